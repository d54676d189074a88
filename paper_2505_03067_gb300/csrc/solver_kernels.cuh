// solver_kernels.cuh -- restarted GMRES (Saad & Schultz 1986, the solver named
// in Sec. 2.4) for the box systems, as ONE persistent cooperative kernel: the
// device code and its instantiation helper (the instances themselves live
// in the solver_inst_*.cu translation units, two each, compiled in
// parallel).
//
// Structure of a launch.  The grid is split into teams of co-resident CTAs;
// each team solves a list of work items, one (system, species) pair each.
// A cycle is
//   R   r = b - A x (FP64), ||r||, ||b||                       -> barrier
//   for j = 0..m-1 (classical Gram-Schmidt in two passes):
//     P1  w = A v_j (7-point stencil) and h_ij = <v_i, w>, i<=j -> barrier
//     P2  w -= sum_i h_ij v_i, ||w||                           -> barrier
//         Givens rotation of the new Hessenberg column (in the Krylov type,
//         redundantly in every CTA)
//   U   x += V y (y from the triangular solve)                 -> barrier
// and the next R pass doubles as the true-residual convergence test.  Krylov
// vectors are stored unnormalised with a scale sigma_i = 1/||v_i||, so no
// pass is spent on normalisation.  With the FP32 basis on tiles at least four
// wide, P1, P2 and U give each thread 4-element chunks of tile rows (16-byte
// vector loads); R and the FP64 basis keep one or two elements per thread.
//
// Reductions are deterministic: every CTA writes its partial sums to a
// double-buffered slot, and after the team barrier every CTA sums the team's
// slots in the same fixed order, so all CTAs hold bit-identical Hessenberg
// data and take identical control decisions without any broadcast.
//
// precision 1 (T = float): the Krylov basis, the operator (FP32 diagonal) and
// the Arnoldi passes run in FP32; R stays FP64 and U adds the FP32 correction
// to the FP64 iterate, so each restart is one step of iterative refinement
// whose inner cycle stops at max(tol, inner_rtol * ||r||).
#pragma once

#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>
#include <algorithm>

#include "mpm_internal.cuh"
#include "step_kernels.cuh"

namespace mpm {

enum { ST_RUN = -1 };

constexpr int kSB = 512;            // default solver CTA size (16 warps); variants also use 1024

struct SpState {
    double beta, bnorm, tol, tol_in;
    double wwb;                       // ||w||^2 before the orthogonalisation (reorthogonalisation test)
    int32_t it, cyc, status, in_cycle, k, done, bad, jsum;
    int32_t reo, nreo;                // second Gram-Schmidt pass due / passes so far
};

// Species are processed in groups of NSG inside one element loop, so the face
// flags and neighbour indices are computed once per element and the loads of
// all species of the group are in flight together.

// G: the type of the small serial least-squares problem (Hessenberg matrix,
// Givens rotations, residual vector, basis scales) -- the Krylov type: FP32
// on the FP32-Krylov path, whose inner solve only has to reach about 1e-6
// relative (the FP64 residual pass decides convergence), FP64 otherwise.  On
// GB300 every FP64 instruction of this one-thread section costs tens of cycles.
template <int MAXM, typename G, int NT>
struct Smem {
    G H[kMaxSpecies][(MAXM + 1) * MAXM];
    G cs[kMaxSpecies][MAXM], sn[kMaxSpecies][MAXM];
    G g[kMaxSpecies][MAXM + 1], sig[kMaxSpecies][MAXM + 1];
    double coef[kMaxSpecies][MAXM + 1];
    float coef32[kMaxSpecies][MAXM + 1];
    double red[NT / 32][kKMax];
    double tot[kKMax];
    SpState sp[kMaxSpecies];
    SysDev sys;
};

template <typename T> __device__ __forceinline__ T warp_sum_t(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// CTA reduction of the group's values acc[g][i] (g active in gm, i < cnt): warp
// sums in the accumulator type, cross-warp sum in FP64 in a fixed order; the
// CTA total of species s0+g, value i lands in out[(s0+g)*kKStride + i].
template <int NSG, int N, typename AccT, int NT>
__device__ __forceinline__ void block_reduce_g(const AccT (&acc)[NSG][N], uint32_t gm, int cnt, int s0,
                                               double (*red)[kKMax], double *out)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int g = 0; g < NSG; ++g) {
        if (!((gm >> g) & 1u)) continue;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (i < cnt) {
                const AccT v = warp_sum_t<AccT>(acc[g][i]);
                if (lane == 0) red[w][(s0 + g) * kKStride + i] = (double)v;
            }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NSG * kKStride; t += NT) {
        const int g = t / kKStride, i = t - g * kKStride;
        if (!((gm >> g) & 1u) || i >= cnt) continue;
        const int slot = (s0 + g) * kKStride + i;
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < NT / 32; ++q) s += red[q][slot];
        out[slot] = s;
    }
    __syncthreads();
}

// Team sum of the slots s*kKStride + i (i < cnt) of the species in smask, in a
// fixed order (lane l adds blocks l, l+32, ...; then a fixed shuffle tree).
template <int NT>
__device__ __forceinline__ void team_reduce(const double *part, int b0, int nb, uint32_t smask, int cnt,
                                            double *tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nslot = kMaxSpecies * cnt;
    for (int q = w; q < nslot; q += NT / 32) {
        const int s = q / cnt, i = q - s * cnt;
        if (!((smask >> s) & 1u)) continue;
        const int slot = s * kKStride + i;
        double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
        int b = lane;
        for (; b + 96 < nb; b += 128) {
            v0 += __ldcg(part + (size_t)(b0 + b) * kKMax + slot);
            v1 += __ldcg(part + (size_t)(b0 + b + 32) * kKMax + slot);
            v2 += __ldcg(part + (size_t)(b0 + b + 64) * kKMax + slot);
            v3 += __ldcg(part + (size_t)(b0 + b + 96) * kKMax + slot);
        }
        for (; b < nb; b += 32) v0 += __ldcg(part + (size_t)(b0 + b) * kKMax + slot);
        const double v = warp_sum((v0 + v1) + (v2 + v3));
        if (lane == 0) tot[slot] = v;
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ const T *diag_of(const SysDev &S, int s);
template <>
__device__ __forceinline__ const double *diag_of<double>(const SysDev &S, int s) { return S.diag[s]; }
template <>
__device__ __forceinline__ const float *diag_of<float>(const SysDev &S, int s) { return S.diag32[s]; }

// Loads of data written before the solve (face flags, rows, neighbour table,
// diffusivity factors): plain cached loads, not the read-only path -- in the
// device-resident step the same kernel wrote them before a grid barrier.
template <typename T>
__device__ __forceinline__ T ldro(const T *p) { return *p; }

// The six neighbour-tile entries of e's tile (-x,+x,-y,+y,-z,+z; 24 bytes,
// 8-byte aligned).  The passes fetch them one iteration ahead together with
// the flag byte, so an element's neighbour indices never wait on a table load.
__device__ __forceinline__ void tile_nbrs(const int32_t *__restrict__ nbr, uint32_t e, int ltv, int32_t (&t)[6])
{
    const int2 *p = reinterpret_cast<const int2 *>(nbr + (size_t)(e >> ltv) * 6);
    const int2 a = ldro(p), b = ldro(p + 1), c = ldro(p + 2);
    t[0] = a.x;
    t[1] = a.y;
    t[2] = b.x;
    t[3] = b.y;
    t[4] = c.x;
    t[5] = c.y;
}

// Neighbour elements of e for its open faces from its tile's entries t
// (closed faces get e; never read).
__device__ __forceinline__ void nbr_elems_t(const int32_t (&t)[6], uint32_t e, uint32_t f, int ltx, int lty, int ltz,
                                            uint32_t (&q)[6])
{
    const int ltv = ltx + lty + ltz;
    const uint32_t v = e & ((1u << ltv) - 1u);
    const uint32_t TX = 1u << ltx, TY = 1u << lty, TZ = 1u << ltz;
    const uint32_t ix = v & (TX - 1), iy = (v >> ltx) & (TY - 1), iz = v >> (ltx + lty);
    q[0] = !(f & F_MX) ? e : (ix > 0 ? e - 1 : ((uint32_t)t[0] << ltv) + (v + TX - 1));
    q[1] = !(f & F_PX) ? e : (ix < TX - 1 ? e + 1 : ((uint32_t)t[1] << ltv) + (v - (TX - 1)));
    q[2] = !(f & F_MY) ? e : (iy > 0 ? e - TX : ((uint32_t)t[2] << ltv) + (v + (TY - 1) * TX));
    q[3] = !(f & F_PY) ? e : (iy < TY - 1 ? e + TX : ((uint32_t)t[3] << ltv) + (v - (TY - 1) * TX));
    q[4] = !(f & F_MZ) ? e : (iz > 0 ? e - TX * TY : ((uint32_t)t[4] << ltv) + (v + (TZ - 1) * TX * TY));
    q[5] = !(f & F_PZ) ? e : (iz < TZ - 1 ? e + TX * TY : ((uint32_t)t[5] << ltv) + (v - (TZ - 1) * TX * TY));
}

// Sum of u over the open faces with closed faces selected to zero (5 adds for
// 6 faces; neighbours read through L2: other CTAs wrote them).
template <typename T>
__device__ __forceinline__ T open_sum_sel(const T *__restrict__ u, uint32_t f, const uint32_t (&q)[6])
{
    T v[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) v[d] = __ldcg(u + q[d]);   // a closed face reads e itself
#pragma unroll
    for (int d = 0; d < 6; ++d) v[d] = (f & (1u << d)) ? v[d] : T(0);
    return ((v[0] + v[1]) + (v[2] + v[3])) + (v[4] + v[5]);
}

// Sum of u over the open faces (neighbours read through L2: other CTAs wrote
// them).  A closed face's index is e itself, so all six loads are issued
// unconditionally, back to back, and the closed ones are selected away.
template <typename T>
__device__ __forceinline__ T open_sum(const T *__restrict__ u, uint32_t f, const uint32_t (&q)[6])
{
    T v[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) v[d] = __ldcg(u + q[d]);
#pragma unroll
    for (int d = 0; d < 6; ++d) v[d] = (f & (1u << d)) ? v[d] : T(0);
    return ((v[0] + v[2]) + v[4]) + ((v[1] + v[3]) + v[5]);
}

// Harmonic-mean variant: sum of D_f u_Q, D_f = 2 D_P D_Q / (D_P + D_Q).
template <typename T>
__device__ __forceinline__ T open_sum_var(const T *__restrict__ u, const double *__restrict__ dfac, uint32_t e,
                                          uint32_t f, const uint32_t (&q)[6], double Ds)
{
    const double dp = Ds * ldro(dfac + e);
    T s = T(0);
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        if (f & (1u << d)) {
            const double dq = Ds * ldro(dfac + q[d]);
            const double hm = (dp + dq > 0.0) ? 2.0 * dp * dq / (dp + dq) : 0.0;
            s += T(hm) * __ldcg(u + q[d]);
        }
    }
    return s;
}

// Every pass handles U elements per thread and iteration (e, e+es, ...,
// spaced one grid stride apart) and issues all their loads before the first
// store: stores through the Krylov base pointer may alias later loads in the
// compiler's eyes, so this ordering is what keeps U elements' loads in flight
// together.  Work items hold one species (s = 0).

template <typename T>
__device__ __forceinline__ T to_basis(double x);
template <>
__device__ __forceinline__ float to_basis<float>(double x) { return f32_rz(x); }
template <>
__device__ __forceinline__ double to_basis<double>(double x) { return x; }

// ---- R: r = b - A x in FP64; u_0 = r (stored in T); sums of r^2 and of b^2
// over mask rows.
template <typename T, int U, bool VAR>
__device__ __forceinline__ void pass_residual_t(const SysDev &S, bool first, uint32_t e0, uint32_t es,
                                                double &aR, double &aB)
{
    // The residual and both norms are FP64 on either path: squares of FP32
    // values would underflow for fields below ~1e-19 and end the solve on a
    // zero norm.
    const uint32_t NE = (uint32_t)S.NE;
    constexpr bool var = VAR;
    const double *x = S.x[0];
    // the flag bytes and the tile's neighbour entries are read-only during the
    // solve: fetch the next iteration's one iteration ahead, so the neighbour
    // loads never wait for them
    const int ltv = S.ltx + S.lty + S.ltz;
    uint32_t fn[U];
    int32_t tn[U][6];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint32_t en = e0 + u * es;
        fn[u] = en < NE ? ldro(S.flags + en) : 0u;
        if (en < NE) tile_nbrs(S.nbr, en, ltv, tn[u]);
    }
    for (uint32_t e = e0; e < NE; e += U * es) {
        uint32_t f[U], q[U][6];
        double xv[U], ns[U], bv[U], dg[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t eu = e + u * es;
            if (eu < NE) nbr_elems_t(tn[u], eu, fn[u], S.ltx, S.lty, S.ltz, q[u]);
            f[u] = fn[u];
            const uint32_t en = e + (U + u) * es;
            fn[u] = en < NE ? ldro(S.flags + en) : 0u;
            if (en < NE) tile_nbrs(S.nbr, en, ltv, tn[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t eu = e + u * es;
            if (eu >= NE) continue;
            xv[u] = __ldcg(x + eu);   // the update may have written it from another CTA
            ns[u] = var ? S.a * open_sum_var<double>(x, S.dfac, eu, f[u], q[u], S.Dsp[0]) : open_sum_sel<double>(x, f[u], q[u]);
            bv[u] = ldro(S.b[0] + eu);
            dg[u] = ldro(S.diag[0] + eu);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t eu = e + u * es;
            if (eu >= NE) continue;
            // r = b - diag x + off * sum_open x_Q  (two fused multiply-adds)
            const double r = var ? bv[u] - (dg[u] * xv[u] - ns[u]) : fma(S.off[0], ns[u], fma(-dg[u], xv[u], bv[u]));
            ((T *)S.V[0])[eu] = to_basis<T>(r);
            aR = fma(r, r, aR);
            if (first && (f[u] & F_MASK)) aB = fma(bv[u], bv[u], aB);
        }
    }
}

// the harmonic-mean (per-voxel D) and the uniform-D form as separate loops
template <typename T, int U>
__device__ __forceinline__ void pass_residual(const SysDev &S, bool first, uint32_t e0, uint32_t es,
                                              double &aR, double &aB)
{
    if (S.dfac) pass_residual_t<T, U, true>(S, first, e0, es, aR, aB);
    else pass_residual_t<T, U, false>(S, first, e0, es, aR, aB);
}

// ---- P1: w = sigma_j A u_j into slot j+1; acc[i] += u_i . w for i <= j
template <typename T, int MAXM, int U, bool VAR, int JJ = -1, int LIM = MAXM>
__device__ __forceinline__ void pass_arnoldi1_t(const SysDev &S, int jr, T sj, uint32_t e0, uint32_t es,
                                                T (&acc)[MAXM + 1], bool want_ww)
{
    const int j = JJ >= 0 ? JJ : jr;   // JJ >= 0: the step index known at compile time
    const uint32_t NE = (uint32_t)S.NE;
    const int64_t vs = S.vstride;
    constexpr bool var = VAR;
    const T offT = (T)(var ? S.a : S.off[0]);
    const T *V = (const T *)S.V[0];
    const T *uj = V + (int64_t)j * vs;
    const T *dgp = diag_of<T>(S, 0);
    const int ltv = S.ltx + S.lty + S.ltz;
    uint32_t fn[U];
    int32_t tn[U][6];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint32_t en = e0 + u * es;
        fn[u] = en < NE ? ldro(S.flags + en) : 0u;
        if (en < NE) tile_nbrs(S.nbr, en, ltv, tn[u]);
    }
    for (uint32_t e = e0; e < NE; e += U * es) {
        uint32_t f[U], q[U][6];
        T xj[U], ns[U], dg[U], w[U], vi[U][LIM];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t eu = e + u * es;
            if (eu < NE) nbr_elems_t(tn[u], eu, fn[u], S.ltx, S.lty, S.ltz, q[u]);
            f[u] = fn[u];
            const uint32_t en = e + (U + u) * es;
            fn[u] = en < NE ? ldro(S.flags + en) : 0u;
            if (en < NE) tile_nbrs(S.nbr, en, ltv, tn[u]);
        }
        // every load of the iteration before the first product: the stencil
        // values and the basis entries u_i(e), i < j, travel together
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t eu = e + u * es;
            if (eu >= NE) continue;
            xj[u] = __ldcg(uj + eu);   // the chunked passes may have written these from other CTAs
            ns[u] = var ? open_sum_var<T>(uj, S.dfac, eu, f[u], q[u], S.Dsp[0]) : open_sum<T>(uj, f[u], q[u]);
            dg[u] = ldro(dgp + eu);
#pragma unroll
            for (int i = 0; i < LIM; ++i) vi[u][i] = i < j ? __ldcg(V + (int64_t)i * vs + eu) : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t eu = e + u * es;
            if (eu >= NE) continue;
            w[u] = sj * (dg[u] * xj[u] - offT * ns[u]);
#pragma unroll
            for (int i = 0; i <= LIM; ++i) {
                if (i < j) acc[i] += vi[u][i] * w[u];
                else if (i == j) acc[i] += xj[u] * w[u];
                else if (i == j + 1 && want_ww) acc[i] += w[u] * w[u];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t eu = e + u * es;
            if (eu < NE) ((T *)S.V[0])[(int64_t)(j + 1) * vs + eu] = w[u];
        }
    }
}

// The basis loops of the FP64 element passes unrolled for the exact step
// index (restart length up to 8): an FP64 instruction whose lanes are all
// predicated off still takes its issue slot of the FP64 pipe, so the loops
// carry no predicated-off iterations.  f receives std::integral_constant<int, J>.
template <typename F>
__device__ __forceinline__ void with_exact(int j, F &&f)
{
    switch (j) {
    case 0: f(std::integral_constant<int, 0>{}); break;
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    default: f(std::integral_constant<int, 7>{}); break;
    }
}

template <typename T, int MAXM>
__device__ __forceinline__ constexpr bool exact_j()
{
    return std::is_same<T, double>::value && MAXM == 8;
}

// The restart buckets above 8: the basis loops of a pass run to the smallest
// multiple of 8 above j (j < MAXM) instead of MAXM, so a loop carries at most
// seven predicated-off iterations.  f receives std::integral_constant<int, LIM>.
template <int MAXM, typename F>
__device__ __forceinline__ void with_limit(int j, F &&f)
{
    if (MAXM <= 8 || j < 8) f(std::integral_constant<int, (MAXM < 8 ? MAXM : 8)>{});
    else if (MAXM <= 16 || j < 16) f(std::integral_constant<int, (MAXM < 16 ? MAXM : 16)>{});
    else if (MAXM <= 24 || j < 24) f(std::integral_constant<int, (MAXM < 24 ? MAXM : 24)>{});
    else f(std::integral_constant<int, MAXM>{});
}

// Four consecutive elements of a vector: one 16-byte load (FP32) or two (FP64).
template <typename T>
struct Q4 {
    T v[4];
};
__device__ __forceinline__ Q4<float> ld4cg(const float *p)
{
    const float4 a = __ldcg(reinterpret_cast<const float4 *>(p));
    return Q4<float>{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Q4<double> ld4cg(const double *p)
{
    const double2 a = __ldcg(reinterpret_cast<const double2 *>(p)), b = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    return Q4<double>{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ Q4<float> ld4ro(const float *p)
{
    const float4 a = ldro(reinterpret_cast<const float4 *>(p));
    return Q4<float>{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Q4<double> ld4ro(const double *p)
{
    const double2 a = ldro(reinterpret_cast<const double2 *>(p)), b = ldro(reinterpret_cast<const double2 *>(p) + 1);
    return Q4<double>{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float *p, const float (&w)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ void st4(double *p, const double (&w)[4])
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(w[0], w[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(w[2], w[3]);
}

// The FP32 basis on tiles at least four wide in x: P1 (uniform D), P2, the
// update and the reorthogonalisation's dots run on 4-element chunks of tile
// rows (FP64 passes are bound by the FP64 rate and keep one element per
// thread).  A pass reads what another pass wrote through L2, whichever thread
// wrote it.
template <typename T>
__device__ __forceinline__ bool use_rows(const SysDev &S)
{
    return std::is_same<T, float>::value && S.ltx >= 2;
}



// ---- P1 for uniform D on tiles at least four wide in x: one 4-element chunk
// of a tile row per thread and iteration.  Its u_j, the chunks at -y, +y, -z,
// +z (same offsets within the tile, or in the neighbour tile), diag and the
// basis rows travel as 16-byte vectors; the two x ends are single loads.  Per
// element the operands and the order of the sum are those of the scalar pass,
// so w is the same bit for bit; the dot products add four elements per thread
// and iteration.  Vectors written during the solve are read through L2.
template <typename T, int MAXM, int LIM = MAXM>
__device__ __forceinline__ void pass_arnoldi1_rows(const SysDev &S, int j, T sj, uint32_t e0, uint32_t es,
                                                   T (&acc)[MAXM + 1], bool want_ww)
{
    const uint32_t NR = (uint32_t)S.NE >> 2;
    const int64_t vs = S.vstride;
    const T offT = (T)S.off[0];
    T *V = (T *)S.V[0];
    const T *uj = V + (int64_t)j * vs;
    const T *dgp = diag_of<T>(S, 0);
    const int ltx = S.ltx, lty = S.lty, ltv = S.ltx + S.lty + S.ltz;
    const uint32_t TX = 1u << ltx, TY = 1u << lty, TZ = 1u << S.ltz, TXY = TX * TY;
    for (uint32_t r = e0; r < NR; r += es) {
        const uint32_t e = r << 2;
        const uint32_t v0 = e & ((1u << ltv) - 1u);
        const uint32_t ix0 = v0 & (TX - 1), iy = (v0 >> ltx) & (TY - 1), iz = v0 >> (ltx + lty);
        int32_t tn[6];
        tile_nbrs(S.nbr, e, ltv, tn);
        const uchar4 fl = ldro(reinterpret_cast<const uchar4 *>(S.flags) + r);
        // element of the neighbour tile across face d at offset o, or e when
        // there is none (every face that way is then closed)
        auto other = [&](int d, uint32_t o) -> uint32_t { return tn[d] >= 0 ? ((uint32_t)tn[d] << ltv) + o : e; };
        const uint32_t qym = iy > 0 ? e - TX : other(2, v0 + (TY - 1) * TX);
        const uint32_t qyp = iy < TY - 1 ? e + TX : other(3, v0 - (TY - 1) * TX);
        const uint32_t qzm = iz > 0 ? e - TXY : other(4, v0 + (TZ - 1) * TXY);
        const uint32_t qzp = iz < TZ - 1 ? e + TXY : other(5, v0 - (TZ - 1) * TXY);
        const uint32_t qxm = ix0 > 0 ? e - 1 : other(0, v0 + TX - 1);
        const uint32_t qxp = ix0 + 4 < TX ? e + 4 : other(1, v0 - ix0);
        const Q4<T> u = ld4cg(uj + e);
        const Q4<T> ym = ld4cg(uj + qym), yp = ld4cg(uj + qyp), zm = ld4cg(uj + qzm), zp = ld4cg(uj + qzp);
        const T xm = __ldcg(uj + qxm), xp = __ldcg(uj + qxp);
        const Q4<T> dg = ld4ro(dgp + e);
        const uint32_t ff[4] = {fl.x, fl.y, fl.z, fl.w};
        T w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t f = ff[k];
            T v[6] = {k > 0 ? u.v[k - 1] : xm, k < 3 ? u.v[k + 1] : xp, ym.v[k], yp.v[k], zm.v[k], zp.v[k]};
#pragma unroll
            for (int d = 0; d < 6; ++d) v[d] = (f & (1u << d)) ? v[d] : T(0);
            const T ns = ((v[0] + v[2]) + v[4]) + ((v[1] + v[3]) + v[5]);
            w[k] = sj * (dg.v[k] * u.v[k] - offT * ns);
        }
#pragma unroll
        for (int i = 0; i < LIM; ++i) {
            if (i < j) {
                const Q4<T> b = ld4cg(V + (int64_t)i * vs + e);
                acc[i] += ((b.v[0] * w[0] + b.v[1] * w[1]) + (b.v[2] * w[2] + b.v[3] * w[3]));
            }
        }
#pragma unroll
        for (int i = 0; i <= LIM; ++i) {
            if (i == j) acc[i] += ((u.v[0] * w[0] + u.v[1] * w[1]) + (u.v[2] * w[2] + u.v[3] * w[3]));
            else if (i == j + 1 && want_ww) acc[i] += ((w[0] * w[0] + w[1] * w[1]) + (w[2] * w[2] + w[3] * w[3]));
        }
        st4(V + (int64_t)(j + 1) * vs + e, w);
    }
}

template <typename T, int MAXM, int U>
__device__ __forceinline__ void pass_arnoldi1(const SysDev &S, int j, T sj, uint32_t e0, uint32_t es,
                                              T (&acc)[MAXM + 1], bool want_ww)
{
    if (exact_j<T, MAXM>()) {
        if (S.dfac)
            with_exact(j, [&](auto J) { pass_arnoldi1_t<T, MAXM, U, true, decltype(J)::value>(S, j, sj, e0, es, acc, want_ww); });
        else
            with_exact(j, [&](auto J) { pass_arnoldi1_t<T, MAXM, U, false, decltype(J)::value>(S, j, sj, e0, es, acc, want_ww); });
    } else {
        with_limit<MAXM>(j, [&](auto L) {
            constexpr int LIM = decltype(L)::value;
            if (S.dfac) pass_arnoldi1_t<T, MAXM, U, true, -1, LIM>(S, j, sj, e0, es, acc, want_ww);
            else if (use_rows<T>(S)) pass_arnoldi1_rows<T, MAXM, LIM>(S, j, sj, e0, es, acc, want_ww);
            else pass_arnoldi1_t<T, MAXM, U, false, -1, LIM>(S, j, sj, e0, es, acc, want_ww);
        });
    }
}

// ---- P2: w -= sum_{i<=j} c_i u_i in place (c_i = h_ij sigma_i); acc += w^2
template <typename T, int MAXM, int U, int JJ = -1, int LIM = MAXM>
__device__ __forceinline__ void pass_arnoldi2_e(const SysDev &S, int jr, const T *c, uint32_t e0, uint32_t es, T &acc)
{
    const int j = JJ >= 0 ? JJ : jr;
    const uint32_t NE = (uint32_t)S.NE;
    const int64_t vs = S.vstride;
    const T *V = (const T *)S.V[0];
    for (uint32_t e = e0; e < NE; e += U * es) {
        T w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t eu = e + u * es;
            if (eu >= NE) continue;
            T t = __ldcg(V + (int64_t)(j + 1) * vs + eu);   // P1 may have written it from another CTA
#pragma unroll
            for (int i = 0; i <= LIM; ++i)
                if (i <= j) t -= c[i] * V[(int64_t)i * vs + eu];
            w[u] = t;
            acc += t * t;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t eu = e + u * es;
            if (eu < NE) ((T *)S.V[0])[(int64_t)(j + 1) * vs + eu] = w[u];
        }
    }
}

template <typename T, int MAXM, int LIM = MAXM>
__device__ __forceinline__ void pass_arnoldi2_rows(const SysDev &S, int j, const T *c, uint32_t e0, uint32_t es, T &acc)
{
    const uint32_t NR = (uint32_t)S.NE >> 2;
    const int64_t vs = S.vstride;
    T *V = (T *)S.V[0];
    for (uint32_t r = e0; r < NR; r += es) {
        const uint32_t e = r << 2;
        Q4<T> t = ld4cg(V + (int64_t)(j + 1) * vs + e);
#pragma unroll
        for (int i = 0; i <= LIM; ++i) {
            if (i <= j) {
                const Q4<T> b = ld4cg(V + (int64_t)i * vs + e);
                const T ci = c[i];
#pragma unroll
                for (int k = 0; k < 4; ++k) t.v[k] -= ci * b.v[k];
            }
        }
        acc += (t.v[0] * t.v[0] + t.v[1] * t.v[1]) + (t.v[2] * t.v[2] + t.v[3] * t.v[3]);
        st4(V + (int64_t)(j + 1) * vs + e, t.v);
    }
}

template <typename T, int MAXM, int U>
__device__ __forceinline__ void pass_arnoldi2(const SysDev &S, int j, const T *c, uint32_t e0, uint32_t es, T &acc)
{
    if (exact_j<T, MAXM>() && !use_rows<T>(S))
        with_exact(j, [&](auto J) { pass_arnoldi2_e<T, MAXM, U, decltype(J)::value>(S, j, c, e0, es, acc); });
    else
        with_limit<MAXM>(j, [&](auto L) {
            constexpr int LIM = decltype(L)::value;
            if (use_rows<T>(S)) pass_arnoldi2_rows<T, MAXM, LIM>(S, j, c, e0, es, acc);
            else pass_arnoldi2_e<T, MAXM, U, -1, LIM>(S, j, c, e0, es, acc);
        });
}

// ---- P1b (reorthogonalisation): acc[i] += u_i . w for i <= j, w in slot j+1
template <typename T, int MAXM, int U, int LIM = MAXM>
__device__ __forceinline__ void pass_dots_e(const SysDev &S, int j, uint32_t e0, uint32_t es, T (&acc)[MAXM + 1])
{
    const uint32_t NE = (uint32_t)S.NE;
    const int64_t vs = S.vstride;
    const T *V = (const T *)S.V[0];
    for (uint32_t e = e0; e < NE; e += U * es) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t eu = e + u * es;
            if (eu >= NE) continue;
            const T w = V[(int64_t)(j + 1) * vs + eu];
#pragma unroll
            for (int i = 0; i <= LIM; ++i)
                if (i <= j) acc[i] += V[(int64_t)i * vs + eu] * w;
        }
    }
}

template <typename T, int MAXM, int LIM = MAXM>
__device__ __forceinline__ void pass_dots_rows(const SysDev &S, int j, uint32_t e0, uint32_t es, T (&acc)[MAXM + 1])
{
    const uint32_t NR = (uint32_t)S.NE >> 2;
    const int64_t vs = S.vstride;
    const T *V = (const T *)S.V[0];
    for (uint32_t r = e0; r < NR; r += es) {
        const uint32_t e = r << 2;
        const Q4<T> w = ld4cg(V + (int64_t)(j + 1) * vs + e);
#pragma unroll
        for (int i = 0; i <= LIM; ++i) {
            if (i <= j) {
                const Q4<T> b = ld4cg(V + (int64_t)i * vs + e);
                acc[i] += (b.v[0] * w.v[0] + b.v[1] * w.v[1]) + (b.v[2] * w.v[2] + b.v[3] * w.v[3]);
            }
        }
    }
}

template <typename T, int MAXM, int U>
__device__ __forceinline__ void pass_dots(const SysDev &S, int j, uint32_t e0, uint32_t es, T (&acc)[MAXM + 1])
{
    with_limit<MAXM>(j, [&](auto L) {
        constexpr int LIM = decltype(L)::value;
        if (use_rows<T>(S)) pass_dots_rows<T, MAXM, LIM>(S, j, e0, es, acc);
        else pass_dots_e<T, MAXM, U, LIM>(S, j, e0, es, acc);
    });
}

// ---- U: x += sum_{i<k} c_i u_i (c_i = y_i sigma_i); the FP32 path adds its
// FP32 correction d to the FP64 iterate.
template <typename T, int MAXM, int U, int KK = -1, int LIM = MAXM>
__device__ __forceinline__ void pass_update_e(const SysDev &S, int kr, const T *c, uint32_t e0, uint32_t es)
{
    const int k = KK >= 0 ? KK : kr;   // KK >= 0: the vector count known at compile time
    const uint32_t NE = (uint32_t)S.NE;
    const int64_t vs = S.vstride;
    const T *V = (const T *)S.V[0];
    double *x = S.x[0];
    for (uint32_t e = e0; e < NE; e += U * es) {
        T d[U];
        double xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t eu = e + u * es;
            if (eu >= NE) continue;
            T t = T(0);
#pragma unroll
            for (int i = 0; i < LIM; ++i)
                if (i < k) t += c[i] * V[(int64_t)i * vs + eu];
            d[u] = t;
            xv[u] = x[eu];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t eu = e + u * es;
            if (eu < NE) x[eu] = xv[u] + (double)d[u];
        }
    }
}

template <typename T, int MAXM, int LIM = MAXM>
__device__ __forceinline__ void pass_update_rows(const SysDev &S, int k, const T *c, uint32_t e0, uint32_t es)
{
    const uint32_t NR = (uint32_t)S.NE >> 2;
    const int64_t vs = S.vstride;
    const T *V = (const T *)S.V[0];
    double *x = S.x[0];
    for (uint32_t r = e0; r < NR; r += es) {
        const uint32_t e = r << 2;
        const Q4<double> xv = ld4cg(x + e);
        T d[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int i = 0; i < LIM; ++i) {
            if (i < k) {
                const Q4<T> b = ld4cg(V + (int64_t)i * vs + e);
                const T ci = c[i];
#pragma unroll
                for (int q = 0; q < 4; ++q) d[q] += ci * b.v[q];
            }
        }
        double xo[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) xo[q] = xv.v[q] + f64_of(d[q]);
        st4(x + e, xo);
    }
}

template <typename T, int MAXM, int U>
__device__ __forceinline__ void pass_update(const SysDev &S, int k, const T *c, uint32_t e0, uint32_t es)
{
    if (exact_j<T, MAXM>() && !use_rows<T>(S))   // k = 1..8 vectors
        with_exact(k - 1, [&](auto J) { pass_update_e<T, MAXM, U, decltype(J)::value + 1>(S, k, c, e0, es); });
    else
        with_limit<MAXM>(k - 1, [&](auto L) {   // i < k <= LIM
            constexpr int LIM = decltype(L)::value;
            if (use_rows<T>(S)) pass_update_rows<T, MAXM, LIM>(S, k, c, e0, es);
            else pass_update_e<T, MAXM, U, -1, LIM>(S, k, c, e0, es);
        });
}

// The persistent GMRES of one CTA of a team (every item of its team in turn).
// Returns early when a team barrier gave up (the abort flag is then set).
template <typename T, int MAXM, int U, int NT>
__device__ __forceinline__ void gmres_body(const SolveArgs &A, Smem<MAXM, T, NT> &sm)
{
    const int tid = threadIdx.x;
    const int team = A.block_team[blockIdx.x];
    const TeamDesc td = A.teams[team];
    const int rank = (int)blockIdx.x - td.first_block, nb = td.nblocks;
    uint32_t *bar = A.bar + 32 * team;
    uint32_t epoch = 0;
    int pbuf = 0;
    const size_t pstride = (size_t)gridDim.x * kKMax;
    const uint32_t e0 = (uint32_t)rank * NT + tid, es = (uint32_t)nb * NT;
    constexpr bool kF32 = std::is_same<T, float>::value;
    const T *coefT = kF32 ? (const T *)&sm.coef32[0][0] : (const T *)&sm.coef[0][0];
    // optional phase timer (CTA 0, thread 0): work, barrier wait, team reduce, serial
    const bool prof = A.prof != nullptr && blockIdx.x == 0 && tid == 0;
    uint64_t tp = prof ? globaltimer_ns() : 0, pacc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int wcat = 4;   // work category of the current pass: 4 R, 5 P1, 6 P2, 7 U
#define MPM_TICK(cat)                                   \
    do {                                                \
        if (prof) {                                     \
            const uint64_t t_ = globaltimer_ns();       \
            pacc[cat] += t_ - tp;                       \
            tp = t_;                                    \
        }                                               \
    } while (0)
#define MPM_BARRIER()                                                              \
    do {                                                                           \
        MPM_TICK(wcat);                                                            \
        if (!team_barrier(bar, epoch, nb, A.abort_flag, A.timeout_ns)) return;     \
        MPM_TICK(1);                                                               \
    } while (0)

    for (int si = td.sys_begin; si < td.sys_end; ++si) {
        const int sys_id = A.sys_order[si];
        const uint64_t t_item0 = globaltimer_ns();
        if (tid == 0) {
            sm.sys = A.sys[sys_id];
            if (sm.sys.NEp) sm.sys.NE = __ldcg(sm.sys.NEp);   // sized on the device (device-resident step)
        }
        __syncthreads();
        const SysDev &S = sm.sys;
        const int NS = S.nspecies;
        if (tid < NS) {
            const bool bad_id = S.err && __ldcg(S.err) != 0;   // cell id outside the rate tables
            SpState &p = sm.sp[tid];
            p.beta = p.bnorm = p.tol = p.tol_in = 0.0;
            p.it = p.cyc = p.in_cycle = p.k = p.bad = p.jsum = 0;
            p.wwb = 0.0;
            p.reo = p.nreo = 0;
            p.done = bad_id ? 1 : 0;
            p.status = bad_id ? MPM_ERR_ARG : ST_RUN;
        }
        __syncthreads();
        bool first = true;
        double *mypart = nullptr;
        for (;;) {
            // ---------------- R: true residual (FP64)
            uint32_t rmask = 0;
            for (int s = 0; s < NS; ++s) if (!sm.sp[s].done) rmask |= 1u << s;
            mypart = A.partials + pbuf * pstride + (size_t)blockIdx.x * kKMax;
            wcat = 4;
            if (rmask & 1u) {
                double a2[1][2] = {{0.0, 0.0}};
                pass_residual<T, U>(S, first, e0, es, a2[0][0], a2[0][1]);
                block_reduce_g<1, 2, double, NT>(a2, 1u, 2, 0, sm.red, mypart);
            }
            MPM_BARRIER();
            team_reduce<NT>(A.partials + pbuf * pstride, td.first_block, nb, rmask, 2, sm.tot);
            MPM_TICK(2);
            pbuf ^= 1;
            if (tid < NS && ((rmask >> tid) & 1u)) {
                SpState &p = sm.sp[tid];
                const double beta = sqrt(sm.tot[tid * kKStride + 0]);
                if (first) {
                    p.bnorm = sqrt(sm.tot[tid * kKStride + 1]);
                    p.tol = fmax(A.rtol * p.bnorm, A.atol);
                }
                p.beta = beta;
                if (!isfinite(beta) || !isfinite(p.bnorm)) { p.status = MPM_ERR_BREAKDOWN; p.done = 1; }
                else if (beta <= p.tol) { p.status = MPM_OK; p.done = 1; }
                else if (p.it >= A.maxit) { p.status = MPM_ERR_NOCONV; p.done = 1; }
                else {
                    p.in_cycle = 1;
                    p.cyc += 1;
                    p.k = 0;
                    for (int i = 0; i <= MAXM; ++i) sm.g[tid][i] = T(0);
                    sm.g[tid][0] = (T)beta;
                    sm.sig[tid][0] = (T)(1.0 / beta);
                    p.tol_in = kF32 ? fmax(0.25 * p.tol, A.inner_rtol * beta) : p.tol;
                }
            }
            first = false;
            __syncthreads();
            MPM_TICK(3);
            bool any = false;
            for (int s = 0; s < NS; ++s) any |= sm.sp[s].in_cycle != 0;
            if (!any) break;

            // ---------------- Arnoldi
            for (int j = 0; j < A.m; ++j) {
                uint32_t cm = 0;
                for (int s = 0; s < NS; ++s) if (sm.sp[s].in_cycle) cm |= 1u << s;
                if (!cm) break;
                mypart = A.partials + pbuf * pstride + (size_t)blockIdx.x * kKMax;
                wcat = 5;
                {
                    T acc[1][MAXM + 1];
#pragma unroll
                    for (int i = 0; i <= MAXM; ++i) acc[0][i] = T(0);
                    pass_arnoldi1<T, MAXM, U>(S, j, sm.sig[0][j], e0, es, acc[0], A.reorth != 0);
                    block_reduce_g<1, MAXM + 1, T, NT>(acc, 1u, j + 1 + (A.reorth != 0), 0, sm.red, mypart);
                }
                MPM_BARRIER();
                team_reduce<NT>(A.partials + pbuf * pstride, td.first_block, nb, cm, j + 1 + (A.reorth != 0), sm.tot);
                MPM_TICK(2);
                pbuf ^= 1;
                // the new Hessenberg column and the projection coefficients, one
                // thread per basis vector (a work item holds one species)
                if (tid <= j && (cm & 1u)) {
                    const int i = tid;
                    const T h = sm.sig[0][i] * (T)sm.tot[i];
                    sm.H[0][i * MAXM + j] = h;
                    const T c = h * sm.sig[0][i];
                    if (kF32) sm.coef32[0][i] = (float)c;
                    else sm.coef[0][i] = (double)c;
                }
                if (tid == 0 && (cm & 1u) && A.reorth) sm.sp[0].wwb = sm.tot[j + 1];
                __syncthreads();
                MPM_TICK(3);
                mypart = A.partials + pbuf * pstride + (size_t)blockIdx.x * kKMax;
                wcat = 6;
                {
                    T acc[1][1] = {{T(0)}};
                    pass_arnoldi2<T, MAXM, U>(S, j, coefT, e0, es, acc[0][0]);
                    block_reduce_g<1, 1, T, NT>(acc, 1u, 1, 0, sm.red, mypart);
                }
                MPM_BARRIER();
                team_reduce<NT>(A.partials + pbuf * pstride, td.first_block, nb, cm, 1, sm.tot);
                MPM_TICK(2);
                pbuf ^= 1;
                // optional second classical Gram-Schmidt pass (opt->reorth) when the
                // orthogonalisation removed most of w: ||w|| < 0.7 ||w_before||
                if (tid < NS && ((cm >> tid) & 1u))
                    sm.sp[tid].reo = A.reorth && sm.tot[tid * kKStride] < 0.49 * sm.sp[tid].wwb ? 1 : 0;
                __syncthreads();
                bool reo = false;   // uniform over the team: every CTA reads the same totals
                for (int s = 0; s < NS; ++s) reo |= ((cm >> s) & 1u) && sm.sp[s].reo;
                if (reo) {
                    mypart = A.partials + pbuf * pstride + (size_t)blockIdx.x * kKMax;
                    wcat = 5;
                    {
                        T acc[1][MAXM + 1];
#pragma unroll
                        for (int i = 0; i <= MAXM; ++i) acc[0][i] = T(0);
                        pass_dots<T, MAXM, U>(S, j, e0, es, acc[0]);
                        block_reduce_g<1, MAXM + 1, T, NT>(acc, 1u, j + 1, 0, sm.red, mypart);
                    }
                    MPM_BARRIER();
                    team_reduce<NT>(A.partials + pbuf * pstride, td.first_block, nb, cm, j + 1, sm.tot);
                    MPM_TICK(2);
                    pbuf ^= 1;
                    if (tid < NS && ((cm >> tid) & 1u)) {
                        for (int i = 0; i <= j; ++i) {   // h_ij += sigma_i (u_i . w); subtract sigma_i^2 (u_i . w) u_i
                            const T d = (T)sm.tot[tid * kKStride + i];
                            sm.H[tid][i * MAXM + j] += sm.sig[tid][i] * d;
                            const T c = sm.sig[tid][i] * sm.sig[tid][i] * d;
                            if (kF32) sm.coef32[tid][i] = (float)c;
                            else sm.coef[tid][i] = (double)c;
                        }
                        sm.sp[tid].nreo += 1;
                    }
                    __syncthreads();
                    MPM_TICK(3);
                    mypart = A.partials + pbuf * pstride + (size_t)blockIdx.x * kKMax;
                    wcat = 6;
                    {
                        T acc[1][1] = {{T(0)}};
                        pass_arnoldi2<T, MAXM, U>(S, j, coefT, e0, es, acc[0][0]);
                        block_reduce_g<1, 1, T, NT>(acc, 1u, 1, 0, sm.red, mypart);
                    }
                    MPM_BARRIER();
                    team_reduce<NT>(A.partials + pbuf * pstride, td.first_block, nb, cm, 1, sm.tot);
                    MPM_TICK(2);
                    pbuf ^= 1;
                }
                if (tid < NS && ((cm >> tid) & 1u)) {
                    SpState &p = sm.sp[tid];
                    T *H = sm.H[tid];
                    T *cs = sm.cs[tid], *sn = sm.sn[tid], *g = sm.g[tid];
                    const T hn = sqrt((T)sm.tot[tid * kKStride]);
                    H[(j + 1) * MAXM + j] = hn;
                    for (int i = 0; i < j; ++i) {
                        const T t0 = H[i * MAXM + j], t1 = H[(i + 1) * MAXM + j];
                        H[i * MAXM + j] = cs[i] * t0 + sn[i] * t1;
                        H[(i + 1) * MAXM + j] = -sn[i] * t0 + cs[i] * t1;
                    }
                    const T aa = H[j * MAXM + j], bb = hn;
                    if (bb == T(0)) { cs[j] = T(1); sn[j] = T(0); }
                    else {
                        const T ri = T(1) / hypot(aa, bb);   // one division (FP64 divisions are long here)
                        cs[j] = aa * ri;
                        sn[j] = bb * ri;
                    }
                    H[j * MAXM + j] = cs[j] * aa + sn[j] * bb;
                    H[(j + 1) * MAXM + j] = T(0);
                    g[j + 1] = -sn[j] * g[j];
                    g[j] = cs[j] * g[j];
                    p.it += 1;
                    p.jsum += j;
                    p.k = j + 1;
                    if (!isfinite(g[j + 1]) || !isfinite(H[j * MAXM + j])) {
                        p.status = MPM_ERR_BREAKDOWN;
                        p.bad = 1;
                        p.done = 1;
                        p.in_cycle = 0;
                    } else if (fabs(g[j + 1]) <= (T)p.tol_in || p.it >= A.maxit || hn <= T(kF32 ? 1e-30 : 1e-300) ||
                               j + 1 == A.m) {
                        p.in_cycle = 0;
                    } else {
                        sm.sig[tid][j + 1] = T(1) / hn;
                    }
                }
                __syncthreads();
                MPM_TICK(3);
            }

            // ---------------- least squares: R y = g (back substitution), coef = y * sigma;
            // the reciprocals of the diagonal first, one thread each, so the
            // sequential substitution has no division
            {
                const SpState &p = sm.sp[0];
                if (!p.bad && tid < p.k) sm.cs[0][tid] = T(1) / sm.H[0][tid * MAXM + tid];   // cs no longer needed
            }
            __syncthreads();
            if (tid < NS) {
                SpState &p = sm.sp[tid];
                if (!p.bad && p.k > 0) {
                    const T *H = sm.H[tid];
                    const T *rd = sm.cs[tid];
                    T *y = kF32 ? (T *)sm.coef32[tid] : (T *)sm.coef[tid];
                    for (int i = p.k - 1; i >= 0; --i) {
                        T acc = sm.g[tid][i];
                        for (int l = i + 1; l < p.k; ++l) acc -= H[i * MAXM + l] * y[l];
                        y[i] = acc * rd[i];
                    }
                    bool fin = true;
                    for (int i = 0; i < p.k; ++i) {
                        y[i] *= sm.sig[tid][i];
                        fin &= isfinite(y[i]) != 0;
                    }
                    if (!fin) { p.status = MPM_ERR_BREAKDOWN; p.bad = 1; p.done = 1; }
                }
            }
            __syncthreads();
            MPM_TICK(3);
            // ---------------- U: x += V y
            wcat = 7;
            if (!sm.sp[0].bad && sm.sp[0].k > 0) pass_update<T, MAXM, U>(S, sm.sp[0].k, coefT, e0, es);
            __syncthreads();
            if (tid < NS) sm.sp[tid].k = 0;
            MPM_BARRIER();
        }
        if (rank == 0 && tid < NS) {
            const SpState &p = sm.sp[tid];
            SysReport *R = A.reports + sys_id;
            R->iters[tid] = p.it;
            R->cycles[tid] = p.cyc;
            R->status[tid] = p.status;
            R->jsum[tid] = p.jsum;
            R->res[tid] = p.beta;
            R->bnorm[tid] = p.bnorm;
            R->reorth[tid] = p.nreo;
            R->t_ns = globaltimer_ns() - t_item0;
        }
        __syncthreads();
    }
    if (prof) {
        MPM_TICK(wcat);
        for (int c = 0; c < 8; ++c) A.prof[c] += pacc[c];
    }
#undef MPM_TICK
#undef MPM_BARRIER
}

// U: elements in flight per thread in the streaming passes; MINB: CTAs per SM
// the register allocation must allow (1: up to 128 registers, 2: up to 64).
template <typename T, int MAXM, int U, int MINB, int NT>
__global__ void __launch_bounds__(NT, MINB) k_gmres(SolveArgs A)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    Smem<MAXM, T, NT> &sm = *reinterpret_cast<Smem<MAXM, T, NT> *>(smraw);
    if ((int)blockIdx.x == A.skip_block) return;    // fault injection: this CTA never arrives
    gmres_body<T, MAXM, U, NT>(A, sm);
}

// ------------------------------------------------------------------ the whole step in one kernel
// Results of the device-resident step for the host (host-mapped memory):
// raw box min[3], max[3] at 0, counts (mask voxels, active tiles) at 64, the
// abort flag at 128, the reports at 256.
struct StepOut {
    const int32_t *box;
    const unsigned long long *count;
    const uint32_t *reports;
    int32_t nrep_words;
    char *host;
    uint32_t *exit_count;          // CTAs that left; the last one copies and resets
};

// What one launch of the whole-step kernel does: the whole step, or (for a
// step whose solve starts from another kernel's initial guess, written
// between the two launches) its first half -- the extraction -- or its
// second half -- the solve, the scatter and the step's results.
enum { STEP_WHOLE = 0, STEP_EXTRACT = 1, STEP_SOLVE = 2 };

struct StepArgs {
    SolveArgs sa;
    ExtractArgs xa;                // xa.bar: the grid barrier; xa.xabort == sa.abort_flag
    BatchSys S;
    StepOut o;
    int32_t mode;                  // STEP_WHOLE, STEP_EXTRACT or STEP_SOLVE
};

// One implicit-Euler step of one lattice: the extraction phases A-E (bbox,
// activity, compaction, gather + rows), a grid barrier, the team solves, a
// grid barrier, the scatter onto the pleural mask (skipped if any wait gave
// up).  The last CTA to leave copies the results to host-mapped memory and
// resets the grid barrier and exit counters for the next step.
template <typename T, int MAXM, int U, int MINB, int NT>
__global__ void __launch_bounds__(NT, MINB) k_step(const __grid_constant__ StepArgs P)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    Smem<MAXM, T, NT> &sm = *reinterpret_cast<Smem<MAXM, T, NT> *>(smraw);
    const int tid = threadIdx.x, nb = gridDim.x, b = blockIdx.x;
    // optional phase timer (CTA 0): extraction up to the grid barrier after
    // it, and the wait for the last team plus the scatter
    const bool prof = P.sa.prof != nullptr && b == 0 && tid == 0;
    uint64_t t0 = prof ? globaltimer_ns() : 0;
    // the box cadence: a full extraction unless the previous step let this one
    // keep the box (its last CTA decided; see the end of this kernel)
    const bool full = P.xa.box_every <= 1 || *(const volatile uint32_t *)&P.xa.cad->refresh_ok == 0u;
    if (b != P.sa.skip_block && P.mode == STEP_EXTRACT) {
        // the extraction alone; the kernel boundary orders it before the guess
        uint32_t epoch = 0;
        if (full) extract_phases<NT>(P.xa, P.S, b, nb, epoch);
        else refresh_phases<NT>(P.xa, P.S, b, nb, epoch);
        if (prof) P.sa.prof[8] += globaltimer_ns() - t0;
    } else if (b != P.sa.skip_block) {              // fault injection: this CTA never arrives
        uint32_t epoch = 0;
        bool ok = true;
        if (P.mode == STEP_WHOLE) {
            ok = full ? extract_phases<NT>(P.xa, P.S, b, nb, epoch) : refresh_phases<NT>(P.xa, P.S, b, nb, epoch);
            ok = ok && team_barrier(P.xa.bar, epoch, nb, P.xa.xabort, P.xa.timeout_ns);
        } else {
            ok = *(volatile int32_t *)P.xa.xabort == 0;   // the extraction launch gave up
        }
        if (prof) {
            const uint64_t t = globaltimer_ns();
            P.sa.prof[8] += t - t0;
        }
        if (ok) gmres_body<T, MAXM, U, NT>(P.sa, sm);
        if (prof) t0 = globaltimer_ns();
        ok = ok && team_barrier(P.xa.bar, epoch, nb, P.xa.xabort, P.xa.timeout_ns);
        if (ok && *(volatile int32_t *)P.xa.xabort == 0) {
            const int64_t NE = __ldcg(&P.xa.dyn->NE);
            const BoxGeo g = P.xa.dyn->g;
            if (g.lt[0] >= 2) {   // 4-element chunks of tile rows
                for (int64_t r = (int64_t)b * NT + tid; r < (NE >> 2); r += (int64_t)nb * NT)
                    scatter_chunk(P.S, g, (uint32_t)r);
            } else {
                for (int64_t e = (int64_t)b * NT + tid; e < NE; e += (int64_t)nb * NT) scatter_elem<true>(P.S, g, e);
            }
        }
        if (prof) P.sa.prof[9] += globaltimer_ns() - t0;
    }
    __syncthreads();
    __shared__ int s_last;
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(P.o.exit_count, 1u) == (unsigned)nb - 1u;
        __threadfence();
    }
    __syncthreads();
    if (!s_last) return;
    if (P.mode == STEP_EXTRACT) {
        // the solve launch reuses the grid barrier and the exit counter
        if (tid == 0) {
            *P.xa.bar = 0u;
            *P.o.exit_count = 0u;
        }
        return;
    }
    int32_t *hb = reinterpret_cast<int32_t *>(P.o.host);
    unsigned long long *hc = reinterpret_cast<unsigned long long *>(P.o.host + 64);
    uint32_t *hr = reinterpret_cast<uint32_t *>(P.o.host + 256);
    if (tid < 6) hb[tid] = __ldcg(P.o.box + tid);
    if (tid < 2) hc[tid] = __ldcg(P.o.count + tid);
    if (tid == 0) *reinterpret_cast<int32_t *>(P.o.host + 128) = *(volatile int32_t *)P.xa.xabort;
    for (int i = tid; i < P.o.nrep_words; i += NT) hr[i] = __ldcg(P.o.reports + i);
    if (tid == 0) {
        // the cadence for the next step: keep the box while fewer than
        // box_every steps used it, no tumour voxel reached its guard band, the
        // box is not empty and no wait gave up
        StepCad *c = P.xa.cad;
        const uint32_t cnt = full ? 1u : c->count + 1u;
        c->count = cnt;
        if (full) c->nfull += 1u;
        const bool keep = P.xa.box_every > 1 && cnt < (uint32_t)P.xa.box_every &&
                          *(volatile uint32_t *)&c->guard_hit == 0u && __ldcg(&P.xa.dyn->NE) > 0 &&
                          *(volatile int32_t *)P.xa.xabort == 0;
        c->refresh_ok = keep ? 1u : 0u;
        *reinterpret_cast<uint32_t *>(P.o.host + 160) = c->nfull;
        *P.xa.bar = 0u;
        *P.o.exit_count = 0u;
    }
}

typedef void (*KernFn)(SolveArgs);

typedef void (*StepFn)(StepArgs);

// A kernel variant: the solve kernel, the whole-step kernel of the same
// instantiation, its dynamic shared memory and CTA size.
struct Variant {
    KernFn fn;
    StepFn stepfn;
    size_t smem;
    int nt;
};

template <typename T, int MAXM, int U, int MINB, int NT>
static Variant var_of()
{
    return Variant{k_gmres<T, MAXM, U, MINB, NT>, k_step<T, MAXM, U, MINB, NT>, sizeof(Smem<MAXM, T, NT>), NT};
}

// Kernel instances <type, restart bucket, elements per thread, CTAs per SM,
// threads>, defined in the solver_inst_*.cu translation units.
Variant inst_f32_8_1_1_512();
Variant inst_f32_8_1_1_768();
Variant inst_f32_8_2_2_512();
Variant inst_f32_8_2_1_512();
Variant inst_f32_8_1_1_1024();
Variant inst_f32_8_1_2_512();
Variant inst_f32_8_1_1_640();
Variant inst_f32_16_1_1_512();
Variant inst_f32_32_1_1_512();
Variant inst_f64_8_2_1_512();
Variant inst_f64_8_1_2_512();
Variant inst_f64_8_1_1_512();
Variant inst_f64_8_1_1_1024();
Variant inst_f64_8_1_1_768();
Variant inst_f64_8_2_1_768();
Variant inst_f64_16_1_1_512();
Variant inst_f64_32_1_1_512();

}  // namespace mpm
