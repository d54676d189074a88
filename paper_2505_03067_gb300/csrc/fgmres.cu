// fgmres.cu -- row a13: the implicit-Euler step of Eq. 1-4 on the box solved by
// right-preconditioned flexible GMRES with the network as the preconditioner,
// device-resident.
//
// One CUDA graph per solve holds every species: for each, a residual launch,
// then a WHILE node over refinement cycles whose body holds a WHILE node over
// Arnoldi steps.  Every scalar (projections, Hessenberg column, Givens
// rotations, residual estimate, loop decisions) lives in device memory and is
// computed by single-block launches inside the graph, which set the WHILE
// conditions themselves (cudaGraphSetConditional): the host waits once per
// solve, for the report.  The graph is kept and relaunched while the solve's
// buffers and scalars are unchanged.
//
// Arithmetic (precision 1): the Krylov vectors V, the preconditioned
// directions Z and w = A z are FP32 with the FP32 operator; every cycle
// starts from the FP64 true residual r = b - A x and ends with the FP64 update
// x_t = x + Z y and its FP64 residual (iterative refinement around one
// flexible GMRES cycle, whose residual estimate stops at max(tol / 4,
// inner_rtol ||r||)).  Precision 0 keeps the same structure with FP64 vectors
// and the estimate stopping at tol.  Gram-Schmidt: classical, two passes (the
// projections of the first are read together with the operator).
//
// Fallback to plain GMRES: a cycle whose FP64 true residual is not below the
// one it started from (or is not finite) is discarded (x and r kept).  The
// solver then sets the network plan's unit count to zero, so every network
// kernel has nothing to do, and continues with z_j = v_j: plain GMRES in the
// same refinement.  The report's fallback flag records it.  A discarded plain
// cycle ends the solve (stagnation: MPM_ERR_NOCONV unless the tolerance is
// met).
#include <cmath>
#include <cstring>
#include <vector>

#include "mpm_internal.cuh"

mpm_status mpm_cnn_pc_plan(mpm_ctx *ctx, mpm_cnn *c, mpm_subgrid *sub, const mpm_lattice *lat, const mpm_params *prm,
                           cudaStream_t st, int32_t **units_out);
mpm_status mpm_cnn_pc_apply(mpm_ctx *ctx, mpm_cnn *c, mpm_subgrid *sub, const mpm_lattice *lat,
                            const mpm_params *prm, int s, const void *v, bool f32, int64_t vstride,
                            const int32_t *vj, const double *vscale, void *z, cudaStream_t st);
int mpm_cnn_pc_launches();
uint64_t mpm_cnn_serial(const mpm_cnn *c);
mpm_status mpm_cnn_check_err(mpm_ctx *ctx, mpm_cnn *c);
mpm::SysDev mpm_make_sysdev(const mpm_subgrid *sub);

namespace mpm {

constexpr int kFgRed = 1024;                  // threads of the single-block launches
constexpr int kSlotNorm = kMaxM + 1;          // partial slots: 0..kMaxM projections, then
constexpr int kSlotMax = kMaxM + 2;           //   ||.||^2, max |.|, ||b||^2 over the in-mask rows
constexpr int kSlotB = kMaxM + 3;
constexpr int kSlots = kMaxM + 4;
constexpr int kUnitsSaved = 32;               // network plan: counters[kUnitsSaved] = listed units
constexpr int kFgKernelsPerStep = 7;          // Arnoldi step, network excluded
constexpr int kFgKernelsPerCycle = 6;
constexpr int kFgKernelsPerSpecies = 2;

// The scalars of one species' solve (device memory); head is copied back for
// the report.
struct FgHead {
    double beta;        // FP64 true residual of the current x
    double bnorm;       // ||b|| over the in-mask rows
    double tol;         // max(rtol ||b||, atol)
    double tol_in;      // where the residual estimate ends a cycle
    double vscale;      // max |v_j| of the current Krylov vector (the network's input scale)
    double vscale0;     // max |r| / beta (for v_0)
    double hn;          // ||w|| after the Gram-Schmidt passes
    double beta_t;      // FP64 residual of the last trial update
    int32_t it, cyc, j, k, status, fallback, accept, done, jsum, stall;
    int32_t pad[6];
};

struct FgState {
    FgHead h;
    double c[kMaxM + 1];                 // projections of the current Gram-Schmidt pass
    double hc[kMaxM + 1];                // column j of the Hessenberg matrix (both passes)
    double H[(kMaxM + 1) * kMaxM];       // row-major, rotated
    double cs[kMaxM], sn[kMaxM], g[kMaxM + 1], y[kMaxM];
};

struct FgArgs {
    SysDev S;
    int32_t s;
    int32_t G;                  // CTAs of the streaming launches
    int64_t NE;                 // stored elements
    int64_t vs;                 // Krylov vector stride (elements)
    double *x, *xt, *r, *rt;    // FP64: iterate, trial iterate, residuals
    const double *b;
    void *V, *Z, *w;            // Krylov basis (m+1), directions (m), work vector (T)
    const void *zc;             // the network's output for the current v_j (T)
    FgState *st;
    double *part;               // [kSlots][G] per-CTA partials
    int32_t m, maxit;
    double rtol, atol, inner_rtol;
    int32_t *units;             // the network plan's counters
    cudaGraphConditionalHandle h_out, h_in;
};

template <typename T>
__device__ __forceinline__ const T *fg_diag(const SysDev &S, int s);
template <>
__device__ __forceinline__ const double *fg_diag<double>(const SysDev &S, int s) { return S.diag[s]; }
template <>
__device__ __forceinline__ const float *fg_diag<float>(const SysDev &S, int s) { return S.diag32[s]; }

// (A u)_e of species s in the arithmetic of T (the 7-point operator of Eq. 4).
template <typename T>
__device__ __forceinline__ T fg_apply(const SysDev &S, int s, const T *__restrict__ u, int64_t e)
{
    const uint32_t f = S.flags[e];
    T ns;
    if (S.dfac) ns = T(S.a) * nbr_sum_var<T>(u, S.dfac, S.nbr, e, f, S.ltx, S.lty, S.ltz, S.Dsp[s]);
    else ns = T(S.off[s]) * nbr_sum<T>(u, S.nbr, e, f, S.ltx, S.lty, S.ltz);
    return fg_diag<T>(S, s)[e] * u[e] - ns;
}

__device__ __forceinline__ double fg_warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block sums of acc[0..nk) into the partials of slots slot0.. (one per CTA).
template <int K>
__device__ __forceinline__ void fg_block_sums(double (&acc)[K], int nk, double *__restrict__ part, int slot0, int G,
                                              double (*sh)[kWarps])
{
#pragma unroll
    for (int u = 0; u < K; ++u) acc[u] = warp_sum(acc[u]);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int u = 0; u < K; ++u) sh[u][wid] = acc[u];
    }
    __syncthreads();
    if ((int)threadIdx.x < nk) {
        double t = 0.0;
        for (int q = 0; q < kWarps; ++q) t += sh[threadIdx.x][q];
        part[(int64_t)(slot0 + threadIdx.x) * G + blockIdx.x] = t;
    }
    __syncthreads();
}

// Block sum (or max) of v into the partial of one slot.
__device__ __forceinline__ void fg_block_one(double v, bool mx, double *__restrict__ part, int slot, int G,
                                             double *sh)
{
    v = mx ? fg_warp_max(v) : warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < kWarps; ++q) t = mx ? fmax(t, sh[q]) : t + sh[q];
        part[(int64_t)slot * G + blockIdx.x] = t;
    }
    __syncthreads();
}

// Sum (or max) of the G partials of a slot by one warp, in a fixed order.
__device__ __forceinline__ double fg_slot(const double *__restrict__ part, int slot, int G, bool mx)
{
    const int lane = threadIdx.x & 31;
    double t = 0.0;
    for (int q = lane; q < G; q += 32) {
        const double v = part[(int64_t)slot * G + q];
        t = mx ? fmax(t, v) : t + v;
    }
    return mx ? fg_warp_max(t) : warp_sum(t);
}

#define FG_LOOP(e) for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < A.NE; e += (int64_t)A.G * kBlock)

// r = b - A x in FP64 (kInit: from x into r; else from the trial xt into rt),
// with the partials of ||r||^2, max |r| and (kInit) ||b||^2 over the in-mask rows.
template <bool kInit>
__global__ void __launch_bounds__(kBlock) k_fg_residual(const __grid_constant__ FgArgs A)
{
    __shared__ double sh[kWarps];
    const double *__restrict__ x = kInit ? A.x : A.xt;
    double *__restrict__ r = kInit ? A.r : A.rt;
    double n2 = 0.0, mx = 0.0, b2 = 0.0;
    FG_LOOP(e) {
        const double b = A.b[e];
        const double re = b - fg_apply<double>(A.S, A.s, x, e);
        r[e] = re;
        n2 += re * re;
        mx = fmax(mx, fabs(re));
        if (kInit && (A.S.flags[e] & F_MASK)) b2 += b * b;
    }
    fg_block_one(n2, false, A.part, kSlotNorm, A.G, sh);
    fg_block_one(mx, true, A.part, kSlotMax, A.G, sh);
    if (kInit) fg_block_one(b2, false, A.part, kSlotB, A.G, sh);
}

// ||b||, beta = ||r||, the tolerance; the network plan restored; the outer
// loop entered unless the start already meets the tolerance.
__global__ void __launch_bounds__(kFgRed) k_fg_init(const __grid_constant__ FgArgs A)
{
    __shared__ double red[3];
    const int wid = threadIdx.x >> 5;
    if (wid < 3) {
        const double t = fg_slot(A.part, wid == 0 ? kSlotNorm : (wid == 1 ? kSlotMax : kSlotB), A.G, wid == 1);
        if ((threadIdx.x & 31) == 0) red[wid] = t;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    FgHead &h = A.st->h;
    h.bnorm = sqrt(red[2]);
    h.beta = sqrt(red[0]);
    h.beta_t = h.beta;
    h.tol = fmax(A.rtol * h.bnorm, A.atol);
    h.it = h.cyc = h.j = h.k = h.jsum = 0;
    h.fallback = h.accept = h.stall = 0;
    h.hn = 0.0;
    h.vscale0 = h.beta > 0.0 ? red[1] / h.beta : 0.0;
    h.vscale = h.vscale0;
    A.units[0] = A.units[kUnitsSaved];
    int done = 1;
    if (!isfinite(h.beta)) h.status = MPM_ERR_BREAKDOWN;
    else if (h.beta <= h.tol) h.status = MPM_OK;
    else {
        h.status = MPM_ERR_NOCONV;
        done = 0;
    }
    h.done = done;
    cudaGraphSetConditional(A.h_out, done ? 0u : 1u);
}

// Start of a cycle: v_0 = r / beta, g = beta e_1, the cycle's threshold.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_fg_cycle(const __grid_constant__ FgArgs A)
{
    const double beta = A.st->h.beta;
    const double inv = 1.0 / beta;
    T *__restrict__ V0 = static_cast<T *>(A.V);
    FG_LOOP(e) V0[e] = T(A.r[e] * inv);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        FgState &S = *A.st;
        S.h.j = 0;
        S.h.k = 0;
        S.g[0] = beta;
        for (int i = 1; i <= A.m; ++i) S.g[i] = 0.0;
        S.h.cyc += 1;
        S.h.tol_in = sizeof(T) == 4 ? fmax(0.25 * S.h.tol, A.inner_rtol * beta) : S.h.tol;
        S.h.vscale = S.h.vscale0;
        cudaGraphSetConditional(A.h_in, 1u);
    }
}

// Arnoldi step j, first pass: z_j (the network's output, v_j after the
// fallback), Z[j] = z_j, w = A z_j, and the partials of <w, v_i>, i <= j.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_fg_arnoldi(const __grid_constant__ FgArgs A)
{
    __shared__ double sh[8][kWarps];
    const FgHead &h = A.st->h;
    const int j = h.j;
    const bool fb = h.fallback != 0;
    const bool zero = !fb && !(h.vscale > 0.0);     // v_j = 0: the network wrote nothing
    const T *__restrict__ V = static_cast<const T *>(A.V);
    const T *__restrict__ zs = fb ? V + (int64_t)j * A.vs : static_cast<const T *>(A.zc);
    T *__restrict__ Zj = static_cast<T *>(A.Z) + (int64_t)j * A.vs;
    T *__restrict__ w = static_cast<T *>(A.w);
    for (int i0 = 0; i0 <= j; i0 += 8) {
        T ac[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) ac[u] = T(0);
        FG_LOOP(e) {
            T we;
            if (i0 == 0) {
                Zj[e] = zero ? T(0) : zs[e];
                we = zero ? T(0) : fg_apply<T>(A.S, A.s, zs, e);
                w[e] = we;
            } else {
                we = w[e];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (i0 + u <= j) ac[u] += we * V[(int64_t)(i0 + u) * A.vs + e];
        }
        double acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = (double)ac[u];
        fg_block_sums<8>(acc, min(8, j + 1 - i0), A.part, i0, A.G, sh);
    }
}

// Projections of a Gram-Schmidt pass: c_i = sum of the partials; the
// Hessenberg column accumulates both passes.
template <int kPass>
__global__ void __launch_bounds__(kFgRed) k_fg_project(const __grid_constant__ FgArgs A)
{
    FgState &S = *A.st;
    const int j = S.h.j;
    for (int i = threadIdx.x >> 5; i <= j; i += kFgRed / 32) {
        const double t = fg_slot(A.part, i, A.G, false);
        if ((threadIdx.x & 31) == 0) {
            S.c[i] = t;
            S.hc[i] = kPass == 1 ? t : S.hc[i] + t;
        }
    }
}

// w -= sum_i c_i v_i; pass 1 then takes the partials of <w, v_i> (the second
// pass's projections), pass 2 those of ||w||^2 and max |w|.
template <typename T, int kPass>
__global__ void __launch_bounds__(kBlock) k_fg_orth(const __grid_constant__ FgArgs A)
{
    __shared__ double sh[8][kWarps];
    __shared__ T cv[kMaxM + 1];
    const FgState &S = *A.st;
    const int j = S.h.j;
    for (int i = threadIdx.x; i <= j; i += kBlock) cv[i] = T(S.c[i]);
    __syncthreads();
    const T *__restrict__ V = static_cast<const T *>(A.V);
    T *__restrict__ w = static_cast<T *>(A.w);
    if (kPass == 1) {
        for (int i0 = 0; i0 <= j; i0 += 8) {
            T ac[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) ac[u] = T(0);
            FG_LOOP(e) {
                T we = w[e];
                if (i0 == 0) {
                    for (int i = 0; i <= j; ++i) we -= cv[i] * V[(int64_t)i * A.vs + e];
                    w[e] = we;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (i0 + u <= j) ac[u] += we * V[(int64_t)(i0 + u) * A.vs + e];
            }
            double acc[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] = (double)ac[u];
            fg_block_sums<8>(acc, min(8, j + 1 - i0), A.part, i0, A.G, sh);
        }
    } else {
        T n2 = T(0);
        double mx = 0.0;
        FG_LOOP(e) {
            T we = w[e];
            for (int i = 0; i <= j; ++i) we -= cv[i] * V[(int64_t)i * A.vs + e];
            w[e] = we;
            n2 += we * we;
            mx = fmax(mx, (double)fabs(we));
        }
        fg_block_one((double)n2, false, A.part, kSlotNorm, A.G, sh[0]);
        fg_block_one(mx, true, A.part, kSlotMax, A.G, sh[0]);
    }
}

// h_{j+1,j} = ||w||, the rotations of column j, the residual estimate |g_{j+1}|
// and whether the cycle goes on (FP64, one thread).
__global__ void __launch_bounds__(kFgRed) k_fg_givens(const __grid_constant__ FgArgs A)
{
    __shared__ double red[2];
    const int wid = threadIdx.x >> 5;
    if (wid < 2) {
        const double t = fg_slot(A.part, wid == 0 ? kSlotNorm : kSlotMax, A.G, wid == 1);
        if ((threadIdx.x & 31) == 0) red[wid] = t;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    FgState &S = *A.st;
    FgHead &h = S.h;
    const int j = h.j;
    const double hn = sqrt(red[0]);
    double *H = S.H;
    for (int i = 0; i <= j; ++i) H[i * kMaxM + j] = S.hc[i];
    for (int i = 0; i < j; ++i) {
        const double t0 = H[i * kMaxM + j], t1 = H[(i + 1) * kMaxM + j];
        H[i * kMaxM + j] = S.cs[i] * t0 + S.sn[i] * t1;
        H[(i + 1) * kMaxM + j] = -S.sn[i] * t0 + S.cs[i] * t1;
    }
    const double aa = H[j * kMaxM + j];
    const double den = hypot(aa, hn);
    double c = 1.0, sn = 0.0;
    if (den != 0.0) {
        c = aa / den;
        sn = hn / den;
    }
    S.cs[j] = c;
    S.sn[j] = sn;
    H[j * kMaxM + j] = c * aa + sn * hn;
    S.g[j + 1] = -sn * S.g[j];
    S.g[j] = c * S.g[j];
    h.it += 1;
    h.jsum += j;
    h.hn = hn;
    h.vscale = hn > 0.0 ? red[1] / hn : 0.0;
    h.j = j + 1;
    h.k = j + 1;
    const double gj = S.g[j + 1];
    const bool stop = !isfinite(gj) || fabs(gj) <= h.tol_in || j + 1 >= A.m || h.it >= A.maxit || hn == 0.0;
    cudaGraphSetConditional(A.h_in, stop ? 0u : 1u);
}

// v_{j+1} = w / h_{j+1,j}.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_fg_normalise(const __grid_constant__ FgArgs A)
{
    const FgHead &h = A.st->h;
    const double hn = h.hn;
    if (!(hn > 0.0) || !isfinite(hn)) return;
    const T inv = T(1.0 / hn);
    T *__restrict__ Vj = static_cast<T *>(A.V) + (int64_t)h.j * A.vs;
    const T *__restrict__ w = static_cast<const T *>(A.w);
    FG_LOOP(e) Vj[e] = w[e] * inv;
}

// y = R^-1 g over the k steps of the cycle (FP64, one thread).
__global__ void k_fg_backsolve(const __grid_constant__ FgArgs A)
{
    if (threadIdx.x != 0) return;
    FgState &S = *A.st;
    const int k = S.h.k;
    for (int i = k - 1; i >= 0; --i) {
        double acc = S.g[i];
        for (int l = i + 1; l < k; ++l) acc -= S.H[i * kMaxM + l] * S.y[l];
        S.y[i] = acc / S.H[i * kMaxM + i];
    }
}

// x_t = x + sum_i y_i z_i (FP64).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_fg_update(const __grid_constant__ FgArgs A)
{
    __shared__ double ys[kMaxM];
    const FgState &S = *A.st;
    const int k = S.h.k;
    for (int i = threadIdx.x; i < k; i += kBlock) ys[i] = S.y[i];
    __syncthreads();
    const T *__restrict__ Z = static_cast<const T *>(A.Z);
    FG_LOOP(e) {
        double xe = A.x[e];
        for (int i = 0; i < k; ++i) xe += ys[i] * (double)Z[(int64_t)i * A.vs + e];
        A.xt[e] = xe;
    }
}

// Accept the trial when its FP64 residual is below beta, else fall back (or,
// already plain, stop); whether the outer loop goes on.
__global__ void __launch_bounds__(kFgRed) k_fg_decide(const __grid_constant__ FgArgs A)
{
    __shared__ double red[2];
    const int wid = threadIdx.x >> 5;
    if (wid < 2) {
        const double t = fg_slot(A.part, wid == 0 ? kSlotNorm : kSlotMax, A.G, wid == 1);
        if ((threadIdx.x & 31) == 0) red[wid] = t;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    FgHead &h = A.st->h;
    const double bt = sqrt(red[0]);
    h.beta_t = bt;
    const bool acc = isfinite(bt) && bt < h.beta;
    h.accept = acc ? 1 : 0;
    if (acc) {
        h.beta = bt;
        h.vscale0 = bt > 0.0 ? red[1] / bt : 0.0;
    } else if (!h.fallback) {
        h.fallback = 1;
        A.units[0] = 0;          // the network's kernels now have nothing to do
    } else {
        h.stall = 1;
    }
    int done = 1;
    if (h.beta <= h.tol) h.status = MPM_OK;
    else if (h.it >= A.maxit || h.stall) h.status = MPM_ERR_NOCONV;
    else done = 0;
    h.done = done;
    cudaGraphSetConditional(A.h_out, done ? 0u : 1u);
}

// x = x_t, r = r_t when the trial was accepted.
__global__ void __launch_bounds__(kBlock) k_fg_commit(const __grid_constant__ FgArgs A)
{
    if (!A.st->h.accept) return;
    FG_LOOP(e) {
        A.x[e] = A.xt[e];
        A.r[e] = A.rt[e];
    }
}

#undef FG_LOOP

}  // namespace mpm

using namespace mpm;

namespace {

// The graph of the last solve and what it was built from.
struct FgCache {
    std::vector<char> key;
    cudaGraphExec_t exec = nullptr;
};

template <typename T>
void key_put(std::vector<char> &k, const T &v)
{
    const char *p = reinterpret_cast<const char *>(&v);
    k.insert(k.end(), p, p + sizeof(T));
}

// A conditional handle in the graph that capturing stream cs records into.
mpm_status cond_handle(mpm_ctx *ctx, cudaStream_t cs, cudaGraphConditionalHandle *h)
{
    cudaStreamCaptureStatus stat;
    cudaGraph_t g = nullptr;
    MPM_CU(cudaStreamGetCaptureInfo(cs, &stat, nullptr, &g, nullptr, nullptr, nullptr));
    if (stat != cudaStreamCaptureStatusActive || !g) return mpm_fail(ctx, MPM_ERR_CUDA, "fgmres: stream not capturing");
    MPM_CU(cudaGraphConditionalHandleCreate(h, g, 0, 0));
    return MPM_OK;
}

// A WHILE node on handle h at the current position of capturing stream cs
// (later work on cs follows it); *body receives its body graph.
mpm_status add_while(mpm_ctx *ctx, cudaStream_t cs, cudaGraphConditionalHandle h, cudaGraph_t *body)
{
    cudaStreamCaptureStatus stat;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    MPM_CU(cudaStreamGetCaptureInfo(cs, &stat, nullptr, &g, &deps, nullptr, &nd));
    if (stat != cudaStreamCaptureStatusActive || !g) return mpm_fail(ctx, MPM_ERR_CUDA, "fgmres: stream not capturing");
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t n = nullptr;
    MPM_CU(cudaGraphAddNode(&n, g, deps, nullptr, nd, &p));
    MPM_CU(cudaStreamUpdateCaptureDependencies(cs, &n, nullptr, 1, cudaStreamSetCaptureDependencies));
    *body = p.conditional.phGraph_out[0];
    return MPM_OK;
}

struct FgPlan {
    mpm_ctx *ctx;
    mpm_cnn *cnn;
    mpm_subgrid *sub;
    const mpm_lattice *lat;
    const mpm_params *prm;
    bool f32;
    int nsp;
    FgArgs A[kMaxSpecies];
};

template <typename T>
mpm_status capture_species(const FgPlan &P, FgArgs A, cudaStream_t cs0, cudaStream_t cs1, cudaStream_t cs2)
{
    mpm_ctx *ctx = P.ctx;
    const int G = A.G;
    mpm_status r = cond_handle(ctx, cs0, &A.h_out);
    if (r != MPM_OK) return r;
    k_fg_residual<true><<<G, kBlock, 0, cs0>>>(A);
    k_fg_init<<<1, kFgRed, 0, cs0>>>(A);
    MPM_CU(cudaGetLastError());
    cudaGraph_t outer = nullptr, inner = nullptr;
    r = add_while(ctx, cs0, A.h_out, &outer);
    if (r != MPM_OK) return r;
    MPM_CU(cudaStreamBeginCaptureToGraph(cs1, outer, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    r = cond_handle(ctx, cs1, &A.h_in);
    if (r == MPM_OK) {
        k_fg_cycle<T><<<G, kBlock, 0, cs1>>>(A);
        r = mpm_cuda_check(ctx, cudaGetLastError(), "fgmres cycle");
    }
    if (r == MPM_OK) r = add_while(ctx, cs1, A.h_in, &inner);
    if (r == MPM_OK) {
        const cudaError_t e = cudaStreamBeginCaptureToGraph(cs2, inner, nullptr, nullptr, 0,
                                                            cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) r = mpm_cuda_check(ctx, e, "fgmres: capture of the Arnoldi body");
        if (r == MPM_OK) {
            r = mpm_cnn_pc_apply(ctx, P.cnn, P.sub, P.lat, P.prm, A.s, A.V, sizeof(T) == 4, A.vs, &A.st->h.j,
                                 &A.st->h.vscale, const_cast<void *>(A.zc), cs2);
            k_fg_arnoldi<T><<<G, kBlock, 0, cs2>>>(A);
            k_fg_project<1><<<1, kFgRed, 0, cs2>>>(A);
            k_fg_orth<T, 1><<<G, kBlock, 0, cs2>>>(A);
            k_fg_project<2><<<1, kFgRed, 0, cs2>>>(A);
            k_fg_orth<T, 2><<<G, kBlock, 0, cs2>>>(A);
            k_fg_givens<<<1, kFgRed, 0, cs2>>>(A);
            k_fg_normalise<T><<<G, kBlock, 0, cs2>>>(A);
            const cudaError_t e2 = cudaGetLastError();
            if (r == MPM_OK) r = mpm_cuda_check(ctx, e2, "fgmres Arnoldi step");
            const cudaError_t e3 = cudaStreamEndCapture(cs2, &inner);
            if (r == MPM_OK) r = mpm_cuda_check(ctx, e3, "fgmres: end of the Arnoldi body capture");
        }
    }
    if (r == MPM_OK) {
        k_fg_backsolve<<<1, 32, 0, cs1>>>(A);
        k_fg_update<T><<<G, kBlock, 0, cs1>>>(A);
        k_fg_residual<false><<<G, kBlock, 0, cs1>>>(A);
        k_fg_decide<<<1, kFgRed, 0, cs1>>>(A);
        k_fg_commit<<<G, kBlock, 0, cs1>>>(A);
        r = mpm_cuda_check(ctx, cudaGetLastError(), "fgmres cycle end");
    }
    const cudaError_t e4 = cudaStreamEndCapture(cs1, &outer);
    if (r == MPM_OK) r = mpm_cuda_check(ctx, e4, "fgmres: end of the cycle capture");
    return r;
}

}  // namespace

void mpm_fgmres_release(mpm_ctx *ctx)
{
    FgCache *C = (FgCache *)ctx->fg_cache;
    if (C) {
        if (C->exec) cudaGraphExecDestroy(C->exec);
        delete C;
    }
    ctx->fg_cache = nullptr;
    for (int i = 0; i < 3; ++i)
        if (ctx->fg_cs[i]) cudaStreamDestroy(ctx->fg_cs[i]);
    for (int i = 0; i < 3; ++i) ctx->fg_cs[i] = nullptr;
}

mpm_status mpm_solve_fgmres_impl(mpm_ctx *ctx, mpm_cnn *cnn, mpm_subgrid *sub, const mpm_lattice *lat,
                                 const mpm_params *prm, const mpm_lattice *scatter_to, const mpm_opts *opt,
                                 mpm_report *rep, cudaStream_t st)
{
    if (!cnn || !sub || !lat || !prm || !opt) return mpm_fail(ctx, MPM_ERR_ARG, "fgmres: null argument");
    if (!sub->extracted || !sub->assembled) return mpm_fail(ctx, MPM_ERR_ARG, "fgmres: subgrid not assembled");
    if (sub->nspecies > 3 || prm->nspecies != sub->nspecies)
        return mpm_fail(ctx, MPM_ERR_ARG, "fgmres: the network covers species 0..2 of the assembled subgrid");
    const int m = opt->restart;
    if (m < 1 || m > MPM_MAX_RESTART || opt->maxit < 1 || !(opt->rtol >= 0.0) || !(opt->atol >= 0.0) ||
        (opt->precision != 0 && opt->precision != 1) || (opt->precision == 1 && !(opt->inner_rtol >= 0.0)))
        return mpm_fail(ctx, MPM_ERR_ARG, "fgmres: bad options");
    const bool f32 = opt->precision == 1;
    const int64_t NE = sub->NE;
    mpm_report R;
    memset(&R, 0, sizeof(R));
    R.box_voxels = (int64_t)sub->n[0] * sub->n[1] * sub->n[2];
    R.mask_voxels = sub->mask_voxels;
    R.stored_voxels = NE;
    const int nsp = sub->nspecies;
    if (NE == 0) {
        if (rep) *rep = R;
        sub->x_fresh = false;
        return scatter_to ? mpm_scatter_impl(ctx, sub, scatter_to, st) : MPM_OK;
    }
    // workspace: species states, partials, x_t / r / r_t, then V, Z, w, zc
    const int G = ctx->num_sms * 4;
    const int64_t vs = (NE + 63) & ~(int64_t)63;
    const size_t ts = f32 ? 4 : 8;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_st = al((size_t)nsp * sizeof(FgState));
    const size_t b_part = al((size_t)kSlots * G * sizeof(double));
    const size_t b_vec = al((size_t)vs * sizeof(double));
    const size_t b_kv = al((size_t)vs * ts);
    const size_t need = b_st + b_part + 3 * b_vec + (size_t)(2 * m + 3) * b_kv;
    mpm_status r = mpm_grow(ctx, (void **)&ctx->d_fg, &ctx->fg_cap, need, "fgmres workspace");
    if (r != MPM_OK) return r;
    char *p = (char *)ctx->d_fg;
    FgState *states = (FgState *)p;
    p += b_st;
    double *part = (double *)p;
    p += b_part;
    double *xt = (double *)p, *rr = (double *)(p + b_vec), *rt = (double *)(p + 2 * b_vec);
    p += 3 * b_vec;
    void *V = p;
    void *Z = p + (size_t)(m + 1) * b_kv;
    void *w = p + (size_t)(2 * m + 1) * b_kv;
    void *zc = p + (size_t)(2 * m + 2) * b_kv;
    const size_t hneed = (size_t)nsp * sizeof(FgHead);
    if (ctx->stage_cap < hneed) {
        if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
        ctx->h_stage = nullptr;
        ctx->stage_cap = 0;
        MPM_CU(cudaMallocHost(&ctx->h_stage, hneed + 4096));
        ctx->stage_cap = hneed + 4096;
    }
    // the network's plan (once per solve), its output zeroed (it writes the
    // in-mask elements only), the start iterates
    int32_t *units = nullptr;
    r = mpm_cnn_pc_plan(ctx, cnn, sub, lat, prm, st, &units);
    if (r != MPM_OK) return r;
    MPM_CU(cudaMemsetAsync(zc, 0, (size_t)vs * ts, st));
    for (int s = 0; s < nsp; ++s)
        if (!opt->x0_given && !sub->x_fresh)
            MPM_CU(cudaMemcpyAsync(sub->x[s], sub->cn[s], (size_t)NE * sizeof(double), cudaMemcpyDeviceToDevice, st));

    FgPlan P;
    memset(&P, 0, sizeof(P));
    P.ctx = ctx;
    P.cnn = cnn;
    P.sub = sub;
    P.lat = lat;
    P.prm = prm;
    P.f32 = f32;
    P.nsp = nsp;
    const SysDev S = mpm_make_sysdev(sub);
    std::vector<char> key;
    key_put(key, mpm_cnn_serial(cnn));
    key_put(key, (const void *)sub->tile_index);
    key_put(key, *lat);
    key_put(key, *prm);
    for (int s = 0; s < nsp; ++s) {
        FgArgs &A = P.A[s];
        memset(&A, 0, sizeof(A));
        A.S = S;
        A.s = s;
        A.G = G;
        A.NE = NE;
        A.vs = vs;
        A.x = sub->x[s];
        A.b = sub->b[s];
        A.xt = xt;
        A.r = rr;
        A.rt = rt;
        A.V = V;
        A.Z = Z;
        A.w = w;
        A.zc = zc;
        A.st = states + s;
        A.part = part;
        A.m = m;
        A.maxit = opt->maxit;
        A.rtol = opt->rtol;
        A.atol = opt->atol;
        A.inner_rtol = f32 ? opt->inner_rtol : 0.0;
        A.units = units;
        key_put(key, A);
    }
    FgCache *C = (FgCache *)ctx->fg_cache;
    if (!C) ctx->fg_cache = C = new FgCache;
    if (!C->exec || C->key != key) {
        if (C->exec) cudaGraphExecDestroy(C->exec);
        C->exec = nullptr;
        C->key.clear();
        for (int i = 0; i < 3; ++i)
            if (!ctx->fg_cs[i]) MPM_CU(cudaStreamCreateWithFlags(&ctx->fg_cs[i], cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        MPM_CU(cudaGraphCreate(&g, 0));
        const int64_t launches0 = ctx->launches;
        cudaError_t e = cudaStreamBeginCaptureToGraph(ctx->fg_cs[0], g, nullptr, nullptr, 0,
                                                      cudaStreamCaptureModeThreadLocal);
        r = e == cudaSuccess ? MPM_OK : mpm_cuda_check(ctx, e, "fgmres: graph capture");
        if (r == MPM_OK) {
            for (int s = 0; s < nsp && r == MPM_OK; ++s)
                r = f32 ? capture_species<float>(P, P.A[s], ctx->fg_cs[0], ctx->fg_cs[1], ctx->fg_cs[2])
                        : capture_species<double>(P, P.A[s], ctx->fg_cs[0], ctx->fg_cs[1], ctx->fg_cs[2]);
            e = cudaStreamEndCapture(ctx->fg_cs[0], &g);
            if (r == MPM_OK) r = mpm_cuda_check(ctx, e, "fgmres: end of the graph capture");
        }
        ctx->launches = launches0;
        if (r == MPM_OK) {
            e = cudaGraphInstantiate(&C->exec, g, 0);
            if (e != cudaSuccess) {
                C->exec = nullptr;
                r = mpm_cuda_check(ctx, e, "fgmres: graph instantiation");
            }
        }
        cudaGraphDestroy(g);
        if (r != MPM_OK) {
            cudaGetLastError();
            return r;
        }
        C->key = key;
    }
    MPM_CU(cudaEventRecord(ctx->ev0, st));
    MPM_CU(cudaGraphLaunch(C->exec, st));
    MPM_CU(cudaEventRecord(ctx->ev1, st));
    MPM_CU(cudaMemcpy2DAsync(ctx->h_stage, sizeof(FgHead), states, sizeof(FgState), sizeof(FgHead), (size_t)nsp,
                             cudaMemcpyDeviceToHost, st));
    MPM_CU(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    R.solve_ms = ms;
    const FgHead *H = (const FgHead *)ctx->h_stage;
    mpm_status worst = MPM_OK;
    for (int s = 0; s < nsp; ++s) {
        R.iters[s] = H[s].it;
        R.cycles[s] = H[s].cyc;
        R.status[s] = H[s].status;
        R.jsum[s] = H[s].jsum;
        R.res[s] = H[s].beta;
        R.bnorm[s] = H[s].bnorm;
        R.reorth[s] = H[s].it;            // every Arnoldi step takes both Gram-Schmidt passes
        R.fallback[s] = H[s].fallback;
        ctx->launches += kFgKernelsPerSpecies + (int64_t)H[s].cyc * kFgKernelsPerCycle +
                         (int64_t)H[s].it * (kFgKernelsPerStep + mpm_cnn_pc_launches());
        const mpm_status ss = (mpm_status)H[s].status;
        if (ss != MPM_OK && (worst == MPM_OK || ss == MPM_ERR_BREAKDOWN)) worst = ss;
    }
    sub->x_fresh = false;
    if (rep) *rep = R;
    r = mpm_cnn_check_err(ctx, cnn);
    if (r != MPM_OK) return r;
    if (scatter_to && worst != MPM_ERR_BREAKDOWN) {
        r = mpm_scatter_impl(ctx, sub, scatter_to, st);
        if (r != MPM_OK) return r;
    }
    if (worst != MPM_OK) mpm_fail(ctx, worst, "fgmres: not every species converged");
    return worst;
}
