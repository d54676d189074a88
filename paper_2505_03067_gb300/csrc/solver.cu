// solver.cu -- restarted GMRES (Saad & Schultz 1986, the solver named in
// Sec. 2.4) for the box systems, as ONE persistent cooperative kernel.
//
// Structure of a launch.  The grid is split into teams of co-resident CTAs;
// each team solves a list of systems, every species of a system in lock step.
// A cycle is
//   R   r = b - A x (FP64), ||r||, ||b||                       -> barrier
//   for j = 0..m-1 (classical Gram-Schmidt in two passes):
//     P1  w = A v_j (7-point stencil) and h_ij = <v_i, w>, i<=j -> barrier
//     P2  w -= sum_i h_ij v_i, ||w||                           -> barrier
//         Givens rotation of the new Hessenberg column (FP64, one thread per
//         species, redundantly in every CTA)
//   U   x += V y (y from the triangular solve)                 -> barrier
// and the next R pass doubles as the true-residual convergence test.  Krylov
// vectors are stored unnormalised with a scale sigma_i = 1/||v_i||, so no
// pass is spent on normalisation.
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
#include <cstring>
#include <type_traits>
#include <vector>
#include <algorithm>

#include "mpm_internal.cuh"

namespace mpm {

enum { ST_RUN = -1 };

struct SpState {
    double beta, bnorm, tol, tol_in;
    int32_t it, cyc, status, in_cycle, k, done, bad, pad;
};

template <int MAXM>
struct Smem {
    double H[kMaxSpecies][(MAXM + 1) * MAXM];
    double cs[kMaxSpecies][MAXM], sn[kMaxSpecies][MAXM];
    double g[kMaxSpecies][MAXM + 1], sig[kMaxSpecies][MAXM + 1], coef[kMaxSpecies][MAXM + 1];
    double red[kWarps][MAXM + 2];
    double tot[kKMax];
    SpState sp[kMaxSpecies];
    SysDev sys;
};

// CTA reduction of cnt per-thread values; thread i < cnt stores the CTA total
// of value i to out[i].
template <int N, typename AccT, int RS>
__device__ __forceinline__ void block_reduce_store(const AccT (&acc)[N], int cnt, double (*red)[RS], double *out)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i < cnt) {
            const double v = warp_sum((double)acc[i]);
            if (lane == 0) red[w][i] = v;
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < kWarps; ++q) s += red[q][threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// Team sum of the slots s*kKStride + i (i < cnt) of the species in smask, in a
// fixed order (lane l adds blocks l, l+32, ...; then a fixed shuffle tree).
__device__ __forceinline__ void team_reduce(const double *part, int b0, int nb, uint32_t smask, int cnt,
                                            double *tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nslot = kMaxSpecies * cnt;
    for (int q = w; q < nslot; q += kWarps) {
        const int s = q / cnt, i = q - s * cnt;
        if (!((smask >> s) & 1u)) continue;
        const int slot = s * kKStride + i;
        double v0 = 0.0, v1 = 0.0;
        int b = lane;
        for (; b + 32 < nb; b += 64) {
            v0 += __ldcg(part + (size_t)(b0 + b) * kKMax + slot);
            v1 += __ldcg(part + (size_t)(b0 + b + 32) * kKMax + slot);
        }
        if (b < nb) v0 += __ldcg(part + (size_t)(b0 + b) * kKMax + slot);
        const double v = warp_sum(v0 + v1);
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

// ---- R: r = b - A x in FP64; u_0 = r (stored in T); sums of r^2 and b^2 (mask rows)
template <typename T>
__device__ __forceinline__ void pass_residual(const SysDev &S, int s, bool first, int64_t e0, int64_t es,
                                              double &accR, double &accB)
{
    T *u0 = (T *)S.V[s];
    const double *__restrict__ x = S.x[s];
    const double *__restrict__ b = S.b[s];
    const double *__restrict__ dg = S.diag[s];
    const bool var = S.dfac != nullptr;
    for (int64_t e = e0; e < S.NE; e += es) {
        const uint32_t f = S.flags[e];
        const double xv = x[e];
        const double ns = var ? S.a * nbr_sum_var<double>(x, S.dfac, S.nbr, e, f, S.ltx, S.lty, S.ltz, S.Dsp[s])
                              : S.off[s] * nbr_sum<double>(x, S.nbr, e, f, S.ltx, S.lty, S.ltz);
        const double bv = b[e];
        const double r = bv - (dg[e] * xv - ns);
        u0[e] = (T)r;
        accR += r * r;
        if (first && (f & F_MASK)) accB += bv * bv;
    }
}

// ---- P1: w = sigma_j A u_j into slot j+1; acc[i] += u_i . w for i <= j
template <typename T, int MAXM>
__device__ __forceinline__ void pass_arnoldi1(const SysDev &S, int s, int j, double sigj, int64_t e0, int64_t es,
                                              T (&acc)[MAXM + 1])
{
    T *V = (T *)S.V[s];
    const int64_t vs = S.vstride;
    const T *uj = V + (int64_t)j * vs;
    T *wv = V + (int64_t)(j + 1) * vs;
    const T *__restrict__ dg = diag_of<T>(S, s);
    const T sj = (T)sigj;
    const bool var = S.dfac != nullptr;
    const T offT = (T)(var ? S.a : S.off[s]);
    for (int64_t e = e0; e < S.NE; e += es) {
        const uint32_t f = S.flags[e];
        const T xj = uj[e];
        const T ns = var ? nbr_sum_var<T>(uj, S.dfac, S.nbr, e, f, S.ltx, S.lty, S.ltz, S.Dsp[s])
                         : nbr_sum<T>(uj, S.nbr, e, f, S.ltx, S.lty, S.ltz);
        const T w = sj * (dg[e] * xj - offT * ns);
        wv[e] = w;
#pragma unroll
        for (int i = 0; i <= MAXM; ++i) {
            if (i < j) acc[i] += V[(int64_t)i * vs + e] * w;
            else if (i == j) acc[i] += xj * w;
        }
    }
}

// ---- P2: w -= sum_{i<=j} c_i u_i in place (c_i = h_ij sigma_i); acc += w^2
template <typename T, int MAXM>
__device__ __forceinline__ void pass_arnoldi2(const SysDev &S, int s, int j, const double *coef, int64_t e0,
                                              int64_t es, T &acc)
{
    T *V = (T *)S.V[s];
    const int64_t vs = S.vstride;
    T *wv = V + (int64_t)(j + 1) * vs;
    T c[MAXM + 1];
#pragma unroll
    for (int i = 0; i <= MAXM; ++i) c[i] = i <= j ? (T)coef[i] : T(0);
    for (int64_t e = e0; e < S.NE; e += es) {
        T w = wv[e];
#pragma unroll
        for (int i = 0; i <= MAXM; ++i)
            if (i <= j) w -= c[i] * V[(int64_t)i * vs + e];
        wv[e] = w;
        acc += w * w;
    }
}

// ---- U: x += sum_{i<k} c_i u_i (c_i = y_i sigma_i); FP32 path: FP32 correction added in FP64
template <typename T, int MAXM>
__device__ __forceinline__ void pass_update(const SysDev &S, int s, int k, const double *coef, int64_t e0, int64_t es)
{
    const T *V = (const T *)S.V[s];
    const int64_t vs = S.vstride;
    double *__restrict__ x = S.x[s];
    T c[MAXM];
#pragma unroll
    for (int i = 0; i < MAXM; ++i) c[i] = i < k ? (T)coef[i] : T(0);
    for (int64_t e = e0; e < S.NE; e += es) {
        T d = T(0);
#pragma unroll
        for (int i = 0; i < MAXM; ++i)
            if (i < k) d += c[i] * V[(int64_t)i * vs + e];
        x[e] += (double)d;
    }
}

template <typename T, int MAXM>
__global__ void __launch_bounds__(kBlock) k_gmres(SolveArgs A)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    Smem<MAXM> &sm = *reinterpret_cast<Smem<MAXM> *>(smraw);
    if ((int)blockIdx.x == A.skip_block) return;    // fault injection: this CTA never arrives
    const int tid = threadIdx.x;
    const int team = A.block_team[blockIdx.x];
    const TeamDesc td = A.teams[team];
    const int rank = (int)blockIdx.x - td.first_block, nb = td.nblocks;
    uint32_t *bar = A.bar + 32 * team;
    uint32_t epoch = 0;
    int pbuf = 0;
    const size_t pstride = (size_t)gridDim.x * kKMax;
    const int64_t e0 = (int64_t)rank * kBlock + tid, es = (int64_t)nb * kBlock;
    constexpr bool kF32 = std::is_same<T, float>::value;

    for (int si = td.sys_begin; si < td.sys_end; ++si) {
        const int sys_id = A.sys_order[si];
        if (tid == 0) sm.sys = A.sys[sys_id];
        __syncthreads();
        const SysDev &S = sm.sys;
        const int NS = S.nspecies;
        if (tid < NS) {
            const bool bad_id = S.err && __ldcg(S.err) != 0;   // cell id outside the rate tables
            SpState &p = sm.sp[tid];
            p.beta = p.bnorm = p.tol = p.tol_in = 0.0;
            p.it = p.cyc = p.in_cycle = p.k = p.bad = 0;
            p.done = bad_id ? 1 : 0;
            p.status = bad_id ? MPM_ERR_ARG : ST_RUN;
        }
        __syncthreads();
        bool first = true;
        for (;;) {
            // ---------------- R: true residual (FP64)
            uint32_t rmask = 0;
            for (int s = 0; s < NS; ++s) if (!sm.sp[s].done) rmask |= 1u << s;
            for (int s = 0; s < NS; ++s) {
                if (!((rmask >> s) & 1u)) continue;
                double acc[2] = {0.0, 0.0};
                pass_residual<T>(S, s, first, e0, es, acc[0], acc[1]);
                block_reduce_store<2, double, MAXM + 2>(acc, 2, sm.red,
                                                        A.partials + pbuf * pstride + (size_t)blockIdx.x * kKMax + s * kKStride);
            }
            if (!team_barrier(bar, epoch, nb, A.abort_flag, A.timeout_ns)) return;
            team_reduce(A.partials + pbuf * pstride, td.first_block, nb, rmask, 2, sm.tot);
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
                    for (int i = 0; i <= MAXM; ++i) sm.g[tid][i] = 0.0;
                    sm.g[tid][0] = beta;
                    sm.sig[tid][0] = 1.0 / beta;
                    p.tol_in = kF32 ? fmax(p.tol, A.inner_rtol * beta) : p.tol;
                }
            }
            first = false;
            __syncthreads();
            bool any = false;
            for (int s = 0; s < NS; ++s) any |= sm.sp[s].in_cycle != 0;
            if (!any) break;

            // ---------------- Arnoldi
            for (int j = 0; j < A.m; ++j) {
                uint32_t cm = 0;
                for (int s = 0; s < NS; ++s) if (sm.sp[s].in_cycle) cm |= 1u << s;
                if (!cm) break;
                for (int s = 0; s < NS; ++s) {
                    if (!((cm >> s) & 1u)) continue;
                    T acc[MAXM + 1];
#pragma unroll
                    for (int i = 0; i <= MAXM; ++i) acc[i] = T(0);
                    pass_arnoldi1<T, MAXM>(S, s, j, sm.sig[s][j], e0, es, acc);
                    block_reduce_store<MAXM + 1, T, MAXM + 2>(acc, j + 1, sm.red,
                                                             A.partials + pbuf * pstride + (size_t)blockIdx.x * kKMax + s * kKStride);
                }
                if (!team_barrier(bar, epoch, nb, A.abort_flag, A.timeout_ns)) return;
                team_reduce(A.partials + pbuf * pstride, td.first_block, nb, cm, j + 1, sm.tot);
                pbuf ^= 1;
                if (tid < NS && ((cm >> tid) & 1u)) {
                    for (int i = 0; i <= j; ++i) {
                        const double h = sm.sig[tid][i] * sm.tot[tid * kKStride + i];
                        sm.H[tid][i * MAXM + j] = h;
                        sm.coef[tid][i] = h * sm.sig[tid][i];
                    }
                }
                __syncthreads();
                for (int s = 0; s < NS; ++s) {
                    if (!((cm >> s) & 1u)) continue;
                    T acc[1] = {T(0)};
                    pass_arnoldi2<T, MAXM>(S, s, j, sm.coef[s], e0, es, acc[0]);
                    block_reduce_store<1, T, MAXM + 2>(acc, 1, sm.red,
                                                      A.partials + pbuf * pstride + (size_t)blockIdx.x * kKMax + s * kKStride);
                }
                if (!team_barrier(bar, epoch, nb, A.abort_flag, A.timeout_ns)) return;
                team_reduce(A.partials + pbuf * pstride, td.first_block, nb, cm, 1, sm.tot);
                pbuf ^= 1;
                if (tid < NS && ((cm >> tid) & 1u)) {
                    SpState &p = sm.sp[tid];
                    double *H = sm.H[tid];
                    double *cs = sm.cs[tid], *sn = sm.sn[tid], *g = sm.g[tid];
                    const double hn = sqrt(sm.tot[tid * kKStride]);
                    H[(j + 1) * MAXM + j] = hn;
                    for (int i = 0; i < j; ++i) {
                        const double t0 = H[i * MAXM + j], t1 = H[(i + 1) * MAXM + j];
                        H[i * MAXM + j] = cs[i] * t0 + sn[i] * t1;
                        H[(i + 1) * MAXM + j] = -sn[i] * t0 + cs[i] * t1;
                    }
                    const double aa = H[j * MAXM + j], bb = hn;
                    if (bb == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
                    else {
                        const double r = hypot(aa, bb);
                        cs[j] = aa / r;
                        sn[j] = bb / r;
                    }
                    H[j * MAXM + j] = cs[j] * aa + sn[j] * bb;
                    H[(j + 1) * MAXM + j] = 0.0;
                    g[j + 1] = -sn[j] * g[j];
                    g[j] = cs[j] * g[j];
                    p.it += 1;
                    p.k = j + 1;
                    if (!isfinite(g[j + 1]) || !isfinite(H[j * MAXM + j])) {
                        p.status = MPM_ERR_BREAKDOWN;
                        p.bad = 1;
                        p.done = 1;
                        p.in_cycle = 0;
                    } else if (fabs(g[j + 1]) <= p.tol_in || p.it >= A.maxit || hn <= 1e-300 || j + 1 == A.m) {
                        p.in_cycle = 0;
                    } else {
                        sm.sig[tid][j + 1] = 1.0 / hn;
                    }
                }
                __syncthreads();
            }

            // ---------------- least squares: R y = g (back substitution)
            if (tid < NS) {
                SpState &p = sm.sp[tid];
                if (!p.bad && p.k > 0) {
                    const double *H = sm.H[tid];
                    double *y = sm.coef[tid];
                    for (int i = p.k - 1; i >= 0; --i) {
                        double acc = sm.g[tid][i];
                        for (int l = i + 1; l < p.k; ++l) acc -= H[i * MAXM + l] * y[l];
                        y[i] = acc / H[i * MAXM + i];
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
            // ---------------- U: x += V y
            for (int s = 0; s < NS; ++s) {
                const SpState &p = sm.sp[s];
                if (p.bad || p.k == 0) continue;
                pass_update<T, MAXM>(S, s, p.k, sm.coef[s], e0, es);
            }
            __syncthreads();
            if (tid < NS) sm.sp[tid].k = 0;
            if (!team_barrier(bar, epoch, nb, A.abort_flag, A.timeout_ns)) return;
        }
        if (rank == 0 && tid < NS) {
            const SpState &p = sm.sp[tid];
            SysReport *R = A.reports + sys_id;
            R->iters[tid] = p.it;
            R->cycles[tid] = p.cyc;
            R->status[tid] = p.status;
            R->res[tid] = p.beta;
            R->bnorm[tid] = p.bnorm;
        }
        __syncthreads();
    }
}

typedef void (*KernFn)(SolveArgs);

template <typename T, int MAXM>
struct KernInfo {
    static KernFn fn() { return k_gmres<T, MAXM>; }
    static size_t smem() { return sizeof(Smem<MAXM>); }
};

static KernFn pick(int prec, int maxm, size_t &smem)
{
    if (prec == 0) {
        if (maxm == 8) { smem = KernInfo<double, 8>::smem(); return KernInfo<double, 8>::fn(); }
        if (maxm == 16) { smem = KernInfo<double, 16>::smem(); return KernInfo<double, 16>::fn(); }
        smem = KernInfo<double, 32>::smem(); return KernInfo<double, 32>::fn();
    }
    if (maxm == 8) { smem = KernInfo<float, 8>::smem(); return KernInfo<float, 8>::fn(); }
    if (maxm == 16) { smem = KernInfo<float, 16>::smem(); return KernInfo<float, 16>::fn(); }
    smem = KernInfo<float, 32>::smem(); return KernInfo<float, 32>::fn();
}

}  // namespace mpm

using namespace mpm;

SysDev mpm_make_sysdev(const mpm_subgrid *sub)
{
    SysDev S;
    memset(&S, 0, sizeof(S));
    S.NE = sub->NE;
    S.ltx = sub->lt[0];
    S.lty = sub->lt[1];
    S.ltz = sub->lt[2];
    S.nspecies = sub->nspecies;
    S.nbr = sub->nbr;
    S.flags = sub->flags;
    S.dfac = sub->dfac;
    S.a = sub->a;
    S.err = sub->err;
    for (int s = 0; s < sub->nspecies; ++s) {
        S.x[s] = sub->x[s];
        S.b[s] = sub->b[s];
        S.diag[s] = sub->diag[s];
        S.diag32[s] = sub->diag32[s];
        S.off[s] = sub->off[s];
        S.Dsp[s] = sub->Dsp[s];
    }
    return S;
}

int mpm_solver_max_blocks(mpm_ctx *ctx, int prec, int m)
{
    const int maxm = m <= 8 ? 8 : (m <= 16 ? 16 : 32);
    size_t smem = 0;
    KernFn fn = pick(prec, maxm, smem);
    if (smem > 48 * 1024) cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, kBlock, smem) != cudaSuccess) return 0;
    return per_sm * ctx->num_sms;
}

static size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

// Longest-first partition of systems onto teams (the batched form).  Each team
// gets a share of the grid proportional to its work, at least one CTA.
static void plan_teams(const std::vector<double> &work, int G, std::vector<TeamDesc> &teams,
                       std::vector<int32_t> &order, std::vector<int32_t> &block_team)
{
    const int nsys = (int)work.size();
    std::vector<int> idx(nsys);
    for (int i = 0; i < nsys; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return work[a] > work[b]; });
    double total = 0.0;
    for (double w : work) total += w;
    const int nteam = std::max(1, std::min(nsys, G));
    std::vector<std::vector<int>> members(nteam);
    std::vector<double> load(nteam, 0.0);
    for (int i : idx) {           // LPT: next-largest system onto the least-loaded team
        int best = 0;
        for (int t = 1; t < nteam; ++t) if (load[t] < load[best]) best = t;
        members[best].push_back(i);
        load[best] += work[i];
    }
    // CTAs proportional to load (largest remainder), at least one each
    std::vector<int> nbk(nteam, 1);
    int left = G - nteam;
    if (left > 0 && total > 0) {
        std::vector<std::pair<double, int>> rem;
        int given = 0;
        for (int t = 0; t < nteam; ++t) {
            const double ideal = load[t] / total * left;
            const int fl = (int)ideal;
            nbk[t] += fl;
            given += fl;
            rem.push_back({ideal - fl, t});
        }
        std::stable_sort(rem.begin(), rem.end(), [](const std::pair<double, int> &a, const std::pair<double, int> &b) {
            return a.first > b.first;
        });
        for (int r = 0; r < left - given && r < (int)rem.size(); ++r) nbk[rem[r].second] += 1;
    }
    teams.clear();
    order.clear();
    block_team.clear();
    int fb = 0;
    for (int t = 0; t < nteam; ++t) {
        TeamDesc d;
        d.first_block = fb;
        d.nblocks = nbk[t];
        d.sys_begin = (int32_t)order.size();
        for (int i : members[t]) order.push_back(i);
        d.sys_end = (int32_t)order.size();
        teams.push_back(d);
        for (int b = 0; b < nbk[t]; ++b) block_team.push_back(t);
        fb += nbk[t];
    }
}

mpm_status mpm_solve_impl(mpm_ctx *ctx, mpm_subgrid *const *subs, const mpm_lattice *const *scatter_to,
                          int32_t nsys, const mpm_opts *opt, mpm_report *reps, cudaStream_t st)
{
    if (!subs || !opt || nsys < 1) return mpm_fail(ctx, MPM_ERR_ARG, "solve: null argument or nsys < 1");
    if (opt->restart < 1 || opt->restart > MPM_MAX_RESTART) return mpm_fail(ctx, MPM_ERR_ARG, "solve: restart out of [1, 32]");
    if (opt->maxit < 1) return mpm_fail(ctx, MPM_ERR_ARG, "solve: maxit < 1");
    if (opt->precision != 0 && opt->precision != 1) return mpm_fail(ctx, MPM_ERR_ARG, "solve: precision must be 0 or 1");
    if (!(opt->rtol >= 0.0) || !(opt->atol >= 0.0)) return mpm_fail(ctx, MPM_ERR_ARG, "solve: negative tolerance");
    if (opt->precision == 1 && !(opt->inner_rtol > 0.0 && opt->inner_rtol < 1.0))
        return mpm_fail(ctx, MPM_ERR_ARG, "solve: inner_rtol must be in (0, 1)");
    for (int i = 0; i < nsys; ++i) {
        if (!subs[i]) return mpm_fail(ctx, MPM_ERR_ARG, "solve: null subgrid");
        if (!subs[i]->assembled) return mpm_fail(ctx, MPM_ERR_ARG, "solve: subgrid not assembled");
    }
    const int m = opt->restart;
    const int maxm = m <= 8 ? 8 : (m <= 16 ? 16 : 32);
    const size_t tsz = opt->precision ? sizeof(float) : sizeof(double);

    // ---- Krylov bases and initial guesses
    std::vector<SysDev> sd(nsys);
    std::vector<double> work(nsys);
    for (int i = 0; i < nsys; ++i) {
        mpm_subgrid *sub = subs[i];
        const int64_t vstride = sub->NE > 0 ? ((sub->NE + 63) / 64) * 64 : 64;
        const size_t per = a256((size_t)(m + 1) * (size_t)vstride * tsz);
        mpm_status r = mpm_grow(ctx, &sub->krylov, &sub->krylov_bytes, per * sub->nspecies, "Krylov basis");
        if (r != MPM_OK) return r;
        if (!opt->x0_given && !sub->x_fresh) {
            for (int s = 0; s < sub->nspecies; ++s)
                MPM_CU(cudaMemcpyAsync(sub->x[s], sub->cn[s], (size_t)sub->NE * sizeof(double), cudaMemcpyDeviceToDevice, st));
            sub->x_fresh = true;
        }
        sd[i] = mpm_make_sysdev(sub);
        sd[i].vstride = vstride;
        for (int s = 0; s < sub->nspecies; ++s) sd[i].V[s] = (char *)sub->krylov + per * s;
        work[i] = (double)sub->NE * sub->nspecies + 1.0;
    }

    // ---- grid and teams
    size_t smem = 0;
    KernFn fn = pick(opt->precision, maxm, smem);
    const int gmax = mpm_solver_max_blocks(ctx, opt->precision, m);
    if (gmax < 1) return mpm_fail(ctx, MPM_ERR_CUDA, "solve: occupancy query failed");
    int G;
    if (opt->nblocks > 0) G = std::min(opt->nblocks, gmax);
    else {
        double tot = 0.0;
        for (double w : work) tot += w;
        // about 4 elements per thread per species at least; at most 2 CTAs per SM
        const double want = tot / (kBlock * 4.0);
        G = (int)std::min<double>(std::min(gmax, 2 * ctx->num_sms), std::max(1.0, want));
        G = std::max(G, std::min(nsys, gmax));
    }
    std::vector<TeamDesc> teams;
    std::vector<int32_t> order, block_team;
    plan_teams(work, G, teams, order, block_team);
    const int nteam = (int)teams.size();

    // ---- descriptors to the device (pinned staging)
    const size_t o_sys = 0;
    const size_t o_team = a256(o_sys + sizeof(SysDev) * nsys);
    const size_t o_order = a256(o_team + sizeof(TeamDesc) * nteam);
    const size_t o_bt = a256(o_order + sizeof(int32_t) * nsys);
    const size_t o_rep = a256(o_bt + sizeof(int32_t) * G);
    const size_t args_need = a256(o_rep + sizeof(SysReport) * nsys);
    mpm_status r = mpm_grow(ctx, &ctx->d_args, &ctx->args_cap, args_need, "solver descriptors");
    if (r != MPM_OK) return r;
    if (ctx->stage_cap < args_need + 256) {
        if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
        ctx->h_stage = nullptr;
        MPM_CU(cudaMallocHost(&ctx->h_stage, args_need + 4096));
        ctx->stage_cap = args_need + 4096;
    }
    MPM_CU(cudaStreamSynchronize(st));   // the staging buffer is reused across calls
    char *hs = (char *)ctx->h_stage;
    memcpy(hs + o_sys, sd.data(), sizeof(SysDev) * nsys);
    memcpy(hs + o_team, teams.data(), sizeof(TeamDesc) * nteam);
    memcpy(hs + o_order, order.data(), sizeof(int32_t) * nsys);
    memcpy(hs + o_bt, block_team.data(), sizeof(int32_t) * G);
    MPM_CU(cudaMemcpyAsync(ctx->d_args, hs, o_rep, cudaMemcpyHostToDevice, st));
    const size_t pneed = 2 * (size_t)G * kKMax * sizeof(double);
    r = mpm_grow(ctx, (void **)&ctx->d_partials, &ctx->partials_cap, pneed, "reduction partials");
    if (r != MPM_OK) return r;
    if (ctx->bar_cap < nteam) {
        if (ctx->d_bar) cudaFree(ctx->d_bar);
        ctx->d_bar = nullptr;
        MPM_CU(cudaMalloc(&ctx->d_bar, (size_t)nteam * 32 * sizeof(uint32_t)));
        ctx->bar_cap = nteam;
    }
    MPM_CU(cudaMemsetAsync(ctx->d_bar, 0, (size_t)nteam * 32 * sizeof(uint32_t), st));
    MPM_CU(cudaMemsetAsync(ctx->d_abort, 0, sizeof(int32_t), st));
    MPM_CU(cudaMemsetAsync((char *)ctx->d_args + o_rep, 0, sizeof(SysReport) * nsys, st));

    SolveArgs sa;
    sa.sys = (const SysDev *)((char *)ctx->d_args + o_sys);
    sa.teams = (const TeamDesc *)((char *)ctx->d_args + o_team);
    sa.sys_order = (const int32_t *)((char *)ctx->d_args + o_order);
    sa.block_team = (const int32_t *)((char *)ctx->d_args + o_bt);
    sa.reports = (SysReport *)((char *)ctx->d_args + o_rep);
    sa.partials = ctx->d_partials;
    sa.bar = ctx->d_bar;
    sa.abort_flag = ctx->d_abort;
    sa.rtol = opt->rtol;
    sa.atol = opt->atol;
    sa.inner_rtol = opt->precision ? opt->inner_rtol : 0.0;
    sa.m = m;
    sa.maxit = opt->maxit;
    sa.timeout_ns = ctx->timeout_ns;
    sa.skip_block = ctx->skip_block;
    void *kargs[] = {&sa};
    MPM_CU(cudaEventRecord(ctx->ev0, st));
    MPM_CU(cudaLaunchCooperativeKernel((const void *)fn, dim3(G), dim3(kBlock), kargs, smem, st));
    MPM_CU(cudaEventRecord(ctx->ev1, st));

    // ---- results
    SysReport *hrep = (SysReport *)(hs + o_rep);
    MPM_CU(cudaMemcpyAsync(hrep, sa.reports, sizeof(SysReport) * nsys, cudaMemcpyDeviceToHost, st));
    int32_t *hflags = (int32_t *)(hs + args_need);
    MPM_CU(cudaMemcpyAsync(hflags, ctx->d_abort, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MPM_CU(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    const bool timed_out = hflags[0] != 0;
    bool bad_id = false;

    mpm_status worst = MPM_OK;
    auto rank_of = [](int s) {
        switch (s) {
        case MPM_OK: return 0;
        case MPM_ERR_NOCONV: return 1;
        case MPM_ERR_BREAKDOWN: return 2;
        case MPM_ERR_ARG: return 3;
        case MPM_ERR_TIMEOUT: return 4;
        default: return 5;
        }
    };
    for (int i = 0; i < nsys; ++i) {
        mpm_subgrid *sub = subs[i];
        sub->x_fresh = false;
        mpm_report R;
        memset(&R, 0, sizeof(R));
        for (int s = 0; s < sub->nspecies; ++s) {
            R.iters[s] = hrep[i].iters[s];
            R.cycles[s] = hrep[i].cycles[s];
            int stt = hrep[i].status[s];
            if (timed_out) stt = MPM_ERR_TIMEOUT;
            else if (stt == ST_RUN) stt = MPM_ERR_NOCONV;
            if (stt == MPM_ERR_ARG) bad_id = true;
            R.status[s] = stt;
            R.res[s] = hrep[i].res[s];
            R.bnorm[s] = hrep[i].bnorm[s];
            if (rank_of(stt) > rank_of(worst)) worst = (mpm_status)stt;
        }
        R.box_voxels = (int64_t)sub->n[0] * sub->n[1] * sub->n[2];
        R.mask_voxels = sub->mask_voxels;
        R.stored_voxels = sub->NE;
        R.solve_ms = ms;
        if (reps) reps[i] = R;
        if (!timed_out && scatter_to && scatter_to[i]) {
            r = mpm_scatter_impl(ctx, sub, scatter_to[i], st);
            if (r != MPM_OK) return r;
        }
    }
    if (timed_out) {
        MPM_CU(cudaMemsetAsync(ctx->d_abort, 0, sizeof(int32_t), st));
        return mpm_fail(ctx, MPM_ERR_TIMEOUT, "solve: a bounded inter-CTA wait expired");
    }
    if (bad_id) return mpm_fail(ctx, MPM_ERR_ARG, "solve: a cell id lies outside the rate tables");
    if (worst != MPM_OK) mpm_fail(ctx, worst, "solve: not every species converged");
    return worst;
}
