// mpm_internal.cuh -- shared declarations of the GB300 solver library.
//
// Data layout in HBM.  A box of dims n[3] is covered by tiles of TX x TY x TZ
// voxels (powers of two).  Only "active" tiles (holding at least one in-mask
// voxel) are stored, tile-major and compacted: element e of a box vector is
// voxel (e & (TV-1)) of active tile (e >> log2 TV), x fastest inside the tile.
// Every per-voxel array (flags, cell ids, iterate, rhs, diagonal, Krylov
// vectors) uses that one flat index, so all streaming passes are plain,
// perfectly coalesced 1D loops and only the 7-point stencil looks at tiles
// (through a 6-entry neighbour table per tile).  Inactive tiles have no
// unknowns (identity rows keeping c^n), so they are never stored or touched.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mpm.h"

namespace mpm {

// flags byte of an element
constexpr uint32_t F_MX = 1u, F_PX = 2u, F_MY = 4u, F_PY = 8u, F_MZ = 16u, F_PZ = 32u;
constexpr uint32_t F_OPEN = 63u;   // any open face
constexpr uint32_t F_MASK = 64u;   // voxel is in the pleural mask (an unknown)
constexpr uint32_t F_BOX = 128u;   // voxel lies inside the box (not tile padding)

constexpr int kBlock = 256;        // threads per CTA of every kernel
constexpr int kWarps = kBlock / 32;
constexpr int kProfSlots = 15;      // phase timer: [-, wait, reduce, serial, R, P1, P2, U, extract, scatter,
                                    //  extraction phases A..E]
constexpr int kMaxSpecies = MPM_MAX_SPECIES;
constexpr int kMaxM = MPM_MAX_RESTART;
constexpr int kKStride = kMaxM + 2;           // partial slots per species
constexpr int kKMax = kMaxSpecies * kKStride; // partial slots per block

// Box geometry of an extraction: box origin and dims in the lattice, tile
// counts and log2 tile dims, lattice row and plane strides.
struct BoxGeo {
    int32_t lo[3], n[3], nt[3];
    int32_t lt[3];
    uint32_t Lx, Ly;
};

// Box coordinates of element e; returns false for tile padding outside the box.
// kCoherent: the tile coordinates were written earlier in the same kernel
// (read through L2, not the read-only path).
template <bool kCoherent = false>
__device__ __forceinline__ bool elem_box(int64_t e, const BoxGeo &g, const int32_t *__restrict__ tile_coord,
                                         int &bx, int &by, int &bz)
{
    const int ltv = g.lt[0] + g.lt[1] + g.lt[2];
    const int64_t tile = e >> ltv;
    const uint32_t v = (uint32_t)(e & ((1 << ltv) - 1));
    const int4 *tcp = reinterpret_cast<const int4 *>(tile_coord) + tile;
    const int4 tc = kCoherent ? __ldcg(tcp) : __ldg(tcp);
    bx = (tc.x << g.lt[0]) + (int)(v & ((1u << g.lt[0]) - 1));
    by = (tc.y << g.lt[1]) + (int)((v >> g.lt[0]) & ((1u << g.lt[1]) - 1));
    bz = (tc.z << g.lt[2]) + (int)(v >> (g.lt[0] + g.lt[1]));
    return bx < g.n[0] && by < g.n[1] && bz < g.n[2];
}

BoxGeo make_geo(const ::mpm_subgrid *sub, const int32_t dims[3]);   // extract.cu

// Running min / max of the (x, y, z) of lattice index e (bounding box, Sec. 2.3).
__device__ __forceinline__ void bbox_upd(uint32_t e, uint32_t Lx, uint32_t Lxy, int (&mn)[3], int (&mx)[3])
{
    const uint32_t k = e / Lxy;
    const uint32_t r = e - k * Lxy;
    const uint32_t j = r / Lx;
    const uint32_t i = r - j * Lx;
    mn[0] = min(mn[0], (int)i); mx[0] = max(mx[0], (int)i);
    mn[1] = min(mn[1], (int)j); mx[1] = max(mx[1], (int)j);
    mn[2] = min(mn[2], (int)k); mx[2] = max(mx[2], (int)k);
}


// The FP32 value of x rounded toward zero, formed from its IEEE-754 bits with
// integer operations: the FP64-to-FP32 conversion instruction shares GB300's
// narrow FP64 pipe with the residual's arithmetic.  Magnitudes below the FP32
// normal range give a signed zero, above it infinity; NaN stays NaN.
__device__ __forceinline__ float f32_rz(double x)
{
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t sgn = hi & 0x80000000u, ex = (hi >> 20) & 0x7ffu;
    const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const int e = (int)ex - 896;   // FP32 biased exponent
    uint32_t bits;
    if (e <= 0) bits = sgn;
    else if (e >= 255) bits = sgn | 0x7f800000u | ((ex == 0x7ffu && ((hi & 0xfffffu) | lo)) ? 0x400000u : 0u);
    else bits = sgn | ((uint32_t)e << 23) | m;
    return __uint_as_float(bits);
}

// The FP64 value of an FP32 x (exact), formed from its IEEE-754 bits with
// integer operations, for the same reason; subnormal inputs give a signed zero.
__device__ __forceinline__ double f64_of(float x)
{
    const uint32_t b = __float_as_uint(x);
    const uint32_t sgn = b & 0x80000000u, ex = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    uint32_t hi, lo;
    if (ex == 0) { hi = sgn; lo = 0u; }
    else if (ex == 0xffu) { hi = sgn | 0x7ff00000u | (m >> 3); lo = m << 29; }
    else { hi = sgn | ((ex + 896u) << 20) | (m >> 3); lo = m << 29; }
    return __hiloint2double((int)hi, (int)lo);
}

// Box from the reduced bounds (Sec. 2.3): lo = max(0, min - margin),
// hi = min(L, max + margin + 1); tile counts of the box.  n[0] = 0 marks an
// empty tumour set.
__device__ __forceinline__ BoxGeo box_geo(const int32_t *__restrict__ mnmx, int32_t margin, int32_t Lx, int32_t Ly,
                                          int32_t Lz, int32_t lt0, int32_t lt1, int32_t lt2)
{
    BoxGeo g;
    const int32_t L[3] = {Lx, Ly, Lz};
    const int32_t lt[3] = {lt0, lt1, lt2};
    const bool empty = mnmx[3] < 0;
    for (int d = 0; d < 3; ++d) {
        const int32_t lo = max(0, mnmx[d] - margin);
        const int32_t hi = (int32_t)min((int64_t)L[d], (int64_t)mnmx[3 + d] + margin + 1);
        g.lo[d] = empty ? 0 : lo;
        g.n[d] = empty ? 0 : hi - lo;
        g.lt[d] = lt[d];
        g.nt[d] = empty ? 0 : (hi - lo + (1 << lt[d]) - 1) >> lt[d];
    }
    g.Lx = (uint32_t)Lx;
    g.Ly = (uint32_t)Ly;
    return g;
}


// Box and element count of a device-resident step, written by the tile scan
// and read by the later stages (the host does not know them yet).
struct StepDyn {
    int64_t NE;
    BoxGeo g;
};

// Coefficients of the implicit-Euler system (Eq. 1-4) shared by every row.
struct AsmCoef {
    int32_t nspecies, ncell, bc_box;
    double dt, a;                       // a = dt / h^2
    double D[kMaxSpecies], mu[kMaxSpecies], cbc[kMaxSpecies];
    const double *k_cell, *q_cell;      // [nspecies][ncell]
};

// Diagonal and right-hand side of the row of an in-mask voxel P, species s:
//   A_PP = 1 + dt (mu_s + k_cell[s][id]) + a (sum_open D_f + 2 D_P n_dir)
//   b_P  = c^n_P + dt q_cell[s][id] + a 2 D_P c_bc n_dir
// with D_f the harmonic mean of D_s fp and D_s dq(d) over the open faces d when
// the diffusivity varies (has_dfac), else D_s on every open face.  n_dir counts
// the faces of P on the box boundary (Dirichlet c_bc there).  dq(d) returns the
// diffusivity factor of the neighbour across face d.
template <typename DQ>
__device__ __forceinline__ void assemble_row(const AsmCoef &C, int s, uint32_t f, int id, int ndir, bool has_dfac,
                                             double fp, DQ dq, double cn, double &dg, double &b)
{
    const double kv = C.mu[s] + C.k_cell[(int64_t)s * C.ncell + id];
    if (has_dfac) {
        const double dp = C.D[s] * fp;
        double acc = 0.0;
        for (int d = 0; d < 6; ++d) {
            if (f & (1u << d)) {
                const double dn = C.D[s] * dq(d);
                acc += (dp + dn > 0.0) ? 2.0 * dp * dn / (dp + dn) : 0.0;
            }
        }
        dg = 1.0 + C.dt * kv + C.a * (acc + 2.0 * dp * ndir);
        b = cn + C.dt * C.q_cell[(int64_t)s * C.ncell + id] + C.a * 2.0 * dp * C.cbc[s] * ndir;
    } else {
        const double Ds = C.D[s];
        dg = 1.0 + C.dt * kv + C.a * Ds * (double)(__popc(f & F_OPEN) + 2 * ndir);
        b = cn + C.dt * C.q_cell[(int64_t)s * C.ncell + id] + C.a * 2.0 * Ds * C.cbc[s] * ndir;
    }
}

// Device view of one extracted, assembled box system.
struct SysDev {
    int64_t NE;                 // stored elements = nact * TV
    const int64_t *NEp;         // if set, the element count is read here on the device
    int32_t ltx, lty, ltz;      // log2 tile dims
    int32_t nspecies;
    const int32_t *nbr;         // [nact][6] neighbour tile (-1 none): -x,+x,-y,+y,-z,+z
    const uint8_t *flags;       // [NE]
    const double *dfac;         // [NE] or null (uniform D)
    double *x[kMaxSpecies];     // iterate (FP64)
    const double *b[kMaxSpecies];
    const double *diag[kMaxSpecies];
    const float *diag32[kMaxSpecies];
    void *V[kMaxSpecies];       // Krylov basis: (m+1) vectors of vstride elements
    int64_t vstride;
    double off[kMaxSpecies];    // dt*D_s/h^2 (uniform D: every open face)
    double a;                   // dt/h^2 (harmonic-mean path)
    double Dsp[kMaxSpecies];    // D_s (harmonic-mean path)
    const int32_t *err;         // set by the assembly when a cell id lies outside the tables
};

// Per-system result written by the solver kernel.
struct SysReport {
    int32_t iters[kMaxSpecies];
    int32_t cycles[kMaxSpecies];
    int32_t status[kMaxSpecies];
    int32_t jsum[kMaxSpecies];
    double res[kMaxSpecies];
    double bnorm[kMaxSpecies];
    int32_t reorth[kMaxSpecies];
    unsigned long long t_ns;    // device time of the item (its team's CTA 0)
};

struct TeamDesc {
    int32_t first_block, nblocks, sys_begin, sys_end;
};

struct SolveArgs {
    const SysDev *sys;
    const int32_t *sys_order;   // systems of team t: sys_order[sys_begin..sys_end)
    const TeamDesc *teams;
    const int32_t *block_team;  // team of each block
    double *partials;           // [2][gridDim][kKMax]
    uint32_t *bar;              // one counter per team, 32 words apart
    int32_t *abort_flag;        // set on a timed-out wait; every block then leaves
    SysReport *reports;         // per system
    double rtol, atol, inner_rtol;
    int32_t m, maxit;
    uint64_t timeout_ns;
    int32_t skip_block;         // fault injection for tests: this block never arrives (-1 none)
    int32_t reorth;             // second Gram-Schmidt pass when ||w|| < 0.7 ||w_before||
    unsigned long long *prof;   // nullable: CTA 0 adds ns spent in [-, wait, reduce, serial, R, P1, P2, U]
};

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u32(uint32_t *p, uint32_t v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Team-wide barrier among `nblocks` co-resident CTAs sharing counter `bar`.
// Each arrival adds 1; the k-th barrier of a launch completes when the counter
// reaches k*nblocks (the counter is zeroed before the launch).  The wait is
// bounded by timeout_ns of wall time; on expiry (or when another block has
// already given up) the global abort flag is raised and false is returned.
__device__ __forceinline__ bool team_barrier(uint32_t *bar, uint32_t &epoch, uint32_t nblocks,
                                             int32_t *abort_flag, uint64_t timeout_ns)
{
    // The CTA barrier orders every thread's earlier writes (the partials)
    // before thread 0's release; the acquire load orders the other CTAs'
    // writes before the barrier that releases this CTA's threads.  The abort
    // flag and the clock are checked every 16 polls.
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        epoch += 1;
        const uint32_t target = epoch * nblocks;
        red_release_add_u32(bar, 1u);
        int ok = 1;
        const uint64_t t0 = globaltimer_ns();
        uint32_t spins = 0;
        for (;;) {
            const uint32_t v = ld_acquire_u32(bar);
            if ((int32_t)(v - target) >= 0) break;
            if ((++spins & 15u) == 0) {
                if (*(volatile int32_t *)abort_flag) { ok = 0; break; }
                if (globaltimer_ns() - t0 > timeout_ns) {
                    atomicExch(abort_flag, 1);
                    ok = 0;
                    break;
                }
            }
            __nanosleep(32);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Neighbour element of e across face `dir` (0..5 = -x,+x,-y,+y,-z,+z) in the
// compact tile-major layout.  Valid only where that face is open (the
// neighbour then lies in an active tile by construction).
struct TileGeo {
    int32_t ltx, lty, ltz;
    __device__ __forceinline__ int32_t ltv() const { return ltx + lty + ltz; }
};

template <typename T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

// Sum over open faces of u at the neighbour (uniform diffusivity), reading
// through L2 (neighbours may belong to another CTA).
template <typename T>
__device__ __forceinline__ T nbr_sum(const T *__restrict__ u, const int32_t *__restrict__ nbr, int64_t e,
                                     uint32_t f, int ltx, int lty, int ltz)
{
    T s = T(0);
    if (!(f & F_OPEN)) return s;
    const int ltv = ltx + lty + ltz;
    const int64_t tile = e >> ltv;
    const uint32_t v = (uint32_t)(e & ((1 << ltv) - 1));
    const uint32_t TX = 1u << ltx, TY = 1u << lty, TZ = 1u << ltz;
    const uint32_t ix = v & (TX - 1), iy = (v >> ltx) & (TY - 1), iz = v >> (ltx + lty);
    const int64_t base = tile << ltv;
    if (f & F_MX) {
        const int64_t q = ix > 0 ? e - 1 : ((int64_t)__ldg(nbr + tile * 6 + 0) << ltv) + (v + TX - 1);
        s += ldcg(u + q);
    }
    if (f & F_PX) {
        const int64_t q = ix < TX - 1 ? e + 1 : ((int64_t)__ldg(nbr + tile * 6 + 1) << ltv) + (v - (TX - 1));
        s += ldcg(u + q);
    }
    if (f & F_MY) {
        const int64_t q = iy > 0 ? e - TX : ((int64_t)__ldg(nbr + tile * 6 + 2) << ltv) + (v + (TY - 1) * TX);
        s += ldcg(u + q);
    }
    if (f & F_PY) {
        const int64_t q = iy < TY - 1 ? e + TX : ((int64_t)__ldg(nbr + tile * 6 + 3) << ltv) + (v - (TY - 1) * TX);
        s += ldcg(u + q);
    }
    if (f & F_MZ) {
        const int64_t q = iz > 0 ? e - TX * TY
                                 : ((int64_t)__ldg(nbr + tile * 6 + 4) << ltv) + (v + (TZ - 1) * TX * TY);
        s += ldcg(u + q);
    }
    if (f & F_PZ) {
        const int64_t q = iz < TZ - 1 ? e + TX * TY
                                      : ((int64_t)__ldg(nbr + tile * 6 + 5) << ltv) + (v - (TZ - 1) * TX * TY);
        s += ldcg(u + q);
    }
    (void)base;
    return s;
}

// Harmonic-mean variant: sum over open faces of D_f u_Q with
// D_f = 2 D_P D_Q / (D_P + D_Q), D_P = Ds * dfac[P] (the caller multiplies by
// dt / h^2).
template <typename T>
__device__ __forceinline__ T nbr_sum_var(const T *__restrict__ u, const double *__restrict__ dfac,
                                         const int32_t *__restrict__ nbr, int64_t e, uint32_t f, int ltx,
                                         int lty, int ltz, double Ds)
{
    const double dp = Ds * __ldg(dfac + e);
    T s = T(0);
    if (!(f & F_OPEN)) return s;
    const int ltv = ltx + lty + ltz;
    const int64_t tile = e >> ltv;
    const uint32_t v = (uint32_t)(e & ((1 << ltv) - 1));
    const uint32_t TX = 1u << ltx, TY = 1u << lty, TZ = 1u << ltz;
    const uint32_t ix = v & (TX - 1), iy = (v >> ltx) & (TY - 1), iz = v >> (ltx + lty);
    int64_t q[6];
    q[0] = ix > 0 ? e - 1 : ((int64_t)__ldg(nbr + tile * 6 + 0) << ltv) + (v + TX - 1);
    q[1] = ix < TX - 1 ? e + 1 : ((int64_t)__ldg(nbr + tile * 6 + 1) << ltv) + (v - (TX - 1));
    q[2] = iy > 0 ? e - TX : ((int64_t)__ldg(nbr + tile * 6 + 2) << ltv) + (v + (TY - 1) * TX);
    q[3] = iy < TY - 1 ? e + TX : ((int64_t)__ldg(nbr + tile * 6 + 3) << ltv) + (v - (TY - 1) * TX);
    q[4] = iz > 0 ? e - TX * TY : ((int64_t)__ldg(nbr + tile * 6 + 4) << ltv) + (v + (TZ - 1) * TX * TY);
    q[5] = iz < TZ - 1 ? e + TX * TY : ((int64_t)__ldg(nbr + tile * 6 + 5) << ltv) + (v - (TZ - 1) * TX * TY);
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        if (f & (1u << d)) {
            const double dq = Ds * __ldg(dfac + q[d]);
            const double hm = (dp + dq > 0.0) ? 2.0 * dp * dq / (dp + dq) : 0.0;
            s += T(hm) * ldcg(u + q[d]);
        }
    }
    return s;
}

}  // namespace mpm

// ------------------------------------------------------------------ host-side objects
struct mpm_ctx {
    int device = 0;
    int num_sms = 0;
    size_t cap = 0;              // workspace cap (0 = none)
    size_t allocated = 0;
    std::string err;
    // scratch
    int32_t *d_box = nullptr;    // bbox result: lo[3] (min), hi[3] (max)
    int64_t *d_count = nullptr;  // mask-voxel count, nact
    int32_t *d_err = nullptr;    // device-side error flags
    double *d_partials = nullptr;
    size_t partials_cap = 0;     // doubles
    uint32_t *d_bar = nullptr;   // barrier counters
    int32_t bar_cap = 0;         // teams
    int32_t *d_abort = nullptr;
    void *d_args = nullptr;      // SysDev[], TeamDesc[], orders, block_team, reports
    size_t args_cap = 0;
    void *h_stage = nullptr;     // pinned staging for descriptors and reports
    size_t stage_cap = 0;
    double *d_tmp = nullptr;     // element scratch for apply_operator
    double *d_fg = nullptr;      // flexible GMRES workspace
    size_t fg_cap = 0;
    size_t tmp_cap = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int64_t launches = 0;        // kernels launched by this context
    int32_t phase_prof = 0;      // record the solver's phase times (test/tuning hook)
    int32_t cnn_layer_prof = 0;  // record CUDA events around the network's convolutions (test hook)
    int32_t solver_variant = 0;  // solver kernel variant (tuning)
    void *batch_graph = nullptr; // captured batched step (solver.cu)
    cudaStream_t cap_stream = nullptr;  // stream used only for graph capture
    cudaStream_t fg_cs[3] = {};  // capture streams of the flexible GMRES graph (fgmres.cu)
    void *fg_cache = nullptr;    // its last graph
    void *d_cpm = nullptr;       // growth driver scratch (cpm.cu)
    size_t cpm_cap = 0;
    void *d_tune = nullptr;      // tuner scratch tables
    size_t tune_cap = 0;
    unsigned long long *d_prof = nullptr;
    unsigned long long h_prof[16] = {};   // phase timer slots (kProfSlots used)
    double last_imbalance = 0.0; // t_max / <t> - 1 over the teams of the last solve
    // team planning of the batched solve (solver.cu); the model is measured
    // by mpm_tune_teams (tune.cu)
    double team_fixed = 3000.0;         // per-pass fixed cost of an item on a team of several CTAs
    double team_fixed1 = 3000.0;        //   and on a one-CTA team (no grid barrier), element-equivalents
    int32_t team_use_iters = 0;         // 1: weight items by item_iters; 2: plan from the measured item times
    double team_beta = 0.0;             // fitted device time per stored element and Arnoldi step (ns)
    uint64_t team_gen = 0;              // bumped when the model changes (captured plans are redone)
    std::vector<double> item_iters;     // per work item of the last solve: Arnoldi steps
    std::vector<double> item_ne;        //   stored elements
    std::vector<double> item_cta;       //   CTAs of its team
    std::vector<double> item_ns;        //   device time (its team's CTA 0)
    std::vector<double> team_ns;        // per team of the last solve: device time
    int64_t step_nfull = 0;      // mpm_step: full extractions so far (MPM_COUNTER_STEP_FULL_EXTRACTIONS)
    // test hooks
    uint64_t timeout_ns = 2000000000ull;
    int32_t skip_block = -1;
};

struct mpm_subgrid {
    bool extracted = false, assembled = false;
    uint64_t gen = 0;                // bumped by every extraction (buffers may move)
    int32_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, n[3] = {0, 0, 0};
    int32_t lt[3] = {2, 2, 2};
    int32_t nt[3] = {0, 0, 0};
    int32_t ldims[3] = {0, 0, 0};    // lattice dims of the extraction
    int32_t ntiles = 0, nact = 0;
    int64_t NE = 0, mask_voxels = 0;
    int64_t NE_cap = 0;              // element capacity of the buffers (device-resident step)
    void *step = nullptr;            // device-resident step state (solver.cu)
    int32_t nspecies = 0;
    bool has_dfac = false;
    bool x_fresh = true;         // iterate still equals c^n
    // geometry buffers (sized by tiles)
    void *geo = nullptr;
    size_t geo_bytes = 0;
    int32_t *tile_index = nullptr;   // [ntiles] compact index or -1
    int32_t *tile_coord = nullptr;   // [nact][4] tile coords (x, y, z, pad)
    int32_t *nbr = nullptr;          // [nact][6]
    int8_t *active = nullptr;        // [ntiles]
    int32_t *err = nullptr;          // assembly error flag (cell id outside the tables)
    // element buffers
    void *elem = nullptr;
    size_t elem_bytes = 0;
    uint8_t *flags = nullptr;
    int32_t *cell = nullptr;
    double *dfac = nullptr;
    double *x[MPM_MAX_SPECIES] = {};
    double *cn[MPM_MAX_SPECIES] = {};
    double *b[MPM_MAX_SPECIES] = {};
    double *diag[MPM_MAX_SPECIES] = {};
    float *diag32[MPM_MAX_SPECIES] = {};
    // Krylov basis
    void *krylov = nullptr;
    size_t krylov_bytes = 0;
    // assembled scalars
    double off[MPM_MAX_SPECIES] = {};
    double a = 0.0;
    double Dsp[MPM_MAX_SPECIES] = {};
};

// ------------------------------------------------------------------ host helpers (api.cu)
mpm_status mpm_fail(mpm_ctx *ctx, mpm_status st, const std::string &msg);
mpm_status mpm_cuda_check(mpm_ctx *ctx, cudaError_t e, const char *what);
mpm_status mpm_grow(mpm_ctx *ctx, void **p, size_t *cap, size_t need, const char *what);

#define MPM_CU(call)                                                       \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return mpm_cuda_check(ctx, e_, #call);      \
    } while (0)

// kernels' host launchers (extract.cu, assemble.cu, solver.cu)
mpm_status mpm_extract_impl(mpm_ctx *ctx, const mpm_lattice *lat, int32_t nspecies, int32_t margin,
                            const int32_t tile[3], mpm_box *out_box, mpm_subgrid *sub, cudaStream_t st);
mpm_status mpm_assemble_impl(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_params *prm, cudaStream_t st);
mpm_status mpm_assemble_check(mpm_ctx *ctx, const mpm_subgrid *sub, const mpm_params *p);
mpm_status mpm_params_check(mpm_ctx *ctx, const mpm_params *p);
mpm_status mpm_lattice_check(mpm_ctx *ctx, const mpm_lattice *lat, int32_t nspecies);
mpm_status mpm_tile_lt(mpm_ctx *ctx, const int32_t tile[3], int32_t lt[3]);
void mpm_asm_coef(const mpm_params *p, mpm::AsmCoef *C);
void mpm_set_assembled_scalars(mpm_subgrid *sub, const mpm_params *p);
mpm_status mpm_scatter_impl(mpm_ctx *ctx, const mpm_subgrid *sub, const mpm_lattice *lat, cudaStream_t st);
mpm_status mpm_refresh_impl(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_lattice *lat, cudaStream_t st);
// batched forms of refresh + assemble and of scatter (batch.cu): one launch for
// all systems; the descriptors live in device memory the caller owns
size_t mpm_batch_desc_bytes(int32_t nsys);
mpm_status mpm_batch_prep_check(mpm_ctx *ctx, mpm_subgrid *const *subs, const mpm_lattice *const *lats,
                                const mpm_params *const *prms, int32_t nsys);
mpm_status mpm_batch_desc_fill(mpm_subgrid *const *subs, const mpm_lattice *const *lats,
                               const mpm_params *const *prms, int32_t nsys, void *host, int64_t *nblocks);
mpm_status mpm_batch_prep_launch(mpm_ctx *ctx, const void *d_desc, int32_t nsys, int64_t nblocks, cudaStream_t st);
mpm_status mpm_batch_scatter_launch(mpm_ctx *ctx, const void *d_desc, int32_t nsys, int64_t nblocks, cudaStream_t st);
// extraction with buffers sized for the whole lattice and no host round trip (extract.cu)
mpm_status mpm_step_buffers(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_lattice *lat, int32_t nspecies, const int32_t lt[3]);

mpm_status mpm_count_active_impl(mpm_ctx *ctx, const mpm_lattice *lat, int32_t margin, const int32_t lt[3],
                                 int64_t *nact, int64_t *mask_voxels, cudaStream_t st);
mpm_status mpm_export_impl(mpm_ctx *ctx, const mpm_subgrid *sub, int32_t what, int32_t s, void *dst,
                           cudaStream_t st);
mpm_status mpm_import_impl(mpm_ctx *ctx, mpm_subgrid *sub, int32_t s, const double *src, cudaStream_t st);
mpm_status mpm_apply_impl(mpm_ctx *ctx, const mpm_subgrid *sub, int32_t s, const double *x, double *y,
                          cudaStream_t st);
mpm_status mpm_solve_impl(mpm_ctx *ctx, mpm_subgrid *const *subs, const mpm_lattice *const *scatter_to,
                          int32_t nsys, const mpm_opts *opt, mpm_report *reps, cudaStream_t st);
mpm_status mpm_batch_step_impl(mpm_ctx *ctx, mpm_subgrid *const *subs, const mpm_lattice *const *lats,
                               const mpm_params *const *prms, int32_t nsys, const mpm_opts *opt, mpm_report *reps,
                               cudaStream_t st);
void mpm_batch_graph_free(mpm_ctx *ctx);
void mpm_fgmres_release(mpm_ctx *ctx);   // fgmres.cu: its graph and capture streams
mpm_status mpm_step_impl(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_lattice *lat, const mpm_params *prm, int32_t margin,
                         const int32_t tile[3], const mpm_opts *opt, mpm_report *rep, mpm_box *out_box, cudaStream_t st);
mpm_status mpm_step_enqueue_impl(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_lattice *lat, const mpm_params *prm,
                                 int32_t margin, const int32_t tile[3], const mpm_opts *opt, cudaStream_t st);
mpm_status mpm_step_wait_impl(mpm_ctx *ctx, mpm_subgrid *sub, mpm_report *rep, mpm_box *out_box, cudaStream_t st);
mpm_status mpm_step_set_network_impl(mpm_ctx *ctx, mpm_subgrid *sub, mpm_cnn *cnn);
mpm_status mpm_solve_fgmres_impl(mpm_ctx *ctx, mpm_cnn *cnn, mpm_subgrid *sub, const mpm_lattice *lat,
                                 const mpm_params *prm, const mpm_lattice *scatter_to, const mpm_opts *opt,
                                 mpm_report *rep, cudaStream_t st);
void mpm_step_free(mpm_ctx *ctx, mpm_subgrid *sub);
void mpm_step_invalidate(mpm_subgrid *sub);
int mpm_batch_graph_active(mpm_ctx *ctx);
