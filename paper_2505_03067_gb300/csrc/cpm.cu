// cpm.cu -- the growth driver coupled to the fields: tumour growth into the
// pleural space and mitosis on the device (the CPM and its Steppables of
// Sec. 2.1 / 2.4; the paper gives no Hamiltonian, so this is one simple
// rule, stated in the C header).
//
// Four launches per step, all stream-ordered, no host round trip:
//   k_cpm_grow     lattice -> scratch: every medium voxel in the mask next to
//                  a tumour cell is taken over with p = p_grow * c_O/(K_O+c_O)
//                  * c_n/(K_n+c_n) (0 below o2_min) by one of its tumour
//                  neighbours (synchronous: every voxel reads the old lattice);
//   k_cpm_stats    per-cell volume and coordinate sums (exact integer atomics,
//                  aggregated over the lanes of a warp that hold one id);
//   k_cpm_plan     one CTA: cells of at least v_div voxels get daughter ids in
//                  increasing id order while the rate tables have room, an
//                  axis each, and their parent's rates;
//   k_cpm_apply    scratch -> lattice: voxels strictly above the parent's
//                  centroid along its axis move to the daughter.
// Randomness: SplitMix64's output function on a counter (seed, step, stream,
// index), so the decisions do not depend on the launch shape.
#include <cmath>
#include <cstring>

#include "mpm_internal.cuh"

namespace mpm {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr int kPlanThreads = 1024;

__device__ __forceinline__ uint64_t splitmix_out(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t cpm_draw(uint64_t seed, int64_t step, int stream, uint64_t idx)
{
    const uint64_t c = ((uint64_t)((4 * step + stream) & ((1 << 24) - 1)) << 40) | idx;
    return splitmix_out(seed + (c + 1ull) * kGamma);
}

struct CpmArgs {
    int32_t *cell;               // lattice cell ids (in: before the step, out: after)
    int32_t *scratch;            // cell ids after growth
    const uint8_t *mask;
    const double *o2, *nut;
    int32_t Lx, Ly, Lz;
    int64_t L;
    double p_grow, K_o2, K_nut, o2_min;
    int32_t v_div;
    int32_t cap;                 // rate-table entries per species
    int32_t nspecies;
    double *k_cell, *q_cell;     // [nspecies][cap]
    int32_t *ncell;              // ids in use (device)
    unsigned long long *vol, *sum;   // [cap], [3][cap]
    int32_t *daughter, *axis;    // [cap + 1] (daughter[cap]: the ids in use before the step), [cap]
    unsigned long long *stats;   // grown, divisions, ids outside the tables
    uint64_t seed;
    int64_t step;
};

// Element loops of the growth and statistics kernels run warp-uniformly:
// every lane of a warp takes every iteration (lanes past the end idle), so
// full-warp collectives are legal inside.
__device__ __forceinline__ int64_t cpm_warp_base() { return (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); }

__global__ void __launch_bounds__(256) k_cpm_grow(const __grid_constant__ CpmArgs A)
{
    const uint32_t Lx = A.Lx, Ly = A.Ly, Lz = A.Lz;
    for (int64_t base = cpm_warp_base(); base < A.L; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = base + (threadIdx.x & 31);
        const bool inr = v < A.L;
        int32_t out = 0;
        bool grew = false;
        if (inr) {
            const int32_t id = A.cell[v];
            out = id;
            if (id == 0 && A.mask[v]) {
                const uint32_t x = (uint32_t)(v % Lx), y = (uint32_t)((v / Lx) % Ly), z = (uint32_t)(v / ((int64_t)Lx * Ly));
                int32_t nb[6];
                nb[0] = x > 0 ? A.cell[v - 1] : 0;
                nb[1] = x + 1 < Lx ? A.cell[v + 1] : 0;
                nb[2] = y > 0 ? A.cell[v - Lx] : 0;
                nb[3] = y + 1 < Ly ? A.cell[v + Lx] : 0;
                nb[4] = z > 0 ? A.cell[v - (int64_t)Lx * Ly] : 0;
                nb[5] = z + 1 < Lz ? A.cell[v + (int64_t)Lx * Ly] : 0;
                uint32_t k = 0;
#pragma unroll
                for (int d = 0; d < 6; ++d) k += nb[d] > 0 ? 1u : 0u;
                const double c0 = A.o2[v], c1 = A.nut[v];
                if (k > 0 && !(c0 < A.o2_min)) {
                    // same operations, same order as the rule's statement (no contraction possible)
                    const double p = A.p_grow * (c0 / (A.K_o2 + c0)) * (c1 / (A.K_nut + c1));
                    const double u = (double)(cpm_draw(A.seed, A.step, 0, (uint64_t)v) >> 11) * 0x1.0p-53;
                    if (u < p) {
                        const uint64_t h = cpm_draw(A.seed, A.step, 1, (uint64_t)v) >> 32;
                        const uint32_t j = (uint32_t)((h * k) >> 32);
                        uint32_t r = 0;
#pragma unroll
                        for (int d = 0; d < 6; ++d)
                            if (nb[d] > 0) {
                                if (r == j) out = nb[d];
                                ++r;
                            }
                        grew = true;
                    }
                }
            }
            A.scratch[v] = out;
        }
        const unsigned g = __ballot_sync(0xffffffffu, grew);
        if ((threadIdx.x & 31) == 0 && g) atomicAdd(A.stats + 0, (unsigned long long)__popc(g));
    }
}

__global__ void __launch_bounds__(256) k_cpm_stats(const __grid_constant__ CpmArgs A)
{
    const uint32_t Lx = A.Lx, Ly = A.Ly;
    for (int64_t base = cpm_warp_base(); base < A.L; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = base + (threadIdx.x & 31);
        const bool inr = v < A.L;
        const int32_t id = inr ? A.scratch[v] : 0;
        const bool bad = inr && (id < 0 || id >= A.cap);
        const bool ok = inr && id > 0 && id < A.cap;
        const unsigned okm = __ballot_sync(0xffffffffu, ok);
        const unsigned badm = __ballot_sync(0xffffffffu, bad);
        if ((threadIdx.x & 31) == 0 && badm) atomicAdd(A.stats + 2, (unsigned long long)__popc(badm));
        if (ok) {
            const uint32_t x = (uint32_t)(v % Lx), y = (uint32_t)((v / Lx) % Ly), z = (uint32_t)(v / ((int64_t)Lx * Ly));
            const unsigned peers = __match_any_sync(okm, id);
            const unsigned n = __popc(peers);
            const unsigned sx = __reduce_add_sync(peers, x), sy = __reduce_add_sync(peers, y),
                           sz = __reduce_add_sync(peers, z);
            if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) {
                atomicAdd(A.vol + id, (unsigned long long)n);
                atomicAdd(A.sum + id, (unsigned long long)sx);
                atomicAdd(A.sum + A.cap + id, (unsigned long long)sy);
                atomicAdd(A.sum + 2 * (int64_t)A.cap + id, (unsigned long long)sz);
            }
        }
    }
}

// One CTA: daughters in increasing parent id order while the tables have room.
__global__ void __launch_bounds__(kPlanThreads) k_cpm_plan(const __grid_constant__ CpmArgs A)
{
    __shared__ int32_t s_warp[kPlanThreads / 32];
    __shared__ int32_t s_next;
    const int nc0 = *A.ncell;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_next = nc0;
    __syncthreads();
    if (threadIdx.x == 0) A.daughter[A.cap] = nc0;      // the ids the apply pass may meet
    for (int c0 = 0; c0 < nc0 && c0 < A.cap; c0 += kPlanThreads) {
        const int id = c0 + threadIdx.x;
        const bool live = id >= 1 && id < nc0 && id < A.cap;
        const bool div = live && A.vol[id] >= (unsigned long long)A.v_div;
        const unsigned b = __ballot_sync(0xffffffffu, div);
        if (lane == 0) s_warp[wid] = __popc(b);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < kPlanThreads / 32; ++w) {
            if (w < wid) before += s_warp[w];
            total += s_warp[w];
        }
        const int rank = before + __popc(b & ((1u << lane) - 1u));
        const int next = s_next;
        if (id < A.cap && id < nc0) {
            int32_t d = -1, ax = 0;
            if (div && next + rank < A.cap) {
                d = next + rank;
                const uint64_t h = cpm_draw(A.seed, A.step, 2, (uint64_t)id) >> 32;
                ax = (int32_t)((h * 3ull) >> 32);
                for (int s = 0; s < A.nspecies; ++s) {
                    A.k_cell[(int64_t)s * A.cap + d] = A.k_cell[(int64_t)s * A.cap + id];
                    A.q_cell[(int64_t)s * A.cap + d] = A.q_cell[(int64_t)s * A.cap + id];
                }
            }
            A.daughter[id] = d;
            A.axis[id] = ax;
        }
        __syncthreads();
        if (threadIdx.x == 0) s_next = min(A.cap, next + total);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        A.stats[1] += (unsigned long long)(s_next - nc0);
        *A.ncell = s_next;
    }
}

__global__ void __launch_bounds__(256) k_cpm_apply(const __grid_constant__ CpmArgs A)
{
    const uint32_t Lx = A.Lx, Ly = A.Ly;
    const int32_t nc0 = A.daughter[A.cap];
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < A.L; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t id = A.scratch[v];
        int32_t out = id;
        if (id > 0 && id < nc0 && id < A.cap) {
            const int32_t d = A.daughter[id];
            if (d >= 0) {
                const int a = A.axis[id];
                const uint64_t c = a == 0 ? (uint64_t)(v % Lx) : a == 1 ? (uint64_t)((v / Lx) % Ly)
                                                                         : (uint64_t)(v / ((int64_t)Lx * Ly));
                if (c * A.vol[id] > A.sum[(int64_t)a * A.cap + id]) out = d;
            }
        }
        A.cell[v] = out;
    }
}

}  // namespace mpm

using namespace mpm;

extern "C" mpm_status mpm_cpm_step(mpm_ctx *ctx, const mpm_lattice *lat, const mpm_params *prm,
                                   const mpm_cpm_params *cp, uint64_t seed, int64_t step, int32_t *ncell_dev,
                                   int64_t *stats_dev, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    if (!lat || !prm || !cp || !ncell_dev || !stats_dev) return mpm_fail(ctx, MPM_ERR_ARG, "cpm_step: null argument");
    if (!lat->cell_id || !lat->mask || prm->nspecies < 2 || !lat->field[0] || !lat->field[1])
        return mpm_fail(ctx, MPM_ERR_ARG, "cpm_step: needs cell ids, the mask and species 0 (O2) and 1 (nutrient)");
    if (!prm->k_cell || !prm->q_cell || prm->ncell < 1 || prm->nspecies > MPM_MAX_SPECIES)
        return mpm_fail(ctx, MPM_ERR_ARG, "cpm_step: rate tables missing");
    const int64_t L = (int64_t)lat->dims[0] * lat->dims[1] * lat->dims[2];
    if (lat->dims[0] < 1 || lat->dims[1] < 1 || lat->dims[2] < 1 || L >= ((int64_t)1 << 31))
        return mpm_fail(ctx, MPM_ERR_ARG, "cpm_step: lattice dims out of range");
    if (!(cp->p_grow >= 0.0) || !(cp->K_o2 >= 0.0) || !(cp->K_nut >= 0.0) || !std::isfinite(cp->o2_min) ||
        cp->v_div < 2 || step < 0)
        return mpm_fail(ctx, MPM_ERR_ARG, "cpm_step: bad growth parameters");
    cudaStream_t st = (cudaStream_t)stream;
    const int cap = prm->ncell;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_scr = al((size_t)L * 4), b_vol = al((size_t)cap * 8), b_sum = al((size_t)cap * 24),
                 b_i = al((size_t)(cap + 1) * 4);
    mpm_status r = mpm_grow(ctx, (void **)&ctx->d_cpm, &ctx->cpm_cap, b_scr + b_vol + b_sum + 2 * b_i,
                            "growth driver scratch");
    if (r != MPM_OK) return r;
    char *p = (char *)ctx->d_cpm;
    CpmArgs A;
    memset(&A, 0, sizeof(A));
    A.cell = const_cast<int32_t *>(lat->cell_id);   // updated in place (documented)
    A.scratch = (int32_t *)p;
    A.vol = (unsigned long long *)(p + b_scr);
    A.sum = (unsigned long long *)(p + b_scr + b_vol);
    A.daughter = (int32_t *)(p + b_scr + b_vol + b_sum);
    A.axis = (int32_t *)(p + b_scr + b_vol + b_sum + b_i);
    A.mask = lat->mask;
    A.o2 = lat->field[0];
    A.nut = lat->field[1];
    A.Lx = lat->dims[0];
    A.Ly = lat->dims[1];
    A.Lz = lat->dims[2];
    A.L = L;
    A.p_grow = cp->p_grow;
    A.K_o2 = cp->K_o2;
    A.K_nut = cp->K_nut;
    A.o2_min = cp->o2_min;
    A.v_div = cp->v_div;
    A.cap = cap;
    A.nspecies = prm->nspecies;
    A.k_cell = const_cast<double *>(prm->k_cell);
    A.q_cell = const_cast<double *>(prm->q_cell);
    A.ncell = ncell_dev;
    A.stats = (unsigned long long *)stats_dev;
    A.seed = seed;
    A.step = step;
    MPM_CU(cudaMemsetAsync(A.vol, 0, b_vol + b_sum, st));
    const int grid = ctx->num_sms * 8;
    k_cpm_grow<<<grid, 256, 0, st>>>(A);
    k_cpm_stats<<<grid, 256, 0, st>>>(A);
    k_cpm_plan<<<1, kPlanThreads, 0, st>>>(A);
    k_cpm_apply<<<grid, 256, 0, st>>>(A);
    ctx->launches += 4;
    return mpm_cuda_check(ctx, cudaGetLastError(), "cpm_step");
}
