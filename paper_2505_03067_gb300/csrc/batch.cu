// batch.cu -- the per-step preparation (Sec. 2.4: copy c^n, the mask and the
// cell ids into the box, then assemble Eq. 1-4) and the scatter of the
// solution back onto the pleural mask, for many systems in one launch each.
//
// A batched step of many small boxes is otherwise a long chain of tiny
// launches (gather, assemble and scatter per system) whose fixed costs add up
// to more than the solve.  Here every system owns a contiguous range of CTAs;
// a CTA finds its system by binary search over the ranges' first CTAs and
// streams kEPT x kBlock elements of it.  The fused preparation reads the
// lattice once per element and computes the rows from those values: the
// neighbours' diffusivity factors come straight from the lattice (an open
// face implies an in-mask, in-box neighbour), so no element waits for
// another.  The rows are those of the separate gather + assembly, bit for
// bit: both call assemble_row with the same values.
#include <algorithm>
#include <climits>
#include <cstring>

#include "mpm_internal.cuh"
#include "step_kernels.cuh"

namespace mpm {

constexpr int kEPT = 4;   // elements per thread

// Descriptor buffer: int64 first_block[nsys + 1], then BatchSys[nsys].
__host__ __device__ __forceinline__ size_t desc_off(int32_t nsys)
{
    return ((size_t)(nsys + 1) * sizeof(int64_t) + 255) & ~(size_t)255;
}

__device__ __forceinline__ int find_sys(const int64_t *__restrict__ blk0, int nsys, int64_t b)
{
    int lo = 0, hi = nsys - 1;   // largest i with blk0[i] <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(blk0 + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_batch_reset_err(const char *__restrict__ buf, int nsys)
{
    const BatchSys *D = reinterpret_cast<const BatchSys *>(buf + desc_off(nsys));
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsys; i += gridDim.x * blockDim.x) *D[i].err = 0;
}

__global__ void __launch_bounds__(kBlock) k_batch_prep(const char *__restrict__ buf, int nsys)
{
    const int64_t *blk0 = reinterpret_cast<const int64_t *>(buf);
    const int i = find_sys(blk0, nsys, blockIdx.x);
    const BatchSys &S = reinterpret_cast<const BatchSys *>(buf + desc_off(nsys))[i];
    const int64_t e0 = (blockIdx.x - blk0[i]) * (int64_t)(kBlock * kEPT);
    const int64_t e1 = min(S.NE, e0 + (int64_t)(kBlock * kEPT));
    const BoxGeo g = S.g;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kBlock) prep_elem<false>(S, g, e);
}

__global__ void __launch_bounds__(kBlock) k_batch_scatter(const char *__restrict__ buf, int nsys)
{
    const int64_t *blk0 = reinterpret_cast<const int64_t *>(buf);
    const int i = find_sys(blk0, nsys, blockIdx.x);
    const BatchSys &S = reinterpret_cast<const BatchSys *>(buf + desc_off(nsys))[i];
    const int64_t e0 = (blockIdx.x - blk0[i]) * (int64_t)(kBlock * kEPT);
    const int64_t e1 = min(S.NE, e0 + (int64_t)(kBlock * kEPT));
    const BoxGeo g = S.g;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kBlock) scatter_elem(S, g, e);
}

// ---------------------------------------------------------------- single system, device-sized
// The device-resident step: the static part of the descriptor (pointers,
// coefficients) is a kernel parameter, the box and element count come from
// the tile scan (StepDyn); the element kernels stride over whatever count
// they find there.  The preparation also builds the neighbour table (the
// first element of each tile), and the scatter's CTA 0 copies the step's
// results to host-mapped memory and resets the box and count slots for the
// next step (so the graph has no memset or copy nodes).
}  // namespace mpm

using namespace mpm;

size_t mpm_batch_desc_bytes(int32_t nsys) { return desc_off(nsys) + sizeof(BatchSys) * (size_t)nsys; }

// The checks of refresh and assembly, for every system of a batch.
mpm_status mpm_batch_prep_check(mpm_ctx *ctx, mpm_subgrid *const *subs, const mpm_lattice *const *lats,
                                const mpm_params *const *prms, int32_t nsys)
{
    for (int i = 0; i < nsys; ++i) {
        const mpm_subgrid *sub = subs[i];
        const mpm_lattice *lat = lats[i];
        if (!sub || !lat || !lat->cell_id || !lat->mask) return mpm_fail(ctx, MPM_ERR_ARG, "batch: null argument");
        if (!sub->extracted) return mpm_fail(ctx, MPM_ERR_ARG, "batch: subgrid not extracted");
        for (int d = 0; d < 3; ++d)
            if (lat->dims[d] != sub->ldims[d])
                return mpm_fail(ctx, MPM_ERR_ARG, "batch: lattice dims differ from the extraction");
        for (int s = 0; s < sub->nspecies; ++s)
            if (!lat->field[s]) return mpm_fail(ctx, MPM_ERR_ARG, "batch: null field pointer");
        if ((lat->dfac != nullptr) != sub->has_dfac)
            return mpm_fail(ctx, MPM_ERR_ARG, "batch: dfac presence differs from the extraction");
        mpm_status r = mpm_assemble_check(ctx, sub, prms[i]);
        if (r != MPM_OK) return r;
    }
    return MPM_OK;
}

// Host image of the descriptor buffer; also sets the subgrids' assembled
// scalars (the solver's descriptors read them).
mpm_status mpm_batch_desc_fill(mpm_subgrid *const *subs, const mpm_lattice *const *lats,
                               const mpm_params *const *prms, int32_t nsys, void *host, int64_t *nblocks)
{
    char *buf = (char *)host;
    memset(buf, 0, mpm_batch_desc_bytes(nsys));
    int64_t *blk0 = reinterpret_cast<int64_t *>(buf);
    BatchSys *D = reinterpret_cast<BatchSys *>(buf + desc_off(nsys));
    int64_t nb = 0;
    for (int i = 0; i < nsys; ++i) {
        mpm_subgrid *sub = subs[i];
        const mpm_lattice *lat = lats[i];
        BatchSys &S = D[i];
        blk0[i] = nb;
        nb += (sub->NE + kBlock * kEPT - 1) / (kBlock * kEPT);
        S.g = make_geo(sub, lat->dims);
        S.NE = sub->NE;
        S.tile_coord = sub->tile_coord;
        S.cell_id = lat->cell_id;
        S.mask = lat->mask;
        S.dfac_lat = lat->dfac;
        S.flags = sub->flags;
        S.cell = sub->cell;
        S.dfac = sub->dfac;
        for (int s = 0; s < sub->nspecies; ++s) {
            S.field[s] = lat->field[s];
            S.x[s] = sub->x[s];
            S.cn[s] = sub->cn[s];
            S.b[s] = sub->b[s];
            S.diag[s] = sub->diag[s];
            S.diag32[s] = sub->diag32[s];
        }
        S.err = sub->err;
        mpm_asm_coef(prms[i], &S.C);
        mpm_set_assembled_scalars(sub, prms[i]);
    }
    blk0[nsys] = nb;
    *nblocks = nb;
    return MPM_OK;
}

mpm_status mpm_batch_prep_launch(mpm_ctx *ctx, const void *d_desc, int32_t nsys, int64_t nblocks, cudaStream_t st)
{
    k_batch_reset_err<<<(nsys + kBlock - 1) / kBlock, kBlock, 0, st>>>((const char *)d_desc, nsys);
    ctx->launches += 1;
    if (nblocks > 0) {
        k_batch_prep<<<(unsigned)nblocks, kBlock, 0, st>>>((const char *)d_desc, nsys);
        ctx->launches += 1;
    }
    MPM_CU(cudaGetLastError());
    return MPM_OK;
}

mpm_status mpm_batch_scatter_launch(mpm_ctx *ctx, const void *d_desc, int32_t nsys, int64_t nblocks, cudaStream_t st)
{
    if (nblocks > 0) {
        k_batch_scatter<<<(unsigned)nblocks, kBlock, 0, st>>>((const char *)d_desc, nsys);
        ctx->launches += 1;
        MPM_CU(cudaGetLastError());
    }
    return MPM_OK;
}

