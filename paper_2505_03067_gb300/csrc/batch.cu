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
#include <cstring>

#include "mpm_internal.cuh"

namespace mpm {

constexpr int kEPT = 4;   // elements per thread

struct BatchSys {
    BoxGeo g;
    int64_t NE;
    const int32_t *tile_coord;
    const int32_t *cell_id;     // lattice
    const uint8_t *mask;        // lattice
    const double *dfac_lat;     // lattice, or null
    double *field[kMaxSpecies]; // lattice fields (read by the preparation, written by the scatter)
    uint8_t *flags;
    int32_t *cell;
    double *dfac;
    double *x[kMaxSpecies], *cn[kMaxSpecies], *b[kMaxSpecies], *diag[kMaxSpecies];
    float *diag32[kMaxSpecies];
    int32_t *err;
    AsmCoef C;
};

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
    const int ns = S.C.nspecies;
    const int64_t e0 = (blockIdx.x - blk0[i]) * (int64_t)(kBlock * kEPT);
    const int64_t e1 = min(S.NE, e0 + (int64_t)(kBlock * kEPT));
    const BoxGeo g = S.g;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kBlock) {
        int bx, by, bz;
        if (!elem_box(e, g, S.tile_coord, bx, by, bz)) {   // tile padding
            S.flags[e] = 0;
            S.cell[e] = 0;
            if (S.dfac) S.dfac[e] = 1.0;
            for (int s = 0; s < ns; ++s) {
                S.x[s][e] = 0.0;
                S.cn[s][e] = 0.0;
                S.diag[s][e] = 1.0;
                S.diag32[s][e] = 1.0f;
                S.b[s][e] = 0.0;
            }
            continue;
        }
        const int64_t sy = g.Lx, sz = (int64_t)g.Lx * g.Ly;
        const int64_t L = (int64_t)(g.lo[0] + bx) + sy * (g.lo[1] + by) + sz * (g.lo[2] + bz);
        uint32_t f = F_BOX;
        if (__ldg(S.mask + L)) {
            f |= F_MASK;
            if (bx > 0 && __ldg(S.mask + L - 1)) f |= F_MX;
            if (bx < g.n[0] - 1 && __ldg(S.mask + L + 1)) f |= F_PX;
            if (by > 0 && __ldg(S.mask + L - sy)) f |= F_MY;
            if (by < g.n[1] - 1 && __ldg(S.mask + L + sy)) f |= F_PY;
            if (bz > 0 && __ldg(S.mask + L - sz)) f |= F_MZ;
            if (bz < g.n[2] - 1 && __ldg(S.mask + L + sz)) f |= F_PZ;
        }
        S.flags[e] = (uint8_t)f;
        int32_t id = __ldg(S.cell_id + L);
        S.cell[e] = id;
        const double fp = S.dfac_lat ? __ldg(S.dfac_lat + L) : 1.0;
        if (S.dfac) S.dfac[e] = fp;
        if (!(f & F_MASK)) {                        // identity row keeping c^n
            for (int s = 0; s < ns; ++s) {
                const double c = __ldg(S.field[s] + L);
                S.x[s][e] = c;
                S.cn[s][e] = c;
                S.diag[s][e] = 1.0;
                S.diag32[s][e] = 1.0f;
                S.b[s][e] = c;
            }
            continue;
        }
        if (id < 0 || id >= S.C.ncell) {
            atomicOr(S.err, 1);
            id = 0;
        }
        const int ndir = S.C.bc_box == 0 ? (bx == 0) + (bx == g.n[0] - 1) + (by == 0) + (by == g.n[1] - 1) +
                                               (bz == 0) + (bz == g.n[2] - 1)
                                         : 0;
        auto dq = [&](int d) -> double {
            const int64_t o = d == 0 ? -1 : d == 1 ? 1 : d == 2 ? -sy : d == 3 ? sy : d == 4 ? -sz : sz;
            return __ldg(S.dfac_lat + L + o);
        };
        for (int s = 0; s < ns; ++s) {
            const double c = __ldg(S.field[s] + L);
            double dg, bb;
            assemble_row(S.C, s, f, id, ndir, S.dfac != nullptr, fp, dq, c, dg, bb);
            S.x[s][e] = c;
            S.cn[s][e] = c;
            S.diag[s][e] = dg;
            S.diag32[s][e] = (float)dg;
            S.b[s][e] = bb;
        }
    }
}

// Sec. 2.4: the box solution onto the pleural mask (in-mask voxels only).
__global__ void __launch_bounds__(kBlock) k_batch_scatter(const char *__restrict__ buf, int nsys)
{
    const int64_t *blk0 = reinterpret_cast<const int64_t *>(buf);
    const int i = find_sys(blk0, nsys, blockIdx.x);
    const BatchSys &S = reinterpret_cast<const BatchSys *>(buf + desc_off(nsys))[i];
    const int64_t e0 = (blockIdx.x - blk0[i]) * (int64_t)(kBlock * kEPT);
    const int64_t e1 = min(S.NE, e0 + (int64_t)(kBlock * kEPT));
    const BoxGeo g = S.g;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kBlock) {
        if (!(S.flags[e] & F_MASK)) continue;
        int bx, by, bz;
        elem_box(e, g, S.tile_coord, bx, by, bz);
        const int64_t L = (int64_t)(g.lo[0] + bx) + (int64_t)g.Lx * ((g.lo[1] + by) + (int64_t)g.Ly * (g.lo[2] + bz));
        for (int s = 0; s < S.C.nspecies; ++s) S.field[s][L] = S.x[s][e];
    }
}

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
