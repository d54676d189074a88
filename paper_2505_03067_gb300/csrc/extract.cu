// extract.cu -- Sec. 2.3 (dynamic bounding box) and the gather/scatter of the
// box sub-grid between the caller's lattice and the library's tile-major
// compact layout (Sec. 2.4: the result is mapped back onto the pleural mask).
#include <climits>
#include <cstring>

#include "mpm_internal.cuh"

namespace mpm {

// ---------------------------------------------------------------- bbox reduction
// Min and max (x, y, z) over voxels with cell_id > 0.  HBM-bound scan of the
// int32 lattice (4 B/voxel): 16-byte loads, four in flight per thread; the
// coordinate arithmetic only runs for tumour voxels.  Per-CTA reduction, then
// six atomics per CTA that found any tumour voxel.
__global__ void __launch_bounds__(kBlock) k_bbox(const int32_t *__restrict__ cell, uint32_t Lx, uint32_t Lxy,
                                                 uint32_t ntot, int vec4, int32_t *__restrict__ out)
{
    int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {-1, -1, -1};
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nth = gridDim.x * blockDim.x;
    uint32_t done = 0;
    if (vec4) {
        const int4 *c4 = reinterpret_cast<const int4 *>(cell);
        const uint32_t n4 = ntot / 4;
        uint32_t q = tid;
        for (; q + 3 * nth < n4; q += 4 * nth) {
            int4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = __ldcs(c4 + q + u * nth);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if ((v[u].x > 0) | (v[u].y > 0) | (v[u].z > 0) | (v[u].w > 0)) {
                    const uint32_t e = 4 * (q + u * nth);
                    if (v[u].x > 0) bbox_upd(e + 0, Lx, Lxy, mn, mx);
                    if (v[u].y > 0) bbox_upd(e + 1, Lx, Lxy, mn, mx);
                    if (v[u].z > 0) bbox_upd(e + 2, Lx, Lxy, mn, mx);
                    if (v[u].w > 0) bbox_upd(e + 3, Lx, Lxy, mn, mx);
                }
            }
        }
        for (; q < n4; q += nth) {
            const int4 v = __ldcs(c4 + q);
            const uint32_t e = 4 * q;
            if (v.x > 0) bbox_upd(e + 0, Lx, Lxy, mn, mx);
            if (v.y > 0) bbox_upd(e + 1, Lx, Lxy, mn, mx);
            if (v.z > 0) bbox_upd(e + 2, Lx, Lxy, mn, mx);
            if (v.w > 0) bbox_upd(e + 3, Lx, Lxy, mn, mx);
        }
        done = n4 * 4;
    }
    for (uint32_t e = done + tid; e < ntot; e += nth)
        if (__ldcs(cell + e) > 0) bbox_upd(e, Lx, Lxy, mn, mx);

    __shared__ int smn[3][kWarps], smx[3][kWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int a = __reduce_min_sync(0xffffffffu, mn[d]);
        const int b = __reduce_max_sync(0xffffffffu, mx[d]);
        if (lane == 0) { smn[d][w] = a; smx[d][w] = b; }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int d = threadIdx.x;
        int a = INT_MAX, b = -1;
        for (int i = 0; i < kWarps; ++i) { a = min(a, smn[d][i]); b = max(b, smx[d][i]); }
        if (b >= 0) { atomicMin(out + d, a); atomicMax(out + 3 + d, b); }
    }
}

// ---------------------------------------------------------------- tiles
// Mark tiles holding an in-mask voxel; count the in-mask voxels of the box.
// One warp per box row (j, k).
__device__ __forceinline__ void tile_active_rows(const uint8_t *__restrict__ mask, const BoxGeo &g,
                                                 int8_t *__restrict__ active, unsigned long long *__restrict__ count)
{
    if (g.n[0] <= 0) return;                  // empty tumour set: no box
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t nwarp = (int64_t)gridDim.x * kWarps;
    const int64_t nrows = (int64_t)g.n[1] * g.n[2];
    unsigned long long cnt = 0;
    for (int64_t row = warp; row < nrows; row += nwarp) {
        const int by = (int)(row % g.n[1]), bz = (int)(row / g.n[1]);
        const int64_t L0 = (int64_t)g.lo[0] + (int64_t)g.Lx * ((int64_t)(g.lo[1] + by) + (int64_t)g.Ly * (g.lo[2] + bz));
        const int64_t trow = ((int64_t)(bz >> g.lt[2]) * g.nt[1] + (by >> g.lt[1])) * g.nt[0];
        for (int bx = lane; bx < g.n[0]; bx += 32) {
            if (__ldg(mask + L0 + bx)) {
                ++cnt;
                active[trow + (bx >> g.lt[0])] = 1;
            }
        }
    }
    cnt = __reduce_add_sync(0xffffffffu, (unsigned)cnt);
    if (lane == 0 && cnt) atomicAdd(count, cnt);
}

__global__ void __launch_bounds__(kBlock) k_tile_active(const uint8_t *__restrict__ mask, const BoxGeo *__restrict__ gp,
                                                        int8_t *__restrict__ active,
                                                        unsigned long long *__restrict__ count)
{
    const BoxGeo g = *gp;
    tile_active_rows(mask, g, active, count);
}

__global__ void k_box_finalize(const int32_t *__restrict__ mnmx, int32_t margin, int32_t Lx, int32_t Ly, int32_t Lz,
                               int32_t lt0, int32_t lt1, int32_t lt2, BoxGeo *__restrict__ g)
{
    if (threadIdx.x != 0) return;
    *g = box_geo(mnmx, margin, Lx, Ly, Lz, lt0, lt1, lt2);
}

// Exclusive scan of the tile activity by one CTA of 1024 threads, 8192 tiles
// per round: every lane reads the activity bytes of 8 tiles as one 8-byte
// word (bytes are 0 or 1; the next round's word is loaded before this one is
// used), warps scan their lanes' counts with shuffles, warp 0 scans the warp
// totals.  Writes the compact index of each tile (-1 if inactive) and the
// coordinates of each active tile in box-tile order; clear: zero the
// activity bytes after use.  Returns the active count (every thread).
__device__ __forceinline__ int32_t tile_scan_body(int8_t *__restrict__ active, const BoxGeo &g,
                                                  int32_t *__restrict__ tile_index, int32_t *__restrict__ tile_coord,
                                                  bool clear)
{
    __shared__ int32_t wsum[32];
    __shared__ int32_t carry;
    const int32_t ntiles = g.n[0] > 0 ? g.nt[0] * g.nt[1] * g.nt[2] : 0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    unsigned long long *aw = reinterpret_cast<unsigned long long *>(active);
    const int32_t nxy = g.nt[0] * g.nt[1];
    unsigned long long wn = 8 * tid < ntiles ? aw[tid] : 0ull;
    for (int32_t base = 0; base < ntiles; base += 8192) {
        const int32_t i0 = base + 8 * tid;
        unsigned long long w = wn;
        const int32_t in = i0 + 8192;
        wn = in < ntiles ? aw[in >> 3] : 0ull;
        if (i0 + 8 > ntiles) w &= i0 >= ntiles ? 0ull : (~0ull >> (8 * (i0 + 8 - ntiles)));
        const int32_t c = __popcll(w & 0x0101010101010101ull);
        int32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int32_t t = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t v = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += v;
            }
            wsum[lane] = t;   // inclusive
        }
        __syncthreads();
        int32_t idx = carry + (warp > 0 ? wsum[warp - 1] : 0) + incl - c;
        if (i0 < ntiles) {
            int32_t tx = i0 % g.nt[0], ty = (i0 / g.nt[0]) % g.nt[1], tz = i0 / nxy;
            for (int k = 0; k < 8; ++k) {
                const int32_t i = i0 + k;
                if (i >= ntiles) break;
                if ((w >> (8 * k)) & 1ull) {
                    tile_index[i] = idx;
                    reinterpret_cast<int4 *>(tile_coord)[idx] = make_int4(tx, ty, tz, 0);
                    ++idx;
                } else {
                    tile_index[i] = -1;
                }
                if (++tx == g.nt[0]) {
                    tx = 0;
                    if (++ty == g.nt[1]) { ty = 0; ++tz; }
                }
            }
            if (clear) aw[i0 >> 3] = 0ull;
        }
        __syncthreads();
        if (tid == 0) carry += wsum[31];
        __syncthreads();
    }
    return carry;
}

__global__ void __launch_bounds__(1024) k_tile_scan(int8_t *__restrict__ active, const BoxGeo *__restrict__ gp,
                                                    int32_t *__restrict__ tile_index,
                                                    int32_t *__restrict__ tile_coord,
                                                    unsigned long long *__restrict__ nact_out)
{
    const BoxGeo g = *gp;
    const int32_t n = tile_scan_body(active, g, tile_index, tile_coord, false);
    if (threadIdx.x == 0) *nact_out = (unsigned long long)n;
}

// Neighbour table of the active tiles; the box and the active count come from
// the device (grid-stride, so any grid covers them).
__global__ void k_tile_nbr(const int32_t *__restrict__ tile_index, const int32_t *__restrict__ tile_coord,
                           const unsigned long long *__restrict__ nactp, const BoxGeo *__restrict__ gp,
                           int32_t *__restrict__ nbr)
{
    const BoxGeo g = *gp;
    const int64_t nact = g.n[0] > 0 ? (int64_t)*nactp : 0;
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nact; a += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c[3] = {tile_coord[4 * a], tile_coord[4 * a + 1], tile_coord[4 * a + 2]};
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            int32_t q[3] = {c[0], c[1], c[2]};
            q[d >> 1] += (d & 1) ? 1 : -1;
            int32_t r = -1;
            if (q[0] >= 0 && q[0] < g.nt[0] && q[1] >= 0 && q[1] < g.nt[1] && q[2] >= 0 && q[2] < g.nt[2])
                r = tile_index[(q[2] * g.nt[1] + q[1]) * g.nt[0] + q[0]];
            nbr[6 * a + d] = r;
        }
    }
}

struct GatherArgs {
    const int32_t *cell_id;
    const uint8_t *mask;
    const double *dfac_lat;
    const double *field[kMaxSpecies];
    int32_t nspecies;
    uint8_t *flags;
    int32_t *cell;
    double *dfac;
    double *x[kMaxSpecies];
    double *cn[kMaxSpecies];
};

// Copy mask-derived face flags, cell ids, dfac and c^n of every stored element.
__global__ void __launch_bounds__(kBlock) k_gather(GatherArgs a, BoxGeo g, const int32_t *__restrict__ tile_coord,
                                                   int64_t NE)
{
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < NE; e += (int64_t)gridDim.x * kBlock) {
        int bx, by, bz;
        if (!elem_box(e, g, tile_coord, bx, by, bz)) {
            a.flags[e] = 0;
            a.cell[e] = 0;
            if (a.dfac) a.dfac[e] = 1.0;
            for (int s = 0; s < a.nspecies; ++s) { a.x[s][e] = 0.0; a.cn[s][e] = 0.0; }
            continue;
        }
        const int64_t sy = g.Lx, sz = (int64_t)g.Lx * g.Ly;
        const int64_t L = (int64_t)(g.lo[0] + bx) + sy * (g.lo[1] + by) + sz * (g.lo[2] + bz);
        uint32_t f = F_BOX;
        if (__ldg(a.mask + L)) {
            f |= F_MASK;
            if (bx > 0 && __ldg(a.mask + L - 1)) f |= F_MX;
            if (bx < g.n[0] - 1 && __ldg(a.mask + L + 1)) f |= F_PX;
            if (by > 0 && __ldg(a.mask + L - sy)) f |= F_MY;
            if (by < g.n[1] - 1 && __ldg(a.mask + L + sy)) f |= F_PY;
            if (bz > 0 && __ldg(a.mask + L - sz)) f |= F_MZ;
            if (bz < g.n[2] - 1 && __ldg(a.mask + L + sz)) f |= F_PZ;
        }
        a.flags[e] = (uint8_t)f;
        a.cell[e] = __ldg(a.cell_id + L);
        if (a.dfac) a.dfac[e] = __ldg(a.dfac_lat + L);
        for (int s = 0; s < a.nspecies; ++s) {
            const double c = __ldg(a.field[s] + L);
            a.x[s][e] = c;
            a.cn[s][e] = c;
        }
    }
}

struct ScatterArgs {
    double *field[kMaxSpecies];
    const double *x[kMaxSpecies];
    int32_t nspecies;
    const uint8_t *flags;
};

// Sec. 2.4: write the box solution onto the pleural mask (in-mask voxels only).
__global__ void __launch_bounds__(kBlock) k_scatter(ScatterArgs a, BoxGeo g, const int32_t *__restrict__ tile_coord,
                                                    int64_t NE)
{
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < NE; e += (int64_t)gridDim.x * kBlock) {
        if (!(a.flags[e] & F_MASK)) continue;
        int bx, by, bz;
        elem_box(e, g, tile_coord, bx, by, bz);
        const int64_t L = (int64_t)(g.lo[0] + bx) + (int64_t)g.Lx * ((g.lo[1] + by) + (int64_t)g.Ly * (g.lo[2] + bz));
        for (int s = 0; s < a.nspecies; ++s) a.field[s][L] = a.x[s][e];
    }
}

// Box-dense <-> compact conversions (tests, warm starts, the standalone operator).
__device__ __forceinline__ int64_t dense_to_elem(int64_t d, const BoxGeo &g, const int32_t *__restrict__ tile_index)
{
    const int bx = (int)(d % g.n[0]);
    const int64_t r = d / g.n[0];
    const int by = (int)(r % g.n[1]), bz = (int)(r / g.n[1]);
    const int32_t t = __ldg(tile_index + ((int64_t)(bz >> g.lt[2]) * g.nt[1] + (by >> g.lt[1])) * g.nt[0] + (bx >> g.lt[0]));
    if (t < 0) return -1;
    const int ix = bx & ((1 << g.lt[0]) - 1), iy = by & ((1 << g.lt[1]) - 1), iz = bz & ((1 << g.lt[2]) - 1);
    return ((int64_t)t << (g.lt[0] + g.lt[1] + g.lt[2])) + ix + ((int64_t)(iy + (iz << g.lt[1])) << g.lt[0]);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_export(const T *__restrict__ src, T dflt, BoxGeo g,
                                                   const int32_t *__restrict__ tile_index, T *__restrict__ dst,
                                                   int64_t nbox)
{
    for (int64_t d = (int64_t)blockIdx.x * kBlock + threadIdx.x; d < nbox; d += (int64_t)gridDim.x * kBlock) {
        const int64_t e = dense_to_elem(d, g, tile_index);
        dst[d] = e >= 0 ? src[e] : dflt;
    }
}

// dense -> compact; only_mask: write in-mask voxels only (import of a guess),
// else every in-box voxel of the active tiles.
__global__ void __launch_bounds__(kBlock) k_import(const double *__restrict__ src, BoxGeo g,
                                                   const int32_t *__restrict__ tile_index,
                                                   const uint8_t *__restrict__ flags, int only_mask,
                                                   double *__restrict__ dst, int64_t nbox)
{
    for (int64_t d = (int64_t)blockIdx.x * kBlock + threadIdx.x; d < nbox; d += (int64_t)gridDim.x * kBlock) {
        const int64_t e = dense_to_elem(d, g, tile_index);
        if (e < 0) continue;
        if (only_mask && !(flags[e] & F_MASK)) continue;
        dst[e] = src[d];
    }
}

// compact -> dense where stored, else the per-voxel default (identity rows)
__global__ void __launch_bounds__(kBlock) k_export_or(const double *__restrict__ src, const double *__restrict__ dflt,
                                                      BoxGeo g, const int32_t *__restrict__ tile_index,
                                                      double *__restrict__ dst, int64_t nbox)
{
    for (int64_t d = (int64_t)blockIdx.x * kBlock + threadIdx.x; d < nbox; d += (int64_t)gridDim.x * kBlock) {
        const int64_t e = dense_to_elem(d, g, tile_index);
        dst[d] = e >= 0 ? src[e] : dflt[d];
    }
}

static int grid_for(int64_t n, int num_sms, int per_sm = 8)
{
    int64_t g = (n + kBlock - 1) / kBlock;
    const int64_t cap = (int64_t)num_sms * per_sm;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

BoxGeo make_geo(const mpm_subgrid *sub, const int32_t dims[3])
{
    BoxGeo g;
    for (int d = 0; d < 3; ++d) {
        g.lo[d] = sub->lo[d];
        g.n[d] = sub->n[d];
        g.nt[d] = sub->nt[d];
        g.lt[d] = sub->lt[d];
    }
    g.Lx = (uint32_t)dims[0];
    g.Ly = (uint32_t)dims[1];
    return g;
}

}  // namespace mpm

using namespace mpm;

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Lattice arguments of an extraction: pointers, species fields, dims.
mpm_status mpm_lattice_check(mpm_ctx *ctx, const mpm_lattice *lat, int32_t nspecies)
{
    if (!lat || !lat->cell_id || !lat->mask) return mpm_fail(ctx, MPM_ERR_ARG, "extract: null argument");
    if (nspecies < 1 || nspecies > MPM_MAX_SPECIES) return mpm_fail(ctx, MPM_ERR_ARG, "extract: nspecies out of range");
    for (int s = 0; s < nspecies; ++s)
        if (!lat->field[s]) return mpm_fail(ctx, MPM_ERR_ARG, "extract: null field pointer");
    const int64_t L = (int64_t)lat->dims[0] * lat->dims[1] * lat->dims[2];
    if (lat->dims[0] < 1 || lat->dims[1] < 1 || lat->dims[2] < 1 || L >= (int64_t)1 << 31)
        return mpm_fail(ctx, MPM_ERR_ARG, "extract: lattice dims out of range");
    return MPM_OK;
}

// log2 tile dims from tile (null: 4x4x4, the fastest solve on thin shells
// among the shapes measured); powers of two <= 64, volume in [32, 1024].
mpm_status mpm_tile_lt(mpm_ctx *ctx, const int32_t tile[3], int32_t lt[3])
{
    lt[0] = lt[1] = lt[2] = 2;
    if (!tile) return MPM_OK;
    for (int d = 0; d < 3; ++d) {
        const int32_t t = tile[d];
        if (t < 1 || t > 64 || (t & (t - 1))) return mpm_fail(ctx, MPM_ERR_ARG, "extract: tile dims must be powers of two <= 64");
        lt[d] = __builtin_ctz((unsigned)t);
    }
    const int tv = 1 << (lt[0] + lt[1] + lt[2]);
    if (tv < 32 || tv > 1024) return mpm_fail(ctx, MPM_ERR_ARG, "extract: tile volume must be in [32, 1024]");
    return MPM_OK;
}

mpm_status mpm_extract_impl(mpm_ctx *ctx, const mpm_lattice *lat, int32_t nspecies, int32_t margin,
                            const int32_t tile[3], mpm_box *out_box, mpm_subgrid *sub, cudaStream_t st)
{
    if (!sub) return mpm_fail(ctx, MPM_ERR_ARG, "extract: null argument");
    mpm_status rc = mpm_lattice_check(ctx, lat, nspecies);
    if (rc != MPM_OK) return rc;
    const int64_t L = (int64_t)lat->dims[0] * lat->dims[1] * lat->dims[2];
    if (margin < 0) return mpm_fail(ctx, MPM_ERR_ARG, "extract: negative margin");
    int32_t lt[3];
    rc = mpm_tile_lt(ctx, tile, lt);
    if (rc != MPM_OK) return rc;

    // ---- a1: bounding box of the tumour voxels
    int32_t init[6] = {INT_MAX, INT_MAX, INT_MAX, -1, -1, -1};
    MPM_CU(cudaMemcpyAsync(ctx->d_box, init, sizeof(init), cudaMemcpyHostToDevice, st));
    const int vec4 = ((uintptr_t)lat->cell_id % 16) == 0;
    k_bbox<<<grid_for(L / 4 + 1, ctx->num_sms, 4), kBlock, 0, st>>>(lat->cell_id, (uint32_t)lat->dims[0],
                                                                     (uint32_t)(lat->dims[0] * lat->dims[1]),
                                                                     (uint32_t)L, vec4, ctx->d_box);
    ctx->launches += 1;
    MPM_CU(cudaGetLastError());
    // box geometry on the device; tile tables sized for the whole lattice, so
    // the only host round trip of the extract comes after the compaction
    BoxGeo *d_geo = (BoxGeo *)(ctx->d_box + 8);
    k_box_finalize<<<1, 32, 0, st>>>(ctx->d_box, margin, lat->dims[0], lat->dims[1], lat->dims[2], lt[0], lt[1], lt[2],
                                     d_geo);
    ctx->launches += 1;
    MPM_CU(cudaGetLastError());
    mpm_subgrid tmp = *sub;   // commit only on success
    const int64_t ntl = (((int64_t)lat->dims[0] + (1 << lt[0]) - 1) >> lt[0]) *
                        (((int64_t)lat->dims[1] + (1 << lt[1]) - 1) >> lt[1]) *
                        (((int64_t)lat->dims[2] + (1 << lt[2]) - 1) >> lt[2]);
    const size_t nt = (size_t)ntl;
    const size_t geo_need = align256(nt * 4) + align256(nt * 16) + align256(nt * 24) + align256(nt) + 256;
    void *const old_geo = sub->geo;
    const bool was_extracted = sub->extracted, was_assembled = sub->assembled;
    mpm_step_invalidate(sub);   // the tile tables are shared with the device-resident step
    sub->extracted = false;   // from here on the subgrid's buffers are rewritten
    sub->assembled = false;
    mpm_status s0 = mpm_grow(ctx, &sub->geo, &sub->geo_bytes, geo_need, "tile tables");
    tmp.geo = sub->geo;
    tmp.geo_bytes = sub->geo_bytes;
    if (s0 != MPM_OK) return s0;
    {
        char *p = (char *)tmp.geo;
        tmp.tile_index = (int32_t *)p; p += align256(nt * 4);
        tmp.tile_coord = (int32_t *)p; p += align256(nt * 16);
        tmp.nbr = (int32_t *)p; p += align256(nt * 24);
        tmp.active = (int8_t *)p; p += align256(nt);
        tmp.err = (int32_t *)p;
    }
    MPM_CU(cudaMemsetAsync(tmp.active, 0, nt, st));
    MPM_CU(cudaMemsetAsync(ctx->d_count, 0, 2 * sizeof(int64_t), st));
    k_tile_active<<<ctx->num_sms * 8, kBlock, 0, st>>>(lat->mask, d_geo, tmp.active, (unsigned long long *)ctx->d_count);
    ctx->launches += 1;
    MPM_CU(cudaGetLastError());
    k_tile_scan<<<1, 1024, 0, st>>>(tmp.active, d_geo, tmp.tile_index, tmp.tile_coord,
                                    (unsigned long long *)(ctx->d_count + 1));
    ctx->launches += 1;
    MPM_CU(cudaGetLastError());
    char *hs = (char *)ctx->h_stage;
    MPM_CU(cudaMemcpyAsync(hs, ctx->d_box, 6 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MPM_CU(cudaMemcpyAsync(hs + 64, ctx->d_count, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    MPM_CU(cudaStreamSynchronize(st));
    const int32_t *hb = (const int32_t *)hs;
    const int64_t *hc = (const int64_t *)(hs + 64);
    if (hb[3] < 0) {
        // no box: the subgrid keeps its previous extraction (its tile tables
        // were not written) unless the tile tables had to grow
        if (sub->geo == old_geo) {
            sub->extracted = was_extracted;
            sub->assembled = was_assembled;
        }
        return mpm_fail(ctx, MPM_ERR_EMPTY, "extract: no tumour voxel (cell_id > 0)");
    }
    MPM_CU(cudaMemsetAsync(tmp.err, 0, sizeof(int32_t), st));
    mpm_box box;
    for (int d = 0; d < 3; ++d) {
        box.lo[d] = hb[d] - margin < 0 ? 0 : hb[d] - margin;
        const int64_t h = (int64_t)hb[3 + d] + margin + 1;
        box.hi[d] = h > lat->dims[d] ? lat->dims[d] : (int32_t)h;
        tmp.lo[d] = box.lo[d];
        tmp.hi[d] = box.hi[d];
        tmp.n[d] = box.hi[d] - box.lo[d];
        tmp.lt[d] = lt[d];
        tmp.nt[d] = (tmp.n[d] + (1 << lt[d]) - 1) >> lt[d];
    }
    tmp.ntiles = tmp.nt[0] * tmp.nt[1] * tmp.nt[2];
    BoxGeo g = make_geo(&tmp, lat->dims);
    tmp.mask_voxels = hc[0];
    tmp.nact = (int32_t)hc[1];
    const int ltv = lt[0] + lt[1] + lt[2];
    tmp.NE = (int64_t)tmp.nact << ltv;
    tmp.nspecies = nspecies;
    tmp.has_dfac = lat->dfac != nullptr;

    // ---- element buffers
    const size_t NE = (size_t)tmp.NE;
    size_t need = align256(NE) + align256(NE * 4) + (tmp.has_dfac ? align256(NE * 8) : 0);
    need += (size_t)nspecies * (4 * align256(NE * 8) + align256(NE * 4));
    s0 = mpm_grow(ctx, &sub->elem, &sub->elem_bytes, need > 0 ? need : 256, "element buffers");
    tmp.elem = sub->elem;
    tmp.elem_bytes = sub->elem_bytes;
    if (s0 != MPM_OK) return s0;
    {
        char *p = (char *)tmp.elem;
        tmp.flags = (uint8_t *)p; p += align256(NE);
        tmp.cell = (int32_t *)p; p += align256(NE * 4);
        tmp.dfac = nullptr;
        if (tmp.has_dfac) { tmp.dfac = (double *)p; p += align256(NE * 8); }
        for (int s = 0; s < MPM_MAX_SPECIES; ++s) {
            tmp.x[s] = tmp.cn[s] = tmp.b[s] = tmp.diag[s] = nullptr;
            tmp.diag32[s] = nullptr;
        }
        for (int s = 0; s < nspecies; ++s) {
            tmp.x[s] = (double *)p; p += align256(NE * 8);
            tmp.cn[s] = (double *)p; p += align256(NE * 8);
            tmp.b[s] = (double *)p; p += align256(NE * 8);
            tmp.diag[s] = (double *)p; p += align256(NE * 8);
            tmp.diag32[s] = (float *)p; p += align256(NE * 4);
        }
    }
    if (tmp.nact > 0) {
        k_tile_nbr<<<(tmp.nact + 127) / 128, 128, 0, st>>>(tmp.tile_index, tmp.tile_coord,
                                                           (const unsigned long long *)(ctx->d_count + 1), d_geo, tmp.nbr);
        ctx->launches += 1;
        MPM_CU(cudaGetLastError());
        GatherArgs ga;
        memset(&ga, 0, sizeof(ga));
        ga.cell_id = lat->cell_id;
        ga.mask = lat->mask;
        ga.dfac_lat = lat->dfac;
        ga.nspecies = nspecies;
        ga.flags = tmp.flags;
        ga.cell = tmp.cell;
        ga.dfac = tmp.dfac;
        for (int s = 0; s < nspecies; ++s) {
            ga.field[s] = lat->field[s];
            ga.x[s] = tmp.x[s];
            ga.cn[s] = tmp.cn[s];
        }
        k_gather<<<grid_for(tmp.NE, ctx->num_sms, 8), kBlock, 0, st>>>(ga, g, tmp.tile_coord, tmp.NE);
        ctx->launches += 1;
        MPM_CU(cudaGetLastError());
    }
    for (int d = 0; d < 3; ++d) tmp.ldims[d] = lat->dims[d];
    tmp.gen = sub->gen + 1;
    tmp.extracted = true;
    tmp.assembled = false;
    tmp.x_fresh = true;
    *sub = tmp;
    if (out_box) *out_box = box;
    return MPM_OK;
}

// Active-tile count of the box for tile dims 2^lt (the tuner's bytes model):
// the same bbox, finalize, activity and compaction kernels as the extract, on
// the context's scratch tables.  Synchronises `st`.
mpm_status mpm_count_active_impl(mpm_ctx *ctx, const mpm_lattice *lat, int32_t margin, const int32_t lt[3],
                                 int64_t *nact, int64_t *mask_voxels, cudaStream_t st)
{
    const int64_t L = (int64_t)lat->dims[0] * lat->dims[1] * lat->dims[2];
    int32_t init[6] = {INT_MAX, INT_MAX, INT_MAX, -1, -1, -1};
    MPM_CU(cudaMemcpyAsync(ctx->d_box, init, sizeof(init), cudaMemcpyHostToDevice, st));
    const int vec4 = ((uintptr_t)lat->cell_id % 16) == 0;
    k_bbox<<<grid_for(L / 4 + 1, ctx->num_sms, 4), kBlock, 0, st>>>(lat->cell_id, (uint32_t)lat->dims[0],
                                                                     (uint32_t)(lat->dims[0] * lat->dims[1]),
                                                                     (uint32_t)L, vec4, ctx->d_box);
    BoxGeo *d_geo = (BoxGeo *)(ctx->d_box + 8);
    k_box_finalize<<<1, 32, 0, st>>>(ctx->d_box, margin, lat->dims[0], lat->dims[1], lat->dims[2], lt[0], lt[1], lt[2],
                                     d_geo);
    const int64_t ntl = (((int64_t)lat->dims[0] + (1 << lt[0]) - 1) >> lt[0]) *
                        (((int64_t)lat->dims[1] + (1 << lt[1]) - 1) >> lt[1]) *
                        (((int64_t)lat->dims[2] + (1 << lt[2]) - 1) >> lt[2]);
    const size_t nt = (size_t)ntl;
    const size_t need = align256(nt * 4) + align256(nt * 16) + align256(nt);
    mpm_status r = mpm_grow(ctx, &ctx->d_tune, &ctx->tune_cap, need, "tuner tables");
    if (r != MPM_OK) return r;
    char *p = (char *)ctx->d_tune;
    int32_t *tile_index = (int32_t *)p; p += align256(nt * 4);
    int32_t *tile_coord = (int32_t *)p; p += align256(nt * 16);
    int8_t *active = (int8_t *)p;
    MPM_CU(cudaMemsetAsync(active, 0, nt, st));
    MPM_CU(cudaMemsetAsync(ctx->d_count, 0, 2 * sizeof(int64_t), st));
    k_tile_active<<<ctx->num_sms * 8, kBlock, 0, st>>>(lat->mask, d_geo, active, (unsigned long long *)ctx->d_count);
    k_tile_scan<<<1, 1024, 0, st>>>(active, d_geo, tile_index, tile_coord, (unsigned long long *)(ctx->d_count + 1));
    ctx->launches += 4;
    MPM_CU(cudaGetLastError());
    int64_t *hc = (int64_t *)ctx->h_stage;
    MPM_CU(cudaMemcpyAsync(hc, ctx->d_count, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    MPM_CU(cudaStreamSynchronize(st));
    *mask_voxels = hc[0];
    *nact = hc[1];
    return MPM_OK;
}

mpm_status mpm_refresh_impl(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_lattice *lat, cudaStream_t st)
{
    if (!sub || !lat || !lat->cell_id || !lat->mask) return mpm_fail(ctx, MPM_ERR_ARG, "refresh: null argument");
    if (!sub->extracted) return mpm_fail(ctx, MPM_ERR_ARG, "refresh: subgrid not extracted");
    for (int d = 0; d < 3; ++d)
        if (lat->dims[d] != sub->ldims[d]) return mpm_fail(ctx, MPM_ERR_ARG, "refresh: lattice dims differ from the extraction");
    for (int s = 0; s < sub->nspecies; ++s)
        if (!lat->field[s]) return mpm_fail(ctx, MPM_ERR_ARG, "refresh: null field pointer");
    if ((lat->dfac != nullptr) != sub->has_dfac) return mpm_fail(ctx, MPM_ERR_ARG, "refresh: dfac presence differs from the extraction");
    sub->assembled = false;
    sub->x_fresh = true;
    if (sub->NE == 0) return MPM_OK;
    GatherArgs ga;
    memset(&ga, 0, sizeof(ga));
    ga.cell_id = lat->cell_id;
    ga.mask = lat->mask;
    ga.dfac_lat = lat->dfac;
    ga.nspecies = sub->nspecies;
    ga.flags = sub->flags;
    ga.cell = sub->cell;
    ga.dfac = sub->dfac;
    for (int s = 0; s < sub->nspecies; ++s) {
        ga.field[s] = lat->field[s];
        ga.x[s] = sub->x[s];
        ga.cn[s] = sub->cn[s];
    }
    BoxGeo g = make_geo(sub, lat->dims);
    k_gather<<<grid_for(sub->NE, ctx->num_sms, 8), kBlock, 0, st>>>(ga, g, sub->tile_coord, sub->NE);
    ctx->launches += 1;
    MPM_CU(cudaGetLastError());
    return MPM_OK;
}

mpm_status mpm_scatter_impl(mpm_ctx *ctx, const mpm_subgrid *sub, const mpm_lattice *lat, cudaStream_t st)
{
    if (!sub || !lat) return mpm_fail(ctx, MPM_ERR_ARG, "scatter: null argument");
    if (!sub->extracted) return mpm_fail(ctx, MPM_ERR_ARG, "scatter: subgrid not extracted");
    for (int s = 0; s < sub->nspecies; ++s)
        if (!lat->field[s]) return mpm_fail(ctx, MPM_ERR_ARG, "scatter: null field pointer");
    for (int d = 0; d < 3; ++d)
        if (sub->hi[d] > lat->dims[d]) return mpm_fail(ctx, MPM_ERR_ARG, "scatter: lattice smaller than the box");
    if (sub->NE == 0) return MPM_OK;
    ScatterArgs a;
    memset(&a, 0, sizeof(a));
    a.nspecies = sub->nspecies;
    a.flags = sub->flags;
    for (int s = 0; s < sub->nspecies; ++s) { a.field[s] = lat->field[s]; a.x[s] = sub->x[s]; }
    BoxGeo g = make_geo(sub, lat->dims);
    k_scatter<<<grid_for(sub->NE, ctx->num_sms, 8), kBlock, 0, st>>>(a, g, sub->tile_coord, sub->NE);
    ctx->launches += 1;
    MPM_CU(cudaGetLastError());
    return MPM_OK;
}

mpm_status mpm_export_impl(mpm_ctx *ctx, const mpm_subgrid *sub, int32_t what, int32_t s, void *dst, cudaStream_t st)
{
    if (!sub || !dst) return mpm_fail(ctx, MPM_ERR_ARG, "export: null argument");
    if (!sub->extracted) return mpm_fail(ctx, MPM_ERR_ARG, "export: subgrid not extracted");
    if ((what == MPM_EXPORT_X || what == MPM_EXPORT_RHS || what == MPM_EXPORT_DIAG) && (s < 0 || s >= sub->nspecies))
        return mpm_fail(ctx, MPM_ERR_ARG, "export: species out of range");
    if ((what == MPM_EXPORT_RHS || what == MPM_EXPORT_DIAG) && !sub->assembled)
        return mpm_fail(ctx, MPM_ERR_ARG, "export: subgrid not assembled");
    const int32_t dims[3] = {sub->n[0], sub->n[1], sub->n[2]};
    BoxGeo g = make_geo(sub, dims);
    const int64_t nbox = (int64_t)sub->n[0] * sub->n[1] * sub->n[2];
    const int grid = grid_for(nbox, ctx->num_sms, 8);
    switch (what) {
    case MPM_EXPORT_X:
        k_export<double><<<grid, kBlock, 0, st>>>(sub->x[s], 0.0, g, sub->tile_index, (double *)dst, nbox);
        ctx->launches += 1; break;
    case MPM_EXPORT_RHS:
        k_export<double><<<grid, kBlock, 0, st>>>(sub->b[s], 0.0, g, sub->tile_index, (double *)dst, nbox);
        ctx->launches += 1; break;
    case MPM_EXPORT_DIAG:
        k_export<double><<<grid, kBlock, 0, st>>>(sub->diag[s], 1.0, g, sub->tile_index, (double *)dst, nbox);
        ctx->launches += 1; break;
    case MPM_EXPORT_FLAGS:
        k_export<uint8_t><<<grid, kBlock, 0, st>>>(sub->flags, (uint8_t)0, g, sub->tile_index, (uint8_t *)dst, nbox);
        ctx->launches += 1; break;
    case MPM_EXPORT_CELL:
        k_export<int32_t><<<grid, kBlock, 0, st>>>(sub->cell, 0, g, sub->tile_index, (int32_t *)dst, nbox);
        ctx->launches += 1; break;
    default:
        return mpm_fail(ctx, MPM_ERR_ARG, "export: unknown field");
    }
    MPM_CU(cudaGetLastError());
    return MPM_OK;
}

mpm_status mpm_import_impl(mpm_ctx *ctx, mpm_subgrid *sub, int32_t s, const double *src, cudaStream_t st)
{
    if (!sub || !src) return mpm_fail(ctx, MPM_ERR_ARG, "import: null argument");
    if (!sub->extracted) return mpm_fail(ctx, MPM_ERR_ARG, "import: subgrid not extracted");
    if (s < 0 || s >= sub->nspecies) return mpm_fail(ctx, MPM_ERR_ARG, "import: species out of range");
    const int32_t dims[3] = {sub->n[0], sub->n[1], sub->n[2]};
    BoxGeo g = make_geo(sub, dims);
    const int64_t nbox = (int64_t)sub->n[0] * sub->n[1] * sub->n[2];
    k_import<<<grid_for(nbox, ctx->num_sms, 8), kBlock, 0, st>>>(src, g, sub->tile_index, sub->flags, 1, sub->x[s], nbox);
    ctx->launches += 1;
    MPM_CU(cudaGetLastError());
    sub->x_fresh = false;
    return MPM_OK;
}

// prediction [V][3] (float, box-dense) -> iterate of every species on in-mask voxels
__global__ void __launch_bounds__(kBlock) k_import_pred(const float *__restrict__ pred, BoxGeo g,
                                                        const int32_t *__restrict__ tile_index,
                                                        const uint8_t *__restrict__ flags, int nspecies,
                                                        double *x0, double *x1, double *x2, int64_t nbox)
{
    for (int64_t d = (int64_t)blockIdx.x * kBlock + threadIdx.x; d < nbox; d += (int64_t)gridDim.x * kBlock) {
        const int64_t e = dense_to_elem(d, g, tile_index);
        if (e < 0 || !(flags[e] & F_MASK)) continue;
        x0[e] = (double)pred[d * 3 + 0];
        if (nspecies > 1) x1[e] = (double)pred[d * 3 + 1];
        if (nspecies > 2) x2[e] = (double)pred[d * 3 + 2];
    }
}

mpm_status mpm_import_pred_impl(mpm_ctx *ctx, mpm_subgrid *sub, const float *pred, cudaStream_t st)
{
    const int32_t dims[3] = {sub->n[0], sub->n[1], sub->n[2]};
    BoxGeo g = make_geo(sub, dims);
    const int64_t nbox = (int64_t)sub->n[0] * sub->n[1] * sub->n[2];
    k_import_pred<<<grid_for(nbox, ctx->num_sms, 8), kBlock, 0, st>>>(pred, g, sub->tile_index, sub->flags,
                                                                      sub->nspecies, sub->x[0], sub->x[1], sub->x[2], nbox);
    ctx->launches += 1;
    MPM_CU(cudaGetLastError());
    sub->x_fresh = false;
    return MPM_OK;
}

// used by mpm_apply_impl (assemble.cu)
mpm_status mpm_dense_to_elems(mpm_ctx *ctx, const mpm_subgrid *sub, const double *src, double *dst, cudaStream_t st)
{
    const int32_t dims[3] = {sub->n[0], sub->n[1], sub->n[2]};
    BoxGeo g = make_geo(sub, dims);
    const int64_t nbox = (int64_t)sub->n[0] * sub->n[1] * sub->n[2];
    MPM_CU(cudaMemsetAsync(dst, 0, (size_t)sub->NE * sizeof(double), st));
    k_import<<<grid_for(nbox, ctx->num_sms, 8), kBlock, 0, st>>>(src, g, sub->tile_index, sub->flags, 0, dst, nbox);
    ctx->launches += 1;
    MPM_CU(cudaGetLastError());
    return MPM_OK;
}

mpm_status mpm_elems_to_dense(mpm_ctx *ctx, const mpm_subgrid *sub, const double *src, const double *dflt_dense,
                              double *dst, cudaStream_t st)
{
    const int32_t dims[3] = {sub->n[0], sub->n[1], sub->n[2]};
    BoxGeo g = make_geo(sub, dims);
    const int64_t nbox = (int64_t)sub->n[0] * sub->n[1] * sub->n[2];
    k_export_or<<<grid_for(nbox, ctx->num_sms, 8), kBlock, 0, st>>>(src, dflt_dense, g, sub->tile_index, dst, nbox);
    ctx->launches += 1;
    MPM_CU(cudaGetLastError());
    return MPM_OK;
}

// ---------------------------------------------------------------- device-resident step
// Buffers of a subgrid sized for the whole lattice: every box of this lattice
// fits, so the step never has to learn the box size on the host before it
// launches the next stage.  Element buffers hold ceil(L/T) tiles of T voxels
// per axis; pointers move only when a buffer grows.
mpm_status mpm_step_buffers(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_lattice *lat, int32_t nspecies, const int32_t lt[3])
{
    const int64_t ntl = (((int64_t)lat->dims[0] + (1 << lt[0]) - 1) >> lt[0]) *
                        (((int64_t)lat->dims[1] + (1 << lt[1]) - 1) >> lt[1]) *
                        (((int64_t)lat->dims[2] + (1 << lt[2]) - 1) >> lt[2]);
    const size_t nt = (size_t)ntl;
    const size_t NE = nt << (lt[0] + lt[1] + lt[2]);
    const bool has_dfac = lat->dfac != nullptr;
    const size_t geo_need = align256(nt * 4) + align256(nt * 16) + align256(nt * 24) + align256(nt) + 256;
    size_t need = align256(NE) + align256(NE * 4) + (has_dfac ? align256(NE * 8) : 0);
    need += (size_t)nspecies * (4 * align256(NE * 8) + align256(NE * 4));
    sub->extracted = false;
    sub->assembled = false;
    mpm_status r = mpm_grow(ctx, &sub->geo, &sub->geo_bytes, geo_need, "tile tables");
    if (r != MPM_OK) return r;
    r = mpm_grow(ctx, &sub->elem, &sub->elem_bytes, need, "element buffers");
    if (r != MPM_OK) return r;
    char *p = (char *)sub->geo;
    sub->tile_index = (int32_t *)p; p += align256(nt * 4);
    sub->tile_coord = (int32_t *)p; p += align256(nt * 16);
    sub->nbr = (int32_t *)p; p += align256(nt * 24);
    sub->active = (int8_t *)p; p += align256(nt);
    sub->err = (int32_t *)p;
    p = (char *)sub->elem;
    sub->flags = (uint8_t *)p; p += align256(NE);
    sub->cell = (int32_t *)p; p += align256(NE * 4);
    sub->dfac = nullptr;
    if (has_dfac) { sub->dfac = (double *)p; p += align256(NE * 8); }
    for (int s = 0; s < MPM_MAX_SPECIES; ++s) {
        sub->x[s] = sub->cn[s] = sub->b[s] = sub->diag[s] = nullptr;
        sub->diag32[s] = nullptr;
    }
    for (int s = 0; s < nspecies; ++s) {
        sub->x[s] = (double *)p; p += align256(NE * 8);
        sub->cn[s] = (double *)p; p += align256(NE * 8);
        sub->b[s] = (double *)p; p += align256(NE * 8);
        sub->diag[s] = (double *)p; p += align256(NE * 8);
        sub->diag32[s] = (float *)p; p += align256(NE * 4);
    }
    for (int d = 0; d < 3; ++d) {
        sub->lt[d] = lt[d];
        sub->ldims[d] = lat->dims[d];
    }
    sub->nspecies = nspecies;
    sub->has_dfac = has_dfac;
    sub->NE_cap = (int64_t)NE;
    return MPM_OK;
}

