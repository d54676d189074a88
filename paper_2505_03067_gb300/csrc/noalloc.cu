// noalloc.cu -- a bounding-box reduction for callers that cannot allocate
// device memory.
//
// mpm_box_extract computes the tumour box with atomics into a context's
// device scratch, and creating a context allocates.  Some callers may not
// allocate at all: code whose device memory is entirely owned by another
// allocator (a framework's caching allocator or a pool fixed at start-up),
// code that must not risk the device-wide synchronisation cudaMalloc and
// cudaFree can cause while other streams run, or a plugin whose host
// application controls every allocation.  mpm_box_bounds_noalloc serves them:
// it needs no context, and its only scratch is the fixed array below, which
// lives in the library image and is held by every GPU that loads the library
// until the process exits.
#include <climits>
#include <mutex>

#include "mpm_internal.cuh"

namespace {

constexpr int kSlabInts = 8;   // per z-slice: min x, min y, max x, max y, any tumour, 3 unused

// Per-z-slice partial bounds.  Every call rewrites the entries of the slices
// it covers before reading them, so nothing needs clearing between calls;
// calls that overlap on the GPU share this array and race.
static __device__ __align__(256) int32_t g_slab_bounds[MPM_NOALLOC_MAX_SLABS * kSlabInts];

// One CTA per z-slice: min/max (x, y) of the voxels with cell id > 0.
__global__ void __launch_bounds__(256) k_slab_bounds(const int32_t *__restrict__ cell, uint32_t Lx, uint32_t Ly,
                                                     int32_t *__restrict__ slabs)
{
    const uint32_t k = blockIdx.x;
    const uint32_t n = Lx * Ly;
    const int32_t *c = cell + (size_t)k * n;
    int mnx = INT_MAX, mny = INT_MAX, mxx = -1, mxy = -1;
    for (uint32_t v = threadIdx.x; v < n; v += blockDim.x) {
        if (__ldg(c + v) > 0) {
            const int y = (int)(v / Lx), x = (int)(v - (uint32_t)y * Lx);
            mnx = min(mnx, x); mxx = max(mxx, x);
            mny = min(mny, y); mxy = max(mxy, y);
        }
    }
    mnx = __reduce_min_sync(0xffffffffu, mnx);
    mny = __reduce_min_sync(0xffffffffu, mny);
    mxx = __reduce_max_sync(0xffffffffu, mxx);
    mxy = __reduce_max_sync(0xffffffffu, mxy);
    __shared__ int s[4][8];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s[0][w] = mnx; s[1][w] = mny; s[2][w] = mxx; s[3][w] = mxy; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            s[0][0] = min(s[0][0], s[0][i]); s[1][0] = min(s[1][0], s[1][i]);
            s[2][0] = max(s[2][0], s[2][i]); s[3][0] = max(s[3][0], s[3][i]);
        }
        int32_t *o = slabs + (size_t)k * kSlabInts;
        o[0] = s[0][0]; o[1] = s[1][0]; o[2] = s[2][0]; o[3] = s[3][0];
        o[4] = s[2][0] >= 0 ? 1 : 0;
    }
}

// One CTA: combine the slices, widen by the margin and clamp (the same box
// rule as mpm_box_extract), write lo[3], hi[3] and a found flag.
__global__ void __launch_bounds__(1024) k_slab_reduce(const int32_t *__restrict__ slabs, int32_t Lx, int32_t Ly,
                                                      int32_t Lz, int32_t margin, int32_t *__restrict__ out)
{
    int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {-1, -1, -1};
    for (int k = threadIdx.x; k < Lz; k += blockDim.x) {
        const int32_t *o = slabs + (size_t)k * kSlabInts;
        if (o[4]) {
            mn[0] = min(mn[0], o[0]); mn[1] = min(mn[1], o[1]); mn[2] = min(mn[2], k);
            mx[0] = max(mx[0], o[2]); mx[1] = max(mx[1], o[3]); mx[2] = max(mx[2], k);
        }
    }
    __shared__ int s[6][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int a = __reduce_min_sync(0xffffffffu, mn[d]);
        const int b = __reduce_max_sync(0xffffffffu, mx[d]);
        if (lane == 0) { s[d][w] = a; s[3 + d][w] = b; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (int)(blockDim.x >> 5);
        const int32_t L[3] = {Lx, Ly, Lz};
        int a[3], b[3];
        for (int d = 0; d < 3; ++d) {
            a[d] = s[d][0];
            b[d] = s[3 + d][0];
            for (int i = 1; i < nw; ++i) { a[d] = min(a[d], s[d][i]); b[d] = max(b[d], s[3 + d][i]); }
        }
        const int found = b[0] >= 0;
        for (int d = 0; d < 3; ++d) {
            out[d] = found ? max(0, a[d] - margin) : 0;
            out[3 + d] = found ? (int32_t)min((int64_t)L[d], (int64_t)b[d] + margin + 1) : 0;
        }
        out[6] = found;
    }
}

// Device address of g_slab_bounds per device ordinal, looked up once.  A
// cudaDeviceReset unloads the module that holds the array, so an address
// cached before a reset is stale afterwards: a process that resets a device
// must not call this entry point on that device again.
std::mutex g_mu;
int32_t *g_ptr[64] = {};

}  // namespace

extern "C" mpm_status mpm_box_bounds_noalloc(const int32_t *cell_id, const int32_t dims[3], int32_t margin,
                                             int32_t *out_box, void *stream)
{
    if (!cell_id || !dims || !out_box || margin < 0) return MPM_ERR_ARG;
    if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1) return MPM_ERR_ARG;
    if ((int64_t)dims[0] * dims[1] * dims[2] >= ((int64_t)1 << 31)) return MPM_ERR_ARG;
    if (dims[2] > MPM_NOALLOC_MAX_SLABS) return MPM_ERR_NOMEM;   // more z-slices than the fixed scratch holds
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); return MPM_ERR_CUDA; }
    int32_t *scratch = nullptr;
    {
        // first call on a device: look up the device address of the static
        // scratch with that device current (no allocation happens here)
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_slab_bounds) != cudaSuccess || !p) { cudaGetLastError(); return MPM_ERR_CUDA; }
            g_ptr[dev] = (int32_t *)p;
        }
        scratch = g_ptr[dev];
    }
    // launched through cudaLaunchKernel so that each launch's own return code
    // is checked: an error left pending by unrelated earlier work is neither
    // consumed nor reported as this call's failure
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t lx = (uint32_t)dims[0], ly = (uint32_t)dims[1];
    const int32_t *cell = cell_id;
    void *a1[] = {(void *)&cell, (void *)&lx, (void *)&ly, (void *)&scratch};
    if (cudaLaunchKernel((const void *)k_slab_bounds, dim3((unsigned)dims[2]), dim3(256), a1, 0, st) != cudaSuccess)
        return MPM_ERR_CUDA;
    int32_t Lx = dims[0], Ly = dims[1], Lz = dims[2], mg = margin;
    int32_t *ob = out_box;
    void *a2[] = {(void *)&scratch, (void *)&Lx, (void *)&Ly, (void *)&Lz, (void *)&mg, (void *)&ob};
    if (cudaLaunchKernel((const void *)k_slab_reduce, dim3(1), dim3(1024), a2, 0, st) != cudaSuccess)
        return MPM_ERR_CUDA;
    return MPM_OK;
}
