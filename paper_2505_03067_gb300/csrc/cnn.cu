// cnn.cu -- the learned warm start: a small 3D CNN evaluated and trained on
// the GPU by the library's own tensor-core kernels (cnn_tc.cuh).  The paper
// has no network; this is one of the faster forms built around its solve.
//
// Network: six 3x3x3 convolutions with zero padding and a bias, channels
// 9 -> 24 -> 24 -> 24 -> 24 -> 24 -> 3, erf-GELU after layers 1-5, a residual
// output pred = c^n + s_out * z6 (the next-step fields), and an activity
// mask: the network sees the pleural space of its box only -- the layer-1
// input and the activations a_1..a_5 are zero at voxels outside the mask or
// the box, as a masked voxel contributes nothing to the finite-volume
// operator (zero flux, Sec. 2.4).
//
// Storage.  bf16 channel-last [voxel][C] buffers indexed like the lattice
// (images of dims L stacked along z): C = 16 for the 9 features (channel 15
// holds a constant 1 at active voxels: its row of the weight gradient is the
// bias gradient; its weights are zero), 24 for hidden activations and
// gradients, 8 for the output gradient; FP32 pre-activations for the backward
// pass.  Parameters: an FP32 master vector in the flat layout
// [W_1, b_1, ..., W_6, b_6], W_l[27][Ci][Co] with tap (dx+1) + 3(dy+1) +
// 9(dz+1), and per layer a bf16 weight image for the forward convolution and
// one for the input gradient (taps flipped, channels swapped), laid out as
// the tensor cores read them from shared memory.
#include <cuda_bf16.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "cnn_tc.cuh"

namespace mpm {

using tc::CnnDom;
using tc::Unit;

constexpr int kLayers = 6;
__host__ __device__ constexpr int chan(int l) { return l == 0 ? 9 : (l == kLayers ? 3 : 24); }
constexpr int kXC = 16;   // feature channels stored per voxel
constexpr int kHC = 24;   // hidden channels stored per voxel
constexpr int kGC6 = 8;   // output-gradient channels stored per voxel

// Stored input channels and MMA N of each layer's forward convolution, and of
// the input-gradient convolution through layer l (l >= 1).
__host__ __device__ constexpr int fwd_ci(int l) { return l == 0 ? kXC : kHC; }
__host__ __device__ constexpr int fwd_no(int l) { return l == kLayers - 1 ? 16 : 32; }
__host__ __device__ constexpr int dg_ci(int l) { return l == kLayers - 1 ? kGC6 : kHC; }

__host__ __device__ constexpr int wimg_bytes(int ci, int no)
{
    return 9 * (3 * (ci / 8) + ((3 * (ci / 8)) & 1)) * (no / 8) * 128;
}

// ---------------------------------------------------------------- weights
struct PrepArgs {
    const float *master;
    long long off[kLayers];
    unsigned char *wf[kLayers];    // forward weight images
    unsigned char *wd[kLayers];    // input-gradient weight images (l >= 1)
    float *bias[kLayers];          // [fwd_no(l)]
};

// Entry e (a bf16 element) of a weight image with input channels CI and N =
// NO: core matrix cm = e / 64 at ((dy+1) * QP + q) * 3 NG + (dz+1) * NG + ng,
// row r, column j.  Forward: value W[t][ci][co]; input gradient:
// W[26 - t][co][ci] (the tap mirrored, input and output channels exchanged).
__device__ float wimg_value(const float *W, int Ci, int Co, int CI, int NO, int e, bool dgrad)
{
    const int KC = CI / 8, QC = 3 * KC, QP = QC + (QC & 1), NG = NO / 8;
    const int cm = e >> 6, w = e & 63, r = w >> 3, j = w & 7;
    const int nn = cm % (3 * NG), rest = cm / (3 * NG);
    const int q = rest % QP, dyi = rest / QP;
    const int dzi = nn / NG, ng = nn % NG;
    if (q >= QC) return 0.0f;
    const int c = q / KC, kc = q % KC;
    const int dx = c - 1, dy = dyi - 1, dz = dzi - 1;
    const int t = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
    const int n = ng * 8 + r, k = kc * 8 + j;   // output, input channel of this convolution
    if (!dgrad) return (k < Ci && n < Co) ? W[((long long)t * Ci + k) * Co + n] : 0.0f;
    // input-gradient convolution of layer (Ci -> Co): its inputs are the Co channels
    return (k < Co && n < Ci) ? W[((long long)(26 - t) * Ci + n) * Co + k] : 0.0f;
}

__global__ void k_prep_weights(PrepArgs P)
{
    const int l = blockIdx.y;
    const int Ci = chan(l), Co = chan(l + 1);
    const float *W = P.master + P.off[l];
    const int nf = wimg_bytes(fwd_ci(l), fwd_no(l)) / 2;
    __nv_bfloat16 *wf = reinterpret_cast<__nv_bfloat16 *>(P.wf[l]);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nf; e += gridDim.x * blockDim.x)
        wf[e] = __float2bfloat16_rn(wimg_value(W, Ci, Co, fwd_ci(l), fwd_no(l), e, false));
    if (l > 0) {
        const int nd = wimg_bytes(dg_ci(l), 32) / 2;
        __nv_bfloat16 *wd = reinterpret_cast<__nv_bfloat16 *>(P.wd[l]);
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nd; e += gridDim.x * blockDim.x)
            wd[e] = __float2bfloat16_rn(wimg_value(W, Ci, Co, dg_ci(l), 32, e, true));
    }
    if (blockIdx.x == 0)
        for (int c = threadIdx.x; c < fwd_no(l); c += blockDim.x) P.bias[l][c] = c < Co ? W[27LL * Ci * Co + c] : 0.0f;
}

// The gradient of layer l's weights and bias from the weight-gradient
// kernel's per-CTA partial sums (summed in CTA order): row m of tap pair p
// holds (dx copy c, channel ci) = ((c * KC + kc) * 8 + j); the bias row is
// the ones column (CI = 24: the pad K-column; CI = 16: feature channel 15).
__global__ void k_wgrad_reduce(const float *__restrict__ partials, int nblk, int CI, int NO, int Ci, int Co,
                               float *__restrict__ grads)
{
    const int KC = CI / 8;
    const int n = 27 * Ci * Co + Co;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int p, m, co;
        if (i < 27 * Ci * Co) {
            const int t = i / (Ci * Co), ci = (i / Co) % Ci;
            co = i % Co;
            const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
            p = (dy + 1) + 3 * (dz + 1);
            m = ((dx + 1) * KC + ci / 8) * 8 + (ci % 8);
        } else {
            co = i - 27 * Ci * Co;
            p = 4;
            m = CI == kHC ? 3 * KC * 8 : (KC + 1) * 8 + 7;
        }
        float s = 0.0f;
        for (int b = 0; b < nblk; ++b) s += partials[(((size_t)b * 9 + p) * 128 + m) * NO + co];
        grads[i] = s;
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ---------------------------------------------------------------- plans
// Candidate unit ci of image mode -> unit record; false if it lies outside its image's box.
__device__ __forceinline__ bool unit_of(const CnnDom &D, int64_t ci, Unit &u)
{
    const int nsx = (D.L[0] + tc::kSlabX - 1) / tc::kSlabX, nsy = (D.L[1] + tc::kSlabY - 1) / tc::kSlabY;
    const int nzs = (D.L[2] + tc::kZSeg - 1) / tc::kZSeg;
    const int i = (int)(ci % nsx);
    int64_t r = ci / nsx;
    const int j = (int)(r % nsy);
    r /= nsy;
    const int kz = (int)(r % nzs);
    const int b = (int)(r / nzs);
    u.b = b;
    u.ox = D.lo[b][0] + i * tc::kSlabX;
    u.oy = D.lo[b][1] + j * tc::kSlabY;
    u.z0 = D.lo[b][2] + kz * tc::kZSeg;
    u.nz = min(tc::kZSeg, D.n[b][2] - kz * tc::kZSeg);
    u.pad0 = u.pad1 = u.pad2 = 0;
    return i * tc::kSlabX < D.n[b][0] && j * tc::kSlabY < D.n[b][1] && u.nz > 0;
}

// Image mode, one warp per candidate unit: any active voxel (in the box, mask set)?
__global__ void k_plan_flags(const __grid_constant__ CnnDom D, const uint8_t *__restrict__ mask, int64_t ncand,
                             uint8_t *__restrict__ flags)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (gridDim.x * (int64_t)blockDim.x) >> 5;
    for (int64_t c = w0; c < ncand; c += nw) {
        Unit u;
        bool any = false;
        if (unit_of(D, c, u)) {
            for (int i = lane; i < tc::kSlabX * tc::kSlabY * u.nz && !any; i += 32) {
                const int x = u.ox + (i & 7), y = u.oy + ((i >> 3) & 15), z = u.z0 + (i >> 7);
                any = tc::in_box(D, u.b, x, y, z) && mask[tc::vox_index(D, u.b, x, y, z)] != 0;
            }
        }
        any = __any_sync(0xffffffffu, any);
        if (lane == 0) flags[c] = any ? 1 : 0;
    }
}

// Image mode, one CTA: the flagged units in candidate order (a fixed order:
// the weight gradient's per-CTA sums depend on it); writes the domain too.
__global__ void __launch_bounds__(1024) k_plan_compact(const __grid_constant__ CnnDom D,
                                                       const uint8_t *__restrict__ flags, int64_t ncand,
                                                       Unit *__restrict__ units, int32_t *__restrict__ counters,
                                                       CnnDom *__restrict__ dom_out)
{
    __shared__ int s_w[32];
    __shared__ int s_base;
    if (threadIdx.x == 0) {
        s_base = 0;
        *dom_out = D;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t c0 = 0; c0 < ncand; c0 += 1024) {
        const int64_t c = c0 + threadIdx.x;
        const bool f = c < ncand && flags[c];
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) s_w[wid] = __popc(bal);
        __syncthreads();
        int off = 0, tot = 0;
        for (int i = 0; i < 32; ++i) {
            if (i < wid) off += s_w[i];
            tot += s_w[i];
        }
        if (f) {
            Unit u;
            unit_of(D, c, u);
            units[s_base + off + __popc(bal & ((1u << lane) - 1u))] = u;
        }
        __syncthreads();
        if (threadIdx.x == 0) s_base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) counters[0] = s_base;
}

// Solver mode: the box of a subgrid (from device memory) on a lattice of dims
// L.  Units are placed along y where the pleural space is: one warp per band
// of the box (8 x columns by a segment of up to 8 depths) marks the band's
// active tile rows (a row of the subgrid's tiles is active when a tile of it
// overlapping the band is stored, i.e. holds an in-mask voxel) and starts a
// unit of 16 rows at the first active tile row, the next one at the first
// active tile row at or after the previous unit's end (or at that end), and
// so on.  Units of a band never overlap and every in-mask voxel of the box
// lies in one.  On the thin pleural shell with 4-row tiles this lists ~10 %
// fewer units and ~7 % fewer active slabs than a fixed 16-row grid.  Unit
// starts lie in [0, n_y) at least 16 rows apart, so a band has at most
// ceil(n_y / 16) units; a listing past `max_units` sets *err and is dropped.
// counters[0] must be zero; the listing order does not matter.
__global__ void __launch_bounds__(256) k_plan_box(const BoxGeo *__restrict__ geo, const int32_t *__restrict__ tile_index,
                                                  int32_t L0, int32_t L1, int32_t L2, Unit *__restrict__ units,
                                                  int32_t *__restrict__ counters, int64_t max_units,
                                                  CnnDom *__restrict__ dom_out, int32_t *__restrict__ err)
{
    const BoxGeo g = *geo;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        CnnDom D;
        memset(&D, 0, sizeof(D));
        D.L[0] = L0;
        D.L[1] = L1;
        D.L[2] = L2;
        D.B = 1;
        for (int d = 0; d < 3; ++d) {
            D.lo[0][d] = g.lo[d];
            D.n[0][d] = g.n[d];
        }
        *dom_out = D;
    }
    if (g.n[0] <= 0) return;
    const int nxb = (g.n[0] + tc::kSlabX - 1) / tc::kSlabX, nzs = (g.n[2] + tc::kZSeg - 1) / tc::kZSeg;
    const int64_t nbands = (int64_t)nxb * nzs;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (gridDim.x * (int64_t)blockDim.x) >> 5;
    const int ty_n = g.nt[1], ly = g.lt[1];
    for (int64_t band = w0; band < nbands; band += nw) {
        const int bx0 = (int)(band % nxb) * tc::kSlabX, bz0 = (int)(band / nxb) * tc::kZSeg;
        const int nx = min(tc::kSlabX, g.n[0] - bx0), nz = min(tc::kZSeg, g.n[2] - bz0);
        const int tx0 = bx0 >> g.lt[0], tx1 = (bx0 + nx - 1) >> g.lt[0];
        const int tz0 = bz0 >> g.lt[2], tz1 = (bz0 + nz - 1) >> g.lt[2];
        int next_free = 0;                        // first box row no unit of this band covers
        for (int t0 = 0; t0 < ty_n; t0 += 32) {
            const int ty = t0 + lane;
            bool a = false;
            if (ty < ty_n)
                for (int tz = tz0; tz <= tz1 && !a; ++tz)
                    for (int tx = tx0; tx <= tx1 && !a; ++tx)
                        a = __ldg(tile_index + ((int64_t)tz * ty_n + ty) * g.nt[0] + tx) >= 0;
            unsigned act = __ballot_sync(0xffffffffu, a);
            // units over these tile rows (warp-uniform walk; lane 0 lists them):
            // each active tile row is covered from its first box row, or from
            // the previous unit's end when that lies inside it, to its end
            while (act) {
                const int b = __ffs(act) - 1;
                act &= act - 1u;
                const int r0 = (t0 + b) << ly, r1 = min((t0 + b + 1) << ly, g.n[1]);
                while (next_free < r1) {
                    const int start = r0 > next_free ? r0 : next_free;
                    if (lane == 0) {
                        const int64_t k = atomicAdd(counters, 1);
                        if (k < max_units) {
                            Unit u;
                            u.b = 0;
                            u.ox = g.lo[0] + bx0;
                            u.oy = g.lo[1] + start;
                            u.z0 = g.lo[2] + bz0;
                            u.nz = nz;
                            u.pad0 = u.pad1 = u.pad2 = 0;
                            units[k] = u;
                        } else {
                            atomicExch(err, 1);
                        }
                    }
                    next_free = start + tc::kSlabY;
                }
            }
        }
    }
}

// ---------------------------------------------------------------- features
// Feature channels of a voxel: c^n of the 3 species scaled (1, 1, 20), one-hot
// medium / tumour, the cell's rates scaled 10 (uptake of species 0 and 1,
// source of species 2), the mask, and channel 15 = 1.
struct FeatSrc {
    const int32_t *cell;
    const double *field[kMaxSpecies];
    int nspecies, ncell;
    const double *k_cell, *q_cell;
};

__device__ __forceinline__ void feat_store(__nv_bfloat16 *xo, const float (&f)[kXC])
{
    uint32_t w[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * c], f[2 * c + 1]);
        w[c] = *reinterpret_cast<uint32_t *>(&h);
    }
    reinterpret_cast<uint4 *>(xo)[0] = make_uint4(w[0], w[1], w[2], w[3]);
    reinterpret_cast<uint4 *>(xo)[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// fld[s]: the value of species s's field channel before scaling
__device__ __forceinline__ void features_of(const FeatSrc &F, int64_t L, const float (&fld)[3], bool with_source,
                                            float (&f)[kXC])
{
    int id = F.cell[L];
    if (id < 0 || id >= F.ncell) id = 0;
#pragma unroll
    for (int c = 0; c < kXC; ++c) f[c] = 0.0f;
    f[0] = fld[0] * 1.0f;
    f[1] = fld[1] * 1.0f;
    f[2] = fld[2] * 20.0f;
    f[3] = id == 0 ? 1.0f : 0.0f;
    f[4] = id > 0 ? 1.0f : 0.0f;
    f[5] = F.nspecies > 0 ? (float)F.k_cell[id] * 10.0f : 0.0f;
    f[6] = F.nspecies > 1 ? (float)F.k_cell[F.ncell + id] * 10.0f : 0.0f;
    f[7] = (with_source && F.nspecies > 2) ? (float)F.q_cell[2 * (long long)F.ncell + id] * 10.0f : 0.0f;
    f[8] = 1.0f;
    f[15] = 1.0f;
}

// Image mode: the box voxels of lattice F (dims = the image dims) into image b:
// mask, features and c^n (FP32).
__global__ void k_feat_image(FeatSrc F, const uint8_t *__restrict__ lmask, int32_t L0, int32_t L1, int32_t L2, int b,
                             int32_t lo0, int32_t lo1, int32_t lo2, int32_t n0, int32_t n1, int32_t n2,
                             uint8_t *__restrict__ mask, __nv_bfloat16 *__restrict__ x, float *__restrict__ f32)
{
    const int64_t nb = (int64_t)n0 * n1 * n2;
    const int64_t img = (int64_t)b * L0 * L1 * L2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += gridDim.x * (int64_t)blockDim.x) {
        const int xx = lo0 + (int)(i % n0);
        const int64_t r = i / n0;
        const int yy = lo1 + (int)(r % n1), zz = lo2 + (int)(r / n1);
        const int64_t L = xx + (int64_t)L0 * (yy + (int64_t)L1 * zz);
        const int64_t v = img + L;
        const uint8_t m = lmask[L] != 0;
        mask[v] = m;
        float fld[3];
        for (int s = 0; s < 3; ++s) fld[s] = s < F.nspecies ? (float)F.field[s][L] : 0.0f;
        for (int s = 0; s < 3; ++s) f32[v * 3 + s] = fld[s];
        float f[kXC];
        features_of(F, L, fld, true, f);
        if (!m) {
#pragma unroll
            for (int c = 0; c < kXC; ++c) f[c] = 0.0f;
        }
        feat_store(x + v * kXC, f);
    }
}

// Image mode: the target of image b = the lattice's fields on the box (FP32).
__global__ void k_target_image(FeatSrc F, int32_t L0, int32_t L1, int32_t L2, int b, int32_t lo0, int32_t lo1,
                               int32_t lo2, int32_t n0, int32_t n1, int32_t n2, float *__restrict__ tgt)
{
    const int64_t nb = (int64_t)n0 * n1 * n2;
    const int64_t img = (int64_t)b * L0 * L1 * L2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += gridDim.x * (int64_t)blockDim.x) {
        const int xx = lo0 + (int)(i % n0);
        const int64_t r = i / n0;
        const int yy = lo1 + (int)(r % n1), zz = lo2 + (int)(r / n1);
        const int64_t L = xx + (int64_t)L0 * (yy + (int64_t)L1 * zz);
        for (int s = 0; s < 3; ++s) tgt[(img + L) * 3 + s] = s < F.nspecies ? (float)F.field[s][L] : 0.0f;
    }
}

// Box coordinates (x, y, z) of a lattice voxel -> its element in the subgrid
// (-1 when its tile is not stored).
__device__ __forceinline__ int64_t elem_of(const BoxGeo &g, const int32_t *__restrict__ tile_index, int x, int y, int z)
{
    const int bx = x - g.lo[0], by = y - g.lo[1], bz = z - g.lo[2];
    const int32_t t = __ldg(tile_index + ((int64_t)(bz >> g.lt[2]) * g.nt[1] + (by >> g.lt[1])) * g.nt[0] + (bx >> g.lt[0]));
    if (t < 0) return -1;
    const int ix = bx & ((1 << g.lt[0]) - 1), iy = by & ((1 << g.lt[1]) - 1), iz = bz & ((1 << g.lt[2]) - 1);
    return ((int64_t)t << (g.lt[0] + g.lt[1] + g.lt[2])) + ix + ((int64_t)(iy + (iz << g.lt[1])) << g.lt[0]);
}

// Solver mode: features of the active voxels of every listed unit (B = 1, the
// lattice itself).  vin == null: c^n from the lattice (the guess); otherwise
// the field channel of species s carries v / m (v: compact vector of the
// subgrid, FP32 or FP64, at vin + (*vj) * vstride elements when vj is set --
// the Krylov vector whose index the solver keeps in device memory; m =
// *vscale), the other fields and the source map are zero (the
// preconditioner's homogeneous problem), and f32 receives the field channels.
struct FeatUnits {
    FeatSrc F;
    const uint8_t *lmask;
    const CnnDom *dom;
    const Unit *units;
    const int32_t *nunits;
    __nv_bfloat16 *x;
    float *f32;
    const void *vin;
    int32_t vin_f32;
    int64_t vstride;
    const int32_t *vj;
    const double *vscale;
    int s;
    const BoxGeo *geo;
    const int32_t *tile_index;
};

__global__ void k_feat_units(const __grid_constant__ FeatUnits A)
{
    const CnnDom &D = *A.dom;
    const int nu = *A.nunits;
    const double m = A.vin ? *A.vscale : 1.0;
    const int64_t voff = A.vin && A.vj ? (int64_t)*A.vj * A.vstride : 0;
    for (int ui = blockIdx.x; ui < nu; ui += gridDim.x) {
        const Unit u = A.units[ui];
        for (int i = threadIdx.x; i < tc::kSlabX * tc::kSlabY * u.nz; i += blockDim.x) {
            const int x = u.ox + (i & 7), y = u.oy + ((i >> 3) & 15), z = u.z0 + (i >> 7);
            if (!tc::in_box(D, 0, x, y, z)) continue;
            const int64_t L = tc::vox_index(D, 0, x, y, z);
            if (!A.lmask[L]) continue;
            float fld[3] = {0.0f, 0.0f, 0.0f};
            if (!A.vin) {
                for (int s = 0; s < 3; ++s) fld[s] = s < A.F.nspecies ? (float)A.F.field[s][L] : 0.0f;
            } else {
                if (m > 0.0) {
                    const int64_t e = elem_of(*A.geo, A.tile_index, x, y, z);
                    if (e >= 0) {
                        const double ve = A.vin_f32 ? (double)static_cast<const float *>(A.vin)[voff + e]
                                                    : static_cast<const double *>(A.vin)[voff + e];
                        fld[A.s] = (float)(ve / m);
                    }
                }
                for (int s = 0; s < 3; ++s) A.f32[L * 3 + s] = fld[s];
            }
            float f[kXC];
            features_of(A.F, L, fld, A.vin == nullptr, f);
            feat_store(A.x + L * kXC, f);
        }
    }
}

// ---------------------------------------------------------------- loss
__device__ __forceinline__ bool active_image_voxel(const CnnDom &D, const uint8_t *__restrict__ mask, int64_t v,
                                                   int64_t V)
{
    const int b = (int)(v / V);
    const int64_t r = v - (int64_t)b * V;
    const int x = (int)(r % D.L[0]), y = (int)((r / D.L[0]) % D.L[1]), z = (int)(r / ((int64_t)D.L[0] * D.L[1]));
    return tc::in_box(D, b, x, y, z) && mask[v];
}

__global__ void k_count_active(const __grid_constant__ CnnDom D, const uint8_t *__restrict__ mask,
                               unsigned long long *__restrict__ n)
{
    const int64_t V = (int64_t)D.L[0] * D.L[1] * D.L[2];
    unsigned c = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V * D.B; v += gridDim.x * (int64_t)blockDim.x)
        c += active_image_voxel(D, mask, v, V) ? 1u : 0u;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(n, (unsigned long long)c);
}

// Masked MSE over the active voxels and 3 species: loss and
// g6 = s_out * dLoss/dpred (bf16, 8 channels, 3..7 zero).
__global__ void k_loss(const __grid_constant__ CnnDom D, const uint8_t *__restrict__ mask, const float *__restrict__ pred,
                       const float *__restrict__ target, float s_out, const unsigned long long *__restrict__ nact,
                       __nv_bfloat16 *__restrict__ g6, double *__restrict__ loss)
{
    const double inv = *nact > 0 ? 1.0 / (3.0 * (double)*nact) : 0.0;
    const int64_t V = (int64_t)D.L[0] * D.L[1] * D.L[2];
    double part = 0.0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V * D.B; v += gridDim.x * (int64_t)blockDim.x) {
        if (!active_image_voxel(D, mask, v, V)) continue;
        __nv_bfloat16 out[kGC6];
#pragma unroll
        for (int c = 0; c < kGC6; ++c) out[c] = __float2bfloat16_rn(0.0f);
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const float d = pred[v * 3 + s] - target[v * 3 + s];
            part += (double)d * d * inv;
            out[s] = __float2bfloat16_rn((float)(s_out * 2.0 * d * inv));
        }
        uint4 u;
        memcpy(&u, out, 16);
        *reinterpret_cast<uint4 *>(g6 + v * kGC6) = u;
    }
    part = warp_sum(part);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, part);
}

// ---------------------------------------------------------------- preconditioner helpers
__global__ void k_pc_amax(const double *__restrict__ v, int64_t n, double *__restrict__ out)
{
    __shared__ double sh[32];
    double m = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(v[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmax(t, sh[i]);
        *out = t;
    }
}

// z[e] = m * pred[s] on the in-mask stored elements of the listed units
// (pred = v / m + s_out z6 from the network's image-mode output).
struct PcOut {
    const CnnDom *dom;
    const Unit *units;
    const int32_t *nunits;
    const uint8_t *lmask;
    const float *pred;            // [V][3] lattice-indexed
    const BoxGeo *geo;
    const int32_t *tile_index;
    const double *vscale;
    int s;
    void *z;                      // FP32 (z_f32) or FP64 compact vector
    int32_t z_f32;
};

__global__ void k_pc_scatter(const __grid_constant__ PcOut P)
{
    const CnnDom &D = *P.dom;
    const int nu = *P.nunits;
    const double m = *P.vscale;
    if (!(m > 0.0)) return;
    for (int ui = blockIdx.x; ui < nu; ui += gridDim.x) {
        const Unit u = P.units[ui];
        for (int i = threadIdx.x; i < tc::kSlabX * tc::kSlabY * u.nz; i += blockDim.x) {
            const int x = u.ox + (i & 7), y = u.oy + ((i >> 3) & 15), z = u.z0 + (i >> 7);
            if (!tc::in_box(D, 0, x, y, z)) continue;
            const int64_t L = tc::vox_index(D, 0, x, y, z);
            if (!P.lmask[L]) continue;
            const int64_t e = elem_of(*P.geo, P.tile_index, x, y, z);
            if (e >= 0) {
                const double z = m * (double)P.pred[L * 3 + P.s];
                if (P.z_f32) static_cast<float *>(P.z)[e] = (float)z;
                else static_cast<double *>(P.z)[e] = z;
            }
        }
    }
}

}  // namespace mpm

using namespace mpm;

struct mpm_cnn {
    uint64_t serial = 0;             // distinct for every network of the process (graph caches)
    cudaEvent_t lev[kLayers + 1] = {};   // around the convolutions (MPM_DEBUG_CNN_LAYER_TIMES)
    bool lev_recorded = false;
    int32_t L[3] = {0, 0, 0};
    int32_t maxB = 0;
    long long V = 0;                 // voxels per image
    bool train = false;
    long long nparams = 0;
    long long off[kLayers] = {};
    float *master = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    unsigned char *wf[kLayers] = {}, *wd[kLayers] = {};
    float *bias[kLayers] = {};
    __nv_bfloat16 *x = nullptr;      // [B V][16]
    uint8_t *mask = nullptr;         // [B V] (image mode)
    float *f32 = nullptr;            // [B V][3] c^n (image mode) / field channels (preconditioner)
    float *target = nullptr;         // [B V][3]
    float *pred = nullptr;           // [B V][3]
    __nv_bfloat16 *a[kLayers - 1] = {};   // activations (inference: a[0], a[1] ping-pong)
    float *z[kLayers - 1] = {};      // pre-activations (training)
    __nv_bfloat16 *g = nullptr, *g2 = nullptr, *g6 = nullptr;
    float *partials = nullptr;
    CnnDom *dom = nullptr;
    Unit *units = nullptr;
    uint8_t *uact = nullptr;         // [units][kActStride] activity bytes of each listed unit
    uint32_t *ubits = nullptr;       // [units] its active slabs
    long long max_units = 0;
    uint8_t *flags = nullptr;
    int32_t *counters = nullptr;     // [0] listed units, [1..15] work counters
    BoxGeo *geo = nullptr;           // host-known box (guess, preconditioner)
    unsigned long long *nact = nullptr;
    double *loss = nullptr;
    int32_t *h_err = nullptr, *d_err = nullptr;   // host-mapped: a bounded wait gave up
    CnnDom hdom;                     // image boxes as loaded
    int step = 0;
    float s_out = 0.01f;
    std::vector<void *> allocs;
};

namespace {

mpm_status cnn_alloc(mpm_ctx *ctx, mpm_cnn *c, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return mpm_fail(ctx, MPM_ERR_NOMEM, "cnn: device allocation failed");
    }
    c->allocs.push_back(*p);
    return MPM_OK;
}

// One forward / input-gradient convolution over the listed units; `slot` is
// its work counter.
// The dynamic shared-memory size of a convolution instance, set once per
// process (outside any stream capture: mpm_cnn_create sets the forward ones).
template <int CI, int NO, int EPI>
mpm_status conv_attr(mpm_ctx *ctx)
{
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(tc::k_conv_tc<CI, NO, EPI>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)tc::ConvSmem<CI, NO>::BYTES);
        if (e != cudaSuccess) return mpm_cuda_check(ctx, e, "cnn convolution: shared-memory attribute");
        attr = true;
    }
    return MPM_OK;
}

template <int CI, int NO, int EPI>
mpm_status conv(mpm_ctx *ctx, mpm_cnn *c, tc::ConvArgs A, int slot, cudaStream_t st)
{
    constexpr int smem = tc::ConvSmem<CI, NO>::BYTES;
    const mpm_status ra = conv_attr<CI, NO, EPI>(ctx);
    if (ra != MPM_OK) return ra;
    A.dom = c->dom;
    A.units = c->units;
    A.nunits = c->counters;
    A.uact = c->uact;
    A.ubits = c->ubits;
    A.work = c->counters + slot;
    A.done = c->counters + 16 + slot;
    A.err = c->d_err;
    A.timeout_ns = ctx->timeout_ns;
    // programmatic dependent launch: the next layer's CTAs start their
    // prologue (weights into shared memory, TMEM) on the SMs this launch has
    // left, and wait (griddepcontrol.wait) for it to complete before reading
    // its output
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctx->num_sms);
    cfg.blockDim = dim3((unsigned)tc::kConvThreads);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, tc::k_conv_tc<CI, NO, EPI>, A);
    ctx->launches += 1;
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFuncAttributes fa;
        memset(&fa, 0, sizeof(fa));
        cudaFuncGetAttributes(&fa, tc::k_conv_tc<CI, NO, EPI>);
        char msg[256];
        snprintf(msg, sizeof(msg), "cnn convolution (%d threads, %d B shared; kernel: max %d threads, %d registers, "
                 "%zu B static shared, %d B dynamic allowed)", tc::kConvThreads, smem, fa.maxThreadsPerBlock,
                 fa.numRegs, fa.sharedSizeBytes, fa.maxDynamicSharedSizeBytes);
        return mpm_cuda_check(ctx, e, msg);
    }
    return MPM_OK;
}

template <int CI, int NO>
mpm_status wgrad(mpm_ctx *ctx, mpm_cnn *c, const __nv_bfloat16 *in, const __nv_bfloat16 *g, int gc, int l,
                 cudaStream_t st)
{
    static bool attr = false;
    constexpr int smem = tc::WgSmem<CI, NO>::BYTES;
    if (!attr) {
        cudaFuncSetAttribute(tc::k_wgrad_tc<CI, NO>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr = true;
    }
    tc::WgradArgs A;
    memset(&A, 0, sizeof(A));
    A.in = in;
    A.g = g;
    A.gc = gc;
    A.mask = c->mask;
    A.dom = c->dom;
    A.units = c->units;
    A.nunits = c->counters;
    A.uact = c->uact;
    A.ubits = c->ubits;
    A.partials = c->partials;
    A.err = c->d_err;
    A.timeout_ns = ctx->timeout_ns;
    tc::k_wgrad_tc<CI, NO><<<ctx->num_sms, tc::kThreads, smem, st>>>(A);
    k_wgrad_reduce<<<64, 256, 0, st>>>(c->partials, ctx->num_sms, CI, NO, chan(l), chan(l + 1), c->grads + c->off[l]);
    ctx->launches += 2;
    return mpm_cuda_check(ctx, cudaGetLastError(), "cnn weight gradient");
}

mpm_status prep(mpm_ctx *ctx, mpm_cnn *c, cudaStream_t st)
{
    PrepArgs P;
    memset(&P, 0, sizeof(P));
    P.master = c->master;
    for (int l = 0; l < kLayers; ++l) {
        P.off[l] = c->off[l];
        P.wf[l] = c->wf[l];
        P.wd[l] = c->wd[l];
        P.bias[l] = c->bias[l];
    }
    k_prep_weights<<<dim3(32, kLayers), 256, 0, st>>>(P);
    ctx->launches += 1;
    return mpm_cuda_check(ctx, cudaGetLastError(), "cnn weight preparation");
}

mpm_status check_err(mpm_ctx *ctx, mpm_cnn *c)
{
    if (*(volatile int32_t *)c->h_err) {
        *(volatile int32_t *)c->h_err = 0;
        return mpm_fail(ctx, MPM_ERR_TIMEOUT, "cnn: a bounded wait in a convolution kernel gave up");
    }
    return MPM_OK;
}

// The listed units' activity bytes and slab masks (once per application,
// for all six layers and the backward pass).
mpm_status unit_act(mpm_ctx *ctx, mpm_cnn *c, const uint8_t *mask, cudaStream_t st)
{
    tc::k_unit_act<<<ctx->num_sms * 4, 256, 0, st>>>(c->dom, mask, c->units, c->counters, c->uact, c->ubits);
    ctx->launches += 1;
    return mpm_cuda_check(ctx, cudaGetLastError(), "cnn unit activity");
}

// Image mode plan over images 0..nimg-1 (their boxes as loaded).
mpm_status plan_images(mpm_ctx *ctx, mpm_cnn *c, int nimg, cudaStream_t st)
{
    CnnDom D = c->hdom;
    D.B = nimg;
    const long long ncand = (long long)nimg * ((c->L[0] + 7) / 8) * ((c->L[1] + 15) / 16) * ((c->L[2] + 7) / 8);
    MPM_CU(cudaMemsetAsync(c->counters, 0, 16 * sizeof(int32_t), st));
    k_plan_flags<<<ctx->num_sms * 4, 256, 0, st>>>(D, c->mask, ncand, c->flags);
    k_plan_compact<<<1, 1024, 0, st>>>(D, c->flags, ncand, c->units, c->counters, c->dom);
    ctx->launches += 2;
    MPM_CU(cudaGetLastError());
    return unit_act(ctx, c, c->mask, st);
}

// The six layers.  Inference (train = false): activations ping-pong in a[0],
// a[1]; training: a[l] and z[l] kept for the backward pass.  The last layer's
// output is described by out_args (image mode: pred / f32; solver mode: the
// iterate).
mpm_status forward_layers(mpm_ctx *ctx, mpm_cnn *c, const uint8_t *mask, bool train, const tc::ConvArgs &out_args,
                          cudaStream_t st)
{
    bool timed = false;
    if (ctx->cnn_layer_prof) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        timed = cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
        for (int i = 0; i <= kLayers && timed; ++i)
            if (!c->lev[i]) timed = cudaEventCreate(&c->lev[i]) == cudaSuccess;
        cudaGetLastError();
        if (timed) MPM_CU(cudaEventRecord(c->lev[0], st));
    }
    for (int l = 0; l < kLayers; ++l) {
        tc::ConvArgs A;
        memset(&A, 0, sizeof(A));
        A.mask = mask;
        A.in = l == 0 ? c->x : (train ? c->a[l - 1] : c->a[(l - 1) & 1]);
        A.wimg = c->wf[l];
        A.bias = c->bias[l];
        mpm_status r;
        if (l < kLayers - 1) {
            A.a_out = train ? c->a[l] : c->a[l & 1];
            A.z_out = train ? c->z[l] : nullptr;
            r = l == 0 ? conv<kXC, 32, tc::EPI_GELU>(ctx, c, A, 1 + l, st)
                       : conv<kHC, 32, tc::EPI_GELU>(ctx, c, A, 1 + l, st);
        } else {
            tc::ConvArgs O = out_args;
            O.mask = mask;
            O.in = A.in;
            O.wimg = A.wimg;
            O.bias = A.bias;
            O.s_out = c->s_out;
            r = conv<kHC, 16, tc::EPI_OUT>(ctx, c, O, 1 + l, st);
        }
        if (r != MPM_OK) return r;
        if (timed) MPM_CU(cudaEventRecord(c->lev[l + 1], st));
    }
    if (timed) c->lev_recorded = true;
    return MPM_OK;
}

FeatSrc feat_src(const mpm_lattice *lat, const mpm_params *prm)
{
    FeatSrc F;
    memset(&F, 0, sizeof(F));
    F.cell = lat->cell_id;
    F.nspecies = prm->nspecies;
    for (int s = 0; s < prm->nspecies && s < kMaxSpecies; ++s) F.field[s] = lat->field[s];
    F.ncell = prm->ncell;
    F.k_cell = prm->k_cell;
    F.q_cell = prm->q_cell;
    return F;
}

mpm_status solver_mode_check(mpm_ctx *ctx, mpm_cnn *c, const mpm_subgrid *sub, const mpm_lattice *lat,
                             const mpm_params *prm, const char *who)
{
    if (!c || !sub || !lat || !prm) return mpm_fail(ctx, MPM_ERR_ARG, std::string(who) + ": null argument");
    if (!sub->extracted) return mpm_fail(ctx, MPM_ERR_ARG, std::string(who) + ": subgrid not extracted");
    for (int d = 0; d < 3; ++d)
        if (lat->dims[d] != c->L[d])
            return mpm_fail(ctx, MPM_ERR_ARG, std::string(who) + ": lattice dims differ from the network's image dims");
    if (sub->nspecies > 3) return mpm_fail(ctx, MPM_ERR_ARG, std::string(who) + ": the network predicts 3 species");
    return MPM_OK;
}

}  // namespace

// ---------------------------------------------------------------- C ABI
extern "C" mpm_status mpm_cnn_create(mpm_ctx *ctx, mpm_cnn **out, const int32_t image_dims[3], int32_t max_images,
                                     int32_t train)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    if (!out || !image_dims || max_images < 1 || max_images > tc::kMaxImages || (train != 0 && train != 1))
        return mpm_fail(ctx, MPM_ERR_ARG, "cnn_create: bad argument");
    for (int d = 0; d < 3; ++d)
        if (image_dims[d] < 1) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_create: bad image dims");
    const long long V = (long long)image_dims[0] * image_dims[1] * image_dims[2];
    if (V * max_images >= (1LL << 31)) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_create: more than 2^31 voxels");
    static std::atomic<uint64_t> serials{0};
    mpm_cnn *c = new mpm_cnn();
    c->serial = ++serials;
    for (int d = 0; d < 3; ++d) c->L[d] = image_dims[d];
    c->maxB = max_images;
    c->V = V;
    c->train = train != 0;
    memset(&c->hdom, 0, sizeof(c->hdom));
    for (int d = 0; d < 3; ++d) c->hdom.L[d] = image_dims[d];
    long long n = 0;
    for (int l = 0; l < kLayers; ++l) {
        c->off[l] = n;
        n += 27LL * chan(l) * chan(l + 1) + chan(l + 1);
    }
    c->nparams = n;
    const size_t VT = (size_t)V * max_images;
    // a band of 8 columns by 8 depths holds at most ceil(n_y / 16) units, on
    // the fixed grid (image mode) and placed along y (solver mode) alike
    c->max_units = (long long)max_images * ((image_dims[0] + 7) / 8) * ((image_dims[1] + 15) / 16) *
                   ((image_dims[2] + 7) / 8);
    mpm_status r = MPM_OK;
    auto A = [&](void **p, size_t b) {
        if (r == MPM_OK) r = cnn_alloc(ctx, c, p, b);
    };
    A((void **)&c->master, n * 4);
    A((void **)&c->grads, n * 4);
    A((void **)&c->m, n * 4);
    A((void **)&c->v, n * 4);
    for (int l = 0; l < kLayers; ++l) {
        A((void **)&c->wf[l], wimg_bytes(fwd_ci(l), fwd_no(l)));
        if (l > 0) A((void **)&c->wd[l], wimg_bytes(dg_ci(l), 32));
        A((void **)&c->bias[l], 32 * 4);
    }
    A((void **)&c->x, VT * kXC * 2);
    A((void **)&c->mask, VT);
    A((void **)&c->f32, VT * 3 * 4);
    A((void **)&c->pred, VT * 3 * 4);
    for (int l = 0; l < (c->train ? kLayers - 1 : 2); ++l) A((void **)&c->a[l], VT * kHC * 2);
    if (c->train) {
        for (int l = 0; l < kLayers - 1; ++l) A((void **)&c->z[l], VT * kHC * 4);
        A((void **)&c->target, VT * 3 * 4);
        A((void **)&c->g, VT * kHC * 2);
        A((void **)&c->g2, VT * kHC * 2);
        A((void **)&c->g6, VT * kGC6 * 2);
        A((void **)&c->partials, (size_t)ctx->num_sms * 9 * 128 * 32 * 4);
    }
    A((void **)&c->dom, sizeof(CnnDom));
    A((void **)&c->units, (size_t)c->max_units * sizeof(Unit));
    A((void **)&c->uact, (size_t)c->max_units * tc::kActStride);
    A((void **)&c->ubits, (size_t)c->max_units * sizeof(uint32_t));
    A((void **)&c->flags, (size_t)c->max_units);
    A((void **)&c->counters, 64 * sizeof(int32_t));
    A((void **)&c->geo, 256);
    A((void **)&c->nact, 256);
    A((void **)&c->loss, 256);
    if (r == MPM_OK) {
        if (cudaHostAlloc((void **)&c->h_err, 64, cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer((void **)&c->d_err, c->h_err, 0) != cudaSuccess) {
            cudaGetLastError();
            r = mpm_fail(ctx, MPM_ERR_NOMEM, "cnn: host-mapped allocation failed");
        } else {
            *c->h_err = 0;
        }
    }
    if (r == MPM_OK) {
        cudaMemset(c->m, 0, n * 4);
        cudaMemset(c->v, 0, n * 4);
        cudaMemset(c->mask, 0, VT);
        cudaMemset(c->counters, 0, 64 * sizeof(int32_t));
        if (cudaDeviceSynchronize() != cudaSuccess) r = mpm_cuda_check(ctx, cudaGetLastError(), "cnn_create");
    }
    // the forward convolutions run inside captured graphs (learned step,
    // flexible GMRES): their attributes are set here, outside any capture
    if (r == MPM_OK) r = conv_attr<kXC, 32, tc::EPI_GELU>(ctx);
    if (r == MPM_OK) r = conv_attr<kHC, 32, tc::EPI_GELU>(ctx);
    if (r == MPM_OK) r = conv_attr<kHC, 16, tc::EPI_OUT>(ctx);
    if (r != MPM_OK) {
        mpm_cnn_destroy(ctx, c);
        return r;
    }
    *out = c;
    return MPM_OK;
}

extern "C" mpm_status mpm_cnn_layer_times(mpm_ctx *ctx, mpm_cnn *c, float ms[6])
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    if (!c || !ms) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_layer_times: null argument");
    if (!c->lev_recorded) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_layer_times: no timed application");
    MPM_CU(cudaEventSynchronize(c->lev[kLayers]));
    for (int l = 0; l < kLayers; ++l) MPM_CU(cudaEventElapsedTime(&ms[l], c->lev[l], c->lev[l + 1]));
    return MPM_OK;
}

extern "C" mpm_status mpm_cnn_destroy(mpm_ctx *ctx, mpm_cnn *c)
{
    (void)ctx;
    if (!c) return MPM_ERR_ARG;
    for (int i = 0; i <= kLayers; ++i)
        if (c->lev[i]) cudaEventDestroy(c->lev[i]);
    for (void *p : c->allocs) cudaFree(p);
    if (c->h_err) cudaFreeHost(c->h_err);
    delete c;
    return MPM_OK;
}

extern "C" mpm_status mpm_cnn_set_params(mpm_ctx *ctx, mpm_cnn *c, const float *host_params, int64_t n, float s_out,
                                         void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    if (!c || !host_params || n != c->nparams) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_set_params: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    MPM_CU(cudaMemcpyAsync(c->master, host_params, n * 4, cudaMemcpyHostToDevice, st));
    MPM_CU(cudaMemsetAsync(c->m, 0, n * 4, st));
    MPM_CU(cudaMemsetAsync(c->v, 0, n * 4, st));
    MPM_CU(cudaStreamSynchronize(st));
    c->step = 0;
    c->s_out = s_out;
    return prep(ctx, c, st);
}

extern "C" mpm_status mpm_cnn_get_params(mpm_ctx *ctx, const mpm_cnn *c, int32_t which, float *host_out, int64_t n,
                                         void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    if (!c || !host_out || n != c->nparams || which < 0 || which > 1 || (which == 1 && !c->train))
        return mpm_fail(ctx, MPM_ERR_ARG, "cnn_get_params: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    MPM_CU(cudaMemcpyAsync(host_out, which == 1 ? c->grads : c->master, n * 4, cudaMemcpyDeviceToHost, st));
    MPM_CU(cudaStreamSynchronize(st));
    return MPM_OK;
}

extern "C" mpm_status mpm_cnn_load_image(mpm_ctx *ctx, mpm_cnn *c, int32_t b, const mpm_lattice *lat,
                                         const mpm_params *prm, const mpm_box *box, int32_t what, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    if (!c || !lat || !prm || !box || b < 0 || b >= c->maxB)
        return mpm_fail(ctx, MPM_ERR_ARG, "cnn_load_image: bad argument");
    if (what != MPM_CNN_INPUT && what != MPM_CNN_TARGET) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_load_image: bad `what`");
    if (what == MPM_CNN_TARGET && !c->train) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_load_image: not a training network");
    for (int d = 0; d < 3; ++d) {
        if (lat->dims[d] != c->L[d])
            return mpm_fail(ctx, MPM_ERR_ARG, "cnn_load_image: lattice dims differ from the image dims");
        if (box->lo[d] < 0 || box->hi[d] > lat->dims[d] || box->hi[d] <= box->lo[d])
            return mpm_fail(ctx, MPM_ERR_ARG, "cnn_load_image: bad box");
    }
    if (!lat->cell_id || !lat->mask || prm->nspecies < 1 || prm->ncell < 1 || !prm->k_cell || !prm->q_cell)
        return mpm_fail(ctx, MPM_ERR_ARG, "cnn_load_image: null lattice array or rate table");
    for (int s = 0; s < prm->nspecies && s < 3; ++s)
        if (!lat->field[s]) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_load_image: null field");
    cudaStream_t st = (cudaStream_t)stream;
    const FeatSrc F = feat_src(lat, prm);
    const int n0 = box->hi[0] - box->lo[0], n1 = box->hi[1] - box->lo[1], n2 = box->hi[2] - box->lo[2];
    if (what == MPM_CNN_INPUT) {
        for (int d = 0; d < 3; ++d) {
            c->hdom.lo[b][d] = box->lo[d];
            c->hdom.n[b][d] = box->hi[d] - box->lo[d];
        }
        k_feat_image<<<ctx->num_sms * 4, 256, 0, st>>>(F, lat->mask, c->L[0], c->L[1], c->L[2], b, box->lo[0],
                                                        box->lo[1], box->lo[2], n0, n1, n2, c->mask, c->x, c->f32);
    } else {
        k_target_image<<<ctx->num_sms * 4, 256, 0, st>>>(F, c->L[0], c->L[1], c->L[2], b, box->lo[0], box->lo[1],
                                                          box->lo[2], n0, n1, n2, c->target);
    }
    ctx->launches += 1;
    return mpm_cuda_check(ctx, cudaGetLastError(), "cnn_load_image");
}

extern "C" mpm_status mpm_cnn_export_features(mpm_ctx *ctx, const mpm_cnn *c, int32_t nimg, void *x_bf16,
                                              uint8_t *mask, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    if (!c || nimg < 1 || nimg > c->maxB || !x_bf16 || !mask)
        return mpm_fail(ctx, MPM_ERR_ARG, "cnn_export_features: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)c->V * nimg;
    MPM_CU(cudaMemcpyAsync(x_bf16, c->x, n * kXC * 2, cudaMemcpyDeviceToDevice, st));
    MPM_CU(cudaMemcpyAsync(mask, c->mask, n, cudaMemcpyDeviceToDevice, st));
    return MPM_OK;
}

extern "C" mpm_status mpm_cnn_export_preact(mpm_ctx *ctx, const mpm_cnn *c, int32_t layer, int32_t nimg, float *dst,
                                            void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    if (!c || !c->train || layer < 1 || layer > kLayers - 1 || nimg < 1 || nimg > c->maxB || !dst)
        return mpm_fail(ctx, MPM_ERR_ARG, "cnn_export_preact: bad argument");
    MPM_CU(cudaMemcpyAsync(dst, c->z[layer - 1], (size_t)c->V * nimg * kHC * 4, cudaMemcpyDeviceToDevice,
                           (cudaStream_t)stream));
    return MPM_OK;
}

extern "C" mpm_status mpm_cnn_forward(mpm_ctx *ctx, mpm_cnn *c, int32_t nimg, float *pred, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    if (!c || nimg < 1 || nimg > c->maxB) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_forward: bad argument");
    mpm_status r = check_err(ctx, c);
    if (r != MPM_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    r = plan_images(ctx, c, nimg, st);
    if (r != MPM_OK) return r;
    tc::ConvArgs O;
    memset(&O, 0, sizeof(O));
    O.f32 = c->f32;
    O.pred = pred ? pred : c->pred;
    return forward_layers(ctx, c, c->mask, false, O, st);
}

extern "C" mpm_status mpm_cnn_train_step(mpm_ctx *ctx, mpm_cnn *c, int32_t nimg, float lr, int32_t apply,
                                         double *loss_out, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    if (!c || !c->train || nimg < 1 || nimg > c->maxB || (apply != 0 && apply != 1))
        return mpm_fail(ctx, MPM_ERR_ARG, "cnn_train_step: bad argument");
    mpm_status r = check_err(ctx, c);
    if (r != MPM_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    r = plan_images(ctx, c, nimg, st);
    if (r != MPM_OK) return r;
    tc::ConvArgs O;
    memset(&O, 0, sizeof(O));
    O.f32 = c->f32;
    O.pred = c->pred;
    r = forward_layers(ctx, c, c->mask, true, O, st);
    if (r != MPM_OK) return r;
    CnnDom D = c->hdom;
    D.B = nimg;
    MPM_CU(cudaMemsetAsync(c->nact, 0, 8, st));
    MPM_CU(cudaMemsetAsync(c->loss, 0, 8, st));
    k_count_active<<<ctx->num_sms * 4, 256, 0, st>>>(D, c->mask, c->nact);
    k_loss<<<ctx->num_sms * 4, 256, 0, st>>>(D, c->mask, c->pred, c->target, c->s_out, c->nact, c->g6, c->loss);
    ctx->launches += 2;
    MPM_CU(cudaGetLastError());
    // backward: each layer's weight gradient from its input and dLoss/dz of
    // its output, then dLoss/dz of the layer below through the input gradient
    __nv_bfloat16 *g = c->g, *gn = c->g2;
    for (int l = kLayers - 1; l >= 0; --l) {
        const __nv_bfloat16 *in = l == 0 ? c->x : c->a[l - 1];
        const __nv_bfloat16 *gl = l == kLayers - 1 ? c->g6 : g;
        if (l == kLayers - 1) r = wgrad<kHC, 16>(ctx, c, in, gl, kGC6, l, st);
        else if (l == 0) r = wgrad<kXC, 32>(ctx, c, in, gl, kHC, l, st);
        else r = wgrad<kHC, 32>(ctx, c, in, gl, kHC, l, st);
        if (r != MPM_OK) return r;
        if (l == 0) break;
        tc::ConvArgs A;
        memset(&A, 0, sizeof(A));
        A.mask = c->mask;
        A.in = gl;
        A.wimg = c->wd[l];
        A.zprev = c->z[l - 1];
        __nv_bfloat16 *dst = l == kLayers - 1 ? g : gn;
        A.g_out = dst;
        const int slot = 7 + (kLayers - 1 - l);
        r = l == kLayers - 1 ? conv<kGC6, 32, tc::EPI_DGRAD>(ctx, c, A, slot, st)
                             : conv<kHC, 32, tc::EPI_DGRAD>(ctx, c, A, slot, st);
        if (r != MPM_OK) return r;
        if (l != kLayers - 1) {
            __nv_bfloat16 *t = g;
            g = gn;
            gn = t;
        }
    }
    if (apply) {
        c->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.0f - powf(b1, (float)c->step), c2 = 1.0f - powf(b2, (float)c->step);
        k_adam<<<ctx->num_sms, 256, 0, st>>>(c->master, c->grads, c->m, c->v, c->nparams, lr, b1, b2, 1e-8f, c1, c2);
        ctx->launches += 1;
        MPM_CU(cudaGetLastError());
        r = prep(ctx, c, st);
        if (r != MPM_OK) return r;
    }
    if (loss_out) {
        MPM_CU(cudaMemcpyAsync(ctx->h_stage, c->loss, 8, cudaMemcpyDeviceToHost, st));
        MPM_CU(cudaStreamSynchronize(st));
        *loss_out = *(double *)ctx->h_stage;
        return check_err(ctx, c);
    }
    return MPM_OK;
}

// The guess of a subgrid's solve with its box in device memory (d_geo): plan
// from the subgrid's tile activity, features from the lattice's c^n, the
// network, and the prediction into the iterate of every species on the
// in-mask stored elements.  Stream work only (graph-capturable).
mpm_status mpm_cnn_enqueue_guess(mpm_ctx *ctx, mpm_cnn *c, mpm_subgrid *sub, const mpm_lattice *lat,
                                 const mpm_params *prm, const BoxGeo *d_geo, cudaStream_t st)
{
    MPM_CU(cudaMemsetAsync(c->counters, 0, 16 * sizeof(int32_t), st));
    k_plan_box<<<ctx->num_sms, 256, 0, st>>>(d_geo, sub->tile_index, lat->dims[0], lat->dims[1], lat->dims[2], c->units,
                                             c->counters, c->max_units, c->dom, c->d_err);
    ctx->launches += 1;
    mpm_status ra = unit_act(ctx, c, lat->mask, st);
    if (ra != MPM_OK) return ra;
    FeatUnits FU;
    memset(&FU, 0, sizeof(FU));
    FU.F = feat_src(lat, prm);
    FU.lmask = lat->mask;
    FU.dom = c->dom;
    FU.units = c->units;
    FU.nunits = c->counters;
    FU.x = c->x;
    k_feat_units<<<ctx->num_sms * 8, 256, 0, st>>>(FU);
    ctx->launches += 1;
    MPM_CU(cudaGetLastError());
    tc::ConvArgs O;
    memset(&O, 0, sizeof(O));
    for (int s = 0; s < 3 && s < prm->nspecies; ++s) {
        O.field[s] = lat->field[s];
        O.xs[s] = sub->x[s];
    }
    O.nspecies = prm->nspecies < 3 ? prm->nspecies : 3;
    O.tile_index = sub->tile_index;
    O.geo = d_geo;
    return forward_layers(ctx, c, lat->mask, false, O, st);
}

// A network used by a device-resident step: its image dims must be the
// lattice's, and it predicts 3 species at most.
mpm_status mpm_cnn_check(mpm_ctx *ctx, mpm_cnn *c, const mpm_lattice *lat, const mpm_params *prm)
{
    for (int d = 0; d < 3; ++d)
        if (lat->dims[d] != c->L[d])
            return mpm_fail(ctx, MPM_ERR_ARG, "learned step: lattice dims differ from the network's image dims");
    if (prm->nspecies > 3) return mpm_fail(ctx, MPM_ERR_ARG, "learned step: the network predicts 3 species");
    return check_err(ctx, c);
}

extern "C" mpm_status mpm_cnn_guess(mpm_ctx *ctx, mpm_cnn *c, mpm_subgrid *sub, const mpm_lattice *lat,
                                    const mpm_params *prm, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    mpm_status r = solver_mode_check(ctx, c, sub, lat, prm, "cnn_guess");
    if (r != MPM_OK) return r;
    r = check_err(ctx, c);
    if (r != MPM_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const BoxGeo g = make_geo(sub, lat->dims);
    MPM_CU(cudaMemcpyAsync(c->geo, &g, sizeof(g), cudaMemcpyHostToDevice, st));
    r = mpm_cnn_enqueue_guess(ctx, c, sub, lat, prm, c->geo, st);
    if (r != MPM_OK) return r;
    sub->x_fresh = false;
    return MPM_OK;
}

// ---------------------------------------------------------------- the network as a preconditioner
// Row a13: flexible GMRES applies z = m * net(v / m) to a Krylov vector v of
// one species (m = max |v|, which puts v in the range the network was trained
// on), with the other fields and the source map at zero (the homogeneous
// problem), and keeps z on the in-mask voxels only.
//
// The plan (box geometry, listed units, per-unit activity) depends on the
// subgrid alone: mpm_cnn_pc_plan computes it once per solve and keeps the
// unit count twice, in counters[0] (read by every network kernel) and in
// counters[kUnitsSaved] (from which a solver restores it: a solver that has
// abandoned the network sets counters[0] = 0, and every network kernel then
// has nothing to do).  Stream work only.
constexpr int kUnitsSaved = 32;

mpm_status mpm_cnn_pc_plan(mpm_ctx *ctx, mpm_cnn *c, mpm_subgrid *sub, const mpm_lattice *lat, const mpm_params *prm,
                           cudaStream_t st, int32_t **units_out)
{
    mpm_status r = solver_mode_check(ctx, c, sub, lat, prm, "cnn_precond");
    if (r != MPM_OK) return r;
    r = check_err(ctx, c);
    if (r != MPM_OK) return r;
    const BoxGeo g = make_geo(sub, lat->dims);
    MPM_CU(cudaMemcpyAsync(c->geo, &g, sizeof(g), cudaMemcpyHostToDevice, st));
    MPM_CU(cudaMemsetAsync(c->counters, 0, 16 * sizeof(int32_t), st));
    k_plan_box<<<ctx->num_sms, 256, 0, st>>>(c->geo, sub->tile_index, lat->dims[0], lat->dims[1], lat->dims[2], c->units,
                                             c->counters, c->max_units, c->dom, c->d_err);
    ctx->launches += 1;
    r = unit_act(ctx, c, lat->mask, st);
    if (r != MPM_OK) return r;
    MPM_CU(cudaMemcpyAsync(c->counters + kUnitsSaved, c->counters, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    if (units_out) *units_out = c->counters;
    return MPM_OK;
}

// z = m * net(v / m)[s] on the in-mask stored elements of the planned units
// (elements elsewhere untouched).  v at v + (*vj) * vstride elements (vj null:
// at v), FP32 or FP64 (f32); m = *vscale (device); z of the same type.  Kernel
// launches only (capturable into a graph body).
mpm_status mpm_cnn_pc_apply(mpm_ctx *ctx, mpm_cnn *c, mpm_subgrid *sub, const mpm_lattice *lat,
                            const mpm_params *prm, int s, const void *v, bool f32, int64_t vstride,
                            const int32_t *vj, const double *vscale, void *z, cudaStream_t st)
{
    FeatUnits FU;
    memset(&FU, 0, sizeof(FU));
    FU.F = feat_src(lat, prm);
    FU.lmask = lat->mask;
    FU.dom = c->dom;
    FU.units = c->units;
    FU.nunits = c->counters;
    FU.x = c->x;
    FU.f32 = c->f32;
    FU.vin = v;
    FU.vin_f32 = f32 ? 1 : 0;
    FU.vstride = vstride;
    FU.vj = vj;
    FU.vscale = vscale;
    FU.s = s;
    FU.geo = c->geo;
    FU.tile_index = sub->tile_index;
    k_feat_units<<<ctx->num_sms * 8, 256, 0, st>>>(FU);
    ctx->launches += 1;
    MPM_CU(cudaGetLastError());
    // image-mode output (pred = field channels + s_out z6) on the lattice-indexed buffer
    tc::ConvArgs O;
    memset(&O, 0, sizeof(O));
    O.pred = c->pred;
    O.f32 = c->f32;
    mpm_status r = forward_layers(ctx, c, lat->mask, false, O, st);
    if (r != MPM_OK) return r;
    PcOut P;
    P.dom = c->dom;
    P.units = c->units;
    P.nunits = c->counters;
    P.lmask = lat->mask;
    P.pred = c->pred;
    P.geo = c->geo;
    P.tile_index = sub->tile_index;
    P.vscale = vscale;
    P.s = s;
    P.z = z;
    P.z_f32 = f32 ? 1 : 0;
    k_pc_scatter<<<ctx->num_sms * 8, 256, 0, st>>>(P);
    ctx->launches += 1;
    return mpm_cuda_check(ctx, cudaGetLastError(), "cnn preconditioner output");
}

uint64_t mpm_cnn_serial(const mpm_cnn *c) { return c->serial; }

// Kernels one mpm_cnn_pc_apply launches.
int mpm_cnn_pc_launches() { return 2 + kLayers; }

mpm_status mpm_cnn_check_err(mpm_ctx *ctx, mpm_cnn *c) { return check_err(ctx, c); }

// One application on compact FP64 vectors (z = 0 off the mask); d_scale: one
// device double of scratch.  Stream work only.
mpm_status mpm_cnn_precond_impl(mpm_ctx *ctx, mpm_cnn *c, mpm_subgrid *sub, const mpm_lattice *lat,
                                const mpm_params *prm, int s, const double *v, double *z, double *d_scale,
                                cudaStream_t st)
{
    if (s < 0 || s > 2) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_precond: the network covers species 0..2");
    MPM_CU(cudaMemsetAsync(z, 0, (size_t)(sub->NE > 0 ? sub->NE : 1) * sizeof(double), st));
    if (sub->NE == 0) return MPM_OK;
    mpm_status r = mpm_cnn_pc_plan(ctx, c, sub, lat, prm, st, nullptr);
    if (r != MPM_OK) return r;
    k_pc_amax<<<1, 1024, 0, st>>>(v, sub->NE, d_scale);
    ctx->launches += 1;
    return mpm_cnn_pc_apply(ctx, c, sub, lat, prm, s, v, false, 0, nullptr, d_scale, z, st);
}

mpm_status mpm_dense_to_elems(mpm_ctx *ctx, const mpm_subgrid *sub, const double *src, double *dst, cudaStream_t st);
mpm_status mpm_elems_to_dense(mpm_ctx *ctx, const mpm_subgrid *sub, const double *src, const double *dflt_dense,
                              double *dst, cudaStream_t st);

extern "C" mpm_status mpm_cnn_precond(mpm_ctx *ctx, mpm_cnn *c, mpm_subgrid *sub, const mpm_lattice *lat,
                                      const mpm_params *prm, int32_t s, const double *v, double *z, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    if (!c || !sub || !lat || !prm || !v || !z) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_precond: null argument");
    if (!sub->extracted) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_precond: subgrid not extracted");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t vec = (size_t)(sub->NE > 0 ? sub->NE : 1);
    mpm_status r = mpm_grow(ctx, (void **)&ctx->d_fg, &ctx->fg_cap, (2 * vec + 8) * sizeof(double), "precond scratch");
    if (r != MPM_OK) return r;
    double *ve = ctx->d_fg, *ze = ve + vec, *scal = ze + vec;
    if (sub->NE > 0) {
        r = mpm_dense_to_elems(ctx, sub, v, ve, st);
        if (r != MPM_OK) return r;
        r = mpm_cnn_precond_impl(ctx, c, sub, lat, prm, s, ve, ze, scal, st);
        if (r != MPM_OK) return r;
    }
    const long long V = (long long)sub->n[0] * sub->n[1] * sub->n[2];
    MPM_CU(cudaMemsetAsync(z, 0, (size_t)V * sizeof(double), st));
    if (sub->NE == 0) return MPM_OK;
    return mpm_elems_to_dense(ctx, sub, ze, z, z, st);
}
