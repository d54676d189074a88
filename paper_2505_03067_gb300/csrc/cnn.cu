// cnn.cu -- the learned warm start: a small 3D CNN trained on the GPU by the
// library's own kernels (the paper has no network; this is one of the faster forms built around its solve).
//
// Network: six 3x3x3 convolutions with zero padding and a bias, channels
// 9 -> 24 -> 24 -> 24 -> 24 -> 24 -> 3, erf-GELU after layers 1-5, and a
// residual output pred = c^n + s_out * z6 (the next-step fields).
//
// Storage: activations are bfloat16, channel-last ([voxel][C], x fastest,
// crops of a batch one after the other) with C = 16 for the 9 input features
// and C = 24 for hidden layers; pre-activations z are kept in FP32 for the
// backward pass.  Weights live as an FP32 master vector (the layout of the
// oracle: per layer W[27][Ci][Co] then b[Co]) plus two bf16 copies per layer:
// the forward layout [27][Co_pad][Ci_pad] and the input-gradient layout (taps
// flipped, channels swapped).
//
// Convolutions (forward and input gradient) are implicit GEMMs on the tensor
// cores with mma.sync m16n8k16 / m16n8k8 (bf16 in, fp32 accumulate): a warp
// owns 16 consecutive voxels of an x-row and all output channels; K runs over
// the 27 taps times the input channels.  The weight gradient is a reduction
// over voxels done in FP32 SIMT with per-CTA partials summed in fixed order.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "mpm_internal.cuh"

namespace mpm {

constexpr int kLayers = 6;
__host__ __device__ constexpr int chan(int l) { return l == 0 ? 9 : (l == kLayers ? 3 : 24); }
constexpr int kInStride = 16;    // channels stored for the 9 input features
constexpr int kHidStride = 24;   // channels stored for hidden activations
constexpr int kOutPad = 8;       // output channels of layer 6 padded to one n-tile

__host__ __device__ constexpr int in_stride(int l) { return l == 0 ? kInStride : kHidStride; }
__host__ __device__ constexpr int out_pad(int l) { return l == kLayers - 1 ? kOutPad : kHidStride; }

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__device__ __forceinline__ void mma16816(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma1688(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t b0)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(b0));
}

enum { EPI_GELU = 0, EPI_OUT = 1, EPI_DGRAD = 2 };

struct ConvArgs {
    const __nv_bfloat16 *in;    // [V][CIN]
    int nx, ny, nz, B;
    const __nv_bfloat16 *W;     // [27][NT*8][CIN]
    const float *bias;          // [NT*8] or null
    float *z_out;               // EPI_GELU: [V][NT*8]
    __nv_bfloat16 *a_out;       // EPI_GELU: [V][NT*8]
    const float *fields;        // EPI_OUT: [V][3]
    float *pred;                // EPI_OUT: [V][3]
    float s_out;
    const float *zprev;         // EPI_DGRAD: [V][NT*8]
    __nv_bfloat16 *g_out;       // EPI_DGRAD: [V][NT*8]
};

__device__ __forceinline__ uint32_t ld_bf2(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

// Implicit-GEMM 3x3x3 convolution, zero padding per crop.  8 warps per CTA,
// each warp one 16-voxel x-segment; weights staged in shared memory.
template <int CIN, int NT, int EPI>
__global__ void __launch_bounds__(256) k_conv3(ConvArgs A)
{
    constexpr int CO = NT * 8;
    extern __shared__ __align__(16) unsigned char cnn_smem[];
    __nv_bfloat16 *Ws = reinterpret_cast<__nv_bfloat16 *>(cnn_smem);
    for (int i = threadIdx.x; i < 27 * CO * CIN / 2; i += blockDim.x)
        reinterpret_cast<uint32_t *>(Ws)[i] = reinterpret_cast<const uint32_t *>(A.W)[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int nsx = (A.nx + 15) >> 4;
    const long long nseg = (long long)nsx * A.ny * A.nz * A.B;
    const long long seg = (long long)blockIdx.x * 8 + warp;
    if (seg >= nseg) return;
    const int sx = (int)(seg % nsx);
    long long r = seg / nsx;
    const int y = (int)(r % A.ny); r /= A.ny;
    const int z = (int)(r % A.nz);
    const int b = (int)(r / A.nz);
    const int x0 = sx << 4;
    float acc[NT][4];
#pragma unroll
    for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.0f;
    const long long crop = (long long)b * A.nz * A.ny * A.nx;
#pragma unroll 1
    for (int t = 0; t < 27; ++t) {
        const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
        const int yy = y + dy, zz = z + dz;
        const bool rowok = yy >= 0 && yy < A.ny && zz >= 0 && zz < A.nz;
        const int xa = x0 + gid + dx, xb = x0 + gid + 8 + dx;
        const bool va = rowok && xa >= 0 && xa < A.nx, vb = rowok && xb >= 0 && xb < A.nx;
        const long long rowbase = crop + ((long long)zz * A.ny + yy) * A.nx;
        const __nv_bfloat16 *pa = A.in + (rowbase + xa) * CIN;
        const __nv_bfloat16 *pb = A.in + (rowbase + xb) * CIN;
        const __nv_bfloat16 *wt = Ws + (size_t)t * CO * CIN;
#pragma unroll
        for (int c0 = 0; c0 + 16 <= CIN; c0 += 16) {
            const uint32_t a0 = va ? ld_bf2(pa + c0 + tig * 2) : 0u;
            const uint32_t a1 = vb ? ld_bf2(pb + c0 + tig * 2) : 0u;
            const uint32_t a2 = va ? ld_bf2(pa + c0 + 8 + tig * 2) : 0u;
            const uint32_t a3 = vb ? ld_bf2(pb + c0 + 8 + tig * 2) : 0u;
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const __nv_bfloat16 *wr = wt + (n * 8 + gid) * CIN + c0 + tig * 2;
                mma16816(acc[n], a0, a1, a2, a3, ld_bf2(wr), ld_bf2(wr + 8));
            }
        }
        if (CIN % 16 == 8) {
            constexpr int c0 = CIN - 8;
            const uint32_t a0 = va ? ld_bf2(pa + c0 + tig * 2) : 0u;
            const uint32_t a1 = vb ? ld_bf2(pb + c0 + tig * 2) : 0u;
#pragma unroll
            for (int n = 0; n < NT; ++n) mma1688(acc[n], a0, a1, ld_bf2(wt + (n * 8 + gid) * CIN + c0 + tig * 2));
        }
    }
    // epilogue: thread holds voxels x0+gid (acc[.][0..1]) and x0+gid+8 (acc[.][2..3]),
    // output channels n*8 + tig*2 + {0, 1}
    const long long obase = crop + ((long long)z * A.ny + y) * A.nx;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int xv = x0 + gid + 8 * h;
        if (xv >= A.nx) continue;
        const long long v = obase + xv;
#pragma unroll
        for (int n = 0; n < NT; ++n) {
            const int co = n * 8 + tig * 2;
            float v0 = acc[n][2 * h], v1 = acc[n][2 * h + 1];
            if (EPI != EPI_DGRAD && A.bias) { v0 += A.bias[co]; v1 += A.bias[co + 1]; }
            if (EPI == EPI_GELU) {
                *reinterpret_cast<float2 *>(A.z_out + v * CO + co) = make_float2(v0, v1);
                *reinterpret_cast<__nv_bfloat162 *>(A.a_out + v * CO + co) = __floats2bfloat162_rn(gelu_f(v0), gelu_f(v1));
            } else if (EPI == EPI_OUT) {
                if (co < 3) A.pred[v * 3 + co] = A.fields[v * 3 + co] + A.s_out * v0;
                if (co + 1 < 3) A.pred[v * 3 + co + 1] = A.fields[v * 3 + co + 1] + A.s_out * v1;
            } else {
                const float2 zp = *reinterpret_cast<const float2 *>(A.zprev + v * CO + co);
                *reinterpret_cast<__nv_bfloat162 *>(A.g_out + v * CO + co) =
                    __floats2bfloat162_rn(v0 * gelu_grad_f(zp.x), v1 * gelu_grad_f(zp.y));
            }
        }
    }
}

// Weight and bias gradient of one layer: dW[t][ci][co] = sum_v in[v+off(t)][ci] g[v][co],
// db[co] = sum_v g[v][co].  Row r < 27*CI is (t, ci); row 27*CI is the bias.
// Each CTA sums its voxel chunks into partials[blockIdx][row][co].
template <int CI, int CIS, int CO, int GS>
__global__ void __launch_bounds__(256) k_wgrad(const __nv_bfloat16 *__restrict__ in,
                                               const __nv_bfloat16 *__restrict__ g, int nx, int ny, int nz, int B,
                                               float *__restrict__ partials)
{
    constexpr int CH = 64;
    constexpr int ROWS = 27 * CI + 1;
    __shared__ float gs[CH][CO];
    __shared__ int cx[CH], cy[CH], cz[CH];
    __shared__ long long cb[CH];
    const long long V = (long long)nx * ny * nz * B;
    const long long nchunk = (V + CH - 1) / CH;
    float acc[(ROWS + 255) / 256][CO];
#pragma unroll
    for (int k = 0; k < (ROWS + 255) / 256; ++k)
#pragma unroll
        for (int c = 0; c < CO; ++c) acc[k][c] = 0.0f;
    for (long long ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
        __syncthreads();
        for (int i = threadIdx.x; i < CH * CO; i += blockDim.x) {
            const int vv = i / CO, c = i - vv * CO;
            const long long v = ch * CH + vv;
            gs[vv][c] = v < V ? __bfloat162float(g[v * GS + c]) : 0.0f;
        }
        for (int i = threadIdx.x; i < CH; i += blockDim.x) {
            long long v = ch * CH + i;
            if (v >= V) v = V - 1;
            cx[i] = (int)(v % nx);
            long long r2 = v / nx;
            cy[i] = (int)(r2 % ny);
            r2 /= ny;
            cz[i] = (int)(r2 % nz);
            cb[i] = (r2 / nz) * (long long)nx * ny * nz;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < (ROWS + 255) / 256; ++k) {
            const int row = threadIdx.x + 256 * k;
            if (row >= ROWS) continue;
            if (row == 27 * CI) {
                for (int vv = 0; vv < CH; ++vv)
#pragma unroll
                    for (int c = 0; c < CO; ++c) acc[k][c] += gs[vv][c];
                continue;
            }
            const int t = row / CI, ci = row - t * CI;
            const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
            for (int vv = 0; vv < CH; ++vv) {
                const int xx = cx[vv] + dx, yy = cy[vv] + dy, zz = cz[vv] + dz;
                if (xx < 0 || xx >= nx || yy < 0 || yy >= ny || zz < 0 || zz >= nz) continue;
                const float a = __bfloat162float(in[(cb[vv] + ((long long)zz * ny + yy) * nx + xx) * CIS + ci]);
#pragma unroll
                for (int c = 0; c < CO; ++c) acc[k][c] += a * gs[vv][c];
            }
        }
    }
#pragma unroll
    for (int k = 0; k < (ROWS + 255) / 256; ++k) {
        const int row = threadIdx.x + 256 * k;
        if (row >= ROWS) continue;
        float *o = partials + ((size_t)blockIdx.x * ROWS + row) * CO;
#pragma unroll
        for (int c = 0; c < CO; ++c) o[c] = acc[k][c];
    }
}

// grads[off + i] = sum over CTAs (fixed order) of partials[b][i], i < n
__global__ void k_wgrad_reduce(const float *__restrict__ partials, int nblk, int n, float *__restrict__ grads)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.0f;
    for (int b = 0; b < nblk; ++b) s += partials[(size_t)b * n + i];
    grads[i] = s;
}

// bf16 forward and input-gradient weight layouts of every layer from the FP32 master.
struct PrepArgs {
    const float *master;
    __nv_bfloat16 *wf[kLayers];
    __nv_bfloat16 *wd[kLayers];
    float *bias[kLayers];
    long long off[kLayers];
};

__global__ void k_prep_weights(PrepArgs P)
{
    const int l = blockIdx.y;
    const int Ci = chan(l), Co = chan(l + 1);
    const int CIS = in_stride(l), COP = out_pad(l);
    const float *W = P.master + P.off[l];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 27 * COP * CIS; i += gridDim.x * blockDim.x) {
        const int t = i / (COP * CIS), rem = i - t * COP * CIS;
        const int co = rem / CIS, ci = rem - co * CIS;
        const float w = (ci < Ci && co < Co) ? W[((long long)t * Ci + ci) * Co + co] : 0.0f;
        P.wf[l][i] = __float2bfloat16_rn(w);
    }
    if (l > 0) {   // input gradient: in = g_l (COP channels), out = grad of a_{l-1} (CIS channels)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 27 * CIS * COP; i += gridDim.x * blockDim.x) {
            const int t = i / (CIS * COP), rem = i - t * CIS * COP;
            const int o = rem / COP, c = rem - o * COP;   // o: input channel of layer l, c: its output channel
            const int tf = 26 - t;
            const float w = (o < Ci && c < Co) ? W[((long long)tf * Ci + o) * Co + c] : 0.0f;
            P.wd[l][i] = __float2bfloat16_rn(w);
        }
    }
    if (blockIdx.x == 0)
        for (int c = threadIdx.x; c < COP; c += blockDim.x) P.bias[l][c] = c < Co ? W[27LL * Ci * Co + c] : 0.0f;
}

// Masked MSE over 3 species: loss partials and g6 = s_out * dLoss/dpred
// (bf16, 8 channels, 3..7 zero).  The mask is input feature 8.
__global__ void k_loss(const float *__restrict__ pred, const float *__restrict__ target,
                       const __nv_bfloat16 *__restrict__ x, long long V, float s_out,
                       const unsigned long long *__restrict__ nmask, __nv_bfloat16 *__restrict__ g6,
                       double *__restrict__ loss)
{
    const double inv = *nmask > 0 ? 1.0 / (3.0 * (double)*nmask) : 0.0;
    double part = 0.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        const float m = __bfloat162float(x[v * kInStride + 8]) > 0.5f ? 1.0f : 0.0f;
        __nv_bfloat16 out[kOutPad];
#pragma unroll
        for (int c = 0; c < kOutPad; ++c) out[c] = __float2bfloat16_rn(0.0f);
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const float d = m * (pred[v * 3 + s] - target[v * 3 + s]);
            part += (double)d * d * inv;
            out[s] = __float2bfloat16_rn((float)(s_out * 2.0 * d * inv));
        }
        uint4 u;
        memcpy(&u, out, 16);
        *reinterpret_cast<uint4 *>(g6 + v * kOutPad) = u;
    }
    part = warp_sum(part);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, part);
}

__global__ void k_count_mask(const __nv_bfloat16 *__restrict__ x, long long V, unsigned long long *__restrict__ n)
{
    unsigned c = 0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x)
        c += __bfloat162float(x[v * kInStride + 8]) > 0.5f ? 1u : 0u;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(n, (unsigned long long)c);
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

// Input features of a box crop of the lattice: c^n of the species (scaled by
// fscale), one-hot medium / tumour, the per-cell rates of the cell (uptake of
// species 0 and 1, source of species 2; scaled by rscale) and the mask.
struct FeatArgs {
    const int32_t *cell;
    const uint8_t *mask;
    const double *field[kMaxSpecies];
    int nspecies, ncell;
    const double *k_cell, *q_cell;
    int lo[3], n[3];
    int Lx, Ly;
    float fscale[3], rscale;
    __nv_bfloat16 *x;    // [V][16]
    float *fields;       // [V][3]
};

__global__ void k_features(FeatArgs F)
{
    const long long V = (long long)F.n[0] * F.n[1] * F.n[2];
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(v % F.n[0]);
        const long long r = v / F.n[0];
        const int j = (int)(r % F.n[1]), k = (int)(r / F.n[1]);
        const long long L = (long long)(F.lo[0] + i) + (long long)F.Lx * ((F.lo[1] + j) + (long long)F.Ly * (F.lo[2] + k));
        int id = F.cell[L];
        if (id < 0 || id >= F.ncell) id = 0;
        float f[kInStride];
#pragma unroll
        for (int c = 0; c < kInStride; ++c) f[c] = 0.0f;
        for (int s = 0; s < 3; ++s) {
            const float c = s < F.nspecies ? (float)F.field[s][L] : 0.0f;
            F.fields[v * 3 + s] = c;
            f[s] = c * F.fscale[s];
        }
        f[3] = id == 0 ? 1.0f : 0.0f;
        f[4] = id > 0 ? 1.0f : 0.0f;
        f[5] = F.nspecies > 0 ? (float)F.k_cell[id] * F.rscale : 0.0f;
        f[6] = F.nspecies > 1 ? (float)F.k_cell[F.ncell + id] * F.rscale : 0.0f;
        f[7] = F.nspecies > 2 ? (float)F.q_cell[2 * (long long)F.ncell + id] * F.rscale : 0.0f;
        f[8] = F.mask[L] ? 1.0f : 0.0f;
#pragma unroll
        for (int c = 0; c < kInStride; c += 2)
            *reinterpret_cast<__nv_bfloat162 *>(F.x + v * kInStride + c) = __floats2bfloat162_rn(f[c], f[c + 1]);
    }
}

}  // namespace mpm

using namespace mpm;

struct mpm_cnn {
    long long maxV = 0;
    long long nparams = 0;
    long long off[kLayers] = {};
    float *master = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *wf[kLayers] = {}, *wd[kLayers] = {};
    float *bias[kLayers] = {};
    float *z[kLayers] = {};           // pre-activations [V][out_pad]
    __nv_bfloat16 *a[kLayers] = {};   // activations (a[5] unused)
    __nv_bfloat16 *g = nullptr, *g2 = nullptr;   // gradient ping-pong [V][24]
    float *pred = nullptr;
    float *partials = nullptr;
    int nblk_w = 0;
    unsigned long long *d_nmask = nullptr;
    double *d_loss = nullptr;
    __nv_bfloat16 *gx = nullptr;      // features of one box (mpm_cnn_guess)
    float *gfields = nullptr;
    int step = 0;
    float s_out = 0.01f;
    std::vector<void *> allocs;
};

static mpm_status cnn_alloc(mpm_ctx *ctx, mpm_cnn *c, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return mpm_fail(ctx, MPM_ERR_NOMEM, "cnn: device allocation failed");
    }
    c->allocs.push_back(*p);
    return MPM_OK;
}

template <int CIN, int NT, int EPI>
static cudaError_t launch_conv(const ConvArgs &A, long long V, cudaStream_t st)
{
    const size_t smem = (size_t)27 * NT * 8 * CIN * sizeof(__nv_bfloat16);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_conv3<CIN, NT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const long long nseg = (long long)((A.nx + 15) / 16) * A.ny * A.nz * A.B;
    (void)V;
    k_conv3<CIN, NT, EPI><<<(unsigned)((nseg + 7) / 8), 256, smem, st>>>(A);
    return cudaGetLastError();
}

mpm_status mpm_import_pred_impl(mpm_ctx *ctx, mpm_subgrid *sub, const float *pred, cudaStream_t st);

extern "C" mpm_status mpm_cnn_create(mpm_ctx *ctx, mpm_cnn **out, int64_t max_voxels)
{
    if (!ctx || !out || max_voxels < 1) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_create: bad argument");
    mpm_cnn *c = new mpm_cnn();
    c->maxV = max_voxels;
    long long n = 0;
    for (int l = 0; l < kLayers; ++l) {
        c->off[l] = n;
        n += 27LL * chan(l) * chan(l + 1) + chan(l + 1);
    }
    c->nparams = n;
    mpm_status r = MPM_OK;
    auto A = [&](void **p, size_t b) { if (r == MPM_OK) r = cnn_alloc(ctx, c, p, b); };
    A((void **)&c->master, n * 4);
    A((void **)&c->grads, n * 4);
    A((void **)&c->m, n * 4);
    A((void **)&c->v, n * 4);
    for (int l = 0; l < kLayers; ++l) {
        A((void **)&c->wf[l], 27 * out_pad(l) * in_stride(l) * 2);
        A((void **)&c->wd[l], 27 * out_pad(l) * in_stride(l) * 2);
        A((void **)&c->bias[l], out_pad(l) * 4);
        A((void **)&c->z[l], (size_t)max_voxels * out_pad(l) * 4);
        if (l < kLayers - 1) A((void **)&c->a[l], (size_t)max_voxels * kHidStride * 2);
    }
    A((void **)&c->g, (size_t)max_voxels * kHidStride * 2);
    A((void **)&c->g2, (size_t)max_voxels * kHidStride * 2);
    A((void **)&c->pred, (size_t)max_voxels * 3 * 4);
    c->nblk_w = 2 * ctx->num_sms;
    A((void **)&c->partials, (size_t)c->nblk_w * (27 * 24 + 1) * 24 * 4);
    A((void **)&c->d_nmask, 256);
    A((void **)&c->d_loss, 256);
    A((void **)&c->gx, (size_t)max_voxels * kInStride * 2);
    A((void **)&c->gfields, (size_t)max_voxels * 3 * 4);
    if (r != MPM_OK) {
        mpm_cnn_destroy(ctx, c);
        return r;
    }
    cudaMemset(c->m, 0, n * 4);
    cudaMemset(c->v, 0, n * 4);
    *out = c;
    return MPM_OK;
}

extern "C" mpm_status mpm_cnn_destroy(mpm_ctx *ctx, mpm_cnn *c)
{
    (void)ctx;
    if (!c) return MPM_ERR_ARG;
    for (void *p : c->allocs) cudaFree(p);
    delete c;
    return MPM_OK;
}

static mpm_status prep(mpm_ctx *ctx, mpm_cnn *c, cudaStream_t st)
{
    PrepArgs P;
    P.master = c->master;
    for (int l = 0; l < kLayers; ++l) {
        P.wf[l] = c->wf[l];
        P.wd[l] = c->wd[l];
        P.bias[l] = c->bias[l];
        P.off[l] = c->off[l];
    }
    k_prep_weights<<<dim3(16, kLayers), 256, 0, st>>>(P);
    ctx->launches += 1;
    MPM_CU(cudaGetLastError());
    return MPM_OK;
}

extern "C" mpm_status mpm_cnn_set_params(mpm_ctx *ctx, mpm_cnn *c, const float *host_params, int64_t n, float s_out, void *stream)
{
    if (!ctx || !c || !host_params || n != c->nparams) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_set_params: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    MPM_CU(cudaMemcpyAsync(c->master, host_params, n * 4, cudaMemcpyHostToDevice, st));
    MPM_CU(cudaMemsetAsync(c->m, 0, n * 4, st));
    MPM_CU(cudaMemsetAsync(c->v, 0, n * 4, st));
    MPM_CU(cudaStreamSynchronize(st));
    c->step = 0;
    c->s_out = s_out;
    return prep(ctx, c, st);
}

extern "C" mpm_status mpm_cnn_get_params(mpm_ctx *ctx, const mpm_cnn *c, int32_t which, float *host_out, int64_t n, void *stream)
{
    if (!ctx || !c || !host_out || n != c->nparams) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_get_params: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    MPM_CU(cudaMemcpyAsync(host_out, which == 1 ? c->grads : c->master, n * 4, cudaMemcpyDeviceToHost, st));
    MPM_CU(cudaStreamSynchronize(st));
    return MPM_OK;
}

extern "C" mpm_status mpm_cnn_features(mpm_ctx *ctx, const mpm_lattice *lat, const mpm_params *prm, const mpm_box *box,
                            void *x_bf16, float *fields, void *stream)
{
    if (!ctx || !lat || !prm || !box || !x_bf16 || !fields) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_features: null argument");
    FeatArgs F;
    memset(&F, 0, sizeof(F));
    F.cell = lat->cell_id;
    F.mask = lat->mask;
    F.nspecies = prm->nspecies;
    for (int s = 0; s < prm->nspecies && s < kMaxSpecies; ++s) F.field[s] = lat->field[s];
    F.ncell = prm->ncell;
    F.k_cell = prm->k_cell;
    F.q_cell = prm->q_cell;
    for (int d = 0; d < 3; ++d) {
        F.lo[d] = box->lo[d];
        F.n[d] = box->hi[d] - box->lo[d];
        if (F.n[d] < 1 || box->lo[d] < 0 || box->hi[d] > lat->dims[d]) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_features: bad box");
    }
    F.Lx = lat->dims[0];
    F.Ly = lat->dims[1];
    F.fscale[0] = 1.0f;
    F.fscale[1] = 1.0f;
    F.fscale[2] = 20.0f;
    F.rscale = 10.0f;
    F.x = (__nv_bfloat16 *)x_bf16;
    F.fields = fields;
    k_features<<<ctx->num_sms * 4, 256, 0, (cudaStream_t)stream>>>(F);
    ctx->launches += 1;
    MPM_CU(cudaGetLastError());
    return MPM_OK;
}

static mpm_status forward(mpm_ctx *ctx, mpm_cnn *c, const void *x, const float *fields, const int32_t dims[3], int B,
                          float *pred, cudaStream_t st)
{
    const long long V = (long long)dims[0] * dims[1] * dims[2] * B;
    if (V > c->maxV) return mpm_fail(ctx, MPM_ERR_ARG, "cnn: more voxels than the network was created for");
    ConvArgs A;
    memset(&A, 0, sizeof(A));
    A.nx = dims[0]; A.ny = dims[1]; A.nz = dims[2]; A.B = B;
    for (int l = 0; l < kLayers; ++l) {
        A.in = l == 0 ? (const __nv_bfloat16 *)x : c->a[l - 1];
        A.W = c->wf[l];
        A.bias = c->bias[l];
        cudaError_t e;
        if (l < kLayers - 1) {
            A.z_out = c->z[l];
            A.a_out = c->a[l];
            e = l == 0 ? launch_conv<16, 3, EPI_GELU>(A, V, st) : launch_conv<24, 3, EPI_GELU>(A, V, st);
        } else {
            A.fields = fields;
            A.pred = pred;
            A.s_out = c->s_out;
            e = launch_conv<24, 1, EPI_OUT>(A, V, st);
        }
        ctx->launches += 1;
        if (e != cudaSuccess) return mpm_cuda_check(ctx, e, "cnn forward conv");
    }
    return MPM_OK;
}

extern "C" mpm_status mpm_cnn_forward(mpm_ctx *ctx, mpm_cnn *c, const void *x_bf16, const float *fields, const int32_t dims[3],
                           int32_t batch, float *pred, void *stream)
{
    if (!ctx || !c || !x_bf16 || !fields || !dims || !pred || batch < 1) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_forward: bad argument");
    return forward(ctx, c, x_bf16, fields, dims, batch, pred, (cudaStream_t)stream);
}

template <int CI, int CIS, int CO, int GS>
static mpm_status wgrad_layer(mpm_ctx *ctx, mpm_cnn *c, const __nv_bfloat16 *in, const __nv_bfloat16 *g,
                              const int32_t dims[3], int B, float *grads_out, cudaStream_t st)
{
    k_wgrad<CI, CIS, CO, GS><<<c->nblk_w, 256, 0, st>>>(in, g, dims[0], dims[1], dims[2], B, c->partials);
    const int n = (27 * CI + 1) * CO;
    k_wgrad_reduce<<<(n + 255) / 256, 256, 0, st>>>(c->partials, c->nblk_w, n, grads_out);
    ctx->launches += 2;
    MPM_CU(cudaGetLastError());
    return MPM_OK;
}

// Forward, loss and the gradient of every parameter into c->grads.
static mpm_status backward(mpm_ctx *ctx, mpm_cnn *c, const void *x, const float *fields, const float *target,
                           const int32_t dims[3], int B, cudaStream_t st)
{
    mpm_status r = forward(ctx, c, x, fields, dims, B, c->pred, st);
    if (r != MPM_OK) return r;
    const long long V = (long long)dims[0] * dims[1] * dims[2] * B;
    MPM_CU(cudaMemsetAsync(c->d_nmask, 0, 8, st));
    MPM_CU(cudaMemsetAsync(c->d_loss, 0, 8, st));
    k_count_mask<<<ctx->num_sms * 4, 256, 0, st>>>((const __nv_bfloat16 *)x, V, c->d_nmask);
    k_loss<<<ctx->num_sms * 4, 256, 0, st>>>(c->pred, target, (const __nv_bfloat16 *)x, V, c->s_out, c->d_nmask,
                                             c->g, c->d_loss);
    ctx->launches += 2;
    MPM_CU(cudaGetLastError());
    // layer 6: g holds dL/dz6 (8 channels)
    __nv_bfloat16 *g = c->g, *gn = c->g2;
    for (int l = kLayers - 1; l >= 0; --l) {
        float *gW = c->grads + c->off[l];
        const __nv_bfloat16 *in = l == 0 ? (const __nv_bfloat16 *)x : c->a[l - 1];
        if (l == kLayers - 1) r = wgrad_layer<24, 24, 3, 8>(ctx, c, in, g, dims, B, gW, st);
        else if (l == 0) r = wgrad_layer<9, 16, 24, 24>(ctx, c, in, g, dims, B, gW, st);
        else r = wgrad_layer<24, 24, 24, 24>(ctx, c, in, g, dims, B, gW, st);
        if (r != MPM_OK) return r;
        if (l == 0) break;
        // dL/dz_{l-1} = conv^T(g; W_l) * gelu'(z_{l-1})
        ConvArgs A;
        memset(&A, 0, sizeof(A));
        A.nx = dims[0]; A.ny = dims[1]; A.nz = dims[2]; A.B = B;
        A.in = g;
        A.W = c->wd[l];
        A.zprev = c->z[l - 1];
        A.g_out = gn;
        cudaError_t e = l == kLayers - 1 ? launch_conv<8, 3, EPI_DGRAD>(A, V, st) : launch_conv<24, 3, EPI_DGRAD>(A, V, st);
        ctx->launches += 1;
        if (e != cudaSuccess) return mpm_cuda_check(ctx, e, "cnn input-gradient conv");
        __nv_bfloat16 *t = g;
        g = gn;
        gn = t;
    }
    return MPM_OK;
}

extern "C" mpm_status mpm_cnn_guess(mpm_ctx *ctx, mpm_cnn *c, mpm_subgrid *sub, const mpm_lattice *lat, const mpm_params *prm,
                         void *stream)
{
    if (!ctx || !c || !sub || !lat || !prm) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_guess: null argument");
    if (!sub->extracted) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_guess: subgrid not extracted");
    if (sub->nspecies > 3) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_guess: the network predicts 3 species");
    const long long V = (long long)sub->n[0] * sub->n[1] * sub->n[2];
    if (V > c->maxV) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_guess: box larger than the network was created for");
    cudaStream_t st = (cudaStream_t)stream;
    mpm_box box;
    for (int d = 0; d < 3; ++d) { box.lo[d] = sub->lo[d]; box.hi[d] = sub->hi[d]; }
    mpm_status r = mpm_cnn_features(ctx, lat, prm, &box, c->gx, c->gfields, stream);
    if (r != MPM_OK) return r;
    r = forward(ctx, c, c->gx, c->gfields, sub->n, 1, c->pred, st);
    if (r != MPM_OK) return r;
    return mpm_import_pred_impl(ctx, sub, c->pred, st);
}

extern "C" mpm_status mpm_cnn_train_step(mpm_ctx *ctx, mpm_cnn *c, const void *x_bf16, const float *fields, const float *target,
                              const int32_t dims[3], int32_t batch, float lr, int32_t apply, double *loss_out,
                              void *stream)
{
    if (!ctx || !c || !x_bf16 || !fields || !target || !dims || batch < 1)
        return mpm_fail(ctx, MPM_ERR_ARG, "cnn_train_step: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    mpm_status r = backward(ctx, c, x_bf16, fields, target, dims, batch, st);
    if (r != MPM_OK) return r;
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
        MPM_CU(cudaMemcpyAsync(ctx->h_stage, c->d_loss, 8, cudaMemcpyDeviceToHost, st));
        MPM_CU(cudaStreamSynchronize(st));
        *loss_out = *(double *)ctx->h_stage;
    }
    return MPM_OK;
}


// ---------------------------------------------------------------- the network as a preconditioner
// Row a13: flexible GMRES applies z = m * net(v / m) to a vector v of one
// species (m = max |v|, which puts v in the range the network was trained
// on), with the other fields and the source map at zero (the homogeneous
// problem), and keeps z on the in-mask voxels only.
namespace mpm {

struct PcArgs {
    BoxGeo g;                      // the subgrid's box
    const int32_t *tile_index;     // box tile -> compact tile (-1: not stored)
    const int32_t *tile_coord;
    const uint8_t *flags;          // compact
    const int32_t *cell;           // lattice
    const uint8_t *mask;           // lattice
    const double *k_cell;
    int nspecies, ncell, s;
    const double *v;               // compact input
    double *z;                     // compact output
    const double *scale;           // device scalar m
    __nv_bfloat16 *x;              // [V][16]
    float *fields;                 // [V][3]
    const float *pred;             // [V][3]
    int64_t NE;
};

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

__global__ void k_pc_features(PcArgs P)
{
    const BoxGeo &g = P.g;
    const long long V = (long long)g.n[0] * g.n[1] * g.n[2];
    const double m = *P.scale;
    const float fscale[3] = {1.0f, 1.0f, 20.0f};
    const int ltv = g.lt[0] + g.lt[1] + g.lt[2];
    for (long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x; d < V; d += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(d % g.n[0]);
        const long long r = d / g.n[0];
        const int j = (int)(r % g.n[1]), k = (int)(r / g.n[1]);
        const int32_t t = P.tile_index[((long long)(k >> g.lt[2]) * g.nt[1] + (j >> g.lt[1])) * g.nt[0] + (i >> g.lt[0])];
        double val = 0.0;
        if (t >= 0 && m > 0.0) {
            const int ix = i & ((1 << g.lt[0]) - 1), iy = j & ((1 << g.lt[1]) - 1), iz = k & ((1 << g.lt[2]) - 1);
            const int64_t e = ((int64_t)t << ltv) + ix + ((int64_t)(iy + (iz << g.lt[1])) << g.lt[0]);
            val = P.v[e] / m;
        }
        const long long L = (long long)(g.lo[0] + i) + (long long)g.Lx * ((g.lo[1] + j) + (long long)g.Ly * (g.lo[2] + k));
        int id = P.cell[L];
        if (id < 0 || id >= P.ncell) id = 0;
        float f[kInStride];
#pragma unroll
        for (int c = 0; c < kInStride; ++c) f[c] = 0.0f;
        const float vf = (float)val;
        for (int c = 0; c < 3; ++c) P.fields[d * 3 + c] = c == P.s ? vf : 0.0f;
        f[P.s] = vf * fscale[P.s];
        f[3] = id == 0 ? 1.0f : 0.0f;
        f[4] = id > 0 ? 1.0f : 0.0f;
        f[5] = P.nspecies > 0 ? (float)P.k_cell[id] * 10.0f : 0.0f;
        f[6] = P.nspecies > 1 ? (float)P.k_cell[P.ncell + id] * 10.0f : 0.0f;
        f[8] = P.mask[L] ? 1.0f : 0.0f;
#pragma unroll
        for (int c = 0; c < kInStride; c += 2)
            *reinterpret_cast<__nv_bfloat162 *>(P.x + d * kInStride + c) = __floats2bfloat162_rn(f[c], f[c + 1]);
    }
}

__global__ void k_pc_out(PcArgs P)
{
    const BoxGeo &g = P.g;
    const double m = *P.scale;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P.NE; e += (int64_t)gridDim.x * blockDim.x) {
        double zv = 0.0;
        if ((P.flags[e] & F_MASK) && m > 0.0) {
            int bx, by, bz;
            elem_box(e, g, P.tile_coord, bx, by, bz);
            const int64_t d = bx + (int64_t)g.n[0] * (by + (int64_t)g.n[1] * bz);
            zv = m * (double)P.pred[d * 3 + P.s];
        }
        P.z[e] = zv;
    }
}

}  // namespace mpm

// z = the network's preconditioner applied to v (compact FP64 vectors of
// species s of sub); d_scale: one device double of scratch.  Stream work only.
mpm_status mpm_cnn_precond_impl(mpm_ctx *ctx, mpm_cnn *c, mpm_subgrid *sub, const mpm_lattice *lat,
                                const mpm_params *prm, int s, const double *v, double *z, double *d_scale,
                                cudaStream_t st)
{
    const long long V = (long long)sub->n[0] * sub->n[1] * sub->n[2];
    if (V > c->maxV) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_precond: box larger than the network was created for");
    if (s < 0 || s > 2) return mpm_fail(ctx, MPM_ERR_ARG, "cnn_precond: the network covers species 0..2");
    PcArgs P;
    memset(&P, 0, sizeof(P));
    P.g = make_geo(sub, lat->dims);
    P.tile_index = sub->tile_index;
    P.tile_coord = sub->tile_coord;
    P.flags = sub->flags;
    P.cell = lat->cell_id;
    P.mask = lat->mask;
    P.k_cell = prm->k_cell;
    P.nspecies = prm->nspecies;
    P.ncell = prm->ncell;
    P.s = s;
    P.v = v;
    P.z = z;
    P.scale = d_scale;
    P.x = c->gx;
    P.fields = c->gfields;
    P.pred = c->pred;
    P.NE = sub->NE;
    k_pc_amax<<<1, 1024, 0, st>>>(v, sub->NE, d_scale);
    k_pc_features<<<ctx->num_sms * 4, 256, 0, st>>>(P);
    ctx->launches += 2;
    MPM_CU(cudaGetLastError());
    mpm_status r = forward(ctx, c, c->gx, c->gfields, sub->n, 1, c->pred, st);
    if (r != MPM_OK) return r;
    k_pc_out<<<ctx->num_sms * 4, 256, 0, st>>>(P);
    ctx->launches += 1;
    MPM_CU(cudaGetLastError());
    return MPM_OK;
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
