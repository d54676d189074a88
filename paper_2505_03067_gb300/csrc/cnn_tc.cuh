// cnn_tc.cuh -- the learned warm start's 3x3x3 convolutions on the fifth-
// generation tensor cores (tcgen05.mma, accumulators in tensor memory), for
// sm_103a.
//
// Domain.  The network runs on B "images" of dims L[3] (x fastest, images
// stacked along z), each with its own box [lo, lo + n).  A voxel is ACTIVE
// when it lies in its image's box and its mask byte is set: the network sees
// the pleural space only (activations are zero at inactive voxels).  Images
// are laid out like a lattice, so a network applied to a solver lattice reads
// and writes lattice-indexed buffers directly.
//
// Work decomposition.  The box of an image is cut into SLABS of 8 (x) x 16 (y)
// x 1 (z) voxels -- M = 128 rows of one MMA -- and slabs into UNITS of kZSeg
// consecutive slabs along z.  A plan kernel lists the units that hold an
// active voxel; a persistent CTA per SM takes units from that list.
//
// Implicit GEMM.  For an output slab at depth z the convolution is
//     D[v][co] = sum over (dy, dz) of sum over (dx, ci) of in[v + (dx,dy,dz)][ci] W[(dx,dy,dz)][ci][co].
// The input halo of a depth (10 x 18 voxels) is staged in shared memory in
// the tensor cores' canonical no-swizzle K-major layout with THREE copies
// shifted by dx = -1, 0, +1 laid side by side along K: the core matrix of
// K-column q = 3-copy index c times the channel chunks, plus the chunk kc,
// for the 8 x-rows of halo row y', sits at y' * GS + q * 128.  A shift in y is
// then a whole number of 8-row core-matrix groups, so the A operand of every
// tap (dy, dz) is the same buffer at another start address: 9 taps x (K/16)
// MMAs per slab read the staged halo in place, with no per-tap copy.  The
// weights of all taps are staged once per CTA in the matching B layout.
//
// Pipeline per CTA.  Halo depths are copied with cp.async (16 B, zero-filled
// for inactive voxels) into a ring of kSlots slots, two depths ahead; one
// thread issues the slab's MMAs into one of two TMEM accumulators and commits
// them to an mbarrier; all eight warps drain the other accumulator (tcgen05.ld)
// through the epilogue while the tensor cores run.
//
// Weight gradient.  dW[(dx,dy,dz)][ci][co] = sum_v in[v + off][ci] g[v][co] is
// a GEMM over voxels with the halo buffer read as an MN-major A operand
// (M = the K-columns of the forward layout, K = voxels along y) and the
// slab's gradient tile as an MN-major B operand; the nine taps accumulate in
// nine TMEM accumulators over all slabs of a CTA, and per-CTA partial sums are
// reduced in a fixed order.
#pragma once

#include <cuda_bf16.h>

#include "mpm_internal.cuh"

namespace mpm {
namespace tc {

constexpr int kSlabX = 8, kSlabY = 16, kZSeg = 8;
constexpr int kHaloX = kSlabX + 2, kHaloY = kSlabY + 2;
constexpr int kSlots = 6;               // halo depths in the shared-memory ring
constexpr int kThreads = 256;           // weight-gradient kernel: 8 warps
constexpr int kEpiWarps = 16;           // forward kernel: 16 epilogue / loader warps ...
constexpr int kConvThreads = 32 * (kEpiWarps + 1);   // ... and one warp that issues the MMAs
constexpr int kMaxImages = 16;

// Device-side description of the images a network application covers.
struct CnnDom {
    int32_t L[3];                       // dims of one image
    int32_t B;                          // images
    int32_t lo[kMaxImages][3];          // box of each image
    int32_t n[kMaxImages][3];           // (n[b][0] == 0: empty image)
};

// A unit: image b, slab origin (ox, oy) in image coordinates, depths
// [z0, z0 + nz) (nz <= kZSeg).
struct Unit {
    int32_t b, ox, oy, z0;
    int32_t nz, pad0, pad1, pad2;
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start address, K-direction
// core-matrix stride (LBO) and M/N-direction stride (SBO), sm_100 version bit.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16 with bf16 A and B, FP32 accumulation.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn, bool b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
                 "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of an mbarrier: false (and *err set) when
// timeout_ns of wall time passed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t timeout_ns, int32_t *err)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try(bar, parity)) return true;
        if (globaltimer_ns() - t0 > timeout_ns) {
            if (err) atomicExch(err, 1);
            return false;
        }
    }
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 lanes x 32 bit, N consecutive columns: thread t of the warp receives
// columns [col, col + N) of lane (warp's lane quarter) * 32 + t.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 16-byte asynchronous global -> shared copy; src_bytes 0 writes zeros.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Wait until at most n of this thread's committed groups are pending.
__device__ __forceinline__ void cp_async_wait(int n)
{
    switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
    case 4: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
    }
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// ---------------------------------------------------------------- layouts
// Input channels CI (8, 16 or 24) -> chunks of 8, K-columns of the 3-copy halo
// (padded to even), shared bytes per halo row and per depth slot.
template <int CI>
struct Halo {
    static constexpr int KC = CI / 8;
    static constexpr int QC = 3 * KC;
    static constexpr int QP = QC + (QC & 1);
    static constexpr int GS = QP * 128;            // bytes per halo row (18 of them per depth)
    static constexpr int SLOT = kHaloY * GS;       // bytes per depth
    static constexpr int NKS = QP / 2;             // MMAs of K = 16 per tap
};

// Weight image of one layer for the forward kernel: for tap pair p = (dy+1) +
// 3 (dz+1), K-column q and output-channel group ng, the 8 x 8 core matrix
// (rows n = ng*8 + r, columns k = q*8 + j) at ((p * QP + q) * NG + ng) * 128 bytes.
template <int CI, int NO>
struct WImg {
    static constexpr int NG = NO / 8;
    static constexpr int BYTES = 9 * Halo<CI>::QP * NG * 128;
};

// Shared memory of the forward kernel.
template <int CI, int NO>
struct ConvSmem {
    static constexpr int W_OFF = 0;
    static constexpr int RING_OFF = (WImg<CI, NO>::BYTES + 1023) & ~1023;
    static constexpr int RING_BYTES = kSlots * Halo<CI>::SLOT;
    static constexpr int ACT_OFF = RING_OFF + RING_BYTES + 2048;   // 2 KB guard after the ring
    static constexpr int ACT_BYTES = (kZSeg + 2) * kHaloY * kHaloX;
    static constexpr int BAR_OFF = (ACT_OFF + ACT_BYTES + 15) & ~15;
    static constexpr int BYTES = BAR_OFF + 64;
};

enum { EPI_GELU = 0, EPI_OUT = 1, EPI_DGRAD = 2 };

struct ConvArgs {
    const __nv_bfloat16 *in;        // [B * V][CI]
    const uint8_t *mask;            // [B * V]
    const CnnDom *dom;
    const Unit *units;
    const int32_t *nunits;
    int32_t *work;                  // dynamic scheduling counter (reset by the plan)
    const unsigned char *wimg;      // weight image (WImg layout)
    const float *bias;              // [NO] (null: none)
    // EPI_GELU: a_out = bf16(gelu(z)) at active voxels, z_out (nullable) = z
    __nv_bfloat16 *a_out;           // [B * V][24]
    float *z_out;                   // [B * V][24]
    // EPI_OUT: pred = c^n + s_out * z (3 channels)
    float s_out;
    const float *f32;               // [B * V][3] c^n (image mode)
    float *pred;                    // [B * V][3] (image mode)
    const double *field[3];         // lattice c^n (solver mode, B = 1)
    double *xs[3];                  // solver iterate (compact elements)
    const int32_t *tile_index;      // box tile -> compact tile (solver mode)
    const BoxGeo *geo;              // the step's box geometry (solver mode)
    int32_t nspecies;
    // EPI_DGRAD: g_out = bf16(D * gelu'(z_prev)) at active voxels
    const float *zprev;             // [B * V][24]
    __nv_bfloat16 *g_out;           // [B * V][24]
    int32_t *err;                   // set on a wait that timed out
    uint64_t timeout_ns;
};

__device__ __forceinline__ int64_t vox_index(const CnnDom &D, int b, int x, int y, int z)
{
    return (((int64_t)b * D.L[2] + z) * D.L[1] + y) * (int64_t)D.L[0] + x;
}

__device__ __forceinline__ bool in_box(const CnnDom &D, int b, int x, int y, int z)
{
    return x >= D.lo[b][0] && x < D.lo[b][0] + D.n[b][0] && y >= D.lo[b][1] && y < D.lo[b][1] + D.n[b][1] &&
           z >= D.lo[b][2] && z < D.lo[b][2] + D.n[b][2];
}

// Active bytes of a unit's halo region (depths z0-1 .. z0+kZSeg, rows
// oy-1 .. oy+16, columns ox-1 .. ox+8) into smem; returns per-slab activity
// in the low kZSeg bits (through *slab_bits, all threads).
template <int NTHR>
__device__ __forceinline__ void load_unit_act(const CnnDom &D, const uint8_t *__restrict__ mask, const Unit &u,
                                              uint8_t *act, uint32_t *slab_bits)
{
    if (threadIdx.x == 0) *slab_bits = 0u;
    __syncthreads();
    constexpr int N = (kZSeg + 2) * kHaloY * kHaloX;
    uint32_t mine = 0u;
    for (int i = threadIdx.x; i < N; i += NTHR) {
        const int xh = i % kHaloX, r = i / kHaloX;
        const int yh = r % kHaloY, j = r / kHaloY;
        const int x = u.ox - 1 + xh, y = u.oy - 1 + yh, z = u.z0 - 1 + j;
        uint8_t a = 0;
        if (in_box(D, u.b, x, y, z)) a = __ldg(mask + vox_index(D, u.b, x, y, z)) != 0;
        act[i] = a;
        if (a && xh >= 1 && xh <= kSlabX && yh >= 1 && yh <= kSlabY && j >= 1 && j <= u.nz) mine |= 1u << (j - 1);
    }
    if (mine) atomicOr(slab_bits, mine);
    __syncthreads();
}

// The 16-byte copies of one halo depth handled by one loader thread, fixed for
// a launch: the k-th covers item tid + k NL of the depth (halo row yh, copy c,
// x row, channel chunk kc); `rel` is its source offset in elements from the
// depth's halo origin, `dst` its shared offset in the slot, `act` its index in
// a depth of the unit's activity bytes (act < 0: no item).
template <int CI, int NL>
struct HaloItems {
    static constexpr int N = kHaloY * 3 * kSlabX * (CI / 8);
    static constexpr int K = (N + NL - 1) / NL;
    int32_t rel[K], dst[K], act[K];
    __device__ __forceinline__ void init(int tid, int L0)
    {
        using H = Halo<CI>;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = tid + k * NL;
            const int kc = i % H::KC;
            int r = i / H::KC;
            const int x = r % kSlabX;
            r /= kSlabX;
            const int c = r % 3, yh = r / 3;
            const int xh = x + c;
            rel[k] = (yh * L0 + xh) * CI + kc * 8;
            dst[k] = yh * H::GS + (c * H::KC + kc) * 128 + x * 16;
            act[k] = i < N ? yh * kHaloX + xh : -1;
        }
    }
};

// cp.async the halo depth j (image depth z0 - 1 + j) of unit u into slot base
// `dst` (3 x-shifted copies, zero-filled where inactive), with the items of
// this thread (it.act < 0: none).
template <int CI, int NL>
__device__ __forceinline__ void load_halo_depth_items(const CnnDom &D, const __nv_bfloat16 *__restrict__ in,
                                                      const Unit &u, const uint8_t *act, int j, uint32_t dst,
                                                      const HaloItems<CI, NL> &it)
{
    const uint8_t *aj = act + j * kHaloY * kHaloX;
    // the halo origin (ox - 1, oy - 1) of this depth; items inside the box only
    // are read (inactive or outside: zero-filled, source unused)
    const int64_t base = (((int64_t)u.b * D.L[2] + (u.z0 - 1 + j)) * D.L[1] + (u.oy - 1)) * (int64_t)D.L[0] + (u.ox - 1);
#pragma unroll
    for (int k = 0; k < HaloItems<CI, NL>::K; ++k) {
        if (it.act[k] < 0) continue;
        const bool ok = aj[it.act[k]] != 0;
        const __nv_bfloat16 *src = ok ? in + (base * CI + it.rel[k]) : in;
        cp_async16(dst + (uint32_t)it.dst[k], src, ok ? 16u : 0u);
    }
}

// ---------------------------------------------------------------- forward / input-gradient convolution
// One persistent CTA per SM; units are taken from the plan's list through an
// atomic counter.  NO: MMA N (output channels padded to 16 or 32).  Warps
// 0..15 load the halo depths and run the epilogue (warp w: TMEM lane quarter
// w & 3, channels 6 (w >> 2) .. 6 (w >> 2) + 5); warp 16 issues the MMAs, so
// a slab's MMAs overlap the previous slab's epilogue.
template <int CI, int NO, int EPI>
__global__ void __launch_bounds__(kConvThreads, 1) k_conv_tc(const __grid_constant__ ConvArgs A)
{
    using H = Halo<CI>;
    using S = ConvSmem<CI, NO>;
    constexpr int NG = WImg<CI, NO>::NG;
    constexpr int NL = 32 * kEpiWarps;            // loader / epilogue threads
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint32_t s_tmem, s_bits;
    __shared__ int32_t s_unit;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + S::BAR_OFF);   // [0], [1]: MMA done per accumulator
    uint8_t *act = sm + S::ACT_OFF;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool mma_warp = warp == kEpiWarps;
    const CnnDom &D = *A.dom;
    const uint32_t wbase = smem_u32(sm + S::W_OFF), rbase = smem_u32(sm + S::RING_OFF);

    // weights into shared memory; zero the ring (pad K-columns stay zero)
    for (int i = tid; i < WImg<CI, NO>::BYTES / 16; i += kConvThreads)
        reinterpret_cast<uint4 *>(sm + S::W_OFF)[i] = __ldg(reinterpret_cast<const uint4 *>(A.wimg) + i);
    for (int i = tid; i < (S::RING_BYTES + 2048) / 16; i += kConvThreads)
        reinterpret_cast<uint4 *>(sm + S::RING_OFF)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) tmem_alloc(&s_tmem, 64);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = s_tmem;
    constexpr uint32_t kIdesc = idesc_bf16(128, NO, false, false);
    // descriptors of the ring and weight bases; a tap's operands are these
    // plus an offset (start-address field in 16-byte units)
    const uint64_t adesc0 = sdesc(rbase, 128u, H::GS), bdesc0 = sdesc(wbase, NG * 128u, 128u);
    // epilogue role
    const int lq = warp & 3, wq = (warp >> 2) & 3;
    const int row = lq * 32 + lane;               // voxel (row & 7, row >> 3) of the slab
    const int ex = row & 7, ey = row >> 3;
    const int c0 = 6 * wq;                        // first channel of this thread
    const bool epi = !mma_warp && (EPI != EPI_OUT || wq == 0);
    HaloItems<CI, NL> items;
    items.init(mma_warp ? 0 : tid, D.L[0]);
    float bias[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) bias[i] = 0.0f;
    if (A.bias && EPI != EPI_DGRAD) {
#pragma unroll
        for (int i = 0; i < 6; ++i)
            if (EPI != EPI_OUT || i < 3) bias[i] = A.bias[c0 + i];
    }
    uint32_t nmma = 0;                            // MMA groups issued (accumulator = nmma & 1)
    const int nunits = *A.nunits;
    bool dead = false;
    for (;;) {
        if (tid == 0) s_unit = atomicAdd(A.work, 1);
        __syncthreads();
        const int ui = s_unit;
        if (ui >= nunits || dead) break;
        const Unit u = A.units[ui];
        load_unit_act<kConvThreads>(D, A.mask, u, act, &s_bits);
        const uint32_t bits = s_bits;
        // depths 0 .. u.nz + 1; prefetch the first kSlots
        const int ndep = u.nz + 2;
        int issued = 0;
        for (; issued < ndep && issued < kSlots; ++issued) {
            if (!mma_warp) load_halo_depth_items<CI, NL>(D, A.in, u, act, issued, rbase + (issued % kSlots) * H::SLOT, items);
            cp_async_commit();
        }
        int prev_k = -1;                          // slab whose epilogue is pending
        uint32_t prev_m = 0;
        for (int k = 0; k <= u.nz && !dead; ++k) {
            const bool have = k < u.nz && ((bits >> k) & 1u);
            if (k < u.nz) {
                // depths k, k+1, k+2 (slices z-1, z, z+1) must have landed
                cp_async_wait(issued - (k + 3) < 0 ? 0 : issued - (k + 3));
                fence_async_smem();
                tc_before_sync();
                __syncthreads();
                tc_after_sync();
                if (have && mma_warp && lane == 0) {
                    const uint32_t dt = tmem + (nmma & 1u) * 32u;
#pragma unroll
                    for (int p = 0; p < 9; ++p) {
                        const int dy = p % 3 - 1, dz = p / 3 - 1;
                        const uint32_t slot = (uint32_t)((k + 1 + dz) % kSlots);
                        const uint64_t a = adesc0 + ((slot * H::SLOT + (uint32_t)(dy + 1) * H::GS) >> 4);
                        const uint64_t b = bdesc0 + ((uint32_t)p * H::QP * NG * 128u >> 4);
#pragma unroll
                        for (int s2 = 0; s2 < H::NKS; ++s2)
                            mma_bf16(dt, a + (uint64_t)(s2 * 16), b + (uint64_t)(s2 * NG * 16), kIdesc,
                                     (p | s2) != 0);
                    }
                    mma_commit(&bars[nmma & 1u]);
                }
            }
            // epilogue of the previous active slab
            if (prev_k >= 0) {
                const uint32_t buf = prev_m & 1u, par = (prev_m >> 1) & 1u;
                const int z = u.z0 + prev_k;
                const int x = u.ox + ex, y = u.oy + ey;
                const bool on = epi && act[((prev_k + 1) * kHaloY + ey + 1) * kHaloX + ex + 1] != 0;
                const int64_t v = on ? vox_index(D, u.b, x, y, z) : 0;
                // operands that do not depend on the MMAs: loaded before the wait
                float pre[6];
                int64_t e = -1;
                double cn[3] = {0.0, 0.0, 0.0};
#pragma unroll
                for (int i = 0; i < 6; ++i) pre[i] = 0.0f;
                if (on) {
                    if (EPI == EPI_DGRAD) {
                        const float2 *zp = reinterpret_cast<const float2 *>(A.zprev + v * 24 + c0);
                        const float2 q0 = zp[0], q1 = zp[1], q2 = zp[2];
                        pre[0] = q0.x; pre[1] = q0.y; pre[2] = q1.x; pre[3] = q1.y; pre[4] = q2.x; pre[5] = q2.y;
                    } else if (EPI == EPI_OUT) {
                        if (A.pred) {
#pragma unroll
                            for (int c = 0; c < 3; ++c) pre[c] = A.f32[v * 3 + c];
                        } else {
                            const BoxGeo &g = *A.geo;
                            const int bx = x - g.lo[0], by = y - g.lo[1], bz = z - g.lo[2];
                            const int32_t t = __ldg(A.tile_index + ((int64_t)(bz >> g.lt[2]) * g.nt[1] + (by >> g.lt[1])) *
                                                                       g.nt[0] + (bx >> g.lt[0]));
                            if (t >= 0) {
                                const int ix = bx & ((1 << g.lt[0]) - 1), iy = by & ((1 << g.lt[1]) - 1),
                                          iz = bz & ((1 << g.lt[2]) - 1);
                                e = ((int64_t)t << (g.lt[0] + g.lt[1] + g.lt[2])) + ix +
                                    ((int64_t)(iy + (iz << g.lt[1])) << g.lt[0]);
                                for (int c = 0; c < A.nspecies && c < 3; ++c) cn[c] = A.field[c][v];
                            }
                        }
                    }
                }
                // one thread waits for the MMAs (the others sleep at the barrier);
                // a wait that gave up ends the whole CTA's work
                bool okw = true;
                if (mma_warp && lane == 0) okw = mbar_wait(&bars[buf], par, A.timeout_ns, A.err);
                dead = !__syncthreads_and(okw);
                tc_after_sync();
                if (!dead && !mma_warp && (EPI != EPI_OUT || wq == 0)) {
                    // columns lo .. lo + 15 of this lane quarter hold channels c0 .. c0 + 5
                    const int lo = c0 & ~7;
                    const uint32_t ta = tmem + buf * 32u + (uint32_t)lo + ((uint32_t)(lq * 32) << 16);
                    float t0[8], t1[8];
                    tmem_ld8(ta, t0);
                    tmem_ld8(ta + 8u, t1);
                    tc_wait_ld();
                    float d[6];
                    switch (wq) {   // warp-uniform: constant register indices in every case
                    case 0: d[0] = t0[0]; d[1] = t0[1]; d[2] = t0[2]; d[3] = t0[3]; d[4] = t0[4]; d[5] = t0[5]; break;
                    case 1: d[0] = t0[6]; d[1] = t0[7]; d[2] = t1[0]; d[3] = t1[1]; d[4] = t1[2]; d[5] = t1[3]; break;
                    case 2: d[0] = t0[4]; d[1] = t0[5]; d[2] = t0[6]; d[3] = t0[7]; d[4] = t1[0]; d[5] = t1[1]; break;
                    default: d[0] = t0[2]; d[1] = t0[3]; d[2] = t0[4]; d[3] = t0[5]; d[4] = t0[6]; d[5] = t0[7]; break;
                    }
                    if (on) {
                        if (EPI == EPI_OUT) {
                            if (A.pred) {
#pragma unroll
                                for (int c = 0; c < 3; ++c) A.pred[v * 3 + c] = pre[c] + A.s_out * (d[c] + bias[c]);
                            } else if (e >= 0) {
                                for (int c = 0; c < A.nspecies && c < 3; ++c) {
                                    const double p = cn[c] + (double)(A.s_out * (d[c] + bias[c]));
                                    A.xs[c][e] = isfinite(p) ? p : cn[c];   // a non-finite guess falls back to c^n
                                }
                            }
                        } else {
                            uint32_t o[3];
                            if (EPI == EPI_GELU) {
                                float zz[6];
#pragma unroll
                                for (int c = 0; c < 6; ++c) zz[c] = d[c] + bias[c];
                                if (A.z_out) {
                                    float2 *zp = reinterpret_cast<float2 *>(A.z_out + v * 24 + c0);
                                    zp[0] = make_float2(zz[0], zz[1]);
                                    zp[1] = make_float2(zz[2], zz[3]);
                                    zp[2] = make_float2(zz[4], zz[5]);
                                }
#pragma unroll
                                for (int c = 0; c < 3; ++c) {
                                    __nv_bfloat162 h = __floats2bfloat162_rn(gelu(zz[2 * c]), gelu(zz[2 * c + 1]));
                                    o[c] = *reinterpret_cast<uint32_t *>(&h);
                                }
                                uint32_t *ap = reinterpret_cast<uint32_t *>(A.a_out + v * 24 + c0);
                                ap[0] = o[0]; ap[1] = o[1]; ap[2] = o[2];
                            } else {   // EPI_DGRAD
#pragma unroll
                                for (int c = 0; c < 3; ++c) {
                                    __nv_bfloat162 h = __floats2bfloat162_rn(d[2 * c] * gelu_grad(pre[2 * c]),
                                                                             d[2 * c + 1] * gelu_grad(pre[2 * c + 1]));
                                    o[c] = *reinterpret_cast<uint32_t *>(&h);
                                }
                                uint32_t *gp = reinterpret_cast<uint32_t *>(A.g_out + v * 24 + c0);
                                gp[0] = o[0]; gp[1] = o[1]; gp[2] = o[2];
                            }
                        }
                    }
                }
                tc_before_sync();
                prev_k = -1;
            }
            if (have) {
                prev_k = k;
                prev_m = nmma;
                nmma += 1;
            }
            // the slot of depth k-1 (read by slabs k-2 .. k-1, whose MMAs every
            // thread has waited for) is refilled with depth k-1+kSlots
            if (!dead && k >= 1 && issued < ndep && issued == k - 1 + kSlots) {
                if (!mma_warp) load_halo_depth_items<CI, NL>(D, A.in, u, act, issued, rbase + (issued % kSlots) * H::SLOT, items);
                cp_async_commit();
                ++issued;
            }
        }
        cp_async_wait(0);
        __syncthreads();
    }
    // leave: all MMAs were waited for (or a wait gave up); free TMEM
    cp_async_wait(0);
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0) tmem_dealloc(tmem, 64);
}

// ---------------------------------------------------------------- weight gradient
// Shared memory of the weight-gradient kernel: the halo ring (its pad column
// q = QC holds ones, so the row block of that column accumulates the bias
// gradient), a guard for the A operand's M overrun, two gradient tiles.
template <int CI, int NO>
struct WgSmem {
    static constexpr int NG = NO / 8;
    static constexpr int RING_OFF = 0;
    static constexpr int RING_BYTES = kSlots * Halo<CI>::SLOT;
    static constexpr int G_OFF = RING_OFF + RING_BYTES + 2048;
    static constexpr int G_BYTES = kSlabY * NG * 128;
    static constexpr int ACT_OFF = G_OFF + 2 * G_BYTES;
    static constexpr int ACT_BYTES = (kZSeg + 2) * kHaloY * kHaloX;
    static constexpr int BAR_OFF = (ACT_OFF + ACT_BYTES + 15) & ~15;
    // more than half an SM's shared memory: one CTA per SM, so a CTA's TMEM
    // allocation never waits for another's
    static constexpr int BYTES = BAR_OFF + 64 > 120 * 1024 ? BAR_OFF + 64 : 120 * 1024;
    static constexpr int TMEM_COLS = 9 * NO <= 256 ? 256 : 512;
};

struct WgradArgs {
    const __nv_bfloat16 *in;        // [B * V][CI] layer input
    const __nv_bfloat16 *g;         // [B * V][GC] dLoss/dz of the layer output
    int32_t gc;                     // channels stored per voxel in g (8 or 24)
    const uint8_t *mask;
    const CnnDom *dom;
    const Unit *units;
    const int32_t *nunits;
    float *partials;                // [gridDim][9][128][NO]
    int32_t *err;
    uint64_t timeout_ns;
};

// Per CTA, over the units i = blockIdx, blockIdx + gridDim, ... (a fixed
// assignment, so the partial sums and their fixed-order reduction are
// reproducible): D_p[m][n] += sum over the slab's voxels v of
// halo_(dy,dz)[v][m] g[v][n] for the nine tap pairs p = (dy, dz), m the row
// (dx copy, channel) of the forward layout's K-columns.
template <int CI, int NO>
__global__ void __launch_bounds__(kThreads, 1) k_wgrad_tc(const __grid_constant__ WgradArgs A)
{
    using H = Halo<CI>;
    using S = WgSmem<CI, NO>;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint32_t s_tmem, s_bits;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + S::BAR_OFF);
    uint8_t *act = sm + S::ACT_OFF;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const CnnDom &D = *A.dom;
    const uint32_t rbase = smem_u32(sm + S::RING_OFF), gbase = smem_u32(sm + S::G_OFF);

    // ring: zeros, ones in the pad column q = QC (CI = 24); gradient tiles: zeros
    for (int i = tid; i < (S::RING_BYTES + 2048) / 16; i += kThreads) {
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        const int off = i * 16;
        if (H::QP > H::QC && off < S::RING_BYTES && ((off % H::GS) / 128) == H::QC)
            w = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);   // bf16 1.0
        reinterpret_cast<uint4 *>(sm + S::RING_OFF)[i] = w;
    }
    for (int i = tid; i < 2 * S::G_BYTES / 16; i += kThreads)
        reinterpret_cast<uint4 *>(sm + S::G_OFF)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) tmem_alloc(&s_tmem, S::TMEM_COLS);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = s_tmem;
    constexpr uint32_t kIdesc = idesc_bf16(128, NO, true, true);
    uint32_t nmma = 0;
    bool ok = true;
    const int nunits = *A.nunits;
    HaloItems<CI, kThreads> items;
    items.init(tid, D.L[0]);
    const int gch = A.gc / 8;                     // real 8-channel chunks of g
    for (int ui = blockIdx.x; ui < nunits && ok; ui += gridDim.x) {
        const Unit u = A.units[ui];
        load_unit_act<kThreads>(D, A.mask, u, act, &s_bits);
        const uint32_t bits = s_bits;
        const int ndep = u.nz + 2;
        int issued = 0;
        for (; issued < ndep && issued < kSlots; ++issued) {
            load_halo_depth_items<CI, kThreads>(D, A.in, u, act, issued, rbase + (issued % kSlots) * H::SLOT, items);
            cp_async_commit();
        }
        for (int k = 0; k < u.nz && ok; ++k) {
            if ((bits >> k) & 1u) {
                const uint32_t m = nmma, buf = m & 1u;
                // the gradient tile buffer was last read by MMA group m - 2
                if (m >= 2 && tid == 0) ok = mbar_wait(&bars[buf], ((m - 2) >> 1) & 1u, A.timeout_ns, A.err);
                ok = __syncthreads_and(ok);
                if (!ok) break;
                // gradient tile of slab k: [y][ng][x][8 channels], zero where inactive
                unsigned char *gt = sm + S::G_OFF + buf * S::G_BYTES;
                for (int i = tid; i < kSlabY * kSlabX * gch; i += kThreads) {
                    const int ch = i % gch, r = i / gch;
                    const int x = r % kSlabX, y = r / kSlabX;
                    uint4 w = make_uint4(0u, 0u, 0u, 0u);
                    if (act[((k + 1) * kHaloY + y + 1) * kHaloX + x + 1])
                        w = __ldg(reinterpret_cast<const uint4 *>(
                            A.g + vox_index(D, u.b, u.ox + x, u.oy + y, u.z0 + k) * A.gc + ch * 8));
                    *reinterpret_cast<uint4 *>(gt + (y * S::NG + ch) * 128 + x * 16) = w;
                }
                cp_async_wait(issued - (k + 3) < 0 ? 0 : issued - (k + 3));
                fence_async_smem();
                tc_before_sync();
                __syncthreads();
                tc_after_sync();
                if (tid == 0) {
                    const uint32_t gb = gbase + buf * S::G_BYTES;
#pragma unroll 1
                    for (int p = 0; p < 9; ++p) {
                        const int dy = p % 3 - 1, dz = p / 3 - 1;
                        const uint32_t slot = (uint32_t)((k + 1 + dz) % kSlots);
                        const uint32_t a0 = rbase + slot * H::SLOT + (uint32_t)(dy + 1) * H::GS;
#pragma unroll
                        for (int s = 0; s < kSlabY / 2; ++s) {
                            const uint64_t ad = sdesc(a0 + 2u * s * H::GS, H::GS, 128u);
                            const uint64_t bd = sdesc(gb + 2u * s * S::NG * 128u, S::NG * 128u, 128u);
                            mma_bf16(tmem + (uint32_t)(p * NO), ad, bd, kIdesc, (m > 0 || s > 0) ? 1u : 0u);
                        }
                    }
                    mma_commit(&bars[buf]);
                }
                nmma = m + 1;
                // every MMA of slabs < k is complete once group m - 1 is: the
                // ring slot of depth k - 1 may then be refilled
                if (m >= 1 && tid == 0) ok = mbar_wait(&bars[(m - 1) & 1u], ((m - 1) >> 1) & 1u, A.timeout_ns, A.err);
                ok = __syncthreads_and(ok);
            } else if (nmma >= 1) {
                if (tid == 0) ok = mbar_wait(&bars[(nmma - 1) & 1u], ((nmma - 1) >> 1) & 1u, A.timeout_ns, A.err);
                ok = __syncthreads_and(ok);
            }
            if (ok && k >= 1 && issued < ndep && issued == k - 1 + kSlots) {
                load_halo_depth_items<CI, kThreads>(D, A.in, u, act, issued, rbase + (issued % kSlots) * H::SLOT, items);
                cp_async_commit();
                ++issued;
            }
        }
        cp_async_wait(0);
        __syncthreads();
    }
    // the last group, then the accumulators to this CTA's partial sums
    if (ok && nmma >= 1 && tid == 0) ok = mbar_wait(&bars[(nmma - 1) & 1u], ((nmma - 1) >> 1) & 1u, A.timeout_ns, A.err);
    ok = __syncthreads_and(ok);
    tc_after_sync();
    const int lq = warp & 3, half = warp >> 2;
    const int row = lq * 32 + lane;
    if (half * 16 < NO) {
        for (int p = 0; p < 9; ++p) {
            float v[16];
            tmem_ld16(tmem + (uint32_t)(p * NO + half * 16) + ((uint32_t)(lq * 32) << 16), v);
            tc_wait_ld();
            float4 *o = reinterpret_cast<float4 *>(A.partials + (((size_t)blockIdx.x * 9 + p) * 128 + row) * NO + half * 16);
            const bool z = nmma == 0 || !ok;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                o[i] = z ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        }
    }
    cp_async_wait(0);
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0) tmem_dealloc(tmem, S::TMEM_COLS);
}

}  // namespace tc
}  // namespace mpm
