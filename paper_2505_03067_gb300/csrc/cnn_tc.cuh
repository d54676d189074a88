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
// Pipeline per CTA (forward kernel).  Loader warps copy halo depths with
// cp.async (16 B, zero-filled for inactive voxels) into a ring of depth
// slots; one warp issues each depth's MMAs (the tap depths folded into N)
// into the accumulators of the slabs it feeds and commits them to
// mbarriers; epilogue warps drain complete slabs (tcgen05.ld) while the
// tensor cores run on.  The weight-gradient kernel runs its own, simpler
// pipeline (kSlots slots, eight warps).
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
// forward kernel: 12 epilogue warps, 6 loader warps and one warp that issues the
// MMAs (19 warps, at most 5 on each SM sub-partition; 96 registers a thread).
// With six loader warps a thread issues 7 halo copies per depth instead of
// 11 with four, whose issue latency held the pipeline back (seven warps gain
// nothing more, five less).
constexpr int kEpiWarps = 12, kLoadWarps = 6;
constexpr int kConvThreads = 32 * (kEpiWarps + kLoadWarps + 1);
constexpr int kFwdSlots = 7;            // halo depths in the forward kernel's ring
// TMEM of the forward kernel: two unit buffers of 256 columns, slab k of a
// unit (k < kZSeg) accumulating in columns NO * (kZSeg - 1 - k) .. + NO of its
// buffer (descending, so the slabs one input depth feeds are adjacent)
constexpr int kTmemBuf = 256;
constexpr int kMaxImages = 16;
// Activity bytes of a unit's halo region (depths z0-1 .. z0+kZSeg, rows
// oy-1 .. oy+16, columns ox-1 .. ox+8: in its image's box and mask set),
// kActStride bytes per unit, and the unit's active slabs (bit k: slab z0+k),
// computed once per network application by k_unit_act.
constexpr int kActBytes = (kZSeg + 2) * kHaloY * kHaloX;
constexpr int kActStride = (kActBytes + 15) & ~15;

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

// The same issued by a converged warp: every lane executes it with the same
// (warp-uniform) operands and one elected lane issues.  Descriptors come as
// their two 32-bit words (the start address and LBO in the low word), so a
// tile offset is one 32-bit add.
__device__ __forceinline__ void mma_bf16_warp(uint32_t d_tmem, uint32_t alo, uint32_t ahi, uint32_t blo, uint32_t bhi,
                                              uint32_t idesc, uint32_t accum)
{
    asm volatile("{\n.reg .pred p, e;\n.reg .b64 a, b;\nelect.sync _|e, 0xffffffff;\nsetp.ne.b32 p, %6, 0;\n"
                 "mov.b64 a, {%1, %2};\nmov.b64 b, {%3, %4};\n"
                 "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %5, p;\n}" ::"r"(d_tmem),
                 "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit_warp(uint64_t *bar)
{
    asm volatile("{\n.reg .pred e;\nelect.sync _|e, 0xffffffff;\n"
                 "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}" ::"r"(smem_u32(bar))
                 : "memory");
}

// Low and high words of a no-swizzle shared-memory descriptor (see sdesc).
__device__ __forceinline__ uint32_t sdesc_lo(uint32_t addr, uint32_t lbo)
{
    return ((addr & 0x3FFFFu) >> 4) | (((lbo >> 4) & 0x3FFFu) << 16);
}
__host__ __device__ constexpr uint32_t sdesc_hi(uint32_t sbo) { return ((sbo >> 4) & 0x3FFFu) | (1u << 14); }

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

// try_wait with a suspend-time hint: the thread sleeps in hardware until the
// phase completes or about `ns` nanoseconds passed, instead of spinning.
__device__ __forceinline__ bool mbar_try_sleep(uint64_t *bar, uint32_t parity, uint32_t ns)
{
    uint32_t ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
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
// Zeros into N consecutive columns of the warp's 32 lanes (tcgen05.st).
__device__ __forceinline__ void tmem_zero8(uint32_t taddr)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr), "r"(0u)
                 : "memory");
}
__device__ __forceinline__ void tmem_zero1(uint32_t taddr)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "r"(0u) : "memory");
}
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tmem_ld1(uint32_t taddr)
{
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    return __uint_as_float(r);
}

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

// 16-byte asynchronous global -> shared copy; src_bytes 0 writes zeros.  The
// copy allocates in L1 (.ca): the three x-shifted halo copies read each
// 16-byte source chunk three times, and the second and third reads hit L1.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
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

// GELU(z) = z Phi(z), Phi(z) = (1 + erf(z / sqrt 2)) / 2, with erf from the
// rational-exponential approximation of Abramowitz & Stegun, Handbook of
// Mathematical Functions, formula 7.1.26 (|error| <= 1.5e-7 for x >= 0):
// erf(x) = 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-x^2), t = 1 / (1 + p x).
// For z < 0, Phi(z) = (1 - erf(|z| / sqrt 2)) / 2.  Far below the bf16 rounding
// of the stored activation (2^-9 relative).
__device__ __forceinline__ float gelu(float z)
{
    const float x = fabsf(z) * 0.70710678118654752f;
    const float t = __frcp_rn(fmaf(0.3275911f, x, 1.0f));
    const float e = exp2f(-1.4426950408889634f * x * x);
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
    const float half_tail = 0.5f * poly * e;   // (1 - erf(x)) / 2
    return z * (z >= 0.0f ? 1.0f - half_tail : half_tail);
}
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

// Weight image of one layer for the forward kernel: for tap row dy, K-column
// q, tap depth dz and output-channel group ng, the 8 x 8 core matrix (rows n =
// ng*8 + r, columns k = q*8 + j) at (((dy+1) * QP + q) * 3 NG + (dz+1) * NG +
// ng) * 128 bytes: the three depths' N blocks are adjacent, so one MMA of N =
// 3 NO applies the taps dz = -1, 0, +1 of an input depth to three output slabs.
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
    static constexpr int RING_BYTES = kFwdSlots * Halo<CI>::SLOT;
    static constexpr int ACT_BYTES = kActStride;
    static constexpr int ACT_OFF = RING_OFF + RING_BYTES;          // two units' activity bytes
    static constexpr int UNIT_OFF = (ACT_OFF + 2 * ACT_BYTES + 15) & ~15;   // two Units + two slab masks
    // mbarriers: full[slots], empty[slots], slab_done[2][kZSeg], tmem_free[2], unit_full[2], unit_empty[2]
    static constexpr int BAR_OFF = (UNIT_OFF + 2 * 32 + 2 * 4 + 15) & ~15;
    static constexpr int NBAR = 2 * kFwdSlots + 2 * kZSeg + 2 + 4;
    // more than half an SM's shared memory: one CTA per SM, so its 512-column
    // TMEM allocation never waits for another CTA's
    static constexpr int BYTES0 = BAR_OFF + NBAR * 8 + 16;
    static constexpr int BYTES = BYTES0 > 120 * 1024 ? BYTES0 : 120 * 1024;
};

enum { EPI_GELU = 0, EPI_OUT = 1, EPI_DGRAD = 2 };

struct ConvArgs {
    const __nv_bfloat16 *in;        // [B * V][CI]
    const uint8_t *mask;            // [B * V]
    const CnnDom *dom;
    const Unit *units;
    const int32_t *nunits;
    const uint8_t *uact;            // [units][kActStride]
    const uint32_t *ubits;          // [units]
    int32_t *work;                  // dynamic scheduling: the next unit (reset by the launch's last CTA)
    int32_t *done;                  //   CTAs finished (reset with it)
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

// The 16-byte copies of one halo depth handled by one loader thread, fixed for
// a launch: the k-th covers item tid + k NL of the depth (halo row yh, copy c,
// channel chunk kc, x row; x fastest, so the eight lanes that fill one core
// matrix write its 128 contiguous bytes -- one shared-memory wavefront, no
// bank conflict -- while a warp still reads the same sectors of the source
// rows); `rel` is its source offset in elements from the depth's halo origin;
// `da` packs its shared offset in the slot (low 16 bits) and its index in a
// depth of the unit's activity bytes (bits 16..23; 255: no item).
template <int CI, int NL>
struct HaloItems {
    static constexpr int N = kHaloY * 3 * kSlabX * (CI / 8);
    static constexpr int K = (N + NL - 1) / NL;
    int32_t rel[K];
    uint32_t da[K];
    __device__ __forceinline__ void init(int tid, int L0)
    {
        using H = Halo<CI>;
        static_assert(kHaloY * kHaloX < 255 && Halo<CI>::SLOT < 65536, "packed halo item");
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = tid + k * NL;
            const int x = i % kSlabX;
            int r = i / kSlabX;
            const int kc = r % H::KC;
            r /= H::KC;
            const int c = r % 3, yh = r / 3;
            const int xh = x + c;
            rel[k] = (yh * L0 + xh) * CI + kc * 8;
            const uint32_t dst = (uint32_t)(yh * H::GS + (c * H::KC + kc) * 128 + x * 16);
            da[k] = dst | ((i < N ? (uint32_t)(yh * kHaloX + xh) : 255u) << 16);
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
        const uint32_t ai = it.da[k] >> 16;
        if (ai == 255u) continue;
        const bool ok = aj[ai] != 0;
        const __nv_bfloat16 *src = ok ? in + (base * CI + it.rel[k]) : in;
        cp_async16(dst + (it.da[k] & 0xFFFFu), src, ok ? 16u : 0u);
    }
}

// One CTA per listed unit (grid-strided): its activity bytes and slab mask.
__global__ void __launch_bounds__(256) k_unit_act(const CnnDom *__restrict__ dom, const uint8_t *__restrict__ mask,
                                                  const Unit *__restrict__ units, const int32_t *__restrict__ nunits,
                                                  uint8_t *__restrict__ uact, uint32_t *__restrict__ ubits)
{
    __shared__ uint32_t s_bits;
    const CnnDom &D = *dom;
    const int nu = *nunits;
    for (int ui = blockIdx.x; ui < nu; ui += gridDim.x) {
        if (threadIdx.x == 0) s_bits = 0u;
        __syncthreads();
        const Unit u = units[ui];
        uint32_t mine = 0u;
        for (int i = threadIdx.x; i < kActStride; i += blockDim.x) {
            uint8_t a = 0;
            if (i < kActBytes) {
                const int xh = i % kHaloX, r = i / kHaloX;
                const int yh = r % kHaloY, j = r / kHaloY;
                const int x = u.ox - 1 + xh, y = u.oy - 1 + yh, z = u.z0 - 1 + j;
                if (in_box(D, u.b, x, y, z)) a = __ldg(mask + vox_index(D, u.b, x, y, z)) != 0;
                if (a && xh >= 1 && xh <= kSlabX && yh >= 1 && yh <= kSlabY && j >= 1 && j <= u.nz)
                    mine |= 1u << (j - 1);
            }
            uact[(size_t)ui * kActStride + i] = a;
        }
        if (mine) atomicOr(&s_bits, mine);
        __syncthreads();
        if (threadIdx.x == 0) ubits[ui] = s_bits;
    }
}

// Copy a unit's activity bytes into shared memory (threads 0..NT-1 of the
// caller's group, one 16-byte load each at most); the caller syncs.
template <int NT>
__device__ __forceinline__ void copy_unit_act(const uint8_t *__restrict__ uact, int ui, uint8_t *act, int t)
{
    const uint4 *src = reinterpret_cast<const uint4 *>(uact + (size_t)ui * kActStride);
    for (int i = t; i < kActStride / 16; i += NT) reinterpret_cast<uint4 *>(act)[i] = __ldg(src + i);
}

// ---------------------------------------------------------------- forward / input-gradient convolution
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar)) : "memory");
}

// Arrive on an mbarrier once every cp.async this thread issued so far has
// landed (the arrival counts toward the phase's expected count).
__device__ __forceinline__ void cp_async_arrive(uint64_t *bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void named_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Bounded wait that also gives up once another role of the CTA gave up (*abort).
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t *bar, uint32_t parity, uint64_t timeout_ns, int32_t *err,
                                                   volatile int32_t *abort)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_sleep(bar, parity, 20000u)) return true;
        if (*abort) return false;
        if (globaltimer_ns() - t0 > timeout_ns) {
            if (err) atomicExch(err, 1);
            *abort = 1;
            return false;
        }
    }
}

// Warp-level bounded wait for phase `parity`: every lane tests the barrier
// (non-blocking) and the warp agrees by a vote, so a phase that is already
// complete costs no divergent branch and no broadcast; otherwise lane 0 waits
// (mbar_wait_or_abort) and broadcasts the outcome.  The whole warp calls it.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, uint32_t parity, uint64_t timeout_ns, int32_t *err,
                                               volatile int32_t *abort)
{
    uint32_t ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    if (__all_sync(0xffffffffu, ok)) return true;
    int w = 1;
    if ((threadIdx.x & 31) == 0) w = mbar_wait_or_abort(bar, parity, timeout_ns, err, abort) ? 1 : 0;
    return __shfl_sync(0xffffffffu, w, 0) != 0;
}

// One persistent CTA per SM over the units i = blockIdx, blockIdx + gridDim,
// ... of the plan's list, as a pipeline of three roles that meet only at
// mbarriers (no CTA-wide barrier in the steady state):
//  - 6 LOADER warps stage, per unit, its activity bytes and slab mask (one of
//    two unit buffers) and then its halo depths into a ring of kFwdSlots
//    slots (cp.async; a slot's mbarrier completes when every loader's copies
//    into it have landed; a slot is refilled once the MMAs that read it
//    completed);
//  - 1 MMA warp (one elected lane) issues, per input depth, 3 tap rows (dy) x
//    (K/16) MMAs of N = up to 3 NO: the depth's halo (the A operand, read
//    once) times the weights of its three tap depths dz, accumulating into
//    the accumulators of the (active) output slabs it feeds, which lie side
//    by side in TMEM and start at zero.  A commit releases the depth's ring
//    slot, and one marks slab j - 2 complete after depth j;
//  - 12 EPILOGUE warps (warp w: TMEM lane quarter w & 3, channels
//    8 (w >> 2) .. 8 (w >> 2) + 7; the output layer: channel w >> 2) drain
//    each complete slab through the epilogue, zero their columns of the
//    unit's TMEM buffer and hand it back.
// NO: MMA N (output channels padded to 16 or 32).
template <int CI, int NO, int EPI>
__global__ void __maxnreg__(96) k_conv_tc(const __grid_constant__ ConvArgs A)
{
    using H = Halo<CI>;
    using S = ConvSmem<CI, NO>;
    constexpr int NG = WImg<CI, NO>::NG;
    constexpr int NE = 32 * kEpiWarps;            // epilogue threads: 0 .. NE-1
    constexpr int NLD = 32 * kLoadWarps;          // loader threads: NE .. NE+NLD-1
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint32_t s_tmem;
    __shared__ int32_t s_abort, s_lstop, s_ui;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + S::BAR_OFF);
    uint64_t *full = bar, *empty = bar + kFwdSlots, *accf = bar + 2 * kFwdSlots, *accu = accf + 2 * kZSeg;
    uint64_t *unitf = accu + 2, *unite = unitf + 2;
    Unit *urec = reinterpret_cast<Unit *>(sm + S::UNIT_OFF);
    uint32_t *ubits = reinterpret_cast<uint32_t *>(sm + S::UNIT_OFF + 64);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const CnnDom &D = *A.dom;
    const uint32_t wbase = smem_u32(sm + S::W_OFF), rbase = smem_u32(sm + S::RING_OFF);
    volatile int32_t *abort = &s_abort;

    // weights into shared memory; zero the ring (pad K-columns stay zero)
    for (int i = tid; i < WImg<CI, NO>::BYTES / 16; i += kConvThreads)
        reinterpret_cast<uint4 *>(sm + S::W_OFF)[i] = __ldg(reinterpret_cast<const uint4 *>(A.wimg) + i);
    for (int i = tid; i < S::RING_BYTES / 16; i += kConvThreads)
        reinterpret_cast<uint4 *>(sm + S::RING_OFF)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) tmem_alloc(&s_tmem, 2 * kTmemBuf);
    if (tid == 0) {
        s_abort = 0;
        s_lstop = 0;
        for (int i = 0; i < kFwdSlots; ++i) {
            mbar_init(&full[i], NLD);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2 * kZSeg; ++i) mbar_init(&accf[i], 1);
        for (int i = 0; i < 2; ++i) mbar_init(&accu[i], kEpiWarps);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&unitf[i], 1);
            mbar_init(&unite[i], kEpiWarps + 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = s_tmem;
    // every accumulator starts at zero: the MMAs always accumulate, and the
    // epilogue zeroes the columns it drained before it hands a buffer back
    if (warp < 4) {
        for (uint32_t c = 0; c < 2 * kTmemBuf; c += 8) tmem_zero8(tmem + c + ((uint32_t)(warp * 32) << 16));
        tc_wait_st();
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    // launched as a programmatic dependent of the previous launch (the layer
    // before): let the next one start its prologue as SMs free up, then wait
    // for the previous one's completion and memory before touching any
    // global data it writes or reads (activations, unit lists, counters)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int nunits = *A.nunits;
    const uint64_t T = A.timeout_ns;

    if (tid >= NE && tid < NE + NLD) {
        // ------------------------------------------------------------ loaders
        // Loader thread 0 alone waits on the mbarriers and publishes the
        // outcome (s_lstop) before a named barrier, so every decision of the
        // loader warps is uniform.
        const int lt = tid - NE;
        HaloItems<CI, NLD> items;
        items.init(lt, D.L[0]);
        // Units are taken from a counter shared by the CTAs (units hold 1..8
        // active slabs, so a fixed assignment leaves CTAs unequally loaded).
        // The next unit's index, activity bytes (one 16-byte share per
        // thread), record and slab mask are fetched a unit ahead, so a unit's
        // start waits on no global round trip; an index past the list is
        // published as the stop record.
        constexpr int kAct16 = kActStride / 16;
        static_assert(kAct16 <= NLD, "one activity share per loader thread");
        const uint4 *uact4 = reinterpret_cast<const uint4 *>(A.uact);
        uint4 actq = make_uint4(0u, 0u, 0u, 0u);
        Unit urow;
        urow.b = urow.ox = urow.oy = urow.z0 = urow.nz = urow.pad0 = urow.pad1 = urow.pad2 = 0;
        uint32_t ubit = 0u;
        if (lt == 0) s_ui = atomicAdd(A.work, 1);
        named_sync(1, NLD);
        int ui = s_ui;
        if (ui < nunits) {
            if (lt < kAct16) actq = __ldg(uact4 + (size_t)ui * kAct16 + lt);
            if (lt == 0) {
                urow = A.units[ui];
                ubit = A.ubits[ui];
            }
        }
        uint32_t dseq = 0;                        // depths issued
        for (int n = 0;; ++n) {
            const int ub = n & 1;
            named_sync(1, NLD);                   // every loader read s_ui
            if (lt == 0) {
                s_ui = ui < nunits ? atomicAdd(A.work, 1) : nunits;
                const bool w = n < 2 || mbar_wait_or_abort(&unite[ub], ((n >> 1) - 1) & 1, T, A.err, abort);
                if (!w || *abort) s_lstop = 1;
            }
            named_sync(1, NLD);
            if (s_lstop) break;
            const int ui_next = s_ui;
            if (ui >= nunits) {
                if (lt == 0) {
                    Unit stop = urow;
                    stop.nz = -1;
                    urec[ub] = stop;
                    mbar_arrive(&unitf[ub]);
                }
                break;
            }
            uint8_t *act = sm + S::ACT_OFF + ub * S::ACT_BYTES;
            if (lt < kAct16) reinterpret_cast<uint4 *>(act)[lt] = actq;
            if (lt == 0) {
                ubits[ub] = ubit;
                urec[ub] = urow;
            }
            named_sync(1, NLD);
            if (lt == 0) mbar_arrive(&unitf[ub]);
            const Unit u = urec[ub];
            if (ui_next < nunits) {
                if (lt < kAct16) actq = __ldg(uact4 + (size_t)ui_next * kAct16 + lt);
                if (lt == 0) {
                    urow = A.units[ui_next];
                    ubit = A.ubits[ui_next];
                }
            }
            ui = ui_next;
            for (int j = 0; j < u.nz + 2; ++j) {
                const uint32_t slot = dseq % kFwdSlots, use = dseq / kFwdSlots;
                if (lt == 0 && use >= 1 && !mbar_wait_or_abort(&empty[slot], (use - 1) & 1, T, A.err, abort))
                    s_lstop = 1;
                named_sync(1, NLD);
                if (s_lstop) break;
                load_halo_depth_items<CI, NLD>(D, A.in, u, act, j, rbase + slot * H::SLOT, items);
                cp_async_arrive(&full[slot]);   // completes the slot's phase once the copies land
                ++dseq;
            }
            if (s_lstop) break;
        }
        cp_async_wait(0);
    } else if (warp == kEpiWarps + kLoadWarps) {
        // ------------------------------------------------------------ MMA issue
        // The whole warp runs this loop on warp-uniform values (shared-memory
        // reads broadcast from lane 0), and one elected lane issues each
        // tcgen05 instruction: operands the compiler can keep in uniform
        // registers let the MMAs issue back to back.
        constexpr uint32_t kId1 = idesc_bf16(128, NO, false, false), kId2 = idesc_bf16(128, 2 * NO, false, false),
                           kId3 = idesc_bf16(128, 3 * NO, false, false);
        const uint32_t tm = __shfl_sync(0xffffffffu, tmem, 0);
        const uint32_t alo0 = sdesc_lo(rbase, 128u), blo0 = sdesc_lo(wbase, 3u * NG * 128u);
        constexpr uint32_t ahi = sdesc_hi(H::GS), bhi = sdesc_hi(128u);
        uint32_t dbase = 0;
        bool ok = true;
        for (int n = 0; ok; ++n) {
            const int ub = n & 1;
            ok = mbar_wait_warp(&unitf[ub], (n >> 1) & 1, T, A.err, abort);
            if (!ok) break;
            const int nz = __shfl_sync(0xffffffffu, urec[ub].nz, 0);
            if (nz < 0) break;                    // the stop record
            const uint32_t bits = __shfl_sync(0xffffffffu, ubits[ub], 0);
            // the unit's TMEM buffer is free once the epilogue drained unit n - 2
            ok = n < 2 || mbar_wait_warp(&accu[ub], ((n >> 1) - 1) & 1, T, A.err, abort);
            if (!ok) break;
            tc_after_sync();
            const uint32_t cbuf = tm + (uint32_t)ub * kTmemBuf;
            for (int j = 0; j < nz + 2; ++j) {
                const uint32_t d = dbase + j, slot = d % kFwdSlots;
                ok = mbar_wait_warp(&full[slot], (d / kFwdSlots) & 1, T, A.err, abort);
                if (!ok) break;
                fence_async_smem();
                tc_after_sync();
                // depth j feeds slabs j (tap dz = -1), j - 1 (dz = 0), j - 2 (dz = +1):
                // the active ones among them, hi .. lo (descending)
                const uint32_t win = (bits & ((1u << nz) - 1u)) >> (j >= 2 ? j - 2 : 0);
                const uint32_t sel = win & (j >= 2 ? 7u : (j == 1 ? 3u : 1u));
                if (sel) {
                    const int base = j >= 2 ? j - 2 : 0;
                    const int hi = base + 31 - __clz(sel), lo = base + __ffs(sel) - 1;
                    const int nsl = hi - lo + 1;
                    const uint32_t idn = nsl == 3 ? kId3 : (nsl == 2 ? kId2 : kId1);
                    const uint32_t dacc = cbuf + (uint32_t)(NO * (kZSeg - 1 - hi));
                    const uint32_t alo = alo0 + slot * (uint32_t)(H::SLOT >> 4);
                    const uint32_t blo = blo0 + (uint32_t)((j - hi) * NG * 8);
                    // the accumulators start at zero (see the epilogue), so every MMA accumulates
#pragma unroll
                    for (int t = 0; t < 3 * H::NKS; ++t) {
                        const int dyi = t / H::NKS, s2 = t % H::NKS;
                        // A: halo row dyi, K-columns 2 s2 .. 2 s2 + 1; B: core matrix (dy, q = 2 s2, dz block j - hi, ng 0)
                        mma_bf16_warp(dacc, alo + (uint32_t)((dyi * H::GS) >> 4) + (uint32_t)(s2 * 16), ahi,
                                      blo + (uint32_t)((dyi * H::QP + 2 * s2) * 3 * NG * 8), bhi, idn, 1u);
                    }
                }
                mma_commit_warp(&empty[slot]);          // no later MMA reads this depth
                if (j >= 2 && j - 2 < nz) mma_commit_warp(&accf[ub * kZSeg + (j - 2)]);   // slab j - 2 complete
            }
            if (!ok) break;
            // one completion per buffer use for every slab barrier
            for (int k = nz; k < kZSeg; ++k) mma_commit_warp(&accf[ub * kZSeg + k]);
            dbase += nz + 2;
            if (lane == 0) mbar_arrive(&unite[ub]);
            __syncwarp();
        }
        __syncwarp();
    } else if (tid < NE) {
        // ------------------------------------------------------------ epilogue
        const int lq = warp & 3, wq = warp >> 2;
        const int row = lq * 32 + lane;           // voxel (row & 7, row >> 3) of the slab
        const int ex = row & 7, ey = row >> 3;
        // first channel of this thread: 8 channels per warp group; the output
        // layer's three channels go one to each warp group (channel wq)
        const int c0 = EPI == EPI_OUT ? wq : 8 * wq;
        // (image mode writes all three predicted channels, solver mode the species')
        const bool reads = EPI != EPI_OUT || wq < (A.pred ? 3 : (A.nspecies < 3 ? A.nspecies : 3));
        float bias[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) bias[i] = 0.0f;
        if (A.bias && EPI != EPI_DGRAD) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (EPI != EPI_OUT || i == 0) bias[i] = A.bias[c0 + i];
        }
        bool ok = true;
        for (int n = 0; ok; ++n) {
            const int ub = n & 1;
            if (lane == 0) ok = mbar_wait_or_abort(&unitf[ub], (n >> 1) & 1, T, A.err, abort);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) break;
            const Unit u = urec[ub];
            if (u.nz < 0) break;                  // the stop record
            const uint32_t bits = ubits[ub];
            const uint8_t *act = sm + S::ACT_OFF + ub * S::ACT_BYTES;
            for (int k = 0; k < u.nz && ok; ++k) {
                if (!((bits >> k) & 1u)) continue;
                const int z = u.z0 + k, x = u.ox + ex, y = u.oy + ey;
                const bool on = reads && act[((k + 1) * kHaloY + ey + 1) * kHaloX + ex + 1] != 0;
                const int64_t v = on ? vox_index(D, u.b, x, y, z) : 0;
                // operands that do not depend on the MMAs: loaded before the wait
                float pre[8];
                int64_t e = -1;
                double cn[3] = {0.0, 0.0, 0.0};
#pragma unroll
                for (int i = 0; i < 8; ++i) pre[i] = 0.0f;
                if (on) {
                    if (EPI == EPI_DGRAD) {
                        const float4 *zp = reinterpret_cast<const float4 *>(A.zprev + v * 24 + c0);
                        const float4 q0 = zp[0], q1 = zp[1];
                        pre[0] = q0.x; pre[1] = q0.y; pre[2] = q0.z; pre[3] = q0.w;
                        pre[4] = q1.x; pre[5] = q1.y; pre[6] = q1.z; pre[7] = q1.w;
                    } else if (EPI == EPI_OUT) {
                        if (A.pred) {
                            pre[0] = A.f32[v * 3 + c0];
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
                                cn[0] = A.field[c0][v];
                            }
                        }
                    }
                }
                ok = mbar_wait_warp(&accf[ub * kZSeg + k], (n >> 1) & 1, T, A.err, abort);
                if (!ok) break;
                tc_after_sync();
                float d[8];
                if (reads) {
                    const uint32_t ta = tmem + (uint32_t)ub * kTmemBuf + (uint32_t)(NO * (kZSeg - 1 - k)) + (uint32_t)c0 +
                                        ((uint32_t)(lq * 32) << 16);
                    if (EPI == EPI_OUT)
                        d[0] = tmem_ld1(ta);
                    else
                        tmem_ld8(ta, d);
                    tc_wait_ld();
                }
                if (on) {
                    if (EPI == EPI_OUT) {
                        if (A.pred) {
                            A.pred[v * 3 + c0] = pre[0] + A.s_out * (d[0] + bias[0]);
                        } else if (e >= 0) {
                            const double p = cn[0] + (double)(A.s_out * (d[0] + bias[0]));
                            A.xs[c0][e] = isfinite(p) ? p : cn[0];   // a non-finite guess falls back to c^n
                        }
                    } else {
                        uint32_t o[4];
                        if (EPI == EPI_GELU) {
                            float zz[8];
#pragma unroll
                            for (int c = 0; c < 8; ++c) zz[c] = d[c] + bias[c];
                            if (A.z_out) {
                                float4 *zp = reinterpret_cast<float4 *>(A.z_out + v * 24 + c0);
                                zp[0] = make_float4(zz[0], zz[1], zz[2], zz[3]);
                                zp[1] = make_float4(zz[4], zz[5], zz[6], zz[7]);
                            }
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                __nv_bfloat162 h = __floats2bfloat162_rn(gelu(zz[2 * c]), gelu(zz[2 * c + 1]));
                                o[c] = *reinterpret_cast<uint32_t *>(&h);
                            }
                            *reinterpret_cast<uint4 *>(A.a_out + v * 24 + c0) = make_uint4(o[0], o[1], o[2], o[3]);
                        } else {   // EPI_DGRAD
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                __nv_bfloat162 h = __floats2bfloat162_rn(d[2 * c] * gelu_grad(pre[2 * c]),
                                                                         d[2 * c + 1] * gelu_grad(pre[2 * c + 1]));
                                o[c] = *reinterpret_cast<uint32_t *>(&h);
                            }
                            *reinterpret_cast<uint4 *>(A.g_out + v * 24 + c0) = make_uint4(o[0], o[1], o[2], o[3]);
                        }
                    }
                }
            }
            // zero this warp's accumulator columns of every slab of the buffer
            // (every MMA accumulates; unit n + 2 starts from these zeros): all
            // MMAs into the buffer completed with its last active slab
            if (ok) {
                const uint32_t tq = tmem + (uint32_t)ub * kTmemBuf + (uint32_t)c0 + ((uint32_t)(lq * 32) << 16);
#pragma unroll
                for (int k = 0; k < kZSeg; ++k) {
                    if (EPI == EPI_OUT)
                        tmem_zero1(tq + (uint32_t)(NO * (kZSeg - 1 - k)));
                    else
                        tmem_zero8(tq + (uint32_t)(NO * (kZSeg - 1 - k)));
                }
                tc_wait_st();
            }
            // this warp is done with the unit's TMEM buffer, activity bytes and records
            tc_before_sync();
            __syncwarp();
            if (ok && lane == 0) {
                mbar_arrive(&accu[ub]);
                mbar_arrive(&unite[ub]);
            }
        }
    }
    // leave: every role finished (or gave up); free TMEM
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0) tmem_dealloc(tmem, 2 * kTmemBuf);
    // the launch's last CTA resets the unit counter for the next launch
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(A.done, 1) == (int)gridDim.x - 1) {
            *A.work = 0;
            *A.done = 0;
            __threadfence();
        }
    }
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
    static constexpr int ACT_BYTES = kActStride;
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
    const uint8_t *uact;            // [units][kActStride]
    const uint32_t *ubits;          // [units]
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
    __shared__ uint32_t s_tmem;
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
        copy_unit_act<kThreads>(A.uact, ui, act, tid);
        __syncthreads();
        const uint32_t bits = A.ubits[ui];
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
