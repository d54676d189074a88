// api.cu -- the C ABI of include/mpm.h: context and subgrid lifetime, memory
// accounting, error plumbing.  No exception crosses the ABI; every entry
// point returns an mpm_status and records a message on the context.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>

#include "mpm_internal.cuh"

mpm_status mpm_fail(mpm_ctx *ctx, mpm_status st, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return st;
}

mpm_status mpm_cuda_check(mpm_ctx *ctx, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return MPM_OK;
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return mpm_fail(ctx, MPM_ERR_NOMEM, m);
    return mpm_fail(ctx, MPM_ERR_CUDA, m);
}

// Grow-only device buffer under the context's cap; the old contents are not kept.
mpm_status mpm_grow(mpm_ctx *ctx, void **p, size_t *cap, size_t need, const char *what)
{
    if (need <= *cap && *p) return MPM_OK;
    size_t want = need + need / 4 + 4096;     // head-room for growing boxes
    if (ctx->cap && ctx->allocated - *cap + want > ctx->cap) {
        want = need;
        if (ctx->allocated - *cap + want > ctx->cap)
            return mpm_fail(ctx, MPM_ERR_NOMEM, std::string(what) + ": workspace cap exceeded");
    }
    if (*p) {
        cudaError_t e = cudaFree(*p);
        if (e != cudaSuccess) return mpm_cuda_check(ctx, e, "cudaFree");
        ctx->allocated -= *cap;
        *p = nullptr;
        *cap = 0;
    }
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return mpm_fail(ctx, MPM_ERR_NOMEM, std::string(what) + ": cudaMalloc of " + std::to_string(want) + " bytes failed");
    }
    *p = q;
    *cap = want;
    ctx->allocated += want;
    return MPM_OK;
}

static void free_sub_buffers(mpm_ctx *ctx, mpm_subgrid *sub)
{
    mpm_step_free(ctx, sub);
    void **bufs[3] = {&sub->geo, &sub->elem, &sub->krylov};
    size_t *caps[3] = {&sub->geo_bytes, &sub->elem_bytes, &sub->krylov_bytes};
    for (int i = 0; i < 3; ++i) {
        if (*bufs[i]) {
            cudaFree(*bufs[i]);
            if (ctx) ctx->allocated -= *caps[i];
        }
        *bufs[i] = nullptr;
        *caps[i] = 0;
    }
}

namespace mpm {
// The bit-level conversions of the FP32 Krylov path, applied elementwise
// (test hook: mpm_debug_convert).
// CUDA's own conversions (round toward zero, and the exact widening) are
// written beside them as the reference.
__global__ void k_debug_convert(const double *__restrict__ in64, float *__restrict__ out32,
                                float *__restrict__ ref32, const float *__restrict__ in32,
                                double *__restrict__ out64, double *__restrict__ ref64, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        out32[i] = f32_rz(in64[i]);
        ref32[i] = __double2float_rz(in64[i]);
        out64[i] = f64_of(in32[i]);
        ref64[i] = (double)in32[i];
    }
}

// The voxels a step updated -- the in-mask voxels of its box -- of every
// field into host fields the device addresses directly (page-locked host
// memory): one box row per CTA iteration, the row's in-mask voxels only.
struct HostBack {
    const double *src[MPM_MAX_SPECIES];
    double *dst[MPM_MAX_SPECIES];
    int32_t n;
};

__global__ void __launch_bounds__(256) k_box_mask_to_host(const uint8_t *__restrict__ mask, HostBack o, int64_t nx,
                                                          int64_t ny, int32_t x0, int32_t y0, int32_t z0, int32_t bx,
                                                          int32_t by, int32_t bz)
{
    const int64_t rows = (int64_t)by * bz;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const int64_t y = y0 + r % by, z = z0 + r / by;
        const int64_t off = (z * ny + y) * nx + x0;
        for (int32_t i = threadIdx.x; i < bx; i += blockDim.x) {
            if (!mask[off + i]) continue;
            for (int s = 0; s < o.n; ++s)
                if (o.dst[s]) o.dst[s][off + i] = o.src[s][off + i];
        }
    }
}
}  // namespace mpm

extern "C" {

mpm_status mpm_create(mpm_ctx **out, size_t workspace_bytes)
{
    if (!out) return MPM_ERR_ARG;
    *out = nullptr;
    mpm_ctx *ctx = new (std::nothrow) mpm_ctx();
    if (!ctx) return MPM_ERR_NOMEM;
    ctx->cap = workspace_bytes;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    int coop = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
    if (e == cudaSuccess && !coop) e = cudaErrorNotSupported;
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_box, 256);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_count, 256);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_err, 256);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_abort, 256);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, 256);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_abort, 0, 256);
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_stage, 1 << 16);
    if (e == cudaSuccess) ctx->stage_cap = 1 << 16;
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        mpm_destroy(ctx);
        return MPM_ERR_CUDA;
    }
    *out = ctx;
    return MPM_OK;
}

mpm_status mpm_destroy(mpm_ctx *ctx)
{
    if (!ctx) return MPM_ERR_ARG;
    mpm_batch_graph_free(ctx);
    mpm_fgmres_release(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    cudaFree(ctx->d_box);
    cudaFree(ctx->d_count);
    cudaFree(ctx->d_err);
    cudaFree(ctx->d_abort);
    cudaFree(ctx->d_partials);
    cudaFree(ctx->d_bar);
    cudaFree(ctx->d_args);
    cudaFree(ctx->d_tmp);
    cudaFree(ctx->d_fg);
    cudaFree(ctx->d_cpm);
    cudaFree(ctx->d_prof);
    cudaFree(ctx->d_tune);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    delete ctx;
    return MPM_OK;
}

const char *mpm_last_error(const mpm_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : "null context";
}

mpm_status mpm_subgrid_create(mpm_ctx *ctx, mpm_subgrid **sub)
{
    if (!ctx || !sub) return mpm_fail(ctx, MPM_ERR_ARG, "subgrid_create: null argument");
    *sub = new (std::nothrow) mpm_subgrid();
    return *sub ? MPM_OK : mpm_fail(ctx, MPM_ERR_NOMEM, "subgrid_create: out of host memory");
}

mpm_status mpm_subgrid_destroy(mpm_ctx *ctx, mpm_subgrid *sub)
{
    if (!sub) return mpm_fail(ctx, MPM_ERR_ARG, "subgrid_destroy: null subgrid");
    free_sub_buffers(ctx, sub);
    delete sub;
    return MPM_OK;
}

mpm_status mpm_subgrid_info(const mpm_subgrid *sub, mpm_subgrid_desc *out)
{
    if (!sub || !out) return MPM_ERR_ARG;
    memset(out, 0, sizeof(*out));
    if (!sub->extracted) return MPM_ERR_ARG;
    for (int d = 0; d < 3; ++d) {
        out->box.lo[d] = sub->lo[d];
        out->box.hi[d] = sub->hi[d];
        out->n[d] = sub->n[d];
        out->tile[d] = 1 << sub->lt[d];
    }
    out->ntiles = sub->ntiles;
    out->nactive = sub->nact;
    out->stored_voxels = sub->NE;
    out->mask_voxels = sub->mask_voxels;
    out->nspecies = sub->nspecies;
    return MPM_OK;
}

mpm_status mpm_box_extract(mpm_ctx *ctx, const mpm_lattice *lat, int32_t nspecies, int32_t margin,
                           const int32_t tile[3], mpm_box *out_box, mpm_subgrid *sub, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    return mpm_extract_impl(ctx, lat, nspecies, margin, tile, out_box, sub, (cudaStream_t)stream);
}

mpm_status mpm_subgrid_refresh(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_lattice *lat, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    return mpm_refresh_impl(ctx, sub, lat, (cudaStream_t)stream);
}

mpm_status mpm_assemble_coeffs(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_params *prm, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    return mpm_assemble_impl(ctx, sub, prm, (cudaStream_t)stream);
}

mpm_status mpm_solve_step(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_lattice *scatter_to, const mpm_opts *opt,
                          mpm_report *rep, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    mpm_subgrid *subs[1] = {sub};
    const mpm_lattice *sc[1] = {scatter_to};
    return mpm_solve_impl(ctx, subs, sc, 1, opt, rep, (cudaStream_t)stream);
}

mpm_status mpm_solve_batch(mpm_ctx *ctx, mpm_subgrid *const *subs, const mpm_lattice *const *scatter_to,
                           int32_t nsys, const mpm_opts *opt, mpm_report *reps, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    return mpm_solve_impl(ctx, subs, scatter_to, nsys, opt, reps, (cudaStream_t)stream);
}

mpm_status mpm_batch_step(mpm_ctx *ctx, mpm_subgrid *const *subs, const mpm_lattice *const *lats,
                          const mpm_params *const *prms, int32_t nsys, const mpm_opts *opt, mpm_report *reps,
                          void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    return mpm_batch_step_impl(ctx, subs, lats, prms, nsys, opt, reps, (cudaStream_t)stream);
}

mpm_status mpm_step(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_lattice *lat, const mpm_params *prm, int32_t margin,
                    const int32_t tile[3], const mpm_opts *opt, mpm_report *rep, mpm_box *out_box, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    return mpm_step_impl(ctx, sub, lat, prm, margin, tile, opt, rep, out_box, (cudaStream_t)stream);
}

mpm_status mpm_step_enqueue(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_lattice *lat, const mpm_params *prm,
                            int32_t margin, const int32_t tile[3], const mpm_opts *opt, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    return mpm_step_enqueue_impl(ctx, sub, lat, prm, margin, tile, opt, (cudaStream_t)stream);
}

mpm_status mpm_step_wait(mpm_ctx *ctx, mpm_subgrid *sub, mpm_report *rep, mpm_box *out_box, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    return mpm_step_wait_impl(ctx, sub, rep, out_box, (cudaStream_t)stream);
}

mpm_status mpm_step_set_network(mpm_ctx *ctx, mpm_subgrid *sub, mpm_cnn *cnn)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    return mpm_step_set_network_impl(ctx, sub, cnn);
}

mpm_status mpm_step_host(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_host_lattice *host, const mpm_lattice *dev,
                         const mpm_params *prm, int32_t margin, const int32_t tile[3], const mpm_opts *opt,
                         int32_t flags, mpm_report *rep, mpm_box *out_box, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    if (!host || !dev || !prm) return mpm_fail(ctx, MPM_ERR_ARG, "step_host: null argument");
    if (flags & ~MPM_HOST_FIELDS_IN) return mpm_fail(ctx, MPM_ERR_ARG, "step_host: unknown flag");
    if (prm->nspecies < 1 || prm->nspecies > MPM_MAX_SPECIES)
        return mpm_fail(ctx, MPM_ERR_ARG, "step_host: nspecies out of range");
    for (int d = 0; d < 3; ++d)
        if (dev->dims[d] < 1) return mpm_fail(ctx, MPM_ERR_ARG, "step_host: lattice dims must be positive");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nx = (size_t)dev->dims[0], ny = (size_t)dev->dims[1], nz = (size_t)dev->dims[2];
    const size_t nvox = nx * ny * nz;
    // the device lattice's buffers are the caller's; this call overwrites them
    if (host->cell_id) {
        if (!dev->cell_id) return mpm_fail(ctx, MPM_ERR_ARG, "step_host: null device cell ids");
        MPM_CU(cudaMemcpyAsync((void *)dev->cell_id, host->cell_id, nvox * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    }
    if (host->mask) {
        if (!dev->mask) return mpm_fail(ctx, MPM_ERR_ARG, "step_host: null device mask");
        MPM_CU(cudaMemcpyAsync((void *)dev->mask, host->mask, nvox, cudaMemcpyHostToDevice, st));
    }
    if (flags & MPM_HOST_FIELDS_IN)
        for (int s = 0; s < prm->nspecies; ++s)
            if (host->field[s] && dev->field[s])
                MPM_CU(cudaMemcpyAsync(dev->field[s], host->field[s], nvox * sizeof(double), cudaMemcpyHostToDevice, st));
    mpm_box box = {{0, 0, 0}, {0, 0, 0}};
    const mpm_status r = mpm_step_impl(ctx, sub, dev, prm, margin, tile, opt, rep, &box, st);
    if (out_box && (r == MPM_OK || r == MPM_ERR_NOCONV || r == MPM_ERR_BREAKDOWN)) *out_box = box;
    if (r != MPM_OK && r != MPM_ERR_NOCONV && r != MPM_ERR_BREAKDOWN) return r;
    // the step's results back to the host.  A host field the device can
    // address (page-locked) receives the in-mask voxels of the box from a
    // kernel -- the only voxels the step wrote, a tenth of the box on a thin
    // shell -- any other one the whole box by a 3-D copy (rows of nx doubles).
    const bool has_box = box.hi[0] > box.lo[0] && box.hi[1] > box.lo[1] && box.hi[2] > box.lo[2];
    mpm::HostBack hb;
    memset(&hb, 0, sizeof(hb));
    hb.n = prm->nspecies;
    bool pageable[MPM_MAX_SPECIES] = {};
    bool any_mapped = false;
    for (int s = 0; s < prm->nspecies && has_box; ++s) {
        if (!host->field[s] || !dev->field[s]) continue;
        cudaPointerAttributes pa;
        memset(&pa, 0, sizeof(pa));
        if (cudaPointerGetAttributes(&pa, host->field[s]) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer) {
            hb.src[s] = dev->field[s];
            hb.dst[s] = (double *)pa.devicePointer;
            any_mapped = true;
        } else {
            cudaGetLastError();
            pageable[s] = true;
        }
    }
    if (any_mapped) {
        const int32_t bx = box.hi[0] - box.lo[0], by = box.hi[1] - box.lo[1], bz = box.hi[2] - box.lo[2];
        mpm::k_box_mask_to_host<<<ctx->num_sms * 8, 256, 0, st>>>(dev->mask, hb, (int64_t)nx, (int64_t)ny, box.lo[0],
                                                                 box.lo[1], box.lo[2], bx, by, bz);
        ctx->launches += 1;
        MPM_CU(cudaGetLastError());
    }
    for (int s = 0; s < prm->nspecies; ++s) {
        if (!pageable[s]) continue;
        cudaMemcpy3DParms p = {};
        p.srcPtr = make_cudaPitchedPtr(dev->field[s], nx * sizeof(double), nx, ny);
        p.dstPtr = make_cudaPitchedPtr(host->field[s], nx * sizeof(double), nx, ny);
        p.srcPos = make_cudaPos((size_t)box.lo[0] * sizeof(double), (size_t)box.lo[1], (size_t)box.lo[2]);
        p.dstPos = p.srcPos;
        p.extent = make_cudaExtent((size_t)(box.hi[0] - box.lo[0]) * sizeof(double), (size_t)(box.hi[1] - box.lo[1]),
                                   (size_t)(box.hi[2] - box.lo[2]));
        p.kind = cudaMemcpyDeviceToHost;
        MPM_CU(cudaMemcpy3DAsync(&p, st));
    }
    MPM_CU(cudaStreamSynchronize(st));
    return r;
}

mpm_status mpm_solve_fgmres_cnn(mpm_ctx *ctx, mpm_cnn *cnn, mpm_subgrid *sub, const mpm_lattice *lat,
                                const mpm_params *prm, const mpm_lattice *scatter_to, const mpm_opts *opt,
                                mpm_report *rep, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    return mpm_solve_fgmres_impl(ctx, cnn, sub, lat, prm, scatter_to, opt, rep, (cudaStream_t)stream);
}

mpm_status mpm_subgrid_export(mpm_ctx *ctx, const mpm_subgrid *sub, int32_t what, int32_t s, void *dst, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    return mpm_export_impl(ctx, sub, what, s, dst, (cudaStream_t)stream);
}

mpm_status mpm_subgrid_import(mpm_ctx *ctx, mpm_subgrid *sub, int32_t s, const double *src, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    return mpm_import_impl(ctx, sub, s, src, (cudaStream_t)stream);
}

mpm_status mpm_apply_operator(mpm_ctx *ctx, const mpm_subgrid *sub, int32_t s, const double *x, double *y,
                              void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    return mpm_apply_impl(ctx, sub, s, x, y, (cudaStream_t)stream);
}

mpm_status mpm_scatter(mpm_ctx *ctx, const mpm_subgrid *sub, const mpm_lattice *lat, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    return mpm_scatter_impl(ctx, sub, lat, (cudaStream_t)stream);
}

mpm_status mpm_debug_set(mpm_ctx *ctx, int32_t key, int64_t value)
{
    if (!ctx) return MPM_ERR_ARG;
    switch (key) {
    case MPM_DEBUG_TIMEOUT_NS:
        if (value <= 0) return mpm_fail(ctx, MPM_ERR_ARG, "debug: timeout must be > 0");
        ctx->timeout_ns = (uint64_t)value;
        return MPM_OK;
    case MPM_DEBUG_SKIP_BLOCK:
        ctx->skip_block = (int32_t)value;
        return MPM_OK;
    case MPM_DEBUG_PHASE_TIMES:
        ctx->phase_prof = value != 0;
        return MPM_OK;
    case MPM_DEBUG_SOLVER_VARIANT:
        if (value < 0 || value > 6) return mpm_fail(ctx, MPM_ERR_ARG, "debug: solver variant out of [0, 6]");
        ctx->solver_variant = (int32_t)value;
        return MPM_OK;
    case MPM_DEBUG_CNN_LAYER_TIMES:
        ctx->cnn_layer_prof = value != 0;
        return MPM_OK;
    default:
        return mpm_fail(ctx, MPM_ERR_ARG, "debug: unknown key");
    }
}

mpm_status mpm_debug_convert(const double *in64, float *out32, float *ref32, const float *in32, double *out64,
                             double *ref64, int64_t n, void *stream)
{
    if (n < 0 || (n > 0 && (!in64 || !out32 || !ref32 || !in32 || !out64 || !ref64))) return MPM_ERR_ARG;
    if (n == 0) return MPM_OK;
    const int nb = (int)std::min<int64_t>((n + 255) / 256, 4096);
    mpm::k_debug_convert<<<nb, 256, 0, (cudaStream_t)stream>>>(in64, out32, ref32, in32, out64, ref64, n);
    return cudaGetLastError() == cudaSuccess ? MPM_OK : MPM_ERR_CUDA;
}

mpm_status mpm_counter_get(const mpm_ctx *ctx, int32_t key, int64_t *value)
{
    if (!ctx || !value) return MPM_ERR_ARG;
    if (key == MPM_COUNTER_LAUNCHES) { *value = ctx->launches; return MPM_OK; }
    if (key == MPM_COUNTER_BATCH_GRAPH) { *value = mpm_batch_graph_active((mpm_ctx *)ctx); return MPM_OK; }
    if (key == MPM_COUNTER_IMBALANCE_PPM) { *value = (int64_t)(ctx->last_imbalance * 1e6 + 0.5); return MPM_OK; }
    if (key == MPM_COUNTER_PHASE_WORK_NS) {
        *value = (int64_t)(ctx->h_prof[4] + ctx->h_prof[5] + ctx->h_prof[6] + ctx->h_prof[7]);
        return MPM_OK;
    }
    if (key >= MPM_COUNTER_PHASE_WAIT_NS && key <= MPM_COUNTER_PHASE_SERIAL_NS) {
        *value = (int64_t)ctx->h_prof[key - MPM_COUNTER_PHASE_WORK_NS];
        return MPM_OK;
    }
    if (key >= MPM_COUNTER_PHASE_BBOX_NS && key <= MPM_COUNTER_PHASE_GATHER_NS) {
        *value = (int64_t)ctx->h_prof[10 + key - MPM_COUNTER_PHASE_BBOX_NS];
        return MPM_OK;
    }
    if (key == MPM_COUNTER_PHASE_EXTRACT_NS || key == MPM_COUNTER_PHASE_SCATTER_NS) {
        *value = (int64_t)ctx->h_prof[key == MPM_COUNTER_PHASE_EXTRACT_NS ? 8 : 9];
        return MPM_OK;
    }
    if (key >= MPM_COUNTER_PHASE_R_NS && key <= MPM_COUNTER_PHASE_U_NS) {
        *value = (int64_t)ctx->h_prof[4 + key - MPM_COUNTER_PHASE_R_NS];
        return MPM_OK;
    }
    if (key == MPM_COUNTER_STEP_FULL_EXTRACTIONS) { *value = ctx->step_nfull; return MPM_OK; }
    return MPM_ERR_ARG;
}

}  // extern "C"
