// fgmres.cu -- row a13: the implicit-Euler step of Eq. 1-4 on the box solved by
// right-preconditioned flexible GMRES with the network as the preconditioner.
//
// Arnoldi runs on A z_j with z_j = M(v_j), M the network applied to the
// vector (mpm_cnn_precond_impl); modified Gram-Schmidt, Givens rotations on
// the host, the update x += Z y from the preconditioned directions, and
// restarts from the true FP64 residual -- the algorithm of the oracle's
// fgmres, in FP64 on the device.  The scalars of one Arnoldi step (the
// projections and the new norm) stay in device memory until the step ends,
// so each step waits for the device once.  This path is not the fast one: a
// network application costs several Arnoldi steps of the plain solver.
#include <cmath>
#include <cstring>
#include <vector>

#include "mpm_internal.cuh"

mpm_status mpm_cnn_precond_impl(mpm_ctx *ctx, mpm_cnn *c, mpm_subgrid *sub, const mpm_lattice *lat,
                                const mpm_params *prm, int s, const double *v, double *z, double *d_scale,
                                cudaStream_t st);
mpm_status mpm_apply_compact(mpm_ctx *ctx, const mpm_subgrid *sub, int32_t s, const double *x, double *y,
                             cudaStream_t st);

namespace mpm {

constexpr int kDotBlocks = 256;

// Partial sums a.b (or a.b over in-mask elements when flags is set) per
// block; the second stage sums the partials in a fixed order, so every dot
// product is reproducible.
__global__ void __launch_bounds__(kBlock) k_fg_dot1(const double *__restrict__ a, const double *__restrict__ b,
                                                    const uint8_t *__restrict__ flags, int64_t n,
                                                    double *__restrict__ part)
{
    __shared__ double sh[kWarps];
    double t = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock)
        if (!flags || (flags[i] & F_MASK)) t += a[i] * b[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int w = 0; w < kWarps; ++w) u += sh[w];
        part[blockIdx.x] = u;
    }
}

__global__ void k_fg_dot2(const double *__restrict__ part, int np, double *__restrict__ out)
{
    if (threadIdx.x != 0) return;
    double u = 0.0;
    for (int i = 0; i < np; ++i) u += part[i];
    *out = u;
}

// y += sgn * (*alpha) * x
__global__ void __launch_bounds__(kBlock) k_fg_axpy(double *__restrict__ y, const double *__restrict__ x, int64_t n,
                                                    const double *__restrict__ alpha, double sgn)
{
    const double a = sgn * *alpha;
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) y[i] += a * x[i];
}

// y = x / sqrt(*sq)  (0 if the norm is 0)
__global__ void __launch_bounds__(kBlock) k_fg_normalise(double *__restrict__ y, const double *__restrict__ x, int64_t n,
                                                         const double *__restrict__ sq)
{
    const double nrm = sqrt(*sq);
    const double a = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) y[i] = a * x[i];
}

// r = b - ax
__global__ void __launch_bounds__(kBlock) k_fg_resid(double *__restrict__ r, const double *__restrict__ b,
                                                     const double *__restrict__ ax, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) r[i] = b[i] - ax[i];
}

// x += y * z (host scalar)
__global__ void __launch_bounds__(kBlock) k_fg_update(double *__restrict__ x, const double *__restrict__ z, int64_t n,
                                                      double y)
{
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) x[i] += y * z[i];
}

}  // namespace mpm

using namespace mpm;

namespace {

struct Fg {
    mpm_ctx *ctx;
    cudaStream_t st;
    int64_t n;
    int grid;
    double *part;
    mpm_status dot(const double *a, const double *b, const uint8_t *flags, double *out)
    {
        k_fg_dot1<<<kDotBlocks, kBlock, 0, st>>>(a, b, flags, n, part);
        k_fg_dot2<<<1, 32, 0, st>>>(part, kDotBlocks, out);
        ctx->launches += 2;
        MPM_CU(cudaGetLastError());
        return MPM_OK;
    }
};

}  // namespace

mpm_status mpm_solve_fgmres_impl(mpm_ctx *ctx, mpm_cnn *cnn, mpm_subgrid *sub, const mpm_lattice *lat,
                                 const mpm_params *prm, const mpm_lattice *scatter_to, const mpm_opts *opt,
                                 mpm_report *rep, cudaStream_t st)
{
    if (!cnn || !sub || !lat || !prm || !opt) return mpm_fail(ctx, MPM_ERR_ARG, "fgmres: null argument");
    if (!sub->extracted || !sub->assembled) return mpm_fail(ctx, MPM_ERR_ARG, "fgmres: subgrid not assembled");
    if (sub->nspecies > 3 || prm->nspecies != sub->nspecies)
        return mpm_fail(ctx, MPM_ERR_ARG, "fgmres: the network covers species 0..2 of the assembled subgrid");
    const int m = opt->restart;
    if (m < 1 || m > MPM_MAX_RESTART || opt->maxit < 1 || !(opt->rtol >= 0.0) || !(opt->atol >= 0.0))
        return mpm_fail(ctx, MPM_ERR_ARG, "fgmres: bad options");
    const int64_t NE = sub->NE;
    const size_t vec = (size_t)(NE > 0 ? NE : 1);
    // workspace: V (m+1), Z (m), w, ax, partials, scalars
    const size_t need = ((size_t)(2 * m + 3) * vec + kDotBlocks + 2 * (MPM_MAX_RESTART + 8)) * sizeof(double);
    mpm_status r = mpm_grow(ctx, (void **)&ctx->d_fg, &ctx->fg_cap, need, "fgmres workspace");
    if (r != MPM_OK) return r;
    double *V = ctx->d_fg;
    double *Z = V + (size_t)(m + 1) * vec;
    double *w = Z + (size_t)m * vec;
    double *ax = w + vec;
    double *part = ax + vec;
    double *sc = part + kDotBlocks;          // device scalars: h[0..m], ||w||^2, beta^2, ||b||^2, m
    const size_t hneed = 2 * (MPM_MAX_RESTART + 8) * sizeof(double);
    if (ctx->stage_cap < hneed + 4096) {
        if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
        ctx->h_stage = nullptr;
        ctx->stage_cap = 0;
        MPM_CU(cudaMallocHost(&ctx->h_stage, hneed + 4096));
        ctx->stage_cap = hneed + 4096;
    }
    double *hsc = (double *)ctx->h_stage;
    Fg F{ctx, st, NE, ctx->num_sms * 4, part};
    const int grid = ctx->num_sms * 4;
    mpm_report R;
    memset(&R, 0, sizeof(R));
    R.box_voxels = (int64_t)sub->n[0] * sub->n[1] * sub->n[2];
    R.mask_voxels = sub->mask_voxels;
    R.stored_voxels = NE;
    MPM_CU(cudaEventRecord(ctx->ev0, st));
    mpm_status worst = MPM_OK;
    for (int s = 0; s < sub->nspecies; ++s) {
        double *x = sub->x[s];
        const double *b = sub->b[s];
        if (!opt->x0_given && !sub->x_fresh)
            MPM_CU(cudaMemcpyAsync(x, sub->cn[s], (size_t)NE * sizeof(double), cudaMemcpyDeviceToDevice, st));
        // ||b|| over the in-mask rows (the stopping rule of the plain solver)
        r = F.dot(b, b, sub->flags, sc + MPM_MAX_RESTART + 3);
        if (r != MPM_OK) return r;
        MPM_CU(cudaMemcpyAsync(hsc, sc + MPM_MAX_RESTART + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
        MPM_CU(cudaStreamSynchronize(st));
        const double bnorm = std::sqrt(hsc[0]);
        const double tol = std::fmax(opt->rtol * bnorm, opt->atol);
        int it = 0, cyc = 0, status = MPM_ERR_NOCONV;
        double beta = 0.0;
        std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
        for (;;) {
            // r = b - A x (into w), beta = ||r||
            r = mpm_apply_compact(ctx, sub, s, x, ax, st);
            if (r != MPM_OK) return r;
            k_fg_resid<<<grid, kBlock, 0, st>>>(w, b, ax, NE);
            ctx->launches += 1;
            r = F.dot(w, w, nullptr, sc + MPM_MAX_RESTART + 2);
            if (r != MPM_OK) return r;
            k_fg_normalise<<<grid, kBlock, 0, st>>>(V, w, NE, sc + MPM_MAX_RESTART + 2);
            ctx->launches += 1;
            MPM_CU(cudaMemcpyAsync(hsc, sc + MPM_MAX_RESTART + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
            MPM_CU(cudaStreamSynchronize(st));
            beta = std::sqrt(hsc[0]);
            if (!std::isfinite(beta)) { status = MPM_ERR_BREAKDOWN; break; }
            if (beta <= tol) { status = MPM_OK; break; }
            if (it >= opt->maxit) { status = MPM_ERR_NOCONV; break; }
            ++cyc;
            std::fill(g.begin(), g.end(), 0.0);
            g[0] = beta;
            int k = 0;
            for (int j = 0; j < m; ++j) {
                double *vj = V + (size_t)j * vec, *zj = Z + (size_t)j * vec;
                r = mpm_cnn_precond_impl(ctx, cnn, sub, lat, prm, s, vj, zj, sc + MPM_MAX_RESTART + 4, st);
                if (r != MPM_OK) return r;
                r = mpm_apply_compact(ctx, sub, s, zj, w, st);
                if (r != MPM_OK) return r;
                for (int i = 0; i <= j; ++i) {   // modified Gram-Schmidt, scalars on the device
                    const double *vi = V + (size_t)i * vec;
                    r = F.dot(w, vi, nullptr, sc + i);
                    if (r != MPM_OK) return r;
                    k_fg_axpy<<<grid, kBlock, 0, st>>>(w, vi, NE, sc + i, -1.0);
                    ctx->launches += 1;
                }
                r = F.dot(w, w, nullptr, sc + MPM_MAX_RESTART + 1);
                if (r != MPM_OK) return r;
                k_fg_normalise<<<grid, kBlock, 0, st>>>(V + (size_t)(j + 1) * vec, w, NE, sc + MPM_MAX_RESTART + 1);
                ctx->launches += 1;
                MPM_CU(cudaGetLastError());
                MPM_CU(cudaMemcpyAsync(hsc, sc, (MPM_MAX_RESTART + 2) * sizeof(double), cudaMemcpyDeviceToHost, st));
                MPM_CU(cudaStreamSynchronize(st));
                const double hn = std::sqrt(hsc[MPM_MAX_RESTART + 1]);
                for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hsc[i];
                for (int i = 0; i < j; ++i) {
                    const double t0 = H[(size_t)i * m + j], t1 = H[(size_t)(i + 1) * m + j];
                    H[(size_t)i * m + j] = cs[i] * t0 + sn[i] * t1;
                    H[(size_t)(i + 1) * m + j] = -sn[i] * t0 + cs[i] * t1;
                }
                const double aa = H[(size_t)j * m + j];
                const double den = std::hypot(aa, hn);
                if (den == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
                else { cs[j] = aa / den; sn[j] = hn / den; }
                H[(size_t)j * m + j] = cs[j] * aa + sn[j] * hn;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                ++it;
                R.jsum[s] += j;
                k = j + 1;
                if (!std::isfinite(g[j + 1])) { status = MPM_ERR_BREAKDOWN; break; }
                if (std::fabs(g[j + 1]) <= tol || it >= opt->maxit || hn == 0.0) break;
            }
            if (status == MPM_ERR_BREAKDOWN) break;
            for (int i = k - 1; i >= 0; --i) {
                double acc = g[i];
                for (int l = i + 1; l < k; ++l) acc -= H[(size_t)i * m + l] * y[l];
                y[i] = acc / H[(size_t)i * m + i];
            }
            for (int i = 0; i < k; ++i) {
                k_fg_update<<<grid, kBlock, 0, st>>>(x, Z + (size_t)i * vec, NE, y[i]);
                ctx->launches += 1;
            }
            MPM_CU(cudaGetLastError());
        }
        R.iters[s] = it;
        R.cycles[s] = cyc;
        R.status[s] = status;
        R.res[s] = beta;
        R.bnorm[s] = bnorm;
        if (status != MPM_OK && (worst == MPM_OK || status == MPM_ERR_BREAKDOWN)) worst = (mpm_status)status;
    }
    sub->x_fresh = false;
    MPM_CU(cudaEventRecord(ctx->ev1, st));
    MPM_CU(cudaEventSynchronize(ctx->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    R.solve_ms = ms;
    if (rep) *rep = R;
    if (scatter_to && worst != MPM_ERR_BREAKDOWN) {
        r = mpm_scatter_impl(ctx, sub, scatter_to, st);
        if (r != MPM_OK) return r;
    }
    if (worst != MPM_OK) mpm_fail(ctx, worst, "fgmres: not every species converged");
    return worst;
}
