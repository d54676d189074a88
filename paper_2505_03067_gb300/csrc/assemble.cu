// assemble.cu -- the implicit-Euler finite-volume system of Eq. 1-4 on the box
// (Sec. 2.4), stored matrix-free: per element a diagonal (FP64 and FP32 copies),
// a right-hand side and the face-flag byte shared by all species; the
// off-diagonal of every open face is -(dt/h^2) D_f.
#include <cstring>

#include "mpm_internal.cuh"

namespace mpm {

struct AsmArgs {
    AsmCoef C;
    int32_t n[3], lt[3];
    const uint8_t *flags;
    const int32_t *cell;
    const double *dfac;
    const int32_t *tile_coord;
    const int32_t *nbr;
    const double *cn[kMaxSpecies];
    double *b[kMaxSpecies];
    double *diag[kMaxSpecies];
    float *diag32[kMaxSpecies];
    int32_t *err;
};

// Rows of the stored elements: in-mask voxels by assemble_row, every other
// element an identity row keeping c^n (tile padding: 0).  The neighbours'
// diffusivity factors come from the compact copy through the tile table.
__global__ void __launch_bounds__(kBlock) k_assemble(AsmArgs A, int64_t NE)
{
    const int ltv = A.lt[0] + A.lt[1] + A.lt[2];
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < NE; e += (int64_t)gridDim.x * kBlock) {
        const uint32_t f = A.flags[e];
        if (!(f & F_MASK)) {                       // padding or masked voxel: identity row
            for (int s = 0; s < A.C.nspecies; ++s) {
                A.diag[s][e] = 1.0;
                A.diag32[s][e] = 1.0f;
                A.b[s][e] = (f & F_BOX) ? A.cn[s][e] : 0.0;
            }
            continue;
        }
        int32_t id = A.cell[e];
        if (id < 0 || id >= A.C.ncell) {
            atomicOr(A.err, 1);
            id = 0;
        }
        const int64_t tile = e >> ltv;
        const uint32_t v = (uint32_t)(e & ((1 << ltv) - 1));
        const uint32_t TX = 1u << A.lt[0], TY = 1u << A.lt[1], TZ = 1u << A.lt[2];
        const uint32_t ix = v & (TX - 1), iy = (v >> A.lt[0]) & (TY - 1), iz = v >> (A.lt[0] + A.lt[1]);
        int ndir = 0;
        if (A.C.bc_box == 0) {
            const int4 tc = __ldg(reinterpret_cast<const int4 *>(A.tile_coord) + tile);
            const int bx = (tc.x << A.lt[0]) + (int)ix;
            const int by = (tc.y << A.lt[1]) + (int)iy;
            const int bz = (tc.z << A.lt[2]) + (int)iz;
            ndir = (bx == 0) + (bx == A.n[0] - 1) + (by == 0) + (by == A.n[1] - 1) + (bz == 0) + (bz == A.n[2] - 1);
        }
        const double fp = A.dfac ? A.dfac[e] : 1.0;
        auto dq = [&](int d) -> double {
            int64_t q;
            switch (d) {
            case 0: q = ix > 0 ? e - 1 : ((int64_t)A.nbr[tile * 6 + 0] << ltv) + (v + TX - 1); break;
            case 1: q = ix < TX - 1 ? e + 1 : ((int64_t)A.nbr[tile * 6 + 1] << ltv) + (v - (TX - 1)); break;
            case 2: q = iy > 0 ? e - TX : ((int64_t)A.nbr[tile * 6 + 2] << ltv) + (v + (TY - 1) * TX); break;
            case 3: q = iy < TY - 1 ? e + TX : ((int64_t)A.nbr[tile * 6 + 3] << ltv) + (v - (TY - 1) * TX); break;
            case 4: q = iz > 0 ? e - TX * TY : ((int64_t)A.nbr[tile * 6 + 4] << ltv) + (v + (TZ - 1) * TX * TY); break;
            default: q = iz < TZ - 1 ? e + TX * TY : ((int64_t)A.nbr[tile * 6 + 5] << ltv) + (v - (TZ - 1) * TX * TY);
            }
            return A.dfac[q];
        };
        for (int s = 0; s < A.C.nspecies; ++s) {
            double dg, b;
            assemble_row(A.C, s, f, id, ndir, A.dfac != nullptr, fp, dq, A.cn[s][e], dg, b);
            A.diag[s][e] = dg;
            A.diag32[s][e] = f32_rz(dg);
            A.b[s][e] = b;
        }
    }
}

// y = A x on the stored elements (FP64 operator): the solver's matvec alone.
__global__ void __launch_bounds__(kBlock) k_apply(SysDev S, int s, const double *__restrict__ x,
                                                  double *__restrict__ y, double a, double Ds)
{
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < S.NE; e += (int64_t)gridDim.x * kBlock) {
        const uint32_t f = S.flags[e];
        double ns;
        if (S.dfac) ns = a * nbr_sum_var<double>(x, S.dfac, S.nbr, e, f, S.ltx, S.lty, S.ltz, Ds);
        else ns = S.off[s] * nbr_sum<double>(x, S.nbr, e, f, S.ltx, S.lty, S.ltz);
        y[e] = S.diag[s][e] * x[e] - ns;
    }
}

}  // namespace mpm

using namespace mpm;

mpm_status mpm_assemble_check(mpm_ctx *ctx, const mpm_subgrid *sub, const mpm_params *p)
{
    if (!sub || !p) return mpm_fail(ctx, MPM_ERR_ARG, "assemble: null argument");
    if (!sub->extracted) return mpm_fail(ctx, MPM_ERR_ARG, "assemble: subgrid not extracted");
    if (p->nspecies != sub->nspecies) return mpm_fail(ctx, MPM_ERR_ARG, "assemble: nspecies differs from the extract");
    return mpm_params_check(ctx, p);
}

mpm_status mpm_params_check(mpm_ctx *ctx, const mpm_params *p)
{
    if (!p) return mpm_fail(ctx, MPM_ERR_ARG, "assemble: null parameters");
    if (p->nspecies < 1 || p->nspecies > MPM_MAX_SPECIES) return mpm_fail(ctx, MPM_ERR_ARG, "assemble: nspecies out of range");
    if (p->ncell < 1 || !p->k_cell || !p->q_cell) return mpm_fail(ctx, MPM_ERR_ARG, "assemble: empty rate tables");
    if (!(p->dt > 0.0) || !(p->h > 0.0)) return mpm_fail(ctx, MPM_ERR_ARG, "assemble: dt and h must be > 0");
    if (p->bc_box != 0 && p->bc_box != 1) return mpm_fail(ctx, MPM_ERR_ARG, "assemble: bc_box must be 0 or 1");
    for (int s = 0; s < p->nspecies; ++s)
        if (!(p->D[s] >= 0.0) || !(p->mu[s] >= 0.0)) return mpm_fail(ctx, MPM_ERR_ARG, "assemble: D and mu must be >= 0");
    return MPM_OK;
}

void mpm_asm_coef(const mpm_params *p, AsmCoef *C)
{
    memset(C, 0, sizeof(*C));
    C->nspecies = p->nspecies;
    C->ncell = p->ncell;
    C->bc_box = p->bc_box;
    C->dt = p->dt;
    C->a = p->dt / (p->h * p->h);
    for (int s = 0; s < p->nspecies; ++s) {
        C->D[s] = p->D[s];
        C->mu[s] = p->mu[s];
        C->cbc[s] = p->c_bc[s];
    }
    C->k_cell = p->k_cell;
    C->q_cell = p->q_cell;
}

// The scalars the solver reads from the subgrid: the uniform-D off-diagonal
// dt D_s / h^2, and a = dt / h^2 with D_s for the harmonic-mean path.
void mpm_set_assembled_scalars(mpm_subgrid *sub, const mpm_params *p)
{
    sub->a = p->dt / (p->h * p->h);
    for (int s = 0; s < MPM_MAX_SPECIES; ++s) {
        sub->off[s] = s < p->nspecies ? sub->a * p->D[s] : 0.0;
        sub->Dsp[s] = s < p->nspecies ? p->D[s] : 0.0;
    }
}

mpm_status mpm_assemble_impl(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_params *p, cudaStream_t st)
{
    mpm_status r = mpm_assemble_check(ctx, sub, p);
    if (r != MPM_OK) return r;
    AsmArgs A;
    memset(&A, 0, sizeof(A));
    mpm_asm_coef(p, &A.C);
    for (int d = 0; d < 3; ++d) { A.n[d] = sub->n[d]; A.lt[d] = sub->lt[d]; }
    for (int s = 0; s < p->nspecies; ++s) {
        A.cn[s] = sub->cn[s];
        A.b[s] = sub->b[s];
        A.diag[s] = sub->diag[s];
        A.diag32[s] = sub->diag32[s];
    }
    A.flags = sub->flags;
    A.cell = sub->cell;
    A.dfac = sub->dfac;
    A.tile_coord = sub->tile_coord;
    A.nbr = sub->nbr;
    A.err = sub->err;
    mpm_set_assembled_scalars(sub, p);
    MPM_CU(cudaMemsetAsync(sub->err, 0, sizeof(int32_t), st));
    if (sub->NE > 0) {
        int64_t g = (sub->NE + kBlock - 1) / kBlock;
        if (g > (int64_t)ctx->num_sms * 8) g = (int64_t)ctx->num_sms * 8;
        k_assemble<<<(int)g, kBlock, 0, st>>>(A, sub->NE);
        ctx->launches += 1;
        MPM_CU(cudaGetLastError());
    }
    sub->assembled = true;
    return MPM_OK;
}

SysDev mpm_make_sysdev(const mpm_subgrid *sub);
mpm_status mpm_dense_to_elems(mpm_ctx *ctx, const mpm_subgrid *sub, const double *src, double *dst, cudaStream_t st);
mpm_status mpm_elems_to_dense(mpm_ctx *ctx, const mpm_subgrid *sub, const double *src, const double *dflt_dense,
                              double *dst, cudaStream_t st);

mpm_status mpm_apply_impl(mpm_ctx *ctx, const mpm_subgrid *sub, int32_t s, const double *x, double *y, cudaStream_t st)
{
    if (!sub || !x || !y) return mpm_fail(ctx, MPM_ERR_ARG, "apply: null argument");
    if (!sub->assembled) return mpm_fail(ctx, MPM_ERR_ARG, "apply: subgrid not assembled");
    if (s < 0 || s >= sub->nspecies) return mpm_fail(ctx, MPM_ERR_ARG, "apply: species out of range");
    const size_t need = 2 * (size_t)(sub->NE > 0 ? sub->NE : 1) * sizeof(double);
    mpm_status r = mpm_grow(ctx, (void **)&ctx->d_tmp, &ctx->tmp_cap, need, "operator scratch");
    if (r != MPM_OK) return r;
    double *xe = ctx->d_tmp, *ye = ctx->d_tmp + (sub->NE > 0 ? sub->NE : 1);
    if (sub->NE > 0) {
        r = mpm_dense_to_elems(ctx, sub, x, xe, st);
        if (r != MPM_OK) return r;
        SysDev S = mpm_make_sysdev(sub);
        int64_t g = (sub->NE + kBlock - 1) / kBlock;
        if (g > (int64_t)ctx->num_sms * 8) g = (int64_t)ctx->num_sms * 8;
        k_apply<<<(int)g, kBlock, 0, st>>>(S, s, xe, ye, sub->a, sub->Dsp[s]);
        ctx->launches += 1;
        MPM_CU(cudaGetLastError());
    }
    return mpm_elems_to_dense(ctx, sub, ye, x, y, st);
}

// y = A x on compact element vectors of species s (no box-dense conversion).
mpm_status mpm_apply_compact(mpm_ctx *ctx, const mpm_subgrid *sub, int32_t s, const double *x, double *y,
                             cudaStream_t st)
{
    if (!sub->assembled) return mpm_fail(ctx, MPM_ERR_ARG, "apply: subgrid not assembled");
    if (sub->NE == 0) return MPM_OK;
    const SysDev S = mpm_make_sysdev(sub);
    int64_t g = (sub->NE + kBlock - 1) / kBlock;
    if (g > (int64_t)ctx->num_sms * 8) g = (int64_t)ctx->num_sms * 8;
    k_apply<<<(int)g, kBlock, 0, st>>>(S, s, x, y, sub->a, sub->Dsp[s]);
    ctx->launches += 1;
    MPM_CU(cudaGetLastError());
    return MPM_OK;
}
