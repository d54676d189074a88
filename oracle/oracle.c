/*
 * oracle.c -- plain, single-threaded FP64 CPU oracle for the box-restricted
 * implicit-Euler finite-volume reaction-diffusion step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py load this library.  The CUDA product path never
 * calls, links or includes it, and it shares no code with that path.
 *
 * Source: Dolganov, Krzhizhanovskaya, Trebeschi, Sheraton, "Multiscale Parallel
 * Simulation of Malignant Pleural Mesothelioma via Adaptive Domain Partitioning"
 * (arXiv 2505.03067).
 *   Eq. 1-2   dC/dt = D lap(C) - S          (oxygen, nutrient; S = consumption)
 *   Eq. 3-4   dC/dt = D lap(C) - mu C       (cytokines IL6, IL8; mu = degradation)
 *   Sec. 2.3  the PDEs are solved only inside a bounding box of the tumour cells
 *             plus a margin.
 *   Sec. 2.4  a structured 3D mesh of the box, finite volumes, first-order
 *             implicit Euler, GMRES (Saad & Schultz 1986); the output is mapped
 *             onto the pleural mask.
 *
 * Readings of what the paper leaves open (each is listed in the design notes):
 *   - the consumption S is linear, S = k_v C, with k_v = mu + k_cell[id], and a
 *     zero-order source q_v = q_cell[id] (secretion) may be added;
 *   - masked voxels (inside the box, outside the pleural mask) are identity
 *     rows that keep c^n; faces between a masked and an unmasked voxel carry no
 *     flux;
 *   - box faces are Dirichlet with the face value fixed half a cell from the
 *     centre (weight 2), or zero flux when bc_box = 1;
 *   - face diffusivities are the harmonic mean of the two cell values;
 *   - the stopping rule is the true residual ||b - A x||_2 <= tol_abs.
 *
 * Everything here is the plain definition: an explicit CSR matrix, a textbook
 * restarted GMRES with modified Gram-Schmidt and Givens rotations, and a dense
 * LU with partial pivoting for small grids.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_NOCONV 3
#define ORC_ERR_BREAKDOWN 4
#define ORC_ERR_NOMEM 7

/* Parameters of one species' system (Eq. 1-4 on the box). */
typedef struct {
    double dt, h;
    double D;              /* diffusivity of the species */
    double mu;             /* uniform first-order decay (Eq. 3-4) */
    double c_bc;           /* Dirichlet value on box faces */
    int32_t bc_box;        /* 0: Dirichlet box faces, 1: zero flux */
    int32_t ncell;         /* number of entries in k_cell / q_cell */
    const double *k_cell;  /* first-order uptake per cell id (id 0 = medium) */
    const double *q_cell;  /* zero-order source per cell id */
} orc_species;

static double face_diffusivity(double dp, double dq)
{
    /* Harmonic mean of the two cell diffusivities (flux continuity across the
     * face for a first-order FV scheme). */
    if (dp + dq <= 0.0) return 0.0;
    return 2.0 * dp * dq / (dp + dq);
}

/*
 * Assemble A and b of one implicit-Euler step (I - dt*L + dt*K) c^{n+1} = c^n + dt*q
 * on the box of dims n[3] (x fastest).  Row P of an in-mask voxel:
 *   A_PP = 1 + dt*k_P + (dt/h^2) * sum_f w_f D_f
 *   A_PQ = -(dt/h^2) D_f        for each open face f to an in-mask neighbour Q
 *   b_P  = c^n_P + dt*q_P + (dt/h^2) * sum_{Dirichlet f} 2 D_P c_bc
 * with w_f = 1 on an interior open face, 2 on a Dirichlet box face, 0 on a face
 * to a masked voxel (zero flux).  A masked voxel has A_PP = 1, b_P = c^n_P.
 * dfac (nullable) scales D per voxel; NULL means uniform D.
 * CSR output: row_ptr[N+1], col/val with room for 7N entries, columns sorted.
 * Returns the number of non-zeros, or -1 if a cell id lies outside the tables.
 */
int64_t orc_assemble(const int32_t n[3], const uint8_t *mask, const int32_t *cell,
                     const double *c_old, const double *dfac, const orc_species *sp,
                     int64_t *row_ptr, int32_t *col, double *val, double *rhs)
{
    const int64_t nx = n[0], ny = n[1], nz = n[2];
    const double a = sp->dt / (sp->h * sp->h);
    int64_t nnz = 0;
    row_ptr[0] = 0;
    for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
    for (int64_t i = 0; i < nx; ++i) {
        const int64_t p = i + nx * (j + ny * k);
        if (!mask[p]) {
            col[nnz] = (int32_t)p; val[nnz] = 1.0; ++nnz;
            rhs[p] = c_old[p];
            row_ptr[p + 1] = nnz;
            continue;
        }
        const int32_t id = cell[p];
        if (id < 0 || id >= sp->ncell) return -1;
        const double dp = sp->D * (dfac ? dfac[p] : 1.0);
        double diag = 1.0 + sp->dt * (sp->mu + sp->k_cell[id]);
        double b = c_old[p] + sp->dt * sp->q_cell[id];
        /* neighbours in ascending flat index: -z, -y, -x, (self), +x, +y, +z */
        const int64_t di[6] = {0, 0, -1, 1, 0, 0};
        const int64_t dj[6] = {0, -1, 0, 0, 1, 0};
        const int64_t dk[6] = {-1, 0, 0, 0, 0, 1};
        int64_t qcol[6]; double qval[6]; int nq = 0;
        for (int f = 0; f < 6; ++f) {
            const int64_t ii = i + di[f], jj = j + dj[f], kk = k + dk[f];
            const int inside = ii >= 0 && ii < nx && jj >= 0 && jj < ny && kk >= 0 && kk < nz;
            if (!inside) {
                if (sp->bc_box == 0) {           /* Dirichlet face, half a cell away */
                    diag += a * 2.0 * dp;
                    b += a * 2.0 * dp * sp->c_bc;
                }
                continue;
            }
            const int64_t q = ii + nx * (jj + ny * kk);
            if (!mask[q]) continue;              /* zero flux towards a masked voxel */
            const double df = face_diffusivity(dp, sp->D * (dfac ? dfac[q] : 1.0));
            diag += a * df;
            qcol[nq] = q; qval[nq] = -a * df; ++nq;
        }
        /* emit lower neighbours, diagonal, upper neighbours (already sorted) */
        int e = 0;
        while (e < nq && qcol[e] < p) { col[nnz] = (int32_t)qcol[e]; val[nnz] = qval[e]; ++nnz; ++e; }
        col[nnz] = (int32_t)p; val[nnz] = diag; ++nnz;
        while (e < nq) { col[nnz] = (int32_t)qcol[e]; val[nnz] = qval[e]; ++nnz; ++e; }
        rhs[p] = b;
        row_ptr[p + 1] = nnz;
    }
    return nnz;
}

/* y = A x for a CSR matrix. */
void orc_csr_matvec(int64_t N, const int64_t *rp, const int32_t *ci, const double *va,
                    const double *x, double *y)
{
    for (int64_t r = 0; r < N; ++r) {
        double s = 0.0;
        for (int64_t e = rp[r]; e < rp[r + 1]; ++e) s += va[e] * x[ci[e]];
        y[r] = s;
    }
}

static double dot(int64_t N, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) s += a[i] * b[i];
    return s;
}

/* r = b - A x, returns ||r||_2 */
static double residual(int64_t N, const int64_t *rp, const int32_t *ci, const double *va,
                       const double *b, const double *x, double *r)
{
    orc_csr_matvec(N, rp, ci, va, x, r);
    for (int64_t i = 0; i < N; ++i) r[i] = b[i] - r[i];
    return sqrt(dot(N, r, r));
}

/*
 * Restarted GMRES(m) (Saad & Schultz 1986) for A x = b, x holding the initial
 * guess on entry and the iterate on exit.  Each cycle: r = b - A x,
 * v_1 = r/||r||; Arnoldi with modified Gram-Schmidt builds the Hessenberg
 * matrix H; Givens rotations reduce H to upper-triangular form and carry
 * ||r|| e_1 into g, whose last entry is the residual norm of the least-squares
 * problem min ||beta e_1 - H y||; then x += V y.  Stops when the TRUE residual
 * satisfies ||b - A x||_2 <= tol_abs, or after maxit Arnoldi steps in total.
 * Returns ORC_OK or ORC_ERR_NOCONV; iterations and the final true residual
 * norm are written to *iters and *res.
 */
int orc_gmres(int64_t N, const int64_t *rp, const int32_t *ci, const double *va,
              const double *b, double *x, int32_t m, double tol_abs, int32_t maxit,
              int32_t *iters, int32_t *cycles, double *res)
{
    if (m < 1 || N < 0) return ORC_ERR_ARG;
    double *V = (double *)malloc(sizeof(double) * (size_t)N * (size_t)(m + 1));
    double *w = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double *H = (double *)calloc((size_t)(m + 1) * (size_t)m, sizeof(double));
    double *cs = (double *)malloc(sizeof(double) * (size_t)m);
    double *sn = (double *)malloc(sizeof(double) * (size_t)m);
    double *g = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    double *y = (double *)malloc(sizeof(double) * (size_t)m);
    if ((!V && N) || !w || !H || !cs || !sn || !g || !y) {
        free(V); free(w); free(H); free(cs); free(sn); free(g); free(y);
        return ORC_ERR_NOMEM;
    }
#define HH(i, j) H[(size_t)(i) * (size_t)m + (size_t)(j)]
    int32_t it = 0, cyc = 0;
    int status = ORC_ERR_NOCONV;
    double beta = 0.0;
    for (;;) {
        beta = residual(N, rp, ci, va, b, x, V);        /* r into v_1 */
        if (beta <= tol_abs) { status = ORC_OK; break; }
        if (it >= maxit) break;
        ++cyc;
        for (int64_t i = 0; i < N; ++i) V[i] /= beta;
        for (int i = 0; i <= m; ++i) g[i] = 0.0;
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m; ++j) {
            double *vj = V + (size_t)j * (size_t)N;
            orc_csr_matvec(N, rp, ci, va, vj, w);
            for (int i = 0; i <= j; ++i) {                   /* modified Gram-Schmidt */
                const double *vi = V + (size_t)i * (size_t)N;
                const double hij = dot(N, w, vi);
                HH(i, j) = hij;
                for (int64_t t = 0; t < N; ++t) w[t] -= hij * vi[t];
            }
            const double hn = sqrt(dot(N, w, w));
            HH(j + 1, j) = hn;
            for (int i = 0; i < j; ++i) {                    /* earlier rotations */
                const double t0 = HH(i, j), t1 = HH(i + 1, j);
                HH(i, j) = cs[i] * t0 + sn[i] * t1;
                HH(i + 1, j) = -sn[i] * t0 + cs[i] * t1;
            }
            const double aa = HH(j, j), bb = HH(j + 1, j);   /* new rotation */
            if (bb == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
            else {
                const double r = hypot(aa, bb);
                cs[j] = aa / r; sn[j] = bb / r;
            }
            HH(j, j) = cs[j] * aa + sn[j] * bb;
            HH(j + 1, j) = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++it;
            k = j + 1;
            if (fabs(g[j + 1]) <= tol_abs || it >= maxit || hn == 0.0) break;
            double *vn = V + (size_t)(j + 1) * (size_t)N;
            for (int64_t t = 0; t < N; ++t) vn[t] = w[t] / hn;
        }
        for (int i = k - 1; i >= 0; --i) {                   /* back substitution */
            double s = g[i];
            for (int l = i + 1; l < k; ++l) s -= HH(i, l) * y[l];
            if (HH(i, i) == 0.0) { status = ORC_ERR_BREAKDOWN; goto done; }
            y[i] = s / HH(i, i);
        }
        for (int i = 0; i < k; ++i) {
            const double *vi = V + (size_t)i * (size_t)N;
            for (int64_t t = 0; t < N; ++t) x[t] += y[i] * vi[t];
        }
    }
done:
    if (res) *res = (status == ORC_ERR_BREAKDOWN) ? residual(N, rp, ci, va, b, x, w) : beta;
    if (iters) *iters = it;
    if (cycles) *cycles = cyc;
#undef HH
    free(V); free(w); free(H); free(cs); free(sn); free(g); free(y);
    return status;
}

/*
 * Dense LU with partial pivoting (Doolittle, row interchanges) of the CSR
 * matrix, then forward and back substitution: x = A^{-1} b.  For grids small
 * enough to hold A densely (the tests use N <= 8^3).
 */
int orc_dense_solve(int64_t N, const int64_t *rp, const int32_t *ci, const double *va,
                    const double *b, double *x)
{
    double *M = (double *)calloc((size_t)N * (size_t)N, sizeof(double));
    int64_t *piv = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    if ((!M && N) || !piv) { free(M); free(piv); return ORC_ERR_NOMEM; }
    for (int64_t r = 0; r < N; ++r)
        for (int64_t e = rp[r]; e < rp[r + 1]; ++e) M[r * N + ci[e]] += va[e];
    for (int64_t r = 0; r < N; ++r) x[r] = b[r];
    for (int64_t c = 0; c < N; ++c) {
        int64_t p = c;
        for (int64_t r = c + 1; r < N; ++r)
            if (fabs(M[r * N + c]) > fabs(M[p * N + c])) p = r;
        piv[c] = p;
        if (M[p * N + c] == 0.0) { free(M); free(piv); return ORC_ERR_BREAKDOWN; }
        if (p != c) {
            for (int64_t t = 0; t < N; ++t) {
                const double tmp = M[c * N + t]; M[c * N + t] = M[p * N + t]; M[p * N + t] = tmp;
            }
            const double tb = x[c]; x[c] = x[p]; x[p] = tb;
        }
        for (int64_t r = c + 1; r < N; ++r) {
            const double l = M[r * N + c] / M[c * N + c];
            M[r * N + c] = l;
            for (int64_t t = c + 1; t < N; ++t) M[r * N + t] -= l * M[c * N + t];
            x[r] -= l * x[c];
        }
    }
    for (int64_t r = N - 1; r >= 0; --r) {
        double s = x[r];
        for (int64_t t = r + 1; t < N; ++t) s -= M[r * N + t] * x[t];
        x[r] = s / M[r * N + r];
    }
    free(M); free(piv);
    return ORC_OK;
}
