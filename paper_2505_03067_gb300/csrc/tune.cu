// tune.cu -- the autotuner of the batched solve.
//
// Tile shape (per system): the candidate that stores the fewest voxels wins,
// ties going to the larger tile (fewer neighbour-table lookups).  This is an
// exact bytes model: the active-tile count of each candidate is computed on
// the device with the extraction's own kernels, so no timing noise enters.
//
// Restart length and kernel variant (per batch): measured.  Each candidate
// (m, variant) solves the whole batch from c^n once to warm up and once
// timed with CUDA events; the fastest wins.  Results go to an optional
// on-disk cache, one line per key: the GPU name, precision, tolerance, and
// for every system its species count with bucketed box dims
// (nearest power of two) and mask occupancy (tenths).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mpm_internal.cuh"

int mpm_solver_max_blocks(mpm_ctx *ctx, int prec, int m, int variant);
int mpm_solver_variants(int prec, int m);

namespace {

const int32_t kTiles[][3] = {{4, 4, 4}, {8, 4, 4}, {8, 8, 4}, {8, 4, 2}, {16, 4, 2}, {8, 8, 2}, {4, 4, 2}, {16, 4, 4}};
const int32_t kRestarts[] = {4, 8, 16};

int ilog2(int v)
{
    int l = 0;
    while ((1 << (l + 1)) <= v) ++l;
    return l;
}

std::string cache_key(mpm_ctx *ctx, mpm_subgrid *const *subs, int nsys, const mpm_opts *opt)
{
    cudaDeviceProp pr;
    std::string k = "gpu=";
    if (cudaGetDeviceProperties(&pr, ctx->device) == cudaSuccess) k += pr.name;
    for (char &c : k) if (c == ' ') c = '_';
    char buf[128];
    snprintf(buf, sizeof(buf), ";prec=%d;rtol=%.0e;n=%d", opt->precision, opt->rtol, nsys);
    k += buf;
    for (int i = 0; i < nsys; ++i) {
        const mpm_subgrid *s = subs[i];
        const double box = (double)s->n[0] * s->n[1] * s->n[2];
        const int occ = box > 0 ? (int)std::lround(10.0 * (double)s->mask_voxels / box) : 0;
        snprintf(buf, sizeof(buf), ";%d:%d,%d,%d,%d", s->nspecies, ilog2(std::max(1, s->n[0])),
                 ilog2(std::max(1, s->n[1])), ilog2(std::max(1, s->n[2])), occ);
        k += buf;
    }
    return k;
}

bool cache_lookup(const char *path, const std::string &key, int &m, int &var)
{
    if (!path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    std::vector<char> line(1 << 16);
    bool found = false;
    while (fgets(line.data(), (int)line.size(), f)) {
        std::string s(line.data());
        const size_t sp = s.rfind(' ');
        if (sp == std::string::npos) continue;
        const size_t sp2 = s.rfind(' ', sp - 1);
        if (sp2 == std::string::npos) continue;
        if (s.compare(0, sp2, key) == 0 && sp2 == key.size()) {
            m = atoi(s.c_str() + sp2 + 1);
            var = atoi(s.c_str() + sp + 1);
            found = true;
        }
    }
    fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, int m, int var)
{
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d\n", key.c_str(), m, var);
    fclose(f);
}

}  // namespace

extern "C" mpm_status mpm_tune_tile(mpm_ctx *ctx, const mpm_lattice *lat, int32_t margin, int32_t out_tile[3],
                                    int64_t *out_stored, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    if (!lat || !lat->cell_id || !lat->mask || !out_tile || margin < 0)
        return mpm_fail(ctx, MPM_ERR_ARG, "tune_tile: null argument");
    const int64_t L = (int64_t)lat->dims[0] * lat->dims[1] * lat->dims[2];
    if (lat->dims[0] < 1 || lat->dims[1] < 1 || lat->dims[2] < 1 || L >= ((int64_t)1 << 31))
        return mpm_fail(ctx, MPM_ERR_ARG, "tune_tile: lattice dims out of range");
    cudaStream_t st = (cudaStream_t)stream;
    int64_t best = -1;
    int best_i = 0;
    for (int i = 0; i < (int)(sizeof(kTiles) / sizeof(kTiles[0])); ++i) {
        const int32_t lt[3] = {ilog2(kTiles[i][0]), ilog2(kTiles[i][1]), ilog2(kTiles[i][2])};
        int64_t nact = 0, mv = 0;
        mpm_status r = mpm_count_active_impl(ctx, lat, margin, lt, &nact, &mv, st);
        if (r != MPM_OK) return r;
        if (mv == 0 && nact == 0 && i == 0) {
            // empty tumour or mask: keep the default tile
        }
        const int64_t stored = nact * kTiles[i][0] * kTiles[i][1] * kTiles[i][2];
        const int tv = kTiles[i][0] * kTiles[i][1] * kTiles[i][2];
        const int btv = kTiles[best_i][0] * kTiles[best_i][1] * kTiles[best_i][2];
        if (best < 0 || stored < best || (stored == best && tv > btv)) {
            best = stored;
            best_i = i;
        }
    }
    for (int d = 0; d < 3; ++d) out_tile[d] = kTiles[best_i][d];
    if (out_stored) *out_stored = best;
    return MPM_OK;
}

extern "C" mpm_status mpm_tune_solver(mpm_ctx *ctx, mpm_subgrid *const *subs, int32_t nsys, mpm_opts *opt,
                                      int32_t *out_variant, const char *cache_path, void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    if (!subs || nsys < 1 || !opt || !out_variant) return mpm_fail(ctx, MPM_ERR_ARG, "tune_solver: null argument");
    for (int i = 0; i < nsys; ++i)
        if (!subs[i] || !subs[i]->assembled) return mpm_fail(ctx, MPM_ERR_ARG, "tune_solver: subgrid not assembled");
    const std::string key = cache_key(ctx, subs, nsys, opt);
    int m = 0, var = 0;
    if (cache_lookup(cache_path, key, m, var)) {
        opt->restart = m;
        *out_variant = var;
        ctx->solver_variant = var;
        return MPM_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int saved_var = ctx->solver_variant;
    double best_ms = 1e300;
    int best_m = opt->restart, best_v = 0;
    for (int32_t mm : kRestarts) {
        const int nvar = mpm_solver_variants(opt->precision, mm);
        for (int v = 0; v < nvar; ++v) {
            mpm_opts o = *opt;
            o.restart = mm;
            o.x0_given = 0;
            ctx->solver_variant = v;
            std::vector<mpm_report> reps(nsys);
            double t = 0.0;
            bool ok = true;
            for (int rep = 0; rep < 2 && ok; ++rep) {
                const mpm_status r = mpm_solve_impl(ctx, subs, nullptr, nsys, &o, reps.data(), st);
                ok = (r == MPM_OK || r == MPM_ERR_NOCONV);
                if (r == MPM_ERR_NOCONV) ok = false;   // a candidate that does not converge is out
                if (ok && rep == 1) t = reps[0].solve_ms;
            }
            if (ok && t < best_ms) {
                best_ms = t;
                best_m = mm;
                best_v = v;
            }
        }
    }
    ctx->solver_variant = saved_var;
    ctx->err.clear();
    if (best_ms >= 1e300) return mpm_fail(ctx, MPM_ERR_NOCONV, "tune_solver: no candidate converged");
    opt->restart = best_m;
    *out_variant = best_v;
    ctx->solver_variant = best_v;
    cache_store(cache_path, key, best_m, best_v);
    // leave the iterates at c^n for the caller's own solve
    for (int i = 0; i < nsys; ++i) {
        mpm_subgrid *sub = subs[i];
        for (int s = 0; s < sub->nspecies; ++s)
            MPM_CU(cudaMemcpyAsync(sub->x[s], sub->cn[s], (size_t)sub->NE * sizeof(double), cudaMemcpyDeviceToDevice, st));
        sub->x_fresh = true;
    }
    return MPM_OK;
}
