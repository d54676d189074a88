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
#include <algorithm>
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

// ------------------------------------------------------------------ team model
// The team planner's model of the batched solve (Sec. 2.5's load imbalance):
// item i costs it_i (F1 + NE_i) element-equivalents on one CTA and
// it_i (F + NE_i / c) on c > 1 CTAs.  Each round solves the batch from c^n,
// fits F1 and F to the measured item times (least squares of the time per
// Arnoldi step against NE_i / c_i with one intercept per regime, all rounds'
// items pooled), takes it_i from the solve just measured, and plans again;
// the round with the smallest imbalance f = t_max / <t> - 1 over the teams
// wins.  Stops after `rounds` rounds or when f has not fallen for two.
namespace {

// Least squares of y = beta x + alpha1 [one CTA] + alpha [several CTAs] over
// the measured items (x = NE / c, y = time per Arnoldi step): F1 =
// alpha1 / beta, F = alpha / beta.  A regime without items keeps its value.
bool fit_fixed(const std::vector<double> &x, const std::vector<double> &y, const std::vector<int> &one, double &F1,
               double &F, double &beta_out)
{
    // normal equations of the three unknowns (beta, alpha1, alpha)
    double a[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, r[3] = {0, 0, 0};
    int n1 = 0, nm = 0;
    for (size_t i = 0; i < x.size(); ++i) {
        const double f[3] = {x[i], one[i] ? 1.0 : 0.0, one[i] ? 0.0 : 1.0};
        n1 += one[i] ? 1 : 0;
        nm += one[i] ? 0 : 1;
        for (int p = 0; p < 3; ++p) {
            r[p] += f[p] * y[i];
            for (int q = 0; q < 3; ++q) a[p][q] += f[p] * f[q];
        }
    }
    if (n1 + nm < 3) return false;
    // drop a regime without measurements
    int keep[3], nk = 0;
    for (int p = 0; p < 3; ++p)
        if (a[p][p] > 0.0) keep[nk++] = p;
    if (nk < 2 || keep[0] != 0) return false;
    double m[3][4];
    for (int p = 0; p < nk; ++p) {
        for (int q = 0; q < nk; ++q) m[p][q] = a[keep[p]][keep[q]];
        m[p][nk] = r[keep[p]];
    }
    for (int c = 0; c < nk; ++c) {   // Gaussian elimination with partial pivoting
        int piv = c;
        for (int p = c + 1; p < nk; ++p)
            if (std::fabs(m[p][c]) > std::fabs(m[piv][c])) piv = p;
        if (!(std::fabs(m[piv][c]) > 0.0)) return false;
        for (int q = 0; q <= nk; ++q) std::swap(m[c][q], m[piv][q]);
        for (int p = 0; p < nk; ++p) {
            if (p == c) continue;
            const double f = m[p][c] / m[c][c];
            for (int q = c; q <= nk; ++q) m[p][q] -= f * m[c][q];
        }
    }
    double sol[3] = {0, -1, -1};
    for (int p = 0; p < nk; ++p) sol[keep[p]] = m[p][nk] / m[p][p];
    const double beta = sol[0];
    if (!(beta > 0.0)) return false;
    beta_out = beta;
    auto clampF = [](double v) { return std::min(1e7, std::max(0.0, v)); };
    if (a[1][1] > 0.0 && sol[1] >= 0.0) F1 = clampF(sol[1] / beta);
    if (a[2][2] > 0.0 && sol[2] >= 0.0) F = clampF(sol[2] / beta);
    return true;
}

std::string teams_key(const std::string &k) { return k + ";teams"; }

// The team planner's inputs (the context's model fields).
struct TeamModel {
    double F1 = 3000.0, F = 3000.0, beta = 0.0;
    int use = 0;
    std::vector<double> iters, ns, cta;
    static TeamModel of(const mpm_ctx *c)
    {
        TeamModel m;
        m.F1 = c->team_fixed1;
        m.F = c->team_fixed;
        m.beta = c->team_beta;
        m.use = c->team_use_iters;
        m.iters = c->item_iters;
        m.ns = c->item_ns;
        m.cta = c->item_cta;
        return m;
    }
    void apply(mpm_ctx *c) const
    {
        c->team_fixed1 = F1;
        c->team_fixed = F;
        c->team_beta = beta;
        c->team_use_iters = use;
        if (use) {
            c->item_iters = iters;
            c->item_ns = ns;
            c->item_cta = cta;
        }
        c->team_gen += 1;
    }
};

// One line per tuning: key F1 F beta f use n, then n Arnoldi steps, n times
// (ns) and n CTA counts of the plan's input, then "|" and the kept plan's
// per-team times (ns).
bool teams_lookup(const char *path, const std::string &key, TeamModel &m, double &f)
{
    if (!path) return false;
    FILE *fp = fopen(path, "r");
    if (!fp) return false;
    std::vector<char> line(1 << 22);
    bool found = false;
    while (fgets(line.data(), (int)line.size(), fp)) {
        std::string s(line.data());
        if (s.compare(0, key.size(), key) != 0 || s.size() <= key.size() || s[key.size()] != ' ') continue;
        const char *p = s.c_str() + key.size();
        char *e = nullptr;
        TeamModel t;
        t.F1 = strtod(p, &e);
        t.F = strtod(e, &e);
        t.beta = strtod(e, &e);
        const double f_ = strtod(e, &e);
        t.use = (int)strtol(e, &e, 10);
        const long n = strtol(e, &e, 10);
        if (n < 0 || n > (1 << 20)) continue;
        bool ok = true;
        for (std::vector<double> *v : {&t.iters, &t.ns, &t.cta}) {
            v->resize(n);
            for (long i = 0; i < n && ok; ++i) {
                char *e2 = nullptr;
                (*v)[i] = strtod(e, &e2);
                ok = e2 != e;
                e = e2;
            }
        }
        if (!ok) continue;
        m = t;
        f = f_;
        found = true;
    }
    fclose(fp);
    return found;
}

void teams_store(const char *path, const std::string &key, const TeamModel &m, double f,
                 const std::vector<double> &team_ns)
{
    if (!path) return;
    FILE *fp = fopen(path, "a");
    if (!fp) return;
    const size_t n = m.iters.size();
    const bool full = m.ns.size() == n && m.cta.size() == n;
    fprintf(fp, "%s %.17g %.17g %.17g %.6g %d %zu", key.c_str(), m.F1, m.F, m.beta, f, full ? m.use : 0,
            full ? n : (size_t)0);
    if (full)
        for (const std::vector<double> *v : {&m.iters, &m.ns, &m.cta})
            for (double x : *v) fprintf(fp, " %.17g", x);
    fprintf(fp, " |");
    for (double v : team_ns) fprintf(fp, " %.0f", v);
    fprintf(fp, "\n");
    fclose(fp);
}

}  // namespace

extern "C" mpm_status mpm_tune_teams(mpm_ctx *ctx, mpm_subgrid *const *subs, int32_t nsys, const mpm_opts *opt,
                                     int32_t rounds, const char *cache_path, double *history, double *out_fixed,
                                     void *stream)
{
    if (!ctx) return MPM_ERR_ARG;
    ctx->err.clear();
    if (!subs || nsys < 1 || !opt || rounds < 1 || rounds > 64)
        return mpm_fail(ctx, MPM_ERR_ARG, "tune_teams: null argument or rounds out of [1, 64]");
    for (int i = 0; i < nsys; ++i)
        if (!subs[i] || !subs[i]->assembled) return mpm_fail(ctx, MPM_ERR_ARG, "tune_teams: subgrid not assembled");
    const std::string key = teams_key(cache_key(ctx, subs, nsys, opt));
    cudaStream_t st = (cudaStream_t)stream;
    if (history)
        for (int r = 0; r <= rounds; ++r) history[3 * r] = history[3 * r + 1] = history[3 * r + 2] = -1.0;
    {
        TeamModel m;
        double f = 0.0;
        if (teams_lookup(cache_path, key, m, f)) {
            m.apply(ctx);
            if (history) {
                history[0] = f;
                history[1] = m.F1;
                history[2] = m.F;
            }
            if (out_fixed) {
                out_fixed[0] = m.F1;
                out_fixed[1] = m.F;
            }
            return MPM_OK;
        }
    }
    mpm_opts o = *opt;
    o.x0_given = 0;
    std::vector<mpm_report> reps(nsys);
    std::vector<double> xs, ys;
    std::vector<int> ones;
    double best_f = 1e300;
    TeamModel best;
    std::vector<double> best_team;
    int since = 0;
    for (int round = 0; round <= rounds; ++round) {
        if (round > 0) {
            double F1 = ctx->team_fixed1, F = ctx->team_fixed, beta = 0.0;
            if (fit_fixed(xs, ys, ones, F1, F, beta)) {
                ctx->team_fixed1 = F1;
                ctx->team_fixed = F;
                ctx->team_beta = beta;
            }
            // odd rounds weight the items by their Arnoldi steps, even rounds
            // plan from their measured times (both from the solve just run)
            ctx->team_use_iters = (round & 1) ? 1 : 2;
        } else {
            ctx->team_use_iters = 0;
        }
        const TeamModel used = TeamModel::of(ctx);
        const mpm_status r = mpm_solve_impl(ctx, subs, nullptr, nsys, &o, reps.data(), st);
        if (r != MPM_OK && r != MPM_ERR_NOCONV) return r;
        const double f = ctx->last_imbalance;
        if (history) {
            history[3 * round] = f;
            history[3 * round + 1] = used.F1;
            history[3 * round + 2] = used.F;
        }
        for (size_t i = 0; i < ctx->item_ns.size(); ++i)
            if (ctx->item_iters[i] > 0.0) {
                xs.push_back((ctx->item_ne[i] + 1.0) / ctx->item_cta[i]);
                ys.push_back(ctx->item_ns[i] / ctx->item_iters[i]);
                ones.push_back(ctx->item_cta[i] <= 1.0 ? 1 : 0);
            }
        if (f < best_f) {
            best_f = f;
            best = used;
            best_team = ctx->team_ns;
            since = 0;
        } else if (++since >= 2 && round >= 2) {
            break;
        }
    }
    ctx->err.clear();
    best.apply(ctx);
    teams_store(cache_path, key, best, best_f, best_team);
    if (out_fixed) {
        out_fixed[0] = best.F1;
        out_fixed[1] = best.F;
    }
    // leave the iterates at c^n for the caller's own solve
    for (int i = 0; i < nsys; ++i) {
        mpm_subgrid *sub = subs[i];
        for (int s = 0; s < sub->nspecies; ++s)
            MPM_CU(cudaMemcpyAsync(sub->x[s], sub->cn[s], (size_t)sub->NE * sizeof(double), cudaMemcpyDeviceToDevice, st));
        sub->x_fresh = true;
    }
    return MPM_OK;
}
