// solver.cu -- host side of the persistent GMRES (Sec. 2.4): kernel variant
// selection, the team planner, launch, report, the batched step and the
// device-resident step as CUDA graphs.  The device code is in
// solver_kernels.cuh.
#include <algorithm>
#include <cstring>
#include <vector>

#include "solver_kernels.cuh"

namespace mpm {

// Kernel variants: variant 0 is the default of each (precision, restart
// bucket), chosen by measurement on the 256^3 shell workload.  FP32, m <= 8:
// 0: one element (or 4-element chunk) per thread at one CTA/SM of 512 threads
// (up to 128 registers), 1: one CTA/SM of 768, 2: two elements at two CTAs/SM
// of 512, 3: two elements at one CTA/SM of 512, 4: one CTA/SM of 1024, 5: two
// CTAs/SM of 512 (64 registers), 6: one CTA/SM of 640.  FP64, m <= 8: 0: two
// elements at one CTA/SM of 512, 1: one element at two CTAs/SM, 2: one
// element at one CTA/SM of 1024, 3: one element at one CTA/SM of 768, 4: two
// elements at one CTA/SM of 768, 5: one element at one CTA/SM of 512.
// The instances live in the solver_inst_*.cu translation units.
static Variant pick(int prec, int maxm, int variant)
{
    if (prec != 0) {
        if (maxm == 16) return inst_f32_16_1_1_512();
        if (maxm == 32) return inst_f32_32_1_1_512();
        switch (variant) {
        case 1: return inst_f32_8_1_1_768();
        case 2: return inst_f32_8_2_2_512();
        case 3: return inst_f32_8_2_1_512();
        case 4: return inst_f32_8_1_1_1024();
        case 5: return inst_f32_8_1_2_512();
        case 6: return inst_f32_8_1_1_640();
        default: return inst_f32_8_1_1_512();
        }
    }
    if (maxm == 16) return inst_f64_16_1_1_512();
    if (maxm == 32) return inst_f64_32_1_1_512();
    switch (variant) {
    case 1: return inst_f64_8_1_2_512();
    case 2: return inst_f64_8_1_1_1024();
    case 3: return inst_f64_8_1_1_768();
    case 4: return inst_f64_8_2_1_768();
    case 5: return inst_f64_8_1_1_512();
    default: return inst_f64_8_2_1_512();
    }
}

}  // namespace mpm

using namespace mpm;

SysDev mpm_make_sysdev(const mpm_subgrid *sub)
{
    SysDev S;
    memset(&S, 0, sizeof(S));
    S.NE = sub->NE;
    S.ltx = sub->lt[0];
    S.lty = sub->lt[1];
    S.ltz = sub->lt[2];
    S.nspecies = sub->nspecies;
    S.nbr = sub->nbr;
    S.flags = sub->flags;
    S.dfac = sub->dfac;
    S.a = sub->a;
    S.err = sub->err;
    for (int s = 0; s < sub->nspecies; ++s) {
        S.x[s] = sub->x[s];
        S.b[s] = sub->b[s];
        S.diag[s] = sub->diag[s];
        S.diag32[s] = sub->diag32[s];
        S.off[s] = sub->off[s];
        S.Dsp[s] = sub->Dsp[s];
    }
    return S;
}

// Co-resident CTAs of a variant's kernel (the solve, or the whole step).
static int variant_max_blocks(mpm_ctx *ctx, const Variant &v, bool step)
{
    const void *f = step ? (const void *)v.stepfn : (const void *)v.fn;
    if (v.smem > 48 * 1024) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, v.nt, v.smem) != cudaSuccess) return 0;
    return per_sm * ctx->num_sms;
}

int mpm_solver_max_blocks(mpm_ctx *ctx, int prec, int m, int variant)
{
    const int maxm = m <= 8 ? 8 : (m <= 16 ? 16 : 32);
    return variant_max_blocks(ctx, pick(prec, maxm, variant), false);
}

// Number of kernel variants of a (precision, restart) bucket (for the tuner).
int mpm_solver_variants(int prec, int m)
{
    if (m > 8) return 1;
    return prec == 1 ? 7 : 6;
}

static size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

// Team plan of the batched form, with the paper's load-imbalance concern
// (Sec. 2.5) in mind.  Item i costs it_i (F1 + NE_i) element-equivalents on a
// one-CTA team and it_i (F + NE_i / c) on a team of c > 1 CTAs: it_i Arnoldi
// passes, each a fixed part (F1: block barriers and the least squares; F:
// grid barriers among the team's CTAs as well) and a streaming part.  Without
// a measured model it_i = 1 and F1 = F = 3000 (set by timing the 64-patch
// batch); mpm_tune_teams fits F1 and F to measured item times and takes it_i
// from the previous solve.  For a candidate makespan T, items whose one-CTA
// cost fits in T are packed first-fit-decreasing onto one-CTA teams of
// capacity T; larger items get ceil(work_i / (T - fix_i)) CTAs of their own.
// The smallest T that fits in G CTAs is kept (binary search), and the spare
// CTAs go to the teams with the most streaming work per CTA.
struct ItemCost {
    double one;      // on one CTA
    double fix;      // fixed part on a team of several CTAs
    double work;     // streaming part (divided by the team's CTAs)
};

static bool try_plan(const std::vector<ItemCost> &ic, const std::vector<int> &idx, int G, double T,
                     std::vector<std::vector<int>> &members, std::vector<int> &nbk)
{
    members.clear();
    nbk.clear();
    std::vector<double> load;
    int used = 0;
    for (int i : idx) {
        const double one = ic[i].one;
        if (one > T) {
            if (T <= ic[i].fix * 1.05) return false;
            const int c = std::max(2, (int)std::ceil(ic[i].work / (T - ic[i].fix)));
            members.push_back({i});
            nbk.push_back(c);
            load.push_back(-1.0);
            used += c;
        } else {
            int t = -1;
            for (size_t k = 0; k < load.size(); ++k)
                if (load[k] >= 0.0 && load[k] + one <= T) { t = (int)k; break; }
            if (t < 0) {
                members.push_back({});
                nbk.push_back(1);
                load.push_back(0.0);
                t = (int)load.size() - 1;
                used += 1;
            }
            members[t].push_back(i);
            load[t] += one;
        }
        if (used > G) return false;
    }
    return used <= G;
}

static void plan_teams(const std::vector<ItemCost> &ic, int G, std::vector<TeamDesc> &teams,
                       std::vector<int32_t> &order, std::vector<int32_t> &block_team)
{
    const int nsys = (int)ic.size();
    std::vector<int> idx(nsys);
    for (int i = 0; i < nsys; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return ic[a].one > ic[b].one; });
    std::vector<std::vector<int>> members;
    std::vector<int> nbk;
    if (nsys == 1) {
        members = {{0}};
        nbk = {G};
    } else {
        double hi = 1.0, lo = 0.0;   // hi: everything on one CTA
        for (int i = 0; i < nsys; ++i) {
            hi += ic[i].one;
            lo = std::max(lo, std::min(ic[i].one, ic[i].fix * 1.05));
        }
        for (int it = 0; it < 60; ++it) {
            const double mid = 0.5 * (lo + hi);
            std::vector<std::vector<int>> m2;
            std::vector<int> n2;
            if (try_plan(ic, idx, G, mid, m2, n2)) hi = mid;
            else lo = mid;
        }
        if (!try_plan(ic, idx, G, hi, members, nbk)) {   // cannot happen for G >= 1; keep a valid plan
            members = {idx};
            nbk = {G};
        }
        int used = 0;
        for (int c : nbk) used += c;
        // spare CTAs to the teams with the most streaming work per CTA
        while (used < G) {
            int best = 0;
            double bw = -1.0;
            for (size_t t = 0; t < members.size(); ++t) {
                double w = 0.0;
                for (int i : members[t]) w += ic[i].work;
                if (w / nbk[t] > bw) { bw = w / nbk[t]; best = (int)t; }
            }
            nbk[best] += 1;
            ++used;
        }
    }
    teams.clear();
    order.clear();
    block_team.clear();
    int fb = 0;
    for (size_t t = 0; t < members.size(); ++t) {
        TeamDesc d;
        d.first_block = fb;
        d.nblocks = nbk[t];
        d.sys_begin = (int32_t)order.size();
        for (int i : members[t]) order.push_back(i);
        d.sys_end = (int32_t)order.size();
        teams.push_back(d);
        for (int b = 0; b < nbk[t]; ++b) block_team.push_back((int32_t)t);
        fb += nbk[t];
    }
}

// ------------------------------------------------------------------ solve plan / enqueue / finish
struct SolvePlan {
    int nsys = 0, nitem = 0, G = 0, nteam = 0;
    size_t smem = 0;
    int nt = kSB;                   // threads per CTA
    KernFn fn = nullptr;
    StepFn stepfn = nullptr;        // the whole-step kernel of the same variant
    std::vector<SysDev> sd;
    std::vector<int> item_sys, item_sp;
    std::vector<TeamDesc> teams;
    std::vector<int32_t> order, block_team;
    size_t o_sys = 0, o_team = 0, o_order = 0, o_bt = 0, o_rep = 0, args_need = 0;
    SolveArgs sa;
};

static mpm_status check_opts(mpm_ctx *ctx, const mpm_opts *opt)
{
    if (!opt) return mpm_fail(ctx, MPM_ERR_ARG, "solve: null options");
    if (opt->restart < 1 || opt->restart > MPM_MAX_RESTART) return mpm_fail(ctx, MPM_ERR_ARG, "solve: restart out of [1, 32]");
    if (opt->maxit < 1) return mpm_fail(ctx, MPM_ERR_ARG, "solve: maxit < 1");
    if (opt->precision != 0 && opt->precision != 1) return mpm_fail(ctx, MPM_ERR_ARG, "solve: precision must be 0 or 1");
    if (opt->reorth != 0 && opt->reorth != 1) return mpm_fail(ctx, MPM_ERR_ARG, "solve: reorth must be 0 or 1");
    if (opt->box_every < 0 || opt->box_guard < 0)
        return mpm_fail(ctx, MPM_ERR_ARG, "solve: box_every and box_guard must not be negative");
    if (!(opt->rtol >= 0.0) || !(opt->atol >= 0.0)) return mpm_fail(ctx, MPM_ERR_ARG, "solve: negative tolerance");
    if (opt->precision == 1 && !(opt->inner_rtol > 0.0 && opt->inner_rtol < 1.0))
        return mpm_fail(ctx, MPM_ERR_ARG, "solve: inner_rtol must be in (0, 1)");
    return MPM_OK;
}

// Host planning: Krylov bases (grown here, never during a capture), one work
// item per (system, species), the grid, the team split and the descriptor
// layout.  reset_x: restore x = c^n where a previous solve moved it (queued
// on st).
// Overrides of the device-resident step (one system): the Krylov stride is
// set by the buffers' element capacity, the work estimate by the previous
// step's element count, the grid by the caller, and the kernel reads the
// element count from the device.
struct PlanOverride {
    int64_t NE_cap, NE_est;
    const int64_t *NEp;
    int G;
};

static mpm_status plan_solve(mpm_ctx *ctx, mpm_subgrid *const *subs, int nsys, const mpm_opts *opt, bool reset_x,
                             cudaStream_t st, SolvePlan &P, const PlanOverride *ov = nullptr)
{
    const int m = opt->restart;
    const int maxm = m <= 8 ? 8 : (m <= 16 ? 16 : 32);
    const size_t tsz = opt->precision ? sizeof(float) : sizeof(double);
    P.nsys = nsys;
    for (int i = 0; i < nsys; ++i) {
        if (!subs[i]) return mpm_fail(ctx, MPM_ERR_ARG, "solve: null subgrid");
        if (!subs[i]->assembled && reset_x) return mpm_fail(ctx, MPM_ERR_ARG, "solve: subgrid not assembled");
    }
    std::vector<double> work;
    for (int i = 0; i < nsys; ++i) {
        mpm_subgrid *sub = subs[i];
        const int64_t ne_v = ov ? ov->NE_cap : sub->NE;
        const int64_t vstride = ne_v > 0 ? ((ne_v + 63) / 64) * 64 : 64;
        const size_t per = a256((size_t)(m + 1) * (size_t)vstride * tsz);
        mpm_status r = mpm_grow(ctx, &sub->krylov, &sub->krylov_bytes, per * sub->nspecies, "Krylov basis");
        if (r != MPM_OK) return r;
        if (reset_x && !opt->x0_given && !sub->x_fresh) {
            for (int s = 0; s < sub->nspecies; ++s)
                MPM_CU(cudaMemcpyAsync(sub->x[s], sub->cn[s], (size_t)sub->NE * sizeof(double), cudaMemcpyDeviceToDevice, st));
            sub->x_fresh = true;
        }
        SysDev full = mpm_make_sysdev(sub);
        if (ov) {
            full.NE = 0;
            full.NEp = ov->NEp;
        }
        for (int s = 0; s < sub->nspecies; ++s) {
            SysDev d = full;
            d.nspecies = 1;
            for (int t = 0; t < kMaxSpecies; ++t) {
                d.x[t] = nullptr; d.b[t] = nullptr; d.diag[t] = nullptr; d.diag32[t] = nullptr; d.V[t] = nullptr;
                d.off[t] = 0.0; d.Dsp[t] = 0.0;
            }
            d.x[0] = full.x[s];
            d.b[0] = full.b[s];
            d.diag[0] = full.diag[s];
            d.diag32[0] = full.diag32[s];
            d.off[0] = full.off[s];
            d.Dsp[0] = full.Dsp[s];
            d.vstride = vstride;
            d.V[0] = (char *)sub->krylov + per * s;
            P.sd.push_back(d);
            work.push_back((double)(ov ? ov->NE_est : sub->NE) + 1.0);
            P.item_sys.push_back(i);
            P.item_sp.push_back(s);
        }
    }
    P.nitem = (int)P.sd.size();
    {
        const Variant v = pick(opt->precision, maxm, ctx->solver_variant);
        P.fn = v.fn;
        P.stepfn = v.stepfn;
        P.smem = v.smem;
        P.nt = v.nt;
    }
    const int gmax = mpm_solver_max_blocks(ctx, opt->precision, m, ctx->solver_variant);
    if (gmax < 1) return mpm_fail(ctx, MPM_ERR_CUDA, "solve: occupancy query failed");
    if (ov && ov->G > 0) P.G = std::min(ov->G, gmax);
    else if (opt->nblocks > 0) P.G = std::min(opt->nblocks, gmax);
    else {
        double tot = 0.0;
        for (double w : work) tot += w;
        // about two elements per thread and item at least
        const double want = tot / (P.nt * 2.0);
        P.G = (int)std::min<double>(gmax, std::max(1.0, want));
        P.G = std::max(P.G, std::min(P.nitem, gmax));
    }
    {
        // the cost model: measured Arnoldi steps per item when the context has
        // them for a batch of this many items, else one pass each
        const bool iters = ctx->team_use_iters && (int)ctx->item_iters.size() == P.nitem;
        const bool timed = ctx->team_use_iters == 2 && iters && (int)ctx->item_ns.size() == P.nitem &&
                           ctx->team_beta > 0.0;
        std::vector<ItemCost> ic(P.nitem);
        for (int i = 0; i < P.nitem; ++i) {
            const double it = iters ? std::max(1.0, ctx->item_iters[i]) : 1.0;
            if (timed) {
                // the measured time of the item on its c CTAs, split into the
                // fixed part (fitted per Arnoldi step) and the streaming part
                // (which c CTAs divided), in ns
                const double a1 = ctx->team_fixed1 * ctx->team_beta, a = ctx->team_fixed * ctx->team_beta;
                const double c = std::max(1.0, ctx->item_cta[i]), t = ctx->item_ns[i];
                const double stream = std::max(0.0, t - it * (c > 1.0 ? a : a1)) * c;
                ic[i].one = it * a1 + stream;
                ic[i].fix = it * a;
                ic[i].work = stream;
            } else {
                ic[i].one = it * (ctx->team_fixed1 + work[i]);
                ic[i].fix = it * ctx->team_fixed;
                ic[i].work = it * work[i];
            }
        }
        plan_teams(ic, P.G, P.teams, P.order, P.block_team);
    }
    P.nteam = (int)P.teams.size();
    P.o_sys = 0;
    P.o_team = a256(P.o_sys + sizeof(SysDev) * P.nitem);
    P.o_order = a256(P.o_team + sizeof(TeamDesc) * P.nteam);
    P.o_bt = a256(P.o_order + sizeof(int32_t) * P.nitem);
    P.o_rep = a256(P.o_bt + sizeof(int32_t) * P.G);
    P.args_need = a256(P.o_rep + sizeof(SysReport) * P.nitem);
    const size_t pneed = 2 * (size_t)P.G * kKMax * sizeof(double);
    mpm_status r = mpm_grow(ctx, (void **)&ctx->d_partials, &ctx->partials_cap, pneed, "reduction partials");
    if (r != MPM_OK) return r;
    SolveArgs &sa = P.sa;
    memset(&sa, 0, sizeof(sa));
    sa.partials = ctx->d_partials;
    sa.rtol = opt->rtol;
    sa.atol = opt->atol;
    sa.inner_rtol = opt->precision ? opt->inner_rtol : 0.0;
    sa.reorth = opt->reorth;
    sa.m = m;
    sa.maxit = opt->maxit;
    sa.timeout_ns = ctx->timeout_ns;
    sa.skip_block = ctx->skip_block;
    return MPM_OK;
}

static void fill_descriptors(const SolvePlan &P, char *h)
{
    memcpy(h + P.o_sys, P.sd.data(), sizeof(SysDev) * P.nitem);
    memcpy(h + P.o_team, P.teams.data(), sizeof(TeamDesc) * P.nteam);
    memcpy(h + P.o_order, P.order.data(), sizeof(int32_t) * P.nitem);
    memcpy(h + P.o_bt, P.block_team.data(), sizeof(int32_t) * P.G);
}

// Queue the solve: counters and reports cleared, then the cooperative launch.
// Only stream work (capturable); descriptors already sit at d_args.
static mpm_status enqueue_solve(mpm_ctx *ctx, SolvePlan &P, char *d_args, uint32_t *d_bar, int32_t *d_abort,
                                unsigned long long *d_prof, cudaStream_t st, bool zeroed = false)
{
    SolveArgs sa = P.sa;
    sa.sys = (const SysDev *)(d_args + P.o_sys);
    sa.teams = (const TeamDesc *)(d_args + P.o_team);
    sa.sys_order = (const int32_t *)(d_args + P.o_order);
    sa.block_team = (const int32_t *)(d_args + P.o_bt);
    sa.reports = (SysReport *)(d_args + P.o_rep);
    sa.bar = d_bar;
    sa.abort_flag = d_abort;
    sa.prof = d_prof;
    if (!zeroed) {   // else a preceding kernel of the same stream zeroed them
        MPM_CU(cudaMemsetAsync(d_bar, 0, (size_t)P.nteam * 32 * sizeof(uint32_t), st));
        MPM_CU(cudaMemsetAsync(d_abort, 0, sizeof(int32_t), st));
        MPM_CU(cudaMemsetAsync(d_args + P.o_rep, 0, sizeof(SysReport) * P.nitem, st));
    }
    if (d_prof) MPM_CU(cudaMemsetAsync(d_prof, 0, kProfSlots * sizeof(unsigned long long), st));
    void *kargs[] = {&sa};
    MPM_CU(cudaLaunchCooperativeKernel((const void *)P.fn, dim3(P.G), dim3(P.nt), kargs, P.smem, st));
    ctx->launches += 1;
    return MPM_OK;
}

static int status_rank(int s)
{
    switch (s) {
    case MPM_OK: return 0;
    case MPM_ERR_NOCONV: return 1;
    case MPM_ERR_BREAKDOWN: return 2;
    case MPM_ERR_ARG: return 3;
    case MPM_ERR_TIMEOUT: return 4;
    default: return 5;
    }
}

// Map the per-item reports back to systems; scatter (queued) unless the solve
// timed out or scatter already ran on the device.
static mpm_status finish_solve(mpm_ctx *ctx, const SolvePlan &P, mpm_subgrid *const *subs, const SysReport *hrep,
                               bool timed_out, float ms, mpm_report *reps, const mpm_lattice *const *scatter_to,
                               cudaStream_t st)
{
    mpm_status worst = MPM_OK;
    bool bad_id = false;
    std::vector<mpm_report> R(P.nsys);
    for (int i = 0; i < P.nsys; ++i) {
        memset(&R[i], 0, sizeof(mpm_report));
        mpm_subgrid *sub = subs[i];
        sub->x_fresh = false;
        R[i].box_voxels = (int64_t)sub->n[0] * sub->n[1] * sub->n[2];
        R[i].mask_voxels = sub->mask_voxels;
        R[i].stored_voxels = sub->NE;
        R[i].solve_ms = ms;
    }
    // the paper's load imbalance f = t_max / <t> - 1 (Sec. 2.5), over CTA
    // teams; the per-item measurements feed the team planner's model
    {
        std::vector<double> tt(P.nteam, 0.0);
        ctx->item_iters.assign(P.nitem, 0.0);
        ctx->item_ne.assign(P.nitem, 0.0);
        ctx->item_cta.assign(P.nitem, 1.0);
        ctx->item_ns.assign(P.nitem, 0.0);
        for (int t = 0; t < P.nteam; ++t)
            for (int k = P.teams[t].sys_begin; k < P.teams[t].sys_end; ++k) {
                const int it = P.order[k];
                tt[t] += (double)hrep[it].t_ns;
                ctx->item_iters[it] = (double)hrep[it].iters[0];
                ctx->item_ne[it] = (double)subs[P.item_sys[it]]->NE;
                ctx->item_cta[it] = (double)P.teams[t].nblocks;
                ctx->item_ns[it] = (double)hrep[it].t_ns;
            }
        ctx->team_ns = tt;
        double mx = 0.0, mean = 0.0;
        for (double v : tt) { mx = std::max(mx, v); mean += v; }
        mean /= std::max(1, P.nteam);
        ctx->last_imbalance = mean > 0.0 ? mx / mean - 1.0 : 0.0;
    }
    for (int it = 0; it < P.nitem; ++it) {
        const int i = P.item_sys[it], s = P.item_sp[it];
        R[i].item_ms[s] = (double)hrep[it].t_ns * 1e-6;
        R[i].iters[s] = hrep[it].iters[0];
        R[i].jsum[s] = hrep[it].jsum[0];
        R[i].cycles[s] = hrep[it].cycles[0];
        int stt = hrep[it].status[0];
        if (timed_out) stt = MPM_ERR_TIMEOUT;
        else if (stt == ST_RUN) stt = MPM_ERR_NOCONV;
        if (stt == MPM_ERR_ARG) bad_id = true;
        R[i].status[s] = stt;
        R[i].res[s] = hrep[it].res[0];
        R[i].bnorm[s] = hrep[it].bnorm[0];
        R[i].reorth[s] = hrep[it].reorth[0];
        if (status_rank(stt) > status_rank(worst)) worst = (mpm_status)stt;
    }
    for (int i = 0; i < P.nsys; ++i) {
        if (reps) reps[i] = R[i];
        if (!timed_out && scatter_to && scatter_to[i]) {
            mpm_status r = mpm_scatter_impl(ctx, subs[i], scatter_to[i], st);
            if (r != MPM_OK) return r;
        }
    }
    if (timed_out) return mpm_fail(ctx, MPM_ERR_TIMEOUT, "solve: a bounded inter-CTA wait expired");
    if (bad_id) return mpm_fail(ctx, MPM_ERR_ARG, "solve: a cell id lies outside the rate tables");
    if (worst != MPM_OK) mpm_fail(ctx, worst, "solve: not every species converged");
    return worst;
}

static mpm_status ensure_stage(mpm_ctx *ctx, size_t need)
{
    if (ctx->stage_cap >= need) return MPM_OK;
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    ctx->h_stage = nullptr;
    ctx->stage_cap = 0;
    MPM_CU(cudaMallocHost(&ctx->h_stage, need));
    ctx->stage_cap = need;
    return MPM_OK;
}

mpm_status mpm_solve_impl(mpm_ctx *ctx, mpm_subgrid *const *subs, const mpm_lattice *const *scatter_to,
                          int32_t nsys, const mpm_opts *opt, mpm_report *reps, cudaStream_t st)
{
    if (!subs || nsys < 1) return mpm_fail(ctx, MPM_ERR_ARG, "solve: null argument or nsys < 1");
    mpm_status r = check_opts(ctx, opt);
    if (r != MPM_OK) return r;
    SolvePlan P;
    r = plan_solve(ctx, subs, nsys, opt, true, st, P);
    if (r != MPM_OK) return r;
    r = mpm_grow(ctx, &ctx->d_args, &ctx->args_cap, P.args_need, "solver descriptors");
    if (r != MPM_OK) return r;
    r = ensure_stage(ctx, P.args_need + 4096);
    if (r != MPM_OK) return r;
    if (ctx->bar_cap < P.nteam) {
        if (ctx->d_bar) cudaFree(ctx->d_bar);
        ctx->d_bar = nullptr;
        ctx->bar_cap = 0;
        MPM_CU(cudaMalloc(&ctx->d_bar, (size_t)P.nteam * 32 * sizeof(uint32_t)));
        ctx->bar_cap = P.nteam;
    }
    if (ctx->phase_prof && !ctx->d_prof) MPM_CU(cudaMalloc(&ctx->d_prof, kProfSlots * sizeof(unsigned long long)));
    // the staging buffer is free: every call that uses it ends with a stream synchronisation
    char *hs = (char *)ctx->h_stage;
    fill_descriptors(P, hs);
    MPM_CU(cudaMemcpyAsync(ctx->d_args, hs, P.o_rep, cudaMemcpyHostToDevice, st));
    MPM_CU(cudaEventRecord(ctx->ev0, st));
    r = enqueue_solve(ctx, P, (char *)ctx->d_args, ctx->d_bar, ctx->d_abort, ctx->phase_prof ? ctx->d_prof : nullptr, st);
    if (r != MPM_OK) return r;
    MPM_CU(cudaEventRecord(ctx->ev1, st));
    SysReport *hrep = (SysReport *)(hs + P.o_rep);
    MPM_CU(cudaMemcpyAsync(hrep, (char *)ctx->d_args + P.o_rep, sizeof(SysReport) * P.nitem, cudaMemcpyDeviceToHost, st));
    int32_t *hflags = (int32_t *)(hs + P.args_need);
    MPM_CU(cudaMemcpyAsync(hflags, ctx->d_abort, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (ctx->phase_prof) MPM_CU(cudaMemcpyAsync(ctx->h_prof, ctx->d_prof, kProfSlots * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    MPM_CU(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    const bool timed_out = hflags[0] != 0;
    r = finish_solve(ctx, P, subs, hrep, timed_out, ms, reps, scatter_to, st);
    if (timed_out) cudaMemsetAsync(ctx->d_abort, 0, sizeof(int32_t), st);
    return r;
}

// ------------------------------------------------------------------ batched step in a CUDA graph
struct BatchGraph {
    bool valid = false;
    bool graph_failed = false;
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
    char *d_args = nullptr;
    size_t args_cap = 0;
    uint32_t *d_bar = nullptr;
    int32_t *d_abort = nullptr;
    int64_t graph_launches = 0;    // kernels in the captured graph
    SolvePlan plan;
    std::vector<char> h_desc;      // batched preparation / scatter descriptors
    char *d_desc = nullptr;
    size_t desc_cap = 0;
    int64_t prep_blocks = 0;
    double *d_partials = nullptr;  // the graph's own reduction buffer (the context's may move)
    size_t partials_cap = 0;
};

static void batch_key(mpm_ctx *ctx, mpm_subgrid *const *subs, const mpm_lattice *const *lats,
                      const mpm_params *const *prms, int nsys, const mpm_opts *opt, std::vector<unsigned char> &k)
{
    auto put = [&](const void *p, size_t n) {
        const unsigned char *c = (const unsigned char *)p;
        k.insert(k.end(), c, c + n);
    };
    put(&nsys, sizeof(nsys));
    put(opt, sizeof(*opt));
    put(&ctx->solver_variant, sizeof(int32_t));
    put(&ctx->timeout_ns, sizeof(uint64_t));
    put(&ctx->skip_block, sizeof(int32_t));
    put(&ctx->team_gen, sizeof(uint64_t));
    for (int i = 0; i < nsys; ++i) {
        put(&subs[i], sizeof(void *));
        put(&subs[i]->gen, sizeof(subs[i]->gen));
        put(&subs[i]->krylov, sizeof(void *));
        put(lats[i], sizeof(mpm_lattice));
        put(prms[i], sizeof(mpm_params));
    }
}

void mpm_batch_graph_free(mpm_ctx *ctx)
{
    BatchGraph *B = (BatchGraph *)ctx->batch_graph;
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    cudaFree(B->d_args);
    cudaFree(B->d_bar);
    cudaFree(B->d_abort);
    cudaFree(B->d_desc);
    cudaFree(B->d_partials);
    delete B;
    ctx->batch_graph = nullptr;
}

mpm_status mpm_batch_step_impl(mpm_ctx *ctx, mpm_subgrid *const *subs, const mpm_lattice *const *lats,
                               const mpm_params *const *prms, int32_t nsys, const mpm_opts *opt, mpm_report *reps,
                               cudaStream_t st)
{
    if (!subs || !lats || !prms || nsys < 1) return mpm_fail(ctx, MPM_ERR_ARG, "batch_step: null argument or nsys < 1");
    mpm_status r = check_opts(ctx, opt);
    if (r != MPM_OK) return r;
    for (int i = 0; i < nsys; ++i)
        if (!subs[i] || !lats[i] || !prms[i] || !subs[i]->extracted)
            return mpm_fail(ctx, MPM_ERR_ARG, "batch_step: null or unextracted system");
    r = mpm_batch_prep_check(ctx, subs, lats, prms, nsys);
    if (r != MPM_OK) return r;
    if (!ctx->batch_graph) ctx->batch_graph = new BatchGraph();
    BatchGraph *B = (BatchGraph *)ctx->batch_graph;
    std::vector<unsigned char> key;
    batch_key(ctx, subs, lats, prms, nsys, opt, key);
    const bool use_graph = !ctx->phase_prof;
    if (!(B->valid && B->key == key) || !use_graph) {
        // (re)build: eager planning first (allocations), then capture
        if (B->exec) cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
        B->valid = false;
        const size_t dbytes = mpm_batch_desc_bytes(nsys);
        B->h_desc.assign(dbytes, 0);
        mpm_batch_desc_fill(subs, lats, prms, nsys, B->h_desc.data(), &B->prep_blocks);
        r = mpm_grow(ctx, (void **)&B->d_desc, &B->desc_cap, dbytes, "batch preparation descriptors");
        if (r != MPM_OK) return r;
        MPM_CU(cudaMemcpyAsync(B->d_desc, B->h_desc.data(), dbytes, cudaMemcpyHostToDevice, st));
        r = mpm_batch_prep_launch(ctx, B->d_desc, nsys, B->prep_blocks, st);
        if (r != MPM_OK) return r;
        for (int i = 0; i < nsys; ++i) { subs[i]->assembled = true; subs[i]->x_fresh = true; }
        B->plan = SolvePlan();
        r = plan_solve(ctx, subs, nsys, opt, false, st, B->plan);
        if (r != MPM_OK) return r;
        r = mpm_grow(ctx, (void **)&B->d_args, &B->args_cap, B->plan.args_need, "batch descriptors");
        if (r != MPM_OK) return r;
        r = mpm_grow(ctx, (void **)&B->d_partials, &B->partials_cap, 2 * (size_t)B->plan.G * kKMax * sizeof(double),
                     "batch reduction partials");
        if (r != MPM_OK) return r;
        B->plan.sa.partials = B->d_partials;
        if (!B->d_bar) {
            MPM_CU(cudaMalloc(&B->d_bar, (size_t)ctx->num_sms * 4 * 32 * sizeof(uint32_t)));
            MPM_CU(cudaMalloc(&B->d_abort, 256));
        }
        if (B->plan.nteam > ctx->num_sms * 4) return mpm_fail(ctx, MPM_ERR_ARG, "batch_step: too many teams");
        r = ensure_stage(ctx, B->plan.args_need + 4096);
        if (r != MPM_OK) return r;
        fill_descriptors(B->plan, (char *)ctx->h_stage);
        MPM_CU(cudaMemcpyAsync(B->d_args, ctx->h_stage, B->plan.o_rep, cudaMemcpyHostToDevice, st));
        MPM_CU(cudaStreamSynchronize(st));   // descriptors in place before any capture
        if (use_graph && !B->graph_failed) {
            // capture on a stream of the context (the caller's may be the legacy
            // default stream, which cannot be captured); the graph is then
            // launched on the caller's stream
            if (!ctx->cap_stream) MPM_CU(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
            cudaStream_t cs = ctx->cap_stream;
            cudaGraph_t g = nullptr;
            const int64_t launches0 = ctx->launches;
            bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                ok = mpm_batch_prep_launch(ctx, B->d_desc, nsys, B->prep_blocks, cs) == MPM_OK;
                ok = ok && enqueue_solve(ctx, B->plan, B->d_args, B->d_bar, B->d_abort, nullptr, cs) == MPM_OK;
                ok = ok && mpm_batch_scatter_launch(ctx, B->d_desc, nsys, B->prep_blocks, cs) == MPM_OK;
                const cudaError_t ec = cudaStreamEndCapture(cs, &g);
                ok = ok && ec == cudaSuccess && g != nullptr;
            }
            B->graph_launches = ctx->launches - launches0;
            ctx->launches = launches0;   // captured, not launched
            if (ok) ok = cudaGraphInstantiate(&B->exec, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            if (ok) {
                B->valid = true;
                B->key = key;
            } else {
                B->exec = nullptr;
                B->graph_failed = true;   // this device or driver cannot capture it: stay eager
            }
        }
    }
    SolvePlan &P = B->plan;
    r = ensure_stage(ctx, P.args_need + 4096);
    if (r != MPM_OK) return r;
    char *hs = (char *)ctx->h_stage;
    MPM_CU(cudaEventRecord(ctx->ev0, st));
    if (B->valid) {
        MPM_CU(cudaGraphLaunch(B->exec, st));
        ctx->launches += B->graph_launches;
    } else {
        // eager form of the same sequence (graph unavailable or phase timing on)
        r = mpm_batch_prep_launch(ctx, B->d_desc, nsys, B->prep_blocks, st);
        if (r != MPM_OK) return r;
        if (ctx->phase_prof && !ctx->d_prof) MPM_CU(cudaMalloc(&ctx->d_prof, kProfSlots * sizeof(unsigned long long)));
        r = enqueue_solve(ctx, P, B->d_args, B->d_bar, B->d_abort, ctx->phase_prof ? ctx->d_prof : nullptr, st);
        if (r != MPM_OK) return r;
        r = mpm_batch_scatter_launch(ctx, B->d_desc, nsys, B->prep_blocks, st);
        if (r != MPM_OK) return r;
    }
    MPM_CU(cudaEventRecord(ctx->ev1, st));
    SysReport *hrep = (SysReport *)(hs + P.o_rep);
    MPM_CU(cudaMemcpyAsync(hrep, B->d_args + P.o_rep, sizeof(SysReport) * P.nitem, cudaMemcpyDeviceToHost, st));
    int32_t *hflags = (int32_t *)(hs + P.args_need);
    MPM_CU(cudaMemcpyAsync(hflags, B->d_abort, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (ctx->phase_prof) MPM_CU(cudaMemcpyAsync(ctx->h_prof, ctx->d_prof, kProfSlots * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    MPM_CU(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    const bool timed_out = hflags[0] != 0;
    for (int i = 0; i < nsys; ++i) subs[i]->assembled = true;
    return finish_solve(ctx, P, subs, hrep, timed_out, ms, reps, nullptr, st);
}

int mpm_batch_graph_active(mpm_ctx *ctx)
{
    BatchGraph *B = (BatchGraph *)ctx->batch_graph;
    return B && B->valid ? 1 : 0;
}

// ------------------------------------------------------------------ device-resident step in a CUDA graph
// One step of one lattice with no host round trip between its stages: the
// extraction, preparation, solve, scatter and the copies of the results all
// run from one graph, with buffers sized for the whole lattice and the box
// and element count passed from kernel to kernel in device memory.
struct StepGraph {
    bool valid = false;
    bool graph_failed = false;
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_launches = 0;
    SolvePlan plan;
    int G = 0;                      // grid of the current plan
    int64_t last_NE = -1;           // element count of the previous step (-1: none)
    char *d_scr = nullptr;          // box (256 B), counts (256 B), abort flag (256 B), StepDyn (256 B)
    char *d_args = nullptr;         // solver descriptors and reports
    size_t args_cap = 0;
    uint32_t *d_bar = nullptr;      // team barrier counters
    double *d_partials = nullptr;
    size_t partials_cap = 0;
    double *d_rates = nullptr;      // rate tables of the preparation
    size_t rates_cap = 0;
    char *d_xscr = nullptr;         // per-CTA extraction partials, grid barrier, exit counter
    size_t xscr_cap = 0;
    char *h_out = nullptr;          // host-mapped: box, counts, abort flag, reports (written by the kernel)
    char *h_out_dev = nullptr;      // its device address
    size_t hout_cap = 0;
    // what mpm_step_wait needs from the last enqueued step
    bool pending = false;
    int32_t margin = 0, lt[3] = {2, 2, 2}, ldims[3] = {0, 0, 0};
    int gmax_key[3] = {-1, -1, -1};  // (precision, restart bucket, variant) of the cached grid limit
    int gmax = 0;
    mpm_cnn *cnn = nullptr;          // the network whose prediction starts each solve (null: c^n)
};

static constexpr size_t kOutBox = 0, kOutCount = 64, kOutAbort = 128, kOutRep = 256;
static constexpr size_t kScrBox = 0, kScrCount = 256, kScrAbort = 512, kScrDyn = 768, kScrCad = 896;
static constexpr size_t kOutNFull = 160;   // full extractions so far (StepCad::nfull)

// Extraction scratch for a grid of nb CTAs: box partials (32 B per CTA), count
// partials (16 B per CTA), then the grid barrier counter and the exit counter.
static size_t xscr_bytes(int nb) { return (size_t)nb * 48 + 512; }

void mpm_step_free(mpm_ctx *ctx, mpm_subgrid *sub)
{
    StepGraph *T = (StepGraph *)sub->step;
    if (!T) return;
    if (ctx) ctx->allocated -= T->args_cap + T->partials_cap + T->rates_cap + T->xscr_cap;
    if (T->exec) cudaGraphExecDestroy(T->exec);
    cudaFree(T->d_scr);
    cudaFree(T->d_args);
    cudaFree(T->d_bar);
    cudaFree(T->d_partials);
    cudaFree(T->d_rates);
    cudaFree(T->d_xscr);
    if (T->h_out) cudaFreeHost(T->h_out);
    delete T;
    sub->step = nullptr;
}

// Another extraction rewrote the subgrid's tables: the step's between-step
// state (activity bytes) must be set up again.
void mpm_step_invalidate(mpm_subgrid *sub)
{
    StepGraph *T = (StepGraph *)sub->step;
    if (T) T->valid = false;
}

// Static descriptor of a device-resident step (host image, passed by value).
static BatchSys step_sys(mpm_subgrid *sub, const mpm_lattice *lat, const mpm_params *prm, const double *d_rates)
{
    BatchSys S;
    memset(&S, 0, sizeof(S));
    S.tile_coord = sub->tile_coord;
    S.cell_id = lat->cell_id;
    S.mask = lat->mask;
    S.dfac_lat = lat->dfac;
    S.flags = sub->flags;
    S.cell = sub->cell;
    S.dfac = sub->dfac;
    for (int s = 0; s < sub->nspecies; ++s) {
        S.field[s] = lat->field[s];
        S.x[s] = sub->x[s];
        S.cn[s] = sub->cn[s];
        S.b[s] = sub->b[s];
        S.diag[s] = sub->diag[s];
        S.diag32[s] = sub->diag32[s];
    }
    S.err = sub->err;
    S.tile_index = sub->tile_index;
    S.nbr = sub->nbr;
    S.dk = d_rates;
    S.dq = d_rates + (size_t)prm->nspecies * prm->ncell;
    mpm_asm_coef(prm, &S.C);
    return S;
}

mpm_status mpm_cnn_enqueue_guess(mpm_ctx *ctx, mpm_cnn *c, mpm_subgrid *sub, const mpm_lattice *lat,
                                 const mpm_params *prm, const BoxGeo *d_geo, cudaStream_t st);
mpm_status mpm_cnn_check(mpm_ctx *ctx, mpm_cnn *c, const mpm_lattice *lat, const mpm_params *prm);

// One step on stream cs (captured or eager): the whole-step kernel, or, with
// a network attached, its extraction launch, the network's guess written
// into the iterate, and its solve launch.
static mpm_status enqueue_step(mpm_ctx *ctx, StepGraph *T, mpm_subgrid *sub, const mpm_lattice *lat,
                               const mpm_params *prm, int32_t margin, const mpm_opts *opt, cudaStream_t cs)
{
    SolvePlan &P = T->plan;
    const int nb = P.G;
    int32_t *d_box = (int32_t *)(T->d_scr + kScrBox);
    int64_t *d_count = (int64_t *)(T->d_scr + kScrCount);
    int32_t *d_abort = (int32_t *)(T->d_scr + kScrAbort);
    StepDyn *d_dyn = (StepDyn *)(T->d_scr + kScrDyn);
    char *d_rep = T->d_args + P.o_rep;
    const size_t rep_bytes = sizeof(SysReport) * P.nitem;
    StepArgs A;
    memset(&A, 0, sizeof(A));
    A.sa = P.sa;
    A.sa.sys = (const SysDev *)(T->d_args + P.o_sys);
    A.sa.teams = (const TeamDesc *)(T->d_args + P.o_team);
    A.sa.sys_order = (const int32_t *)(T->d_args + P.o_order);
    A.sa.block_team = (const int32_t *)(T->d_args + P.o_bt);
    A.sa.reports = (SysReport *)d_rep;
    A.sa.bar = T->d_bar;
    A.sa.abort_flag = d_abort;
    A.sa.prof = ctx->phase_prof ? ctx->d_prof : nullptr;
    ExtractArgs &X = A.xa;
    X.cell_id = lat->cell_id;
    X.mask = lat->mask;
    for (int d = 0; d < 3; ++d) { X.L[d] = lat->dims[d]; X.lt[d] = sub->lt[d]; }
    X.margin = margin;
    X.vec4 = ((uintptr_t)lat->cell_id % 16) == 0;
    X.part_box = (int32_t *)T->d_xscr;
    X.part_cnt = (unsigned long long *)(T->d_xscr + (size_t)nb * 32);
    X.bar = (uint32_t *)(T->d_xscr + (size_t)nb * 48);
    X.xabort = d_abort;
    X.timeout_ns = ctx->timeout_ns;
    X.box_out = d_box;
    X.geo_out = (BoxGeo *)(d_box + 8);
    X.count_out = (unsigned long long *)d_count;
    X.dyn = d_dyn;
    X.active = sub->active;
    X.tile_index = sub->tile_index;
    X.tile_coord = sub->tile_coord;
    X.err = sub->err;
    X.sbar = T->d_bar;
    X.nsbar = P.nteam * 32;
    X.srep = (uint32_t *)d_rep;
    X.nrep_words = (int32_t)(rep_bytes / 4);
    X.ra.nspecies = prm->nspecies;
    X.ra.ncell = prm->ncell;
    X.ra.dt = prm->dt;
    for (int s = 0; s < prm->nspecies; ++s) X.ra.mu[s] = prm->mu[s];
    X.ra.k_cell = prm->k_cell;
    X.ra.q_cell = prm->q_cell;
    X.ra.dk = T->d_rates;
    X.ra.dq = T->d_rates + (size_t)prm->nspecies * prm->ncell;
    X.prof = ctx->phase_prof ? ctx->d_prof : nullptr;
    X.cad = (StepCad *)(T->d_scr + kScrCad);
    X.box_every = opt->box_every;
    X.box_guard = opt->box_guard;
    A.S = step_sys(sub, lat, prm, T->d_rates);
    A.o.box = d_box;
    A.o.count = (const unsigned long long *)d_count;
    A.o.reports = (const uint32_t *)d_rep;
    A.o.nrep_words = (int32_t)(rep_bytes / 4);
    A.o.host = T->h_out_dev;
    A.o.exit_count = (uint32_t *)(T->d_xscr + (size_t)nb * 48 + 256);
    if (ctx->phase_prof) MPM_CU(cudaMemsetAsync(ctx->d_prof, 0, kProfSlots * sizeof(unsigned long long), cs));
    void *kargs[] = {&A};
    if (!T->cnn) {
        A.mode = STEP_WHOLE;
        MPM_CU(cudaLaunchCooperativeKernel((const void *)P.stepfn, dim3(nb), dim3(P.nt), kargs, P.smem, cs));
        ctx->launches += 1;
    } else {
        A.mode = STEP_EXTRACT;
        MPM_CU(cudaLaunchCooperativeKernel((const void *)P.stepfn, dim3(nb), dim3(P.nt), kargs, P.smem, cs));
        mpm_status r = mpm_cnn_enqueue_guess(ctx, T->cnn, sub, lat, prm, &d_dyn->g, cs);
        if (r != MPM_OK) return r;
        A.mode = STEP_SOLVE;
        MPM_CU(cudaLaunchCooperativeKernel((const void *)P.stepfn, dim3(nb), dim3(P.nt), kargs, P.smem, cs));
        ctx->launches += 2;
    }
    if (ctx->phase_prof)
        MPM_CU(cudaMemcpyAsync(ctx->h_prof, ctx->d_prof, kProfSlots * sizeof(unsigned long long), cudaMemcpyDeviceToHost, cs));
    return MPM_OK;
}

// Grid of the persistent solve for S items of NE elements (the sizing of
// plan_solve: about two elements per thread and item, at least one CTA per
// item, at most the co-resident maximum).
static int step_grid(int64_t NE, int S, int gmax, int nt)
{
    const double want = (double)S * (double)(NE + 1) / (nt * 2.0);
    int G = (int)std::min<double>(gmax, std::max(1.0, want));
    return std::max(G, std::min(S, gmax));
}

mpm_status mpm_step_enqueue_impl(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_lattice *lat, const mpm_params *prm,
                                 int32_t margin, const int32_t tile[3], const mpm_opts *opt, cudaStream_t st)
{
    if (!sub || !prm) return mpm_fail(ctx, MPM_ERR_ARG, "step: null argument");
    mpm_status r = mpm_params_check(ctx, prm);
    if (r != MPM_OK) return r;
    r = mpm_lattice_check(ctx, lat, prm->nspecies);
    if (r != MPM_OK) return r;
    if (margin < 0) return mpm_fail(ctx, MPM_ERR_ARG, "step: negative margin");
    r = check_opts(ctx, opt);
    if (r != MPM_OK) return r;
    if (opt->x0_given) return mpm_fail(ctx, MPM_ERR_ARG, "step: x0_given is not supported (the step starts from c^n)");
    int32_t lt[3];
    r = mpm_tile_lt(ctx, tile, lt);
    if (r != MPM_OK) return r;
    if (!sub->step) sub->step = new StepGraph();
    StepGraph *T = (StepGraph *)sub->step;
    if (T->cnn) {
        r = mpm_cnn_check(ctx, T->cnn, lat, prm);
        if (r != MPM_OK) return r;
    }
    const int S = prm->nspecies;
    // buffers for the whole lattice (pointers move only when they grow)
    const void *old_geo = sub->geo, *old_elem = sub->elem;
    r = mpm_step_buffers(ctx, sub, lat, S, lt);
    if (r != MPM_OK) return r;
    if (sub->geo != old_geo || sub->elem != old_elem) T->valid = false;
    // grid: from the previous step's element count, kept while within 25%;
    // at most the co-resident CTAs of the whole-step kernel
    const int maxm = opt->restart <= 8 ? 8 : (opt->restart <= 16 ? 16 : 32);
    const Variant var = pick(opt->precision, maxm, ctx->solver_variant);
    if (T->gmax_key[0] != opt->precision || T->gmax_key[1] != maxm || T->gmax_key[2] != ctx->solver_variant) {
        T->gmax = variant_max_blocks(ctx, var, true);   // occupancy query: once per variant
        T->gmax_key[0] = opt->precision;
        T->gmax_key[1] = maxm;
        T->gmax_key[2] = ctx->solver_variant;
    }
    const int gmax = T->gmax;
    if (gmax < 1) return mpm_fail(ctx, MPM_ERR_CUDA, "step: occupancy query failed");
    const int64_t NE_est = T->last_NE >= 0 ? T->last_NE : sub->NE_cap;
    int G = opt->nblocks > 0 ? std::min(opt->nblocks, gmax) : step_grid(NE_est, S, gmax, var.nt);
    if (opt->nblocks <= 0 && T->G > 0 && T->G <= gmax && G >= T->G * 4 / 5 && G <= T->G * 5 / 4) G = T->G;
    if (!T->d_scr) {
        MPM_CU(cudaMalloc(&T->d_scr, 1024));
        MPM_CU(cudaMemset(T->d_scr, 0, 1024));
        MPM_CU(cudaMalloc(&T->d_bar, (size_t)ctx->num_sms * 4 * 32 * sizeof(uint32_t)));
        T->valid = false;
    }
    auto make_key = [&](std::vector<unsigned char> &key) {
        key.clear();
        auto put = [&](const void *p, size_t n) {
            const unsigned char *c = (const unsigned char *)p;
            key.insert(key.end(), c, c + n);
        };
        put(lat, sizeof(mpm_lattice));
        put(prm, sizeof(mpm_params));
        put(opt, sizeof(mpm_opts));
        put(&margin, sizeof(margin));
        put(lt, 3 * sizeof(int32_t));
        put(&G, sizeof(G));
        put(&ctx->solver_variant, sizeof(int32_t));
        put(&ctx->timeout_ns, sizeof(uint64_t));
        put(&ctx->skip_block, sizeof(int32_t));
        put(&sub->geo, sizeof(void *));
        put(&sub->elem, sizeof(void *));
        put(&sub->krylov, sizeof(void *));
        put(&T->cnn, sizeof(void *));
    };
    std::vector<unsigned char> key;
    make_key(key);
    const bool use_graph = !ctx->phase_prof;
    if (!(T->valid && T->key == key) || !use_graph) {
        if (T->exec) cudaGraphExecDestroy(T->exec);
        T->exec = nullptr;
        T->valid = false;
        // solver plan: stride from the capacity, grid G, element count from the device
        PlanOverride ov;
        ov.NE_cap = sub->NE_cap;
        ov.NE_est = NE_est;
        ov.NEp = &((const StepDyn *)(T->d_scr + kScrDyn))->NE;
        ov.G = G;
        mpm_set_assembled_scalars(sub, prm);   // read into the solver's descriptors
        T->plan = SolvePlan();
        r = plan_solve(ctx, &sub, 1, opt, false, st, T->plan, &ov);
        if (r != MPM_OK) return r;
        make_key(key);   // the Krylov basis may have grown
        r = mpm_grow(ctx, (void **)&T->d_args, &T->args_cap, T->plan.args_need, "step solver descriptors");
        if (r != MPM_OK) return r;
        r = mpm_grow(ctx, (void **)&T->d_partials, &T->partials_cap, 2 * (size_t)T->plan.G * kKMax * sizeof(double),
                     "step reduction partials");
        if (r != MPM_OK) return r;
        T->plan.sa.partials = T->d_partials;
        r = mpm_grow(ctx, (void **)&T->d_rates, &T->rates_cap, 2 * (size_t)prm->nspecies * prm->ncell * sizeof(double),
                     "step rate tables");
        if (r != MPM_OK) return r;
        r = mpm_grow(ctx, (void **)&T->d_xscr, &T->xscr_cap, xscr_bytes(T->plan.G), "step extraction scratch");
        if (r != MPM_OK) return r;
        if (T->plan.nteam > ctx->num_sms * 4) return mpm_fail(ctx, MPM_ERR_ARG, "step: too many teams");
        const size_t hneed = kOutRep + sizeof(SysReport) * T->plan.nitem;
        if (T->hout_cap < hneed) {
            if (T->h_out) cudaFreeHost(T->h_out);
            T->h_out = T->h_out_dev = nullptr;
            T->hout_cap = 0;
            MPM_CU(cudaHostAlloc((void **)&T->h_out, hneed, cudaHostAllocMapped));
            T->hout_cap = hneed;
            MPM_CU(cudaHostGetDevicePointer((void **)&T->h_out_dev, T->h_out, 0));
        }
        if (ctx->phase_prof && !ctx->d_prof) MPM_CU(cudaMalloc(&ctx->d_prof, kProfSlots * sizeof(unsigned long long)));
        r = ensure_stage(ctx, T->plan.args_need + 4096);
        if (r != MPM_OK) return r;
        fill_descriptors(T->plan, (char *)ctx->h_stage);
        MPM_CU(cudaMemcpyAsync(T->d_args, ctx->h_stage, T->plan.o_rep, cudaMemcpyHostToDevice, st));
        // between-step state at its initial values: activity bytes, grid barrier
        // and exit counters, team barrier counters and the abort flag at zero
        {
            const int64_t ntl = (((int64_t)lat->dims[0] + (1 << lt[0]) - 1) >> lt[0]) *
                                (((int64_t)lat->dims[1] + (1 << lt[1]) - 1) >> lt[1]) *
                                (((int64_t)lat->dims[2] + (1 << lt[2]) - 1) >> lt[2]);
            MPM_CU(cudaMemsetAsync(sub->active, 0, (size_t)ntl, st));
            MPM_CU(cudaMemsetAsync(T->d_xscr, 0, xscr_bytes(T->plan.G), st));
            MPM_CU(cudaMemsetAsync(T->d_scr, 0, 1024, st));
            MPM_CU(cudaMemsetAsync(T->d_bar, 0, (size_t)ctx->num_sms * 4 * 32 * sizeof(uint32_t), st));
        }
        MPM_CU(cudaStreamSynchronize(st));   // descriptors and slots in place before any capture
        T->G = G;
        if (use_graph && !T->graph_failed) {
            if (!ctx->cap_stream) MPM_CU(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
            cudaStream_t cs = ctx->cap_stream;
            cudaGraph_t g = nullptr;
            const int64_t launches0 = ctx->launches;
            bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                ok = enqueue_step(ctx, T, sub, lat, prm, margin, opt, cs) == MPM_OK;
                const cudaError_t ec = cudaStreamEndCapture(cs, &g);
                ok = ok && ec == cudaSuccess && g != nullptr;
            }
            T->graph_launches = ctx->launches - launches0;
            ctx->launches = launches0;
            if (ok) ok = cudaGraphInstantiate(&T->exec, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            if (ok) {
                T->valid = true;
                T->key = key;
            } else {
                T->exec = nullptr;
                T->graph_failed = true;   // stay eager on this device or driver
            }
        }
    }
    if (T->valid) {
        MPM_CU(cudaGraphLaunch(T->exec, st));
        ctx->launches += T->graph_launches;
    } else {
        r = enqueue_step(ctx, T, sub, lat, prm, margin, opt, st);
        if (r != MPM_OK) return r;
    }
    T->pending = true;
    T->margin = margin;
    for (int d = 0; d < 3; ++d) {
        T->lt[d] = lt[d];
        T->ldims[d] = lat->dims[d];
    }
    return MPM_OK;
}

// Waits for the subgrid's enqueued steps and reports the last one.
mpm_status mpm_step_wait_impl(mpm_ctx *ctx, mpm_subgrid *sub, mpm_report *rep, mpm_box *out_box, cudaStream_t st)
{
    if (!sub) return mpm_fail(ctx, MPM_ERR_ARG, "step_wait: null subgrid");
    StepGraph *T = (StepGraph *)sub->step;
    if (!T || !T->pending) return mpm_fail(ctx, MPM_ERR_ARG, "step_wait: no step was enqueued on this subgrid");
    MPM_CU(cudaStreamSynchronize(st));
    T->pending = false;
    const int32_t margin = T->margin;
    const int32_t *lt = T->lt;
    mpm_status r;
    const volatile int32_t *hb = (const volatile int32_t *)(T->h_out + kOutBox);
    const volatile int64_t *hc = (const volatile int64_t *)(T->h_out + kOutCount);
    ctx->step_nfull = *(const volatile uint32_t *)(T->h_out + kOutNFull);
    if (*(const volatile int32_t *)(T->h_out + kOutAbort) != 0) {
        // a bounded wait expired: nothing was scattered; set the between-step state up again
        T->valid = false;
        sub->extracted = false;
        sub->assembled = false;
        return mpm_fail(ctx, MPM_ERR_TIMEOUT, "step: a bounded inter-CTA wait expired");
    }
    const bool timed_out = false;
    // the solve's own time: the longest work item (the kernel is one launch per step)
    float ms = 0.f;
    for (int it = 0; it < T->plan.nitem; ++it)
        ms = std::max(ms, (float)(((const SysReport *)(T->h_out + kOutRep))[it].t_ns * 1e-6));
    sub->gen += 1;
    if (hb[3] < 0) {   // no tumour voxel: nothing was solved or written
        sub->extracted = false;
        sub->assembled = false;
        sub->NE = 0;
        T->last_NE = 0;
        return mpm_fail(ctx, MPM_ERR_EMPTY, "step: no tumour voxel (cell_id > 0)");
    }
    mpm_box box;
    for (int d = 0; d < 3; ++d) {
        box.lo[d] = hb[d] - margin < 0 ? 0 : hb[d] - margin;
        const int64_t h = (int64_t)hb[3 + d] + margin + 1;
        box.hi[d] = h > T->ldims[d] ? T->ldims[d] : (int32_t)h;
        sub->lo[d] = box.lo[d];
        sub->hi[d] = box.hi[d];
        sub->n[d] = box.hi[d] - box.lo[d];
        sub->nt[d] = (sub->n[d] + (1 << lt[d]) - 1) >> lt[d];
    }
    sub->ntiles = sub->nt[0] * sub->nt[1] * sub->nt[2];
    sub->mask_voxels = hc[0];
    sub->nact = (int32_t)hc[1];
    sub->NE = (int64_t)sub->nact << (lt[0] + lt[1] + lt[2]);
    sub->extracted = true;
    sub->assembled = true;
    T->last_NE = sub->NE;
    if (out_box) *out_box = box;
    r = finish_solve(ctx, T->plan, &sub, (const SysReport *)(T->h_out + kOutRep), timed_out, ms, rep, nullptr, st);
    sub->x_fresh = false;
    return r;
}

// Attach (or detach, cnn = null) the network whose prediction starts the
// solves of this subgrid's device-resident steps.
mpm_status mpm_step_set_network_impl(mpm_ctx *ctx, mpm_subgrid *sub, mpm_cnn *cnn)
{
    if (!sub) return mpm_fail(ctx, MPM_ERR_ARG, "step_set_network: null subgrid");
    if (!sub->step) sub->step = new StepGraph();
    StepGraph *T = (StepGraph *)sub->step;
    if (T->pending) return mpm_fail(ctx, MPM_ERR_ARG, "step_set_network: a step is pending (call mpm_step_wait)");
    T->cnn = cnn;
    return MPM_OK;
}

mpm_status mpm_step_impl(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_lattice *lat, const mpm_params *prm, int32_t margin,
                         const int32_t tile[3], const mpm_opts *opt, mpm_report *rep, mpm_box *out_box, cudaStream_t st)
{
    mpm_status r = mpm_step_enqueue_impl(ctx, sub, lat, prm, margin, tile, opt, st);
    if (r != MPM_OK) return r;
    return mpm_step_wait_impl(ctx, sub, rep, out_box, st);
}
