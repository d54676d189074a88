"""Batched solves: many uneven pleural-shell patches x 3 species in one
persistent launch (mpm_solve_batch) and the graph-captured fixed-box step
(mpm_batch_step), against single-system solves and the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_2505_03067_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_03067_gb300 import build, mpm
    build.build()
    return mpm


@pytest.fixture(scope="module")
def patches():
    ps = W.patches()
    # a spread of sizes: the 6 smallest, 2 middle and the largest patch
    order = sorted(range(len(ps)), key=lambda i: ps[i].lattice.cell_id.size)
    pick = order[:6] + order[31:33] + order[-1:]
    return [ps[i] for i in pick]


def _oracle_steps(wl, nsteps):
    ref = wl.lattice.copy()
    for _ in range(nsteps):
        rep = oracle.step(ref, wl.params, wl.margin, rtol=0.0, atol=1e-12)
        assert rep["status"] == oracle.OK
    return ref


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_step_graph_matches_oracle(M, patches, precision):
    ctx = M.Context()
    lats = [M.DeviceLattice(p.lattice) for p in patches]
    prms = [M.DeviceParams(p.params) for p in patches]
    bs = M.BatchStepper(ctx, lats, prms, [p.margin for p in patches])
    if precision == 0:
        opts = M.make_opts(rtol=0.0, atol=1e-12, restart=8, maxit=500)
    else:
        opts = M.make_opts(rtol=1e-9, restart=8, maxit=500, precision=1, inner_rtol=1e-6)
    for step in range(3):
        st, reps = bs.step(opts)
        assert st == M.OK
        if step >= 1:
            assert bs.graph_active()
    for p, lat, rep in zip(patches, lats, reps):
        ref = _oracle_steps(p, 3)
        got = lat.fields_numpy()
        m = p.lattice.mask > 0
        for s in range(3):
            if precision == 0:
                assert np.max(np.abs(got[s] - ref.fields[s])) <= 1e-10
            else:
                assert np.linalg.norm(got[s][m] - ref.fields[s][m]) <= 3e-9 * np.linalg.norm(ref.fields[s][m])


def test_solve_batch_matches_single_solves(M, patches):
    ctx = M.Context()
    opts = M.make_opts(rtol=0.0, atol=1e-12, restart=8, maxit=500)
    lats_b = [M.DeviceLattice(p.lattice) for p in patches]
    subs = []
    for p, lat in zip(patches, lats_b):
        sub = ctx.subgrid_create()
        sub.mpm_box_extract(lat, 3, p.margin)
        sub.mpm_assemble_coeffs(M.DeviceParams(p.params))
        subs.append(sub)
    st, reps = M.mpm_solve_batch(ctx, subs, opts, scatter_to=lats_b)
    assert st == M.OK
    for p, lat in zip(patches, lats_b):
        lat1 = M.DeviceLattice(p.lattice)
        M.StepSolver(ctx, lat1, M.DeviceParams(p.params), p.margin).step(opts)
        assert np.max(np.abs(lat.fields_numpy() - lat1.fields_numpy())) <= 1e-10


def test_refresh_equals_re_extract(M):
    wl = W.random_case(31, (24, 20, 18), nspecies=3)
    ctx = M.Context()
    lat = M.DeviceLattice(wl.lattice)
    sub = ctx.subgrid_create()
    sub.mpm_box_extract(lat, 3, wl.margin)
    lat.fields.mul_(0.5)
    sub.mpm_subgrid_refresh(lat)
    x_ref = [sub.mpm_subgrid_export(M.EXPORT_X, s).cpu().numpy() for s in range(3)]
    sub2 = ctx.subgrid_create()
    sub2.mpm_box_extract(lat, 3, wl.margin)
    for s in range(3):
        assert np.array_equal(x_ref[s], sub2.mpm_subgrid_export(M.EXPORT_X, s).cpu().numpy())


@pytest.mark.parametrize("dfac,bc_box", [(False, 0), (True, 0), (True, 1)])
def test_batched_preparation_equals_per_system_assembly(M, dfac, bc_box):
    """The one-launch refresh + assembly of every system of a batched step gives,
    element for element, the rows, c^n and flags of the per-system refresh and
    assembly (uniform and harmonic-mean diffusivity, both box conditions)."""
    shapes = [((9, 7, 5), 3), ((21, 13, 11), 2), ((33, 17, 25), 3), ((5, 5, 5), 1), ((40, 9, 12), 4)]
    wls = [W.random_case(40 + i, dims, nspecies=ns, dfac=dfac) for i, (dims, ns) in enumerate(shapes)]
    ctx = M.Context()
    lats = [M.DeviceLattice(w.lattice) for w in wls]
    prms = [M.DeviceParams(w.params, bc_box=bc_box) for w in wls]
    bs = M.BatchStepper(ctx, lats, prms, [w.margin for w in wls], tile=(4, 4, 2))
    st, reps = bs.step(M.make_opts(rtol=1e-10, restart=8, maxit=500))
    assert st == M.OK
    for w, sub_b in zip(wls, bs.subs):
        lat1 = M.DeviceLattice(w.lattice)
        sub = ctx.subgrid_create()
        sub.mpm_box_extract(lat1, w.params.nspecies, w.margin, (4, 4, 2))
        sub.mpm_assemble_coeffs(M.DeviceParams(w.params, bc_box=bc_box))
        for what in (M.EXPORT_FLAGS, M.EXPORT_CELL):
            assert np.array_equal(sub_b.mpm_subgrid_export(what, 0).cpu().numpy(),
                                  sub.mpm_subgrid_export(what, 0).cpu().numpy())
        for s in range(w.params.nspecies):
            for what in (M.EXPORT_RHS, M.EXPORT_DIAG):
                assert np.array_equal(sub_b.mpm_subgrid_export(what, s).cpu().numpy(),
                                      sub.mpm_subgrid_export(what, s).cpu().numpy())


def test_batch_step_flags_only_the_system_with_a_bad_cell_id(M):
    ctx = M.Context()
    ps = [W.random_case(50 + i, (16, 12, 10), nspecies=2) for i in range(3)]
    bad = ps[1].lattice.cell_id.copy()
    idx = np.flatnonzero((ps[1].lattice.mask > 0).ravel() & (bad.ravel() > 0))[0]
    bad.reshape(-1)[idx] = ps[1].params.ncell + 3
    ps[1].lattice.cell_id = bad
    lats = [M.DeviceLattice(p.lattice) for p in ps]
    prms = [M.DeviceParams(p.params) for p in ps]
    bs = M.BatchStepper(ctx, lats, prms, [p.margin for p in ps])
    st, reps = bs.step(M.make_opts(rtol=1e-10, restart=8, maxit=500), allow=(M.ERR_NOCONV, M.ERR_ARG))
    assert st == M.ERR_ARG
    assert [set(r["status"]) for r in reps] == [{M.OK}, {M.ERR_ARG}, {M.OK}]


def test_team_model_replanning_keeps_results_within_the_residual_bound(M, tmp_path):
    """NEXT-3: the team planner's measured model (mpm_tune_teams) re-plans the
    64-patch batch; every plan's solution meets the tolerance, and two plans'
    solutions differ by no more than the sum of their residual bounds
    (||x - x*|| <= ||r|| since A's eigenvalues are >= 1).  The kept round's f
    is the smallest measured, a cache hit restores the same model, and the
    captured batch step plans with it."""
    ps = W.patches()
    ctx = M.Context()
    opts = M.make_opts(rtol=1e-9, restart=8, maxit=800, precision=1, inner_rtol=1e-6)
    lats = [M.DeviceLattice(p.lattice) for p in ps]
    subs = []
    for p, lat in zip(ps, lats):
        sub = ctx.subgrid_create()
        sub.mpm_box_extract(lat, 3, p.margin)
        sub.mpm_assemble_coeffs(M.DeviceParams(p.params))
        subs.append(sub)
    st, reps0 = M.mpm_solve_batch(ctx, subs, opts)
    assert st == M.OK
    x0 = [[sub.mpm_subgrid_export(M.EXPORT_X, s).cpu().numpy() for s in range(3)] for sub in subs]
    cache = str(tmp_path / "tune.txt")
    tt = ctx.mpm_tune_teams(subs, opts, 6, cache)
    assert len(tt["f"]) >= 3 and min(tt["fixed"]) >= 0.0
    st, reps1 = M.mpm_solve_batch(ctx, subs, opts)
    assert st == M.OK
    f_new = ctx.imbalance()
    for i, sub in enumerate(subs):
        for s in range(3):
            r0, r1 = reps0[i]["res"][s], reps1[i]["res"][s]
            assert r1 <= 1e-9 * reps1[i]["bnorm"][s]
            x1 = sub.mpm_subgrid_export(M.EXPORT_X, s).cpu().numpy()
            assert np.linalg.norm(x1 - x0[i][s]) <= r0 + r1 + 1e-14
    assert min(tt["f"]) <= tt["f"][0]
    # the cache restores the model without timing
    ctx2 = M.Context()
    tt2 = ctx2.mpm_tune_teams(subs, opts, 6, cache)
    assert tt2["fixed"] == tt["fixed"] and len(tt2["f"]) == 1
    print("team tuning f per round", tt["f"], "F1, F per round", tt["fixed_per_round"], "f of the next solve",
          f_new)
