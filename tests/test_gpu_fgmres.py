"""Row a13 on the GPU: the network as the right preconditioner of flexible
GMRES (mpm_cnn_precond, mpm_solve_fgmres_cnn), against the oracle's network
preconditioner, its flexible GMRES and the dense solve."""
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


def _setup(M, ctx, seed, dims, net_params, s_out, dfac=False):
    wl = W.random_case(seed, dims, nspecies=3, dfac=dfac)
    lat = M.DeviceLattice(wl.lattice)
    prm = M.DeviceParams(wl.params)
    sub = ctx.subgrid_create()
    box = sub.mpm_box_extract(lat, 3, wl.margin)
    sub.mpm_assemble_coeffs(prm)
    cnn = M.CNN(ctx, wl.lattice.dims, 1, net_params, s_out=s_out)
    return wl, lat, prm, sub, box, cnn


def _zero_output_params(M, seed):
    p = M.cnn_init_params(seed, last_scale=0.0).copy()
    p[-3:] = 0.0
    return p


@pytest.mark.parametrize("s", [0, 1, 2])
def test_preconditioner_matches_oracle(M, s):
    import torch
    ctx = M.Context()
    params = M.cnn_init_params(3, last_scale=1.0)
    wl, lat, prm, sub, box, cnn = _setup(M, ctx, 30 + s, (14, 11, 9), params, 0.3)
    mb = oracle.box_view(wl.lattice.mask, box)
    cb = oracle.box_view(wl.lattice.cell_id, box)
    rng = np.random.default_rng(40 + s)
    v = np.where(mb > 0, rng.normal(size=mb.shape), 0.0)
    z = cnn.precond(sub, lat, prm, s, torch.from_numpy(v).cuda()).cpu().numpy()
    zo = oracle.cnn_precond(v, s, cb, mb, wl.params, params.astype(np.float64), 0.3)
    vm = np.where(mb > 0, v.astype(np.float32).astype(np.float64), 0.0)
    scale = np.max(np.abs(zo - vm))
    assert scale > 0.0
    # the network's part z - v at the forward tolerance of test_gpu_cnn (1e-2
    # of its largest magnitude element by element, bf16 rounding flips), plus
    # FP32 rounding of v / m
    assert np.max(np.abs(z - zo)) <= 1e-2 * scale + 1e-6 * np.max(np.abs(v))
    assert np.all(z[mb == 0] == 0.0)


def test_zero_output_network_is_gmres(M):
    """A network with a zero output layer reproduces its input: FGMRES is
    GMRES (the oracle's fgmres, modified Gram-Schmidt against the device's
    two classical passes), same solution; no fallback."""
    ctx = M.Context()
    wl, lat, prm, sub, box, cnn = _setup(M, ctx, 33, (16, 12, 10), _zero_output_params(M, 4), 0.3)
    opts = M.make_opts(rtol=1e-11, restart=8, maxit=500)
    rep = cnn.solve_fgmres(sub, lat, prm, opts, scatter_to=lat)
    assert rep["status_code"] == M.OK and rep["fallback"] == [0, 0, 0]
    mb = oracle.box_view(wl.lattice.mask, box)
    cb = oracle.box_view(wl.lattice.cell_id, box)
    got = lat.fields_numpy()
    for s in range(3):
        A, b = oracle.assemble(mb, cb, oracle.box_view(wl.lattice.fields[s], box), wl.params, s)
        xs = oracle.dense_solve(A, b).reshape(mb.shape)
        tol = 1e-11 * np.linalg.norm(b[mb > 0])
        xo, io = oracle.fgmres(A, b, oracle.box_view(wl.lattice.fields[s], box),
                               lambda u: np.where(mb.reshape(-1) > 0, u.astype(np.float32).astype(np.float64), 0.0),
                               8, tol, 500)
        assert abs(rep["iters"][s] - io["iters"]) <= 1, (s, rep["iters"][s], io["iters"])
        assert rep["res"][s] <= tol
        g = oracle.box_view(got[s], box)
        assert np.linalg.norm((g - xs)[mb > 0]) <= rep["res"][s] + 1e-12


def _mask_round32(mb):
    return lambda u: np.where(mb.reshape(-1) > 0, u.astype(np.float32).astype(np.float64), 0.0)


@pytest.mark.parametrize("dfac", [False, True])
def test_mixed_zero_output_network_matches_refined_oracle(M, dfac):
    """FP32 cycles inside FP64 refinement (precision 1) against the oracle's
    fgmres_refined with the same map (FP32 rounding of v on the mask): the
    cycle count is equal, the Arnoldi steps within one per cycle (FP32
    rounding order decides where an estimate crosses its threshold), the true
    residual meets 1e-10 (below FP32's precision) and the solution is the
    dense solve's within the residual bound."""
    ctx = M.Context()
    wl, lat, prm, sub, box, cnn = _setup(M, ctx, 36, (17, 13, 11), _zero_output_params(M, 4), 0.3, dfac)
    opts = M.make_opts(rtol=1e-10, restart=8, maxit=800, precision=1, inner_rtol=1e-4)
    rep = cnn.solve_fgmres(sub, lat, prm, opts, scatter_to=lat)
    assert rep["status_code"] == M.OK and rep["fallback"] == [0, 0, 0]
    mb = oracle.box_view(wl.lattice.mask, box)
    cb = oracle.box_view(wl.lattice.cell_id, box)
    db = None if wl.lattice.dfac is None else oracle.box_view(wl.lattice.dfac, box)
    got = lat.fields_numpy()
    for s in range(3):
        c0 = oracle.box_view(wl.lattice.fields[s], box)
        A, b = oracle.assemble(mb, cb, c0, wl.params, s, 0, db)
        tol = 1e-10 * np.linalg.norm(b.reshape(-1)[mb.reshape(-1) > 0])
        xo, io = oracle.fgmres_refined(A, b, c0, _mask_round32(mb), 8, tol, 800, inner=np.float32, inner_rtol=1e-4)
        assert io["status"] == oracle.OK and not io["fallback"]
        assert rep["cycles"][s] == io["cycles"], (s, rep["cycles"][s], io["cycles"])
        assert abs(rep["iters"][s] - io["iters"]) <= rep["cycles"][s], (s, rep["iters"][s], io["iters"])
        g = oracle.box_view(got[s], box)
        r = b.reshape(-1) - A.matvec(g.reshape(-1))
        assert np.linalg.norm(r) <= tol
        assert abs(np.linalg.norm(r) - rep["res"][s]) <= 1e-6 * tol
        xs = oracle.dense_solve(A, b).reshape(mb.shape)
        assert np.linalg.norm((g - xs)[mb > 0]) <= rep["res"][s] + 1e-12


def _huge_params(M):
    return (M.cnn_init_params(3, last_scale=1.0) * np.float32(1e30)).astype(np.float32)


@pytest.mark.parametrize("precision", [0, 1])
def test_nonfinite_network_falls_back_to_plain_gmres(M, precision):
    """A host-made bad network (weights x 1e30: its output overflows) fails
    the first cycle of every species; the solve drops it, goes on as plain
    GMRES and ends MPM_OK with the fallback flag set.  Against the oracle's
    fgmres_refined with a non-finite preconditioner: same cycles, the Arnoldi
    steps within one per cycle, the solution within the residual bound."""
    ctx = M.Context()
    wl, lat, prm, sub, box, cnn = _setup(M, ctx, 37, (15, 12, 10), _huge_params(M), 0.3)
    opts = M.make_opts(rtol=1e-10, restart=8, maxit=800, precision=precision, inner_rtol=1e-4)
    rep = cnn.solve_fgmres(sub, lat, prm, opts, scatter_to=lat)
    assert rep["status_code"] == M.OK
    assert rep["fallback"] == [1, 1, 1]
    mb = oracle.box_view(wl.lattice.mask, box)
    cb = oracle.box_view(wl.lattice.cell_id, box)
    got = lat.fields_numpy()
    inner = np.float32 if precision else np.float64
    for s in range(3):
        c0 = oracle.box_view(wl.lattice.fields[s], box)
        A, b = oracle.assemble(mb, cb, c0, wl.params, s)
        tol = 1e-10 * np.linalg.norm(b.reshape(-1)[mb.reshape(-1) > 0])
        xo, io = oracle.fgmres_refined(A, b, c0, lambda v: np.full_like(v, np.nan), 8, tol, 800, inner=inner,
                                       inner_rtol=1e-4)
        assert io["status"] == oracle.OK and io["fallback"]
        assert rep["cycles"][s] == io["cycles"], (s, rep["cycles"][s], io["cycles"])
        assert abs(rep["iters"][s] - io["iters"]) <= rep["cycles"][s], (s, rep["iters"][s], io["iters"])
        g = oracle.box_view(got[s], box)
        assert np.linalg.norm((b.reshape(-1) - A.matvec(g.reshape(-1)))) <= tol
        xs = oracle.dense_solve(A, b).reshape(mb.shape)
        assert np.linalg.norm((g - xs)[mb > 0]) <= rep["res"][s] + 1e-12
    # the network is used again by the next solve (the plan restores it)
    rep2 = cnn.solve_fgmres(sub, lat, prm, opts)
    assert rep2["fallback"] == [1, 1, 1]


@pytest.mark.parametrize("precision", [0, 1])
def test_random_network_fgmres_matches_refined_oracle(M, precision):
    """A random network as the preconditioner, FP64 and FP32-in-FP64: the
    device solve and the oracle's fgmres_refined with the oracle's network
    preconditioner take the same cycles (Arnoldi steps within one per cycle:
    bf16 rounding flips move the directions slightly) and meet the same
    tolerance; no fallback fires."""
    ctx = M.Context()
    params = M.cnn_init_params(5, last_scale=0.3)
    wl, lat, prm, sub, box, cnn = _setup(M, ctx, 38, (14, 12, 10), params, 0.2)
    opts = M.make_opts(rtol=1e-9, restart=8, maxit=800, precision=precision, inner_rtol=1e-4)
    rep = cnn.solve_fgmres(sub, lat, prm, opts, scatter_to=lat)
    assert rep["status_code"] == M.OK and rep["fallback"] == [0, 0, 0]
    mb = oracle.box_view(wl.lattice.mask, box)
    cb = oracle.box_view(wl.lattice.cell_id, box)
    got = lat.fields_numpy()
    inner = np.float32 if precision else np.float64
    for s in range(3):
        c0 = oracle.box_view(wl.lattice.fields[s], box)
        A, b = oracle.assemble(mb, cb, c0, wl.params, s)
        tol = 1e-9 * np.linalg.norm(b.reshape(-1)[mb.reshape(-1) > 0])
        pc = lambda v, s=s: oracle.cnn_precond(v.reshape(mb.shape), s, cb, mb, wl.params,
                                               params.astype(np.float64), 0.2).reshape(-1)
        xo, io = oracle.fgmres_refined(A, b, c0, pc, 8, tol, 800, inner=inner, inner_rtol=1e-4)
        assert io["status"] == oracle.OK and not io["fallback"]
        assert abs(rep["cycles"][s] - io["cycles"]) <= 1, (s, rep["cycles"][s], io["cycles"])
        assert abs(rep["iters"][s] - io["iters"]) <= max(2, rep["cycles"][s]), (s, rep["iters"][s], io["iters"])
        g = oracle.box_view(got[s], box)
        assert np.linalg.norm((b.reshape(-1) - A.matvec(g.reshape(-1)))) <= tol


@pytest.mark.parametrize("dfac", [False, True])
def test_network_preconditioned_fgmres_solves_the_step(M, dfac):
    """A random network (a poor but nonlinear preconditioner): every species
    reaches the true-residual tolerance and the dense solution within the
    residual bound; voxels off the mask keep c^n."""
    ctx = M.Context()
    params = M.cnn_init_params(5, last_scale=0.3)
    wl, lat, prm, sub, box, cnn = _setup(M, ctx, 34, (15, 13, 11), params, 0.2, dfac)
    opts = M.make_opts(rtol=1e-10, restart=8, maxit=800)
    rep = cnn.solve_fgmres(sub, lat, prm, opts, scatter_to=lat)
    assert rep["status_code"] == M.OK
    mb = oracle.box_view(wl.lattice.mask, box)
    cb = oracle.box_view(wl.lattice.cell_id, box)
    db = None if wl.lattice.dfac is None else oracle.box_view(wl.lattice.dfac, box)
    got = lat.fields_numpy()
    for s in range(3):
        A, b = oracle.assemble(mb, cb, oracle.box_view(wl.lattice.fields[s], box), wl.params, s, 0, db)
        xs = oracle.dense_solve(A, b).reshape(mb.shape)
        assert rep["res"][s] <= 1e-10 * rep["bnorm"][s]
        g = oracle.box_view(got[s], box)
        assert np.linalg.norm((g - xs)[mb > 0]) <= rep["res"][s] + 1e-12
        assert np.array_equal(g[mb == 0], oracle.box_view(wl.lattice.fields[s], box)[mb == 0])


def test_guess_then_fgmres(M):
    ctx = M.Context()
    params = M.cnn_init_params(6, last_scale=0.2)
    wl, lat, prm, sub, box, cnn = _setup(M, ctx, 35, (12, 12, 12), params, 0.05)
    cnn.guess(sub, lat, prm)
    rep = cnn.solve_fgmres(sub, lat, prm, M.make_opts(rtol=1e-9, restart=8, maxit=800, x0_given=1))
    assert rep["status_code"] == M.OK and all(r <= 1e-9 * b for r, b in zip(rep["res"], rep["bnorm"]))


def test_mixed_fgmres_growth512_meets_tolerance(M):
    """The 512x384x384 growing tumour at its last (largest) step: the box
    extracted, FP32-in-FP64 flexible GMRES preconditioned by an untrained
    network (a poor but finite map), then a network that overflows (the
    fallback); the true residual recomputed by the oracle meets 1e-6 both
    times."""
    import torch
    wl, extra = W.growth512()
    ctx = M.Context()
    W.grow(wl, wl.steps - 1, extra)
    lat = M.DeviceLattice(wl.lattice)
    prm = M.DeviceParams(wl.params)
    sub = ctx.subgrid_create()
    box = sub.mpm_box_extract(lat, 3, wl.margin)
    sub.mpm_assemble_coeffs(prm)
    mb = oracle.box_view(wl.lattice.mask, box)
    cb = oracle.box_view(wl.lattice.cell_id, box)
    systems = [oracle.assemble(mb, cb, oracle.box_view(wl.lattice.fields[s], box), wl.params, s) for s in range(3)]
    opts = M.make_opts(rtol=1e-6, restart=8, maxit=500, precision=1, inner_rtol=1e-6)
    for params, fb in ((M.cnn_init_params(4, last_scale=0.1), 0), (_huge_params(M), 1)):
        cnn = M.CNN(ctx, wl.lattice.dims, 1, params, s_out=0.01)
        rep = cnn.solve_fgmres(sub, lat, prm, opts)
        assert rep["status_code"] == M.OK and rep["fallback"] == [fb] * 3, rep
        for s in range(3):
            x = sub.mpm_subgrid_export(M.EXPORT_X, s).cpu().numpy().reshape(mb.shape)
            A, b = systems[s]
            r = b.reshape(-1) - A.matvec(np.where(mb > 0, x, oracle.box_view(wl.lattice.fields[s], box)).reshape(-1))
            assert np.linalg.norm(r) <= 1e-6 * np.linalg.norm(b.reshape(-1)[mb.reshape(-1) > 0]), (fb, s)
        del cnn
        torch.cuda.empty_cache()
