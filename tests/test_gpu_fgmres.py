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
    GMRES (the oracle's, same modified Gram-Schmidt), same solution."""
    ctx = M.Context()
    wl, lat, prm, sub, box, cnn = _setup(M, ctx, 33, (16, 12, 10), _zero_output_params(M, 4), 0.3)
    opts = M.make_opts(rtol=1e-11, restart=8, maxit=500)
    rep = cnn.solve_fgmres(sub, lat, prm, opts, scatter_to=lat)
    assert rep["status_code"] == M.OK
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
