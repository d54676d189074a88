"""The learned form of the device-resident step (mpm_step_set_network): the
extraction launch, the network's guess written into the iterate and the solve
launch in one CUDA graph.  Checked against the oracle: the guess inside the
step is the network's prediction, the solution is the oracle's (the guess
changes where GMRES starts, not what it converges to), the growing tumour on
its full 512x384x384 lattice meets 1e-6 on the FP32-in-FP64 path, and a
network whose prediction is not finite leaves c^n (the plain step, bit for
bit)."""
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


def _features_np(lat, params):
    f32 = np.float32
    cid = np.where((lat.cell_id >= 0) & (lat.cell_id < params.ncell), lat.cell_id, 0)
    S = params.nspecies
    shape = lat.cell_id.shape
    fld = [lat.fields[s].astype(f32) if s < S else np.zeros(shape, f32) for s in range(3)]
    X = np.zeros(shape + (9,))
    X[..., 0] = oracle.bf16(fld[0])
    X[..., 1] = oracle.bf16(fld[1])
    X[..., 2] = oracle.bf16(fld[2] * f32(20))
    X[..., 3] = cid == 0
    X[..., 4] = cid > 0
    if S > 0:
        X[..., 5] = oracle.bf16(params.k_cell[0][cid].astype(f32) * f32(10))
    if S > 1:
        X[..., 6] = oracle.bf16(params.k_cell[1][cid].astype(f32) * f32(10))
    if S > 2:
        X[..., 7] = oracle.bf16(params.q_cell[2][cid].astype(f32) * f32(10))
    X[..., 8] = lat.mask > 0
    X[lat.mask == 0] = 0.0
    return X


def _net(M, ctx, dims, seed=2, last_scale=0.3, s_out=0.05):
    params = M.cnn_init_params(seed, last_scale=last_scale)
    return M.CNN(ctx, dims, 1, params, s_out=s_out), params


def test_guess_inside_the_step_is_the_network_prediction(M):
    # rtol = 1 stops every species at its first residual: the iterate the step
    # scatters is the guess itself
    ctx = M.Context()
    wl = W.random_case(81, (37, 21, 18), nspecies=3)
    wl.margin = 2
    lat, prm = M.DeviceLattice(wl.lattice), M.DeviceParams(wl.params)
    cnn, params = _net(M, ctx, wl.lattice.dims)
    solver = M.StepSolver(ctx, lat, prm, wl.margin)
    solver.set_network(cnn)
    rep = solver.step(M.make_opts(rtol=1.0, restart=8, maxit=50))
    assert rep["status_code"] == M.OK and rep["iters"] == [0, 0, 0]
    box = rep["box"]
    assert box == oracle.bbox(wl.lattice.cell_id, wl.margin)
    bx = oracle.box_slices(box)
    X = _features_np(wl.lattice, wl.params)[bx]
    F = np.moveaxis(wl.lattice.fields.astype(np.float32).astype(np.float64), 0, -1)[bx]
    p_o, _ = oracle.cnn_forward(X, F, oracle.bf16(params.astype(np.float64)), 0.05)
    m = wl.lattice.mask[bx] > 0
    got = lat.fields_numpy()
    for s in range(3):
        z6g = (got[s][bx] - wl.lattice.fields[s][bx]) / 0.05
        z6o = (p_o[..., s] - F[..., s]) / 0.05
        assert np.max(np.abs(z6g[m] - z6o[m])) <= 1e-2 * np.max(np.abs(z6o[m])) + 1e-6, s
        assert np.array_equal(got[s][bx][~m], wl.lattice.fields[s][bx][~m])


@pytest.mark.parametrize("precision", [0, 1])
def test_learned_step_converges_to_the_oracle(M, precision):
    ctx = M.Context()
    wl = W.random_case(82, (29, 23, 17), nspecies=3)
    ref = wl.lattice.copy()
    oracle.step(ref, wl.params, wl.margin, rtol=0.0, atol=1e-13)
    res = {}
    for learned in (False, True):
        lat, prm = M.DeviceLattice(wl.lattice), M.DeviceParams(wl.params)
        solver = M.StepSolver(ctx, lat, prm, wl.margin)
        if learned:
            cnn, _ = _net(M, ctx, wl.lattice.dims)
            solver.set_network(cnn)
        opts = (M.make_opts(rtol=0.0, atol=1e-13, restart=16, maxit=500) if precision == 0 else
                M.make_opts(rtol=1e-6, restart=16, maxit=500, precision=1, inner_rtol=1e-5))
        rep = solver.step(opts)
        assert rep["status_code"] == M.OK
        res[learned] = (rep, lat.fields_numpy())
    rep, got = res[True]
    if precision == 0:
        assert np.max(np.abs(got - ref.fields)) <= 1e-10
    else:
        box = rep["box"]
        mb = oracle.box_view(wl.lattice.mask, box) > 0
        for s in range(3):
            g, r = oracle.box_view(got[s], box)[mb], oracle.box_view(ref.fields[s], box)[mb]
            assert np.linalg.norm(g - r) <= 1e-6 * np.linalg.norm(r)
    # the guess moved where GMRES started
    assert res[True][0]["iters"] != res[False][0]["iters"] or not np.array_equal(res[True][1], res[False][1])


def test_nonfinite_prediction_leaves_cn(M):
    ctx = M.Context()
    wl = W.random_case(83, (21, 19, 15), nspecies=3)
    outs = []
    for learned in (False, True):
        lat, prm = M.DeviceLattice(wl.lattice), M.DeviceParams(wl.params)
        solver = M.StepSolver(ctx, lat, prm, wl.margin)
        if learned:
            huge = (M.cnn_init_params(3, last_scale=1.0) * np.float32(1e30)).astype(np.float32)
            cnn = M.CNN(ctx, wl.lattice.dims, 1, huge, s_out=0.05)
            solver.set_network(cnn)
        rep = solver.step(M.make_opts(rtol=1e-10, restart=16, maxit=500))
        assert rep["status_code"] == M.OK
        outs.append((rep["iters"], lat.fields_numpy()))
    assert outs[0][0] == outs[1][0]
    assert np.array_equal(outs[0][1], outs[1][1])


def test_learned_mixed_growth512_steps_meet_tolerance(M):
    """The 512x384x384 growing tumour, FP32-in-FP64 solve from the network's
    guess (an untrained network: a poor guess GMRES must still correct), box
    re-extracted every step, true residual recomputed by the oracle."""
    import torch
    wl, extra = W.growth512()
    ctx = M.Context()
    lat = M.DeviceLattice(wl.lattice)
    prm = M.DeviceParams(wl.params)
    solver = M.StepSolver(ctx, lat, prm, wl.margin)
    cnn, _ = _net(M, ctx, wl.lattice.dims, seed=4, last_scale=0.1, s_out=0.01)
    solver.set_network(cnn)
    opts = M.make_opts(rtol=1e-6, restart=8, maxit=500, precision=1, inner_rtol=1e-6)
    for t in (0, 100, 199):
        W.grow(wl, t, extra)
        lat.cell_id.copy_(torch.from_numpy(wl.lattice.cell_id))
        before = wl.lattice.copy()
        before.fields = lat.fields_numpy()
        rep = solver.step(opts)
        assert rep["status_code"] == M.OK
        box = rep["box"]
        assert box == oracle.bbox(before.cell_id, wl.margin)
        after = lat.fields_numpy()
        mb = oracle.box_view(before.mask, box)
        cb = oracle.box_view(before.cell_id, box)
        for s in range(3):
            A, b = oracle.assemble(mb, cb, oracle.box_view(before.fields[s], box), wl.params, s)
            r = b.reshape(-1) - A.matvec(oracle.box_view(after[s], box).reshape(-1))
            assert np.linalg.norm(r) <= 1e-6 * np.linalg.norm(b.reshape(-1)[mb.reshape(-1) > 0]), (t, s)
        outside = np.ones(before.mask.shape, bool)
        outside[oracle.box_slices(box)] = False
        outside |= before.mask == 0
        assert np.array_equal(after[:, outside], before.fields[:, outside])


def test_growth512_guess_matches_oracle_on_sampled_voxels(M):
    """The network's guess at full size, in the launch configuration the
    benchmark times (the learned step graph on the 512x384x384 growing tumour
    at its last, largest state): a tolerance of 1e3 ||b|| stops every species
    at its first residual, so the fields the step scatters are the prediction.  Sampled
    in-mask voxels of the box are checked one by one against the oracle's
    network on the voxel's receptive field (radius 6 for six 3x3x3 layers,
    clipped to the box: the network sees the box only), at the bound of the
    whole-box test."""
    import torch
    from types import SimpleNamespace
    wl, extra = W.growth512()
    W.grow(wl, wl.steps - 1, extra)
    ctx = M.Context()
    lat = M.DeviceLattice(wl.lattice)
    prm = M.DeviceParams(wl.params)
    solver = M.StepSolver(ctx, lat, prm, wl.margin)
    s_out = 0.05
    cnn, params = _net(M, ctx, wl.lattice.dims, seed=5, last_scale=0.3, s_out=s_out)
    solver.set_network(cnn)
    rep = solver.step(M.make_opts(rtol=1e3, restart=8, maxit=50))
    assert rep["status_code"] == M.OK and rep["iters"] == [0, 0, 0]
    box = rep["box"]
    assert box == oracle.bbox(wl.lattice.cell_id, wl.margin)
    (lx, ly, lz), (hx, hy, hz) = box
    got = [lat.fields[s].cpu().numpy() for s in range(3)]
    P = oracle.bf16(params.astype(np.float64))
    rng = np.random.default_rng(11)
    mz, my, mx = np.nonzero(wl.lattice.mask[lz:hz, ly:hy, lx:hx])
    pick = rng.choice(len(mx), size=24, replace=False)
    z6g, z6o = [], []
    for i in pick:
        x, y, z = lx + mx[i], ly + my[i], lz + mz[i]
        x0, x1 = max(lx, x - 6), min(hx, x + 7)
        y0, y1 = max(ly, y - 6), min(hy, y + 7)
        z0, z1 = max(lz, z - 6), min(hz, z + 7)
        sl = (slice(z0, z1), slice(y0, y1), slice(x0, x1))
        sub = SimpleNamespace(cell_id=wl.lattice.cell_id[sl], mask=wl.lattice.mask[sl],
                              fields=wl.lattice.fields[(slice(None),) + sl])
        X = _features_np(sub, wl.params)
        F = np.moveaxis(sub.fields.astype(np.float32).astype(np.float64), 0, -1)
        p_o, _ = oracle.cnn_forward(X, F, P, s_out)
        c = (z - z0, y - y0, x - x0)
        for s in range(3):
            z6o.append((p_o[c + (s,)] - F[c + (s,)]) / s_out)
            z6g.append((got[s][z, y, x] - wl.lattice.fields[s][z, y, x]) / s_out)
    z6g, z6o = np.array(z6g), np.array(z6o)
    assert np.max(np.abs(z6g - z6o)) <= 1e-2 * np.max(np.abs(z6o)) + 1e-6
    # voxels of the box outside the mask keep c^n
    outside = wl.lattice.mask[lz:hz, ly:hy, lx:hx] == 0
    for s in range(3):
        assert np.array_equal(got[s][lz:hz, ly:hy, lx:hx][outside], wl.lattice.fields[s][lz:hz, ly:hy, lx:hx][outside])
