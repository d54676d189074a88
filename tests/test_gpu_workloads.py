"""The other workloads at their full sizes, in the launch configuration the
benchmark times: the 32^3 sphere (FP64, 1e-10), the 64 batched patches (tuned,
graph-replayed) and the 512x384x384 growing tumour (re-extracted every step).
Large outputs are checked through properties that hold at any size: the true
FP64 residual recomputed by the oracle's assembly and CSR matvec, the
maximum principle and the untouched voxels outside box or mask."""
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


def _true_rel_residuals(before, after, params, margin, box):
    """||b - A x|| / ||b|| per species, A and b from the oracle on the state before the step."""
    mb = oracle.box_view(before.mask, box)
    cb = oracle.box_view(before.cell_id, box)
    out = []
    for s in range(params.nspecies):
        A, b = oracle.assemble(mb, cb, oracle.box_view(before.fields[s], box), params, s)
        x = oracle.box_view(after[s], box).reshape(-1)
        r = b.reshape(-1) - A.matvec(x)
        m = mb.reshape(-1) > 0
        out.append(float(np.linalg.norm(r) / np.linalg.norm(b.reshape(-1)[m])))
    return out


def test_growth512_steps_re_extract_and_meet_tolerance(M):
    import torch
    wl, extra = W.growth512()
    ctx = M.Context()
    lat = M.DeviceLattice(wl.lattice)
    prm = M.DeviceParams(wl.params)
    solver = M.StepSolver(ctx, lat, prm, wl.margin)
    opts = M.make_opts(rtol=1e-6, restart=8, maxit=500, precision=1, inner_rtol=1e-6)
    boxes = []
    for t in (0, 100, 200):
        W.grow(wl, t, extra)
        lat.cell_id.copy_(torch.from_numpy(wl.lattice.cell_id))
        before = wl.lattice.copy()
        before.fields = lat.fields_numpy()
        rep = solver.step(opts)
        assert rep["status_code"] == M.OK
        boxes.append(rep["box"])
        after = lat.fields_numpy()
        box = rep["box"]
        assert box == oracle.bbox(before.cell_id, wl.margin)
        rr = _true_rel_residuals(before, after, wl.params, wl.margin, box)
        assert max(rr) <= 1e-6, rr
        outside = np.ones(before.mask.shape, bool)
        outside[oracle.box_slices(box)] = False
        outside |= before.mask == 0
        assert np.array_equal(after[:, outside], before.fields[:, outside])
        assert after[0].min() >= -1e-9 and after[0].max() <= 1.0 + 1e-9   # maximum principle (q = 0, c_b = 1)
    vol = [np.prod(np.array(b[1]) - np.array(b[0])) for b in boxes]
    assert vol[0] < vol[1] < vol[2]


def test_growth512_early_step_matches_oracle_elementwise(M):
    import torch
    wl, extra = W.growth512()
    W.grow(wl, 10, extra)
    ref = wl.lattice.copy()
    ro = oracle.step(ref, wl.params, wl.margin, rtol=0.0, atol=1e-11)
    ctx = M.Context()
    lat = M.DeviceLattice(wl.lattice)
    rep = M.StepSolver(ctx, lat, M.DeviceParams(wl.params), wl.margin).step(
        M.make_opts(rtol=0.0, atol=1e-11, restart=8, maxit=500))
    assert rep["box"] == ro["box"]
    got = lat.fields_numpy()
    sl = oracle.box_slices(ro["box"])
    assert np.max(np.abs(got[(slice(None),) + sl] - ref.fields[(slice(None),) + sl])) <= 1e-10


def test_patches64_tuned_graph_batch(M):
    ps = W.patches()
    ctx = M.Context()
    lats = [M.DeviceLattice(p.lattice) for p in ps]
    prms = [M.DeviceParams(p.params) for p in ps]
    bs = M.BatchStepper(ctx, lats, prms, [p.margin for p in ps], tune_tiles=True)
    opts = M.make_opts(rtol=1e-6, restart=8, maxit=500, precision=1, inner_rtol=1e-6)
    m, var = bs.tune(opts)
    assert m in (4, 8, 16) and 0 <= var <= 6
    befores = [p.lattice.copy() for p in ps]
    st, reps = bs.step(opts)
    assert st == M.OK
    st, reps2 = bs.step(opts)
    assert bs.graph_active()
    # first step of a sample of patches against the oracle's residual
    lats2 = [M.DeviceLattice(p.lattice) for p in ps[:8]]
    bs2 = M.BatchStepper(ctx, lats2, [M.DeviceParams(p.params) for p in ps[:8]], [p.margin for p in ps[:8]],
                         tune_tiles=True)
    st, reps3 = bs2.step(opts)
    for p, b, lat, rep in zip(ps[:8], befores[:8], lats2, reps3):
        box = ((0, 0, 0), tuple(int(v) for v in p.lattice.cell_id.shape[::-1]))
        rr = _true_rel_residuals(b, lat.fields_numpy(), p.params, p.margin, box)
        assert max(rr) <= 1e-6, rr


def test_sphere32_spec_tolerance_fp64(M):
    wl = W.sphere32()
    ctx = M.Context()
    lat = M.DeviceLattice(wl.lattice)
    solver = M.StepSolver(ctx, lat, M.DeviceParams(wl.params), wl.margin)
    for _ in range(wl.steps):
        before = wl.lattice.copy()
        before.fields = lat.fields_numpy()
        rep = solver.step(M.make_opts(rtol=wl.rtol, restart=wl.restart, maxit=500))
        assert rep["status_code"] == M.OK
        rr = _true_rel_residuals(before, lat.fields_numpy(), wl.params, wl.margin, rep["box"])
        assert rr[0] <= 1e-10
