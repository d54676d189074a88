"""The device growth driver (mpm_cpm_step) against the oracle's cpm_step, bit
for bit: cell ids, the number of ids in use, the rate tables written for the
daughters and the counters, step after step; then coupled to the solver (the
device step advances the fields, the driver grows the tumour on them)."""
import numpy as np
import pytest

import oracle
from paper_2505_03067_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CP = dict(p_grow=0.6, K_o2=0.2, K_nut=0.3, o2_min=0.05, v_div=60)


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_03067_gb300 import build, mpm
    build.build()
    return mpm


def _blob_case(seed, dims, ncell=40, cap=400):
    rng = np.random.default_rng(seed)
    wl = W.random_case(seed, dims, nspecies=3)
    Lz, Ly, Lx = wl.lattice.cell_id.shape
    cell = np.zeros((Lz, Ly, Lx), np.int32)
    zz, yy, xx = np.indices(cell.shape)
    c = np.array([Lz, Ly, Lx]) / 2
    ball = (zz - c[0]) ** 2 + (yy - c[1]) ** 2 + (xx - c[2]) ** 2 <= (min(dims) / 4) ** 2
    cell[ball] = rng.integers(1, ncell, size=int(ball.sum()))
    wl.lattice.cell_id = cell
    wl.lattice.mask[ball] = 1
    k = np.zeros((3, cap))
    q = np.zeros((3, cap))
    k[:, :ncell] = rng.uniform(0.01, 0.1, (3, ncell))
    q[:, :ncell] = rng.uniform(0.01, 0.1, (3, ncell))
    k[:, 0] = q[:, 0] = 0.0
    wl.params = W.dataclasses.replace(wl.params, k_cell=k, q_cell=q)
    for s in range(2):
        wl.lattice.fields[s] = rng.uniform(0.0, 1.0, cell.shape)
    return wl, ncell


def _run_pair(M, wl, ncell, steps, seed, cp=CP, solver_opts=None):
    ctx = M.Context()
    lat = M.DeviceLattice(wl.lattice)
    prm = M.DeviceParams(wl.params)
    g = M.GrowthDriver(ctx, lat, prm, ncell, seed=seed, **cp)
    solver = M.StepSolver(ctx, lat, prm, wl.margin) if solver_opts else None
    cell = wl.lattice.cell_id.copy()
    k, q = wl.params.k_cell.copy(), wl.params.q_cell.copy()
    nc = ncell
    grown = div = 0
    for t in range(steps):
        if solver:
            rep = solver.step(solver_opts)
            assert rep["status_code"] == M.OK
        f = lat.fields_numpy()
        cell, k, q, nc, st = oracle.cpm_step(cell, wl.lattice.mask, f[0], f[1], k, q, nc, cp, seed, t)
        grown += st["grown"]
        div += st["divisions"]
        g.step()
        got = lat.cell_id.cpu().numpy()
        assert np.array_equal(got, cell), (t, int(np.sum(got != cell)))
        cnt = g.counts()
        assert cnt["ncell"] == nc and cnt["grown"] == grown and cnt["divisions"] == div and cnt["bad_ids"] == 0
        assert np.array_equal(prm.k.cpu().numpy(), k[:wl.params.nspecies])
        assert np.array_equal(prm.q.cpu().numpy(), q[:wl.params.nspecies])
    return grown, div


def test_growth_steps_match_the_oracle_bit_for_bit(M):
    wl, nc = _blob_case(91, (71, 53, 47))
    grown, div = _run_pair(M, wl, nc, 8, seed=123)
    assert grown > 1000 and div > 10


def test_table_capacity_stops_divisions(M):
    wl, nc = _blob_case(92, (40, 36, 30), ncell=40, cap=45)
    grown, div = _run_pair(M, wl, nc, 4, seed=5, cp=dict(CP, v_div=8))
    assert div == 5


def test_growth_coupled_to_the_solver(M):
    """Fields from the device step, the tumour from the device driver; the
    oracle's driver on the same fields takes the same decisions."""
    wl, nc = _blob_case(93, (60, 50, 44))
    opts = M.make_opts(rtol=1e-8, restart=16, maxit=500)
    grown, div = _run_pair(M, wl, nc, 6, seed=77, solver_opts=opts)
    assert grown > 0
