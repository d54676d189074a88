"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact for the box extraction (integers, bytes, copies); FP64 solves within
1e-10 max-abs of the oracle when both are driven to ||r||_2 <= 1e-13 (the error
of each is then below its residual, ||A^-1||_2 <= 1); the FP32-in-FP64 path
within 1e-6 relative to the FP64 oracle solution with its own true residual
below 1e-6 ||b||.
"""
import numpy as np
import pytest

import oracle
from paper_2505_03067_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TILES = [(8, 8, 4), (4, 4, 4), (32, 4, 2), (8, 4, 1), (16, 16, 4)]


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_03067_gb300 import build, mpm
    build.build()
    return mpm


@pytest.fixture(scope="module")
def ctx(M):
    return M.Context()


def _expected_flags(mask_box):
    m = mask_box > 0
    f = np.zeros(mask_box.shape, np.uint8)
    f[m] |= 64
    nz, ny, nx = m.shape
    sh = [((slice(None), slice(None), slice(1, None)), (slice(None), slice(None), slice(0, -1)), 1),   # -x
          ((slice(None), slice(None), slice(0, -1)), (slice(None), slice(None), slice(1, None)), 2),   # +x
          ((slice(None), slice(1, None), slice(None)), (slice(None), slice(0, -1), slice(None)), 4),   # -y
          ((slice(None), slice(0, -1), slice(None)), (slice(None), slice(1, None), slice(None)), 8),   # +y
          ((slice(1, None), slice(None), slice(None)), (slice(0, -1), slice(None), slice(None)), 16),  # -z
          ((slice(0, -1), slice(None), slice(None)), (slice(1, None), slice(None), slice(None)), 32)]  # +z
    for me, nb, bit in sh:
        both = m[me] & m[nb]
        f[me] |= (both * bit).astype(np.uint8)
    return f


def _active_tiles(mask_box, tile):
    tx, ty, tz = tile
    nz, ny, nx = mask_box.shape
    act = np.zeros(mask_box.shape, bool)
    for k in range(0, nz, tz):
        for j in range(0, ny, ty):
            for i in range(0, nx, tx):
                blk = mask_box[k:k + tz, j:j + ty, i:i + tx]
                if blk.any():
                    act[k:k + tz, j:j + ty, i:i + tx] = True
    return act


CASES = [(0, (21, 13, 11)), (1, (8, 8, 8)), (2, (33, 17, 5)), (3, (1, 1, 1)), (4, (40, 3, 9)), (5, (17, 29, 23))]


@pytest.mark.parametrize("seed,dims", CASES)
@pytest.mark.parametrize("tile", TILES[:3])
def test_extract_is_bit_exact(M, ctx, seed, dims, tile):
    wl = W.random_case(seed, dims, nspecies=3, dfac=(seed % 2 == 0))
    if seed == 3:
        wl.lattice.cell_id[:] = 1
        wl.lattice.mask[:] = 1
    lat = M.DeviceLattice(wl.lattice)
    sub = ctx.subgrid_create()
    box = sub.mpm_box_extract(lat, 3, wl.margin, tile)
    assert box == oracle.bbox(wl.lattice.cell_id, wl.margin)
    mb = oracle.box_view(wl.lattice.mask, box)
    act = _active_tiles(mb, tile)
    info = sub.info()
    assert info["mask_voxels"] == int(mb.sum())
    assert info["stored_voxels"] == info["nactive"] * tile[0] * tile[1] * tile[2]
    flags = sub.mpm_subgrid_export(M.EXPORT_FLAGS).cpu().numpy()
    exp = np.where(act, _expected_flags(mb) | 128, 0).astype(np.uint8)
    assert np.array_equal(flags, exp)
    cell = sub.mpm_subgrid_export(M.EXPORT_CELL).cpu().numpy()
    assert np.array_equal(cell, np.where(act, oracle.box_view(wl.lattice.cell_id, box), 0))
    for s in range(3):
        x = sub.mpm_subgrid_export(M.EXPORT_X, s).cpu().numpy()
        assert np.array_equal(x, np.where(act, oracle.box_view(wl.lattice.fields[s], box), 0.0))
    sub.destroy()


@pytest.mark.parametrize("seed,dims", CASES[:3] + CASES[4:])
@pytest.mark.parametrize("bc_box", [0, 1])
def test_assembly_and_operator_match_oracle_csr(M, ctx, seed, dims, bc_box):
    import torch
    wl = W.random_case(seed, dims, nspecies=3, dfac=(seed % 2 == 1))
    lat = M.DeviceLattice(wl.lattice)
    prm = M.DeviceParams(wl.params, bc_box=bc_box)
    sub = ctx.subgrid_create()
    box = sub.mpm_box_extract(lat, 3, wl.margin, (8, 4, 2))
    sub.mpm_assemble_coeffs(prm)
    mb, cb, = (oracle.box_view(a, box) for a in (wl.lattice.mask, wl.lattice.cell_id))
    dfb = None if wl.lattice.dfac is None else oracle.box_view(wl.lattice.dfac, box)
    rng = np.random.default_rng(seed + 100)
    for s in range(3):
        A, b = oracle.assemble(mb, cb, oracle.box_view(wl.lattice.fields[s], box), wl.params, s, bc_box, dfb)
        D = np.zeros(A.N)
        for r in range(A.N):
            for e in range(A.row_ptr[r], A.row_ptr[r + 1]):
                if A.col[e] == r:
                    D[r] = A.val[e]
        act = _active_tiles(mb, (8, 4, 2))
        dg = sub.mpm_subgrid_export(M.EXPORT_DIAG, s).cpu().numpy().reshape(-1)
        rhs = sub.mpm_subgrid_export(M.EXPORT_RHS, s).cpu().numpy().reshape(-1)
        a = act.reshape(-1)
        assert np.max(np.abs(dg[a] - D[a]) / np.abs(D[a])) < 1e-14
        assert np.max(np.abs(rhs[a] - b.reshape(-1)[a])) <= 1e-14 * max(1.0, np.abs(b).max())
        x = rng.uniform(-1, 1, mb.shape)
        y = sub.mpm_apply_operator(s, torch.from_numpy(x).cuda()).cpu().numpy().reshape(-1)
        yref = A.matvec(x)
        assert np.max(np.abs(y - yref)) <= 1e-13 * max(1.0, np.abs(yref).max())
    sub.destroy()


def _gpu_step(M, ctx, wl, opts, tile=None, lat=None, prm=None, allow=None, fused=True):
    lat = lat or M.DeviceLattice(wl.lattice)
    prm = prm or M.DeviceParams(wl.params)
    solver = M.StepSolver(ctx, lat, prm, wl.margin, tile, fused=fused)
    rep = solver.step(opts, allow=allow if allow is not None else (M.ERR_NOCONV,))
    return lat, rep


@pytest.mark.parametrize("seed,dims", CASES)
@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("fused", [True, False])
def test_fp64_solve_matches_oracle(M, ctx, seed, dims, tile, fused):
    wl = W.random_case(seed, dims, nspecies=3, dfac=(seed % 3 == 0))
    ref = wl.lattice.copy()
    ro = oracle.step(ref, wl.params, wl.margin, rtol=0.0, atol=1e-13)
    lat, rep = _gpu_step(M, ctx, wl, M.make_opts(rtol=0.0, atol=1e-13, restart=16, maxit=2000), tile, fused=fused)
    assert rep["box"] == ro["box"] and rep["mask_voxels"] == ro["mask_voxels"]
    assert rep["status_code"] == M.OK
    assert all(r <= 1e-13 for r in rep["res"])
    got = lat.fields_numpy()
    assert np.max(np.abs(got - ref.fields)) <= 1e-10


@pytest.mark.parametrize("restart", [2, 5, 8, 30])
def test_restart_lengths_agree(M, ctx, restart):
    wl = W.random_case(9, (19, 18, 17), nspecies=3)
    ref = wl.lattice.copy()
    oracle.step(ref, wl.params, wl.margin, rtol=0.0, atol=1e-13)
    lat, rep = _gpu_step(M, ctx, wl, M.make_opts(rtol=0.0, atol=1e-13, restart=restart, maxit=5000))
    assert rep["status_code"] == M.OK
    if restart < 8:
        assert max(rep["cycles"]) > 1
    assert np.max(np.abs(lat.fields_numpy() - ref.fields)) <= 1e-10


def test_sphere32_ten_steps_fp64(M, ctx):
    """The 32^3 single-species workload, 10 implicit-Euler steps, GMRES(30): parity
    run with both sides at ||r||_2 <= 1e-13 per step (10 steps add at most 1e-12
    each), max-abs within 1e-10; then the 1e-10-relative run, whose distance to the
    parity solution is bounded by the sum of its per-step residual norms."""
    wl = W.sphere32()
    ref = wl.lattice.copy()
    for _ in range(wl.steps):
        assert oracle.step(ref, wl.params, wl.margin, rtol=0.0, atol=1e-13)["status"] == oracle.OK
    lat = M.DeviceLattice(wl.lattice)
    prm = M.DeviceParams(wl.params)
    solver = M.StepSolver(ctx, lat, prm, wl.margin)
    for _ in range(wl.steps):
        rep = solver.step(M.make_opts(rtol=0.0, atol=1e-13, restart=30, maxit=1000))
        assert rep["status_code"] == M.OK and rep["box"] == ((0, 0, 0), (32, 32, 32))
    assert np.max(np.abs(lat.fields_numpy() - ref.fields)) <= 1e-10
    lat2 = M.DeviceLattice(wl.lattice)
    solver2 = M.StepSolver(ctx, lat2, prm, wl.margin)
    bound = 0.0
    for _ in range(wl.steps):
        rep = solver2.step(M.make_opts(rtol=wl.rtol, restart=30, maxit=1000))
        assert rep["status_code"] == M.OK
        assert rep["res"][0] <= 1e-10 * rep["bnorm"][0]
        bound += rep["res"][0]
    assert np.max(np.abs(lat2.fields_numpy() - ref.fields)) <= bound + 1e-12


@pytest.mark.parametrize("seed,dims", CASES[:3] + [(6, (45, 37, 29))])
def test_mixed_precision_within_1e6_of_fp64(M, ctx, seed, dims):
    wl = W.random_case(seed, dims, nspecies=3)
    ref = wl.lattice.copy()
    oracle.step(ref, wl.params, wl.margin, rtol=0.0, atol=1e-13)
    lat, rep = _gpu_step(M, ctx, wl, M.make_opts(rtol=1e-6, restart=16, maxit=500, precision=1, inner_rtol=1e-5))
    assert rep["status_code"] == M.OK
    got = lat.fields_numpy()
    box = rep["box"]
    mb = oracle.box_view(wl.lattice.mask, box) > 0
    for s in range(3):
        assert rep["res"][s] <= 1e-6 * rep["bnorm"][s]
        g = oracle.box_view(got[s], box)[mb]
        r = oracle.box_view(ref.fields[s], box)[mb]
        assert np.linalg.norm(g - r) <= 1e-6 * np.linalg.norm(r)
        # the residual claimed by the GPU, recomputed by the oracle on the GPU's answer
        A, b = oracle.assemble(oracle.box_view(wl.lattice.mask, box), oracle.box_view(wl.lattice.cell_id, box),
                               oracle.box_view(wl.lattice.fields[s], box), wl.params, s)
        xr = oracle.box_view(got[s], box).reshape(-1)
        assert abs(np.linalg.norm(b.reshape(-1) - A.matvec(xr)) - rep["res"][s]) <= 1e-9 * rep["bnorm"][s]


@pytest.mark.parametrize("scale", [1e-20, 1e-30])
@pytest.mark.parametrize("fused", [True, False])
def test_mixed_precision_tiny_fields(M, ctx, scale, fused):
    # every concentration, boundary value and source scaled by 1e-20 / 1e-30:
    # the solution scales exactly (the system is linear), and the FP32 path
    # must neither stop on an underflowed norm nor break down
    wl = W.random_case(31, (23, 17, 13), nspecies=3)
    wl.lattice.fields *= scale
    wl.params.c_bc *= scale
    wl.params.q_cell *= scale
    ref = wl.lattice.copy()
    oracle.step(ref, wl.params, wl.margin, rtol=1e-12)
    lat, rep = _gpu_step(M, ctx, wl, M.make_opts(rtol=1e-6, restart=16, maxit=500, precision=1, inner_rtol=1e-5),
                         fused=fused)
    assert rep["status_code"] == M.OK
    got = lat.fields_numpy()
    box = rep["box"]
    mb = oracle.box_view(wl.lattice.mask, box) > 0
    for s in range(3):
        assert 0.0 < rep["bnorm"][s] and rep["res"][s] <= 1e-6 * rep["bnorm"][s]
        assert rep["iters"][s] > 0
        g = oracle.box_view(got[s], box)[mb]
        r = oracle.box_view(ref.fields[s], box)[mb]
        assert np.linalg.norm(g - r) <= 1e-6 * np.linalg.norm(r)


def test_deterministic(M, ctx):
    wl = W.random_case(2, (33, 17, 25), nspecies=3)
    outs = []
    for _ in range(2):
        lat, rep = _gpu_step(M, ctx, wl, M.make_opts(rtol=1e-8, restart=16, maxit=500))
        outs.append(lat.fields_numpy())
    assert np.array_equal(outs[0], outs[1])


# ---------------------------------------------------------------- edge cases and failures
def test_empty_tumour_is_reported_and_changes_nothing(M, ctx):
    wl = W.random_case(1, (9, 9, 9))
    wl.lattice.cell_id[:] = 0
    lat = M.DeviceLattice(wl.lattice)
    sub = ctx.subgrid_create()
    assert sub.mpm_box_extract(lat, 3, 2) is None
    assert np.array_equal(lat.fields_numpy(), wl.lattice.fields)


def test_tumour_outside_mask_has_no_unknowns(M, ctx):
    wl = W.random_case(4, (12, 12, 12))
    wl.lattice.mask[:] = 0
    lat, rep = _gpu_step(M, ctx, wl, M.make_opts())
    assert rep["status_code"] == M.OK and rep["stored_voxels"] == 0
    assert np.array_equal(lat.fields_numpy(), wl.lattice.fields)


def test_single_voxel_tumour_margin_clamped(M, ctx):
    wl = W.random_case(5, (10, 11, 12), nspecies=2)
    wl.lattice.cell_id[:] = 0
    wl.lattice.cell_id[0, 0, 9] = 3
    ref = wl.lattice.copy()
    ro = oracle.step(ref, wl.params, 3, rtol=0.0, atol=1e-13)
    wl.margin = 3
    lat, rep = _gpu_step(M, ctx, wl, M.make_opts(rtol=0.0, atol=1e-13, restart=8))
    assert rep["box"] == ro["box"] == ((6, 0, 0), (10, 4, 4))
    assert np.max(np.abs(lat.fields_numpy() - ref.fields)) <= 1e-10


def test_maxit_reports_noconv_and_keeps_best_iterate(M, ctx):
    wl = W.random_case(3, (16, 16, 16), nspecies=3)
    lat, rep = _gpu_step(M, ctx, wl, M.make_opts(rtol=1e-14, restart=8, maxit=1))
    assert rep["status_code"] == M.ERR_NOCONV
    assert all(st == M.ERR_NOCONV for st in rep["status"]) and rep["iters"] == [1, 1, 1]
    assert not np.array_equal(lat.fields_numpy(), wl.lattice.fields)


def test_nan_input_reports_breakdown(M, ctx):
    wl = W.random_case(3, (16, 16, 16), nspecies=3)
    box = oracle.bbox(wl.lattice.cell_id, wl.margin)
    sl = oracle.box_slices(box)
    inm = np.argwhere(wl.lattice.mask[sl] > 0)[0]
    wl.lattice.fields[1][sl][tuple(inm)] = np.nan
    lat, rep = _gpu_step(M, ctx, wl, M.make_opts(), allow=(M.ERR_BREAKDOWN,))
    assert rep["status_code"] == M.ERR_BREAKDOWN
    assert rep["status"][1] == M.ERR_BREAKDOWN
    assert rep["status"][0] == M.OK and rep["status"][2] == M.OK


def test_cell_id_outside_tables_is_an_argument_error(M, ctx):
    wl = W.random_case(3, (16, 16, 16), nspecies=1)
    wl.lattice.cell_id[wl.lattice.mask > 0] = 999
    lat = M.DeviceLattice(wl.lattice)
    prm = M.DeviceParams(wl.params)
    sub = ctx.subgrid_create()
    sub.mpm_box_extract(lat, 1, 1)
    sub.mpm_assemble_coeffs(prm)
    with pytest.raises(M.MpmError) as ei:
        sub.mpm_solve_step(M.make_opts())
    assert ei.value.status == M.ERR_ARG
    # later solves on a clean subgrid work again
    wl2 = W.random_case(3, (16, 16, 16), nspecies=1)
    lat2, rep = _gpu_step(M, M.Context(), wl2, M.make_opts())
    assert rep["status_code"] == M.OK


def test_missing_partner_cta_times_out_and_context_survives(M):
    """A CTA that never arrives (host-set skip flag): its partners' bounded waits
    expire, the solve returns MPM_ERR_TIMEOUT, and the same context then solves."""
    c = M.Context()
    wl = W.random_case(2, (33, 17, 25), nspecies=3)
    c.debug_set(M.DEBUG_TIMEOUT_NS, 50_000_000)
    c.debug_set(M.DEBUG_SKIP_BLOCK, 0)
    lat = M.DeviceLattice(wl.lattice)
    prm = M.DeviceParams(wl.params)
    solver = M.StepSolver(c, lat, prm, wl.margin)
    with pytest.raises(M.MpmError) as ei:
        solver.step(M.make_opts(nblocks=4))
    assert ei.value.status == M.ERR_TIMEOUT
    assert np.array_equal(lat.fields_numpy(), wl.lattice.fields)
    c.debug_set(M.DEBUG_SKIP_BLOCK, -1)
    rep = solver.step(M.make_opts(nblocks=4))
    assert rep["status_code"] == M.OK


# ---------------------------------------------------------------- full-size workload
@pytest.fixture(scope="module")
def shell256():
    return W.shell256()


@pytest.mark.parametrize("precision", [0, 1])
def test_shell256_first_step_matches_oracle(M, ctx, shell256, precision):
    """The 256^3 three-species pleural-shell workload, first step, through the
    device-resident step the benchmark times (default grid and tile), compared
    with the oracle on every in-mask voxel of the box."""
    wl = shell256
    ref = wl.lattice.copy()
    ro = oracle.step(ref, wl.params, wl.margin, rtol=0.0, atol=1e-11)
    assert ro["status"] == oracle.OK
    if precision == 0:
        opts = M.make_opts(rtol=0.0, atol=1e-11, restart=16, maxit=500)
    else:
        opts = M.make_opts(rtol=1e-6, restart=16, maxit=500, precision=1, inner_rtol=1e-5)
    lat, rep = _gpu_step(M, ctx, wl, opts)
    assert rep["status_code"] == M.OK and rep["box"] == ro["box"]
    assert rep["mask_voxels"] == ro["mask_voxels"]
    got = lat.fields_numpy()
    box = ro["box"]
    mb = oracle.box_view(wl.lattice.mask, box) > 0
    for s in range(3):
        g = oracle.box_view(got[s], box)[mb]
        r = oracle.box_view(ref.fields[s], box)[mb]
        if precision == 0:
            assert np.max(np.abs(g - r)) <= 1e-10
        else:
            assert np.linalg.norm(g - r) <= 1e-6 * np.linalg.norm(r)


def test_four_species_il8(M, ctx):
    """Eq. 1-4 with all four species (O2, nutrient, IL6, IL8): the same kernels with S = 4."""
    wl = W.random_case(40, (23, 19, 17), nspecies=4)
    ref = wl.lattice.copy()
    oracle.step(ref, wl.params, wl.margin, rtol=0.0, atol=1e-13)
    lat, rep = _gpu_step(M, ctx, wl, M.make_opts(rtol=0.0, atol=1e-13, restart=8, maxit=2000))
    assert rep["status_code"] == M.OK and len(rep["iters"]) == 4
    assert np.max(np.abs(lat.fields_numpy() - ref.fields)) <= 1e-10


# ---------------------------------------------------------------- device-resident step
def _grow_cells(wl, r, centre):
    """Tumour = mask voxels within radius r of centre, ids by octant (1..8)."""
    lz, ly, lx = wl.lattice.cell_id.shape
    z, y, x = np.meshgrid(np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    d = np.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2)
    ids = 1 + (x > centre[0]) + 2 * (y > centre[1]) + 4 * (z > centre[2])
    return np.where((d <= r) & (wl.lattice.mask > 0), ids, 0).astype(np.int32)


@pytest.mark.parametrize("precision", [0, 1])
def test_device_resident_step_follows_a_moving_growing_tumour(M, ctx, precision):
    """Eight steps of one graph-replayed step while the tumour grows and moves:
    the box (and so the element count and the solver's re-planned grid) changes
    between replays; every step matches the oracle's step on the same lattice."""
    import torch
    wl = W.random_case(21, (48, 40, 36), nspecies=3, ncell=9)
    ref = wl.lattice.copy()
    lat = M.DeviceLattice(wl.lattice)
    prm = M.DeviceParams(wl.params)
    solver = M.StepSolver(ctx, lat, prm, wl.margin, (4, 4, 2))
    if precision == 0:
        opts = M.make_opts(rtol=0.0, atol=1e-13, restart=8, maxit=2000)
    else:
        opts = M.make_opts(rtol=1e-9, restart=8, maxit=2000, precision=1, inner_rtol=1e-6)
    boxes = []
    for k, (r, c) in enumerate([(1.5, (8, 9, 10)), (3, (9, 10, 10)), (6, (12, 12, 12)), (10, (16, 14, 14)),
                                (4, (30, 20, 20)), (14, (24, 20, 18)), (20, (24, 20, 18)), (2, (40, 30, 28))]):
        cid = _grow_cells(wl, r, c)
        if not (cid > 0).any():
            continue
        ref.cell_id = cid
        lat.cell_id.copy_(torch.from_numpy(cid))
        ro = oracle.step(ref, wl.params, wl.margin, rtol=0.0, atol=1e-13)
        rep = solver.step(opts)
        assert rep["status_code"] == M.OK and rep["box"] == ro["box"], (k, rep["box"], ro["box"])
        assert rep["mask_voxels"] == ro["mask_voxels"]
        boxes.append(rep["box"])
        got = lat.fields_numpy()
        if precision == 0:
            assert np.max(np.abs(got - ref.fields)) <= 1e-10, k
        else:
            for s in range(3):
                assert np.linalg.norm(got[s] - ref.fields[s]) <= 3e-8 * np.linalg.norm(ref.fields[s]), (k, s)
            lat.fields.copy_(torch.from_numpy(ref.fields))   # keep both sides on the same c^n
    assert len(set(boxes)) >= 6


def test_device_resident_step_empty_then_tumour(M, ctx):
    """No tumour voxel: MPM_ERR_EMPTY and the lattice unchanged; once a tumour
    appears the same subgrid steps it."""
    import torch
    wl = W.random_case(22, (20, 18, 16), nspecies=2)
    cid = wl.lattice.cell_id.copy()
    wl.lattice.cell_id[:] = 0
    lat = M.DeviceLattice(wl.lattice)
    solver = M.StepSolver(ctx, lat, M.DeviceParams(wl.params), wl.margin)
    opts = M.make_opts(rtol=0.0, atol=1e-13, restart=8, maxit=500)
    rep = solver.step(opts)
    assert rep["status_code"] == M.ERR_EMPTY and rep["box"] is None
    assert np.array_equal(lat.fields_numpy(), wl.lattice.fields)
    lat.cell_id.copy_(torch.from_numpy(cid))
    ref = wl.lattice.copy()
    ref.cell_id = cid
    ro = oracle.step(ref, wl.params, wl.margin, rtol=0.0, atol=1e-13)
    rep = solver.step(opts)
    assert rep["status_code"] == M.OK and rep["box"] == ro["box"]
    assert np.max(np.abs(lat.fields_numpy() - ref.fields)) <= 1e-10
    # and back to empty: nothing is written
    before = lat.fields_numpy()
    lat.cell_id.zero_()
    assert solver.step(opts)["status_code"] == M.ERR_EMPTY
    assert np.array_equal(lat.fields_numpy(), before)


def test_device_resident_step_replays_one_graph(M):
    """After the first call the step is one graph launch of one cooperative
    kernel (extraction, assembly, solve, scatter), and the exports see the
    step's extraction."""
    c = M.Context()
    wl = W.random_case(23, (26, 22, 20), nspecies=3)
    lat = M.DeviceLattice(wl.lattice)
    solver = M.StepSolver(c, lat, M.DeviceParams(wl.params), wl.margin)
    opts = M.make_opts(rtol=1e-10, restart=8, maxit=500)
    solver.step(opts)
    l0 = c.launches()
    for _ in range(3):
        assert solver.step(opts)["status_code"] == M.OK
    assert c.launches() - l0 == 3
    info = solver.sub.info()
    box = oracle.bbox(wl.lattice.cell_id, wl.margin)
    assert info["box"] == box
    flags = solver.sub.mpm_subgrid_export(M.EXPORT_FLAGS).cpu().numpy()
    mb = oracle.box_view(wl.lattice.mask, box)
    assert int(((flags & 64) > 0).sum()) == int(mb.sum())


def test_queued_steps_equal_waited_steps(M, ctx):
    """Steps queued back to back (mpm_step_enqueue, one mpm_step_wait at the end)
    give the lattice of the same steps waited for one by one, bit for bit (a
    fixed grid, so both use one plan); a wait with nothing queued is an
    argument error."""
    wl = W.random_case(24, (30, 26, 22), nspecies=3)
    opts = M.make_opts(rtol=1e-10, restart=8, maxit=500, nblocks=8)
    lat1, lat2 = M.DeviceLattice(wl.lattice), M.DeviceLattice(wl.lattice)
    prm = M.DeviceParams(wl.params)
    s1 = M.StepSolver(ctx, lat1, prm, wl.margin)
    s2 = M.StepSolver(ctx, lat2, prm, wl.margin)
    reps = [s1.step(opts) for _ in range(4)]
    for _ in range(4):
        s2.step_async(opts)
    last = s2.wait()
    assert last["status_code"] == M.OK and last["box"] == reps[-1]["box"]
    assert last["iters"] == reps[-1]["iters"]
    assert np.array_equal(lat1.fields_numpy(), lat2.fields_numpy())
    with pytest.raises(M.MpmError) as ei:
        s2.wait()
    assert ei.value.status == M.ERR_ARG


# ---------------------------------------------------------------- optional reorthogonalisation
@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("seed,dims", [(7, (23, 19, 15)), (2, (33, 17, 5))])
def test_reorthogonalised_fp64_solve_matches_oracle(M, ctx, seed, dims, fused):
    """opt.reorth = 1 adds a second Gram-Schmidt pass to every Arnoldi step
    whose ||w|| dropped below 0.7 of its norm before orthogonalisation; the
    solution is the same linear system's, so it meets the oracle at the same
    bound, and the pass count is reported.  With A near a multiple of the
    identity most of A u_j lies along u_j, so the test fires on most steps."""
    wl = W.random_case(seed, dims, nspecies=3, dfac=True)
    ref = wl.lattice.copy()
    oracle.step(ref, wl.params, wl.margin, rtol=0.0, atol=1e-13)
    got = {}
    for ro in (0, 1):
        lat, rep = _gpu_step(M, ctx, wl, M.make_opts(rtol=0.0, atol=1e-13, restart=16, maxit=3000, reorth=ro),
                             fused=fused)
        assert rep["status_code"] == M.OK
        assert all(r <= 1e-13 for r in rep["res"])
        assert np.max(np.abs(lat.fields_numpy() - ref.fields)) <= 1e-10
        got[ro] = rep
    assert got[0]["reorth"] == [0, 0, 0]
    assert all(0 < n <= it for n, it in zip(got[1]["reorth"], got[1]["iters"]))
    # a second pass can only tighten the basis: no species needs many more steps
    assert all(b <= a + 2 for a, b in zip(got[0]["iters"], got[1]["iters"]))


def test_reorthogonalised_mixed_precision(M, ctx):
    wl = W.random_case(6, (45, 37, 29), nspecies=3)
    ref = wl.lattice.copy()
    oracle.step(ref, wl.params, wl.margin, rtol=0.0, atol=1e-13)
    lat, rep = _gpu_step(M, ctx, wl, M.make_opts(rtol=1e-6, restart=16, maxit=500, precision=1, inner_rtol=1e-5,
                                                  reorth=1))
    assert rep["status_code"] == M.OK and min(rep["reorth"]) > 0
    box = rep["box"]
    mb = oracle.box_view(wl.lattice.mask, box) > 0
    for s in range(3):
        assert rep["res"][s] <= 1e-6 * rep["bnorm"][s]
        g = oracle.box_view(lat.fields_numpy()[s], box)[mb]
        r = oracle.box_view(ref.fields[s], box)[mb]
        assert np.linalg.norm(g - r) <= 1e-6 * np.linalg.norm(r)


def test_reorth_flag_out_of_range_is_an_argument_error(M, ctx):
    wl = W.random_case(3, (16, 16, 16), nspecies=1)
    with pytest.raises(M.MpmError) as ei:
        _gpu_step(M, ctx, wl, M.make_opts(reorth=2))
    assert ei.value.status == M.ERR_ARG


# ---------------------------------------------------------------- host buffers (mpm_step_host)
@pytest.mark.parametrize("pinned", [True, False])
def test_step_from_host_buffers_follows_a_moving_tumour(M, ctx, pinned):
    """mpm_step_host: the host's cell ids (and on the first call its mask and
    fields) go in, the step's results come back (page-locked host fields: the
    in-mask voxels of the box, by a kernel; pageable ones: the whole box, by a
    3-D copy); the device lattice starts out wrong (zero cell ids, mask and
    fields), so the answer can only come from the copies.  Each step meets
    the oracle's step, and after each the host fields equal the device fields
    bit for bit."""
    import torch
    wl = W.random_case(23, (40, 36, 30), nspecies=3, ncell=9)
    ref = wl.lattice.copy()
    zero = wl.lattice.copy()
    zero.cell_id = np.zeros_like(zero.cell_id)
    zero.mask = np.zeros_like(zero.mask)
    zero.fields = np.zeros_like(zero.fields)
    lat = M.DeviceLattice(zero)
    prm = M.DeviceParams(wl.params)
    solver = M.StepSolver(ctx, lat, prm, wl.margin, (4, 4, 4))
    h_mask = torch.from_numpy(np.ascontiguousarray(wl.lattice.mask, np.uint8)).pin_memory()
    h_fields = torch.from_numpy(np.ascontiguousarray(wl.lattice.fields))
    if pinned:
        h_fields = h_fields.pin_memory()
    assert h_fields.is_pinned() == pinned
    opts = M.make_opts(rtol=0.0, atol=1e-13, restart=8, maxit=2000)
    for k, (r, c) in enumerate([(3, (8, 9, 10)), (6, (12, 12, 12)), (4, (25, 20, 16)), (9, (20, 18, 15))]):
        cid = _grow_cells(wl, r, c)
        ref.cell_id = cid
        h_cell = torch.from_numpy(np.ascontiguousarray(cid, np.int32)).pin_memory()
        ro = oracle.step(ref, wl.params, wl.margin, rtol=0.0, atol=1e-13)
        first = k == 0
        rep = solver.step_host(h_cell, h_fields, opts, mask=h_mask if first else None, fields_in=first)
        assert rep["status_code"] == M.OK and rep["box"] == ro["box"], (k, rep["box"], ro["box"])
        assert np.max(np.abs(h_fields.numpy() - ref.fields)) <= 1e-10, k
        assert np.array_equal(h_fields.numpy(), lat.fields_numpy()), k
        assert np.array_equal(lat.cell_id.cpu().numpy(), cid)


def test_step_from_host_buffers_rejects_unknown_flags(M, ctx):
    import ctypes as C
    wl = W.random_case(3, (16, 16, 16), nspecies=1)
    lat = M.DeviceLattice(wl.lattice)
    prm = M.DeviceParams(wl.params)
    sub = ctx.subgrid_create()
    h = M.mpm_host_lattice()
    rep, box = M.mpm_report(), M.mpm_box()
    st = ctx.lib.mpm_step_host(ctx.ptr, sub.h, C.byref(h), C.byref(lat.struct()), C.byref(prm.struct), wl.margin,
                               None, C.byref(M.make_opts()), 2, C.byref(rep), C.byref(box), None)
    assert st == M.ERR_ARG
    sub.destroy()


@pytest.mark.parametrize("tile", [(4, 4, 4), (8, 4, 1), (16, 4, 2), (2, 4, 4), (4, 2, 8)])
@pytest.mark.parametrize("dfac", [False, True])
def test_device_resident_step_rows_equal_composition(M, ctx, tile, dfac):
    """The device-resident step's gather + rows (4-element chunks of tile rows
    when tiles are at least four wide and D is uniform, one element per thread
    otherwise) against mpm_box_extract + mpm_assemble_coeffs, on a box whose x
    extent leaves partial chunks: flags and cell ids bit for bit; the rows bit
    for bit where both evaluate the same expression (per-voxel D), and within
    an ulp where the step sums per-cell table entries (uniform D: the tables
    round dt*q and a*D*n before the sums the assembly fuses into FMAs)."""
    wl = W.random_case(31, (37, 23, 19), nspecies=3, dfac=dfac)
    lat1 = M.DeviceLattice(wl.lattice)
    lat2 = M.DeviceLattice(wl.lattice)
    prm = M.DeviceParams(wl.params)
    solver = M.StepSolver(ctx, lat1, prm, wl.margin, tile)
    rep = solver.step(M.make_opts(rtol=1e-8, restart=8, maxit=500))
    assert rep["status_code"] == M.OK
    sub2 = ctx.subgrid_create()
    box = sub2.mpm_box_extract(lat2, 3, wl.margin, tile)
    sub2.mpm_assemble_coeffs(prm)
    assert box == rep["box"]
    for what in (M.EXPORT_FLAGS, M.EXPORT_CELL):
        a = solver.sub.mpm_subgrid_export(what).cpu().numpy()
        b = sub2.mpm_subgrid_export(what).cpu().numpy()
        assert np.array_equal(a, b), what
    for s in range(3):
        for what in (M.EXPORT_RHS, M.EXPORT_DIAG):
            a = solver.sub.mpm_subgrid_export(what, s).cpu().numpy()
            b = sub2.mpm_subgrid_export(what, s).cpu().numpy()
            if dfac:
                assert np.array_equal(a, b), (what, s)
            else:
                assert np.all(np.abs(a - b) <= 2.3e-16 * np.abs(b)), (what, s, np.max(np.abs(a - b)))
    sub2.destroy()


def test_device_resident_step_many_tiles_equals_composition(M, ctx):
    """A box of more than 64 Ki tiles (4x4x2 tiles on a ~130^3 box), where the
    device-resident step counts the active tiles in a phase of its own before
    the compaction: the same flags, cell ids and tile order as the composition
    path, rows within an ulp (rate tables), and the same solution within the
    residual bound."""
    wl = W.random_case(41, (144, 140, 136), nspecies=2, ncell=9)
    cid = _grow_cells(wl, 64, (72, 70, 68))
    wl.lattice.cell_id = cid
    lat1 = M.DeviceLattice(wl.lattice)
    lat2 = M.DeviceLattice(wl.lattice)
    prm = M.DeviceParams(wl.params)
    tile = (4, 4, 2)
    opts = M.make_opts(rtol=1e-12, restart=8, maxit=2000)
    solver = M.StepSolver(ctx, lat1, prm, wl.margin, tile)
    rep = solver.step(opts)
    assert rep["status_code"] == M.OK
    info = solver.sub.info()
    assert info["ntiles"] > 65536
    sub2 = ctx.subgrid_create()
    box = sub2.mpm_box_extract(lat2, 2, wl.margin, tile)
    assert box == rep["box"]
    for what in (M.EXPORT_FLAGS, M.EXPORT_CELL):
        assert np.array_equal(solver.sub.mpm_subgrid_export(what).cpu().numpy(),
                              sub2.mpm_subgrid_export(what).cpu().numpy()), what
    sub2.mpm_assemble_coeffs(prm)
    for s in range(2):
        a = solver.sub.mpm_subgrid_export(M.EXPORT_RHS, s).cpu().numpy()
        b = sub2.mpm_subgrid_export(M.EXPORT_RHS, s).cpu().numpy()
        assert np.all(np.abs(a - b) <= 2.3e-16 * np.abs(b)), s
    r2 = sub2.mpm_solve_step(opts, scatter_to=lat2)
    assert r2["status_code"] == M.OK
    # both solutions are within ||r||_2 <= 1e-12 ||b||_2 of the exact one (||A^-1||_2 <= 1)
    bound = 1e-12 * sum(max(a, b) for a, b in zip(rep["bnorm"], r2["bnorm"]))
    assert np.max(np.abs(lat1.fields_numpy() - lat2.fields_numpy())) <= bound
    sub2.destroy()


# ---------------------------------------------------------------- box cadence (Sec. 2.3: a box every 50 MCS)
def test_box_cadence_static_tumour_is_bit_identical(M):
    """box_every = 4 on a tumour that does not move: the steps in between keep
    the box, tiles and neighbour table and re-gather c^n and the rows, which
    gives the every-step extraction's results bit for bit; 10 steps take 3 full
    extractions (steps 0, 4, 8)."""
    c = M.Context()
    wl = W.random_case(19, (30, 26, 22), nspecies=3)
    outs = []
    for every in (1, 4):
        lat = M.DeviceLattice(wl.lattice)
        solver = M.StepSolver(c, lat, M.DeviceParams(wl.params), wl.margin)
        opts = M.make_opts(rtol=1e-10, restart=8, maxit=500, box_every=every)
        for _ in range(10):
            rep = solver.step(opts)
            assert rep["status_code"] == M.OK
        outs.append(lat.fields_numpy())
        assert c.counter(M.COUNTER_STEP_FULL_EXTRACTIONS) == (10 if every == 1 else 3)
    assert np.array_equal(outs[0], outs[1])


def test_box_cadence_keeps_the_box_and_the_guard_refreshes_it(M, ctx):
    """A growing tumour with box_every = 50 and a guard band of 2 voxels (the
    margin is 4): while the tumour stays clear of the band the box is kept (the
    oracle, solving on the same kept box, agrees at 1e-10); once a tumour voxel
    enters the band, the next step extracts a new box, the bounding box of
    that step's tumour."""
    wl = W.random_case(21, (48, 40, 36), nspecies=3, ncell=9)
    wl.margin = 4
    ref = wl.lattice.copy()
    lat = M.DeviceLattice(wl.lattice)
    solver = M.StepSolver(ctx, lat, M.DeviceParams(wl.params), wl.margin, (4, 4, 2))
    opts = M.make_opts(rtol=0.0, atol=1e-13, restart=8, maxit=2000, box_every=50, box_guard=2)
    kept, refreshed = 0, 0
    box = None
    pending_refresh = True
    for k, r in enumerate([3.0, 3.0, 3.6, 4.2, 5.0, 5.0, 6.0, 7.5, 7.5, 9.0]):
        cid = _grow_cells(wl, r, (20, 18, 16))
        ref.cell_id = cid
        lat.cell_id.copy_(__import__("torch").from_numpy(cid))
        rep = solver.step(opts)
        assert rep["status_code"] == M.OK
        fresh = oracle.bbox(cid, wl.margin)
        if pending_refresh:
            assert rep["box"] == fresh, k          # a full extraction
            refreshed += 1
        else:
            assert rep["box"] == box, k            # the kept box
            kept += 1
        box = rep["box"]
        ro = oracle.step(ref, wl.params, wl.margin, rtol=0.0, atol=1e-13, box=box)
        assert np.max(np.abs(lat.fields_numpy() - ref.fields)) <= 1e-10, k
        # the guard: a tumour voxel within 2 of a box face inside the lattice
        (lx, ly, lz), (hx, hy, hz) = box
        zz, yy, xx = np.nonzero(cid > 0)
        L = (cid.shape[2], cid.shape[1], cid.shape[0])
        near = False
        for c_, lo, hi, n in ((xx, lx, hx, L[0]), (yy, ly, hy, L[1]), (zz, lz, hz, L[2])):
            inb = (c_ >= lo) & (c_ < hi)
            near |= bool(np.any(inb & (c_ < lo + 2) & (lo > 0))) or bool(np.any(inb & (c_ >= hi - 2) & (hi < n)))
        pending_refresh = near
    assert kept >= 3 and refreshed >= 2


def test_box_cadence_rejects_negative_values(M, ctx):
    wl = W.random_case(3, (16, 16, 16), nspecies=1)
    for kw in ({"box_every": -1}, {"box_guard": -2}):
        with pytest.raises(M.MpmError) as ei:
            _gpu_step(M, ctx, wl, M.make_opts(**kw))
        assert ei.value.status == M.ERR_ARG
