"""The allocation-free bounding box (mpm_box_bounds_noalloc) against the CPU
oracle's bounding box (Sec. 2.3) and against mpm_box_extract, on two calls in a
row.

Callers that may not allocate device memory (their memory belongs to another
allocator, or they cannot afford the synchronisation an allocation can cause)
use this entry point; its scratch is a fixed array inside the library that
every call reuses, so the second call also checks that nothing left over from
the first one leaks into its answer.  Integer output: compared exactly.
"""
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


def _extract_box(M, ctx, wl, margin):
    lat = M.DeviceLattice(wl.lattice)
    sub = ctx.subgrid_create()
    box = sub.mpm_box_extract(lat, wl.params.nspecies, margin)
    sub.destroy()
    return box


def _noalloc_box(M, wl, margin):
    import torch
    cell = torch.from_numpy(np.ascontiguousarray(wl.lattice.cell_id)).cuda()
    out = torch.full((7,), -7, dtype=torch.int32, device="cuda")
    st = M.mpm_box_bounds_noalloc(cell, margin, out)
    assert st == M.OK
    torch.cuda.synchronize()
    o = out.cpu().numpy().tolist()
    return None if o[6] == 0 else (tuple(o[0:3]), tuple(o[3:6]))


def test_noalloc_box_matches_extract_on_two_calls_in_a_row(M):
    ctx = M.Context()
    cases = [(W.random_case(21, (37, 29, 23), nspecies=1), 2),   # first call: a large box
             (W.random_case(22, (9, 14, 31), nspecies=1), 0)]    # second call: a different, smaller lattice
    cases[1][0].lattice.cell_id[:] = 0
    cases[1][0].lattice.cell_id[17, 3, 5] = 4                   # a single tumour voxel
    for wl, margin in cases:
        got = _noalloc_box(M, wl, margin)
        assert got == oracle.bbox(wl.lattice.cell_id, margin)
        assert got == _extract_box(M, ctx, wl, margin)


def test_noalloc_box_margin_clamped_against_the_oracle(M):
    # tumour voxels on opposite lattice faces and a margin larger than the
    # lattice: every bound is clamped (lo to 0, hi to L)
    wl = W.random_case(24, (19, 11, 7), nspecies=1)
    c = wl.lattice.cell_id
    c[:] = 0
    c[0, 5, 18] = 3
    c[6, 0, 2] = 1
    for margin in (0, 1, 4, 40):
        assert _noalloc_box(M, wl, margin) == oracle.bbox(c, margin)
    # a single interior voxel, clamped on one side only
    c[:] = 0
    c[3, 9, 1] = 2
    for margin in (0, 2, 5):
        assert _noalloc_box(M, wl, margin) == oracle.bbox(c, margin)


def test_noalloc_box_empty_and_full_lattices(M):
    ctx = M.Context()
    wl = W.random_case(23, (16, 8, 12), nspecies=1)
    wl.lattice.cell_id[:] = 0
    assert _noalloc_box(M, wl, 3) is None and oracle.bbox(wl.lattice.cell_id, 3) is None
    wl.lattice.cell_id[:] = 2
    assert _noalloc_box(M, wl, 1) == oracle.bbox(wl.lattice.cell_id, 1) == _extract_box(M, ctx, wl, 1) \
        == ((0, 0, 0), (16, 8, 12))


def test_noalloc_rejects_lattices_taller_than_its_scratch(M):
    import torch
    cell = torch.zeros((M.NOALLOC_MAX_SLABS + 1, 1, 1), dtype=torch.int32, device="cuda")
    out = torch.zeros(7, dtype=torch.int32, device="cuda")
    assert M.mpm_box_bounds_noalloc(cell, 0, out) == M.ERR_NOMEM


def test_noalloc_wrapper_rejects_bad_tensors(M):
    import torch
    cell = torch.zeros((4, 4, 4), dtype=torch.int32, device="cuda")
    out = torch.zeros(7, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        M.mpm_box_bounds_noalloc(cell.cpu(), 0, out)
    with pytest.raises(ValueError):
        M.mpm_box_bounds_noalloc(cell.to(torch.int64), 0, out)
    with pytest.raises(ValueError):
        M.mpm_box_bounds_noalloc(cell.transpose(0, 2), 0, out)
    with pytest.raises(ValueError):
        M.mpm_box_bounds_noalloc(cell, 0, out[:6])
