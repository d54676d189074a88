"""The allocation-free bounding box (mpm_box_bounds_noalloc) against the box of
mpm_box_extract, on two calls in a row.

Callers that may not allocate device memory (their memory belongs to another
allocator, or they cannot afford the synchronisation an allocation can cause)
use this entry point; its scratch is a fixed array inside the library that
every call reuses, so the second call also checks that nothing left over from
the first one leaks into its answer.  Integer output: compared exactly.
"""
import numpy as np
import pytest

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
        assert _noalloc_box(M, wl, margin) == _extract_box(M, ctx, wl, margin)


def test_noalloc_box_empty_and_full_lattices(M):
    ctx = M.Context()
    wl = W.random_case(23, (16, 8, 12), nspecies=1)
    wl.lattice.cell_id[:] = 0
    assert _noalloc_box(M, wl, 3) is None
    wl.lattice.cell_id[:] = 2
    assert _noalloc_box(M, wl, 1) == _extract_box(M, ctx, wl, 1) == ((0, 0, 0), (16, 8, 12))


def test_noalloc_rejects_lattices_taller_than_its_scratch(M):
    import torch
    cell = torch.zeros((M.NOALLOC_MAX_SLABS + 1, 1, 1), dtype=torch.int32, device="cuda")
    out = torch.zeros(7, dtype=torch.int32, device="cuda")
    assert M.mpm_box_bounds_noalloc(cell, 0, out) == M.ERR_NOMEM
