"""Pins of the growth driver's oracle (oracle.cpm_step; no GPU).

The generator is SplitMix64's published output sequence; the vectorised step
equals the voxel-by-voxel transcription of the rules; closed forms fix the
growth rule (p = 0: nothing; p >= 1: one layer of 6-neighbour dilation inside
the mask; hypoxia: nothing), mitosis (a brick splits into two equal halves
along the drawn axis, the daughter takes the next id and the parent's rates,
no room in the tables: no division) and the growth probability (binomial
frequency on a large interface).  A wrong neighbour order, a flipped
comparison, a centroid off by one or a dropped mask fails one of them.
"""
import numpy as np
import pytest

import oracle

CP = {"p_grow": 0.6, "K_o2": 0.2, "K_nut": 0.3, "o2_min": 0.05, "v_div": 40}


def test_generator_is_splitmix64():
    # SplitMix64 from state 1234567: its first five outputs (Steele, Lea and
    # Flood 2014; the sequence every implementation of it reproduces)
    got = oracle.cpm_draw(1234567, 0, 0, np.arange(5)).tolist()
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
                   16408922859458223821]
    # streams and steps draw other words
    a = oracle.cpm_draw(7, 3, 0, np.arange(1000))
    b = oracle.cpm_draw(7, 3, 1, np.arange(1000))
    c = oracle.cpm_draw(7, 4, 0, np.arange(1000))
    assert len(set(a.tolist()) | set(b.tolist()) | set(c.tolist())) == 3000
    u = (oracle.cpm_draw(11, 0, 0, np.arange(200000)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)


def _case(seed, dims=(7, 6, 9), ncell=6, cap=12):
    rng = np.random.default_rng(seed)
    Lz, Ly, Lx = dims
    cell = np.zeros(dims, np.int32)
    blob = rng.random(dims) < 0.35
    cell[blob] = rng.integers(1, ncell, size=int(blob.sum()))
    mask = (rng.random(dims) < 0.85).astype(np.uint8)
    mask[cell > 0] = 1
    o2 = rng.uniform(0.0, 1.0, dims)
    nut = rng.uniform(0.0, 1.0, dims)
    k = np.zeros((3, cap))
    q = np.zeros((3, cap))
    k[:, 1:ncell] = rng.uniform(0.01, 0.1, (3, ncell - 1))
    q[:, 1:ncell] = rng.uniform(0.01, 0.1, (3, ncell - 1))
    return cell, mask, o2, nut, k, q, ncell


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_vectorised_step_equals_the_voxel_loops(seed):
    cell, mask, o2, nut, k, q, nc = _case(seed)
    cp = dict(CP, v_div=6)
    for step in range(3):
        a = oracle.cpm_step(cell, mask, o2, nut, k, q, nc, cp, 99 + seed, step)
        b = oracle.cpm_step_loops(cell, mask, o2, nut, k, q, nc, cp, 99 + seed, step)
        assert np.array_equal(a[0], b[0]) and a[3] == b[3] and a[4] == b[4]
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
        cell, k, q, nc = a[0], a[1], a[2], a[3]
    assert nc > 6   # divisions happened


def test_no_growth_at_zero_probability_or_hypoxia():
    cell, mask, o2, nut, k, q, nc = _case(4)
    big = dict(CP, v_div=10 ** 9)
    out, _, _, n2, st = oracle.cpm_step(cell, mask, o2, nut, k, q, nc, dict(big, p_grow=0.0), 5, 0)
    assert np.array_equal(out, cell) and st["grown"] == 0 and n2 == nc
    out, _, _, _, st = oracle.cpm_step(cell, mask, np.full_like(o2, 0.01), nut, k, q, nc, dict(big, p_grow=5.0), 5, 0)
    assert np.array_equal(out, cell) and st["grown"] == 0


def test_certain_growth_is_one_dilation_inside_the_mask():
    cell, mask, o2, nut, k, q, nc = _case(5)
    o2 = np.full_like(o2, 1.0)
    nut = np.full_like(nut, 1.0)
    cp = dict(CP, p_grow=10.0, v_div=10 ** 9)   # p > 1 wherever the rule allows growth
    out, _, _, _, st = oracle.cpm_step(cell, mask, o2, nut, k, q, nc, cp, 6, 0)
    t = cell > 0
    dil = t.copy()
    dil[:, :, 1:] |= t[:, :, :-1]
    dil[:, :, :-1] |= t[:, :, 1:]
    dil[:, 1:, :] |= t[:, :-1, :]
    dil[:, :-1, :] |= t[:, 1:, :]
    dil[1:, :, :] |= t[:-1, :, :]
    dil[:-1, :, :] |= t[1:, :, :]
    want = t | (dil & (mask > 0))
    assert np.array_equal(out > 0, want)
    assert st["grown"] == int(want.sum() - t.sum())
    # every new voxel took the id of one of its tumour neighbours
    nb = oracle._nbr_ids(cell)
    new = (out > 0) & ~t
    assert np.all(np.any(nb[:, new] == out[new][None], axis=0))


def test_brick_divides_into_equal_halves_along_the_drawn_axis():
    dims = (10, 9, 11)
    cell = np.zeros(dims, np.int32)
    cell[2:6, 3:9, 1:9] = 1           # 8 (x) x 6 (y) x 4 (z) = 192 voxels
    mask = np.ones(dims, np.uint8)
    k = np.zeros((3, 4))
    q = np.zeros((3, 4))
    k[:, 1] = [0.01, 0.02, 0.03]
    q[:, 1] = [0.04, 0.05, 0.06]
    cp = dict(CP, p_grow=0.0, v_div=192)
    seen = set()
    for step in range(12):
        out, k2, q2, nc, st = oracle.cpm_step(cell, mask, np.ones(dims), np.ones(dims), k, q, 2, cp, 3, step)
        assert nc == 3 and st["divisions"] == 1
        assert np.sum(out == 1) == 96 and np.sum(out == 2) == 96
        assert np.array_equal(k2[:, 2], k[:, 1]) and np.array_equal(q2[:, 2], q[:, 1])
        z, y, x = np.nonzero(out == 2)
        axis = [a for a, c in enumerate((x, y, z)) if np.ptp(c) < np.ptp(np.nonzero(cell)[2 - a])]
        assert len(axis) == 1
        a = axis[0]
        lo = (1, 3, 2)[a]
        ext = (8, 6, 4)[a]
        assert np.min((x, y, z)[a]) == lo + ext // 2      # strictly above the centroid
        seen.add(a)
    assert seen == {0, 1, 2}
    # a full table: no division
    out, _, _, nc, st = oracle.cpm_step(cell, mask, np.ones(dims), np.ones(dims), k[:, :2], q[:, :2], 2, cp, 3, 0)
    assert nc == 2 and st["divisions"] == 0 and np.array_equal(out, cell)


def test_growth_frequency_is_the_probability():
    dims = (40, 64, 64)
    cell = np.zeros(dims, np.int32)
    cell[:20] = 1
    mask = np.ones(dims, np.uint8)
    o2 = np.full(dims, 0.6)
    nut = np.full(dims, 0.9)
    cp = dict(CP, v_div=10 ** 9)
    p = cp["p_grow"] * (0.6 / (cp["K_o2"] + 0.6)) * (0.9 / (cp["K_nut"] + 0.9))
    out, _, _, _, st = oracle.cpm_step(cell, mask, o2, nut, np.zeros((3, 2)), np.zeros((3, 2)), 2, cp, 8, 0)
    n = 64 * 64     # the layer z = 20
    assert np.all(out[21:] == 0) and st["grown"] == int(np.sum(out[20] > 0))
    assert abs(st["grown"] / n - p) <= 5 * np.sqrt(p * (1 - p) / n)
