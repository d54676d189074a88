"""Seeded synthetic workloads for the box-restricted reaction-diffusion step.

This module holds geometry and random draws only: pleural-shell masks, Voronoi
tumour-cell labels, per-cell rate tables and initial fields.  It contains none of
the solver's arithmetic, so both the CUDA path and the CPU oracle may consume
what it produces.

The paper (Dolganov et al., arXiv 2505.03067) builds its domain from segmented
CT scans (Sec. 2.1) and seeds a cluster of epithelioid tumour cells in the
pleural space; neither the scans nor the model parameters are published.  These
generators stand in for them with the same structure: a thin shell between two
concentric ellipsoids (the pleural space), a clustered tumour made of Voronoi
"cells" (the CPM agents, cell id > 0, medium = 0), and per-cell uptake or
secretion rates.

Array convention (shared with the C ABI): a lattice of dims (Lx, Ly, Lz) is a
numpy array of shape (Lz, Ly, Lx) in C order, so the flat index of voxel
(i, j, k) is i + Lx*(j + Ly*k), x fastest.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MAX_SPECIES = 4


@dataclasses.dataclass
class Params:
    """Per-species physical parameters of Eq. 1-4.

    k_cell[s, id] is the first-order uptake rate of cell id for species s and
    q_cell[s, id] its zero-order source (secretion); index 0 is the medium.
    mu[s] is a uniform first-order decay (Eq. 3-4).
    """
    nspecies: int
    dt: float
    h: float
    D: np.ndarray        # [S] float64
    mu: np.ndarray       # [S] float64
    c_bc: np.ndarray     # [S] float64, Dirichlet value on box faces
    k_cell: np.ndarray   # [S, ncell] float64
    q_cell: np.ndarray   # [S, ncell] float64

    @property
    def ncell(self) -> int:
        return int(self.k_cell.shape[1])


@dataclasses.dataclass
class Lattice:
    """A CPM lattice with its fields (shape (Lz, Ly, Lx) per array)."""
    cell_id: np.ndarray           # int32
    mask: np.ndarray              # uint8, 1 = pleural space
    fields: np.ndarray            # float64 [S, Lz, Ly, Lx]
    dfac: np.ndarray | None = None  # optional float64 diffusivity factor per voxel

    @property
    def dims(self) -> tuple[int, int, int]:
        z, y, x = self.cell_id.shape
        return (x, y, z)

    def copy(self) -> "Lattice":
        return Lattice(self.cell_id.copy(), self.mask.copy(), self.fields.copy(),
                       None if self.dfac is None else self.dfac.copy())


@dataclasses.dataclass
class Workload:
    name: str
    lattice: Lattice
    params: Params
    margin: int
    steps: int
    rtol: float
    restart: int
    bc_box: int = 0          # 0 Dirichlet box faces, 1 zero flux


def _grid(dims):
    lx, ly, lz = dims
    z, y, x = np.meshgrid(np.arange(lz, dtype=np.float64), np.arange(ly, dtype=np.float64),
                          np.arange(lx, dtype=np.float64), indexing="ij")
    return x, y, z


def _voronoi_labels(points: np.ndarray, seeds: np.ndarray) -> np.ndarray:
    """Index of the nearest seed for each point (ties resolved by the k-d tree)."""
    from scipy.spatial import cKDTree
    _, idx = cKDTree(seeds).query(points, k=1)
    return idx.astype(np.int32)


def shell_mask(dims, center, outer, inner) -> np.ndarray:
    """Voxels inside the outer ellipsoid and outside the inner one (semi-axes in x,y,z)."""
    lx, ly, lz = dims
    cx, cy, cz = center
    zz = (np.arange(lz) - cz)[:, None, None]
    yy = (np.arange(ly) - cy)[None, :, None]
    xx = (np.arange(lx) - cx)[None, None, :]
    eo = (xx / outer[0]) ** 2 + (yy / outer[1]) ** 2 + (zz / outer[2]) ** 2 <= 1.0
    ei = (xx / inner[0]) ** 2 + (yy / inner[1]) ** 2 + (zz / inner[2]) ** 2 <= 1.0
    return (eo & ~ei).astype(np.uint8)


# --------------------------------------------------------------------------- c1
def sphere32(seed: int = 1, n: int = 32, radius: float = 8.0, ncells: int = 50) -> Workload:
    """Plain FP64 single-species case: 32^3 box, all voxels in the domain, a solid
    tumour sphere of radius 8 at the centre split into 50 Voronoi cells (ids 1..50),
    D = 1, dt = 0.1, uptake k = 0.05 on tumour, c0 = c_bc = 1, 10 steps, GMRES(30)
    to 1e-10.  The margin covers the whole lattice, so the box is 32^3."""
    rng = np.random.default_rng(seed)
    dims = (n, n, n)
    x, y, z = _grid(dims)
    c = (n - 1) / 2.0
    tumour = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2 <= radius * radius
    seeds = []
    while len(seeds) < ncells:
        p = rng.uniform(-radius, radius, size=3)
        if p @ p <= radius * radius:
            seeds.append(p + c)
    seeds = np.array(seeds)
    pts = np.stack([x[tumour], y[tumour], z[tumour]], axis=1)
    cell_id = np.zeros(x.shape, np.int32)
    cell_id[tumour] = _voronoi_labels(pts, seeds) + 1
    mask = np.ones(x.shape, np.uint8)
    fields = np.ones((1,) + x.shape, np.float64)
    k_cell = np.zeros((1, ncells + 1))
    k_cell[0, 1:] = 0.05
    params = Params(1, 0.1, 1.0, np.array([1.0]), np.array([0.0]), np.array([1.0]),
                    k_cell, np.zeros_like(k_cell))
    return Workload("sphere32", Lattice(cell_id, mask, fields), params, margin=n,
                    steps=10, rtol=1e-10, restart=30)


# --------------------------------------------------------------------------- c2
SHELL256_OUTER = (110.0, 90.0, 120.0)
SHELL256_INNER = (100.0, 80.0, 110.0)
SHELL256_REGION = ((128, 64, 80), (128, 128, 96))   # origin, size (x, y, z)


def three_species_params(rng, ncell: int, dt: float = 0.05, mu_cyt: float = 0.01) -> Params:
    """O2 and nutrient: per-cell uptake k ~ U[0.01, 0.1] on tumour; cytokine (IL6-like):
    uniform decay mu = 0.01 plus per-cell secretion q ~ U[0.01, 0.1] on tumour.
    D = (1, 0.5, 0.2); Dirichlet values (1, 1, 0)."""
    k = np.zeros((3, ncell + 1))
    q = np.zeros((3, ncell + 1))
    k[0, 1:] = rng.uniform(0.01, 0.1, ncell)
    k[1, 1:] = rng.uniform(0.01, 0.1, ncell)
    q[2, 1:] = rng.uniform(0.01, 0.1, ncell)
    return Params(3, dt, 1.0, np.array([1.0, 0.5, 0.2]), np.array([0.0, 0.0, mu_cyt]),
                  np.array([1.0, 1.0, 0.0]), k, q)


def shell256(seed: int = 2, ncells: int = 2000, n: int = 256) -> Workload:
    """Three species on a 256^3 lattice: pleural-shell mask between ellipsoids with
    semi-axes (110, 90, 120) and (100, 80, 110) centred at 127.5; about 2000 Voronoi
    tumour cells seeded in the shell inside the 128x128x96 region at (128, 64, 80)
    (every shell voxel of that region belongs to its nearest seed); bbox margin 4;
    dt = 0.05; 20 steps."""
    rng = np.random.default_rng(seed)
    dims = (n, n, n)
    c = (n - 1) / 2.0
    mask = shell_mask(dims, (c, c, c), SHELL256_OUTER, SHELL256_INNER)
    (ox, oy, oz), (sx, sy, sz) = SHELL256_REGION
    region = np.zeros(mask.shape, bool)
    region[oz:oz + sz, oy:oy + sy, ox:ox + sx] = True
    cand = np.flatnonzero((mask > 0) & region)
    zz, yy, xx = np.unravel_index(cand, mask.shape)
    pts = np.stack([xx, yy, zz], axis=1).astype(np.float64)
    pick = rng.choice(len(cand), size=ncells, replace=False)
    seeds = pts[pick] + rng.uniform(-0.5, 0.5, size=(ncells, 3))
    cell_id = np.zeros(mask.shape, np.int32)
    cell_id.reshape(-1)[cand] = _voronoi_labels(pts, seeds) + 1
    params = three_species_params(rng, ncells)
    fields = np.empty((3,) + mask.shape)
    fields[0] = 1.0
    fields[1] = 1.0
    fields[2] = 0.0
    return Workload("shell256", Lattice(cell_id, mask, fields), params, margin=4,
                    steps=20, rtol=1e-6, restart=30)


# --------------------------------------------------------------------------- c3
def patches(seed: int = 3, npatch: int = 64, lo: int = 16, hi: int = 96,
            mean_cell: float = 100.0) -> list[Workload]:
    """Independent pleural-shell patches for the batched solve: per-axis box dims
    drawn log-uniformly in [16, 96]; each patch is a crop of a 256^3 shell (as in
    shell256) centred on a random shell voxel, cut into Voronoi cells of ~100 voxels;
    whole cells become tumour in seeded order until a tumour occupancy drawn from
    U[5%, 40%] of the shell voxels is reached.  The margin covers the patch, so each
    box is the whole patch."""
    rng = np.random.default_rng(seed)
    n = 256
    c = (n - 1) / 2.0
    shell = shell_mask((n, n, n), (c, c, c), SHELL256_OUTER, SHELL256_INNER)
    shell_idx = np.flatnonzero(shell)
    out = []
    for p in range(npatch):
        d = np.exp(rng.uniform(math.log(lo), math.log(hi), size=3)).round().astype(int)
        d = np.clip(d, lo, hi)
        centre = np.array(np.unravel_index(shell_idx[rng.integers(len(shell_idx))], shell.shape))[::-1]
        o = np.clip(centre - d // 2, 0, n - d)
        crop = shell[o[2]:o[2] + d[2], o[1]:o[1] + d[1], o[0]:o[0] + d[0]].copy()
        cand = np.flatnonzero(crop)
        cell_id = np.zeros(crop.shape, np.int32)
        ncells = max(1, int(round(len(cand) / mean_cell)))
        zz, yy, xx = np.unravel_index(cand, crop.shape)
        pts = np.stack([xx, yy, zz], axis=1).astype(np.float64)
        pick = rng.choice(len(cand), size=ncells, replace=False)
        seeds = pts[pick] + rng.uniform(-0.5, 0.5, size=(ncells, 3))
        lab = _voronoi_labels(pts, seeds)
        occ = rng.uniform(0.05, 0.40)
        sizes = np.bincount(lab, minlength=ncells)
        tum = np.zeros(ncells, bool)
        acc = 0
        for cidx in rng.permutation(ncells):
            if acc >= occ * len(cand):
                break
            tum[cidx] = True
            acc += sizes[cidx]
        ids = np.zeros(ncells, np.int32)
        ids[tum] = np.arange(1, int(tum.sum()) + 1, dtype=np.int32)
        cell_id.reshape(-1)[cand] = ids[lab]
        ncell_t = int(tum.sum())
        params = three_species_params(rng, ncell_t)
        fields = np.empty((3,) + crop.shape)
        fields[0] = 1.0
        fields[1] = 1.0
        fields[2] = 0.0
        out.append(Workload(f"patch{p}", Lattice(cell_id, crop.astype(np.uint8), fields), params,
                            margin=int(max(d)), steps=50, rtol=1e-6, restart=30))
    return out


# --------------------------------------------------------------------------- c5
GROWTH_DIMS = (512, 384, 384)
GROWTH_OUTER = (230.0, 175.0, 175.0)
GROWTH_INNER = (215.0, 160.0, 160.0)
GROWTH_FINAL = ((192, 64, 64), (320, 256, 256))      # origin, size (x, y, z)


def growth_box(t: int, steps: int = 200):
    """Box (lo, hi) of the growth front at step t: linear from a 64^3 box centred on
    the +x cap of the shell to the final 320x256x256 region over `steps` steps."""
    (fx, fy, fz), (sx, sy, sz) = GROWTH_FINAL
    flo = np.array([fx, fy, fz], float)
    fhi = flo + np.array([sx, sy, sz], float)
    cap = np.array([(GROWTH_DIMS[0] - 1) / 2.0 + 0.5 * (GROWTH_OUTER[0] + GROWTH_INNER[0]),
                    (GROWTH_DIMS[1] - 1) / 2.0, (GROWTH_DIMS[2] - 1) / 2.0])
    ilo = cap - 32.0
    ihi = cap + 32.0
    shift = np.minimum(0.0, fhi - ihi)       # keep the initial box inside the final region
    ilo, ihi = ilo + shift, ihi + shift
    a = min(1.0, max(0.0, t / float(steps)))
    return ilo + a * (flo - ilo), ihi + a * (fhi - ihi)


def growth512(seed: int = 5, mean_cell: float = 200.0, dims=GROWTH_DIMS):
    """Full growing tumour on a 512x384x384 lattice: shell mask between ellipsoids
    (230,175,175)/(215,160,160); Voronoi cells over the shell inside the final
    320x256x256 region; returns (workload at t=0, seed positions, cell labels of the
    candidate voxels, candidate voxel indices).  `grow(wl, t, extra)` re-labels which
    cells are tumour at step t."""
    rng = np.random.default_rng(seed)
    lx, ly, lz = dims
    mask = shell_mask(dims, ((lx - 1) / 2.0, (ly - 1) / 2.0, (lz - 1) / 2.0), GROWTH_OUTER, GROWTH_INNER)
    (ox, oy, oz), (sx, sy, sz) = GROWTH_FINAL
    region = np.zeros(mask.shape, bool)
    region[oz:oz + sz, oy:oy + sy, ox:ox + sx] = True
    cand = np.flatnonzero((mask > 0) & region)
    zz, yy, xx = np.unravel_index(cand, mask.shape)
    pts = np.stack([xx, yy, zz], axis=1).astype(np.float64)
    ncells = max(1, int(round(len(cand) / mean_cell)))
    pick = rng.choice(len(cand), size=ncells, replace=False)
    seeds = pts[pick] + rng.uniform(-0.5, 0.5, size=(ncells, 3))
    lab = _voronoi_labels(pts, seeds)
    params = three_species_params(rng, ncells)
    fields = np.empty((3,) + mask.shape)
    fields[0] = 1.0
    fields[1] = 1.0
    fields[2] = 0.0
    wl = Workload("growth512", Lattice(np.zeros(mask.shape, np.int32), mask, fields), params,
                  margin=4, steps=200, rtol=1e-6, restart=30)
    extra = {"seeds": seeds, "labels": lab, "cand": cand}
    grow(wl, 0, extra)
    return wl, extra


def growth_crop(seed: int = 6, mean_cell: float = 200.0):
    """Another instance of the growing-tumour geometry (another seed: other
    Voronoi cells and rates) cut to its final growth region plus the margin,
    324x264x264 voxels: every step's bounding box lies inside the crop and is
    the full 512x384x384 lattice's box moved by the crop origin (the tumour
    never comes nearer a crop face than the margin, except at the lattice's
    own +x face, which the crop keeps).  Returns (workload, extra) like
    growth512; extra["cand"] indexes the crop.  This is the learned warm
    start's training trajectory for the growing tumour."""
    wl, extra = growth512(seed=seed, mean_cell=mean_cell)
    (fx, fy, fz), (sx, sy, sz) = GROWTH_FINAL
    m = wl.margin
    lx, ly, lz = GROWTH_DIMS
    lo = (max(0, fx - m), max(0, fy - m), max(0, fz - m))
    hi = (min(lx, fx + sx + m), min(ly, fy + sy + m), min(lz, fz + sz + m))
    sl = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
    lat = wl.lattice
    crop = Lattice(np.ascontiguousarray(lat.cell_id[sl]), np.ascontiguousarray(lat.mask[sl]),
                   np.ascontiguousarray(lat.fields[(slice(None),) + sl]))
    zz, yy, xx = np.unravel_index(extra["cand"], lat.cell_id.shape)
    nx, ny = hi[0] - lo[0], hi[1] - lo[1]
    cand = ((zz - lo[2]) * ny + (yy - lo[1])) * nx + (xx - lo[0])
    seeds = extra["seeds"] - np.array(lo, float)
    cw = Workload("growth_crop", crop, wl.params, margin=m, steps=wl.steps, rtol=wl.rtol, restart=wl.restart)
    return cw, {"seeds": seeds, "labels": extra["labels"], "cand": cand, "origin": lo}


def grow(wl: Workload, t: int, extra) -> None:
    """Mark as tumour (id = cell index + 1) every cell whose seed lies in growth_box(t)."""
    lo, hi = growth_box(t, wl.steps)
    if "origin" in extra:
        lo, hi = lo - np.array(extra["origin"], float), hi - np.array(extra["origin"], float)
    s = extra["seeds"]
    inside = np.all((s >= lo) & (s < hi), axis=1)
    ids = np.where(inside, np.arange(1, len(s) + 1, dtype=np.int32), 0).astype(np.int32)
    cid = wl.lattice.cell_id.reshape(-1)
    cid[extra["cand"]] = ids[extra["labels"]]


# --------------------------------------------------------------------------- small cases
def random_case(seed: int, dims, nspecies: int = 3, p_mask: float = 0.8, p_tumour: float = 0.3,
                ncell: int = 7, dfac: bool = False, blob: bool = True) -> Workload:
    """Small random lattice for parity tests: random mask (optionally a blob so that
    the mask is mostly connected), random cell ids, random fields and rate tables."""
    rng = np.random.default_rng(seed)
    lx, ly, lz = dims
    shape = (lz, ly, lx)
    if blob:
        x, y, z = _grid(dims)
        c = np.array([(lx - 1) / 2, (ly - 1) / 2, (lz - 1) / 2])
        r = np.sqrt(((x - c[0]) / max(lx, 1)) ** 2 + ((y - c[1]) / max(ly, 1)) ** 2
                    + ((z - c[2]) / max(lz, 1)) ** 2)
        mask = ((r < 0.45) | (rng.random(shape) < p_mask * 0.5)).astype(np.uint8)
    else:
        mask = (rng.random(shape) < p_mask).astype(np.uint8)
    cell_id = np.where(rng.random(shape) < p_tumour, rng.integers(1, ncell, size=shape), 0).astype(np.int32)
    fields = rng.uniform(0.0, 2.0, size=(nspecies,) + shape)
    k = np.zeros((nspecies, ncell))
    q = np.zeros((nspecies, ncell))
    k[:, 1:] = rng.uniform(0.0, 0.5, size=(nspecies, ncell - 1))
    q[:, 1:] = rng.uniform(0.0, 0.5, size=(nspecies, ncell - 1))
    params = Params(nspecies, float(rng.uniform(0.05, 0.5)), 1.0,
                    rng.uniform(0.1, 2.0, nspecies), rng.uniform(0.0, 0.1, nspecies),
                    rng.uniform(0.0, 2.0, nspecies), k, q)
    df = rng.uniform(0.2, 3.0, size=shape) if dfac else None
    return Workload(f"random{seed}", Lattice(cell_id, mask, fields, df), params, margin=1,
                    steps=2, rtol=1e-12, restart=30)


# --------------------------------------------------------------------------- learned warm start
def sphere_training_case(rng, n: int = 32, three_species=None, homogeneous: bool = False) -> Workload:
    """A 32^3 training lattice around the 32^3 sphere workload: every voxel in the
    domain, a solid tumour sphere of radius U[4, 12] at a random centre split into
    ~50 Voronoi cells; species 0 as in the sphere workload (D = 1, dt = 0.1,
    c0 = c_b = 1) with per-cell uptake U[0.01, 0.1].  Species 1-2 either carry the
    shell workload's nutrient and cytokine (D 0.5 / 0.2, per-cell uptake /
    secretion U[0.01, 0.1], cytokine decay 0.01, c_b 1 / 0) or are absent (all
    zero), as in the single-species workload.  homogeneous: the same operators
    with every boundary value and source at zero and one species, drawn at
    random, carrying three Gaussian bumps (centres uniform, widths U[2, 8],
    amplitudes U[-1, 1]) while the others are zero -- the next step is then
    A^-1 applied to that field, the map the network approximates as a
    preconditioner."""
    dims = (n, n, n)
    x, y, z = _grid(dims)
    r = rng.uniform(4.0, 12.0)
    c = rng.uniform(r * 0.5, n - 1 - r * 0.5, size=3)
    tumour = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 <= r * r
    if not tumour.any():
        tumour[int(c[2]), int(c[1]), int(c[0])] = True
    pts = np.stack([x[tumour], y[tumour], z[tumour]], axis=1)
    ncells = max(1, min(50, len(pts)))
    seeds = pts[rng.choice(len(pts), ncells, replace=False)] + rng.uniform(-0.5, 0.5, (ncells, 3))
    cell_id = np.zeros(x.shape, np.int32)
    cell_id[tumour] = _voronoi_labels(pts, seeds) + 1
    three = bool(rng.random() < 0.5) if three_species is None else three_species
    k = np.zeros((3, ncells + 1))
    q = np.zeros((3, ncells + 1))
    k[0, 1:] = rng.uniform(0.01, 0.1, ncells)
    fields = np.zeros((3,) + x.shape)
    fields[0] = 1.0
    if three:
        k[1, 1:] = rng.uniform(0.01, 0.1, ncells)
        q[2, 1:] = rng.uniform(0.01, 0.1, ncells)
        fields[1] = 1.0
        params = Params(3, 0.1, 1.0, np.array([1.0, 0.5, 0.2]), np.array([0.0, 0.0, 0.01]),
                        np.array([1.0, 1.0, 0.0]), k, q)
    else:
        params = Params(3, 0.1, 1.0, np.array([1.0, 1.0, 1.0]), np.zeros(3), np.array([1.0, 0.0, 0.0]), k, q)
    if homogeneous:
        sp = int(rng.integers(0, 3 if three else 1))
        fields = np.zeros((3,) + x.shape)
        for _ in range(3):
            cc = rng.uniform(0, n - 1, size=3)
            w = rng.uniform(2.0, 8.0)
            fields[sp] += rng.uniform(-1.0, 1.0) * np.exp(-((x - cc[0]) ** 2 + (y - cc[1]) ** 2 + (z - cc[2]) ** 2)
                                                         / (2 * w * w))
        params = Params(3, params.dt, params.h, params.D, params.mu, np.zeros(3), params.k_cell, np.zeros_like(q))
    return Workload("sphere_train", Lattice(cell_id, np.ones(x.shape, np.uint8), fields), params, margin=n,
                    steps=10, rtol=1e-10, restart=30)


def with_capacity(params: Params, capacity: int) -> Params:
    """The same parameters with rate tables of `capacity` entries per species
    (new entries zero): room for the daughters of the growth driver."""
    S, n = params.k_cell.shape
    if capacity < n:
        raise ValueError("capacity below the current table size")
    k = np.zeros((S, capacity))
    q = np.zeros((S, capacity))
    k[:, :n] = params.k_cell
    q[:, :n] = params.q_cell
    return dataclasses.replace(params, k_cell=k, q_cell=q)
