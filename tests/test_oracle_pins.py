"""Pins of the CPU oracle against what the mathematics fixes (no GPU).

Every check here comes from outside the oracle: closed-form eigenmodes of the
discrete operator, exact steady states, conservation and maximum-principle
invariants, brute force on tiny lattices, and library routines for the special
cases that reduce to them.  A dropped term, a wrong sign, a wrong face weight
or a transposed index in oracle.c fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2505_03067_gb300 import workloads as W


def _params(S=1, dt=0.1, h=1.0, D=1.0, mu=0.0, c_bc=0.0, k=None, q=None, ncell=2):
    kk = np.zeros((S, ncell)) if k is None else np.asarray(k, float).reshape(S, ncell)
    qq = np.zeros((S, ncell)) if q is None else np.asarray(q, float).reshape(S, ncell)
    return W.Params(S, dt, h, np.full(S, D, float), np.full(S, mu, float), np.full(S, c_bc, float), kk, qq)


def _solve(mask, cell, c, params, s=0, bc_box=0, dfac=None, lu=False, tol=1e-14):
    A, b = oracle.assemble(mask, cell, c, params, s, bc_box, dfac)
    if lu:
        return oracle.dense_solve(A, b).reshape(c.shape)
    x, info = oracle.gmres(A, b, c, 30, tol * max(1.0, float(np.linalg.norm(b))), 5000)
    assert info["status"] == oracle.OK
    return x.reshape(c.shape)


def _mode(n, a, kind):
    """Separable discrete mode on a box of dims n=(nx,ny,nz): product over axes of
    sin(a pi (i+1/2)/n) (Dirichlet at half-cell faces, DST-II) or cos(...) (zero flux)."""
    f = np.sin if kind == "sin" else np.cos
    vx = f(a[0] * np.pi * (np.arange(n[0]) + 0.5) / n[0])
    vy = f(a[1] * np.pi * (np.arange(n[1]) + 0.5) / n[1])
    vz = f(a[2] * np.pi * (np.arange(n[2]) + 0.5) / n[2])
    return vz[:, None, None] * vy[None, :, None] * vx[None, None, :]


def _lam(n, a, h):
    return 4.0 / h ** 2 * sum(math.sin(ad * math.pi / (2 * nd)) ** 2 for ad, nd in zip(a, n))


# ---------------------------------------------------------------- closed-form eigenmodes
@pytest.mark.parametrize("n,a,h,D,dt", [((6, 5, 4), (1, 1, 1), 1.0, 1.0, 0.1),
                                         ((6, 5, 4), (3, 2, 4), 1.0, 0.7, 0.3),
                                         ((8, 8, 8), (8, 1, 5), 0.5, 1.3, 0.05),
                                         ((7, 3, 1), (2, 3, 1), 2.0, 0.2, 1.0)])
def test_dirichlet_eigenmode_decays_by_closed_form(n, a, h, D, dt):
    """With c_bc = 0 on every box face, every voxel in the mask and no reaction, the
    DST-II mode u is an eigenvector: c^{n+1} = u / (1 + dt D lambda),
    lambda = (4/h^2) sum_d sin^2(a_d pi / (2 n_d))."""
    shape = (n[2], n[1], n[0])
    u = _mode(n, a, "sin")
    p = _params(dt=dt, h=h, D=D)
    x = _solve(np.ones(shape, np.uint8), np.zeros(shape, np.int32), u, p)
    expect = u / (1.0 + dt * D * _lam(n, a, h))
    assert np.max(np.abs(x - expect)) < 1e-12
    x2 = _solve(np.ones(shape, np.uint8), np.zeros(shape, np.int32), u, p, lu=True)
    assert np.max(np.abs(x2 - expect)) < 1e-12


@pytest.mark.parametrize("n,a", [((6, 5, 4), (1, 2, 3)), ((5, 5, 5), (0, 4, 1)), ((9, 2, 3), (8, 1, 0))])
def test_zero_flux_eigenmode_decays_by_closed_form(n, a):
    """With zero flux on every box face (bc_box = 1) the DCT-II mode cos(a pi (i+1/2)/n)
    is an eigenvector with the same lambda."""
    shape = (n[2], n[1], n[0])
    u = _mode(n, a, "cos")
    p = _params(dt=0.2, D=0.9, c_bc=123.0)   # c_bc must not matter with zero flux
    x = _solve(np.ones(shape, np.uint8), np.zeros(shape, np.int32), u, p, bc_box=1)
    assert np.max(np.abs(x - u / (1.0 + 0.2 * 0.9 * _lam(n, a, 1.0)))) < 1e-12


def test_affine_dirichlet_mode():
    """c_bc = 1 and c = 1 + eps u: the constant part is the steady state and the mode
    decays as before, so c^{n+1} = 1 + eps u / (1 + dt D lambda) (pins the Dirichlet
    right-hand side 2 D c_bc at half-cell faces)."""
    n, a = (6, 7, 5), (2, 1, 3)
    shape = (n[2], n[1], n[0])
    u = _mode(n, a, "sin")
    p = _params(dt=0.25, D=1.1, c_bc=1.0)
    x = _solve(np.ones(shape, np.uint8), np.zeros(shape, np.int32), 1.0 + 0.3 * u, p)
    assert np.max(np.abs(x - (1.0 + 0.3 * u / (1.0 + 0.25 * 1.1 * _lam(n, a, 1.0))))) < 1e-12


def test_mode_decay_over_steps_through_step_driver():
    """Ten implicit-Euler steps through the full step driver (bbox, gather, solve,
    scatter): the mode decays by (1 + dt D lambda)^-10."""
    n, a = (10, 9, 8), (1, 2, 1)
    shape = (n[2], n[1], n[0])
    u = _mode(n, a, "sin")
    lat = W.Lattice(np.ones(shape, np.int32), np.ones(shape, np.uint8), u[None].copy())
    p = _params(dt=0.1, D=1.0, ncell=2)
    for _ in range(10):
        rep = oracle.step(lat, p, margin=20, rtol=0.0, atol=1e-14)
        assert rep["status"] == oracle.OK
    assert np.max(np.abs(lat.fields[0] - u * (1.0 + 0.1 * _lam(n, a, 1.0)) ** -10)) < 1e-12


# ---------------------------------------------------------------- exact steady state with uptake
@pytest.mark.parametrize("nx,k,D,h", [(12, 0.05, 1.0, 1.0), (9, 0.3, 0.5, 2.0), (20, 1.0, 0.2, 1.0)])
def test_uptake_steady_state_1d(nx, k, D, h):
    """A 1D chain (the centre line of an nx x 3 x 3 box whose other voxels are masked,
    so its y/z faces carry no flux) with Dirichlet x ends and uniform uptake k.  The
    discrete steady state is c_i = cosh(theta (i - m)), cosh(theta) = 1 + k h^2/(2D),
    m = (nx-1)/2, with the boundary value fixed by the half-cell ghost
    c_bc = (c_{-1} + c_0)/2.  From that state one step with any dt changes nothing."""
    th = math.acosh(1.0 + k * h * h / (2.0 * D))
    m = (nx - 1) / 2.0
    prof = np.cosh(th * (np.arange(nx) - m))
    c_bc = 0.5 * (math.cosh(th * (-1 - m)) + math.cosh(th * (0 - m)))
    shape = (3, 3, nx)
    mask = np.zeros(shape, np.uint8)
    mask[1, 1, :] = 1
    cell = np.zeros(shape, np.int32)
    cell[1, 1, :] = 1
    c = np.full(shape, 7.0)
    c[1, 1, :] = prof
    for dt in (0.01, 1.0, 1e3):
        p = _params(dt=dt, h=h, D=D, c_bc=c_bc, k=[0.0, k])
        x = _solve(mask, cell, c, p, lu=True)
        assert np.max(np.abs(x[1, 1, :] - prof)) < 1e-10 * prof.max()
        assert np.all(x[mask == 0] == 7.0)          # masked voxels keep c^n exactly


# ---------------------------------------------------------------- harmonic-mean face diffusivity
@pytest.mark.parametrize("d1,d2", [(1.0, 1.0), (1.0, 3.0), (0.2, 5.0)])
def test_two_voxel_series_conductance(d1, d2):
    """Two voxels with zero flux elsewhere exchange mass through one face whose
    conductance is that of two half-cells in series, 1/(h/(2 D1) + h/(2 D2)).
    Total mass is kept and the difference decays by 1/(1 + 2 (dt/h) G)."""
    h, dt, D0 = 1.5, 0.4, 0.8
    G = 1.0 / (h / (2 * D0 * d1) + h / (2 * D0 * d2))
    shape = (1, 1, 2)
    c = np.array([[[1.0, 0.25]]])
    p = _params(dt=dt, h=h, D=D0)
    x = _solve(np.ones(shape, np.uint8), np.zeros(shape, np.int32), c, p, bc_box=1,
               dfac=np.array([[[d1, d2]]]), lu=True)
    assert abs(x.sum() - c.sum()) < 1e-14
    assert abs((x[0, 0, 0] - x[0, 0, 1]) - 0.75 / (1.0 + 2.0 * dt / h * G)) < 1e-14


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_uniform_field_is_invariant(seed):
    """c = c0 with no reaction stays c0 (to 1e-14) with zero flux on the box, with
    Dirichlet c_bc = c0, with any mask and any diffusivity factor."""
    rng = np.random.default_rng(seed)
    shape = (5, 6, 7)
    mask = (rng.random(shape) < 0.7).astype(np.uint8)
    dfac = rng.uniform(0.1, 4.0, shape)
    c0 = 0.37
    c = np.full(shape, c0)
    for bc_box in (0, 1):
        p = _params(dt=0.5, D=1.7, c_bc=c0)
        x = _solve(mask, np.zeros(shape, np.int32), c, p, bc_box=bc_box, dfac=dfac)
        assert np.max(np.abs(x - c0)) < 1e-14


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_mass_balance_zero_flux(seed):
    """With zero flux at every box and mask face, the total change over the mask is
    exactly dt times the net source: sum(c^{n+1} - c^n) = dt sum(q - k c^{n+1}),
    k including the uniform decay mu."""
    rng = np.random.default_rng(seed)
    shape = (6, 5, 8)
    mask = (rng.random(shape) < 0.75).astype(np.uint8)
    ncell = 5
    cell = rng.integers(0, ncell, shape).astype(np.int32)
    k = rng.uniform(0, 0.4, ncell)
    q = rng.uniform(0, 0.6, ncell)
    mu = 0.07
    dt = 0.3
    c = rng.uniform(0, 2, shape)
    p = _params(dt=dt, D=0.9, mu=mu, k=k, q=q, ncell=ncell)
    x = _solve(mask, cell, c, p, bc_box=1, dfac=rng.uniform(0.3, 2.0, shape))
    m = mask > 0
    lhs = np.sum(x[m] - c[m])
    rhs = dt * np.sum(q[cell[m]] - (k[cell[m]] + mu) * x[m])
    assert abs(lhs - rhs) < 1e-12
    assert np.all(x[~m] == c[~m])


def test_mass_balance_dirichlet_boundary_flux():
    """Dirichlet variant: the change also includes the flux through box faces,
    dt * sum over box-face voxels and faces of 2 D (c_bc - c^{n+1}_P) / h^2."""
    rng = np.random.default_rng(7)
    n = (5, 4, 6)
    shape = (n[2], n[1], n[0])
    c = rng.uniform(0, 2, shape)
    dt, D, h, cb = 0.2, 0.6, 1.0, 1.3
    p = _params(dt=dt, D=D, h=h, c_bc=cb)
    x = _solve(np.ones(shape, np.uint8), np.zeros(shape, np.int32), c, p)
    nf = np.zeros(shape)
    nf[:, :, 0] += 1; nf[:, :, -1] += 1
    nf[:, 0, :] += 1; nf[:, -1, :] += 1
    nf[0, :, :] += 1; nf[-1, :, :] += 1
    flux = np.sum(nf * 2 * D * (cb - x) / h ** 2)
    assert abs(np.sum(x - c) - dt * flux) < 1e-12


@pytest.mark.parametrize("seed", [0, 1])
def test_maximum_principle(seed):
    """A is an M-matrix: with q = 0 and non-negative data,
    0 <= c^{n+1} <= max(max c^n, c_bc)."""
    rng = np.random.default_rng(seed)
    shape = (7, 6, 5)
    mask = (rng.random(shape) < 0.8).astype(np.uint8)
    c = rng.uniform(0, 1, shape)
    k = rng.uniform(0, 0.5, 4)
    for cb in (0.0, 0.5, 3.0):
        p = _params(dt=0.7, D=1.2, c_bc=cb, k=k, ncell=4)
        x = _solve(mask, rng.integers(0, 4, shape).astype(np.int32), c, p)
        assert x.min() >= -1e-12
        assert x.max() <= max(c.max(), cb) + 1e-12


def test_operator_is_symmetric_m_matrix():
    """A is symmetric, has a positive diagonal, non-positive off-diagonals and
    lambda_min >= 1 (diffusion part PSD, k >= 0)."""
    wl = W.random_case(5, (5, 4, 6), nspecies=1, dfac=True)
    box = oracle.bbox(wl.lattice.cell_id, 2)
    args = [oracle.box_view(a, box) for a in (wl.lattice.mask, wl.lattice.cell_id, wl.lattice.fields[0])]
    A, _ = oracle.assemble(*args, wl.params, 0, 0, oracle.box_view(wl.lattice.dfac, box))
    M = A.dense()
    assert np.array_equal(M, M.T)
    off = M - np.diag(np.diag(M))
    assert np.all(off <= 0) and np.all(np.diag(M) > 0)
    assert np.linalg.eigvalsh(M).min() >= 1.0 - 1e-12


# ---------------------------------------------------------------- special cases = library routines
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_dense_lu_matches_numpy_and_gmres(seed):
    """The oracle's dense LU agrees with numpy.linalg.solve on the same matrix, and
    restarted GMRES (restart 30 and restart 3) agrees with the LU within the
    residual bound ||x - x*||_inf <= ||A^-1||_2 ||r||_2 <= ||r||_2."""
    wl = W.random_case(seed, (8, 7, 8), nspecies=1, dfac=(seed == 2))
    box = oracle.bbox(wl.lattice.cell_id, 1)
    mb, cb_, fb = (oracle.box_view(a, box) for a in (wl.lattice.mask, wl.lattice.cell_id, wl.lattice.fields[0]))
    dfb = None if wl.lattice.dfac is None else oracle.box_view(wl.lattice.dfac, box)
    A, b = oracle.assemble(mb, cb_, fb, wl.params, 0, 0, dfb)
    assert A.N <= 512
    x_lu = oracle.dense_solve(A, b)
    x_np = np.linalg.solve(A.dense(), b.reshape(-1))
    assert np.max(np.abs(x_lu - x_np)) < 1e-13
    for m in (30, 3):
        x, info = oracle.gmres(A, b, fb, m, 1e-13, 10000)
        assert info["status"] == oracle.OK and info["res"] <= 1e-13
        assert np.max(np.abs(x - x_lu)) <= 1e-13 + 1e-14


def test_gmres_maxit_reports_noconv():
    wl = W.random_case(3, (6, 6, 6), nspecies=1)
    box = oracle.bbox(wl.lattice.cell_id, 1)
    mb, cb_, fb = (oracle.box_view(a, box) for a in (wl.lattice.mask, wl.lattice.cell_id, wl.lattice.fields[0]))
    A, b = oracle.assemble(mb, cb_, fb, wl.params, 0)
    x, info = oracle.gmres(A, b, fb, 30, 1e-14, 1)
    assert info["status"] == oracle.ERR_NOCONV and info["iters"] == 1


# ---------------------------------------------------------------- bbox / gather / scatter by brute force
def _bbox_brute(cell, margin):
    Lz, Ly, Lx = cell.shape
    lo = [None, None, None]
    hi = [None, None, None]
    for k in range(Lz):
        for j in range(Ly):
            for i in range(Lx):
                if cell[k, j, i] > 0:
                    for d, v in enumerate((i, j, k)):
                        lo[d] = v if lo[d] is None else min(lo[d], v)
                        hi[d] = v if hi[d] is None else max(hi[d], v)
    if lo[0] is None:
        return None
    L = (Lx, Ly, Lz)
    return (tuple(max(0, lo[d] - margin) for d in range(3)),
            tuple(min(L[d], hi[d] + margin + 1) for d in range(3)))


@pytest.mark.parametrize("seed", range(6))
def test_bbox_brute_force(seed):
    rng = np.random.default_rng(seed)
    shape = tuple(int(v) for v in rng.integers(1, 17, 3))
    cases = [np.zeros(shape, np.int32),                         # empty
             np.where(rng.random(shape) < 0.05, 3, 0).astype(np.int32),
             np.ones(shape, np.int32),                          # full lattice
             np.where(rng.random(shape) < 0.5, -1, 0).astype(np.int32)]  # negative ids are not tumour
    one = np.zeros(shape, np.int32)
    one[tuple(int(rng.integers(0, s)) for s in shape)] = 9      # single voxel
    cases.append(one)
    for cell in cases:
        for margin in (0, 1, 3, 40):
            assert oracle.bbox(cell, margin) == _bbox_brute(cell, margin)


def test_step_touches_only_in_mask_box_voxels():
    """Sec. 2.4: the box solution is mapped onto the pleural mask; voxels outside the
    box or outside the mask keep their values bit for bit."""
    wl = W.random_case(11, (14, 12, 10), nspecies=2)
    lat = wl.lattice.copy()
    rep = oracle.step(lat, wl.params, margin=1)
    box = rep["box"]
    inbox = np.zeros(lat.mask.shape, bool)
    inbox[oracle.box_slices(box)] = True
    changed_ok = inbox & (lat.mask > 0)
    for s in range(2):
        assert np.array_equal(lat.fields[s][~changed_ok], wl.lattice.fields[s][~changed_ok])
        assert np.any(lat.fields[s][changed_ok] != wl.lattice.fields[s][changed_ok])


def test_empty_tumour_reports_empty():
    wl = W.random_case(1, (5, 5, 5))
    wl.lattice.cell_id[:] = 0
    assert oracle.step(wl.lattice, wl.params, 2)["status"] == oracle.ERR_EMPTY


def test_step_on_a_kept_box():
    """oracle.step(box=...) solves on a box kept from an earlier step: given the
    step's own bounding box it is the plain step bit for bit, and with a smaller
    kept box the voxels outside it keep c^n."""
    wl = W.random_case(5, (14, 12, 10), nspecies=2)
    a, b = wl.lattice.copy(), wl.lattice.copy()
    box = oracle.bbox(wl.lattice.cell_id, wl.margin)
    oracle.step(a, wl.params, wl.margin, rtol=0.0, atol=1e-12)
    oracle.step(b, wl.params, wl.margin, rtol=0.0, atol=1e-12, box=box)
    assert np.array_equal(a.fields, b.fields)
    (lx, ly, lz), (hx, hy, hz) = box
    small = ((lx + 1, ly + 1, lz + 1), (hx - 1, hy - 1, hz - 1))
    c = wl.lattice.copy()
    oracle.step(c, wl.params, wl.margin, rtol=0.0, atol=1e-12, box=small)
    out = np.ones(c.fields.shape[1:], bool)
    out[oracle.box_slices(small)] = False
    assert np.array_equal(c.fields[:, out], wl.lattice.fields[:, out])
    assert not np.array_equal(c.fields, wl.lattice.fields)
