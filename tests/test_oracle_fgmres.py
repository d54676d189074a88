"""Pins of the oracle's flexible GMRES and of the network preconditioner (no GPU).

The linear system has one solution (A is a nonsingular M-matrix), so every
preconditioner must lead FGMRES to it; beyond that, the identity reduces
FGMRES to GMRES step for step, an exact inverse converges in one step, and a
network whose output layer is zero reproduces its input field, i.e. the
identity on the mask.  An update from the Arnoldi vectors instead of the
preconditioned directions, or a preconditioner applied on the wrong side,
fails the checks with a non-identity M.
"""
import numpy as np
import pytest

import oracle
from paper_2505_03067_gb300 import workloads as W


def _system(seed, dims=(9, 8, 7), s=0, dfac=False):
    wl = W.random_case(seed, dims, nspecies=3, dfac=dfac)
    lat, p = wl.lattice, wl.params
    A, b = oracle.assemble(lat.mask, lat.cell_id, lat.fields[s], p, s, 0, lat.dfac)
    return wl, A, b.reshape(-1), lat.fields[s].reshape(-1).copy()


def _net_params(seed, last_scale=1.0):
    rng = np.random.default_rng(seed)
    out = []
    ch = oracle.CNN_CHANNELS
    for l, (ci, co) in enumerate(zip(ch[:-1], ch[1:])):
        w = rng.normal(size=27 * ci * co) * np.sqrt(2.0 / (27 * ci)) * (last_scale if l == 5 else 1.0)
        out += [w, 0.01 * rng.normal(size=co)]
    p = np.concatenate(out)
    assert p.size == oracle.cnn_nparams()
    return p


@pytest.mark.parametrize("seed", [1, 2])
def test_identity_preconditioner_is_gmres(seed):
    wl, A, b, c = _system(seed)
    tol = 1e-11 * np.linalg.norm(b)
    xg, ig = oracle.gmres(A, b, c, 8, tol, 500)
    xf, inf = oracle.fgmres(A, b, c, lambda v: v, 8, tol, 500)
    assert ig["status"] == inf["status"] == oracle.OK
    assert ig["iters"] == inf["iters"] and ig["cycles"] == inf["cycles"]
    assert np.max(np.abs(xf - xg)) <= 1e-12 * np.max(np.abs(xg))


def test_exact_inverse_converges_in_one_step():
    wl, A, b, c = _system(3)
    xs = oracle.dense_solve(A, b)
    r0 = b - A.matvec(c)
    _, info = oracle.fgmres(A, b, c, lambda v: oracle.dense_solve(A, v), 8, 1e-10 * np.linalg.norm(r0), 50)
    assert info["status"] == oracle.OK and info["iters"] == 1 and info["cycles"] == 1
    x, _ = oracle.fgmres(A, b, c, lambda v: oracle.dense_solve(A, v), 8, 1e-12 * np.linalg.norm(b), 50)
    assert np.max(np.abs(x - xs)) <= 1e-10


@pytest.mark.parametrize("seed,dfac", [(4, False), (5, True)])
def test_non_identity_preconditioners_reach_the_solution(seed, dfac):
    wl, A, b, c = _system(seed, dfac=dfac)
    xs = oracle.dense_solve(A, b)
    d = A.dense().diagonal()
    rng = np.random.default_rng(seed)
    perm = rng.permutation(b.size)
    for M in (lambda v: v / d,                       # Jacobi
              lambda v: v + 0.3 * v[perm],           # a fixed nonsymmetric mixing
              lambda v: np.tanh(v) + 0.1 * v):       # nonlinear (flexible)
        x, info = oracle.fgmres(A, b, c, M, 6, 1e-12 * np.linalg.norm(b), 3000)
        assert info["status"] == oracle.OK, info
        # ||x - x*||_2 <= ||A^-1||_2 ||r||_2 <= ||r||_2 (lambda_min(A) >= 1)
        assert np.linalg.norm(x - xs) <= info["res"] + 1e-13


def _csr_of(Md, dims):
    rp, col, val = [0], [], []
    for r in range(Md.shape[0]):
        nz = np.flatnonzero(Md[r])
        col += list(nz)
        val += list(Md[r, nz])
        rp.append(len(col))
    return oracle.CSR(dims, np.array(rp, np.int64), np.array(col, np.int32), np.array(val, np.float64))


@pytest.mark.parametrize("kind", ["jacobi", "mixing"])
def test_linear_preconditioner_equals_gmres_on_the_product(kind):
    """For a fixed matrix M, right-preconditioned FGMRES from x0 is GMRES on
    (A M) u = b - A x0 from u = 0, with x = x0 + M u: same iteration count,
    same solution."""
    wl, A, b, c = _system(11, dims=(7, 6, 5))
    N = b.size
    Ad = A.dense()
    if kind == "jacobi":
        Md = np.diag(1.0 / Ad.diagonal())
    else:
        rng = np.random.default_rng(12)
        Md = np.eye(N) + 0.3 * np.eye(N)[rng.permutation(N)]
    r0 = b - A.matvec(c)
    tol = 1e-10 * np.linalg.norm(r0)
    AM = _csr_of(Ad @ Md, A.n)
    u, ig = oracle.gmres(AM, r0, np.zeros(N), 5, tol, 400)
    x, inf = oracle.fgmres(A, b, c, lambda v: Md @ v, 5, tol, 400)
    assert ig["status"] == inf["status"] == oracle.OK
    assert ig["iters"] == inf["iters"] and ig["cycles"] == inf["cycles"]
    assert np.max(np.abs(x - (c + Md @ u))) <= 1e-9 * np.max(np.abs(x))


def test_zero_output_layer_network_is_the_identity_on_the_mask():
    wl, A, b, c = _system(6)
    lat, p = wl.lattice, wl.params
    net = _net_params(7, last_scale=0.0)
    net[-3:] = 0.0                               # output layer all zero: pred = input field
    rng = np.random.default_rng(8)
    v = rng.normal(size=lat.mask.shape)
    for s in range(3):
        z = oracle.cnn_precond(v, s, lat.cell_id, lat.mask, p, net, s_out=0.5)
        vf = v.astype(np.float32).astype(np.float64)
        m = np.max(np.abs(v))
        exp = np.where(lat.mask > 0, m * (v / m).astype(np.float32).astype(np.float64), 0.0)
        assert np.max(np.abs(z - exp)) <= 1e-15 * m, s
        assert np.max(np.abs(z - np.where(lat.mask > 0, vf, 0.0))) <= 1e-6 * m


def test_network_preconditioned_fgmres_reaches_the_solution():
    wl, A, b, c = _system(9, dims=(8, 7, 6))
    lat, p = wl.lattice, wl.params
    net = _net_params(10, last_scale=0.3)
    s = 1
    A, b = oracle.assemble(lat.mask, lat.cell_id, lat.fields[s], p, s)
    b = b.reshape(-1)
    c = lat.fields[s].reshape(-1)
    xs = oracle.dense_solve(A, b)

    def M(v):
        return oracle.cnn_precond(v.reshape(lat.mask.shape), s, lat.cell_id, lat.mask, p, net, 0.2).reshape(-1)

    x, info = oracle.fgmres(A, b, c, M, 6, 1e-11 * np.linalg.norm(b), 400)
    assert info["status"] == oracle.OK, info
    assert np.linalg.norm(x - xs) <= info["res"] + 1e-12
    # the preconditioner only acts on the mask: identity rows keep c^n
    out = lat.mask.reshape(-1) == 0
    assert np.array_equal(x[out], c[out])


# ---------------------------------------------------------------- refined FGMRES with the fallback
# Pins of oracle.fgmres_refined: in FP64 with every cycle accepted it is the
# restarted (F)GMRES of oracle.gmres / oracle.fgmres cycle for cycle (a wrong
# rotation, update or Gram-Schmidt pass changes the iteration count or the
# solution); in FP32 the refinement still reaches an FP64 tolerance; a
# preconditioner that returns non-finite or zero directions is dropped after
# one cycle, and the rest of the solve is then plain GMRES step for step.

@pytest.mark.parametrize("seed", [1, 2])
def test_refined_fp64_identity_is_restarted_gmres(seed):
    wl, A, b, c = _system(seed)
    tol = 1e-11 * np.linalg.norm(b)
    xg, ig = oracle.gmres(A, b, c, 8, tol, 500)
    xr, ir = oracle.fgmres_refined(A, b, c, lambda v: v, 8, tol, 500, inner=np.float64)
    assert ig["status"] == ir["status"] == oracle.OK and not ir["fallback"]
    assert ig["iters"] == ir["iters"] and ig["cycles"] == ir["cycles"]
    assert np.max(np.abs(xr - xg)) <= 1e-12 * np.max(np.abs(xg))


def test_refined_fp64_jacobi_is_fgmres():
    wl, A, b, c = _system(6, dfac=True)
    d = A.dense().diagonal()
    tol = 1e-11 * np.linalg.norm(b)
    xf, inf = oracle.fgmres(A, b, c, lambda v: v / d, 5, tol, 500)
    xr, ir = oracle.fgmres_refined(A, b, c, lambda v: v / d, 5, tol, 500, inner=np.float64)
    assert inf["iters"] == ir["iters"] and inf["cycles"] == ir["cycles"] and not ir["fallback"]
    assert np.max(np.abs(xr - xf)) <= 1e-12 * np.max(np.abs(xf))


@pytest.mark.parametrize("seed,dfac", [(7, False), (8, True)])
def test_refined_fp32_reaches_fp64_tolerance(seed, dfac):
    """FP32 cycles inside FP64 refinement meet a tolerance far below FP32's
    precision; the cycles end early (inner_rtol), so there are several."""
    wl, A, b, c = _system(seed, dfac=dfac)
    xs = oracle.dense_solve(A, b)
    d = A.dense().diagonal()
    tol = 1e-11 * np.linalg.norm(b)
    for M in (lambda v: v, lambda v: v / d, lambda v: np.tanh(v) + 0.1 * v):
        x, info = oracle.fgmres_refined(A, b, c, M, 8, tol, 2000, inner=np.float32, inner_rtol=1e-4)
        assert info["status"] == oracle.OK and not info["fallback"], info
        assert info["res"] <= tol and info["cycles"] >= 2
        r = b - A.matvec(x)
        assert abs(np.linalg.norm(r) - info["res"]) <= 1e-3 * info["res"]
        assert np.linalg.norm(x - xs) <= info["res"] + 1e-13


@pytest.mark.parametrize("inner", [np.float32, np.float64])
@pytest.mark.parametrize("bad", ["nan", "zero"])
def test_failing_preconditioner_falls_back_to_plain_gmres(inner, bad):
    """The failed cycle costs one Arnoldi step (its estimate or h_{1,0} ends it)
    and leaves x and r as they were: the result is the plain solve's, bit for
    bit, one cycle and one step later."""
    wl, A, b, c = _system(9)
    tol = 1e-10 * np.linalg.norm(b)
    M = (lambda v: np.full_like(v, np.nan)) if bad == "nan" else (lambda v: np.zeros_like(v))
    xp, ip = oracle.fgmres_refined(A, b, c, lambda v: v, 8, tol, 500, inner=inner, inner_rtol=1e-4)
    xb, ib = oracle.fgmres_refined(A, b, c, M, 8, tol, 500, inner=inner, inner_rtol=1e-4)
    assert ip["status"] == ib["status"] == oracle.OK
    assert not ip["fallback"] and ib["fallback"]
    assert ib["iters"] == ip["iters"] + 1 and ib["cycles"] == ip["cycles"] + 1
    assert np.array_equal(xb, xp)


def test_refined_stagnation_stops_before_maxit():
    """With tolerance 0 the refinement reaches the rounding floor, where a
    cycle no longer reduces the FP64 residual: the solver drops the
    preconditioner once, stalls on the next failure and returns NOCONV long
    before maxit."""
    wl, A, b, c = _system(10)
    x, info = oracle.fgmres_refined(A, b, c, lambda v: v, 8, 0.0, 100000, inner=np.float32, inner_rtol=1e-4)
    assert info["status"] == oracle.ERR_NOCONV and info["fallback"]
    assert info["iters"] < 1000
    assert info["res"] <= 1e-13 * np.linalg.norm(b)
