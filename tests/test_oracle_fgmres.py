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
