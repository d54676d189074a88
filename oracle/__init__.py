"""CPU oracle for the box-restricted implicit-Euler FV reaction-diffusion step.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py may import this package; the product path (the CUDA library and
its binding) never does, and this package imports nothing from it.

Plain FP64, single thread.  The arithmetic-heavy parts (CSR assembly, GMRES,
dense LU, the CNN reference) live in the C files next to this module; the step
driver below is the plain definition of the method (arXiv 2505.03067):

* Sec. 2.3 (Bounding Box Mesh): the box is the bounding box of every tumour
  voxel (cell id > 0) widened by a margin and clamped to the lattice.
* Sec. 2.4 (Implementation): each species is advanced by one implicit-Euler
  step of Eq. 1-4 discretised by first-order finite volumes on the box mesh
  and solved with GMRES; the result is mapped back onto the pleural mask, so
  only in-mask voxels of the box change.

Stopping rule (the paper gives none): true residual ||b - A x||_2 <=
max(rtol * ||b_mask||_2, atol), norms over the in-mask rows (masked rows are
identity rows whose residual is zero from the initial guess c^n on).
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "lib")
_SOURCES = ["oracle.c", "cnn_oracle.c"]
_lib = None

OK, ERR_ARG, ERR_EMPTY, ERR_NOCONV, ERR_BREAKDOWN = 0, 1, 2, 3, 4
# -ffp-contract=off: no fused multiply-add contraction on any target
BUILD_FLAGS = ["-O3", "-ffp-contract=off"]


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/lib/liboracle.so with BUILD_FLAGS.  No
    -march=native: the oracle must give the same results on every host it is
    built on (an x86 build machine and the Arm host of the GPU), and a
    target-specific build may contract a*b+c into fused multiply-adds."""
    os.makedirs(_LIBDIR, exist_ok=True)
    so = os.path.join(_LIBDIR, "liboracle.so")
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    if not force and os.path.exists(so) and all(os.path.getmtime(so) >= os.path.getmtime(s) for s in srcs):
        return so
    tmp = so + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc"] + BUILD_FLAGS + ["-std=c11", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"])
    os.replace(tmp, so)
    return so


class _Species(C.Structure):
    _fields_ = [("dt", C.c_double), ("h", C.c_double), ("D", C.c_double), ("mu", C.c_double),
                ("c_bc", C.c_double), ("bc_box", C.c_int32), ("ncell", C.c_int32),
                ("k_cell", C.c_void_p), ("q_cell", C.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_assemble.restype = C.c_int64
        _lib.orc_gmres.restype = C.c_int
        _lib.orc_dense_solve.restype = C.c_int
        _lib.orc_csr_matvec.restype = None
    return _lib


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None else C.c_void_p(0)


@dataclasses.dataclass
class CSR:
    n: tuple
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def N(self):
        return len(self.row_ptr) - 1

    def dense(self) -> np.ndarray:
        A = np.zeros((self.N, self.N))
        for r in range(self.N):
            for e in range(self.row_ptr[r], self.row_ptr[r + 1]):
                A[r, self.col[e]] += self.val[e]
        return A

    def matvec(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, np.float64).reshape(-1)
        y = np.empty_like(x)
        lib().orc_csr_matvec(C.c_int64(self.N), _p(self.row_ptr), _p(self.col), _p(self.val), _p(x), _p(y))
        return y


# ---------------------------------------------------------------- Sec. 2.3: bounding box
def bbox(cell_id: np.ndarray, margin: int):
    """Bounding box of all voxels with cell id > 0, widened by `margin` and clamped:
    lo = max(0, min - margin), hi = min(L, max + margin + 1) per axis (x, y, z).
    Returns None when there is no tumour voxel."""
    zz, yy, xx = np.nonzero(cell_id > 0)
    if len(xx) == 0:
        return None
    Lz, Ly, Lx = cell_id.shape
    lo = [max(0, int(a.min()) - margin) for a in (xx, yy, zz)]
    hi = [min(L, int(a.max()) + margin + 1) for a, L in ((xx, Lx), (yy, Ly), (zz, Lz))]
    return tuple(lo), tuple(hi)


def box_slices(box):
    (lx, ly, lz), (hx, hy, hz) = box
    return (slice(lz, hz), slice(ly, hy), slice(lx, hx))


def box_view(a: np.ndarray, box) -> np.ndarray:
    """Copy of the box region of a lattice array (the gather)."""
    return np.ascontiguousarray(a[box_slices(box)])


# ---------------------------------------------------------------- Sec. 2.4: FV assembly
def assemble(mask_box, cell_box, c_box, params, s: int, bc_box: int = 0, dfac_box=None):
    """CSR matrix A and right-hand side b of species s on the box (see oracle.c)."""
    nz, ny, nx = mask_box.shape
    N = nx * ny * nz
    mask_box = np.ascontiguousarray(mask_box, np.uint8)
    cell_box = np.ascontiguousarray(cell_box, np.int32)
    c_box = np.ascontiguousarray(c_box, np.float64)
    k = np.ascontiguousarray(params.k_cell[s], np.float64)
    q = np.ascontiguousarray(params.q_cell[s], np.float64)
    df = None if dfac_box is None else np.ascontiguousarray(dfac_box, np.float64)
    sp = _Species(params.dt, params.h, float(params.D[s]), float(params.mu[s]), float(params.c_bc[s]),
                  bc_box, params.ncell, k.ctypes.data, q.ctypes.data)
    n = (C.c_int32 * 3)(nx, ny, nz)
    rp = np.empty(N + 1, np.int64)
    col = np.empty(7 * N, np.int32)
    val = np.empty(7 * N, np.float64)
    rhs = np.empty(N, np.float64)
    nnz = lib().orc_assemble(n, _p(mask_box), _p(cell_box), _p(c_box), _p(df), C.byref(sp),
                             _p(rp), _p(col), _p(val), _p(rhs))
    if nnz < 0:
        raise ValueError("cell id outside the rate tables")
    return CSR((nx, ny, nz), rp, col[:nnz].copy(), val[:nnz].copy()), rhs.reshape(mask_box.shape)


def gmres(A: CSR, b, x0, restart: int = 30, tol_abs: float = 1e-12, maxit: int = 10000):
    """Restarted GMRES(m) with MGS Arnoldi and Givens rotations (oracle.c)."""
    b = np.ascontiguousarray(b, np.float64).reshape(-1)
    x = np.array(x0, np.float64).reshape(-1).copy()
    it = C.c_int32(0)
    cyc = C.c_int32(0)
    res = C.c_double(0)
    st = lib().orc_gmres(C.c_int64(A.N), _p(A.row_ptr), _p(A.col), _p(A.val), _p(b), _p(x),
                         C.c_int32(restart), C.c_double(tol_abs), C.c_int32(maxit),
                         C.byref(it), C.byref(cyc), C.byref(res))
    return x, {"status": st, "iters": it.value, "cycles": cyc.value, "res": res.value}


def dense_solve(A: CSR, b):
    b = np.ascontiguousarray(b, np.float64).reshape(-1)
    x = np.empty_like(b)
    st = lib().orc_dense_solve(C.c_int64(A.N), _p(A.row_ptr), _p(A.col), _p(A.val), _p(b), _p(x))
    if st != OK:
        raise RuntimeError(f"dense solve failed: {st}")
    return x


# ---------------------------------------------------------------- one step of the method
def step(lat, params, margin: int, bc_box: int = 0, rtol: float = 1e-12, atol: float = 0.0,
         restart: int = 30, maxit: int = 10000, solver: str = "gmres", x0=None, box=None):
    """Advance every species of `lat` (a workloads.Lattice, modified in place) by one
    implicit-Euler step inside the bounding box; returns a report dict.  `x0`
    optionally gives per-species initial guesses on the box (default c^n).
    `box` (lo, hi) solves on a box kept from an earlier step instead of this
    step's bounding box: Sec. 2.3 refreshes the box only every 50 MCS and the
    steps in between keep it."""
    if box is None:
        box = bbox(lat.cell_id, margin)
    if box is None:
        return {"status": ERR_EMPTY, "box": None}
    sl = box_slices(box)
    mask_box = box_view(lat.mask, box)
    cell_box = box_view(lat.cell_id, box)
    dfac_box = None if lat.dfac is None else box_view(lat.dfac, box)
    inm = mask_box > 0
    rep = {"status": OK, "box": box, "iters": [], "cycles": [], "res": [], "bnorm": [],
           "mask_voxels": int(inm.sum()), "box_voxels": int(mask_box.size)}
    for s in range(params.nspecies):
        c_box = box_view(lat.fields[s], box)
        A, b = assemble(mask_box, cell_box, c_box, params, s, bc_box, dfac_box)
        bnorm = float(np.sqrt(np.sum(b[inm] ** 2)))
        tol = max(rtol * bnorm, atol)
        if solver == "lu":
            x = dense_solve(A, b)
            info = {"status": OK, "iters": 0, "cycles": 0,
                    "res": float(np.linalg.norm(b.reshape(-1) - A.matvec(x)))}
        else:
            guess = c_box if x0 is None else x0[s]
            x, info = gmres(A, b, guess, restart, tol, maxit)
        x = x.reshape(mask_box.shape)
        # Sec. 2.4: the solution is mapped onto the pleural mask
        lat.fields[s][sl][inm] = x[inm]
        rep["iters"].append(info["iters"])
        rep["cycles"].append(info["cycles"])
        rep["res"].append(info["res"])
        rep["bnorm"].append(bnorm)
        if info["status"] != OK:
            rep["status"] = info["status"]
    return rep


# ---------------------------------------------------------------- CNN reference (cnn_oracle.c)
CNN_CHANNELS = (9, 24, 24, 24, 24, 24, 3)


def _cnn_lib():
    L = lib()
    if not getattr(L, "_cnn_ready", False):
        L.orc_bf16.restype = C.c_double
        L.orc_bf16.argtypes = [C.c_double]
        L.orc_gelu.restype = C.c_double
        L.orc_gelu.argtypes = [C.c_double]
        L.orc_gelu_grad.restype = C.c_double
        L.orc_gelu_grad.argtypes = [C.c_double]
        L.orc_cnn_nparams.restype = C.c_int64
        L.orc_cnn_loss.restype = C.c_double
        L._cnn_ready = True
    return L


def bf16(a):
    """Round to bfloat16 (nearest even), returned as float64."""
    a = np.array(a, np.float64, copy=True)
    _cnn_lib().orc_bf16_array(C.c_int64(a.size), _p(a))
    return a


def gelu(z):
    return _cnn_lib().orc_gelu(float(z))


def gelu_grad(z):
    return _cnn_lib().orc_gelu_grad(float(z))


def cnn_nparams() -> int:
    return int(_cnn_lib().orc_cnn_nparams())


def conv3(x, W, b=None):
    """x: (nz, ny, nx, Ci); W: (27, Ci, Co); zero padding; returns (nz, ny, nx, Co)."""
    x = np.ascontiguousarray(x, np.float64)
    nz, ny, nx, Ci = x.shape
    W = np.ascontiguousarray(W, np.float64)
    Co = W.shape[2]
    out = np.empty((nz, ny, nx, Co))
    bb = None if b is None else np.ascontiguousarray(b, np.float64)
    _cnn_lib().orc_conv3(nx, ny, nz, Ci, Co, _p(x), _p(W), _p(bb), _p(out))
    return out


def conv3_dgrad(gout, W, Ci):
    gout = np.ascontiguousarray(gout, np.float64)
    nz, ny, nx, Co = gout.shape
    gin = np.empty((nz, ny, nx, Ci))
    _cnn_lib().orc_conv3_dgrad(nx, ny, nz, Ci, Co, _p(gout), _p(np.ascontiguousarray(W, np.float64)), _p(gin))
    return gin


def conv3_wgrad(x, gout):
    x = np.ascontiguousarray(x, np.float64)
    gout = np.ascontiguousarray(gout, np.float64)
    nz, ny, nx, Ci = x.shape
    Co = gout.shape[3]
    gW = np.empty((27, Ci, Co))
    gb = np.empty(Co)
    _cnn_lib().orc_conv3_wgrad(nx, ny, nz, Ci, Co, _p(x), _p(gout), _p(gW), _p(gb))
    return gW, gb


def cnn_forward(x, fields, params, s_out, round_act=True):
    """x: (nz, ny, nx, 9); fields: (nz, ny, nx, 3); params: flat [W1, b1, ..., W6, b6].
    Returns pred (nz, ny, nx, 3) and the (z, a) buffers for cnn_backward."""
    x = np.ascontiguousarray(x, np.float64)
    nz, ny, nx, _ = x.shape
    V = nx * ny * nz
    f = np.ascontiguousarray(fields, np.float64)
    P = np.ascontiguousarray(params, np.float64)
    z = np.zeros(6 * V * 24)
    a = np.zeros(5 * V * 24)
    pred = np.empty((nz, ny, nx, 3))
    _cnn_lib().orc_cnn_forward(nx, ny, nz, _p(x), _p(f), _p(P), C.c_double(s_out), int(round_act), _p(z), _p(a),
                               _p(pred))
    return pred, (z, a)


def cnn_loss(pred, target, mask):
    pred = np.ascontiguousarray(pred, np.float64)
    target = np.ascontiguousarray(target, np.float64)
    m = np.ascontiguousarray(mask, np.uint8)
    g = np.empty_like(pred)
    L = _cnn_lib().orc_cnn_loss(C.c_int64(m.size), _p(pred), _p(target), _p(m), _p(g))
    return float(L), g


def cnn_backward(x, params, s_out, cache, gpred, round_grad=False):
    x = np.ascontiguousarray(x, np.float64)
    nz, ny, nx, _ = x.shape
    z, a = cache
    P = np.ascontiguousarray(params, np.float64)
    g = np.empty_like(P)
    _cnn_lib().orc_cnn_backward(nx, ny, nz, _p(x), _p(P), C.c_double(s_out), _p(z), _p(a),
                                _p(np.ascontiguousarray(gpred, np.float64)), int(round_grad), _p(g))
    return g


def adam(p, g, m, v, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    """In place on p, m, v (float64 arrays)."""
    _cnn_lib().orc_adam(C.c_int64(p.size), _p(p), _p(np.ascontiguousarray(g, np.float64)), _p(m), _p(v),
                        C.c_double(lr), C.c_double(b1), C.c_double(b2), C.c_double(eps), int(t))


def cnn_param_slices():
    """(W, b) slices of each layer in the flat parameter vector."""
    out, o = [], 0
    for l in range(6):
        ci, co = CNN_CHANNELS[l], CNN_CHANNELS[l + 1]
        out.append((slice(o, o + 27 * ci * co), slice(o + 27 * ci * co, o + 27 * ci * co + co), ci, co))
        o += 27 * ci * co + co
    return out


# ---------------------------------------------------------------- flexible GMRES with the network (row a13)
def fgmres(A: CSR, b, x0, M, restart: int = 30, tol_abs: float = 1e-12, maxit: int = 10000):
    """Right-preconditioned flexible GMRES(m): the Arnoldi process runs on
    A z_j with z_j = M(v_j) for a preconditioner M that may change from one
    application to the next, modified Gram-Schmidt, Givens rotations for the
    least-squares problem, and the update x += Z y from the preconditioned
    directions; a cycle restarts from the true residual.  Plain NumPy."""
    b = np.asarray(b, np.float64).reshape(-1)
    x = np.array(x0, np.float64).reshape(-1).copy()
    it = cyc = 0
    status = ERR_NOCONV
    while True:
        r = b - A.matvec(x)
        beta = float(np.sqrt(r @ r))
        if not np.isfinite(beta):
            status = ERR_BREAKDOWN
            break
        if beta <= tol_abs:
            status = OK
            break
        if it >= maxit:
            break
        cyc += 1
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        k = 0
        for j in range(restart):
            z = np.asarray(M(V[j]), np.float64).reshape(-1)
            Z.append(z)
            w = A.matvec(z)
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            hn = float(np.sqrt(w @ w))
            H[j + 1, j] = hn
            for i in range(j):
                t0, t1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * t0 + sn[i] * t1
                H[i + 1, j] = -sn[i] * t0 + cs[i] * t1
            den = float(np.hypot(H[j, j], hn))
            cs[j], sn[j] = (1.0, 0.0) if den == 0.0 else (H[j, j] / den, hn / den)
            H[j, j] = cs[j] * H[j, j] + sn[j] * hn
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            if hn > 0.0:
                V.append(w / hn)
            if abs(g[j + 1]) <= tol_abs or it >= maxit or hn == 0.0:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        for i in range(k):
            x = x + y[i] * Z[i]
    r = b - A.matvec(x)
    return x, {"status": status, "iters": it, "cycles": cyc, "res": float(np.sqrt(r @ r))}


def fgmres_refined(A: CSR, b, x0, M, restart: int = 8, tol_abs: float = 1e-12, maxit: int = 10000,
                   inner=np.float32, inner_rtol: float = 0.0):
    """Flexible GMRES inside iterative refinement, with the fallback to plain
    GMRES: the solver of the learned path (the network as the right
    preconditioner of a flexible Krylov method; mixed precision as iterative
    refinement around a low-precision inner solve).  Plain NumPy.

    Each refinement step takes the FP64 true residual r = b - A x, beta =
    ||r||, and runs ONE flexible GMRES(m) cycle on A d = r: the Krylov vectors
    v_j, the directions z_j = M(v_j) and w = A z_j are stored in `inner`
    precision (for FP32 with A's coefficients rounded to FP32), Gram-Schmidt is
    classical in two passes, the Hessenberg matrix, Givens rotations and the
    least-squares solve are FP64.  The cycle ends when the residual estimate
    |g_{j+1}| falls to max(tol / 4, inner_rtol * beta) (FP32; tol for FP64),
    after m steps, at maxit steps in all, or on a zero or non-finite
    h_{j+1,j} / estimate.  The trial x_t = x + Z y (FP64) replaces x when
    ||b - A x_t|| < beta; otherwise it is dropped and the solve continues
    with M = identity (plain GMRES), or, already plain, stops (stagnation).
    Returns x and {status, iters, cycles, res, fallback}."""
    with np.errstate(all="ignore"):          # a failing preconditioner may return inf / NaN
        return _fgmres_refined(A, b, x0, M, restart, tol_abs, maxit, inner, inner_rtol)


def _fgmres_refined(A, b, x0, M, restart, tol_abs, maxit, inner, inner_rtol):
    b = np.asarray(b, np.float64).reshape(-1)
    x = np.array(x0, np.float64).reshape(-1).copy()
    f32 = np.dtype(inner) == np.float32
    if f32:
        q = lambda u: np.asarray(u, np.float64).astype(np.float32).astype(np.float64)
        A_in = dataclasses.replace(A, val=q(A.val))
    else:
        q = lambda u: np.asarray(u, np.float64)
        A_in = A
    m = restart
    r = b - A.matvec(x)
    beta = float(np.sqrt(r @ r))
    it = cyc = 0
    fallback = False
    if not np.isfinite(beta):
        return x, {"status": ERR_BREAKDOWN, "iters": 0, "cycles": 0, "res": beta, "fallback": False}
    if beta <= tol_abs:
        return x, {"status": OK, "iters": 0, "cycles": 0, "res": beta, "fallback": False}
    while True:
        cyc += 1
        tol_in = max(0.25 * tol_abs, inner_rtol * beta) if f32 else tol_abs
        V = [q(r / beta)]
        Z = []
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0
        for j in range(m):
            z = V[j] if fallback else q(M(V[j]))
            Z.append(z)
            w = q(A_in.matvec(z))
            col = np.zeros(j + 1)
            for _ in range(2):                       # classical Gram-Schmidt, two passes
                c = np.array([w @ V[i] for i in range(j + 1)])
                w = q(w - sum(c[i] * V[i] for i in range(j + 1)))
                col += c
            hn = float(np.sqrt(w @ w))
            H[:j + 1, j] = col
            for i in range(j):
                t0, t1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * t0 + sn[i] * t1
                H[i + 1, j] = -sn[i] * t0 + cs[i] * t1
            den = float(np.hypot(H[j, j], hn))
            cs[j], sn[j] = (1.0, 0.0) if den == 0.0 else (H[j, j] / den, hn / den)
            H[j, j] = cs[j] * H[j, j] + sn[j] * hn
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            if hn > 0.0 and np.isfinite(hn):
                V.append(q(w / hn))
            if not np.isfinite(g[j + 1]) or abs(g[j + 1]) <= tol_in or it >= maxit or hn == 0.0:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        xt = x.copy()
        for i in range(k):
            xt = xt + y[i] * Z[i]
        rt = b - A.matvec(xt)
        bt = float(np.sqrt(rt @ rt))
        stall = False
        if np.isfinite(bt) and bt < beta:
            x, r, beta = xt, rt, bt
        elif not fallback:
            fallback = True
        else:
            stall = True
        if beta <= tol_abs:
            status = OK
            break
        if it >= maxit or stall:
            status = ERR_NOCONV
            break
    return x, {"status": status, "iters": it, "cycles": cyc, "res": beta, "fallback": fallback}


def cnn_precond_inputs(v_box, s, cell_box, mask_box, params):
    """Inputs of the network used as a preconditioner for species s: the
    network's nine channels with the field of species s set to v (scaled as
    the features scale it: 1, 1, 20 for species 0, 1, 2), the other fields and
    the source map at zero (homogeneous problem), the medium / tumour one-hot,
    the uptake maps 10 k_0, 10 k_1 and the mask; BF16-rounded like the device
    features.  Returns x (nz, ny, nx, 9) and fields (nz, ny, nx, 3)."""
    nz, ny, nx = mask_box.shape
    x = np.zeros((nz, ny, nx, 9))
    f = np.zeros((nz, ny, nx, 3))
    fscale = (1.0, 1.0, 20.0)
    vf = np.asarray(v_box, np.float64).astype(np.float32).astype(np.float64)
    f[..., s] = vf
    x[..., s] = bf16((vf * np.float32(fscale[s])).astype(np.float32))
    cid = np.where((cell_box >= 0) & (cell_box < params.ncell), cell_box, 0)
    x[..., 3] = (cid == 0)
    x[..., 4] = (cid > 0)
    if params.nspecies > 0:
        x[..., 5] = bf16((np.float32(10.0) * params.k_cell[0][cid].astype(np.float32)).astype(np.float32))
    if params.nspecies > 1:
        x[..., 6] = bf16((np.float32(10.0) * params.k_cell[1][cid].astype(np.float32)).astype(np.float32))
    x[..., 8] = (mask_box > 0)
    return x, f


def cnn_precond(v_box, s, cell_box, mask_box, params, net_params, s_out):
    """The network as a (nonlinear) right preconditioner for species s: with
    m = max |v|, z = m * net(v / m)[s] on the in-mask voxels, 0 elsewhere
    (m scales v into the range the network was trained on)."""
    v = np.asarray(v_box, np.float64)
    m = float(np.max(np.abs(v)))
    if m == 0.0:
        return np.zeros_like(v)
    x, f = cnn_precond_inputs(v / m, s, cell_box, mask_box, params)
    pred, _ = cnn_forward(x, f, bf16(np.asarray(net_params, np.float64)), s_out)
    return np.where(mask_box > 0, m * pred[..., s], 0.0)


# ---------------------------------------------------------------- growth driver (a reading of Sec. 2.1 / 2.4)
# The paper drives the fields from CompuCell3D's CPM (proliferation, mitosis,
# death through Steppables) and gives no Hamiltonian.  This is the simple
# growth / mitosis rule the GPU driver implements, written out plainly:
#
# 1. Growth.  Every medium voxel (cell id 0) inside the pleural mask with at
#    least one tumour neighbour (6-neighbourhood, lattice faces closed) is
#    taken over with probability p = p_grow * c_O/(K_O + c_O) * c_n/(K_n + c_n)
#    (O2 = species 0, nutrient = species 1 at that voxel; p = 0 where
#    c_O < o2_min), by the j-th of its k tumour neighbours in the order
#    -x, +x, -y, +y, -z, +z.  All voxels read the lattice as it was before
#    the step (synchronous update).
# 2. Mitosis.  After growth every cell with at least v_div voxels divides, in
#    increasing id order while the rate tables have room: the daughter gets
#    the next free id and the parent's rates, and takes the parent's voxels
#    strictly above the parent's centroid along an axis drawn per cell
#    (coord * volume > sum of coords, exact integers).
#
# Random numbers: one counter-based generator on both sides, the SplitMix64
# output function (Steele, Lea and Flood, OOPSLA 2014) applied to
# seed + (c + 1) * 0x9E3779B97F4A7C15 with the counter c = (4 step + stream)
# << 40 | index: stream 0 (growth draw u = top 53 bits / 2^53), 1 (neighbour
# choice j = (top 32 bits * k) >> 32) per voxel, 2 (axis = (top 32 bits * 3)
# >> 32) per cell.
SPLITMIX_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64_out(z):
    """The SplitMix64 output (mix) function of 64-bit words (NumPy uint64)."""
    z = np.asarray(z, np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def cpm_draw(seed: int, step: int, stream: int, idx):
    """64 random bits for (seed, step, stream, index), index an integer array."""
    idx = np.asarray(idx, np.uint64)
    c = (np.uint64((4 * step + stream) & ((1 << 24) - 1)) << np.uint64(40)) | idx
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _M64) + (c + np.uint64(1)) * np.uint64(SPLITMIX_GAMMA)
    return splitmix64_out(z)


def _nbr_ids(cell):
    """[6, Lz, Ly, Lx] ids of the -x, +x, -y, +y, -z, +z neighbours (0 off the lattice)."""
    p = np.pad(cell, 1)
    Lz, Ly, Lx = cell.shape
    c = (slice(1, Lz + 1), slice(1, Ly + 1), slice(1, Lx + 1))
    return np.stack([p[c[0], c[1], 0:Lx], p[c[0], c[1], 2:Lx + 2], p[c[0], 0:Ly, c[2]], p[c[0], 2:Ly + 2, c[2]],
                     p[0:Lz, c[1], c[2]], p[2:Lz + 2, c[1], c[2]]])


def cpm_step(cell_id, mask, o2, nut, k_cell, q_cell, ncell: int, cp: dict, seed: int, step: int):
    """One growth + mitosis step (rules above).  cell_id (Lz, Ly, Lx) int32,
    o2 / nut float64 of the same shape, k_cell / q_cell [S][capacity] float64,
    ncell ids in use.  Returns (cell_id, k_cell, q_cell, ncell, stats) with
    stats = {grown, divisions}; the inputs are not modified."""
    cell = np.asarray(cell_id, np.int32)
    Lz, Ly, Lx = cell.shape
    v = np.arange(cell.size, dtype=np.uint64).reshape(cell.shape)
    nb = _nbr_ids(cell)
    tum = nb > 0
    k = tum.sum(axis=0)
    cand = (cell == 0) & (np.asarray(mask) > 0) & (k > 0)
    c0 = np.asarray(o2, np.float64)
    c1 = np.asarray(nut, np.float64)
    with np.errstate(all="ignore"):
        p = cp["p_grow"] * (c0 / (cp["K_o2"] + c0)) * (c1 / (cp["K_nut"] + c1))
    p = np.where(c0 < cp["o2_min"], 0.0, p)
    u = (cpm_draw(seed, step, 0, v) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    grow = cand & (u < p)
    h2 = cpm_draw(seed, step, 1, v) >> np.uint64(32)
    j = ((h2 * k.astype(np.uint64)) >> np.uint64(32)).astype(np.int64)
    # the j-th tumour neighbour: position of the (j+1)-th True along axis 0
    rank = np.cumsum(tum, axis=0) - 1
    pick = np.argmax(tum & (rank == j[None]), axis=0)
    chosen = np.take_along_axis(nb, pick[None], axis=0)[0]
    new = np.where(grow, chosen, cell).astype(np.int32)
    # mitosis
    cap = k_cell.shape[1]
    ids = new.reshape(-1)
    zz, yy, xx = np.indices(new.shape)
    coords = [xx.reshape(-1).astype(np.int64), yy.reshape(-1).astype(np.int64), zz.reshape(-1).astype(np.int64)]
    vol = np.bincount(ids, minlength=cap).astype(np.int64)
    sums = [np.zeros(cap, np.int64) for _ in range(3)]
    for a in range(3):
        np.add.at(sums[a], ids, coords[a])
    k_new = np.array(k_cell, np.float64, copy=True)
    q_new = np.array(q_cell, np.float64, copy=True)
    daughter = np.full(cap, -1, np.int64)
    axis = np.zeros(cap, np.int64)
    nc = ncell
    for cid in range(1, ncell):
        if vol[cid] >= cp["v_div"] and nc < cap:
            daughter[cid] = nc
            h3 = int(cpm_draw(seed, step, 2, np.array([cid]))[0]) >> 32
            axis[cid] = (h3 * 3) >> 32
            k_new[:, nc] = k_new[:, cid]
            q_new[:, nc] = q_new[:, cid]
            nc += 1
    d = daughter[ids]
    a = axis[ids]
    cpos = np.where(a == 0, coords[0], np.where(a == 1, coords[1], coords[2]))
    spos = np.where(a == 0, sums[0][ids], np.where(a == 1, sums[1][ids], sums[2][ids]))
    move = (ids > 0) & (d >= 0) & (cpos * vol[ids] > spos)
    out = np.where(move, d, ids).astype(np.int32).reshape(new.shape)
    return out, k_new, q_new, nc, {"grown": int(grow.sum()), "divisions": int(nc - ncell)}


def cpm_step_loops(cell_id, mask, o2, nut, k_cell, q_cell, ncell: int, cp: dict, seed: int, step: int):
    """cpm_step written voxel by voxel in plain Python (tiny lattices only):
    the rules above, literally."""
    cell = np.asarray(cell_id, np.int32)
    Lz, Ly, Lx = cell.shape
    new = cell.copy()
    grown = 0
    for z in range(Lz):
        for y in range(Ly):
            for x in range(Lx):
                if cell[z, y, x] != 0 or not mask[z, y, x]:
                    continue
                nbrs = []
                for dz, dy, dx in ((0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)):
                    zz, yy, xx = z + dz, y + dy, x + dx
                    if 0 <= zz < Lz and 0 <= yy < Ly and 0 <= xx < Lx and cell[zz, yy, xx] > 0:
                        nbrs.append(int(cell[zz, yy, xx]))
                if not nbrs:
                    continue
                c0, c1 = float(o2[z, y, x]), float(nut[z, y, x])
                if c0 < cp["o2_min"]:
                    continue
                p = cp["p_grow"] * (c0 / (cp["K_o2"] + c0)) * (c1 / (cp["K_nut"] + c1))
                vi = x + Lx * (y + Ly * z)
                u = (int(cpm_draw(seed, step, 0, np.array([vi]))[0]) >> 11) * 2.0 ** -53
                if u < p:
                    h2 = int(cpm_draw(seed, step, 1, np.array([vi]))[0]) >> 32
                    new[z, y, x] = nbrs[(h2 * len(nbrs)) >> 32]
                    grown += 1
    cap = k_cell.shape[1]
    k_new = np.array(k_cell, np.float64, copy=True)
    q_new = np.array(q_cell, np.float64, copy=True)
    vol = {}
    sums = {}
    for z in range(Lz):
        for y in range(Ly):
            for x in range(Lx):
                c = int(new[z, y, x])
                if c > 0:
                    vol[c] = vol.get(c, 0) + 1
                    s = sums.setdefault(c, [0, 0, 0])
                    s[0] += x
                    s[1] += y
                    s[2] += z
    plan = {}
    nc = ncell
    for cid in range(1, ncell):
        if vol.get(cid, 0) >= cp["v_div"] and nc < cap:
            h3 = int(cpm_draw(seed, step, 2, np.array([cid]))[0]) >> 32
            plan[cid] = (nc, (h3 * 3) >> 32)
            k_new[:, nc] = k_new[:, cid]
            q_new[:, nc] = q_new[:, cid]
            nc += 1
    out = new.copy()
    for z in range(Lz):
        for y in range(Ly):
            for x in range(Lx):
                c = int(new[z, y, x])
                if c in plan:
                    d, a = plan[c]
                    if (x, y, z)[a] * vol[c] > sums[c][a]:
                        out[z, y, x] = d
    return out, k_new, q_new, nc, {"grown": grown, "divisions": nc - ncell}
