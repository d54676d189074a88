"""Thin Python binding of the C ABI in include/mpm.h (argument marshalling only).

Every entry point keeps its C name.  PyTorch provides device memory and
streams; every step of the method runs in the CUDA library.  There is no
fallback: if libmpm.so is missing or no GPU is present, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

MAX_SPECIES = 4
MAX_RESTART = 32
NOALLOC_MAX_SLABS = 4096

OK, ERR_ARG, ERR_EMPTY, ERR_NOCONV, ERR_BREAKDOWN, ERR_TIMEOUT, ERR_CUDA, ERR_NOMEM = range(8)
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_EMPTY", "ERR_NOCONV", "ERR_BREAKDOWN", "ERR_TIMEOUT", "ERR_CUDA", "ERR_NOMEM"]
EXPORT_X, EXPORT_RHS, EXPORT_DIAG, EXPORT_FLAGS, EXPORT_CELL = range(5)
DEBUG_TIMEOUT_NS, DEBUG_SKIP_BLOCK, DEBUG_PHASE_TIMES, DEBUG_SOLVER_VARIANT, DEBUG_CNN_LAYER_TIMES = 1, 2, 3, 4, 5
COUNTER_STEP_FULL_EXTRACTIONS = 19
CNN_INPUT, CNN_TARGET = 0, 1

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libmpm.so")

# symbols declared in include/mpm.h
SYMBOLS = ["mpm_create", "mpm_destroy", "mpm_last_error", "mpm_subgrid_create", "mpm_subgrid_destroy",
           "mpm_subgrid_info", "mpm_box_extract", "mpm_assemble_coeffs", "mpm_solve_step", "mpm_solve_batch",
           "mpm_subgrid_export", "mpm_subgrid_import", "mpm_apply_operator", "mpm_scatter", "mpm_debug_set",
           "mpm_counter_get", "mpm_box_bounds_noalloc", "mpm_subgrid_refresh", "mpm_batch_step",
           "mpm_tune_tile", "mpm_tune_solver", "mpm_tune_teams", "mpm_cnn_create", "mpm_cnn_destroy", "mpm_cnn_set_params",
           "mpm_cnn_get_params", "mpm_cnn_load_image", "mpm_cnn_export_features", "mpm_cnn_export_preact", "mpm_cnn_forward", "mpm_cnn_train_step", "mpm_cnn_guess", "mpm_cnn_layer_times",
           "mpm_step", "mpm_step_enqueue", "mpm_step_wait", "mpm_solve_fgmres_cnn", "mpm_cnn_precond",
           "mpm_step_host", "mpm_debug_convert", "mpm_step_set_network", "mpm_cpm_step"]


class mpm_box(C.Structure):
    _fields_ = [("lo", C.c_int32 * 3), ("hi", C.c_int32 * 3)]

    def as_tuple(self):
        return tuple(self.lo), tuple(self.hi)


class mpm_lattice(C.Structure):
    _fields_ = [("dims", C.c_int32 * 3), ("cell_id", C.c_void_p), ("mask", C.c_void_p), ("dfac", C.c_void_p),
                ("field", C.c_void_p * MAX_SPECIES)]


class mpm_host_lattice(C.Structure):
    _fields_ = [("cell_id", C.c_void_p), ("mask", C.c_void_p), ("field", C.c_void_p * MAX_SPECIES)]


HOST_FIELDS_IN = 1


class mpm_params(C.Structure):
    _fields_ = [("nspecies", C.c_int32), ("ncell", C.c_int32), ("dt", C.c_double), ("h", C.c_double),
                ("D", C.c_double * MAX_SPECIES), ("mu", C.c_double * MAX_SPECIES),
                ("c_bc", C.c_double * MAX_SPECIES), ("k_cell", C.c_void_p), ("q_cell", C.c_void_p),
                ("bc_box", C.c_int32)]


class mpm_opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("restart", C.c_int32), ("maxit", C.c_int32),
                ("precision", C.c_int32), ("inner_rtol", C.c_double), ("x0_given", C.c_int32),
                ("nblocks", C.c_int32), ("reorth", C.c_int32), ("box_every", C.c_int32), ("box_guard", C.c_int32)]


class mpm_report(C.Structure):
    _fields_ = [("iters", C.c_int32 * MAX_SPECIES), ("cycles", C.c_int32 * MAX_SPECIES),
                ("status", C.c_int32 * MAX_SPECIES), ("jsum", C.c_int32 * MAX_SPECIES),
                ("res", C.c_double * MAX_SPECIES),
                ("bnorm", C.c_double * MAX_SPECIES), ("box_voxels", C.c_int64), ("mask_voxels", C.c_int64),
                ("stored_voxels", C.c_int64), ("solve_ms", C.c_double), ("item_ms", C.c_double * MAX_SPECIES),
                ("reorth", C.c_int32 * MAX_SPECIES), ("fallback", C.c_int32 * MAX_SPECIES)]

    def as_dict(self, nspecies):
        return {"iters": list(self.iters[:nspecies]), "cycles": list(self.cycles[:nspecies]),
                "status": list(self.status[:nspecies]), "jsum": list(self.jsum[:nspecies]),
                "res": list(self.res[:nspecies]),
                "bnorm": list(self.bnorm[:nspecies]), "box_voxels": self.box_voxels,
                "mask_voxels": self.mask_voxels, "stored_voxels": self.stored_voxels, "solve_ms": self.solve_ms,
                "item_ms": list(self.item_ms[:nspecies]), "reorth": list(self.reorth[:nspecies]),
                "fallback": list(self.fallback[:nspecies])}


class mpm_cpm_params(C.Structure):
    _fields_ = [("p_grow", C.c_double), ("K_o2", C.c_double), ("K_nut", C.c_double), ("o2_min", C.c_double),
                ("v_div", C.c_int32), ("reserved", C.c_int32)]


class mpm_subgrid_desc(C.Structure):
    _fields_ = [("box", mpm_box), ("n", C.c_int32 * 3), ("tile", C.c_int32 * 3), ("ntiles", C.c_int32),
                ("nactive", C.c_int32), ("stored_voxels", C.c_int64), ("mask_voxels", C.c_int64),
                ("nspecies", C.c_int32)]


_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libmpm.so (built by paper_2505_03067_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = C.CDLL(path)
    P = C.c_void_p
    sig = {
        "mpm_create": [C.POINTER(P), C.c_size_t],
        "mpm_destroy": [P],
        "mpm_last_error": [P],
        "mpm_subgrid_create": [P, C.POINTER(P)],
        "mpm_subgrid_destroy": [P, P],
        "mpm_subgrid_info": [P, C.POINTER(mpm_subgrid_desc)],
        "mpm_box_extract": [P, C.POINTER(mpm_lattice), C.c_int32, C.c_int32, C.POINTER(C.c_int32),
                            C.POINTER(mpm_box), P, P],
        "mpm_assemble_coeffs": [P, P, C.POINTER(mpm_params), P],
        "mpm_subgrid_refresh": [P, P, C.POINTER(mpm_lattice), P],
        "mpm_cnn_create": [P, C.POINTER(P), C.POINTER(C.c_int32), C.c_int32, C.c_int32],
        "mpm_cnn_destroy": [P, P],
        "mpm_cnn_set_params": [P, P, P, C.c_int64, C.c_float, P],
        "mpm_cnn_get_params": [P, P, C.c_int32, P, C.c_int64, P],
        "mpm_cnn_load_image": [P, P, C.c_int32, C.POINTER(mpm_lattice), C.POINTER(mpm_params), C.POINTER(mpm_box),
                               C.c_int32, P],
        "mpm_cnn_forward": [P, P, C.c_int32, P, P],
        "mpm_cnn_export_features": [P, P, C.c_int32, P, P, P],
        "mpm_cnn_export_preact": [P, P, C.c_int32, C.c_int32, P, P],
        "mpm_cnn_train_step": [P, P, C.c_int32, C.c_float, C.c_int32, C.POINTER(C.c_double), P],
        "mpm_cnn_guess": [P, P, P, C.POINTER(mpm_lattice), C.POINTER(mpm_params), P],
        "mpm_cnn_layer_times": [P, P, P],
        "mpm_solve_fgmres_cnn": [P, P, P, C.POINTER(mpm_lattice), C.POINTER(mpm_params), C.POINTER(mpm_lattice),
                                 C.POINTER(mpm_opts), C.POINTER(mpm_report), P],
        "mpm_cnn_precond": [P, P, P, C.POINTER(mpm_lattice), C.POINTER(mpm_params), C.c_int32, P, P, P],
        "mpm_tune_tile": [P, C.POINTER(mpm_lattice), C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int64), P],
        "mpm_tune_solver": [P, C.POINTER(P), C.c_int32, C.POINTER(mpm_opts), C.POINTER(C.c_int32), C.c_char_p, P],
        "mpm_tune_teams": [P, C.POINTER(P), C.c_int32, C.POINTER(mpm_opts), C.c_int32, C.c_char_p, P, P, P],
        "mpm_batch_step": [P, C.POINTER(P), C.POINTER(C.POINTER(mpm_lattice)), C.POINTER(C.POINTER(mpm_params)),
                           C.c_int32, C.POINTER(mpm_opts), C.POINTER(mpm_report), P],
        "mpm_solve_step": [P, P, C.POINTER(mpm_lattice), C.POINTER(mpm_opts), C.POINTER(mpm_report), P],
        "mpm_step": [P, P, C.POINTER(mpm_lattice), C.POINTER(mpm_params), C.c_int32, C.POINTER(C.c_int32),
                     C.POINTER(mpm_opts), C.POINTER(mpm_report), C.POINTER(mpm_box), P],
        "mpm_step_enqueue": [P, P, C.POINTER(mpm_lattice), C.POINTER(mpm_params), C.c_int32, C.POINTER(C.c_int32),
                             C.POINTER(mpm_opts), P],
        "mpm_step_wait": [P, P, C.POINTER(mpm_report), C.POINTER(mpm_box), P],
        "mpm_step_host": [P, P, C.POINTER(mpm_host_lattice), C.POINTER(mpm_lattice), C.POINTER(mpm_params), C.c_int32,
                          C.POINTER(C.c_int32), C.POINTER(mpm_opts), C.c_int32, C.POINTER(mpm_report),
                          C.POINTER(mpm_box), P],
        "mpm_solve_batch": [P, C.POINTER(P), C.POINTER(C.POINTER(mpm_lattice)), C.c_int32, C.POINTER(mpm_opts),
                            C.POINTER(mpm_report), P],
        "mpm_subgrid_export": [P, P, C.c_int32, C.c_int32, P, P],
        "mpm_subgrid_import": [P, P, C.c_int32, P, P],
        "mpm_apply_operator": [P, P, C.c_int32, P, P, P],
        "mpm_scatter": [P, P, C.POINTER(mpm_lattice), P],
        "mpm_debug_set": [P, C.c_int32, C.c_int64],
        "mpm_counter_get": [P, C.c_int32, C.POINTER(C.c_int64)],
        "mpm_box_bounds_noalloc": [P, C.POINTER(C.c_int32), C.c_int32, P, P],
        "mpm_debug_convert": [P, P, P, P, P, P, C.c_int64, P],
        "mpm_cpm_step": [P, C.POINTER(mpm_lattice), C.POINTER(mpm_params), C.POINTER(mpm_cpm_params), C.c_uint64,
                         C.c_int64, P, P, P],
        "mpm_step_set_network": [P, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_char_p if name == "mpm_last_error" else C.c_int
    _lib = lib
    return lib


class MpmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ------------------------------------------------------------------ marshalling helpers
class DeviceLattice:
    """A lattice held in device memory (torch tensors) and its mpm_lattice view."""

    def __init__(self, lat, device="cuda"):
        import torch
        self.cell_id = torch.from_numpy(np.ascontiguousarray(lat.cell_id, np.int32)).to(device)
        self.mask = torch.from_numpy(np.ascontiguousarray(lat.mask, np.uint8)).to(device)
        self.dfac = None if lat.dfac is None else torch.from_numpy(np.ascontiguousarray(lat.dfac, np.float64)).to(device)
        self.fields = torch.from_numpy(np.ascontiguousarray(lat.fields, np.float64)).to(device)
        self.nspecies = int(self.fields.shape[0])
        self.dims = (int(lat.cell_id.shape[2]), int(lat.cell_id.shape[1]), int(lat.cell_id.shape[0]))

    def struct(self) -> mpm_lattice:
        s = mpm_lattice()
        s.dims[:] = self.dims
        s.cell_id = self.cell_id.data_ptr()
        s.mask = self.mask.data_ptr()
        s.dfac = self.dfac.data_ptr() if self.dfac is not None else None
        for k in range(self.nspecies):
            s.field[k] = self.fields[k].data_ptr()
        return s

    def fields_numpy(self) -> np.ndarray:
        return self.fields.cpu().numpy()


class DeviceParams:
    def __init__(self, params, bc_box=0, device="cuda"):
        import torch
        S = params.nspecies
        self.k = torch.from_numpy(np.ascontiguousarray(params.k_cell[:S], np.float64)).to(device)
        self.q = torch.from_numpy(np.ascontiguousarray(params.q_cell[:S], np.float64)).to(device)
        p = mpm_params()
        p.nspecies = S
        p.ncell = int(params.k_cell.shape[1])
        p.dt = float(params.dt)
        p.h = float(params.h)
        for s in range(S):
            p.D[s] = float(params.D[s])
            p.mu[s] = float(params.mu[s])
            p.c_bc[s] = float(params.c_bc[s])
        p.k_cell = self.k.data_ptr()
        p.q_cell = self.q.data_ptr()
        p.bc_box = int(bc_box)
        self.struct = p


def make_opts(rtol=1e-6, atol=0.0, restart=30, maxit=1000, precision=0, inner_rtol=1e-5, x0_given=0,
              nblocks=0, reorth=0, box_every=1, box_guard=0) -> mpm_opts:
    o = mpm_opts()
    o.rtol, o.atol, o.restart, o.maxit = rtol, atol, restart, maxit
    o.precision, o.inner_rtol, o.x0_given, o.nblocks = precision, inner_rtol, x0_given, nblocks
    o.reorth, o.box_every, o.box_guard = reorth, box_every, box_guard
    return o


class Context:
    """Owns an mpm_ctx; the methods are the C entry points with Python arguments."""

    def __init__(self, workspace_bytes: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the solver has no CPU path")
        self.lib = load()
        torch.cuda.init()
        self.ptr = C.c_void_p()
        self._check(self.lib.mpm_create(C.byref(self.ptr), workspace_bytes), "mpm_create")

    def _check(self, st, what, allow=()):
        if st != OK and st not in allow:
            msg = self.lib.mpm_last_error(self.ptr).decode() if self.ptr else what
            raise MpmError(st, f"{what}: {msg}")
        return st

    def close(self):
        if self.ptr:
            self.lib.mpm_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def error(self) -> str:
        return self.lib.mpm_last_error(self.ptr).decode()

    def counter(self, key: int) -> int:
        v = C.c_int64(0)
        self._check(self.lib.mpm_counter_get(self.ptr, key, C.byref(v)), "mpm_counter_get")
        return int(v.value)

    def launches(self) -> int:
        return self.counter(1)

    def imbalance(self) -> float:
        """The paper's load imbalance f = t_max / <t> - 1 over the CTA teams of the last solve."""
        return self.counter(11) / 1e6

    def phase_times_us(self) -> dict:
        """CTA-0 time split of the last solve (needs debug_set(DEBUG_PHASE_TIMES, 1))."""
        return {k: self.counter(c) / 1e3 for k, c in (("work", 2), ("wait", 3), ("reduce", 4), ("serial", 5),
                                                      ("R", 6), ("P1", 7), ("P2", 8), ("U", 9),
                                                      ("extract", 12), ("scatter", 13), ("x_bbox", 14),
                                                      ("x_activity", 15), ("x_count", 16), ("x_compact", 17),
                                                      ("x_gather", 18))}

    def debug_set(self, key: int, value: int):
        self._check(self.lib.mpm_debug_set(self.ptr, key, value), "mpm_debug_set")

    def mpm_tune_tile(self, lat: "DeviceLattice", margin: int, stream=None):
        t = (C.c_int32 * 3)()
        n = C.c_int64(0)
        ls = lat.struct()
        self._check(self.lib.mpm_tune_tile(self.ptr, C.byref(ls), margin, t, C.byref(n), _stream_ptr(stream)),
                    "mpm_tune_tile")
        return tuple(t), int(n.value)

    def mpm_tune_solver(self, subs, opts: "mpm_opts", cache_path=None, stream=None):
        n = len(subs)
        hs = (C.c_void_p * n)(*[s.h.value for s in subs])
        v = C.c_int32(0)
        cp = cache_path.encode() if cache_path else None
        self._check(self.lib.mpm_tune_solver(self.ptr, hs, n, C.byref(opts), C.byref(v), cp, _stream_ptr(stream)),
                    "mpm_tune_solver")
        return int(opts.restart), int(v.value)

    def mpm_tune_teams(self, subs, opts: "mpm_opts", rounds: int = 6, cache_path=None, stream=None):
        """The team planner's measured model (mpm_tune_teams): returns the
        imbalance f of every round run and the kept per-pass fixed cost F."""
        n = len(subs)
        hs = (C.c_void_p * n)(*[s.h.value for s in subs])
        hist = (C.c_double * (3 * (rounds + 1)))()
        F = (C.c_double * 2)()
        cp = cache_path.encode() if cache_path else None
        self._check(self.lib.mpm_tune_teams(self.ptr, hs, n, C.byref(opts), rounds, cp, hist, F,
                                            _stream_ptr(stream)), "mpm_tune_teams")
        h = [tuple(hist[3 * r:3 * r + 3]) for r in range(rounds + 1) if hist[3 * r] >= 0.0]
        return {"f": [v[0] for v in h], "fixed_per_round": [(v[1], v[2]) for v in h],
                "fixed": (float(F[0]), float(F[1]))}

    def subgrid_create(self) -> "Subgrid":
        h = C.c_void_p()
        self._check(self.lib.mpm_subgrid_create(self.ptr, C.byref(h)), "mpm_subgrid_create")
        return Subgrid(self, h)


class Subgrid:
    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.h = handle
        self.nspecies = 0

    def destroy(self):
        if self.h:
            self.ctx.lib.mpm_subgrid_destroy(self.ctx.ptr, self.h)
            self.h = C.c_void_p()

    def info(self) -> dict:
        d = mpm_subgrid_desc()
        self.ctx._check(self.ctx.lib.mpm_subgrid_info(self.h, C.byref(d)), "mpm_subgrid_info")
        return {"box": d.box.as_tuple(), "n": tuple(d.n), "tile": tuple(d.tile), "ntiles": d.ntiles,
                "nactive": d.nactive, "stored_voxels": d.stored_voxels, "mask_voxels": d.mask_voxels,
                "nspecies": d.nspecies}

    def mpm_box_extract(self, lat: DeviceLattice, nspecies: int, margin: int, tile=None, stream=None):
        box = mpm_box()
        ls = lat.struct()
        t = (C.c_int32 * 3)(*tile) if tile is not None else None
        st = self.ctx.lib.mpm_box_extract(self.ctx.ptr, C.byref(ls), nspecies, margin, t, C.byref(box), self.h,
                                          _stream_ptr(stream))
        self.ctx._check(st, "mpm_box_extract", allow=(ERR_EMPTY,))
        if st == ERR_EMPTY:
            return None
        self.nspecies = nspecies
        return box.as_tuple()

    def mpm_subgrid_refresh(self, lat: DeviceLattice, stream=None):
        ls = lat.struct()
        self.ctx._check(self.ctx.lib.mpm_subgrid_refresh(self.ctx.ptr, self.h, C.byref(ls), _stream_ptr(stream)),
                        "mpm_subgrid_refresh")

    def mpm_assemble_coeffs(self, prm: DeviceParams, stream=None):
        self.ctx._check(self.ctx.lib.mpm_assemble_coeffs(self.ctx.ptr, self.h, C.byref(prm.struct),
                                                         _stream_ptr(stream)), "mpm_assemble_coeffs")

    def mpm_solve_step(self, opts: mpm_opts, scatter_to: DeviceLattice | None = None, stream=None,
                       allow=(ERR_NOCONV,)):
        rep = mpm_report()
        ls = scatter_to.struct() if scatter_to is not None else None
        st = self.ctx.lib.mpm_solve_step(self.ctx.ptr, self.h, C.byref(ls) if ls is not None else None,
                                         C.byref(opts), C.byref(rep), _stream_ptr(stream))
        self.ctx._check(st, "mpm_solve_step", allow=allow)
        d = rep.as_dict(self.nspecies)
        d["status_code"] = st
        return d

    def mpm_step(self, lat: DeviceLattice, prm: "DeviceParams", margin: int, opts: mpm_opts, tile=None,
                 stream=None, allow=(ERR_NOCONV,)):
        """One device-resident step (mpm_step): box, compaction, assembly, solve
        and scatter from one CUDA graph; the report gains "box" (None if no
        tumour voxel) and "status_code"."""
        rep = mpm_report()
        box = mpm_box()
        ls = lat.struct()
        t = (C.c_int32 * 3)(*tile) if tile is not None else None
        st = self.ctx.lib.mpm_step(self.ctx.ptr, self.h, C.byref(ls), C.byref(prm.struct), margin, t,
                                   C.byref(opts), C.byref(rep), C.byref(box), _stream_ptr(stream))
        self.ctx._check(st, "mpm_step", allow=tuple(allow) + (ERR_EMPTY,))
        if st == ERR_EMPTY:
            return {"status_code": ERR_EMPTY, "box": None}
        self.nspecies = int(prm.struct.nspecies)
        d = rep.as_dict(self.nspecies)
        d["status_code"] = st
        d["box"] = box.as_tuple()
        return d

    def mpm_step_host(self, cell_id, mask, fields, lat: DeviceLattice, prm: "DeviceParams", margin: int,
                      opts: mpm_opts, fields_in=False, tile=None, stream=None, allow=(ERR_NOCONV,)):
        """mpm_step with the inputs in host memory: `cell_id` (int32), `mask`
        (uint8) and `fields` ([S, Lz, Ly, Lx] float64) are contiguous CPU
        tensors (None: the device copy is current); `fields` receives the
        voxels the step updated (the in-mask voxels of its box when `fields`
        is pinned, else the whole box)."""
        h = mpm_host_lattice()
        for name, t in (("cell_id", cell_id), ("mask", mask)):
            if t is not None:
                assert t.device.type == "cpu" and t.is_contiguous() and t.numel() == lat.cell_id.numel()
                setattr(h, name, t.data_ptr())
        if fields is not None:
            assert fields.device.type == "cpu" and fields.is_contiguous() and fields.dtype == lat.fields.dtype
            assert fields.shape == lat.fields.shape
            for s_ in range(fields.shape[0]):
                h.field[s_] = fields[s_].data_ptr()
        rep = mpm_report()
        box = mpm_box()
        ls = lat.struct()
        t = (C.c_int32 * 3)(*tile) if tile is not None else None
        st = self.ctx.lib.mpm_step_host(self.ctx.ptr, self.h, C.byref(h), C.byref(ls), C.byref(prm.struct), margin, t,
                                        C.byref(opts), HOST_FIELDS_IN if fields_in else 0, C.byref(rep),
                                        C.byref(box), _stream_ptr(stream))
        self.ctx._check(st, "mpm_step_host", allow=tuple(allow) + (ERR_EMPTY,))
        if st == ERR_EMPTY:
            return {"status_code": ERR_EMPTY, "box": None}
        self.nspecies = int(prm.struct.nspecies)
        d = rep.as_dict(self.nspecies)
        d["status_code"] = st
        d["box"] = box.as_tuple()
        return d

    def mpm_step_enqueue(self, lat: DeviceLattice, prm: "DeviceParams", margin: int, opts: mpm_opts, tile=None,
                         stream=None):
        """Queue one device-resident step (mpm_step_enqueue); no wait."""
        ls = lat.struct()
        t = (C.c_int32 * 3)(*tile) if tile is not None else None
        self.ctx._check(self.ctx.lib.mpm_step_enqueue(self.ctx.ptr, self.h, C.byref(ls), C.byref(prm.struct), margin,
                                                      t, C.byref(opts), _stream_ptr(stream)), "mpm_step_enqueue")
        self.nspecies = int(prm.struct.nspecies)

    def mpm_step_wait(self, stream=None, allow=(ERR_NOCONV,)):
        """Wait for the queued steps and report the last one (as mpm_step)."""
        rep = mpm_report()
        box = mpm_box()
        st = self.ctx.lib.mpm_step_wait(self.ctx.ptr, self.h, C.byref(rep), C.byref(box), _stream_ptr(stream))
        self.ctx._check(st, "mpm_step_wait", allow=tuple(allow) + (ERR_EMPTY,))
        if st == ERR_EMPTY:
            return {"status_code": ERR_EMPTY, "box": None}
        d = rep.as_dict(self.nspecies)
        d["status_code"] = st
        d["box"] = box.as_tuple()
        return d

    def mpm_subgrid_export(self, what: int, s: int = 0, stream=None):
        import torch
        info = self.info()
        nx, ny, nz = info["n"]
        dt = {EXPORT_X: torch.float64, EXPORT_RHS: torch.float64, EXPORT_DIAG: torch.float64,
              EXPORT_FLAGS: torch.uint8, EXPORT_CELL: torch.int32}[what]
        out = torch.empty((nz, ny, nx), dtype=dt, device="cuda")
        self.ctx._check(self.ctx.lib.mpm_subgrid_export(self.ctx.ptr, self.h, what, s, C.c_void_p(out.data_ptr()),
                                                        _stream_ptr(stream)), "mpm_subgrid_export")
        return out

    def mpm_subgrid_import(self, s: int, src, stream=None):
        self.ctx._check(self.ctx.lib.mpm_subgrid_import(self.ctx.ptr, self.h, s, C.c_void_p(src.data_ptr()),
                                                        _stream_ptr(stream)), "mpm_subgrid_import")

    def mpm_apply_operator(self, s: int, x, stream=None):
        import torch
        y = torch.empty_like(x)
        self.ctx._check(self.ctx.lib.mpm_apply_operator(self.ctx.ptr, self.h, s, C.c_void_p(x.data_ptr()),
                                                        C.c_void_p(y.data_ptr()), _stream_ptr(stream)),
                        "mpm_apply_operator")
        return y

    def mpm_scatter(self, lat: DeviceLattice, stream=None):
        ls = lat.struct()
        self.ctx._check(self.ctx.lib.mpm_scatter(self.ctx.ptr, self.h, C.byref(ls), _stream_ptr(stream)),
                        "mpm_scatter")


def mpm_box_bounds_noalloc(cell_id, margin: int, out_box, stream=None) -> int:
    """Bounding box of a device int32 lattice (torch tensor of shape (Lz, Ly, Lx))
    into out_box (device int32 tensor of 7 entries), without any allocation by
    the library; returns the mpm_status."""
    import torch
    if not (isinstance(cell_id, torch.Tensor) and cell_id.is_cuda and cell_id.dtype == torch.int32
            and cell_id.is_contiguous() and cell_id.dim() == 3):
        raise ValueError("mpm_box_bounds_noalloc: cell_id must be a contiguous 3-D int32 CUDA tensor (Lz, Ly, Lx)")
    if not (isinstance(out_box, torch.Tensor) and out_box.is_cuda and out_box.dtype == torch.int32
            and out_box.is_contiguous() and out_box.numel() >= 7):
        raise ValueError("mpm_box_bounds_noalloc: out_box must be a contiguous int32 CUDA tensor of >= 7 entries")
    if cell_id.device != out_box.device:
        raise ValueError("mpm_box_bounds_noalloc: cell_id and out_box must be on the same device")
    lib = load()
    lz, ly, lx = (int(v) for v in cell_id.shape)
    dims = (C.c_int32 * 3)(lx, ly, lz)
    return lib.mpm_box_bounds_noalloc(C.c_void_p(cell_id.data_ptr()), dims, margin,
                                      C.c_void_p(out_box.data_ptr()), _stream_ptr(stream))


def mpm_debug_convert(in64, in32, stream=None):
    """The FP32 Krylov path's bit-level conversions on device tensors (test
    hook): returns (f32_rz(in64), __double2float_rz(in64), f64_of(in32),
    (double) in32)."""
    import torch
    if not (in64.is_cuda and in64.dtype == torch.float64 and in64.is_contiguous() and in32.is_cuda
            and in32.dtype == torch.float32 and in32.is_contiguous() and in32.numel() == in64.numel()):
        raise ValueError("mpm_debug_convert: contiguous CUDA float64 and float32 tensors of equal size")
    n = in64.numel()
    out32, ref32 = (torch.empty(n, dtype=torch.float32, device=in64.device) for _ in range(2))
    out64, ref64 = (torch.empty(n, dtype=torch.float64, device=in64.device) for _ in range(2))
    ptr = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    st = load().mpm_debug_convert(ptr(in64), ptr(out32), ptr(ref32), ptr(in32), ptr(out64), ptr(ref64), n,
                                  _stream_ptr(stream))
    if st != OK:
        raise MpmError(st, "mpm_debug_convert failed")
    return out32, ref32, out64, ref64


def mpm_solve_batch(ctx: Context, subs, opts: mpm_opts, scatter_to=None, stream=None, allow=(ERR_NOCONV,)):
    n = len(subs)
    hs = (C.c_void_p * n)(*[s.h.value for s in subs])
    lat_structs = []
    lat_ptrs = None
    if scatter_to is not None:
        lat_structs = [None if l is None else l.struct() for l in scatter_to]
        lat_ptrs = (C.POINTER(mpm_lattice) * n)(*[C.pointer(l) if l is not None else C.POINTER(mpm_lattice)()
                                                  for l in lat_structs])
    reps = (mpm_report * n)()
    st = ctx.lib.mpm_solve_batch(ctx.ptr, hs, lat_ptrs, n, C.byref(opts), reps, _stream_ptr(stream))
    ctx._check(st, "mpm_solve_batch", allow=allow)
    return st, [reps[i].as_dict(subs[i].nspecies) for i in range(n)]


class BatchStepper:
    """Fixed-box batched steps of many systems (mpm_batch_step): every system is
    extracted once, then each step refreshes, assembles, solves all (system,
    species) pairs in one persistent launch and scatters, replayed from a CUDA
    graph after the first call."""

    def __init__(self, ctx: Context, lats, prms, margins, tile=None, tune_tiles=False):
        self.ctx = ctx
        self.lats, self.prms = list(lats), list(prms)
        self.subs = []
        self.tiles = []
        for lat, m in zip(self.lats, margins):
            sub = ctx.subgrid_create()
            t = ctx.mpm_tune_tile(lat, m)[0] if tune_tiles else tile
            self.tiles.append(t)
            box = sub.mpm_box_extract(lat, lat.nspecies, m, t)
            if box is None:
                raise MpmError(ERR_EMPTY, "batch system without tumour")
            self.subs.append(sub)
        n = len(self.subs)
        self._hs = (C.c_void_p * n)(*[s.h.value for s in self.subs])
        self._ls = [l.struct() for l in self.lats]
        self._lp = (C.POINTER(mpm_lattice) * n)(*[C.pointer(l) for l in self._ls])
        self._pp = (C.POINTER(mpm_params) * n)(*[C.pointer(p.struct) for p in self.prms])
        self._reps = (mpm_report * n)()
        for sub, prm in zip(self.subs, self.prms):
            sub.mpm_assemble_coeffs(prm)

    def tune(self, opts: mpm_opts, cache_path=None, team_rounds: int = 6):
        """Restart length and kernel variant for this batch (mpm_tune_solver),
        then the team planner's measured model (mpm_tune_teams; team_rounds 0
        skips it).  Returns (restart, variant); the team rounds' imbalances
        are kept in self.team_tuning."""
        m, var = self.ctx.mpm_tune_solver(self.subs, opts, cache_path)
        self.team_tuning = (self.ctx.mpm_tune_teams(self.subs, opts, team_rounds, cache_path)
                            if team_rounds > 0 else None)
        return m, var

    def step(self, opts: mpm_opts, stream=None, allow=(ERR_NOCONV,)):
        n = len(self.subs)
        st = self.ctx.lib.mpm_batch_step(self.ctx.ptr, self._hs, self._lp, self._pp, n, C.byref(opts), self._reps,
                                         _stream_ptr(stream))
        self.ctx._check(st, "mpm_batch_step", allow=allow)
        return st, [self._reps[i].as_dict(self.subs[i].nspecies) for i in range(n)]

    def graph_active(self) -> bool:
        return self.ctx.counter(10) == 1


class StepSolver:
    """One implicit-Euler step of every species on a device lattice.  By
    default the device-resident mpm_step (one CUDA graph per step); with
    fused=False the composition mpm_box_extract -> mpm_assemble_coeffs ->
    mpm_solve_step (with scatter)."""

    def __init__(self, ctx: Context, lat: DeviceLattice, prm: DeviceParams, margin: int, tile=None, fused=True):
        self.ctx, self.lat, self.prm, self.margin, self.tile = ctx, lat, prm, margin, tile
        self.fused = fused
        self.sub = ctx.subgrid_create()

    def set_network(self, cnn: "CNN | None"):
        """Start every later device-resident step's solve from the network's
        prediction (mpm_step_set_network); None: from c^n."""
        self.cnn = cnn
        self.ctx._check(self.ctx.lib.mpm_step_set_network(self.ctx.ptr, self.sub.h, cnn.h if cnn is not None else None),
                        "mpm_step_set_network")

    def step_async(self, opts: mpm_opts, stream=None):
        """Queue one device-resident step (read the result with wait())."""
        self.sub.mpm_step_enqueue(self.lat, self.prm, self.margin, opts, self.tile, stream)

    def wait(self, stream=None, allow=(ERR_NOCONV,)):
        return self.sub.mpm_step_wait(stream, allow)

    def step_host(self, cell_id, fields, opts: mpm_opts, mask=None, fields_in=False, stream=None,
                  allow=(ERR_NOCONV,)):
        """One step from host buffers (mpm_step_host): the cell ids (and the
        mask, and with fields_in the fields) in, the step's results out."""
        return self.sub.mpm_step_host(cell_id, mask, fields, self.lat, self.prm, self.margin, opts, fields_in,
                                      self.tile, stream, allow)

    def step(self, opts: mpm_opts, stream=None, allow=(ERR_NOCONV,)):
        if self.fused:
            return self.sub.mpm_step(self.lat, self.prm, self.margin, opts, self.tile, stream, allow)
        box = self.sub.mpm_box_extract(self.lat, self.lat.nspecies, self.margin, self.tile, stream)
        if box is None:
            return {"status_code": ERR_EMPTY, "box": None}
        self.sub.mpm_assemble_coeffs(self.prm, stream)
        rep = self.sub.mpm_solve_step(opts, scatter_to=self.lat, stream=stream, allow=allow)
        rep["box"] = box
        return rep


CNN_CHANNELS = (9, 24, 24, 24, 24, 24, 3)
CNN_NPARAMS = sum(27 * a * b + b for a, b in zip(CNN_CHANNELS[:-1], CNN_CHANNELS[1:]))


def cnn_init_params(seed: int = 0, last_scale: float = 0.1):
    """He-style random initial parameters (float32, flat layout of include/mpm.h)."""
    rng = np.random.default_rng(seed)
    out = []
    for l, (ci, co) in enumerate(zip(CNN_CHANNELS[:-1], CNN_CHANNELS[1:])):
        w = rng.normal(size=27 * ci * co) * np.sqrt(2.0 / (27 * ci))
        if l == 5:
            w *= last_scale
        out += [w, np.zeros(co)]
    return np.concatenate(out).astype(np.float32)


class GrowthDriver:
    """The device growth driver (mpm_cpm_step) on a device lattice: tumour
    growth into the mask driven by O2 and nutrient, and mitosis.  The rate
    tables of `prm` must have room for the daughters (capacity = their
    ncell); `ncell` is the number of ids in use at the start."""

    def __init__(self, ctx: Context, lat: DeviceLattice, prm: DeviceParams, ncell: int, p_grow: float = 0.6,
                 K_o2: float = 0.2, K_nut: float = 0.3, o2_min: float = 0.05, v_div: int = 400, seed: int = 1):
        import torch
        self.ctx, self.lat, self.prm, self.seed = ctx, lat, prm, seed
        self.cp = mpm_cpm_params(p_grow, K_o2, K_nut, o2_min, v_div, 0)
        self.ncell = torch.tensor([ncell], dtype=torch.int32, device="cuda")
        self.stats = torch.zeros(3, dtype=torch.int64, device="cuda")
        self.t = 0

    def step(self, stream=None):
        """One growth + mitosis step (queued on `stream`)."""
        ls = self.lat.struct()
        st = self.ctx.lib.mpm_cpm_step(self.ctx.ptr, C.byref(ls), C.byref(self.prm.struct), C.byref(self.cp),
                                       C.c_uint64(self.seed), self.t, C.c_void_p(self.ncell.data_ptr()),
                                       C.c_void_p(self.stats.data_ptr()), _stream_ptr(stream))
        self.ctx._check(st, "mpm_cpm_step")
        self.t += 1

    def counts(self) -> dict:
        s = self.stats.cpu().tolist()
        return {"ncell": int(self.ncell.item()), "grown": s[0], "divisions": s[1], "bad_ids": s[2]}


class CNN:
    """The learned warm start's network (mpm_cnn_*) on up to max_images images
    of dims image_dims = (Lx, Ly, Lz); tensors are torch CUDA tensors."""

    def __init__(self, ctx: Context, image_dims, max_images: int = 1, params=None, s_out: float = 0.01,
                 train: bool = False):
        self.ctx = ctx
        self.h = C.c_void_p()
        self.dims = tuple(int(v) for v in image_dims)
        self.V = self.dims[0] * self.dims[1] * self.dims[2]
        self.max_images = int(max_images)
        self.train = bool(train)
        d = (C.c_int32 * 3)(*self.dims)
        ctx._check(ctx.lib.mpm_cnn_create(ctx.ptr, C.byref(self.h), d, self.max_images, int(bool(train))),
                   "mpm_cnn_create")
        self.set_params(cnn_init_params() if params is None else params, s_out)

    def close(self):
        if self.h:
            self.ctx.lib.mpm_cnn_destroy(self.ctx.ptr, self.h)
            self.h = C.c_void_p()

    def set_params(self, params, s_out: float = 0.01, stream=None):
        p = np.ascontiguousarray(params, np.float32)
        self.s_out = s_out
        self.ctx._check(self.ctx.lib.mpm_cnn_set_params(self.ctx.ptr, self.h, C.c_void_p(p.ctypes.data), p.size,
                                                        C.c_float(s_out), _stream_ptr(stream)), "mpm_cnn_set_params")

    def get(self, which: int = 0, stream=None) -> np.ndarray:
        out = np.empty(CNN_NPARAMS, np.float32)
        self.ctx._check(self.ctx.lib.mpm_cnn_get_params(self.ctx.ptr, self.h, which, C.c_void_p(out.ctypes.data),
                                                        out.size, _stream_ptr(stream)), "mpm_cnn_get_params")
        return out

    def load_image(self, b: int, lat: DeviceLattice, prm: DeviceParams, box, what: int = 0, stream=None):
        """Image b from lattice `lat` on box ((lo), (hi)): what = CNN_INPUT
        (features of its fields) or CNN_TARGET (its fields as the target)."""
        (lo, hi) = box
        bx = mpm_box()
        bx.lo[:] = [int(v) for v in lo]
        bx.hi[:] = [int(v) for v in hi]
        ls = lat.struct()
        self.ctx._check(self.ctx.lib.mpm_cnn_load_image(self.ctx.ptr, self.h, int(b), C.byref(ls),
                                                        C.byref(prm.struct), C.byref(bx), int(what),
                                                        _stream_ptr(stream)), "mpm_cnn_load_image")

    def export_features(self, nimg: int = 1, stream=None):
        """(x [nimg * voxels][16] bf16, mask [nimg * voxels] uint8) as loaded."""
        import torch
        x = torch.zeros((nimg * self.V, 16), dtype=torch.bfloat16, device="cuda")
        m = torch.zeros(nimg * self.V, dtype=torch.uint8, device="cuda")
        self.ctx._check(self.ctx.lib.mpm_cnn_export_features(self.ctx.ptr, self.h, int(nimg), C.c_void_p(x.data_ptr()),
                                                             C.c_void_p(m.data_ptr()), _stream_ptr(stream)),
                        "mpm_cnn_export_features")
        return x, m

    def export_preact(self, layer: int, nimg: int = 1, stream=None):
        """FP32 pre-activations of `layer` (1..5) from the last train_step, [nimg * voxels][24]."""
        import torch
        z = torch.zeros((nimg * self.V, 24), dtype=torch.float32, device="cuda")
        self.ctx._check(self.ctx.lib.mpm_cnn_export_preact(self.ctx.ptr, self.h, int(layer), int(nimg),
                                                           C.c_void_p(z.data_ptr()), _stream_ptr(stream)),
                        "mpm_cnn_export_preact")
        return z

    def forward(self, nimg: int = 1, pred=None, stream=None):
        """pred [nimg * image voxels][3] FP32 (written at the active voxels)."""
        import torch
        if pred is None:
            pred = torch.zeros((nimg * self.V, 3), dtype=torch.float32, device="cuda")
        self.ctx._check(self.ctx.lib.mpm_cnn_forward(self.ctx.ptr, self.h, int(nimg), C.c_void_p(pred.data_ptr()),
                                                     _stream_ptr(stream)), "mpm_cnn_forward")
        return pred

    def train_step(self, nimg: int, lr: float, apply: bool = True, stream=None) -> float:
        loss = C.c_double(0)
        self.ctx._check(self.ctx.lib.mpm_cnn_train_step(self.ctx.ptr, self.h, int(nimg), C.c_float(lr), int(apply),
                                                        C.byref(loss), _stream_ptr(stream)), "mpm_cnn_train_step")
        return float(loss.value)

    def guess(self, sub: Subgrid, lat: DeviceLattice, prm: DeviceParams, stream=None):
        ls = lat.struct()
        self.ctx._check(self.ctx.lib.mpm_cnn_guess(self.ctx.ptr, self.h, sub.h, C.byref(ls), C.byref(prm.struct),
                                                   _stream_ptr(stream)), "mpm_cnn_guess")

    def layer_times(self):
        """Device ms of the six convolutions of the last application timed with
        DEBUG_CNN_LAYER_TIMES on (mpm_cnn_layer_times)."""
        ms = (C.c_float * 6)()
        self.ctx._check(self.ctx.lib.mpm_cnn_layer_times(self.ctx.ptr, self.h, ms), "mpm_cnn_layer_times")
        return list(ms)

    def precond(self, sub: Subgrid, lat: DeviceLattice, prm: DeviceParams, s: int, v, stream=None):
        """The FGMRES preconditioner on a box-dense FP64 tensor v (mpm_cnn_precond)."""
        import torch
        z = torch.empty_like(v)
        ls = lat.struct()
        self.ctx._check(self.ctx.lib.mpm_cnn_precond(self.ctx.ptr, self.h, sub.h, C.byref(ls), C.byref(prm.struct),
                                                     int(s), v.data_ptr(), z.data_ptr(), _stream_ptr(stream)),
                        "mpm_cnn_precond")
        return z

    def solve_fgmres(self, sub: Subgrid, lat: DeviceLattice, prm: DeviceParams, opts: mpm_opts,
                     scatter_to: DeviceLattice | None = None, stream=None, allow=(ERR_NOCONV,)):
        """Flexible GMRES with this network as the right preconditioner
        (mpm_solve_fgmres_cnn) on an assembled subgrid."""
        rep = mpm_report()
        ls = lat.struct()
        ss = scatter_to.struct() if scatter_to is not None else None
        st = self.ctx.lib.mpm_solve_fgmres_cnn(self.ctx.ptr, self.h, sub.h, C.byref(ls), C.byref(prm.struct),
                                               C.byref(ss) if ss is not None else None, C.byref(opts),
                                               C.byref(rep), _stream_ptr(stream))
        self.ctx._check(st, "mpm_solve_fgmres_cnn", allow=allow)
        d = rep.as_dict(sub.nspecies)
        d["status_code"] = st
        return d
