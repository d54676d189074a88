"""Training and use of the learned warm start (marshalling only: every step runs
in the library's kernels through the C ABI).

Training data come from the library's own FP64 solver, generated on the GPU
while training: B trajectories of 32^3 lattices (workloads.sphere_training_case)
are advanced one implicit-Euler step at a time; each step gives a pair
(features of c^n, c^{n+1}) per trajectory, and the batch of B pairs makes one
Adam step (mpm_cnn_train_step).  A trajectory restarts from a new random
lattice after `traj_len` steps.
"""
from __future__ import annotations

import time

import numpy as np

from . import mpm
from . import workloads as W


class _Traj:
    def __init__(self, ctx, rng, n, homogeneous_frac=0.0):
        self.wl = W.sphere_training_case(rng, n, homogeneous=bool(rng.random() < homogeneous_frac))
        self.lat = mpm.DeviceLattice(self.wl.lattice)
        self.prm = mpm.DeviceParams(self.wl.params)
        self.solver = mpm.StepSolver(ctx, self.lat, self.prm, self.wl.margin)
        self.age = 0


def train(ctx: mpm.Context, samples: int = 20000, batch: int = 8, n: int = 32, lr: float = 2e-3,
          traj_len: int = 12, seed: int = 4, params=None, log_every: int = 0, homogeneous_frac: float = 0.25):
    """Train a fresh network (or `params`) on `samples` pairs; returns (CNN, history).
    A fraction homogeneous_frac of the trajectories are homogeneous problems
    (zero sources and boundary values), whose pairs (v, A^-1 v) teach the
    network the map it applies as the FGMRES preconditioner."""
    rng = np.random.default_rng(seed)
    cnn = mpm.CNN(ctx, (n, n, n), batch, mpm.cnn_init_params(seed) if params is None else params, s_out=0.01,
                  train=True)
    trajs = [_Traj(ctx, rng, n, homogeneous_frac) for _ in range(batch)]
    opts = mpm.make_opts(rtol=1e-10, restart=16, maxit=500)
    box = ((0, 0, 0), (n, n, n))
    hist = []
    t0 = time.time()
    nsteps = max(1, samples // batch)
    for it in range(nsteps):
        for b, tr in enumerate(trajs):
            if tr.age >= traj_len:
                tr.solver.sub.destroy()
                trajs[b] = tr = _Traj(ctx, rng, n, homogeneous_frac)
            cnn.load_image(b, tr.lat, tr.prm, box, mpm.CNN_INPUT)
            tr.solver.step(opts)
            cnn.load_image(b, tr.lat, tr.prm, box, mpm.CNN_TARGET)
            tr.age += 1
        # cosine decay of the learning rate
        lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * it / nsteps))
        loss = cnn.train_step(batch, lr_t)
        hist.append(loss)
        if log_every and it % log_every == 0:
            print(f"step {it}/{nsteps} loss {loss:.3e} ({time.time() - t0:.1f} s)", flush=True)
    return cnn, {"loss": hist, "seconds": time.time() - t0, "samples": nsteps * batch}


def evaluate_sphere32(ctx: mpm.Context, cnn, rtol: float = 1e-6, precision: int = 0, steps: int = 10):
    """The 32^3 sphere workload advanced `steps` steps twice from the same state:
    with x0 = c^n and with x0 = the network's prediction.  Returns Arnoldi steps
    and device time (solve, plus the network's forward for the learned form)."""
    import torch
    wl = W.sphere32()
    out = {}
    for learned in (False, True):
        lat = mpm.DeviceLattice(wl.lattice)
        prm = mpm.DeviceParams(wl.params)
        sub = ctx.subgrid_create()
        its, ms, res = [], 0.0, []
        stream = torch.cuda.current_stream()
        for _ in range(steps):
            sub.mpm_box_extract(lat, 1, wl.margin)
            sub.mpm_assemble_coeffs(prm)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if learned:
                cnn.guess(sub, lat, prm)
            rep = sub.mpm_solve_step(mpm.make_opts(rtol=rtol, restart=30, maxit=500, precision=precision,
                                                   inner_rtol=1e-6, x0_given=int(learned)), scatter_to=lat)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            its.append(rep["iters"][0])
            res.append(rep["res"][0] / rep["bnorm"][0])
        out["learned" if learned else "plain"] = {"iters_per_step": float(np.mean(its)), "ms_per_step": ms / steps,
                                                 "max_rel_res": float(max(res)), "final": lat.fields_numpy()}
    return out


def evaluate_fgmres_sphere32(ctx: mpm.Context, cnn, rtol: float = 1e-6, steps: int = 10, restart: int = 8,
                             precision: int = 0, inner_rtol: float = 1e-6):
    """The 32^3 sphere workload advanced `steps` steps by flexible GMRES with the
    network as the right preconditioner (mpm_solve_fgmres_cnn; precision 1:
    FP32 cycles inside FP64 refinement), from x0 = c^n and from the learned
    guess.  Returns Arnoldi steps, the steps whose solve fell back to plain
    GMRES, and device time per step (extraction and assembly excluded, as in
    evaluate_sphere32)."""
    import torch
    wl = W.sphere32()
    out = {}
    for guess in (False, True):
        lat = mpm.DeviceLattice(wl.lattice)
        prm = mpm.DeviceParams(wl.params)
        sub = ctx.subgrid_create()
        its, ms, res, fb = [], 0.0, [], 0
        stream = torch.cuda.current_stream()
        for _ in range(steps):
            sub.mpm_box_extract(lat, 1, wl.margin)
            sub.mpm_assemble_coeffs(prm)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if guess:
                cnn.guess(sub, lat, prm)
            rep = cnn.solve_fgmres(sub, lat, prm, mpm.make_opts(rtol=rtol, restart=restart, maxit=500,
                                                                precision=precision, inner_rtol=inner_rtol,
                                                                x0_given=int(guess)), scatter_to=lat)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            its.append(rep["iters"][0])
            res.append(rep["res"][0] / rep["bnorm"][0])
            fb += rep["fallback"][0]
        out["guess_fgmres" if guess else "fgmres"] = {"iters_per_step": float(np.mean(its)),
                                                       "ms_per_step": ms / steps, "max_rel_res": float(max(res)),
                                                       "fallback_steps": fb, "final": lat.fields_numpy()}
    return out


def train_growth(ctx: mpm.Context, wl=None, extra=None, epochs: int = 4, lr: float = 2e-3, seed: int = 7,
                 params=None, rtol: float = 1e-10, log_every: int = 0, s_out: float = 0.01):
    """Train a network for the growing tumour on the trajectory of another
    instance of its geometry (workloads.growth_crop, seed 6 by default):
    `epochs` passes over its 200 steps; every step the tumour grows, the
    step's box (the allocation-free bounding box) and the features of c^n
    are loaded, the FP64 solver advances the lattice to c^{n+1} (rtol 1e-10,
    the target) and one Adam step follows.  Returns (CNN, history)."""
    import torch
    if wl is None:
        wl, extra = W.growth_crop()
    lat = mpm.DeviceLattice(wl.lattice)
    prm = mpm.DeviceParams(wl.params)
    init = lat.fields.clone()
    cand = torch.from_numpy(np.ascontiguousarray(extra["cand"])).cuda()
    labels = torch.from_numpy(extra["labels"].astype(np.int64)).cuda()
    cnn = mpm.CNN(ctx, wl.lattice.dims, 1, mpm.cnn_init_params(seed) if params is None else params, s_out=s_out,
                  train=True)
    solver = mpm.StepSolver(ctx, lat, prm, wl.margin)
    opts = mpm.make_opts(rtol=rtol, restart=16, maxit=500)
    out_box = torch.zeros(8, dtype=torch.int32, device="cuda")
    hist = []
    t0 = time.time()
    n_total = epochs * wl.steps
    it = 0
    for ep in range(epochs):
        lat.fields.copy_(init)
        for t in range(wl.steps):
            lo, hi = W.growth_box(t, wl.steps)
            lo, hi = lo - np.array(extra["origin"], float), hi - np.array(extra["origin"], float)
            inside = np.all((extra["seeds"] >= lo) & (extra["seeds"] < hi), axis=1)
            ids = torch.from_numpy(np.where(inside, np.arange(1, len(inside) + 1), 0).astype(np.int32)).cuda()
            lat.cell_id.view(-1)[cand] = ids[labels]
            st = mpm.mpm_box_bounds_noalloc(lat.cell_id, wl.margin, out_box)
            if st != mpm.OK:
                raise mpm.MpmError(st, "mpm_box_bounds_noalloc failed")
            o = out_box.cpu().numpy().tolist()
            if not o[6]:
                continue
            box = (tuple(o[0:3]), tuple(o[3:6]))
            cnn.load_image(0, lat, prm, box, mpm.CNN_INPUT)
            solver.step(opts)
            cnn.load_image(0, lat, prm, box, mpm.CNN_TARGET)
            lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * it / n_total))
            hist.append(cnn.train_step(1, lr_t))
            it += 1
            if log_every and it % log_every == 0:
                print(f"epoch {ep} step {t} loss {hist[-1]:.3e} ({time.time() - t0:.1f} s)", flush=True)
    return cnn, {"loss": hist, "seconds": time.time() - t0, "samples": it}
