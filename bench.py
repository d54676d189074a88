#!/usr/bin/env python3
"""Benchmark of the box-restricted implicit-Euler reaction-diffusion step.

Metric: species-voxel-steps/s at 1e-6 relative residual (sum over steps and
species of the in-mask voxels of the box, per second), plain FP64 GMRES against
the learned + mixed-precision form (the network's guess, then FP32 GMRES inside
FP64 refinement), on the full growing tumour: a 512x384x384 int32 CPM lattice
with a pleural-shell mask whose tumour grows so the bounding box (margin 4)
expands from ~61^3 to 302x264x264 voxels over 200 steps, re-extracted every
step, 3 species.

One bench step = one implicit-Euler step of the whole hot path through the C
ABI (mpm_step_enqueue): bounding box, tile compaction, gather + assembly, [the
network's guess,] GMRES for the three species and the scatter onto the mask,
all in one CUDA graph.  The K timed steps are sampled evenly over the 200-step
growth (t = 0, 200/K, ...); the tumour of step t is set on the device before
the step, outside the timing.  The lattice is resident in HBM (2.2 GB, larger
than L2) and L2 is flushed (256 MB write) before every timed step; every timed
step's report is checked (status, true FP64 residual <= 1e-6 ||b||).  `e2e`
repeats sampled steps through mpm_step_host with the lattice in pinned host
memory.  The network is trained first, on the trajectory of another instance
of the geometry (seed 6), by the library's own kernels.

--impl reference times the CPU oracle (single thread) on the first K steps of
the same workload (a bounded sample: the late steps' boxes take the oracle
seconds each).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "species-voxel-steps/s at 1e-6 rel. residual: plain FP64 GMRES vs learned+mixed"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def solver_bytes(rep, NM, NE, bT):
    """Algorithmic bytes of one solver launch: per in-mask voxel (the unknowns,
    NM) and species, R = x, b, diag64 (8 each) + write u0 (bT);
    P1_j = u_j, diag, u_0..u_{j-1} + write w = (j+3) bT; P2_j = read w,
    u_0..u_j + write w = (j+3) bT; U = read V (k bT) + x r/w (16); plus the
    flag byte of every stored element (NE) in every pass."""
    tot = 0
    for s in range(len(rep["iters"])):
        it, C, js = rep["iters"][s], rep["cycles"][s], rep["jsum"][s]
        R = 24 + bT
        P = it * 6 * bT + 2 * bT * js
        U = 16 * C + bT * it
        passes = (C + 1) + 2 * it + C
        tot += NM * (R * (C + 1) + P + U) + NE * passes
    return tot


def step_bytes(rep, L, S, bT, tile_vol=64):
    """Algorithmic bytes of one device-resident step (one kernel): the bounding
    box reads the int32 lattice (4 B per voxel); the tile activity reads the box
    mask (1 B per box voxel); the gather + rows read mask, cell id and S fields
    and write flags, cell id and per species x, c^n, b, diag (8 B) and the FP32
    diag (4 B) of every stored element, plus per active tile its coordinates,
    index and neighbour table (44 B); the solve is solver_bytes; the scatter
    reads flags and x and writes the fields of the in-mask voxels."""
    NM, NE, box = rep["mask_voxels"], rep["stored_voxels"], rep["box_voxels"]
    extract = 4 * L + box + NE * (1 + 4 + 8 * S) + NE * (5 + 36 * S) + (NE // tile_vol) * 44
    scatter = NE + NM * 16 * S
    return extract + solver_bytes(rep, NM, NE, bT) + scatter


def solver_fp64_ops(rep, NM, fp32):
    """FP64 instructions of one solver launch per the same pass structure (an FMA,
    an add or a convert each count one): R 10; FP64 path P1_j 8 + (j+1), P2_j
    (j+2), U k; FP32 path U 1 per cycle (x += d)."""
    tot = 0
    for s in range(len(rep["iters"])):
        it, C, js = rep["iters"][s], rep["cycles"][s], rep["jsum"][s]
        r = 10 * (C + 1)
        if fp32:
            r += 2 * C
        else:
            r += it * 8 + (js + it) + (js + 2 * it) + it
        tot += NM * r
    return tot


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def replica_value(units: float, ms_local: float, world: int, device=None):
    """Whole-job throughput of N independent replicas: every rank processed
    `units` in `ms_local` ms; the job time is the maximum over ranks (one
    all-reduce, measurement only) and value = world * units / t_max."""
    t = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return world * units / (t / 1e3), t


def _timed(fn, stream, flush, i):
    import torch
    flush.fill_(i & 255)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    out = fn()
    b.record(stream)
    b.synchronize()
    return out, a.elapsed_time(b)


def _timed_queued(solver, opts, stream, flush, i):
    """One device-resident step queued behind its L2 flush (68 us of device work,
    longer than the host's work to queue the step) and bracketed by its own
    events, so the host's per-step work stays off the timeline; then waited for."""
    import torch
    flush.fill_(i & 255)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    solver.step_async(opts)
    b.record(stream)
    rep = solver.wait()
    b.synchronize()
    return rep, a.elapsed_time(b)


def bench_sphere32(mpm, W, ctx, stream, flush, warmup):
    """32^3 single species, FP64 GMRES(30) to 1e-10 relative, 10 steps."""
    wl = W.sphere32()
    lat = mpm.DeviceLattice(wl.lattice)
    init = lat.fields.clone()
    solver = mpm.StepSolver(ctx, lat, mpm.DeviceParams(wl.params), wl.margin)
    opts = mpm.make_opts(rtol=wl.rtol, restart=wl.restart, maxit=1000)
    for _ in range(warmup):
        solver.step(opts)
    lat.fields.copy_(init)
    ms, units, its = 0.0, 0, []
    for i in range(wl.steps):
        # queued step (its events bracket only the step), then waited for: the
        # residual of every step is checked
        rep, t = _timed_queued(solver, opts, stream, flush, i)
        assert rep["status_code"] == mpm.OK and rep["res"][0] <= wl.rtol * rep["bnorm"][0]
        ms += t
        units += rep["mask_voxels"]
        its.append(rep["iters"][0])
    return {"value": units / (ms / 1e3), "unit": "species-voxel-steps/s", "ms_per_step": ms / wl.steps,
            "path": "FP64 GMRES(30), rtol 1e-10", "steps": wl.steps, "iters_per_step": sum(its) / len(its)}


def bench_patches64(mpm, W, ctx, stream, flush, warmup, steps=50):
    """64 uneven pleural-shell patches x 3 species: one graph-replayed batched step
    (refresh, assemble, one persistent solve of all 192 systems, scatter),
    tiles and restart/variant from the tuner, FP32 inside FP64 refinement."""
    ps = W.patches()
    lats = [mpm.DeviceLattice(p.lattice) for p in ps]
    inits = [l.fields.clone() for l in lats]
    prms = [mpm.DeviceParams(p.params) for p in ps]
    bs = mpm.BatchStepper(ctx, lats, prms, [p.margin for p in ps], tune_tiles=True)
    opts = mpm.make_opts(rtol=1e-6, restart=8, maxit=1000, precision=1, inner_rtol=1e-6)
    m, var = bs.tune(opts)
    for _ in range(warmup):
        bs.step(opts)
    for l, f in zip(lats, inits):
        l.fields.copy_(f)
    ms, units, imb = 0.0, 0, []
    for i in range(steps):
        (st, reps), t = _timed(lambda: bs.step(opts), stream, flush, i)
        assert st == mpm.OK
        ms += t
        units += sum(r["mask_voxels"] * 3 for r in reps)
        imb.append(ctx.imbalance())
    stored = sum(r["stored_voxels"] for r in reps)
    return {"value": units / (ms / 1e3), "unit": "species-voxel-steps/s", "ms_per_step": ms / steps, "steps": steps,
            "systems": 3 * len(ps), "tuned": {"restart": m, "variant": var,
                                              "tiles": sorted(set(map(tuple, bs.tiles)))},
            "graph": bs.graph_active(), "stored_voxels": stored,
            "team_model": {"f_per_tuning_round": bs.team_tuning["f"],
                           "fixed_F1_F_per_round": bs.team_tuning["fixed_per_round"],
                           "kept_F1_F": bs.team_tuning["fixed"],
                           "note": "mpm_tune_teams: item cost it (F1 + NE) on one CTA, it (F + NE / c) on c > 1, "
                                   "F1 and F fitted to measured item times, it from the previous solve; round 0 is "
                                   "the unmeasured model"},
            "imbalance_f": {"mean": float(np.mean(imb)), "max": float(np.max(imb)),
                            "definition": "t_max/<t> - 1 over the CTA teams of the persistent launch"},
            "mask_voxels": sum(r["mask_voxels"] for r in reps)}


C5_STEPS = 200
CNN_FLOPS_PER_VOXEL = 2 * 27 * (9 * 24 + 4 * 24 * 24 + 24 * 3)   # 139 968: the network's convolutions


def c5_schedule(K):
    """The K sampled steps of the 200-step growth."""
    return [int(k * C5_STEPS // K) for k in range(K)]


def c5_workload(K):
    ts = c5_schedule(K)
    return ("growth512: 512x384x384 int32 CPM lattice, pleural-shell mask (ellipsoids 230/175/175 and "
            "215/160/160), ~9.8k Voronoi tumour cells growing so the bbox+4 expands from 61x87x83 to "
            f"302x264x264 over 200 steps, re-extracted every step; {K} steps sampled at t = "
            f"{ts[0]}, {ts[1] if K > 1 else ts[0]}, ..., {ts[-1]} (every {C5_STEPS / K:g}); 3 species, "
            "D=(1,0.5,0.2), dt=0.05, per-cell rates U[0.01,0.1], rtol 1e-6")


class Growth:
    """The growing tumour and its device-side tumour update."""

    def __init__(self, W):
        import torch
        self.W = W
        self.wl, self.extra = W.growth512()
        self.cand = torch.from_numpy(self.extra["cand"]).cuda()
        self.labels = torch.from_numpy(self.extra["labels"].astype(np.int64)).cuda()

    def set_tumour(self, lat, t):
        import torch
        lo, hi = self.W.growth_box(t, self.wl.steps)
        inside = np.all((self.extra["seeds"] >= lo) & (self.extra["seeds"] < hi), axis=1)
        ids = torch.from_numpy(np.where(inside, np.arange(1, len(inside) + 1), 0).astype(np.int32)).cuda()
        lat.cell_id.view(-1)[self.cand] = ids[self.labels]


def c5_tile(mpm, g, ctx):
    """The tile of the growing tumour's steps: the tuner's pick (the tile
    storing the fewest voxels, mpm_tune_tile) on the largest, last state."""
    lat = mpm.DeviceLattice(g.wl.lattice)
    g.set_tumour(lat, C5_STEPS - 1)
    tile, stored = ctx.mpm_tune_tile(lat, g.wl.margin)
    del lat
    return tile, stored


def run_c5_path(mpm, g, ctx, stream, flush, opts, K, warmup, cnn=None, sampler=None, tile=None):
    """K sampled steps of the growing tumour on one path, every report checked."""
    import torch
    wl = g.wl
    lat = mpm.DeviceLattice(wl.lattice)
    init = lat.fields.clone()
    prm = mpm.DeviceParams(wl.params)
    solver = mpm.StepSolver(ctx, lat, prm, wl.margin, tile=tile)
    if cnn is not None:
        solver.set_network(cnn)
    g.set_tumour(lat, 0)
    for _ in range(warmup):
        solver.step(opts)
    lat.fields.copy_(init)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    l0 = ctx.launches()
    ms, units, reps, its = 0.0, 0, [], []
    kbytes = kops = 0
    bT = 4 if opts.precision else 8
    L = wl.lattice.cell_id.size
    for i, t in enumerate(c5_schedule(K)):
        g.set_tumour(lat, t)
        rep, dt = _timed_queued(solver, opts, stream, flush, i)
        assert rep["status_code"] == mpm.OK, (t, rep)
        assert all(r <= wl.rtol * b for r, b in zip(rep["res"], rep["bnorm"])), (t, rep)
        ms += dt
        units += rep["mask_voxels"] * wl.params.nspecies
        kbytes += step_bytes(rep, L, wl.params.nspecies, bT, int(np.prod(tile)) if tile else 64)
        kops += solver_fp64_ops(rep, rep["mask_voxels"], bool(opts.precision))
        reps.append(rep)
        its.append(sum(rep["iters"]) / len(rep["iters"]))
    launches = ctx.launches() - l0
    clocks = sampler.stop() if sampler else None
    # after the timed steps: one more step on the last state with the phase
    # timers on (CTA 0's split of the step: extraction, the solver's passes and
    # its waits), not part of any timed figure
    ctx.debug_set(mpm.DEBUG_PHASE_TIMES, 1)
    prep = solver.step(opts)
    phases = {k: round(v, 1) for k, v in ctx.phase_times_us().items()}
    phases["iters"] = prep["iters"]
    ctx.debug_set(mpm.DEBUG_PHASE_TIMES, 0)
    # the solver phase alone on the last state (CTA 0's team time "work"; the
    # three species' teams run side by side): its FP64 instructions per the
    # pass model over the in-mask unknowns (algorithmic) and over every stored
    # element (what the passes execute), and its algorithmic bytes, against
    # the whole GPU's FP64 issue rate at 2070 MHz and the measured HBM peak
    sec = phases["work"] * 1e-6
    fp32 = bool(opts.precision)
    if sec > 0:
        pk = fp64_peak_instr(2070.0)
        phases["solver_fp64_frac_algorithmic"] = solver_fp64_ops(prep, prep["mask_voxels"], fp32) / sec / pk
        phases["solver_fp64_frac_executed"] = solver_fp64_ops(prep, prep["stored_voxels"], fp32) / sec / pk
        phases["solver_hbm_frac"] = (solver_bytes(prep, prep["mask_voxels"], prep["stored_voxels"], 4 if fp32 else 8)
                                     / sec / 1e9 / _peaks()[0])
        phases["stored_mask_box"] = [prep["stored_voxels"], prep["mask_voxels"], prep["box_voxels"]]
    out = {"value": units / (ms / 1e3), "ms_per_step": ms / K, "steps_checked": len(reps),
           "phase_us_last_state": phases,
           "arnoldi_steps_per_species_step": float(np.mean(its)), "kernel_ms": ms, "kernel_bytes": kbytes,
           "kernel_fp64_ops": kops, "units": units, "launches": launches,
           "box_voxels_first_last": [reps[0]["box_voxels"], reps[-1]["box_voxels"]],
           "mask_voxels_first_last": [reps[0]["mask_voxels"], reps[-1]["mask_voxels"]],
           "max_rel_res": max(r / b for rep in reps for r, b in zip(rep["res"], rep["bnorm"]))}
    return out, clocks, (solver, lat, prm, init)


def run_c5_fgmres(mpm, g, ctx, stream, flush, okw, K, warmup, cnn, tile=None):
    """K sampled steps of the growing tumour by flexible GMRES with the network
    as the right preconditioner from its guess (mpm_solve_fgmres_cnn, one
    graph per solve): extraction, assembly, guess, solve and scatter per step,
    timed by CUDA events around the step (the solve's one host wait for its
    report included), every report checked."""
    import torch
    wl = g.wl
    lat = mpm.DeviceLattice(wl.lattice)
    init = lat.fields.clone()
    prm = mpm.DeviceParams(wl.params)
    sub = ctx.subgrid_create()
    S = wl.params.nspecies
    opts = mpm.make_opts(x0_given=1, **okw)

    def one():
        sub.mpm_box_extract(lat, S, wl.margin, tile=tile)
        sub.mpm_assemble_coeffs(prm)
        cnn.guess(sub, lat, prm)
        return cnn.solve_fgmres(sub, lat, prm, opts, scatter_to=lat)

    g.set_tumour(lat, 0)
    for _ in range(warmup):
        one()
    lat.fields.copy_(init)
    torch.cuda.synchronize()
    l0 = ctx.launches()
    ms, units, its, fb, mx = 0.0, 0, [], 0, 0.0
    for i, t in enumerate(c5_schedule(K)):
        g.set_tumour(lat, t)
        flush.fill_(i & 255)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rep = one()
        b.record(stream)
        b.synchronize()
        assert rep["status_code"] == mpm.OK, (t, rep)
        assert all(r <= wl.rtol * bb for r, bb in zip(rep["res"], rep["bnorm"])), (t, rep)
        ms += a.elapsed_time(b)
        units += rep["mask_voxels"] * S
        its.append(sum(rep["iters"]) / S)
        fb += sum(rep["fallback"])
        mx = max(mx, max(r / bb for r, bb in zip(rep["res"], rep["bnorm"])))
    out = {"value": units / (ms / 1e3), "ms_per_step": ms / K, "steps_checked": K,
           "arnoldi_steps_per_species_step": float(np.mean(its)),
           "network_applications_per_step": float(np.mean(its)) * S + 1,
           "fallback_solves": fb, "solves": K * S, "max_rel_res": mx, "launches": ctx.launches() - l0}
    sub.destroy()
    del lat
    return out


def bench_growth_cpm(mpm, W, ctx, stream, flush, K, warmup):
    """The 512x384x384 tumour grown by the device growth driver instead of the
    script: from the scripted initial tumour (t = 0), K steps of (growth +
    mitosis launches, then the device-resident FP32-in-FP64 step with the box
    re-extracted), both queued on one stream between CUDA events; every step's
    report checked."""
    import torch
    wl, extra = W.growth512()
    W.grow(wl, 0, extra)
    ncell0 = wl.params.ncell
    wl.params = W.with_capacity(wl.params, 8 * ncell0)
    lat = mpm.DeviceLattice(wl.lattice)
    prm = mpm.DeviceParams(wl.params)
    drv = mpm.GrowthDriver(ctx, lat, prm, ncell0, p_grow=0.6, K_o2=0.2, K_nut=0.3, o2_min=0.05, v_div=400, seed=2026)
    solver = mpm.StepSolver(ctx, lat, prm, wl.margin)
    opts = mpm.make_opts(rtol=wl.rtol, restart=8, maxit=1000, precision=1, inner_rtol=1e-6)
    for _ in range(warmup):
        solver.step(opts)
    ms_cpm = ms_pde = 0.0
    units = 0
    boxes = []
    for i in range(K):
        flush.fill_(i & 255)
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        drv.step(stream=stream)
        b.record(stream)
        solver.step_async(opts)
        c.record(stream)
        rep = solver.wait()
        c.synchronize()
        assert rep["status_code"] == mpm.OK, (i, rep)
        assert all(r <= wl.rtol * bb for r, bb in zip(rep["res"], rep["bnorm"])), (i, rep)
        ms_cpm += a.elapsed_time(b)
        ms_pde += b.elapsed_time(c)
        units += rep["mask_voxels"] * wl.params.nspecies
        boxes.append(rep["box_voxels"])
    cnt = drv.counts()
    out = {"value": units / (ms_pde / 1e3), "unit": "species-voxel-steps/s", "pde_ms_per_step": ms_pde / K,
           "growth_ms_per_step": ms_cpm / K, "steps_checked": K, "box_voxels_first_last": [boxes[0], boxes[-1]],
           "cells_first_last": [ncell0 - 1, cnt["ncell"] - 1], "grown_voxels": cnt["grown"],
           "divisions": cnt["divisions"],
           "driver": "mpm_cpm_step: growth into the mask with p = 0.6 c_O/(0.2 + c_O) c_n/(0.3 + c_n) (0 below "
                     "c_O = 0.05), mitosis at 400 voxels, SplitMix64 counter draws (seed 2026)",
           "path": "FP32 GMRES(8) inside FP64 refinement, device-resident step, rtol 1e-6"}
    del solver, drv, lat
    return out


def fp64_peak_instr(sm_mhz, nsm=152):
    """FP64 thread-instructions per second the SMs can issue: 2 per clock per SM
    (GB300's FP64 rate, 1.25 TFLOP/s counting an FMA as 2 flops, at 2.07 GHz)."""
    return 2.0 * nsm * sm_mhz * 1e6


def cnn_guess_time(mpm, ctx, cnn, solver, stream, flush, reps=3):
    """Device time of the network's guess alone (plan, features, six
    convolutions) on the subgrid's current extraction: mpm_cnn_guess bracketed
    by CUDA events after an L2 flush, median of `reps`."""
    import torch
    ts = []
    for i in range(reps + 1):
        flush.fill_(i & 255)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        cnn.guess(solver.sub, solver.lat, solver.prm)
        b.record(stream)
        b.synchronize()
        if i:
            ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def cnn_layer_roofline(mpm, ctx, cnn, solver, stream, flush, active, reps=5):
    """Roofline of the headline's dominant kernel, the hidden-layer convolution
    k_conv_tc<24, 32, 0> (four of the guess's six launches): CUDA events around
    each convolution launch of the guess on the last state (the library records
    them on the guess's stream, MPM_DEBUG_CNN_LAYER_TIMES), median over `reps`
    guesses after L2 flushes; algorithmic flops per launch = active voxels x 27 x
    24 x 24 x 2.  DRAM traffic per launch: the committed ncu record of that
    kernel (a capture on the crop's largest state) scaled by the active voxels,
    valid while the kernel sources are unchanged."""
    import torch
    ctx.debug_set(mpm.DEBUG_CNN_LAYER_TIMES, 1)
    per = []
    for i in range(reps):
        flush.fill_(i & 255)
        cnn.guess(solver.sub, solver.lat, solver.prm)
        per.append(cnn.layer_times())
    ctx.debug_set(mpm.DEBUG_CNN_LAYER_TIMES, 0)
    med = [float(np.median([p[l] for p in per])) for l in range(6)]
    hid = float(np.mean(med[1:5]))
    flops = active * 27 * 24 * 24 * 2
    achieved = flops / (hid / 1e3) / 1e12
    rec = _traffic_record_cnn()
    traffic = rec["dram_bytes_per_launch"] * active / rec["active_voxels"] if rec else None
    return {"bound": "tensor", "kernel": "k_conv_tc<24, 32, 0> (hidden-layer 3x3x3 convolution, tcgen05)",
            "achieved": achieved, "peak": 1980.0, "unit": "TFLOP/s", "frac": achieved / 1980.0,
            "traffic": traffic, "flops_per_launch": flops, "ms_per_launch": hid, "layer_ms": med,
            "peak_source": "measured bf16 burst (MEASURED_PEAKS.json bf16_tflops)",
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the same kernel on the "
                               "growth crop's largest state, scaled by active voxels (profiles/conv_tc_traffic.json)"
                               if rec else "no record for the current kernel sources")}


def _traffic_record_cnn():
    p = os.path.join(ROOT, "profiles", "conv_tc_traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    h = hashlib.sha256()
    for f in ("cnn_tc.cuh",):
        h.update(open(os.path.join(ROOT, "paper_2505_03067_gb300", "csrc", f), "rb").read())
    return d if d.get("source_sha256") == h.hexdigest() else None


def bench_learned(mpm, ctx, samples=20000):
    """The learned solver: train the network on `samples` pairs generated by the
    FP64 solver on the GPU (32^3 sphere-like lattices, a quarter of them
    homogeneous problems), then time the 32^3 sphere workload to 1e-6 with
    x0 = c^n and with x0 = the network's prediction, FP64 and FP32-in-FP64
    (device time includes features + forward), and with flexible GMRES using
    the network as the right preconditioner (from c^n and from the guess)."""
    from paper_2505_03067_gb300 import learned
    cnn, hist = learned.train(ctx, samples=samples)
    out = {"train_seconds": hist["seconds"], "samples": hist["samples"],
           "loss_first_last": [float(np.mean(hist["loss"][:5])), float(np.mean(hist["loss"][-20:]))]}
    for name, prec in (("fp64", 0), ("mixed", 1)):
        ev = learned.evaluate_sphere32(ctx, cnn, rtol=1e-6, precision=prec)
        for k in ("plain", "learned"):
            e = ev[k]
            out[f"{name}_{k}"] = {"value": 32 ** 3 / (e["ms_per_step"] / 1e3), "ms_per_step": e["ms_per_step"],
                                  "iters_per_step": e["iters_per_step"], "max_rel_res": e["max_rel_res"]}
    # row a13: flexible GMRES with the network as the right preconditioner,
    # device-resident (one graph per solve), FP64 and FP32 cycles in FP64 refinement
    for name, prec in (("fp64", 0), ("mixed", 1)):
        ev = learned.evaluate_fgmres_sphere32(ctx, cnn, rtol=1e-6, precision=prec)
        for k in ("fgmres", "guess_fgmres"):
            e = ev[k]
            out[f"{name}_{k}"] = {"value": 32 ** 3 / (e["ms_per_step"] / 1e3), "ms_per_step": e["ms_per_step"],
                                  "iters_per_step": e["iters_per_step"], "max_rel_res": e["max_rel_res"],
                                  "fallback_steps": e["fallback_steps"]}
    cnn.close()
    return out


def oracle_c5_steps(W, nsteps):
    """The oracle on the first nsteps steps of the growing tumour (t = 0, 1, ...)."""
    import oracle
    wl, extra = W.growth512()
    lat = wl.lattice
    units = 0
    dt = 0.0
    for t in range(nsteps):
        W.grow(wl, t, extra)
        t0 = time.perf_counter()
        rep = oracle.step(lat, wl.params, wl.margin, rtol=wl.rtol, restart=wl.restart)
        dt += time.perf_counter() - t0
        units += rep["mask_voxels"] * wl.params.nspecies
    return units, dt


def cpu_baseline(W, nsteps):
    import oracle
    oracle.build()
    units, dt = oracle_c5_steps(W, nsteps)
    return {"value": units / dt, "unit": "species-voxel-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"the first {nsteps} implicit-Euler steps (t = 0..{nsteps - 1}) of growth512 (all 3 species, "
                      f"every in-mask voxel of the box), single-threaded C/NumPy oracle (gcc "
                      f"{' '.join(oracle.BUILD_FLAGS)}), GMRES(30) to 1e-6, {dt:.2f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_2505_03067_gb300 import workloads as W
    import oracle
    oracle.build()
    units, _ = oracle_c5_steps(W, min(args.warmup, 2))   # warm-up (loads, first touches)
    units, dt = oracle_c5_steps(W, args.steps)
    v = units / dt
    line = {"metric": METRIC, "value": v, "unit": "species-voxel-steps/s", "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": c5_workload(args.steps),
                       "path": "CPU oracle, FP64 MGS-GMRES(30)",
                       "sample": f"the first {args.steps} steps of the 200-step growth (t = 0..{args.steps - 1}): "
                                 "the bounded sample of the same workload"},
            "cpu_baseline": {"value": v, "unit": "species-voxel-steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {args.steps} implicit-Euler steps of growth512 (single-threaded "
                                       f"oracle, gcc {' '.join(oracle.BUILD_FLAGS)})"},
            "e2e": {"value": v, "unit": "species-voxel-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def bench_shell256(mpm, W, ctx, stream, flush, K, warmup):
    """The 256^3 pleural shell (2000 Voronoi tumour cells, 20 steps): plain
    FP64 against FP32 GMRES(8) inside FP64 refinement, and the same with the
    box cadence of Sec. 2.3 (a full extraction every 50 steps, a 2-voxel
    guard band; this tumour does not move, so every timed step keeps the box).
    Every step's report is checked."""
    wl = W.shell256()
    S = wl.params.nspecies
    out = {}
    for name, extra in (("fp64", dict(precision=0)), ("mixed", dict(precision=1, inner_rtol=1e-6)),
                        ("mixed_cadence50", dict(precision=1, inner_rtol=1e-6, box_every=50, box_guard=2))):
        opts = mpm.make_opts(rtol=wl.rtol, restart=8, maxit=1000, **extra)
        lat = mpm.DeviceLattice(wl.lattice)
        init = lat.fields.clone()
        solver = mpm.StepSolver(ctx, lat, mpm.DeviceParams(wl.params), wl.margin)
        for _ in range(warmup):
            solver.step(opts)
        lat.fields.copy_(init)
        ms, units, kbytes, kops = 0.0, 0, 0, 0
        bT = 4 if extra["precision"] else 8
        for i in range(K):
            rep, t = _timed_queued(solver, opts, stream, flush, i)
            assert rep["status_code"] == mpm.OK, rep
            assert all(r <= wl.rtol * b for r, b in zip(rep["res"], rep["bnorm"])), rep
            ms += t
            units += rep["mask_voxels"] * S
            kbytes += step_bytes(rep, wl.lattice.cell_id.size, S, bT)
            kops += solver_fp64_ops(rep, rep["mask_voxels"], bool(extra["precision"]))
        out[name] = {"value": units / (ms / 1e3), "ms_per_step": ms / K, "steps_checked": K,
                     "iters_last_step": rep["iters"], "box_voxels": rep["box_voxels"],
                     "mask_voxels": rep["mask_voxels"], "stored_voxels": rep["stored_voxels"],
                     "achieved_gbs": kbytes / (ms / 1e3) / 1e9, "fp64_tinstr": kops / (ms / 1e3) / 1e12}
        del solver, lat
    return {"unit": "species-voxel-steps/s", "paths": out,
            "workload": "shell256: 256^3 lattice, pleural shell (110/90/120, 100/80/110), 2000 Voronoi tumour "
                        f"cells in a 128x128x96 region, bbox+4, 3 species, dt=0.05, {K} implicit-Euler steps, rtol 1e-6"}


def cnn_only(args):
    """The network alone: the guess (plan, features, six tcgen05 convolutions)
    on the growing tumour's training crop (324x264x264, about 4 GB on the
    device) at its last, largest step, `--steps` launches after `--warmup`,
    each timed by CUDA events after an L2 flush.  Prints one JSON line (not
    the benchmark's line): a small case to profile the convolution kernels."""
    import torch
    from paper_2505_03067_gb300 import mpm
    from paper_2505_03067_gb300 import workloads as W
    wl, extra = W.growth_crop()
    W.grow(wl, wl.steps - 1, extra)
    ctx = mpm.Context()
    lat = mpm.DeviceLattice(wl.lattice)
    prm = mpm.DeviceParams(wl.params)
    sub = ctx.subgrid_create()
    sub.mpm_box_extract(lat, wl.params.nspecies, wl.margin)
    sub.mpm_assemble_coeffs(prm)
    act = sub.info()["mask_voxels"]
    cnn = mpm.CNN(ctx, wl.lattice.dims, 1, mpm.cnn_init_params(7), s_out=0.01)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ts = []
    for i in range(args.warmup + args.steps):
        flush.fill_(i & 255)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        cnn.guess(sub, lat, prm)
        b.record(stream)
        b.synchronize()
        if i >= args.warmup:
            ts.append(a.elapsed_time(b))
    ms = float(np.median(ts))
    print(json.dumps({"mode": "cnn_only", "workload": "growth_crop seed 6 at t = 199 (324x264x264 lattice)",
                      "active_voxels": act, "ms_per_guess_median": ms, "launches_timed": args.steps,
                      "tflops": act * CNN_FLOPS_PER_VOXEL / (ms / 1e3) / 1e12}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=40)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--restart", type=int, default=8)
    ap.add_argument("--c5-epochs", type=int, default=3, help="passes over the training trajectory (200 steps each)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-workloads", action="store_true", help="skip the 256^3, 32^3, 64-patch sub-lines")
    ap.add_argument("--train-samples", type=int, default=20000)
    ap.add_argument("--cnn-only", action="store_true", help="time the network alone on a small case (profiling)")
    ap.add_argument("--shell256-only", action="store_true",
                    help="the 256^3 shell sub-line alone (FP64, mixed, cadence paths; a few GB: profiling)")
    ap.add_argument("--c5-only", choices=["fp64", "mixed"], default=None,
                    help="one path of the growing tumour alone, no network (profiling the step kernel)")
    ap.add_argument("--c5-tile", choices=["tuned", "default"], default="tuned",
                    help="tile of the growing tumour's steps: the tuner's pick on the last state, or 4x4x4")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.cnn_only:
        return cnn_only(args)
    if args.c5_only:
        import torch
        from paper_2505_03067_gb300 import mpm
        from paper_2505_03067_gb300 import workloads as W
        ctx = mpm.Context()
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        extra = dict(precision=0) if args.c5_only == "fp64" else dict(precision=1, inner_rtol=1e-6)
        g = Growth(W)
        opts = mpm.make_opts(rtol=g.wl.rtol, restart=args.restart, maxit=1000, **extra)
        tile = c5_tile(mpm, g, ctx)[0] if args.c5_tile == "tuned" else None
        res, _, _ = run_c5_path(mpm, g, ctx, torch.cuda.current_stream(), flush, opts, args.steps, args.warmup,
                                tile=tile)
        keys = ("value", "ms_per_step", "steps_checked", "arnoldi_steps_per_species_step", "phase_us_last_state")
        print(json.dumps({"mode": "c5_only", "path": args.c5_only, "tile": tile, **{k: res[k] for k in keys}}),
              flush=True)
        return 0
    if args.shell256_only:
        import torch
        from paper_2505_03067_gb300 import mpm
        from paper_2505_03067_gb300 import workloads as W
        ctx = mpm.Context()
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        print(json.dumps({"mode": "shell256_only", **bench_shell256(mpm, W, ctx, torch.cuda.current_stream(), flush,
                                                                     args.steps, args.warmup)}), flush=True)
        return 0

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    from paper_2505_03067_gb300 import learned, mpm
    from paper_2505_03067_gb300 import workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    ctx = mpm.Context()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    K = args.steps
    g = Growth(W)
    S = g.wl.params.nspecies

    # ---- the network of the learned form: trained on another instance of the
    # geometry (seed 6, cut to its growth region) by the library's kernels
    cnn_t, hist = learned.train_growth(ctx, epochs=args.c5_epochs)
    params, s_out = cnn_t.get(0), cnn_t.s_out
    cnn_t.close()
    torch.cuda.empty_cache()
    cnn = mpm.CNN(ctx, g.wl.lattice.dims, 1, params, s_out=s_out)
    training = {"trajectory": "growth_crop seed 6: the growth geometry with other cells and rates, 324x264x264 crop "
                              "of its growth region, 200 steps per epoch of the FP64 solver at rtol 1e-10",
                "epochs": args.c5_epochs, "adam_steps": hist["samples"], "seconds": hist["seconds"],
                "loss_first_last": ([float(np.mean(hist["loss"][:10])), float(np.mean(hist["loss"][-20:]))]
                                    if hist["loss"] else None)}

    # ---- the tile of every path: the tuner's pick on the largest state
    tile, tile_stored = c5_tile(mpm, g, ctx) if args.c5_tile == "tuned" else (None, None)

    # ---- the three paths on the same sampled steps
    peak, src = _peaks()
    mixed = dict(precision=1, inner_rtol=1e-6)
    plan = (("fp64", dict(precision=0), None), ("mixed", mixed, None), ("learned_mixed", mixed, cnn))
    results, clocks, keep = {}, None, None
    for name, extra, net in plan:
        opts = mpm.make_opts(rtol=g.wl.rtol, restart=args.restart, maxit=1000, **extra)
        headline = name == "learned_mixed"
        barrier()
        res, clk, kp = run_c5_path(mpm, g, ctx, stream, flush, opts, K, args.warmup, net,
                                   ClockSampler(local) if headline else None, tile=tile)
        barrier()
        _, ms_max = replica_value(res["units"], res["kernel_ms"], world, "cuda")
        res["value"] = replica_value(res["units"], ms_max, world)[0]
        if headline:
            clocks, keep = clk, (kp, opts)
            res["cnn_ms_last_step"] = cnn_guess_time(mpm, ctx, net, kp[0], stream, flush)
            res["roofline_conv"] = cnn_layer_roofline(mpm, ctx, net, kp[0], stream, flush,
                                                      res["mask_voxels_first_last"][1])
        else:
            del kp
        results[name] = res
        torch.cuda.empty_cache()

    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    for name, r in results.items():
        sec = r["kernel_ms"] / 1e3
        if name == "learned_mixed":
            # the network alone, timed on the last (largest) state; the rest of the step is the two step launches
            last_mask = r["mask_voxels_first_last"][1]
            t_cnn = r["cnn_ms_last_step"] / 1e3
            r["roofline_cnn"] = {"bound": "tensor", "kernel": "the network's guess on the last sampled state: plan, "
                                 "features and six tcgen05 convolutions (k_conv_tc)",
                                 "achieved": last_mask * CNN_FLOPS_PER_VOXEL / t_cnn / 1e12,
                                 "peak": 1980.0, "unit": "TFLOP/s", "peak_source": "measured bf16 burst "
                                 "(MEASURED_PEAKS.json bf16_tflops)",
                                 "flops_per_launch": last_mask * CNN_FLOPS_PER_VOXEL, "ms": r["cnn_ms_last_step"]}
            r["roofline_cnn"]["frac"] = r["roofline_cnn"]["achieved"] / 1980.0
        r["roofline_hbm"] = {"bound": "hbm", "achieved": r["kernel_bytes"] / sec / 1e9, "peak": peak, "unit": "GB/s",
                             "frac": r["kernel_bytes"] / sec / 1e9 / peak,
                             "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)",
                             "note": "algorithmic bytes of the step launches (extraction, solve, scatter) over the "
                                     "whole step's time" + (" including the network's" if name == "learned_mixed" else "")}
        pk = fp64_peak_instr(sm_mhz)
        r["roofline_fp64"] = {"bound": "fp64", "unit": "T FP64 instr/s", "achieved": r["kernel_fp64_ops"] / sec / 1e12,
                              "peak": pk / 1e12, "frac": r["kernel_fp64_ops"] / sec / pk,
                              "peak_source": "2 FP64 thread-instructions per clock per SM x 152 SMs at the median "
                                             "SM clock under load (the FP64 pipe: an ALU bound)"}

    head = results["learned_mixed"]
    # the dominant kernel of the headline step: the hidden-layer convolution
    # (four of the network's six launches) when the network takes at least
    # half the step, else the step launches' HBM roofline
    t_step_last = head["kernel_ms"] / K
    if head["cnn_ms_last_step"] >= 0.5 * t_step_last:
        roofline = dict(head["roofline_conv"])
    else:
        roofline = dict(head["roofline_hbm"])
        roofline["traffic"] = None

    # ---- end to end through the public API with host buffers (mpm_step_host)
    (solver, lat, prm, init), opts = keep
    wl, extra = g.wl, g.extra
    W.grow(wl, 0, extra)
    h_cell = torch.from_numpy(wl.lattice.cell_id).pin_memory()
    h_mask = lat.mask.cpu().pin_memory()
    h_fields = init.cpu().pin_memory()
    solver.step_host(h_cell, h_fields, opts, mask=h_mask, fields_in=True)
    barrier()
    ne = max(1, min(args.e2e_steps, K))
    e_ms, e_units, bo = 0.0, 0, 0
    for i, t in enumerate(c5_schedule(ne)):
        W.grow(wl, t, extra)
        h_cell.numpy()[...] = wl.lattice.cell_id
        flush.fill_(i & 255)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        erep = solver.step_host(h_cell, h_fields, opts)
        b.record(stream)
        b.synchronize()
        assert erep["status_code"] == mpm.OK, erep
        assert all(r <= wl.rtol * bb for r, bb in zip(erep["res"], erep["bnorm"])), erep
        e_ms += a.elapsed_time(b)
        e_units += erep["mask_voxels"] * S
        # pinned host fields: the step's in-mask voxels come back (8 B per species each)
        bo += S * 8 * erep["mask_voxels"]
    barrier()
    e2e_value, _ = replica_value(e_units, e_ms, world, "cuda")
    e2e = {"value": e2e_value, "unit": "species-voxel-steps/s", "h2d_bytes_per_step": h_cell.numel() * 4,
           "d2h_bytes_per_step": bo // ne, "steps": ne,
           "note": f"mpm_step_host per step (one synchronous C-ABI call, learned + mixed path) at {ne} steps sampled "
                   "over the growth: the 512x384x384 int32 cell-id lattice copied in from pinned host memory, the "
                   "step, and the voxels the step updated (the in-mask voxels of its box) of the 3 FP64 fields written back "
                   "to the pinned host fields by a kernel; the mask "
                   "and the initial fields went in once before the timed steps"}
    del solver, lat

    keys = ("value", "ms_per_step", "steps_checked", "arnoldi_steps_per_species_step", "max_rel_res",
            "box_voxels_first_last", "mask_voxels_first_last", "roofline_hbm", "roofline_fp64",
            "phase_us_last_state")
    paths = {k: {kk: v[kk] for kk in keys} for k, v in results.items()}
    paths["learned_mixed"]["roofline_cnn"] = head["roofline_cnn"]
    paths["learned_mixed"]["roofline_conv"] = head["roofline_conv"]
    paths["learned_mixed"]["cnn_ms_last_step"] = head["cnn_ms_last_step"]
    # row a13 on the same steps: the network as the right preconditioner of
    # FP32 flexible GMRES inside FP64 refinement, from its guess
    barrier()
    paths["learned_fgmres_mixed"] = run_c5_fgmres(
        mpm, g, ctx, stream, flush, dict(rtol=g.wl.rtol, restart=args.restart, maxit=1000, **mixed), K,
        args.warmup, cnn, tile=tile)
    barrier()
    line = {"metric": METRIC, "value": head["value"], "unit": "species-voxel-steps/s", "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64 + bf16 network",
            "data": "synthetic",
            "config": {"workload": c5_workload(K),
                       "path": "learned_mixed: the network's guess (trained on seed 6), then FP32 GMRES(8) inside "
                               "FP64 refinement (inner cycle to max(tol/4, 1e-6 ||r||)); compared with plain FP64 "
                               "GMRES(8) (paths.fp64) and FP32-in-FP64 from c^n (paths.mixed) on the same steps",
                       "step": "mpm_step_enqueue: one CUDA graph per step (extraction + assembly launch, the network, "
                               "persistent GMRES + scatter launch)",
                       "tile": {"xyz": tile or [4, 4, 4], "source": ("mpm_tune_tile on the last state (fewest stored "
                                                                       f"voxels: {tile_stored})") if tile else "default"},
                       "l2": "flushed (256 MB write) before every timed step; lattice (2.2 GB) > L2",
                       "network_training": training, "parallelism": f"replicas x{world}"},
            "paths": paths, "roofline": roofline, "e2e": e2e, "gpu_launches": head["launches"], "clocks": clocks}
    if not args.no_workloads:
        line["workloads"] = {"growth512_cpm": bench_growth_cpm(mpm, W, ctx, stream, flush, 50, args.warmup),
                             "shell256": bench_shell256(mpm, W, ctx, stream, flush, 20, args.warmup),
                             "sphere32": bench_sphere32(mpm, W, ctx, stream, flush, args.warmup),
                             "patches64": bench_patches64(mpm, W, ctx, stream, flush, args.warmup),
                             "learned_sphere32": bench_learned(mpm, ctx, args.train_samples)}
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(W, args.cpu_steps)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
