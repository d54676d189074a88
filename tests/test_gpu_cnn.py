"""The learned warm start's network on the GPU (bf16 tensor-core convolutions,
FP32 accumulation) against the FP64 CNN oracle with the GPU's bf16 storage
points reproduced: forward, every parameter gradient, Adam, training, and the
network's prediction used as the solver's initial guess."""
import numpy as np
import pytest

import oracle
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


def _case(M, ctx, seed, dims, batch):
    """Features and fields of `batch` random lattices of dims (x fastest)."""
    import torch
    xs, fs, wls = [], [], []
    for b in range(batch):
        wl = W.random_case(seed + b, dims, nspecies=3, blob=True)
        wl.lattice.fields[2] *= 0.05
        lat = M.DeviceLattice(wl.lattice)
        prm = M.DeviceParams(wl.params)
        box = ((0, 0, 0), dims)
        cnn = M.CNN(ctx, 1)
        x, f = cnn.features(lat, prm, box)
        cnn.close()
        xs.append(x)
        fs.append(f)
        wls.append(wl)
    return torch.cat(xs), torch.cat(fs), wls


def _np(t):
    return t.float().cpu().numpy().astype(np.float64)


def test_features_are_the_documented_channels(M):
    ctx = M.Context()
    dims = (11, 6, 5)
    x, f, (wl,) = _case(M, ctx, 3, dims, 1)
    X = _np(x).reshape(dims[2], dims[1], dims[0], 16)
    lat = wl.lattice
    assert np.array_equal(_np(f).reshape(dims[2], dims[1], dims[0], 3), np.moveaxis(lat.fields, 0, -1).astype(np.float32))
    assert np.array_equal(X[..., 0], oracle.bf16(lat.fields[0]))
    assert np.array_equal(X[..., 2], oracle.bf16(20 * lat.fields[2].astype(np.float32)))
    assert np.array_equal(X[..., 3], (lat.cell_id == 0).astype(float))
    assert np.array_equal(X[..., 4], (lat.cell_id > 0).astype(float))
    assert np.array_equal(X[..., 5], oracle.bf16(10 * wl.params.k_cell[0][lat.cell_id].astype(np.float32)))
    assert np.array_equal(X[..., 7], oracle.bf16(10 * wl.params.q_cell[2][lat.cell_id].astype(np.float32)))
    assert np.array_equal(X[..., 8], lat.mask.astype(float))
    assert np.all(X[..., 9:] == 0)


@pytest.mark.parametrize("dims,batch", [((13, 9, 7), 2), ((32, 8, 6), 1), ((5, 17, 3), 3)])
def test_forward_and_gradients_match_oracle(M, dims, batch):
    import torch
    ctx = M.Context()
    x, f, wls = _case(M, ctx, 10, dims, batch)
    V = dims[0] * dims[1] * dims[2]
    params = M.cnn_init_params(seed=1, last_scale=1.0)
    params[-3:] = [0.1, -0.2, 0.05]
    cnn = M.CNN(ctx, V * batch, params, s_out=0.3)
    pred = cnn.forward(x, f, dims, batch)
    rng = np.random.default_rng(2)
    target = torch.from_numpy((_np(f) + 0.3 * rng.normal(size=(V * batch, 3))).astype(np.float32)).cuda()
    loss = cnn.train_step(x, f, target, dims, batch, lr=0.0, apply=False)
    g_gpu = cnn.get(1).astype(np.float64)
    P = oracle.bf16(params.astype(np.float64))
    X = _np(x).reshape(batch, dims[2], dims[1], dims[0], 16)[..., :9]
    F = _np(f).reshape(batch, dims[2], dims[1], dims[0], 3)
    T = _np(target).reshape(batch, dims[2], dims[1], dims[0], 3)
    pr = _np(pred).reshape(batch, dims[2], dims[1], dims[0], 3)
    g_or = np.zeros_like(P)
    L_or = 0.0
    nm_tot = sum(int(w.lattice.mask.sum()) for w in wls)
    for b in range(batch):
        p_o, cache = oracle.cnn_forward(X[b], F[b], P, 0.3)
        z6g = (pr[b] - F[b]) / 0.3
        z6o = (p_o - F[b]) / 0.3
        assert np.max(np.abs(z6g - z6o)) <= 1e-2 * np.max(np.abs(z6o)), b
        # loss over the whole batch: per-crop losses weighted by their mask counts
        Lb, gp = oracle.cnn_loss(p_o, T[b], wls[b].lattice.mask)
        nm = int(wls[b].lattice.mask.sum())
        L_or += Lb * nm / nm_tot
        g_or += oracle.cnn_backward(X[b], P, 0.3, cache, gp * nm / nm_tot, round_grad=True)
    assert abs(loss - L_or) <= 1e-2 * L_or
    for l, (sw, sb, ci, co) in enumerate(oracle.cnn_param_slices()):
        for sl in (sw, sb):
            err = np.linalg.norm(g_gpu[sl] - g_or[sl]) / np.linalg.norm(g_or[sl])
            assert err <= 2e-2, (l, err)


def test_adam_step_matches_oracle(M):
    import torch
    ctx = M.Context()
    dims = (16, 8, 8)
    x, f, wls = _case(M, ctx, 20, dims, 1)
    params = M.cnn_init_params(seed=3)
    cnn = M.CNN(ctx, x.shape[0], params)
    target = (f + 0.01).contiguous()
    cnn.train_step(x, f, target, dims, 1, lr=0.0, apply=False)
    g = cnn.get(1).astype(np.float64)
    cnn.set_params(params)
    cnn.train_step(x, f, target, dims, 1, lr=1e-3, apply=True)
    p_gpu = cnn.get(0).astype(np.float64)
    p = params.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    oracle.adam(p, g, m, v, lr=1e-3, t=1)
    assert np.max(np.abs(p_gpu - p)) <= 1e-6


def test_training_reduces_the_loss(M):
    ctx = M.Context()
    dims = (16, 16, 8)
    x, f, wls = _case(M, ctx, 30, dims, 2)
    target = (f * 0.97 + 0.01).contiguous()
    cnn = M.CNN(ctx, x.shape[0], M.cnn_init_params(seed=4), s_out=0.05)
    losses = [cnn.train_step(x, f, target, dims, 2, lr=3e-3) for _ in range(60)]
    assert losses[-1] < 0.3 * losses[0]


def test_guess_seeds_the_solver(M):
    ctx = M.Context()
    wl = W.sphere32()
    lat = M.DeviceLattice(wl.lattice)
    prm = M.DeviceParams(wl.params)
    sub = ctx.subgrid_create()
    sub.mpm_box_extract(lat, 1, wl.margin)
    sub.mpm_assemble_coeffs(prm)
    cnn = M.CNN(ctx, 32 ** 3, M.cnn_init_params(seed=5), s_out=0.01)
    cnn.guess(sub, lat, prm)
    x0 = sub.mpm_subgrid_export(M.EXPORT_X, 0).cpu().numpy()
    assert not np.array_equal(x0, wl.lattice.fields[0])
    rep = sub.mpm_solve_step(M.make_opts(rtol=0.0, atol=1e-12, restart=30, maxit=500, x0_given=1), scatter_to=lat)
    assert rep["status_code"] == M.OK
    ref = wl.lattice.copy()
    oracle.step(ref, wl.params, wl.margin, rtol=0.0, atol=1e-12)
    assert np.max(np.abs(lat.fields_numpy() - ref.fields)) <= 1e-10


def test_trained_network_gain_on_sphere32(M):
    """Train on GPU-generated pairs (the FP64 solver's own steps), then measure on
    the 32^3 sphere workload what the network's guess gains over x0 = c^n: the
    initial relative residual of the first step (a solve with rtol = 1 stops at
    its first residual and reports it) and the Arnoldi steps to 1e-6 over 10
    steps.  Both answers meet the tolerance and agree within its bound."""
    from paper_2505_03067_gb300 import learned
    ctx = M.Context()
    cnn, hist = learned.train(ctx, samples=4000)
    assert np.mean(hist["loss"][-20:]) < 0.2 * np.mean(hist["loss"][:5])
    wl = W.sphere32()
    r0 = {}
    for use in (False, True):
        lat = M.DeviceLattice(wl.lattice)
        prm = M.DeviceParams(wl.params)
        sub = ctx.subgrid_create()
        sub.mpm_box_extract(lat, 1, wl.margin)
        sub.mpm_assemble_coeffs(prm)
        if use:
            cnn.guess(sub, lat, prm)
        rep = sub.mpm_solve_step(M.make_opts(rtol=1.0, restart=8, maxit=10, x0_given=int(use)))
        r0[use] = rep["res"][0] / rep["bnorm"][0]
    assert r0[True] < 0.5 * r0[False], r0
    ev = learned.evaluate_sphere32(ctx, cnn, rtol=1e-6)
    assert ev["learned"]["max_rel_res"] <= 1e-6 and ev["plain"]["max_rel_res"] <= 1e-6
    assert ev["learned"]["iters_per_step"] <= ev["plain"]["iters_per_step"]
    assert np.max(np.abs(ev["learned"]["final"] - ev["plain"]["final"])) <= 10 * 2e-6 * np.sqrt(32 ** 3)
    # row a13: the same network as the right preconditioner of flexible GMRES
    fg = learned.evaluate_fgmres_sphere32(ctx, cnn, rtol=1e-6)
    for k in ("fgmres", "guess_fgmres"):
        assert fg[k]["max_rel_res"] <= 1e-6, k
        assert np.max(np.abs(fg[k]["final"] - ev["plain"]["final"])) <= 10 * 2e-6 * np.sqrt(32 ** 3), k
