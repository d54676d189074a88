"""The learned warm start's network on the GPU (tcgen05 bf16 convolutions with
FP32 accumulation, block-sparse over the active voxels) against the FP64 CNN
oracle with the GPU's bf16 storage points reproduced: the staged features bit
for bit, the forward pass and every parameter gradient element by element,
Adam, training, the activity mask's invariance, and the network's prediction
used as the solver's initial guess.

Tolerances.  Layer 1's pre-activations see identical bf16 inputs and
weights on both sides and differ only by FP32 against FP64 accumulation of
at most 27 x 9 products (rounding ~ sqrt(243) 2^-24 of the terms' size, a few
times 1e-6): Z1_TOL = 5e-5 of their largest magnitude, element by element.
Deeper, both sides round the same values to bf16 at the same points, so they differ where the FP32 (GPU) and FP64 (oracle) value of an
activation straddle a bf16 rounding boundary: about one activation in 2000
moves by one bf16 unit (2^-8 relative), which moves each output it feeds by
~2^-8 w / |z| ~ 2e-4 of its scale.  An output of layer 6 depends on 13^3
voxels x 24 channels x 5 layers ~ 260 000 activations, ~130 of them flipped:
a random sum of ~130 such terms, sqrt(130) x 2e-4 ~ 2e-3 RMS, up to about
four times that at the worst of thousands of outputs.  So the forward is
checked element by element at FORWARD_MAX = 1e-2 of max |z6| and in the
mean at FORWARD_RMS = 3e-3 of rms |z6|; the gradients (sums over the voxels
of products of two such quantities, with the bf16-stored dLoss/dz flipping the
same way) per layer at GRAD_MAX = 2e-2 of the layer's largest gradient and
GRAD_RMS = 5e-3 of its rms."""
import numpy as np
import pytest

import oracle
from paper_2505_03067_gb300 import workloads as W

pytestmark = pytest.mark.gpu

Z1_TOL = 5e-5
FORWARD_MAX, FORWARD_RMS = 1e-2, 3e-3
GRAD_MAX, GRAD_RMS = 2e-2, 5e-3


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_03067_gb300 import build, mpm
    build.build()
    return mpm


def _features_np(lat, params):
    """The nine input channels written out from their definition (FP32
    products rounded to bf16), zero outside the mask, and c^n in FP32."""
    f32 = np.float32
    cid = np.where((lat.cell_id >= 0) & (lat.cell_id < params.ncell), lat.cell_id, 0)
    S = params.nspecies
    shape = lat.cell_id.shape
    fld = [lat.fields[s].astype(f32) if s < S else np.zeros(shape, f32) for s in range(3)]
    X = np.zeros(shape + (9,))
    X[..., 0] = oracle.bf16(fld[0])
    X[..., 1] = oracle.bf16(fld[1])
    X[..., 2] = oracle.bf16(fld[2] * f32(20))
    X[..., 3] = cid == 0
    X[..., 4] = cid > 0
    if S > 0:
        X[..., 5] = oracle.bf16(params.k_cell[0][cid].astype(f32) * f32(10))
    if S > 1:
        X[..., 6] = oracle.bf16(params.k_cell[1][cid].astype(f32) * f32(10))
    if S > 2:
        X[..., 7] = oracle.bf16(params.q_cell[2][cid].astype(f32) * f32(10))
    X[..., 8] = lat.mask > 0
    X[lat.mask == 0] = 0.0
    return X, np.stack(fld, -1).astype(np.float64)


def _images(M, seed, dims, batch, box_fn=None, p_mask=0.8):
    out = []
    for b in range(batch):
        wl = W.random_case(seed + b, dims, nspecies=3, blob=True, p_mask=p_mask)
        wl.lattice.fields[2] *= 0.05
        box = ((0, 0, 0), dims) if box_fn is None else box_fn(b)
        tgt = wl.lattice.copy()
        tgt.fields = (wl.lattice.fields + 0.3 * np.random.default_rng(seed + 100 + b).normal(size=tgt.fields.shape))
        out.append((wl, box, tgt))
    return out


def _load(M, cnn, imgs):
    keep = []
    for b, (wl, box, tgt) in enumerate(imgs):
        lat, prm = M.DeviceLattice(wl.lattice), M.DeviceParams(wl.params)
        tl = M.DeviceLattice(tgt)
        cnn.load_image(b, lat, prm, box, M.CNN_INPUT)
        if cnn.train:
            cnn.load_image(b, tl, prm, box, M.CNN_TARGET)
        keep += [lat, prm, tl]
    return keep


def _np(t):
    return t.float().cpu().numpy().astype(np.float64)


def _params(M):
    params = M.cnn_init_params(seed=1, last_scale=1.0)
    params[-3:] = [0.1, -0.2, 0.05]
    return params


def _check_forward_and_gradients(M, dims, batch, box_fn=None, p_mask=0.8, seed=10):
    ctx = M.Context()
    params = _params(M)
    cnn = M.CNN(ctx, dims, batch, params, s_out=0.3, train=True)
    imgs = _images(M, seed, dims, batch, box_fn, p_mask)
    keep = _load(M, cnn, imgs)
    pred = cnn.forward(batch)
    loss = cnn.train_step(batch, lr=0.0, apply=False)
    g_gpu = cnn.get(1).astype(np.float64)
    V = dims[0] * dims[1] * dims[2]
    pr = _np(pred).reshape(batch, dims[2], dims[1], dims[0], 3)
    P = oracle.bf16(params.astype(np.float64))
    g_or = np.zeros_like(P)
    L_or = 0.0
    n_tot = 0
    per = []
    for wl, box, tgt in imgs:
        X, F = _features_np(wl.lattice, wl.params)
        bx = oracle.box_slices(box)
        T = np.moveaxis(tgt.fields, 0, -1).astype(np.float32).astype(np.float64)
        m = (wl.lattice.mask > 0)[bx]
        per.append((X[bx], F[bx], T[bx], m))
        n_tot += int(m.sum())
    z1g = _np(cnn.export_preact(1, batch)).reshape(batch, dims[2], dims[1], dims[0], 24)
    sw1, sb1, ci1, co1 = oracle.cnn_param_slices()[0]
    dz6, z6s, z1err = [], [], 0.0
    for b, (X, F, T, m) in enumerate(per):
        box = imgs[b][1]
        p_o, cache = oracle.cnn_forward(X, F, P, 0.3)
        # layer 1 alone: identical bf16 inputs and weights, FP32 vs FP64 sums
        z1o = oracle.conv3(np.where(m[..., None], X, 0.0), P[sw1].reshape(27, ci1, co1), P[sb1])
        z1err = max(z1err, np.max(np.abs(z1g[b][oracle.box_slices(box)][m] - z1o[m])) / np.max(np.abs(z1o[m])))
        z6o = (p_o - F) / 0.3
        z6g = (pr[b][oracle.box_slices(box)] - F) / 0.3
        dz6.append((z6g - z6o)[m].reshape(-1))
        z6s.append(z6o[m].reshape(-1))
        Lb, gp = oracle.cnn_loss(p_o, T, m.astype(np.uint8))
        nm = int(m.sum())
        L_or += Lb * nm / n_tot
        g_or += oracle.cnn_backward(X, P, 0.3, cache, gp * nm / n_tot, round_grad=True)
    dz6, z6s = np.concatenate(dz6), np.concatenate(z6s)
    f_max = np.max(np.abs(dz6)) / np.max(np.abs(z6s))
    f_rms = np.sqrt(np.mean(dz6 ** 2) / np.mean(z6s ** 2))
    report = [f"z1 {z1err:.1e}", f"z6 max {f_max:.1e} rms {f_rms:.1e}", f"loss {abs(loss - L_or) / L_or:.1e}"]
    gerr = []
    for l, (sw, sb, ci, co) in enumerate(oracle.cnn_param_slices()):
        for name, sl in (("W", sw), ("b", sb)):
            d = g_gpu[sl] - g_or[sl]
            e_max = np.max(np.abs(d)) / np.max(np.abs(g_or[sl]))
            e_rms = np.linalg.norm(d) / np.linalg.norm(g_or[sl])
            gerr.append((l + 1, name, e_max, e_rms))
            report.append(f"g{l + 1}{name} max {e_max:.1e} rms {e_rms:.1e}")
    print("cnn parity", dims, batch, "; ".join(report))
    assert z1err <= Z1_TOL, report
    assert f_max <= FORWARD_MAX and f_rms <= FORWARD_RMS, report
    assert abs(loss - L_or) <= 1e-3 * L_or, report
    for l, name, e_max, e_rms in gerr:
        assert e_max <= GRAD_MAX and e_rms <= GRAD_RMS, (l, name, report)
    del keep


def test_features_are_the_documented_channels(M):
    ctx = M.Context()
    dims = (11, 6, 5)
    cnn = M.CNN(ctx, dims, 2, s_out=0.3)
    imgs = _images(M, 3, dims, 2, box_fn=lambda b: ((0, 0, 0), dims) if b == 0 else ((2, 1, 1), (9, 6, 4)))
    keep = _load(M, cnn, imgs)
    x, msk = cnn.export_features(2)
    x = _np(x).reshape(2, dims[2], dims[1], dims[0], 16)
    msk = msk.cpu().numpy().reshape(2, dims[2], dims[1], dims[0])
    for b, (wl, box, _) in enumerate(imgs):
        X, _ = _features_np(wl.lattice, wl.params)
        bx = oracle.box_slices(box)
        assert np.array_equal(msk[b][bx], (wl.lattice.mask[bx] > 0).astype(np.uint8))
        assert np.array_equal(x[b][bx][..., :9], X[bx])
        assert np.all(x[b][bx][..., 9:15] == 0)
        assert np.array_equal(x[b][bx][..., 15], (wl.lattice.mask[bx] > 0).astype(float))
    del keep


@pytest.mark.parametrize("dims,batch", [((13, 9, 7), 2), ((32, 8, 6), 1), ((5, 17, 3), 3), ((19, 33, 20), 1)])
def test_forward_and_gradients_match_oracle(M, dims, batch):
    _check_forward_and_gradients(M, dims, batch)


def test_partial_boxes_and_sparse_masks(M):
    """Boxes inside the image (ragged against the 8 x 16 slabs, at image
    faces and away from them) and a sparse mask (whole units inactive)."""
    dims = (29, 37, 19)
    boxes = [((3, 5, 2), (26, 36, 17)), ((0, 0, 0), (17, 21, 19)), ((11, 2, 7), (29, 37, 12))]
    _check_forward_and_gradients(M, dims, 3, box_fn=lambda b: boxes[b], p_mask=0.15, seed=40)


def test_training_batch_size_32cubed_times_8(M):
    _check_forward_and_gradients(M, (32, 32, 32), 8, seed=60)


def test_inactive_voxels_do_not_change_active_outputs(M):
    """Lattice data outside the mask or outside the box (fields, cell ids)
    do not change the prediction at active voxels: bit for bit."""
    ctx = M.Context()
    dims = (21, 18, 14)
    box = ((2, 3, 1), (19, 17, 13))
    cnn = M.CNN(ctx, dims, 1, _params(M), s_out=0.3)
    wl = W.random_case(70, dims, nspecies=3, blob=True, p_mask=0.5)
    preds = []
    for variant in range(2):
        lat = wl.lattice.copy()
        if variant:
            out = np.ones(lat.mask.shape, bool)
            out[oracle.box_slices(box)] = lat.mask[oracle.box_slices(box)] == 0
            lat.fields[:, out] = 123.0
            lat.cell_id[out] = 3
        dl, dp = M.DeviceLattice(lat), M.DeviceParams(wl.params)
        cnn.load_image(0, dl, dp, box, M.CNN_INPUT)
        preds.append(_np(cnn.forward(1)).reshape(dims[2], dims[1], dims[0], 3))
    act = np.zeros(wl.lattice.mask.shape, bool)
    act[oracle.box_slices(box)] = wl.lattice.mask[oracle.box_slices(box)] > 0
    assert np.array_equal(preds[0][act], preds[1][act])


def test_adam_step_matches_oracle(M):
    ctx = M.Context()
    dims = (16, 8, 8)
    params = M.cnn_init_params(seed=3)
    cnn = M.CNN(ctx, dims, 1, params, train=True)
    imgs = _images(M, 20, dims, 1)
    keep = _load(M, cnn, imgs)
    cnn.train_step(1, lr=0.0, apply=False)
    g = cnn.get(1).astype(np.float64)
    cnn.set_params(params)
    cnn.train_step(1, lr=1e-3, apply=True)
    p_gpu = cnn.get(0).astype(np.float64)
    p = params.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    oracle.adam(p, g, m, v, lr=1e-3, t=1)
    assert np.max(np.abs(p_gpu - p)) <= 1e-6
    del keep


def test_training_reduces_the_loss(M):
    ctx = M.Context()
    dims = (16, 16, 8)
    cnn = M.CNN(ctx, dims, 2, M.cnn_init_params(seed=4), s_out=0.05, train=True)
    imgs = _images(M, 30, dims, 2)
    for wl, box, tgt in imgs:
        tgt.fields = wl.lattice.fields * 0.97 + 0.01
    keep = _load(M, cnn, imgs)
    losses = [cnn.train_step(2, lr=3e-3) for _ in range(100)]
    assert losses[-1] < 0.4 * losses[0]
    del keep


def test_guess_seeds_the_solver(M):
    ctx = M.Context()
    wl = W.sphere32()
    lat = M.DeviceLattice(wl.lattice)
    prm = M.DeviceParams(wl.params)
    sub = ctx.subgrid_create()
    sub.mpm_box_extract(lat, 1, wl.margin)
    sub.mpm_assemble_coeffs(prm)
    cnn = M.CNN(ctx, (32, 32, 32), 1, M.cnn_init_params(seed=5), s_out=0.01)
    cnn.guess(sub, lat, prm)
    x0 = sub.mpm_subgrid_export(M.EXPORT_X, 0).cpu().numpy()
    assert not np.array_equal(x0, wl.lattice.fields[0])
    # the guess is c^n + s_out z6 of the network on this machine: the oracle's prediction
    X, F = _features_np(wl.lattice, wl.params)
    p_o, _ = oracle.cnn_forward(X, F, oracle.bf16(M.cnn_init_params(seed=5).astype(np.float64)), 0.01)
    z6o = (p_o[..., 0] - F[..., 0]) / 0.01
    z6g = (x0 - wl.lattice.fields[0]) / 0.01
    assert np.max(np.abs(z6g - z6o)) <= FORWARD_MAX * np.max(np.abs(z6o)) + 1e-9
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
