"""Pins of the CNN reference (no GPU): convolution special cases with closed
forms, the adjoint identities that define its input and weight gradients, the
full backward pass against central finite differences, the activity mask
(inactive voxels influence nothing; all-active is the plain network), the
bf16-stored-gradient backward against the chain rule written out, GELU
against the erf formula, Adam's first step in closed form, and bfloat16
rounding against PyTorch's conversion."""
import math

import numpy as np
import pytest

import oracle


def test_center_tap_identity_kernel_is_identity():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(4, 5, 6, 3))
    W = np.zeros((27, 3, 3))
    W[13] = np.eye(3)               # tap (0, 0, 0)
    b = np.array([0.5, -1.0, 2.0])
    assert np.allclose(oracle.conv3(x, W, b), x + b, rtol=0, atol=1e-15)


def test_shift_kernel_moves_the_field():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(4, 5, 6, 1))
    W = np.zeros((27, 1, 1))
    W[14] = 1.0                     # tap dx = +1: out[i] = x[i+1], zero past the edge
    out = oracle.conv3(x, W)
    assert np.array_equal(out[:, :, :-1], x[:, :, 1:])
    assert np.all(out[:, :, -1] == 0)


def test_box_kernel_counts_in_domain_neighbours():
    x = np.ones((3, 4, 5, 1))
    W = np.ones((27, 1, 1))
    out = oracle.conv3(x, W)[..., 0]
    def cnt(i, n):
        return 3 - (i == 0) - (i == n - 1) if n > 1 else 1
    for k in range(3):
        for j in range(4):
            for i in range(5):
                assert out[k, j, i] == cnt(i, 5) * cnt(j, 4) * cnt(k, 3)


def test_dgrad_and_wgrad_are_the_adjoints():
    """<conv(x; W), y> = <x, dgrad(y; W)> = <W, wgrad(x, y)> (bias zero)."""
    rng = np.random.default_rng(2)
    x = rng.normal(size=(4, 3, 5, 7))
    W = rng.normal(size=(27, 7, 5))
    y = rng.normal(size=(4, 3, 5, 5))
    lhs = np.sum(oracle.conv3(x, W) * y)
    assert abs(lhs - np.sum(x * oracle.conv3_dgrad(y, W, 7))) < 1e-10 * abs(lhs)
    gW, gb = oracle.conv3_wgrad(x, y)
    assert abs(lhs - np.sum(W * gW)) < 1e-10 * abs(lhs)
    assert np.allclose(gb, y.sum(axis=(0, 1, 2)))


def test_gelu_matches_erf_formula():
    for z in (-3.0, -0.7, 0.0, 0.3, 2.5):
        assert abs(oracle.gelu(z) - 0.5 * z * (1 + math.erf(z / math.sqrt(2)))) < 1e-15
        h = 1e-6
        fd = (oracle.gelu(z + h) - oracle.gelu(z - h)) / (2 * h)
        assert abs(oracle.gelu_grad(z) - fd) < 1e-8


def _rand_params(rng, scale=0.3):
    n = oracle.cnn_nparams()
    assert n == sum(27 * a * b + b for a, b in zip(oracle.CNN_CHANNELS[:-1], oracle.CNN_CHANNELS[1:]))
    return rng.normal(scale=scale, size=n) / np.sqrt(27 * 24)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(3)
    shape = (3, 4, 5)
    x = rng.normal(size=shape + (9,))
    f = rng.normal(size=shape + (3,))
    t = rng.normal(size=shape + (3,))
    mask = (rng.random(shape) < 0.8).astype(np.uint8)
    P = _rand_params(rng, 3.0)
    s_out = 0.7

    def loss(p):
        pred, _ = oracle.cnn_forward(x, f, p, s_out, round_act=False)
        return oracle.cnn_loss(pred, t, mask)[0]

    pred, cache = oracle.cnn_forward(x, f, P, s_out, round_act=False)
    _, gp = oracle.cnn_loss(pred, t, mask)
    g = oracle.cnn_backward(x, P, s_out, cache, gp)
    idx = rng.choice(P.size, 60, replace=False)
    for sl_w, sl_b, _, _ in oracle.cnn_param_slices():   # at least one weight and the bias of every layer
        idx = np.concatenate([idx, [sl_w.start + 5, sl_b.start]])
    h = 2e-3
    for i in idx:
        e = np.zeros_like(P)
        e[i] = h
        # fourth-order central difference
        fd = (-loss(P + 2 * e) + 8 * loss(P + e) - 8 * loss(P - e) + loss(P - 2 * e)) / (12 * h)
        assert abs(g[i] - fd) <= 1e-6 * max(1e-3, abs(fd)), (i, g[i], fd)


def test_zero_last_layer_returns_the_fields():
    rng = np.random.default_rng(4)
    shape = (2, 3, 4)
    P = _rand_params(rng)
    sl_w, sl_b, _, _ = oracle.cnn_param_slices()[5]
    P[sl_w] = 0
    P[sl_b] = 0
    f = rng.normal(size=shape + (3,))
    pred, _ = oracle.cnn_forward(rng.normal(size=shape + (9,)), f, P, 0.5)
    assert np.array_equal(pred, f)


def test_adam_first_step_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m = np.zeros(3)
    v = np.zeros(3)
    oracle.adam(p, g, m, v, lr=0.01, t=1)
    assert np.allclose(p, np.array([1.0, -2.0, 0.5]) - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_bf16_rounding():
    assert oracle.bf16([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5])[0:4].tolist() == [1.0, 1.0, 1.0 + 2 ** -6, -2.5]
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(5).normal(size=1000) * 10 ** np.random.default_rng(6).uniform(-5, 5, 1000)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).double().numpy()
    assert np.array_equal(oracle.bf16(x), ref)


def _masked_case(rng, shape, p_act=0.6):
    x = rng.normal(size=shape + (9,))
    act = rng.random(shape) < p_act
    x[..., 8] = act
    return x, act


def _plain_forward(x, f, P, s_out, act):
    """The network written out from oracle.conv3, GELU and bf16 rounding, with
    the activity mask applied to the layer-1 input and to a_1..a_5."""
    gelu = np.vectorize(oracle.gelu)
    a = np.where(act[..., None], x, 0.0)
    for l, (sw, sb, ci, co) in enumerate(oracle.cnn_param_slices()):
        z = oracle.conv3(a, P[sw].reshape(27, ci, co), P[sb])
        if l < 5:
            a = np.where(act[..., None], oracle.bf16(gelu(z)), 0.0)
    return f + s_out * z


def test_all_active_and_masked_network_written_out():
    rng = np.random.default_rng(7)
    shape = (4, 3, 5)
    P = oracle.bf16(_rand_params(rng))
    f = rng.normal(size=shape + (3,))
    for p_act in (1.0, 0.5):
        x, act = _masked_case(rng, shape, p_act)
        pred, _ = oracle.cnn_forward(x, f, P, 0.3)
        assert np.array_equal(pred, _plain_forward(x, f, P, 0.3, act))


def test_inactive_voxels_do_not_influence_active_outputs():
    rng = np.random.default_rng(8)
    shape = (5, 4, 6)
    P = oracle.bf16(_rand_params(rng, 3.0))
    f = rng.normal(size=shape + (3,))
    x, act = _masked_case(rng, shape, 0.5)
    pred, (z, a) = oracle.cnn_forward(x, f, P, 0.3)
    x2 = x.copy()
    x2[~act, :8] = rng.normal(size=(int((~act).sum()), 8)) * 100.0
    f2 = f.copy()
    f2[~act] = 7.0
    pred2, (_, a2) = oracle.cnn_forward(x2, f2, P, 0.3)
    assert np.array_equal(pred[act], pred2[act])
    V = act.size
    for l in range(5):
        al = a[l * V * 24:(l + 1) * V * 24].reshape(shape + (24,))
        assert np.all(al[~act] == 0.0) and np.array_equal(al, a2[l * V * 24:(l + 1) * V * 24].reshape(al.shape))


def test_bf16_stored_gradient_backward_is_the_chain_rule():
    """The backward pass that stores each dLoss/dz in bf16 (as the GPU does)
    equals the chain rule written out layer by layer from the pinned pieces
    (conv3_wgrad, conv3_dgrad, gelu_grad, bf16) with bf16 applied to every
    stored dLoss/dz and the activity mask applied to each."""
    rng = np.random.default_rng(9)
    shape = (3, 4, 5)
    V = int(np.prod(shape))
    P = oracle.bf16(_rand_params(rng, 3.0))
    f = rng.normal(size=shape + (3,))
    t = rng.normal(size=shape + (3,))
    x, act = _masked_case(rng, shape, 0.7)
    s_out = 0.4
    pred, (z, a) = oracle.cnn_forward(x, f, P, s_out)
    _, gp = oracle.cnn_loss(pred, t, act.astype(np.uint8))
    got = oracle.cnn_backward(x, P, s_out, (z, a), gp, round_grad=True)

    gelu_grad = np.vectorize(oracle.gelu_grad)
    slices = oracle.cnn_param_slices()
    zs = [z[l * V * 24:l * V * 24 + V * slices[l][3]].reshape(shape + (slices[l][3],)) for l in range(6)]
    acts = [a[l * V * 24:(l + 1) * V * 24].reshape(shape + (24,)) for l in range(5)]
    want = np.zeros_like(P)
    g = oracle.bf16(s_out * gp)                                   # dLoss/dz_6, stored in bf16
    for l in range(5, -1, -1):
        sw, sb, ci, co = slices[l]
        inp = np.where(act[..., None], x, 0.0) if l == 0 else acts[l - 1]
        gW, gb = oracle.conv3_wgrad(inp, g)
        want[sw] = gW.reshape(-1)
        want[sb] = gb
        if l == 0:
            break
        gin = oracle.conv3_dgrad(g, P[sw].reshape(27, ci, co), ci)      # dLoss/da_l
        g = oracle.bf16(np.where(act[..., None], gin * gelu_grad(zs[l - 1]), 0.0))
    assert np.array_equal(got, want)
    # and it differs from the unrounded backward by bf16-sized amounts only
    ref = oracle.cnn_backward(x, P, s_out, (z, a), gp)
    assert not np.array_equal(got, ref)
    assert np.linalg.norm(got - ref) <= 2e-2 * np.linalg.norm(ref)
