"""The forward convolution's GELU evaluates erf by Abramowitz & Stegun,
Handbook of Mathematical Functions, formula 7.1.26 (a published rational-
exponential approximation with |error| <= 1.5e-7 on x >= 0).  These checks pin
that formula, as the kernel evaluates it in FP32, against the exact erf, and
bound the GELU error it causes far below the bf16 rounding (2^-9 relative) of
the stored activation.  The GPU parity tests then compare whole layers with
the oracle's exact-erf GELU."""
import math

import numpy as np

P = 0.3275911
A = (0.254829592, -0.284496736, 1.421413741, -1.453152027, 1.061405429)


def erfc_half_as(x, dtype):
    """(1 - erf(x)) / 2 for x >= 0, evaluated in `dtype` the way the kernel does
    (Horner in t, exp(-x^2) as 2^(-x^2 log2 e))."""
    x = x.astype(dtype)
    t = dtype(1.0) / (dtype(P) * x + dtype(1.0))
    poly = t * (dtype(A[0]) + t * (dtype(A[1]) + t * (dtype(A[2]) + t * (dtype(A[3]) + t * dtype(A[4])))))
    return dtype(0.5) * poly * np.exp2(dtype(-1.4426950408889634) * x * x)


def gelu_as(z, dtype=np.float32):
    z = z.astype(dtype)
    h = erfc_half_as(np.abs(z) * dtype(0.70710678118654752), dtype)
    return z * np.where(z >= 0, dtype(1.0) - h, h)


def test_formula_error_within_published_bound():
    x = np.linspace(0.0, 8.0, 400001)
    exact = np.array([math.erf(v) for v in x])
    approx = 1.0 - 2.0 * erfc_half_as(x, np.float64)
    assert np.max(np.abs(approx - exact)) <= 1.5e-7


def test_fp32_gelu_error_far_below_bf16_rounding():
    z = np.linspace(-10.0, 10.0, 200001)
    exact = np.array([0.5 * v * (1.0 + math.erf(v / math.sqrt(2.0))) for v in z])
    got = gelu_as(z).astype(np.float64)
    err = np.abs(got - exact)
    # absolute error at most ~4e-7 * (1 + |z|); bf16 keeps 8 significant bits
    assert np.all(err <= 4e-7 * (1.0 + np.abs(z)))
    big = np.abs(exact) > 1e-3
    assert np.max(err[big] / np.abs(exact[big])) < 2.0 ** -12


def test_special_values():
    z = np.array([0.0, -0.0, 1e-30, -1e-30, 30.0, -30.0], np.float32)
    g = gelu_as(z)
    assert g[0] == 0.0 and g[1] == 0.0
    assert abs(g[2] - 0.5e-30) < 1e-36 and abs(g[3] + 0.5e-30) < 1e-36
    assert g[4] == np.float32(30.0)
    assert g[5] == 0.0 or abs(g[5]) < 1e-30
