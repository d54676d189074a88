"""The FP32 Krylov path's bit-level conversions (f32_rz, f64_of) against CUDA's
own conversions and against NumPy, on random bit patterns and on the edge
values of the two formats.

f32_rz rounds an FP64 value toward zero to FP32 with integer operations on its
IEEE-754 bits; f64_of widens an FP32 value exactly.  Both differ from IEEE in
two stated ranges, checked here as stated: FP64 magnitudes below FP32's normal
range (2^-126) and FP32 subnormals give a signed zero, and FP64 magnitudes of
2^128 and above give an infinity (IEEE round-toward-zero gives the largest
finite FP32).  Everything else must match bit for bit.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_03067_gb300 import build, mpm
    build.build()
    return mpm


def _f64(hi_exp, mant=0, sign=0):
    return np.array([(sign << 63) | (hi_exp << 52) | mant], np.uint64).view(np.float64)[0]


def _inputs(seed=11, n=200000):
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64) | (rng.integers(0, 2, size=n, dtype=np.uint64) << 63)
    x = bits.view(np.float64)
    # bias most draws into and around FP32's exponent range
    e = rng.integers(0x370, 0x490, size=n // 2, dtype=np.uint64)
    x2 = ((bits[: n // 2] & np.uint64(0x800FFFFFFFFFFFFF)) | (e << np.uint64(52))).view(np.float64)
    edges = []
    for ex in (0x37F, 0x380, 0x381, 0x382, 0x47D, 0x47E, 0x47F, 0x480):
        for m in (0, 1, 0xFFFFFFFFFFFFF, 0x8000000000000, 0x1FFFFFFF, 0x20000000):
            for sg in (0, 1):
                edges.append(_f64(ex, m, sg))
    edges += [0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 1e-20, -1e-20, 3.4028234663852886e38,
              np.float64(np.finfo(np.float32).max) * (1 + 2 ** -30)]
    x = np.concatenate([x, x2, np.array(edges, np.float64)])
    f_bits = rng.integers(0, 2 ** 32, size=x.size, dtype=np.uint64).astype(np.uint32)
    f = f_bits.view(np.float32)
    f_edges = np.array([0x00000001, 0x80000001, 0x007FFFFF, 0x807FFFFF, 0x00800000, 0x80800000, 0x7F7FFFFF,
                        0x7F800000, 0xFF800000, 0x7FC00000, 0x00000000, 0x80000000], np.uint32).view(np.float32)
    f[: f_edges.size] = f_edges
    return x, f


def _np_rz(x):
    """Round toward zero to FP32 in NumPy: round to nearest, then step back
    toward zero where that moved away from it."""
    with np.errstate(over="ignore", invalid="ignore"):
        f = x.astype(np.float32)
        away = np.isfinite(x) & (np.abs(f.astype(np.float64)) > np.abs(x))
        f[away] = np.nextafter(f[away], np.float32(0))
    return f


def test_f32_rz_and_f64_of_against_cuda_and_numpy(M):
    import torch
    x, f = _inputs()
    out32, ref32, out64, ref64 = (t.cpu().numpy() for t in
                                  M.mpm_debug_convert(torch.from_numpy(x).cuda(), torch.from_numpy(f).cuda()))
    ax = np.abs(x)
    nan = np.isnan(x)
    tiny = ~nan & (ax < 2.0 ** -126)
    huge = ~nan & (ax >= 2.0 ** 128)
    mid = ~nan & ~tiny & ~huge
    b_out, b_ref = out32.view(np.uint32), ref32.view(np.uint32)
    # the FP32 normal range: bit for bit CUDA's round toward zero, and NumPy's
    assert np.array_equal(b_out[mid], b_ref[mid])
    assert np.array_equal(b_out[mid], _np_rz(x[mid]).view(np.uint32))
    # below it: a zero of the input's sign (CUDA keeps a subnormal)
    sgn = (x.view(np.uint64) >> np.uint64(63)).astype(np.uint32) << np.uint32(31)
    assert np.array_equal(b_out[tiny], sgn[tiny])
    # 2^128 and above, infinities included: an infinity of the input's sign
    assert np.array_equal(b_out[huge], sgn[huge] | np.uint32(0x7F800000))
    assert np.isnan(out32[nan]).all()
    assert mid.sum() > 100000 and tiny.sum() > 1000 and huge.sum() > 1000

    fnan = np.isnan(f)
    sub = ~fnan & (np.abs(f) < np.float32(2.0 ** -126)) & (f != 0)
    rest = ~fnan & ~sub
    assert np.array_equal(out64[rest].view(np.uint64), ref64[rest].view(np.uint64))
    assert np.array_equal(out64[rest], f[rest].astype(np.float64))
    fs = (f.view(np.uint32) >> np.uint32(31)).astype(np.uint64) << np.uint64(63)
    assert np.array_equal(out64[sub].view(np.uint64), fs[sub])
    assert np.isnan(out64[fnan]).all()
    assert sub.sum() >= 4
