"""The two-term FP16 split the tensor-core query projection relies on, checked in numpy.

The window side is split by Veltkamp's method in FP32 (t = 8193 x, x_hi = t - (t - x),
x_lo = x - x_hi), the basis side by rounding (x_hi = fp16(x), x_lo = fp16(x - x_hi)); the
projection accumulates u_hi b_hi + u_lo b_hi + u_hi b_lo, dropping u_lo b_lo.  These tests pin
what that arithmetic guarantees, independently of the kernel: x_hi is exact in FP16 in its
normal range, x_hi + x_lo = x exactly in FP32, the FP16 rounding of x_lo loses at most 2^-23 |x|
(an absolute 2^-25 below |x| = 2^-3, where x_lo is an FP16 subnormal), the three products land
far inside the 2^-17 ||u|| the GPU test allows per coordinate before the FP16 rounding, and
leaving out a cross term breaks that bound at the largest of many coordinates."""
import numpy as np

F32 = np.float32


def _veltkamp(x):
    x = x.astype(F32)
    t = (x * F32(8193.0)).astype(F32)
    hi = (t - (t - x).astype(F32)).astype(F32)
    lo = (x - hi).astype(F32)
    return hi, lo


def test_veltkamp_high_part_is_exact_in_fp16_and_the_split_is_exact():
    rng = np.random.default_rng(5)
    mags = 2.0 ** rng.uniform(-14, 15.9, 200_000)
    x = (mags * rng.choice([-1.0, 1.0], mags.size)).astype(F32)
    hi, lo = _veltkamp(x)
    assert np.all(hi.astype(np.float16).astype(F32) == hi)           # 11 significant bits, in range
    assert np.all((hi + lo).astype(F32) == x)                          # the split loses nothing
    lo16 = lo.astype(np.float16).astype(np.float64)
    assert np.all(np.abs(lo16 - lo.astype(np.float64)) <= np.maximum(2.0 ** -23 * np.abs(x.astype(np.float64)),
                                                                     2.0 ** -25))
    assert np.all(np.abs(lo) <= 2.0 ** -11 * np.abs(x))


def test_a_flat_window_keeps_an_exact_zero():
    hi, lo = _veltkamp(np.zeros(8, F32))
    assert np.all(hi == 0) and np.all(lo == 0)


def _split16(x):
    hi = x.astype(np.float16)
    return hi, (x - hi.astype(F32)).astype(F32).astype(np.float16)


def test_three_products_stay_inside_the_projection_tolerance():
    """Windows of D = 192 values (standard normal, and with entries spanning six decades) against
    32 orthonormal basis vectors: the exact products of the FP16 parts (what the tensor core
    multiplies), summed exactly, stay within 2^-20 ||u|| of u . b for every coordinate, far inside
    the GPU test's 2^-17 ||u|| (the FP32 accumulation of 3 D products adds a few 2^-24 ||u||).
    Leaving out u_lo b_hi moves each coordinate by about 2^-12.8 ||u|| / sqrt(D) (random signs),
    which passes 2^-17 ||u|| at the largest of the 16,000 coordinates."""
    rng = np.random.default_rng(7)
    D, n, d = 192, 500, 32
    B = np.linalg.qr(rng.standard_normal((D, d)))[0].T.astype(F32)  # d x D, orthonormal rows
    b_hi, b_lo = _split16(B)
    bh, bl = b_hi.astype(np.float64), b_lo.astype(np.float64)
    for scale in (np.ones((n, D)), 10.0 ** rng.uniform(-3, 3, (n, D))):
        U = (rng.standard_normal((n, D)) * scale).astype(F32)
        u_hi, u_lo = _veltkamp(U)
        uh, ul = u_hi.astype(np.float64), u_lo.astype(np.float16).astype(np.float64)
        exact = U.astype(np.float64) @ B.astype(np.float64).T
        nu = np.linalg.norm(U.astype(np.float64), axis=1)[:, None]
        three = uh @ bh.T + ul @ bh.T + uh @ bl.T
        assert np.max(np.abs(three - exact) / nu) <= 2.0 ** -20
        dropped = uh @ bh.T + uh @ bl.T
        assert np.max(np.abs(dropped - exact) / nu) > 2.0 ** -17
