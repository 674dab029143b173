"""The three-term FP16 split of the FP32 kernel's tensor-core lag grid (CPU).

The kernel scales each row of coefficients by the power of two that puts its
largest |z| in [2^14, 2^15), splits every value v into FP16 terms h1 = fp16(v),
h2 = fp16(v - h1), h3 = fp16(v - h1 - h2) (round to nearest even, as
cvt.rn.f16x2.f32), does the same to the weights, and sums six of the nine
cross products (z1 w1, z2 w1, z1 w2, z1 w3, z2 w2, z3 w1).  This test checks the
arithmetic facts that design rests on, in numpy: the FP32 differences are
exact, the split leaves less than 2^-33 of the row's largest value, and the six
products carry the dot product to within 2^-30 of sum |z w| plus, for terms
that reach FP16's subnormal range (at most 2^-25 each), 2^-38 of the largest
|z| and |w| times the other side's sum -- far below the FP32 evaluation's own
rounding.
"""
import numpy as np


def _row_scale(z):
    mx = np.float32(np.abs(z).max())
    eb = int(np.frombuffer(mx.tobytes(), dtype=np.uint32)[0] >> 23) & 0xFF
    return np.float32(2.0 ** (141 - eb))


def _split3(v):
    v = np.asarray(v, dtype=np.float32)
    h1 = v.astype(np.float16)
    r1 = v - h1.astype(np.float32)
    assert np.array_equal(r1.astype(np.float64), v.astype(np.float64) - h1.astype(np.float64))  # exact
    h2 = r1.astype(np.float16)
    r2 = r1 - h2.astype(np.float32)
    assert np.array_equal(r2.astype(np.float64), r1.astype(np.float64) - h2.astype(np.float64))  # exact
    h3 = r2.astype(np.float16)
    return h1.astype(np.float64), h2.astype(np.float64), h3.astype(np.float64)


def _rows(rng, n, k):
    # magnitudes spread over many binades inside a row, and rows of very different scale
    z = rng.standard_normal((n, k)) * 10.0 ** rng.uniform(-6, 2, (n, k))
    z *= 10.0 ** rng.uniform(-20, 20, (n, 1))
    return z.astype(np.float32)


def test_row_scale_puts_the_largest_value_in_range():
    rng = np.random.default_rng(1)
    for z in _rows(rng, 500, 32):
        s = _row_scale(z)
        m = float(np.abs(z * s).max())
        assert 2.0 ** 14 <= m < 2.0 ** 15
        # a power of two: scaling is exact
        assert np.array_equal((z * s).astype(np.float64), z.astype(np.float64) * float(s))


def test_three_terms_leave_less_than_2_pow_minus_33():
    rng = np.random.default_rng(2)
    for z in _rows(rng, 500, 32):
        v = z * _row_scale(z)
        h1, h2, h3 = _split3(v)
        res = np.abs(v.astype(np.float64) - (h1 + h2 + h3))
        assert res.max() <= 2.0 ** -33 * np.abs(v).max()


def test_six_products_carry_the_dot_product():
    rng = np.random.default_rng(3)
    n, k = 400, 16
    z = _rows(rng, n, k)
    w = (rng.uniform(-2, 2, (97, k)) * 10.0 ** rng.uniform(-4, 0, (97, k))).astype(np.float32)
    wsh = 15 - int(np.frexp(np.abs(w).max())[1])
    ws = (w * np.float32(2.0 ** wsh)).astype(np.float32)
    assert np.abs(ws).max() < 2.0 ** 15
    w1, w2, w3 = _split3(ws)
    aw = np.abs(ws).astype(np.float64)
    for zr in z:
        zs = zr * _row_scale(zr)
        z1, z2, z3 = _split3(zs)
        six = (w1 @ z1 + w1 @ z2 + w2 @ z1 + w3 @ z1 + w2 @ z2 + w1 @ z3)
        exact = ws.astype(np.float64) @ zs.astype(np.float64)
        az = np.abs(zs).astype(np.float64)
        bound = 2.0 ** -30 * (aw @ az) + 2.0 ** -38 * (az.max() * aw.sum(1) + aw.max() * az.sum())
        assert np.all(np.abs(six - exact) <= bound)
        # below 2^-28 of max|z| max|w|, where one FP32 rounding of a product is up to 2^-24 of it
        assert np.abs(six - exact).max() <= 2.0 ** -28 * az.max() * aw.max()
