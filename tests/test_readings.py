"""Equivalences the kernels rely on where they evaluate the method's tests in
another form than the oracle (CPU, numpy; no GPU).

CW84's overshoot tests on a parabola of zone value a0 between edges L and R,
dA (a0 - (L + R)/2) > dA^2 / 6 and -dA^2 / 6 > dA (a0 - (L + R)/2) with
dA = R - L, hold exactly when |x| > 2|y| and |y| > 2|x| respectively, for
x = a0 - L and y = R - a0 of one sign; and van Leer's dl dr > 0 is the test
that dl and dr share a sign.  The product forms and the comparisons agree
wherever the products neither round across their threshold nor underflow.
"""
import numpy as np

from paper_2007_05218_gb300 import inputs


def _samples(n, seed):
    u = inputs.uniform01(seed, 0, np.arange(3 * n)).reshape(3, n)
    a0 = 2.0 * u[0] - 1.0
    L = a0 - (2.0 * u[1] - 1.0) * 10.0 ** (-3.0 * u[2])
    R = a0 + (2.0 * inputs.uniform01(seed, 1, np.arange(n)) - 1.0) * 10.0 ** (-3.0 * u[2][::-1])
    return a0, L, R


def test_cw84_product_tests_are_the_twice_comparisons():
    a0, L, R = _samples(200_000, 11)
    x, y = a0 - L, R - a0
    one_sign = x * y > 0
    dA = R - L
    mid = a0 - 0.5 * (L + R)
    left = dA * mid > dA * dA / 6.0      # L overshoots: replaced by 3 a0 - 2 R
    right = -(dA * dA) / 6.0 > dA * mid  # R overshoots: replaced by 3 a0 - 2 L
    # away from the boundary |x| = 2|y| (where both forms may round either way)
    clear = np.abs(np.abs(x) - 2.0 * np.abs(y)) > 1e-9 * (np.abs(x) + np.abs(y))
    clear &= np.abs(np.abs(y) - 2.0 * np.abs(x)) > 1e-9 * (np.abs(x) + np.abs(y))
    m = one_sign & clear
    assert m.sum() > 100_000
    assert np.array_equal(left[m], (np.abs(x) > 2.0 * np.abs(y))[m])
    assert np.array_equal(right[m], (np.abs(y) > 2.0 * np.abs(x))[m])
    # both kinds of overshoot occur in the sample
    assert left[m].any() and right[m].any() and (~left[m] & ~right[m]).any()


def _cw84_limit(a0, L, R):
    """CW84's monotonicity limiter in the comparison form (no flattening)."""
    x, y = a0 - L, R - a0
    one_sign = x * y > 0
    lo = one_sign & (np.abs(x) > 2.0 * np.abs(y))
    hi = one_sign & ~lo & (np.abs(y) > 2.0 * np.abs(x))
    Ln = np.where(~one_sign, a0, np.where(lo, a0 - 2.0 * y, L))
    Rn = np.where(~one_sign, a0, np.where(hi, a0 + 2.0 * x, R))
    return Ln, Rn


def test_cw84_limited_edges_are_continuous_across_the_test_boundary():
    """An edge just inside and just outside |x| = 2|y| gives edges within
    the distance of the two inputs, so either rounding of the test gives
    nearly the same parabola."""
    a0, _, R = _samples(10_000, 12)
    y = R - a0
    for eps in (1e-6, 1e-9):
        L_in = a0 - 2.0 * y * (1.0 - eps)    # |x| just below 2|y|: kept
        L_out = a0 - 2.0 * y * (1.0 + eps)   # just above: replaced by a0 - 2y
        Li, Ri = _cw84_limit(a0, L_in, R)
        Lo, Ro = _cw84_limit(a0, L_out, R)
        bound = 4.0 * eps * np.abs(y) + 8.0 * np.spacing(np.abs(a0) + 2.0 * np.abs(y))
        assert np.all(np.abs(Li - Lo) <= bound)
        np.testing.assert_array_equal(Ri, Ro)


def test_van_leer_product_test_is_the_sign_test_until_it_underflows():
    a0, L, R = _samples(100_000, 13)
    dl, dr = a0 - L, R - a0
    np.testing.assert_array_equal(dl * dr > 0, np.sign(dl) * np.sign(dr) > 0)
    # factors of 1e-170 and 3e-200: the product underflows to zero, the sign test still sees one sign
    dl_t, dr_t = 1e-170, 3e-200
    assert not (dl_t * dr_t > 0)
    assert np.sign(dl_t) == np.sign(dr_t) != 0
