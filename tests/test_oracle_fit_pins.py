"""Pins of the least-squares fit oracle (CPU only).

The fit (Section III.B, case study 2) minimises the summed squared error of a
polynomial of order m over each column's samples.  The oracle follows the
paper's normal equations and explicit inverse; these tests check it against
facts that do not come from those equations: exact recovery of polynomial
data, interpolation through m+1 points, the textbook closed form of the
straight-line fit, an SVD-based library least-squares solve of the
Vandermonde system, the defining minimum property, and exact Q16 codes of
the hand example H1 (A=1, G=68813, O=-478413).
"""
import numpy as np
import pytest

import oracle
import synth

RNG = np.random.default_rng(20150521)


def _fit(x, y, order, q16=False):
    x = np.ascontiguousarray(np.asarray(x, np.uint16).reshape(len(x), -1))
    y = np.asarray(y, np.float64)
    y = np.ascontiguousarray(y.reshape(len(y), -1)) if y.ndim > 1 else np.ascontiguousarray(y)
    return oracle.polyfit(x, y, order, q16=q16)


def _vander(x, order):
    return np.vander(np.asarray(x, np.float64), order + 1, increasing=True)


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("n", [None, 6, 40])
def test_polynomial_data_is_recovered_exactly(order, n):
    n = order + 1 if n is None else n
    for trial in range(20):
        x = RNG.choice(4096, size=n, replace=False)
        # dyadic coefficients: y is exact in fp64, the fit's only error is rounding
        a = RNG.integers(-64, 64, size=order + 1) / np.array([1, 64, 65536, 2 ** 24][:order + 1])
        y = sum(float(a[k]) * x.astype(np.float64) ** k for k in range(order + 1))
        coef, st = _fit(x, y, order)
        assert st[0] == 0
        # compare in the column's natural scale: coefficient k times 4096^k
        scale = 4096.0 ** np.arange(order + 1)
        np.testing.assert_allclose(coef[0] * scale, a * scale, rtol=0, atol=1e-6 * max(1.0, np.abs(a * scale).max()))


@pytest.mark.parametrize("order", [1, 2, 3])
def test_m_plus_one_points_are_interpolated(order):
    for trial in range(20):
        x = RNG.choice(16384, size=order + 1, replace=False)
        y = RNG.uniform(-1000, 17000, size=order + 1)
        coef, st = _fit(x, y, order)
        assert st[0] == 0
        fx = _vander(x, order) @ coef[0]
        # normal equations square the conditioning of the (scaled) Vandermonde matrix
        kappa = np.linalg.cond(_vander(x / 16384.0, order))
        np.testing.assert_allclose(fx, y, rtol=0, atol=100 * kappa ** 2 * 2.2e-16 * np.abs(y).max())


def test_straight_line_matches_the_closed_form():
    for trial in range(50):
        n = int(RNG.integers(2, 30))
        x = RNG.integers(0, 65536, size=n).astype(np.uint16)
        if len(np.unique(x)) < 2:
            continue
        y = RNG.normal(1000, 300, size=n)
        coef, st = _fit(x, y, 1)
        xf = x.astype(np.float64)
        # textbook regression line through the centroid: slope = Sxy / Sxx
        xm, ym = xf.mean(), y.mean()
        slope = np.sum((xf - xm) * (y - ym)) / np.sum((xf - xm) ** 2)
        icpt = ym - slope * xm
        np.testing.assert_allclose(coef[0, 1], slope, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(coef[0, 0], icpt, rtol=1e-9, atol=1e-6)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_matches_svd_least_squares_on_noisy_calibration_lines(order):
    # flat-field lines of the calibration recipe, 12 bits, 6 lines x 300 detectors
    x, y = synth.calib(synth.CALIB_SEED, 6, 300, 12)
    coef, st = oracle.polyfit(x, y, order)
    assert (st == 0).all()
    for c in range(0, 300, 7):
        # scaled abscissa so that the library solve is well conditioned; convert back exactly
        t = x[:, c].astype(np.float64) / 4096.0
        sol, *_ = np.linalg.lstsq(_vander(t, order), y, rcond=None)
        ref = sol / 4096.0 ** np.arange(order + 1)
        V = _vander(x[:, c], order)
        # compare the fitted values at the samples (well conditioned) and the coefficients
        np.testing.assert_allclose(V @ coef[c], V @ ref, rtol=0, atol=1e-7)
        np.testing.assert_allclose(coef[c] * 4096.0 ** np.arange(order + 1), sol, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_result_is_the_minimum(order):
    for trial in range(10):
        n = int(RNG.integers(order + 2, 20))
        x = RNG.choice(4096, size=n, replace=False)
        y = RNG.uniform(0, 4095, size=n)
        coef, st = _fit(x, y, order)
        V = _vander(x, order)
        base = np.sum((y - V @ coef[0]) ** 2)
        for k in range(order + 1):
            step = 1e-2 / 4096.0 ** k
            for sgn in (-1, 1):
                a = coef[0].copy()
                a[k] += sgn * step
                assert np.sum((y - V @ a) ** 2) > base
        # first-order conditions: residual orthogonal to every power of x
        r = y - V @ coef[0]
        scale = np.abs(V).max(axis=0) * np.abs(y).max() * n
        assert np.all(np.abs(V.T @ r) <= 1e-9 * scale)


def test_too_few_distinct_abscissae_is_singular():
    x = np.array([[7, 9], [7, 9], [7, 12], [7, 9]], np.uint16)  # column 0: one value; column 1: two
    y = np.array([1.0, 2.0, 3.0, 4.0])
    coef, st = oracle.polyfit(x, y, 1)
    assert st.tolist() == [1, 0] and np.isnan(coef[0]).all() and np.isfinite(coef[1]).all()
    coef, st = oracle.polyfit(x, y, 2)
    assert st.tolist() == [1, 1]
    x[3, 1] = 20
    assert oracle.polyfit(x, y, 2)[1].tolist() == [1, 0]


def test_q16_codes_of_the_hand_example():
    # H1: A=1, G=68813, O=-478413 in Q16.  Data exactly on that polynomial give the codes back.
    a = np.array([-478413, 68813, 1], np.float64) / 65536.0
    x = np.array([0, 700, 1500, 2000, 3100, 4095], np.uint16)
    y = a[0] + a[1] * x + a[2] * x.astype(np.float64) ** 2
    coef, st, q = _fit(x, y, 2, q16=True)
    assert st[0] == 0 and q[:, 0].tolist() == [1, 68813, -478413]
    # order 1 on straight-line data: A is 0
    y1 = a[0] + a[1] * x
    coef, st, q = _fit(x, y1, 1, q16=True)
    assert st[0] == 0 and q[:, 0].tolist() == [0, 68813, -478413]
    # a gain of 40000 does not fit in Q16 int32: status 2, codes 0
    coef, st, q = _fit(x, 40000.0 * x, 1, q16=True)
    assert st[0] == 2 and q[:, 0].tolist() == [0, 0, 0]
    # rounding half away from zero: O = 2.5 / 65536 and -2.5 / 65536 -> codes 3 and -3
    for o, want in ((2.5, 3), (-2.5, -3)):
        coef, st, q = _fit(x, o / 65536.0 + x, 1, q16=True)
        assert q[:, 0].tolist() == [0, 65536, want]


def test_per_column_targets_and_shared_targets_agree():
    x, y = synth.calib(synth.CALIB_SEED, 6, 200, 14, dead_frac=0.05)
    c1, s1 = oracle.polyfit(x, y, 2)
    c2, s2 = oracle.polyfit(x, np.ascontiguousarray(np.repeat(y[:, None], 200, axis=1)), 2)
    assert (s1 == s2).all() and (s1 == 1).sum() > 0
    ok = s1 == 0
    np.testing.assert_array_equal(c1[ok], c2[ok])


def test_fit_inverts_the_calibration_response():
    # the flat-field recipe reads x ~ b + h L + q L^2; the order-2 fit of L on x is close to its inverse
    x, y = synth.calib(synth.CALIB_SEED, 12, 500, 12)
    coef, st = oracle.polyfit(x, y, 2)
    pred = np.stack([_vander(x[:, c], 2) @ coef[c] for c in range(500)], axis=1)
    unclipped = ((x > 0) & (x < 4095)).all(axis=0)
    assert unclipped.sum() > 400
    # noise sigma 2 DN in x and gains near 1: residuals of a few DN
    assert np.abs(pred - y[:, None])[:, unclipped].max() < 12.0
