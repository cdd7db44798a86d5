"""Parity of the CUDA least-squares fit with the oracle (GPU).

Both sides solve the paper's normal equations in fp64, by different but
backward-stable routes (the oracle by the explicit inverse the paper writes,
the kernel by a Cholesky factorisation), so the coefficients agree to within
what the conditioning allows.  The tolerance is derived per column: in the
scaled basis t = x / 2^bits, where the coefficients b_k = a_k 2^(bits k) are of
comparable size, both results carry a relative error of order
kappa(V_t)^2 * eps (the normal matrix squares the condition number of the
Vandermonde matrix V_t), so the test allows 1000 * (m+1) * kappa^2 * eps of
the larger of |b| and |y|.  Status codes are integers decided exactly (a
count of distinct abscissae) and must match exactly.  Q16 codes are rounded
from fp64 values on both sides and must match wherever the oracle's value is
farther than the tolerance from a rounding boundary.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

import paper_1505_05655_gb300 as lutc  # noqa: E402
from paper_1505_05655_gb300 import _lib  # noqa: E402

EPS = np.finfo(np.float64).eps


def _tolerances(x, y, order, bits, coef_ref):
    """Per-column absolute tolerance on the scaled coefficients b_k = a_k 2^(bits k)."""
    ncols = x.shape[1]
    s = float(1 << bits)
    t = x.astype(np.float64) / s
    V = t[:, :, None] ** np.arange(order + 1)  # [n, ncols, m+1]
    kappa = np.linalg.cond(np.transpose(V, (1, 0, 2)))
    yabs = np.abs(y).max(axis=0) if y.ndim == 2 else np.full(ncols, np.abs(y).max())
    b = np.abs(coef_ref * s ** np.arange(order + 1)).max(axis=1)
    return 1000 * (order + 1) * kappa ** 2 * EPS * np.maximum(np.nan_to_num(b), yabs), kappa


def _check(x, y, order, bits, q16=False, x_pad=0, y_pad=0):
    n, ncols = x.shape
    xd = torch.zeros((n, ncols + x_pad), dtype=torch.uint16, device="cuda")[:, :ncols]
    xd.copy_(torch.from_numpy(x))
    if y.ndim == 2:
        yd = torch.zeros((n, ncols + y_pad), dtype=torch.float64, device="cuda")[:, :ncols]
        yd.copy_(torch.from_numpy(y))
    else:
        yd = torch.from_numpy(y).cuda()
    res = lutc.fit(xd, yd, order, q16=q16)
    torch.cuda.synchronize()
    ref = oracle.polyfit(x, np.ascontiguousarray(y), order, q16=q16)
    coef, st = res[0].cpu().numpy(), res[1].cpu().numpy()
    np.testing.assert_array_equal(st == 1, ref[1] == 1)  # singular columns: exact decision
    ok = ref[1] == 0
    tol, kappa = _tolerances(x, y, order, bits, ref[0])
    scale = float(1 << bits) ** np.arange(order + 1)
    diff = np.abs(coef - ref[0]) * scale
    bad = ok & ~(diff <= tol[:, None]).all(axis=1)
    assert not bad.any(), (np.flatnonzero(bad)[:5], diff[bad][:3], tol[bad][:3], kappa[bad][:3])
    assert np.isnan(coef[ref[1] == 1]).all()
    if q16:
        codes, rcodes = res[2].cpu().numpy(), ref[2]
        v = np.stack([ref[0][:, 2] if order >= 2 else np.zeros(ncols), ref[0][:, 1], ref[0][:, 0]]) * 65536.0
        # distance to the nearest rounding boundary, in code units, against the tolerance in code units
        dist = np.abs(np.abs(v) - np.floor(np.abs(v)) - 0.5)
        tol_codes = np.stack([tol / scale[min(2, order)] if order >= 2 else np.zeros_like(tol), tol / scale[1], tol]) * 65536.0
        clear = (dist > tol_codes) | ~np.isfinite(v)
        same = codes == rcodes
        assert (same | ~clear).all()
        np.testing.assert_array_equal(st[ok & (ref[1] != 2)], ref[1][ok & (ref[1] != 2)])
        # status 2 (out of range) is decided on |v| against 2^31 - 0.5: exact unless v sits on the edge
        assert ((st == 2) == (ref[1] == 2)).mean() > 0.999
    return res, ref


@pytest.mark.parametrize("order", [1, 2, 3])
def test_paper_shape_flat_field(order):
    # 6 calibration lines x 6000 detectors, 12-bit, 1 % dead detectors
    x, y = synth.calib(synth.CALIB_SEED, 6, 6000, 12, dead_frac=0.01)
    res, ref = _check(x, y, order, 12, q16=order <= 2)
    assert (ref[1] == 1).sum() > 20


@pytest.mark.parametrize("bits", [8, 10, 14, 16])
def test_bit_depths_and_ragged_width(bits):
    x, y = synth.calib(synth.CALIB_SEED + bits, 9, 3001, bits, dead_frac=0.003)
    for order in (1, 2, 3):
        _check(x, y, order, bits, q16=order <= 2, x_pad=13)


def test_per_sample_targets_with_padded_rows():
    rng = np.random.default_rng(7)
    n, ncols = 11, 1777
    x = rng.integers(0, 4096, size=(n, ncols)).astype(np.uint16)
    y = rng.normal(2000, 500, size=(n, ncols))
    for order in (1, 2, 3):
        _check(x, y, order, 12, q16=order <= 2, x_pad=5, y_pad=3)


def test_many_lines_and_many_columns():
    x, y = synth.calib(synth.CALIB_SEED + 1, 64, 24001, 14, dead_frac=0.001)
    _check(x, y, 2, 14, q16=True)


def test_singular_columns_and_out_of_range_codes():
    n, ncols = 6, 130
    x = np.tile(np.array([100, 900, 1700, 2500, 3300, 4000], np.uint16)[:, None], (1, ncols))
    y = np.tile(np.linspace(0, 4000, n)[:, None], (1, ncols))
    for c in range(0, 40):
        k = c % 4  # k + 1 distinct values
        x[:, c] = x[np.minimum(np.arange(n), k), c]
    y[:, 60:70] = 40000.0 * x[:, 60:70]  # gain 40000: outside Q16 int32
    for order in (1, 2, 3):
        res, ref = _check(x, np.ascontiguousarray(y), order, 12, q16=order <= 2)
        st = res[1].cpu().numpy()
        assert (st[:40] == 1).sum() == sum(1 for c in range(40) if c % 4 + 1 < order + 1)
        if order <= 2:
            assert (st[60:70] == 2).all() and (res[2].cpu().numpy()[:, 60:70] == 0).all()


def test_fit_feeds_the_lut():
    # calibration -> Q16 codes -> detector LUT, against the oracle's chain on the same codes
    x, y = synth.calib(synth.CALIB_SEED + 2, 6, 2048, 12)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    coef, st, codes = lutc.fit(xd, yd, 2, q16=True)
    rc = oracle.polyfit(x, y, 2, q16=True)
    agree = (codes.cpu().numpy() == rc[2]).all(axis=0)
    assert agree.mean() > 0.99
    A, G, O = codes[0].contiguous(), codes[1].contiguous(), codes[2].contiguous()
    lut = lutc.lutgen(A, G, O, 12).cpu().numpy()
    ref = oracle.lutgen(rc[2][0], rc[2][1], rc[2][2], 12)
    np.testing.assert_array_equal(lut[agree], ref[agree])
    # the LUT of the codes follows the fitted polynomial to within the Q16 rounding of the codes
    # (half a code on each of A, G, O: (x^2 + x + 1) / 2^17) plus the final rounding to a DN
    c = coef.cpu().numpy()
    xf = x.astype(np.float64)
    f = c[None, :, 0] + c[None, :, 1] * xf + c[None, :, 2] * xf ** 2
    D = lut[np.arange(2048)[None, :], x].astype(np.float64)
    bound = (xf ** 2 + xf + 1) / 131072.0 + 1.0
    assert (np.abs(D - np.clip(f, 0, 4095)) <= bound)[:, agree].all()


def test_arguments_are_checked():
    lib = _lib.lib()
    x = torch.zeros((6, 100), dtype=torch.uint16, device="cuda")
    y = torch.zeros(6, dtype=torch.float64, device="cuda")
    coef = torch.empty((100, 4), dtype=torch.float64, device="cuda")
    st = torch.empty(100, dtype=torch.int32, device="cuda")
    q = torch.empty((3, 100), dtype=torch.int32, device="cuda")
    E = _lib.LUTC_EINVAL
    args = lambda n, order, q16=None, xp=200: (x.data_ptr(), xp, y.data_ptr(), 0, n, 100, order, coef.data_ptr(),
                                               st.data_ptr(), q16, None)
    assert lib.lutc_fit(*args(6, 0)) == E
    assert lib.lutc_fit(*args(6, 4)) == E
    assert lib.lutc_fit(*args(3, 3)) == E  # n < order + 1
    assert lib.lutc_fit(*args(6, 3, q.data_ptr())) == E  # no Q16 form of a cubic
    assert lib.lutc_fit(*args(6, 1, xp=198)) == E
    assert lib.lutc_fit(x.data_ptr(), 200, y.data_ptr(), 0, 6, 0, 1, None, None, None, None) == 0
    assert lib.lutc_fit(*args(6, 2, q.data_ptr())) == 0
    torch.cuda.synchronize()
    assert (st.cpu() == 1).all()  # all-zero columns: one distinct abscissa
