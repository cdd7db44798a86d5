"""Pins of the CPU oracle to facts fixed outside it (CPU only).

Each test checks the oracle against something it does not compute itself:
hand-worked values (``tests/golden``), closed forms (identity and offset
responses), an independent exact-rational statement of the rounding, library
routines (numpy sort / bincount / fancy indexing) and pure-Python brute force
on tiny rasters.  A plausible slip in the oracle -- a dropped rounding term,
truncating instead of flooring a negative sum, a transposed table index, an
off-by-one percentile rank, a missed clamp -- fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _exact_entry(A, G, O, x, bits):
    """Step (L) stated independently: round half up of the exact rational, then clamp."""
    M = (1 << bits) - 1
    v = math.floor(Fraction(A * x * x + G * x + O, 65536) + Fraction(1, 2))
    return min(max(v, 0), M)


def _exact_S(v, lo, hi):
    """Step (S) stated independently: round half up of 255 (v - lo) / (hi - lo), clamped."""
    if hi == lo or v <= lo:
        return 0
    return min(255, math.floor(Fraction(255 * (v - lo), hi - lo) + Fraction(1, 2)))


def _read_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- step (L)

def test_lut_hand_examples():
    rows = _read_rows("lut_hand_examples.txt")
    assert len(rows) >= 10
    for name, A, G, O, bits, x, s, expected in rows:
        A, G, O, bits, x, s, expected = map(int, (A, G, O, bits, x, s, expected))
        assert A * x * x + G * x + O + 32768 == s, (name, x)  # the worked sum itself
        assert oracle.lut_entry(A, G, O, x, bits) == expected, (name, x)
        lut = oracle.lutgen(np.array([A], np.int32), np.array([G], np.int32), np.array([O], np.int32), bits)
        assert int(lut[0, x]) == expected, (name, x)


@pytest.mark.parametrize("bits", [8, 10, 12, 14, 16])
def test_identity_response_gives_identity_lut(bits):
    n = 3
    lut = oracle.lutgen(np.zeros(n, np.int32), np.full(n, 65536, np.int32), np.zeros(n, np.int32), bits)
    ref = np.arange(1 << bits, dtype=np.uint16)
    for c in range(n):
        np.testing.assert_array_equal(lut[c], ref)


@pytest.mark.parametrize("k", [-7, 0, 5, 300, -5000])
def test_pure_offset_shifts_and_clamps(k):
    bits = 12
    M = (1 << bits) - 1
    lut = oracle.lutgen(np.zeros(1, np.int32), np.full(1, 65536, np.int32), np.full(1, k * 65536, np.int32), bits)
    x = np.arange(1 << bits)
    np.testing.assert_array_equal(lut[0], np.clip(x + k, 0, M).astype(np.uint16))


@pytest.mark.parametrize("bits", [8, 10, 12, 14, 16])
def test_lut_matches_exact_rational(bits):
    rng = np.random.default_rng(100 + bits)
    M = (1 << bits) - 1
    extremes = [-(2 ** 31), 2 ** 31 - 1, -1, 0, 1]
    cols = []
    for _ in range(40):
        cols.append((int(rng.integers(-3, 4)), int(rng.integers(50000, 80000)), int(rng.integers(-2_000_000, 2_000_000))))
    for a in extremes:
        for g in extremes:
            cols.append((a, g, int(rng.choice(extremes))))
    A = np.array([c[0] for c in cols], np.int32)
    G = np.array([c[1] for c in cols], np.int32)
    O = np.array([c[2] for c in cols], np.int32)
    lut = oracle.lutgen(A, G, O, bits)
    xs = sorted(set([0, 1, 2, M // 3, M // 2, M - 1, M] + [int(v) for v in rng.integers(0, M + 1, 40)]))
    for c, (a, g, o) in enumerate(cols):
        for x in xs:
            assert int(lut[c, x]) == _exact_entry(a, g, o, x, bits), (a, g, o, x, bits)


def test_lut_monotone_for_nonnegative_curvature():
    rng = np.random.default_rng(7)
    bits = 12
    A = rng.integers(0, 3, 64).astype(np.int32)
    G = rng.integers(1, 90000, 64).astype(np.int32)
    O = rng.integers(-2_000_000, 2_000_000, 64).astype(np.int32)
    lut = oracle.lutgen(A, G, O, bits).astype(np.int64)
    assert np.all(np.diff(lut, axis=1) >= 0)


# ---------------------------------------------------------------- step (P)

def test_apply_identity_lut_returns_input():
    rng = np.random.default_rng(1)
    bits = 12
    img = rng.integers(0, 1 << bits, (37, 53)).astype(np.uint16)
    lut = np.tile(np.arange(1 << bits, dtype=np.uint16), (53, 1))
    np.testing.assert_array_equal(oracle.apply_u16(img, lut, bits), img)


@pytest.mark.parametrize("bits", [8, 10, 12])
def test_apply_is_per_column_gather(bits):
    rng = np.random.default_rng(bits)
    M = (1 << bits) - 1
    h, w = 29, 41
    img = rng.integers(0, 65536, (h, w)).astype(np.uint16)  # also DN above M
    img[0, :] = M
    lut = rng.integers(0, 1 << bits, (w, 1 << bits)).astype(np.uint16)
    expect = lut[np.arange(w)[None, :], np.minimum(img, M)]  # numpy fancy indexing
    np.testing.assert_array_equal(oracle.apply_u16(img, lut, bits), expect)
    # a non-contiguous (pitched) view gives the same answer
    big = np.zeros((h, w + 11), np.uint16)
    big[:, :w] = img
    np.testing.assert_array_equal(oracle.apply_u16(big[:, :w], lut, bits), expect)


# ---------------------------------------------------------------- step (H)

@pytest.mark.parametrize("bits", [10, 12, 14])
def test_hist_sums_to_pixel_count_and_matches_bincount(bits):
    rng = np.random.default_rng(bits + 50)
    h, w = 31, 47
    M = (1 << bits) - 1
    img = rng.integers(0, 1 << bits, (h, w)).astype(np.uint16)
    ident = oracle.lutgen(np.zeros(w, np.int32), np.full(w, 65536, np.int32), np.zeros(w, np.int32), bits)
    hi = oracle.hist(img, ident, bits)
    assert int(hi.sum()) == h * w
    np.testing.assert_array_equal(hi, np.bincount(img.ravel(), minlength=M + 1).astype(np.uint64))
    # with a real response the histogram is the bincount of the corrected band
    A = rng.integers(-1, 2, w).astype(np.int32)
    G = rng.integers(58982, 72090, w).astype(np.int32)
    O = rng.integers(-1310720, 1310720, w).astype(np.int32)
    lut = oracle.lutgen(A, G, O, bits)
    corr = lut[np.arange(w)[None, :], img]
    np.testing.assert_array_equal(oracle.hist(img, lut, bits), np.bincount(corr.ravel(), minlength=M + 1).astype(np.uint64))


def test_hist_dead_column_spike():
    bits = 12
    h, w = 20, 10
    img = np.full((h, w), 1000, np.uint16)
    img[:, [2, 5, 7]] = 0  # three dead detectors
    A = np.zeros(w, np.int32)
    G = np.full(w, 65536, np.int32)
    O = np.zeros(w, np.int32)
    O[[2, 5, 7]] = 3 * 65536  # dead columns read D[c][0] = 3
    hi = oracle.hist(img, oracle.lutgen(A, G, O, bits), bits)
    assert int(hi[3]) == 3 * h and int(hi[1000]) == 7 * h and int(hi.sum()) == h * w


# ---------------------------------------------------------------- step (S)

def test_stretch_golden():
    rows = _read_rows("stretch_examples.txt")
    bits = 12
    it = iter(rows)
    checked = 0
    for row in it:
        if row[0] == "values":
            vals = np.array(list(map(int, row[1:])))
            hist = np.bincount(vals, minlength=1 << bits).astype(np.uint64)
            lo_hi = next(it)
            S, lo, hi = oracle.stretch(hist, bits)
            assert (lo, hi) == (int(lo_hi[1]), int(lo_hi[2]))
            checked += 1
        elif row[0] == "hist":
            pairs = list(map(int, row[1:]))
            hist = np.zeros(1 << bits, np.uint64)
            for v, n in zip(pairs[0::2], pairs[1::2]):
                hist[v] = n
            lo_hi = next(it)
            S, lo, hi = oracle.stretch(hist, bits)
            assert (lo, hi) == (int(lo_hi[1]), int(lo_hi[2]))
            srow = next(it)
            assert srow[0] == "S"
            sv = list(map(int, srow[1:]))
            for v, s in zip(sv[0::2], sv[1::2]):
                assert int(S[v]) == s, v
            checked += 1
    assert checked == 2


@pytest.mark.parametrize("n", [1, 2, 7, 49, 50, 51, 99, 100, 101, 1000, 4321])
def test_stretch_percentiles_by_sorting(n):
    bits = 10
    rng = np.random.default_rng(n)
    vals = rng.integers(0, 1 << bits, n)
    hist = np.bincount(vals, minlength=1 << bits).astype(np.uint64)
    S, lo, hi = oracle.stretch(hist, bits)
    s = np.sort(vals)  # library sort; rank k = ceil(pN / 100), 1-based
    assert lo == int(s[(2 * n + 99) // 100 - 1])
    assert hi == int(s[(98 * n + 99) // 100 - 1])
    for v in range(1 << bits):
        assert int(S[v]) == _exact_S(v, lo, hi), v
    if hi > lo:
        assert S[lo] == 0 and S[hi] == 255
    assert np.all(np.diff(S.astype(np.int64)) >= 0)


def test_stretch_degenerate_cases():
    bits = 12
    hist = np.zeros(1 << bits, np.uint64)
    hist[777] = 1234  # constant band: hi == lo -> all zero
    S, lo, hi = oracle.stretch(hist, bits)
    assert lo == hi == 777 and not S.any()
    S, lo, hi = oracle.stretch(np.zeros(1 << bits, np.uint64), bits)  # empty band
    assert lo == hi == 0 and not S.any()
    hist = np.zeros(1 << bits, np.uint64)
    hist[0] = 1
    hist[4095] = 1  # two pixels: rank 1 -> lo = 0, rank 2 -> hi = 4095
    S, lo, hi = oracle.stretch(hist, bits)
    assert (lo, hi) == (0, 4095) and S[0] == 0 and S[4095] == 255 and S[2048] == 128


# ---------------------------------------------------------------- steps (C), (A)

def test_compose_then_apply_equals_stretch_after_detector():
    rng = np.random.default_rng(3)
    bits = 12
    h, w = 23, 19
    img = rng.integers(0, 1 << bits, (h, w)).astype(np.uint16)
    A = rng.integers(-1, 2, w).astype(np.int32)
    G = rng.integers(58982, 72090, w).astype(np.int32)
    O = rng.integers(-1310720, 1310720, w).astype(np.int32)
    lut = oracle.lutgen(A, G, O, bits)
    S = rng.integers(0, 256, 1 << bits).astype(np.uint8)
    clut = oracle.compose(lut, S, bits)
    np.testing.assert_array_equal(oracle.apply_u8(img, clut, bits), S[oracle.apply_u16(img, lut, bits)])


def _brute_force_correct(raster, A, G, O, bits):
    """Pure-Python statement of the whole correction on a tiny raster."""
    M = (1 << bits) - 1
    bands, h, w = raster.shape
    out = np.zeros((bands, h, w), np.uint8)
    lohis = []
    for b in range(bands):
        corr = [[_exact_entry(int(A[b][c]), int(G[b][c]), int(O[b][c]), min(int(raster[b, y, c]), M), bits)
                 for c in range(w)] for y in range(h)]
        flat = sorted(v for row in corr for v in row)
        n = len(flat)
        lo = flat[-(-2 * n // 100) - 1]
        hi = flat[-(-98 * n // 100) - 1]
        lohis.append((lo, hi))
        for y in range(h):
            for c in range(w):
                out[b, y, c] = _exact_S(corr[y][c], lo, hi)
    return out, lohis


@pytest.mark.parametrize("bits,h,w", [(8, 5, 7), (10, 9, 4), (12, 6, 13)])
def test_correct_image_brute_force(bits, h, w):
    rng = np.random.default_rng(bits * 1000 + h)
    bands = 2
    raster = rng.integers(0, 1 << bits, (bands, h, w)).astype(np.uint16)
    raster[0, 0, 0] = 65535  # above M: reads entry M
    A = rng.integers(-2, 3, (bands, w)).astype(np.int32)
    G = rng.integers(50000, 80000, (bands, w)).astype(np.int32)
    O = rng.integers(-3_000_000, 3_000_000, (bands, w)).astype(np.int32)
    out, (hist, S, lohi) = oracle.correct_image(raster, A, G, O, bits, stretch=True, with_tables=True)
    ref, ref_lohi = _brute_force_correct(raster, A, G, O, bits)
    np.testing.assert_array_equal(out, ref)
    assert [tuple(map(int, r)) for r in lohi] == ref_lohi
    assert [int(hh.sum()) for hh in hist] == [h * w] * bands
    # detector-only output is the per-pixel exact entry
    out16 = oracle.correct_image(raster, A, G, O, bits, stretch=False)
    M = (1 << bits) - 1
    for b in range(bands):
        for y in range(h):
            for c in range(w):
                assert int(out16[b, y, c]) == _exact_entry(int(A[b, c]), int(G[b, c]), int(O[b, c]),
                                                           min(int(raster[b, y, c]), M), bits)
