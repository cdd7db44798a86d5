"""Pins of the demosaic oracle (CPU only).

Bilinear demosaicing (Section III.A) keeps a pixel's own colour and averages
the neighbours of each missing colour among its 8 direct neighbours.  The
oracle states that per pixel; these tests check it against a mosaic worked by
hand, flat fields, exact reproduction of linear intensity ramps away from the
border, the four-case description in the paper (orthogonal / diagonal /
horizontal / vertical pairs), mirror and transpose symmetries that relate the
four CFA patterns, and the detector-correction order (correct, then
interpolate).
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "demosaic_hand_example.txt")
RNG = np.random.default_rng(104)


def _golden():
    mosaic, pixels = [], []
    for line in open(GOLDEN):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "mosaic":
            mosaic.append([int(v) for v in line[1:]])
        elif line[0] == "pixel":
            pixels.append([int(v) for v in line[1:]])
    return np.array(mosaic, np.uint16), pixels


def test_hand_worked_mosaic():
    img, pixels = _golden()
    out = oracle.demosaic(img, "rggb")
    for y, x, r, g, b in pixels:
        assert out[:, y, x].tolist() == [r, g, b], (y, x)


@pytest.mark.parametrize("pattern", list(oracle.PATTERNS))
def test_flat_field_stays_flat(pattern):
    img = np.full((7, 9), 1234, np.uint16)
    assert (oracle.demosaic(img, pattern) == 1234).all()


def _cfa(pattern, h, w):
    """Colour index (0 R, 1 G, 2 B) of every photosite, from the pattern's name."""
    cells = {c: i for i, c in enumerate("rgb")}
    name = pattern
    cell = np.array([[cells[name[0]], cells[name[1]]], [cells[name[2]], cells[name[3]]]])
    return np.tile(cell, ((h + 1) // 2, (w + 1) // 2))[:h, :w]


@pytest.mark.parametrize("pattern", list(oracle.PATTERNS))
def test_linear_ramps_are_reproduced_inside(pattern):
    # each colour plane is an integer linear ramp with even slopes: every neighbour average of a
    # symmetric pair or quad equals the centre value exactly
    h, w = 12, 14
    yy, xx = np.mgrid[0:h, 0:w]
    planes = np.stack([100 + 2 * xx + 4 * yy, 3000 - 6 * xx + 2 * yy, 500 + 8 * xx + 10 * yy]).astype(np.uint16)
    cfa = _cfa(pattern, h, w)
    mosaic = np.choose(cfa, planes).astype(np.uint16)
    out = oracle.demosaic(mosaic, pattern)
    np.testing.assert_array_equal(out[:, 1:-1, 1:-1], planes[:, 1:-1, 1:-1])


def test_the_four_cases_of_the_paper():
    # red pixel: G from the 4 orthogonal, B from the 4 diagonal neighbours; blue pixel: the reverse;
    # green pixel in a red row: R from left/right, B from up/down; in a blue row: the reverse
    img = RNG.integers(0, 65536, size=(10, 10)).astype(np.uint16)
    out = oracle.demosaic(img, "rggb").astype(np.int64)
    v = img.astype(np.int64)
    avg = lambda *a: (sum(a) + len(a) // 2) // len(a)
    for y in range(1, 9):
        for x in range(1, 9):
            orth = avg(v[y - 1, x], v[y + 1, x], v[y, x - 1], v[y, x + 1])
            diag = avg(v[y - 1, x - 1], v[y - 1, x + 1], v[y + 1, x - 1], v[y + 1, x + 1])
            horiz, vert = avg(v[y, x - 1], v[y, x + 1]), avg(v[y - 1, x], v[y + 1, x])
            if y % 2 == 0 and x % 2 == 0:
                want = (v[y, x], orth, diag)
            elif y % 2 == 1 and x % 2 == 1:
                want = (diag, orth, v[y, x])
            elif y % 2 == 0:
                want = (horiz, v[y, x], vert)
            else:
                want = (vert, v[y, x], horiz)
            assert tuple(out[:, y, x]) == want, (y, x)


def test_mirror_and_transpose_relate_the_patterns():
    img = RNG.integers(0, 4096, size=(9, 12)).astype(np.uint16)
    # mirroring the columns of an RGGB mosaic gives a GRBG mosaic (12 columns: even width)
    np.testing.assert_array_equal(oracle.demosaic(np.ascontiguousarray(img[:, ::-1]), "grbg"),
                                  oracle.demosaic(img, "rggb")[:, :, ::-1])
    # mirroring the rows (9 rows: odd height) keeps row parity: RGGB stays RGGB
    np.testing.assert_array_equal(oracle.demosaic(np.ascontiguousarray(img[::-1]), "rggb"),
                                  oracle.demosaic(img, "rggb")[:, ::-1])
    # transposing swaps the two green sites and keeps R and B: RGGB -> RGGB, GRBG -> GBRG
    np.testing.assert_array_equal(oracle.demosaic(np.ascontiguousarray(img.T), "rggb"),
                                  np.transpose(oracle.demosaic(img, "rggb"), (0, 2, 1)))
    np.testing.assert_array_equal(oracle.demosaic(np.ascontiguousarray(img.T), "gbrg"),
                                  np.transpose(oracle.demosaic(img, "grbg"), (0, 2, 1)))


def test_degenerate_shapes():
    assert oracle.demosaic(np.zeros((0, 5), np.uint16)).shape == (3, 0, 5)
    one = oracle.demosaic(np.array([[77]], np.uint16), "rggb")
    assert one[:, 0, 0].tolist() == [77, 0, 0]  # no neighbour of the missing colours
    row = oracle.demosaic(np.array([[10, 20, 30]], np.uint16), "rggb")
    assert row[:, 0, 1].tolist() == [20, 20, 0] and row[:, 0, 0].tolist() == [10, 20, 0]


def test_correction_comes_before_interpolation():
    h, w, bits = 16, 20, 12
    img = synth.raster(9, 1, h, w, bits)[0]
    A, G, O = synth.coeffs(9, 0, w)
    lut = oracle.lutgen(A, G, O, bits)
    fused = oracle.demosaic(img, "gbrg", lut=lut, bits=bits)
    corrected = oracle.apply_u16(img, lut, bits)
    np.testing.assert_array_equal(fused, oracle.demosaic(np.ascontiguousarray(corrected), "gbrg"))
    # identity coefficients: the correction is the identity
    ident = oracle.lutgen(np.zeros(w, np.int32), np.full(w, 65536, np.int32), np.zeros(w, np.int32), bits)
    np.testing.assert_array_equal(oracle.demosaic(img, "rggb", lut=ident, bits=bits), oracle.demosaic(img, "rggb"))
