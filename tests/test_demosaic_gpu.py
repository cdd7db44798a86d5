"""Parity of the CUDA bilinear demosaic with the oracle (GPU).

Integer arithmetic throughout: tolerance zero.  Shapes span several tiles
(128 x 32 or 128 x 64 on the TMA-fed path, which raw frames take above 4 M
pixels; 128 x 16 or 128 x 32 on the plain one) with ragged right and bottom edges, tiles whose halo leaves the image,
degenerate images one pixel wide or high, unaligned rows on both sides, coefficient
rows off a 16-byte boundary (no TMA staging of the coefficients), all
four CFA patterns, with and without the fused detector correction (int32 and
int64 columns), the paper's 2048 x 2048 16-bit frame in full and a frame
larger than L2 on sampled row bands.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

import paper_1505_05655_gb300 as lutc  # noqa: E402
from paper_1505_05655_gb300 import _lib  # noqa: E402

PATTERNS = list(oracle.PATTERNS)


def _raw(seed, h, w, bits, pad=0):
    img = np.zeros((h, w + pad), np.uint16)
    if h and w:
        img[:, :w] = synth.raster(seed, 1, h, w, bits, sat_frac=0.002)[0]
    return img


def _gpu(img, w, pattern, bits, coeffs=None, in_off=0, out_pad=0):
    h = img.shape[0]
    # in_off shifts the raster by whole elements inside a larger buffer (2-byte aligned, not 16)
    buf = torch.zeros(img.size + 8, dtype=torch.uint16, device="cuda")
    buf[in_off:in_off + img.size] = torch.from_numpy(img.reshape(-1)).cuda()
    raw = buf[in_off:in_off + img.size].view(img.shape)[:, :w]
    out = torch.full((3, h, w + out_pad), 0xBEEF, dtype=torch.uint16, device="cuda")[:, :, :w]
    kw = {}
    if coeffs is not None:
        kw = dict(A=torch.from_numpy(coeffs[0]).cuda(), G=torch.from_numpy(coeffs[1]).cuda(),
                  O=torch.from_numpy(coeffs[2]).cuda())
    lutc.demosaic(raw, pattern, bits, out=out, **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _ref(img, w, pattern, bits, coeffs=None):
    lut = oracle.lutgen(*coeffs, bits) if coeffs is not None else None
    return oracle.demosaic(np.ascontiguousarray(img[:, :w]), pattern, lut=lut, bits=bits)


SHAPES = [(67, 300), (33, 129), (32, 128), (64, 256), (100, 1030), (1, 1), (1, 7), (2, 2), (5, 1), (3, 9), (130, 8)]


@pytest.mark.parametrize("pattern", PATTERNS)
@pytest.mark.parametrize("h,w", SHAPES)
def test_raw_values(pattern, h, w):
    img = _raw(11 + h + w, h, w, 16)
    np.testing.assert_array_equal(_gpu(img, w, pattern, 16), _ref(img, w, pattern, 16))


@pytest.mark.parametrize("pattern", PATTERNS)
@pytest.mark.parametrize("bits", [10, 12, 14])
def test_fused_detector_correction(pattern, bits):
    h, w = 97, 517
    img = _raw(bits, h, w, bits)
    A, G, O = synth.coeffs(bits, 0, w)
    # a few columns whose range needs the int64 evaluation, and DN above M
    A[::37] = 900
    img[::5, ::7] = 65535
    np.testing.assert_array_equal(_gpu(img, w, pattern, bits, (A, G, O)), _ref(img, w, pattern, bits, (A, G, O)))


# 16-byte aligned rows: the vector staging path, ragged in both directions, pitches padded to 16 bytes
ALIGNED_SHAPES = [(67, 304, 0), (100, 1032, 0), (35, 144, 0), (34, 152, 0), (300, 1160, 0), (97, 300, 4), (259, 517, 3),
              (1000, 2048, 0), (66, 144, 0), (130, 152, 0)]


@pytest.mark.parametrize("pattern", PATTERNS)
@pytest.mark.parametrize("h,w,pad", ALIGNED_SHAPES)
def test_aligned_rows_raw_and_corrected(pattern, h, w, pad):
    bits = 12
    img = _raw(7 + h + w, h, w, bits, pad=pad)
    assert (img.strides[0] % 16) == 0
    A, G, O = synth.coeffs(7 + h, 0, w)
    A[::29] = 900  # int64 columns
    np.testing.assert_array_equal(_gpu(img, w, pattern, bits), _ref(img, w, pattern, bits))
    np.testing.assert_array_equal(_gpu(img, w, pattern, bits, (A, G, O)), _ref(img, w, pattern, bits, (A, G, O)))


@pytest.mark.parametrize("bits", [8, 10, 14, 15, 16])
@pytest.mark.parametrize("h,w", [(66, 152), (129, 304), (197, 1032)])
def test_aligned_rows_corrected_every_bit_depth(bits, h, w):
    # the TMA-fed corrected path at every bit depth (two DN clamped per instruction up to 15 bits,
    # one at 16) on frames of one, two and four 64-row tiles, ragged; int64 columns and DN above M
    img = _raw(40 + bits + h, h, w, bits)
    img[::9, ::11] = 65535
    A, G, O = synth.coeffs(40 + bits, 0, w)
    A[::31] = 900
    for pattern in ("rggb", "grbg"):
        np.testing.assert_array_equal(_gpu(img, w, pattern, bits, (A, G, O)), _ref(img, w, pattern, bits, (A, G, O)))


@pytest.mark.parametrize("in_off,pad,out_pad", [(1, 3, 1), (3, 0, 5), (0, 8, 0), (5, 1, 3)])
def test_unaligned_rows(in_off, pad, out_pad):
    h, w = 45, 263
    img = _raw(3, h, w, 12, pad=pad)
    A, G, O = synth.coeffs(3, 0, w)
    for coeffs in (None, (A, G, O)):
        got = _gpu(img, w, "grbg", 12, coeffs, in_off=in_off, out_pad=out_pad)
        np.testing.assert_array_equal(got, _ref(img, w, "grbg", 12, coeffs))


@pytest.mark.parametrize("coef_off", [1, 2, 3])
def test_unaligned_coefficient_rows(coef_off):
    # aligned raster rows (tiles through TMA) but coefficient rows 4 bytes off a 16-byte boundary:
    # the coefficients cannot travel with the tiles and are loaded per tile instead
    h, w, bits = 67, 304, 12
    img = _raw(9 + coef_off, h, w, bits)
    A, G, O = synth.coeffs(9 + coef_off, 0, w)
    A[::29] = 900  # int64 columns

    def shifted(a):
        buf = torch.zeros(w + 4, dtype=torch.int32, device="cuda")
        buf[coef_off:coef_off + w] = torch.from_numpy(a).cuda()
        return buf[coef_off:coef_off + w]

    for pattern in ("rggb", "gbrg"):
        out = lutc.demosaic(torch.from_numpy(img).cuda(), pattern, bits, A=shifted(A), G=shifted(G), O=shifted(O))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), _ref(img, w, pattern, bits, (A, G, O)))


@pytest.mark.parametrize("h,w,pad", [(2050, 2048, 0), (1031, 4104, 8), (2100, 2000, 0)])
def test_raw_frames_above_4m_pixels_take_the_tma_kernel(h, w, pad):
    # raw frames of more than 4 M pixels with aligned rows run the TMA-fed persistent kernel (smaller
    # raw frames the block-per-tile one): ragged in both directions, every pattern, 16-bit
    assert h * w > (1 << 22)
    img = _raw(60 + h, h, w, 16, pad=pad)
    assert (img.strides[0] % 16) == 0
    for pattern in PATTERNS:
        np.testing.assert_array_equal(_gpu(img, w, pattern, 16), _ref(img, w, pattern, 16))


def test_paper_frame_2048_16bit():
    img = _raw(2048, 2048, 2048, 16)
    for pattern in ("rggb", "gbrg"):
        np.testing.assert_array_equal(_gpu(img, 2048, pattern, 16), _ref(img, 2048, pattern, 16))


def test_large_frame_sampled_rows():
    # 8192 x 16384 (256 MB in, larger than L2): row bands checked against the oracle on a crop that
    # keeps at least one extra row above and below (the crop's own border rows are not compared) and
    # starts on an even row, so the crop has the frame's CFA phase
    h, w, bits = 8192, 16384, 12
    img = synth.raster(77, 1, h, w, bits)[0]
    A, G, O = synth.coeffs(77, 0, w)
    raw = torch.from_numpy(img).cuda()
    out = lutc.demosaic(raw, "bggr", bits, A=torch.from_numpy(A).cuda(), G=torch.from_numpy(G).cuda(),
                        O=torch.from_numpy(O).cuda())
    torch.cuda.synchronize()
    lut = oracle.lutgen(A, G, O, bits)
    for y0 in (0, 31, 32, 4095, 8190):
        a, b = max(0, (y0 - 1) // 2 * 2), min(h, y0 + 4)
        ref = oracle.demosaic(np.ascontiguousarray(img[a:b]), "bggr", lut=lut, bits=bits)
        lo = y0 - a if a > 0 else 0
        hi = (b - a) - (1 if b < h else 0)
        np.testing.assert_array_equal(out[:, a + lo:a + hi].cpu().numpy(), ref[:, lo:hi])


def test_arguments_are_checked():
    lib = _lib.lib()
    img = torch.zeros((4, 16), dtype=torch.uint16, device="cuda")
    out = torch.zeros((3, 4, 16), dtype=torch.uint16, device="cuda")
    r = lutc.raster_desc(img, 12)
    E = _lib.LUTC_EINVAL
    assert lib.lutc_demosaic(r, None, 4, out.data_ptr(), 32, None) == E
    assert lib.lutc_demosaic(r, None, 0, out.data_ptr(), 30, None) == E
    assert lib.lutc_demosaic(r, None, 0, None, 32, None) == E
    two = lutc.raster_desc(torch.zeros((2, 4, 16), dtype=torch.uint16, device="cuda"), 12)
    assert lib.lutc_demosaic(two, None, 0, out.data_ptr(), 32, None) == E
    assert lib.lutc_demosaic(r, None, 0, out.data_ptr(), 32, None) == 0
    torch.cuda.synchronize()


def test_task_interface_matches_direct_call():
    import ctypes
    h, w, bits = 40, 200, 12
    img = _raw(5, h, w, bits)
    A, G, O = synth.coeffs(5, 0, w)
    d = [torch.from_numpy(a).cuda() for a in (img, A, G, O)]
    out = torch.zeros((3, h, w), dtype=torch.uint16, device="cuda")
    lutc.submit(_lib.LUTC_TASK_DEMOSAIC, "width=%d,height=%d,bits=%d,pattern=gbrg" % (w, h, bits), d, [out])
    ref = lutc.demosaic(d[0], "gbrg", bits, A=d[1], G=d[2], O=d[3])
    assert torch.equal(out, ref)
    lib = _lib.lib()
    ins = (ctypes.c_void_p * 1)(d[0].data_ptr())
    outs = (ctypes.c_void_p * 1)(out.data_ptr())
    assert lib.lutc_submit(_lib.LUTC_TASK_DEMOSAIC, b"width=200,height=40,bits=12,pattern=xyzw", ins, 1, outs, 1,
                           None, 0, None) == _lib.LUTC_EINVAL
