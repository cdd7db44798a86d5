"""CPU oracle of detector LUT generation, LUT-based image correction, the per-detector fit and demosaicing.

TEST INFRASTRUCTURE ONLY: the plain, slow reference that the CUDA library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm may import it.  It shares no code
with the CUDA path; the definitions it follows are stated in
``lutc_oracle.c`` (steps L, P, H, S, C, A there), ``lsq_oracle.c``
(steps F1-F4 of the least-squares fit) and ``bayer_oracle.c`` (bilinear
demosaicing).

The C sources are compiled with the host ``gcc`` on first use (or by
:func:`build`, :func:`build_lsq` and :func:`build_bayer`) into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lutc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liblutc_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (host gcc, plain -O2, single threaded)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32, i64, p = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        lib.oracle_lut_entry.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, i64, i32]
        lib.oracle_lut_entry.restype = i64
        lib.oracle_lutgen.argtypes = [p, p, p, i32, i32, p]
        lib.oracle_lutgen.restype = None
        lib.oracle_apply_u16.argtypes = [p, i64, i32, i32, i32, p, p, i64]
        lib.oracle_apply_u16.restype = None
        lib.oracle_hist.argtypes = [p, i64, i32, i32, i32, p, p]
        lib.oracle_hist.restype = None
        lib.oracle_stretch.argtypes = [p, i32, p, p]
        lib.oracle_stretch.restype = None
        lib.oracle_compose.argtypes = [p, p, i32, i32, p]
        lib.oracle_compose.restype = None
        lib.oracle_apply_u8.argtypes = [p, i64, i32, i32, i32, p, p, i64]
        lib.oracle_apply_u8.restype = None
        lib.oracle_correct_image.argtypes = [p, i64, i32, i32, i32, i32, p, p, p, i32, p, i64, p, p, p]
        lib.oracle_correct_image.restype = i32
        _lib = lib
    return _lib


def _c(a: np.ndarray, dtype) -> np.ndarray:
    a = np.asarray(a)
    assert a.dtype == dtype, (a.dtype, dtype)
    return a


def _rows(img: np.ndarray):
    """(height, width, pitch in elements) of a 2-D array with contiguous rows."""
    assert img.ndim == 2 and img.strides[1] == img.itemsize
    return img.shape[0], img.shape[1], img.strides[0] // img.itemsize


def lut_entry(A: int, G: int, O: int, x: int, bits: int) -> int:
    """One entry of the detector LUT (step L)."""
    return int(_load().oracle_lut_entry(int(A), int(G), int(O), int(x), int(bits)))


def lutgen(A, G, O, bits: int) -> np.ndarray:
    """Detector LUT ``[ncols, 2^bits]`` uint16 (step L)."""
    A = np.ascontiguousarray(_c(A, np.int32))
    G = np.ascontiguousarray(_c(G, np.int32))
    O = np.ascontiguousarray(_c(O, np.int32))
    n = A.shape[0]
    lut = np.empty((n, 1 << bits), np.uint16)
    _load().oracle_lutgen(A.ctypes.data, G.ctypes.data, O.ctypes.data, n, bits, lut.ctypes.data)
    return lut


def apply_u16(img: np.ndarray, lut: np.ndarray, bits: int) -> np.ndarray:
    """Detector-corrected band (step P)."""
    img = _c(img, np.uint16)
    h, w, pitch = _rows(img)
    lut = np.ascontiguousarray(_c(lut, np.uint16))
    assert lut.shape == (w, 1 << bits)
    out = np.empty((h, w), np.uint16)
    _load().oracle_apply_u16(img.ctypes.data, pitch, w, h, bits, lut.ctypes.data, out.ctypes.data, w)
    return out


def hist(img: np.ndarray, lut: np.ndarray, bits: int) -> np.ndarray:
    """Histogram of corrected DN of one band (step H), 2^bits uint64 bins."""
    img = _c(img, np.uint16)
    h, w, pitch = _rows(img)
    lut = np.ascontiguousarray(_c(lut, np.uint16))
    assert lut.shape == (w, 1 << bits)
    out = np.empty(1 << bits, np.uint64)
    _load().oracle_hist(img.ctypes.data, pitch, w, h, bits, lut.ctypes.data, out.ctypes.data)
    return out


def stretch(hist_: np.ndarray, bits: int):
    """(S uint8[2^bits], lo, hi) of one band's histogram (step S)."""
    hist_ = np.ascontiguousarray(_c(hist_, np.uint64))
    assert hist_.shape == (1 << bits,)
    S = np.empty(1 << bits, np.uint8)
    lohi = np.empty(2, np.int32)
    _load().oracle_stretch(hist_.ctypes.data, bits, S.ctypes.data, lohi.ctypes.data)
    return S, int(lohi[0]), int(lohi[1])


def compose(lut: np.ndarray, S: np.ndarray, bits: int) -> np.ndarray:
    """Composed per-column uint8 LUT (step C)."""
    lut = np.ascontiguousarray(_c(lut, np.uint16))
    S = np.ascontiguousarray(_c(S, np.uint8))
    n = lut.shape[0]
    out = np.empty((n, 1 << bits), np.uint8)
    _load().oracle_compose(lut.ctypes.data, S.ctypes.data, n, bits, out.ctypes.data)
    return out


def apply_u8(img: np.ndarray, clut: np.ndarray, bits: int) -> np.ndarray:
    """uint8 output band through a composed LUT (step A)."""
    img = _c(img, np.uint16)
    h, w, pitch = _rows(img)
    clut = np.ascontiguousarray(_c(clut, np.uint8))
    assert clut.shape == (w, 1 << bits)
    out = np.empty((h, w), np.uint8)
    _load().oracle_apply_u8(img.ctypes.data, pitch, w, h, bits, clut.ctypes.data, out.ctypes.data, w)
    return out


def correct_image(raster: np.ndarray, A, G, O, bits: int, stretch: bool = True, with_tables: bool = False):
    """Whole correction of a planar raster ``[bands, height, width]``.

    Returns the uint8 (stretch) or uint16 (detector only) raster, and with
    ``with_tables`` also ``(hist [bands, 2^bits], S [bands, 2^bits], lohi [bands, 2])``.
    """
    raster = _c(raster, np.uint16)
    assert raster.ndim == 3
    bands, h, w = raster.shape
    if raster.size == 0:
        pitch = max(w, 1)  # nothing is read
    else:
        assert raster.strides[2] == 2
        pitch = raster.strides[1] // 2
        assert bands == 1 or raster.strides[0] == h * raster.strides[1], "bands must be stacked at height * pitch"
    A = np.ascontiguousarray(_c(A, np.int32)).reshape(bands, w)
    G = np.ascontiguousarray(_c(G, np.int32)).reshape(bands, w)
    O = np.ascontiguousarray(_c(O, np.int32)).reshape(bands, w)
    L = 1 << bits
    out = np.empty((bands, h, w), np.uint8 if stretch else np.uint16)
    hist_ = np.zeros((bands, L), np.uint64)
    S = np.zeros((bands, L), np.uint8)
    lohi = np.zeros((bands, 2), np.int32)
    rc = _load().oracle_correct_image(raster.ctypes.data, pitch, w, h, bands, bits,
                                      A.ctypes.data, G.ctypes.data, O.ctypes.data, int(bool(stretch)),
                                      out.ctypes.data, w, hist_.ctypes.data, S.ctypes.data, lohi.ctypes.data)
    if rc != 0:
        raise MemoryError("oracle_correct_image could not allocate its tables")
    if with_tables:
        return out, (hist_, S, lohi)
    return out


# ----------------------------------------------------------------------------- least-squares fit (lsq_oracle.c)

_LSQ_SRC = os.path.join(_HERE, "lsq_oracle.c")
_LSQ_LIB = os.path.join(_HERE, "_build", "liblsq_oracle.so")
_lsq = None


def build_lsq(force: bool = False) -> str:
    """Compile the fit oracle (host gcc, -O2, no fused multiply-add)."""
    if force or not os.path.exists(_LSQ_LIB) or os.path.getmtime(_LSQ_LIB) < os.path.getmtime(_LSQ_SRC):
        os.makedirs(os.path.dirname(_LSQ_LIB), exist_ok=True)
        tmp = _LSQ_LIB + ".%d.tmp" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _LSQ_SRC, "-o", tmp,
                        "-lm"], check=True)
        os.replace(tmp, _LSQ_LIB)
    return _LSQ_LIB


def _load_lsq():
    global _lsq
    if _lsq is None:
        lib = ctypes.CDLL(build_lsq())
        i32, i64, p = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        lib.oracle_polyfit.argtypes = [p, i64, p, i64, i32, i32, i32, p, p, p]
        lib.oracle_polyfit.restype = None
        _lsq = lib
    return _lsq


def polyfit(x, y, order: int, q16: bool = False):
    """Per-column least-squares fit of order 1-3 (steps F1-F4 of lsq_oracle.c).

    x: ``[n, ncols]`` uint16 (contiguous rows); y: ``[n, ncols]`` float64, or ``[n]`` (one target
    per line).  Returns ``(coef [ncols, order+1] float64, status [ncols] int32)`` and, with
    ``q16``, also ``[3, ncols]`` int32 codes (A, G, O).
    """
    x = _c(x, np.uint16)
    y = _c(y, np.float64)
    n, ncols, xp = _rows(x)
    if y.ndim == 1:
        assert y.shape[0] == n and y.strides[0] == 8
        yp = 0
    else:
        assert y.shape == (n, ncols)
        _, _, yp = _rows(y)
    assert 1 <= order <= 3 and not (q16 and order > 2)
    coef = np.empty((ncols, order + 1), np.float64)
    status = np.empty(ncols, np.int32)
    codes = np.empty((3, ncols), np.int32) if q16 else None
    _load_lsq().oracle_polyfit(x.ctypes.data, xp, y.ctypes.data, yp, n, ncols, order, coef.ctypes.data,
                               status.ctypes.data, codes.ctypes.data if q16 else None)
    return (coef, status, codes) if q16 else (coef, status)


# ----------------------------------------------------------------------------- bilinear demosaic (bayer_oracle.c)

_BAYER_SRC = os.path.join(_HERE, "bayer_oracle.c")
_BAYER_LIB = os.path.join(_HERE, "_build", "libbayer_oracle.so")
_bayer = None
PATTERNS = {"rggb": 0, "bggr": 1, "grbg": 2, "gbrg": 3}


def build_bayer(force: bool = False) -> str:
    """Compile the demosaic oracle (host gcc, -O2)."""
    if force or not os.path.exists(_BAYER_LIB) or os.path.getmtime(_BAYER_LIB) < os.path.getmtime(_BAYER_SRC):
        os.makedirs(os.path.dirname(_BAYER_LIB), exist_ok=True)
        tmp = _BAYER_LIB + ".%d.tmp" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _BAYER_SRC, "-o", tmp], check=True)
        os.replace(tmp, _BAYER_LIB)
    return _BAYER_LIB


def _load_bayer():
    global _bayer
    if _bayer is None:
        lib = ctypes.CDLL(build_bayer())
        i32, i64, p = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        lib.oracle_demosaic.argtypes = [p, i64, i32, i32, i32, p, i32, p, i64]
        lib.oracle_demosaic.restype = None
        _bayer = lib
    return _bayer


def demosaic(img: np.ndarray, pattern: str = "rggb", lut: np.ndarray | None = None, bits: int = 16) -> np.ndarray:
    """Bilinear demosaic of one CFA raster (definition in bayer_oracle.c): ``[3, H, W]`` uint16 R, G, B.

    With ``lut`` (``[W, 2^bits]`` uint16, e.g. from :func:`lutgen`) every value is corrected first.
    """
    img = _c(img, np.uint16)
    if img.size == 0:
        return np.zeros((3,) + img.shape, np.uint16)
    h, w, pitch = _rows(img)
    out = np.empty((3, h, w), np.uint16)
    if lut is not None:
        lut = np.ascontiguousarray(_c(lut, np.uint16))
        assert lut.shape == (w, 1 << bits)
    _load_bayer().oracle_demosaic(img.ctypes.data, pitch, w, h, PATTERNS[pattern],
                                  lut.ctypes.data if lut is not None else None, bits, out.ctypes.data, max(w, 1))
    return out
