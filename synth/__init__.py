"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

The module draws raw uint16 detector scenes and per-column Q16 coefficient
triples (see ``synth.c`` for the recipe) and defines the named workloads the
tests and the benchmark use.  It performs none of the correction arithmetic.

The C source is compiled on first use with the host ``gcc`` into
``synth/_build/libsynth.so`` (or explicitly with :func:`build`).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "_build", "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into a shared library (host gcc, no GPU needed)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-pthread",
                        _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, i32, f64, p = ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        lib.synth_hash.argtypes = [u64, u64, u64]
        lib.synth_hash.restype = u64
        lib.synth_u01.argtypes = [u64, u64, u64]
        lib.synth_u01.restype = f64
        lib.synth_scene.argtypes = [u64, i32, i32, i32, i32, f64, f64, p, ctypes.c_int64, i32]
        lib.synth_scene.restype = i32
        lib.synth_coeffs.argtypes = [u64, i32, i32, p, p, p]
        lib.synth_coeffs.restype = None
        lib.synth_batch_spec.argtypes = [u64, i32, p, p, p, p]
        lib.synth_calib.argtypes = [u64, i32, i32, i32, f64, p, ctypes.c_int64, p]
        lib.synth_calib.restype = None
        lib.synth_batch_spec.restype = None
        _lib = lib
    return _lib


def u01(seed: int, stream: int, index: int) -> float:
    return _load().synth_u01(seed, stream, index)


def scene(seed: int, band: int, height: int, width: int, bits: int, *, dead_frac: float = 0.0,
          sat_frac: float = 0.0, out: np.ndarray | None = None, nthreads: int = 0) -> np.ndarray:
    """One band, ``out[y, x]`` uint16 of shape (height, pitch >= width)."""
    if out is None:
        out = np.empty((height, width), dtype=np.uint16)
    assert out.dtype == np.uint16 and out.ndim == 2 and out.shape[0] == height and out.shape[1] >= width
    assert out.strides[1] == 2, "rows must be contiguous"
    pitch = out.strides[0] // 2
    rc = _load().synth_scene(seed, band, width, height, bits, dead_frac, sat_frac,
                             out.ctypes.data, pitch, nthreads)
    if rc != 0:
        raise ValueError("synth_scene rejected its arguments")
    return out


def coeffs(seed: int, band: int, width: int):
    """(A, G, O) int32 arrays of one band's Q16 quadratic, gain and offset."""
    A = np.empty(width, np.int32)
    G = np.empty(width, np.int32)
    O = np.empty(width, np.int32)
    _load().synth_coeffs(seed, band, width, A.ctypes.data, G.ctypes.data, O.ctypes.data)
    return A, G, O


def raster(seed: int, bands: int, height: int, width: int, bits: int, *, dead_frac: float = 0.0,
           sat_frac: float = 0.0, out: np.ndarray | None = None, nthreads: int = 0) -> np.ndarray:
    """Planar band-sequential raster ``[bands, height, width]`` (last axis may be padded)."""
    if out is None:
        out = np.empty((bands, height, width), dtype=np.uint16)
    for b in range(bands):
        scene(seed, b, height, width, bits, dead_frac=dead_frac, sat_frac=sat_frac,
              out=out[b], nthreads=nthreads)
    return out


def coeff_set(seed: int, bands: int, width: int):
    """Per-band coefficients stacked as three ``[bands, width]`` int32 arrays."""
    A = np.empty((bands, width), np.int32)
    G = np.empty((bands, width), np.int32)
    O = np.empty((bands, width), np.int32)
    for b in range(bands):
        A[b], G[b], O[b] = coeffs(seed, b, width)
    return A, G, O


def batch_spec(seed: int, n: int):
    """Image specifications ``(width, height, bits, bands)`` of an n-image batch."""
    w = np.empty(n, np.int32)
    h = np.empty(n, np.int32)
    b = np.empty(n, np.int32)
    nb = np.empty(n, np.int32)
    _load().synth_batch_spec(seed, n, w.ctypes.data, h.ctypes.data, b.ctypes.data, nb.ctypes.data)
    return w, h, b, nb


@dataclass(frozen=True)
class Workload:
    """A named synthetic workload: planar uint16 scene, its bit depth and seed."""
    name: str
    bands: int
    height: int
    width: int
    bits: int
    seed: int
    stretch: bool
    dead_frac: float = 0.0
    sat_frac: float = 0.0

    @property
    def pixels(self) -> int:
        return self.bands * self.height * self.width


#: The single-scene workloads.  ``tiny``: detector correction only, uint16 out.
#: ``scene``: full pipeline on a 4-band 12000 x 12000 12-bit scene.
#: ``large14``: full pipeline on a 3-band 24000 x 24000 14-bit scene with dead
#: columns and saturated pixels.
WORKLOADS = {
    "tiny": Workload("tiny", 1, 1024, 1024, 12, 1505, False),
    "scene": Workload("scene", 4, 12000, 12000, 12, 1506, True),
    "large14": Workload("large14", 3, 24000, 24000, 14, 1507, True, dead_frac=0.01, sat_frac=0.001),
}

#: batch of 256 mixed images, and the serving mixture (64 sensors)
BATCH_SEED = 1508
BATCH_IMAGES = 256
SERVE_SEED = 1509
SERVE_SENSORS = 64


def batch_image_seed(seed: int, i: int) -> int:
    """Seed of image i of a batch (each image draws its own scene and coefficients)."""
    return seed * 1000003 + 7919 * (i + 1)


def batch_images(seed: int = BATCH_SEED, n: int = BATCH_IMAGES, nthreads: int = 0, pitch_multiple: int = 8):
    """The mixed batch: a list of dicts with raw ``[bands, H, pitch]`` uint16 (rows padded to a
    multiple of ``pitch_multiple`` elements; the image is ``raw[:, :, :width]``), A, G, O
    ``[bands, width]`` and the image's width, height, bits, bands."""
    w, h, b, nb = batch_spec(seed, n)
    out = []
    for i in range(n):
        W, H, bits, bands = int(w[i]), int(h[i]), int(b[i]), int(nb[i])
        pitch = -(-W // pitch_multiple) * pitch_multiple
        s = batch_image_seed(seed, i)
        raw = np.zeros((bands, H, pitch), np.uint16)
        raster(s, bands, H, W, bits, out=raw[:, :, :W], nthreads=nthreads)
        A, G, O = coeff_set(s, bands, W)
        out.append(dict(raw=raw, A=A, G=G, O=O, width=W, height=H, bits=bits, bands=bands))
    return out


CALIB_SEED = 1510


def calib(seed: int, n: int, width: int, bits: int, *, dead_frac: float = 0.0):
    """Flat-field calibration scan lines: ``(x [n, width] uint16, y [n] float64 levels)``."""
    x = np.empty((n, width), np.uint16)
    y = np.empty(n, np.float64)
    _load().synth_calib(seed, n, width, bits, dead_frac, x.ctypes.data, width, y.ctypes.data)
    return x, y
