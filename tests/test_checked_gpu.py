"""The bounds-checking build of the library (GPU).

compute-sanitizer is not available, so the library has a debug variant
(``-DLUTC_CHECKED``, loaded under ``LUTC_CHECKED=1``): its TMA-fed kernels check
every shared-memory tile offset, histogram bin, stretch-table index and output
row/column against the job's extents and record ``LUTC_EINVAL`` in the device
status word instead of making the access.  A child process runs the fused
correction (single images, detector-only, a mixed batch) and the TMA-fed
demosaic on ragged shapes through that build: every output must equal the
oracle and the status word must stay 0.
"""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import ctypes
    import numpy as np
    import torch
    import oracle
    import synth
    import paper_1505_05655_gb300 as lutc
    from paper_1505_05655_gb300 import _build, _lib

    assert _lib.checked()
    lib = _lib.lib()
    assert lib._name == _build.CHECKED_LIB, lib._name
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    checked = 0

    # fused correction through the TMA path: 16-byte aligned rows, ragged tiles, three bit depths
    for bands, h, w, bits in ((3, 130, 1032, 12), (2, 77, 2056, 10), (1, 301, 520, 14)):
        raw = synth.raster(h + w, bands, h, w, bits, sat_frac=0.001)
        A, G, O = synth.coeff_set(h + w, bands, w)
        for stretch in (True, False):
            out = lutc.correct_image(d(raw), d(A), d(G), d(O), bits, stretch=stretch)
            ref = oracle.correct_image(raw, A, G, O, bits, stretch=stretch)
            np.testing.assert_array_equal(out.cpu().numpy(), ref)
            checked += 1

    # a mixed batch through the batched TMA kernels
    ims = synth.batch_images(synth.BATCH_SEED + 11, n=12)
    images = []
    for im in ims:
        raw = d(im["raw"])[:, :, :im["width"]]
        images.append((raw, d(im["A"]), d(im["G"]), d(im["O"]), im["bits"], None, True))
    outs = lutc.batch_correct(images)
    for im, out in zip(ims[:6], outs):
        ref = oracle.correct_image(np.ascontiguousarray(im["raw"][:, :, :im["width"]]), im["A"], im["G"], im["O"],
                                   im["bits"])
        np.testing.assert_array_equal(out.cpu().numpy(), ref)
        checked += 1

    # the TMA-fed demosaic, raw and with the detector correction
    for h, w in ((67, 304), (35, 144), (300, 1160)):
        img = synth.raster(7 + h, 1, h, w, 12)[0]
        A, G, O = synth.coeffs(7 + h, 0, w)
        out = lutc.demosaic(d(img), "gbrg", 12)
        np.testing.assert_array_equal(out.cpu().numpy(), oracle.demosaic(img, "gbrg", bits=12))
        out = lutc.demosaic(d(img), "rggb", 12, A=d(A), G=d(G), O=d(O))
        ref = oracle.demosaic(img, "rggb", lut=oracle.lutgen(A, G, O, 12), bits=12)
        np.testing.assert_array_equal(out.cpu().numpy(), ref)
        checked += 2

    torch.cuda.synchronize()
    status = ctypes.c_int(-1)
    assert lib.lutc_device_status(ctypes.byref(status), None) == 0
    print("CHECKED", checked, "STATUS", status.value)
""")


def test_checked_build_runs_clean():
    env = dict(os.environ, LUTC_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1500)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "STATUS 0" in r.stdout, r.stdout[-2000:]
