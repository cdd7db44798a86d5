"""lutc_correct_image_static: the correction for callers that cannot allocate (GPU).

Some callers of this library cannot allocate device memory -- a plain C
client with no device allocator of its own, a loop where an allocation would
stall the device, a framework that owns every device allocation -- so they
cannot provide the scratch workspace lutc_correct_image wants.
lutc_correct_image_static takes that scratch from a fixed device array
inside the library instead.  These tests call it through the C ABI and check:

  * on two calls in a row (two different rasters, so the second call cannot
    pass by reusing the first call's tables) its output equals the output of
    lutc_correct_image with a caller-provided workspace and the oracle's; the
    method is integer arithmetic, so the tolerance is zero;
  * the detector-only mode (no scratch used) on the same rasters;
  * tables of the large 14-bit configuration (3 bands of 16384 bins) and the
    largest table set that fits the 1 MiB array (7 bands at 14 bits);
  * the limit: one band more is LUTC_ENOMEM, and a malformed call on an
    oversized raster is still LUTC_EINVAL.

That calls overlapping on the GPU race on the shared array is documented in
the header, not tested here.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

import paper_1505_05655_gb300 as lutc  # noqa: E402
from paper_1505_05655_gb300 import _lib  # noqa: E402


def _case(seed, bands, h, w, bits, **kw):
    raw = synth.raster(seed, bands, h, w, bits, **kw)
    A, G, O = synth.coeff_set(seed, bands, w)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return (raw, A, G, O), (d(raw), d(A), d(G), d(O))


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _with_workspace(raw, A, G, O, bits, flags):
    lib = _lib.lib()
    desc = lutc.raster_desc(raw, bits)
    cd = lutc.coeff_descs(A, G, O)
    out = torch.empty(raw.shape, dtype=torch.uint8 if flags else torch.uint16, device="cuda")
    ws = torch.empty(max(256, lib.lutc_correct_image_workspace(ctypes.byref(desc))), dtype=torch.uint8, device="cuda")
    rc = lib.lutc_correct_image(ctypes.byref(desc), cd, flags, ctypes.c_void_p(out.data_ptr()),
                                out.stride(1) * out.element_size(), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                _stream())
    assert rc == 0, rc
    return out


def _static(raw, A, G, O, bits, flags):
    lib = _lib.lib()
    desc = lutc.raster_desc(raw, bits)
    cd = lutc.coeff_descs(A, G, O)
    out = torch.empty(raw.shape, dtype=torch.uint8 if flags else torch.uint16, device="cuda")
    out.view(torch.uint8).fill_(0xA5)  # a stale value must not survive
    rc = lib.lutc_correct_image_static(ctypes.byref(desc), cd, flags, ctypes.c_void_p(out.data_ptr()),
                                       out.stride(1) * out.element_size(), _stream())
    assert rc == 0, rc
    return out


def _check(host, dev, bits, flags):
    got = _static(*dev, bits, flags)
    ref = _with_workspace(*dev, bits, flags)
    torch.cuda.synchronize()
    got, ref = got.cpu().numpy(), ref.cpu().numpy()
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(got, oracle.correct_image(*host, bits, stretch=bool(flags)))


@pytest.mark.parametrize("flags", [_lib.LUTC_STRETCH, 0])
def test_static_scratch_matches_workspace_entry_point_and_oracle(flags):
    # two calls in a row on different rasters: a 12-bit one taking the TMA-fed kernels (aligned rows)
    # and a 14-bit one of odd width taking the strip kernels; the second call's tables must not
    # depend on what the first left in the array
    cases = [(_case(4242, 3, 333, 2104, 12), 12), (_case(4343, 2, 257, 3001, 14, sat_frac=0.001), 14)]
    for (host, dev), bits in cases:
        _check(host, dev, bits, flags)


def test_static_scratch_holds_the_large_14_bit_tables():
    # the large 14-bit configuration's table set (3 bands x 16384 bins, dead columns and saturated
    # pixels), then the largest set the array holds (7 bands at 14 bits), then the first again
    big = _case(4444, 3, 160, 2048, 14, dead_frac=0.01, sat_frac=0.001)
    full = _case(4545, 7, 64, 512, 14)
    desc = lutc.raster_desc(full[1][0], 14)
    assert _lib.lib().lutc_correct_image_workspace(ctypes.byref(desc)) <= _lib.LUTC_STATIC_SCRATCH_BYTES
    for host, dev in (big, full, big):
        _check(host, dev, 14, _lib.LUTC_STRETCH)


def test_static_scratch_rejects_oversized_tables():
    lib = _lib.lib()
    for bands, bits in ((8, 14), (2, 16), (4, 15)):
        raw = torch.zeros((bands, 8, 256), dtype=torch.uint16, device="cuda")
        A = torch.zeros((bands, 256), dtype=torch.int32, device="cuda")
        desc = lutc.raster_desc(raw, bits)
        assert lib.lutc_correct_image_workspace(ctypes.byref(desc)) > _lib.LUTC_STATIC_SCRATCH_BYTES
        out = torch.zeros(raw.shape, dtype=torch.uint8, device="cuda")
        cd = lutc.coeff_descs(A, A, A)
        call = lambda flags, o=out: lib.lutc_correct_image_static(ctypes.byref(desc), cd, flags,
                                                                  ctypes.c_void_p(o.data_ptr()), 256, _stream())
        assert call(_lib.LUTC_STRETCH) == _lib.LUTC_ENOMEM
        # malformed calls are refused as malformed first, whatever the size
        assert call(_lib.LUTC_STRETCH | 0x100) == _lib.LUTC_EINVAL
        assert lib.lutc_correct_image_static(ctypes.byref(desc), None, _lib.LUTC_STRETCH,
                                             ctypes.c_void_p(out.data_ptr()), 256, _stream()) == _lib.LUTC_EINVAL
        assert lib.lutc_correct_image_static(ctypes.byref(desc), cd, _lib.LUTC_STRETCH, None, 256,
                                             _stream()) == _lib.LUTC_EINVAL
        torch.cuda.synchronize()
        assert int(out.sum()) == 0  # nothing was written
