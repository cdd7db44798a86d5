"""lutc_correct_image_static: the correction for callers that cannot allocate (GPU).

Some callers of this library cannot allocate device memory -- a plain C
client with no device allocator of its own, a loop where an allocation would
stall the device, a framework that owns every device allocation -- so they
cannot provide the scratch workspace lutc_correct_image wants.
lutc_correct_image_static takes that scratch from a fixed device array
inside the library instead.  This test calls it through the C ABI and checks
that, on two calls in a row (on two different rasters, so the second call
cannot pass by reusing the first call's tables), its output is identical to
the output of lutc_correct_image with a caller-provided workspace; the
method is integer arithmetic, so the tolerance is zero.  It also checks the
size limit is enforced.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

import paper_1505_05655_gb300 as lutc  # noqa: E402
from paper_1505_05655_gb300 import _lib  # noqa: E402


def _case(seed, bands, h, w, bits):
    raw = torch.from_numpy(synth.raster(seed, bands, h, w, bits)).cuda()
    A, G, O = (torch.from_numpy(a).cuda() for a in synth.coeff_set(seed, bands, w))
    return raw, A, G, O


def _with_workspace(raw, A, G, O, bits):
    lib = _lib.lib()
    desc = lutc.raster_desc(raw, bits)
    cd = lutc.coeff_descs(A, G, O)
    out = torch.empty(raw.shape, dtype=torch.uint8, device="cuda")
    ws = torch.empty(lib.lutc_correct_image_workspace(ctypes.byref(desc)), dtype=torch.uint8, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.lutc_correct_image(ctypes.byref(desc), cd, _lib.LUTC_STRETCH, ctypes.c_void_p(out.data_ptr()),
                                out.stride(1), ctypes.c_void_p(ws.data_ptr()), ws.numel(), st)
    assert rc == 0, rc
    return out


def _static(raw, A, G, O, bits):
    lib = _lib.lib()
    desc = lutc.raster_desc(raw, bits)
    cd = lutc.coeff_descs(A, G, O)
    out = torch.empty(raw.shape, dtype=torch.uint8, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.lutc_correct_image_static(ctypes.byref(desc), cd, _lib.LUTC_STRETCH, ctypes.c_void_p(out.data_ptr()),
                                       out.stride(1), st)
    assert rc == 0, rc
    return out


def test_static_scratch_matches_workspace_entry_point():
    cases = [_case(4242, 3, 333, 2100, 12), _case(4343, 2, 257, 3001, 14)]
    for raw, A, G, O, bits in ((*cases[0], 12), (*cases[1], 14)):
        ref = _with_workspace(raw, A, G, O, bits)
        got = _static(raw, A, G, O, bits)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())


def test_static_scratch_rejects_oversized_tables():
    lib = _lib.lib()
    raw = torch.zeros((4, 8, 64), dtype=torch.uint16, device="cuda")
    A = torch.zeros((4, 64), dtype=torch.int32, device="cuda")
    desc = lutc.raster_desc(raw, 16)  # 4 bands x 65536 bins: tables larger than the fixed array
    assert lib.lutc_correct_image_workspace(ctypes.byref(desc)) > (1 << 20)
    out = torch.empty(raw.shape, dtype=torch.uint8, device="cuda")
    rc = lib.lutc_correct_image_static(ctypes.byref(desc), lutc.coeff_descs(A, A, A), _lib.LUTC_STRETCH,
                                       ctypes.c_void_p(out.data_ptr()), 64, None)
    assert rc == _lib.LUTC_ENOMEM
