"""The task interface and the GPU-information utility on the GPU (GPU).

Every task submitted through ``lutc_submit`` must give, byte for byte, what
the direct entry point gives on the same buffers, and the fused task what
the oracle gives.  The device listing must agree with what the runtime
reports for the same device.
"""
import ctypes
import xml.etree.ElementTree as ET

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

import paper_1505_05655_gb300 as lutc  # noqa: E402
from paper_1505_05655_gb300 import _lib  # noqa: E402

BANDS, H, W, BITS = 3, 300, 1000, 12


@pytest.fixture(scope="module")
def data():
    A, G, O = synth.coeff_set(7100, BANDS, W)
    raw = synth.raster(7101, BANDS, H, W, BITS, sat_frac=0.001)
    d = dict(raw=raw, A=A, G=G, O=O)
    d.update({k + "_d": torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in d.items()})
    return d


def _params(**kw):
    return ",".join(f"{k}={v}" for k, v in kw.items())


def test_lutgen_task(data):
    for b in range(BANDS):
        lut = torch.empty((W, 1 << BITS), dtype=torch.uint16, device="cuda")
        lutc.submit(_lib.LUTC_TASK_LUTGEN, _params(width=W, bits=BITS),
                    [data["A_d"][b], data["G_d"][b], data["O_d"][b]], [lut])
        ref = lutc.lutgen(data["A_d"][b], data["G_d"][b], data["O_d"][b], BITS)
        assert torch.equal(lut, ref)


def test_hist_stretch_compose_apply_tasks(data):
    p = _params(width=W, height=H, bands=BANDS, bits=BITS)
    h = torch.empty((BANDS, 1 << BITS), dtype=torch.uint64, device="cuda")
    lutc.submit(_lib.LUTC_TASK_HIST, p, [data["raw_d"], data["A_d"], data["G_d"], data["O_d"]], [h])
    assert torch.equal(h, lutc.hist(data["raw_d"], data["A_d"], data["G_d"], data["O_d"], BITS))
    S = torch.empty((BANDS, 1 << BITS), dtype=torch.uint8, device="cuda")
    lohi = torch.empty((BANDS, 2), dtype=torch.int32, device="cuda")
    lutc.submit(_lib.LUTC_TASK_STRETCH, _params(bands=BANDS, bits=BITS), [h], [S, lohi])
    S_ref, lohi_ref = lutc.stretch(h, BITS)
    assert torch.equal(S, S_ref) and torch.equal(lohi, lohi_ref)
    luts = torch.stack([lutc.lutgen(data["A_d"][b], data["G_d"][b], data["O_d"][b], BITS) for b in range(BANDS)])
    cluts = torch.empty((BANDS, W, 1 << BITS), dtype=torch.uint8, device="cuda")
    for b in range(BANDS):
        lutc.submit(_lib.LUTC_TASK_COMPOSE, _params(width=W, bits=BITS), [luts[b], S[b]], [cluts[b]])
        assert torch.equal(cluts[b], lutc.compose(luts[b], S[b], BITS))
    o16 = torch.empty((BANDS, H, W), dtype=torch.uint16, device="cuda")
    lutc.submit(_lib.LUTC_TASK_APPLY, p + ",table=u16", [data["raw_d"], luts], [o16])
    assert torch.equal(o16, lutc.apply_u16(data["raw_d"], luts, BITS))
    o8 = torch.empty((BANDS, H, W), dtype=torch.uint8, device="cuda")
    lutc.submit(_lib.LUTC_TASK_APPLY, p + ",table=u8", [data["raw_d"], cluts], [o8])
    assert torch.equal(o8, lutc.apply_u8(data["raw_d"], cluts, BITS))
    np.testing.assert_array_equal(o8.cpu().numpy(), oracle.correct_image(data["raw"], data["A"], data["G"],
                                                                          data["O"], BITS))


@pytest.mark.parametrize("stretch", [1, 0])
def test_correct_image_task(data, stretch):
    p = _params(width=W, height=H, bands=BANDS, bits=BITS, stretch=stretch)
    out = torch.empty((BANDS, H, W), dtype=torch.uint8 if stretch else torch.uint16, device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    lutc.submit(_lib.LUTC_TASK_CORRECT_IMAGE, p, [data["raw_d"], data["A_d"], data["G_d"], data["O_d"]], [out], ws)
    ref = lutc.correct_image(data["raw_d"], data["A_d"], data["G_d"], data["O_d"], BITS, stretch=bool(stretch))
    assert torch.equal(out, ref)
    if stretch:
        np.testing.assert_array_equal(out.cpu().numpy(), oracle.correct_image(data["raw"], data["A"], data["G"],
                                                                               data["O"], BITS))
    # a workspace too small is refused, nothing launched
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    if stretch:
        with pytest.raises(lutc.LutcError):
            lutc.submit(_lib.LUTC_TASK_CORRECT_IMAGE, p, [data["raw_d"], data["A_d"], data["G_d"], data["O_d"]],
                        [out], small)


def test_device_info_lists_this_gpu():
    root = ET.fromstring(lutc.device_info())
    assert int(root.get("count")) == torch.cuda.device_count() >= 1
    g = root.findall("gpu")[0]
    prop = torch.cuda.get_device_properties(0)
    assert g.find("name").text == prop.name
    assert g.find("compute_capability").text == f"{prop.major}.{prop.minor}"
    assert int(g.find("multiprocessor_count").text) == prop.multi_processor_count
    assert int(g.find("total_global_memory").text) == prop.total_memory
    assert int(g.find("warp_size").text) == 32
    # the same document through the task interface, into a host buffer
    buf = ctypes.create_string_buffer(1 << 16)
    outs = (ctypes.c_void_p * 1)(ctypes.addressof(buf))
    rc = _lib.lib().lutc_submit(_lib.LUTC_TASK_DEVICE_INFO, b"capacity=65536", None, 0, outs, 1, None, 0, None)
    assert rc == 0 and buf.value.decode() == lutc.device_info()
