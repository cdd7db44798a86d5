"""The fused correction of rasters in host memory (GPU).

lutc_correct_image_host pipelines the copies in, both passes and the copies
out in chunks of rows.  Whatever the chunking, the result must equal the
device-resident call and the oracle byte for byte (tolerance zero).
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

import paper_1505_05655_gb300 as lutc  # noqa: E402
from paper_1505_05655_gb300 import _lib  # noqa: E402


def _coeffs(seed, bands, w):
    A, G, O = synth.coeff_set(seed, bands, w)
    return A, G, O, [torch.from_numpy(a).cuda() for a in (A, G, O)]


@pytest.mark.parametrize("bands,h,w,bits,pad", [(3, 700, 1300, 12, 0), (1, 9000, 6000, 12, 0), (2, 333, 517, 14, 3),
                                                 (4, 64, 256, 10, 8), (1, 1, 1, 12, 0), (2, 5000, 5000, 12, 1),
                                                 (2, 300, 700, 16, 0), (1, 1, 20000, 12, 0), (3, 2049, 8, 8, 5)])
def test_pinned_host_raster(bands, h, w, bits, pad):
    raw = torch.zeros((bands, h, w + pad), dtype=torch.uint16).pin_memory()
    raw[:, :, :w] = torch.from_numpy(synth.raster(3 + bits, bands, h, w, bits, sat_frac=0.001))
    A, G, O, d = _coeffs(3 + bits, bands, w)
    view = raw[:, :, :w]
    out = lutc.correct_image_host(view, *d, bits)
    torch.cuda.synchronize()
    ref_dev = lutc.correct_image(view.cuda(), *d, bits).cpu()
    assert torch.equal(out, ref_dev)
    if bands * h * w <= 4_000_000:
        np.testing.assert_array_equal(out.numpy(), oracle.correct_image(np.ascontiguousarray(view.numpy()), A, G, O,
                                                                        bits))


def test_detector_only_and_pageable_memory():
    bands, h, w, bits = 2, 1200, 2048, 12
    raw = torch.from_numpy(synth.raster(8, bands, h, w, bits))  # pageable
    A, G, O, d = _coeffs(8, bands, w)
    out = lutc.correct_image_host(raw, *d, bits, stretch=False)
    torch.cuda.synchronize()
    assert out.dtype == torch.uint16
    assert torch.equal(out, lutc.correct_image(raw.cuda(), *d, bits, stretch=False).cpu())
    out8 = lutc.correct_image_host(raw, *d, bits)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out8.numpy(), oracle.correct_image(raw.numpy(), A, G, O, bits))


def test_back_to_back_calls_on_one_stream_reuse_the_workspace():
    bands, h, w, bits = 2, 3000, 4000, 12
    A, G, O, d = _coeffs(9, bands, w)
    raws = [torch.from_numpy(synth.raster(20 + k, bands, h, w, bits)).pin_memory() for k in range(3)]
    r0 = lutc.raster_desc(raws[0].cuda(), bits)
    ws = torch.empty(_lib.lib().lutc_correct_image_host_workspace(r0, 1), dtype=torch.uint8, device="cuda")
    outs = [lutc.correct_image_host(r, *d, bits, workspace=ws) for r in raws]
    torch.cuda.synchronize()
    for r, o in zip(raws, outs):
        assert torch.equal(o, lutc.correct_image(r.cuda(), *d, bits).cpu())


def test_small_workspace_is_refused():
    raw = torch.zeros((1, 100, 300), dtype=torch.uint16)
    A, G, O, d = _coeffs(1, 1, 300)
    with pytest.raises(lutc.LutcError) as e:
        lutc.correct_image_host(raw, *d, 12, workspace=torch.empty(1024, dtype=torch.uint8, device="cuda"))
    assert e.value.status == _lib.LUTC_ENOMEM


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_frame_sequences_equal_single_calls(n):
    bands, h, w, bits = 2, 1100, 3000, 12
    A, G, O, d = _coeffs(17, bands, w)
    frames = [torch.from_numpy(synth.raster(30 + k, bands, h, w, bits)).pin_memory() for k in range(n)]
    outs = lutc.correct_frames_host(frames, *d, bits)
    torch.cuda.synchronize()
    for f, o in zip(frames, outs):
        assert torch.equal(o, lutc.correct_image(f.cuda(), *d, bits).cpu())
    # detector only, padded rows (strided copies), frames from pageable memory
    frames = [torch.zeros((bands, h, w + 5), dtype=torch.uint16)[:, :, :w] for _ in range(n)]
    for k, f in enumerate(frames):
        f.copy_(torch.from_numpy(synth.raster(40 + k, bands, h, w, bits)))
    outs = lutc.correct_frames_host(frames, *d, bits, stretch=False)
    torch.cuda.synchronize()
    for f, o in zip(frames, outs):
        assert torch.equal(o, lutc.correct_image(f.contiguous().cuda(), *d, bits, stretch=False).cpu())
