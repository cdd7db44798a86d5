"""Batched correction (lutc_batch_*) against the oracle and against one call per image (GPU).

A batch must give, for every image, exactly what lutc_correct_image gives for
that image alone, which must equal the oracle: integer arithmetic, tolerance
zero.  The mixes below cover images the persistent TMA kernels take (aligned
rows, width >= 256, up to 15 bits) and images they hand to the one-by-one
path (unaligned rows, narrow, 16-bit, empty), stretch and detector-only
images, graph capture and replay, the autotuner and the one-shot call.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

import paper_1505_05655_gb300 as lutc  # noqa: E402


def _image(seed, bands, h, w, bits, pad=None, stretch=True):
    pitch = w if pad is None else w + pad
    raw = np.zeros((bands, h, pitch), np.uint16)
    if h * w:
        synth.raster(seed, bands, h, w, bits, out=raw[:, :, :w], sat_frac=0.001)
    A, G, O = synth.coeff_set(seed, bands, w)
    return dict(raw=raw, A=A, G=G, O=O, width=w, height=h, bits=bits, bands=bands, stretch=stretch)


def _device(im):
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    raw = torch.from_numpy(im["raw"]).cuda()[:, :, :im["width"]]
    out = torch.empty((im["bands"], im["height"], im["width"]), dtype=torch.uint8 if im["stretch"] else torch.uint16,
                      device="cuda")
    return (raw, d(im["A"]), d(im["G"]), d(im["O"]), im["bits"], out, im["stretch"])


def _oracle(im):
    raw = im["raw"][:, :, :im["width"]]
    if im["stretch"]:
        return oracle.correct_image(raw, im["A"], im["G"], im["O"], im["bits"], stretch=True, with_tables=True)
    return oracle.correct_image(raw, im["A"], im["G"], im["O"], im["bits"], stretch=False), None


MIX = [
    (1, 300, 700, 12, 4, True),        # rows padded to a 16-byte multiple
    (3, 97, 2500, 10, 4, True),
    (4, 64, 517, 14, 3, True),        # pitch padded to a 16-byte multiple
    (1, 1000, 256, 12, None, True),
    (3, 33, 4100, 14, 4, True),
    (2, 120, 999, 12, 2, True),       # rows not 16-byte aligned: one-by-one path
    (1, 50, 100, 12, None, True),     # narrower than one TMA box: one-by-one path
    (1, 80, 600, 16, None, True),     # 16-bit: one-by-one path
    (2, 70, 1300, 12, 4, False),      # detector only, uint16 out
    (1, 0, 640, 12, None, True),      # empty
    (3, 211, 1234, 10, 6, True),
    (1, 7, 8192, 12, None, True),
]


@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("column_threads", [0, 64, 256])
def test_mixed_batch_matches_oracle(use_graph, column_threads):
    ims = [_image(100 + i, b, h, w, bits, pad, st) for i, (b, h, w, bits, pad, st) in enumerate(MIX)]
    dev = [_device(im) for im in ims]
    batch = lutc.Batch(dev, column_threads=column_threads, use_graph=use_graph)
    for rep in range(2):  # the second run replays the graph (or relaunches) over the same buffers
        for t in batch.outputs():
            t.view(torch.uint8).zero_()
        batch.run()
        torch.cuda.synchronize()
        for i, im in enumerate(ims):
            ref, tables = _oracle(im)
            np.testing.assert_array_equal(batch.outputs()[i].cpu().numpy(), ref, err_msg="image %d" % i)
            if im["stretch"] and im["height"] * im["width"]:
                h, S, lohi = batch.tables(i, im["bands"], im["bits"])
                np.testing.assert_array_equal(h, tables[0], err_msg="hist of image %d" % i)
                np.testing.assert_array_equal(lohi, tables[2], err_msg="lo/hi of image %d" % i)
                np.testing.assert_array_equal(S, tables[1], err_msg="S of image %d" % i)
    batch.close()


def test_autotuner_picks_a_valid_configuration():
    ims = [_image(300 + i, b, h, w, bits, pad, st) for i, (b, h, w, bits, pad, st) in enumerate(MIX[:5])]
    dev = [_device(im) for im in ims]
    cfg, ms = lutc.batch_autotune(dev, reps=2)
    assert cfg.column_threads in (64, 128, 256) and cfg.use_graph == 1 and ms > 0
    batch = lutc.Batch(dev, config=cfg)
    batch.run()
    torch.cuda.synchronize()
    for i, im in enumerate(ims):
        np.testing.assert_array_equal(batch.outputs()[i].cpu().numpy(), _oracle(im)[0])
    batch.close()


@pytest.mark.parametrize("tuned", [False, True])
def test_one_shot_batch_correct(tuned):
    # lutc_batch_correct: plan, one run, release; with the automatic and with an autotuned configuration
    ims = [_image(500 + i, b, h, w, bits, pad, st) for i, (b, h, w, bits, pad, st) in enumerate(MIX)]
    dev = [_device(im) for im in ims]
    cfg = lutc.batch_autotune(dev, reps=1)[0] if tuned else None
    for t in (d[5] for d in dev):
        t.view(torch.uint8).fill_(0xA5)
    outs = lutc.batch_correct(dev, config=cfg)
    torch.cuda.synchronize()
    for i, im in enumerate(ims):
        np.testing.assert_array_equal(outs[i].cpu().numpy(), _oracle(im)[0], err_msg="image %d" % i)


def test_full_batch_workload_equals_per_image_calls_and_the_oracle():
    """The 256-image mixed workload: every image equals its own single call and the oracle, and every
    stretch image's histogram, lo/hi and S (lutc_batch_tables) equal the oracle's."""
    import concurrent.futures as cf
    import os
    ims = synth.batch_images()
    for im in ims:
        im["stretch"] = True
    dev = [_device(im) for im in ims]
    batch = lutc.Batch(dev)
    batch.run()
    torch.cuda.synchronize()
    for i, (raw, A, G, O, bits, out, stretch) in enumerate(dev):
        single = lutc.correct_image(raw, A, G, O, bits)
        assert torch.equal(single, out), "image %d differs from its single call" % i
    torch.cuda.synchronize()
    got = [(d[5].cpu().numpy(), batch.tables(i, ims[i]["bands"], ims[i]["bits"])) for i, d in enumerate(dev)]
    batch.close()
    # the oracle on every image, spread over the host's cores (ctypes releases the GIL in the oracle)
    threads = max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1))

    def differs(i):  # compared in the worker, so that only `threads` oracle results are alive at once
        ref, tables = _oracle(ims[i])
        out, (h, S, lohi) = got[i]
        bad = [name for name, a, b in (("image", out, ref), ("hist", h, tables[0]), ("lo/hi", lohi, tables[2]),
                                       ("S", S, tables[1])) if not np.array_equal(a, b)]
        return "%s of image %d (%d-bit)" % ("/".join(bad), i, ims[i]["bits"]) if bad else None

    with cf.ThreadPoolExecutor(threads) as ex:
        bad = [m for m in ex.map(differs, range(len(ims))) if m]
    assert not bad, "differ from the oracle: " + "; ".join(bad[:10])
