"""Canary bytes around every output (GPU).

compute-sanitizer is not available, so out-of-bounds writes are caught the
plain way: each output lives inside a larger buffer filled with a canary
pattern (guard regions before and after it, and padding at the end of every
row), the call runs, and every byte outside the exact result region must
still hold the canary.  Shapes are ragged so that partial vectors, partial
tiles and the right and bottom edges are all exercised, on the TMA-fed and
the plain kernels.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

import paper_1505_05655_gb300 as lutc  # noqa: E402

GUARD = 4096  # bytes before and after each output


class Guarded:
    """A [planes, rows, width] output of `dtype` with `pad` extra elements per row, inside guards."""

    def __init__(self, planes, rows, width, dtype, pad, device="cuda", canary=0xA5):
        self.shape = (planes, rows, width)
        self.dtype = dtype
        self.esize = torch.empty((), dtype=dtype).element_size()
        self.pitch = width + pad
        n = planes * rows * self.pitch * self.esize
        self.buf = torch.full((GUARD + n + GUARD,), canary, dtype=torch.uint8, device=device)
        if device != "cuda":
            self.buf = self.buf.pin_memory()
        self.canary = canary
        body = self.buf[GUARD:GUARD + n].view(dtype).view(planes, rows, self.pitch)
        self.view = body[:, :, :width]

    def check(self):
        b = self.buf.cpu().numpy()
        assert (b[:GUARD] == self.canary).all(), "write before the output"
        assert (b[-GUARD:] == self.canary).all(), "write after the output"
        body = b[GUARD:-GUARD].reshape(self.shape[0], self.shape[1], self.pitch * self.esize)
        assert (body[:, :, self.shape[2] * self.esize:] == self.canary).all(), "write into the row padding"


def _data(seed, bands, h, w, bits, pad_in=0):
    raw = np.zeros((bands, h, w + pad_in), np.uint16)
    raw[:, :, :w] = synth.raster(seed, bands, h, w, bits, sat_frac=0.001)
    A, G, O = synth.coeff_set(seed, bands, w)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return d(raw)[:, :, :w], d(A), d(G), d(O)


# (bands, h, w, pad_in, pad_out): aligned rows (TMA) and unaligned (strip kernels), ragged tails
SHAPES = [(2, 77, 1031, 0, 9), (1, 33, 2048, 8, 16), (3, 130, 300, 3, 1), (1, 5, 7, 1, 3)]


@pytest.mark.parametrize("bands,h,w,pad_in,pad_out", SHAPES)
@pytest.mark.parametrize("stretch", [True, False])
def test_correct_image_writes_only_its_output(bands, h, w, pad_in, pad_out, stretch):
    raw, A, G, O = _data(h + w, bands, h, w, 12, pad_in)
    out = Guarded(bands, h, w, torch.uint8 if stretch else torch.uint16, pad_out)
    lutc.correct_image(raw, A, G, O, 12, stretch=stretch, out=out.view)
    torch.cuda.synchronize()
    out.check()
    ref = oracle.correct_image(raw.cpu().numpy(), A.cpu().numpy(), G.cpu().numpy(), O.cpu().numpy(), 12,
                               stretch=stretch)
    np.testing.assert_array_equal(out.view.cpu().numpy(), ref)


def _guarded_flat(nbytes, dtype, shape, canary=0x5A):
    buf = torch.full((GUARD + nbytes + GUARD,), canary, dtype=torch.uint8, device="cuda")
    return buf, buf[GUARD:GUARD + nbytes].view(dtype).view(*shape)


def _guards_intact(buf, canary=0x5A):
    b = buf.cpu().numpy()
    return (b[:GUARD] == canary).all() and (b[-GUARD:] == canary).all()


@pytest.mark.parametrize("bands,h,w,pad_in,pad_out", SHAPES[:3])
def test_table_steps_write_only_their_outputs(bands, h, w, pad_in, pad_out):
    bits = 10
    L = 1 << bits
    raw, A, G, O = _data(7 * h, bands, h, w, bits, pad_in)
    lbuf, luts = _guarded_flat(bands * w * L * 2, torch.uint16, (bands, w, L))
    for b in range(bands):
        lutc.lutgen(A[b], G[b], O[b], bits, out=luts[b])
    hbuf, H = _guarded_flat(bands * L * 8, torch.uint64, (bands, L))
    lutc.hist(raw, A, G, O, bits, out=H)
    sbuf, S = _guarded_flat(bands * L, torch.uint8, (bands, L))
    qbuf, lohi = _guarded_flat(bands * 8, torch.int32, (bands, 2))
    lutc.stretch(H, bits, S=S, lohi=lohi)
    cbuf, clut = _guarded_flat(bands * w * L, torch.uint8, (bands, w, L))
    for b in range(bands):
        lutc.compose(luts[b], S[b], bits, out=clut[b])
    o8 = Guarded(bands, h, w, torch.uint8, pad_out)
    lutc.apply_u8(raw, clut, bits, out=o8.view)
    o16 = Guarded(bands, h, w, torch.uint16, pad_out)
    lutc.apply_u16(raw, luts, bits, out=o16.view)
    o2 = Guarded(bands, h, w, torch.uint8, pad_out + 1)
    lutc.apply_stretch(raw, A, G, O, bits, S, out=o2.view)
    torch.cuda.synchronize()
    for t in (lbuf, hbuf, sbuf, qbuf, cbuf):
        assert _guards_intact(t)
    o8.check()
    o16.check()
    o2.check()
    assert torch.equal(o8.view, o2.view)


@pytest.mark.parametrize("h,w,pad_in,pad_out", [(67, 300, 4, 8), (35, 144, 0, 1), (100, 1031, 1, 3), (3, 9, 0, 2)])
@pytest.mark.parametrize("correct", [False, True])
def test_demosaic_writes_only_its_planes(h, w, pad_in, pad_out, correct):
    raw, A, G, O = _data(3 * h + w, 1, h, w, 12, pad_in)
    out = Guarded(3, h, w, torch.uint16, pad_out)
    kw = dict(A=A[0], G=G[0], O=O[0]) if correct else {}
    lutc.demosaic(raw[0], "gbrg", 12, out=out.view, **kw)
    torch.cuda.synchronize()
    out.check()


def test_batch_writes_only_its_outputs():
    ims = synth.batch_images(synth.BATCH_SEED + 5, n=10)
    images, guards = [], []
    for k, im in enumerate(ims):
        d = torch.from_numpy(im["raw"]).cuda()[:, :, :im["width"]]
        A, G, O = (torch.from_numpy(a).cuda() for a in (im["A"], im["G"], im["O"]))
        g = Guarded(im["bands"], im["height"], im["width"], torch.uint8, 16 if k % 2 else 3)
        guards.append(g)
        images.append((d, A, G, O, im["bits"], g.view, True))
    b = lutc.Batch(images)
    b.run()
    torch.cuda.synchronize()
    b.close()
    for g in guards:
        g.check()


@pytest.mark.parametrize("stretch", [True, False])
def test_host_path_writes_only_its_host_output(stretch):
    bands, h, w = 2, 3000, 1023
    raw = torch.from_numpy(synth.raster(11, bands, h, w, 12)).pin_memory()
    A, G, O = (torch.from_numpy(a).cuda() for a in synth.coeff_set(11, bands, w))
    out = Guarded(bands, h, w, torch.uint8 if stretch else torch.uint16, 5, device="cpu")
    lutc.correct_image_host(raw, A, G, O, 12, stretch=stretch, out=out.view)
    torch.cuda.synchronize()
    out.check()
    frames = [Guarded(bands, h, w, torch.uint8 if stretch else torch.uint16, 3, device="cpu") for _ in range(3)]
    lutc.correct_frames_host([raw, raw, raw], A, G, O, 12, stretch=stretch, outs=[f.view for f in frames])
    torch.cuda.synchronize()
    for f in frames:
        f.check()
        assert torch.equal(f.view, out.view)


def test_fit_writes_only_its_outputs():
    n, ncols, order = 6, 1001, 2
    x, y = synth.calib(synth.CALIB_SEED, n, ncols, 12, dead_frac=0.01)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    cb, coef = _guarded_flat(ncols * (order + 1) * 8, torch.float64, (ncols, order + 1), 0x3C)
    sb, st = _guarded_flat(ncols * 4, torch.int32, (ncols,), 0x3C)
    qb, q = _guarded_flat(3 * ncols * 4, torch.int32, (3, ncols), 0x3C)
    lutc.fit(xd, yd, order, q16=True, coef=coef, status=st, codes=q)
    torch.cuda.synchronize()
    for t in (cb, sb, qb):
        assert _guards_intact(t, 0x3C)
