"""Parity of the CUDA path with the CPU oracle, element by element, bit-exact (GPU).

All arithmetic of the method is integer, so the tolerance is zero everywhere:
tables, histograms, lo/hi, stretch tables and every output pixel must be
identical.  Shapes span several column strips (8 x 256 columns each) and row
groups with ragged tails; edge cases cover empty rasters, single rows and
columns, unaligned pitches and base pointers (the generic path), DN above
2^bits - 1, dead columns, constant bands (hi == lo) and columns whose
response needs 64-bit evaluation.
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


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy()


def make_case(seed, bands, h, w, bits, dead=0.0, sat=0.0, extreme_cols=0):
    raw = synth.raster(seed, bands, h, w, bits, dead_frac=dead, sat_frac=sat)
    A, G, O = synth.coeff_set(seed, bands, w)
    if extreme_cols:
        rng = np.random.default_rng(seed)
        cols = rng.choice(w, size=min(w, extreme_cols), replace=False)
        A[:, cols] = rng.integers(-(2 ** 31), 2 ** 31 - 1, (bands, len(cols)))
        G[:, cols] = rng.integers(-(2 ** 31), 2 ** 31 - 1, (bands, len(cols)))
        O[:, cols] = rng.integers(-(2 ** 31), 2 ** 31 - 1, (bands, len(cols)))
    return raw, A, G, O


def pitched_device_raster(raw: np.ndarray, pad_elems: int, offset_elems: int = 0) -> torch.Tensor:
    """A device view [bands, h, w] whose rows have a pitch of w + pad_elems and start offset_elems in."""
    bands, h, w = raw.shape
    pitch = w + pad_elems
    flat = np.full(offset_elems + bands * h * pitch + 8, 0xBEEF, np.uint16)
    flat[offset_elems:offset_elems + bands * h * pitch].reshape(bands, h, pitch)[:, :, :w] = raw
    d = torch.from_numpy(flat).cuda()
    return d[offset_elems:offset_elems + bands * h * pitch].view(bands, h, pitch)[:, :, :w]


# ----------------------------------------------------------------------------- step (L)

@pytest.mark.parametrize("bits", [8, 10, 12, 14, 15, 16])
def test_lutgen(bits):
    raw, A, G, O = make_case(10 + bits, 1, 1, 37, bits, extreme_cols=9)
    lut = lutc.lutgen(dev(A[0]), dev(G[0]), dev(O[0]), bits)
    np.testing.assert_array_equal(host(lut), oracle.lutgen(A[0], G[0], O[0], bits))


# ----------------------------------------------------------------------------- steps (P), (C), (A), (S) one by one

@pytest.mark.parametrize("pad,off", [(0, 0), (8, 0), (3, 0), (0, 1)])
def test_apply_u16_and_plain_chain(pad, off):
    bits = 12
    raw, A, G, O = make_case(21, 2, 67, 1029, bits)
    raw[0, 0, :5] = [4096, 65535, 5000, 4095, 0]  # DN above M read entry M
    luts = np.stack([oracle.lutgen(A[b], G[b], O[b], bits) for b in range(2)])
    d_raw = pitched_device_raster(raw, pad, off)
    d_lut = torch.empty((2, 1029, 1 << bits), dtype=torch.uint16, device="cuda")
    for b in range(2):
        lutc.lutgen(dev(A[b]), dev(G[b]), dev(O[b]), bits, out=d_lut[b])
    np.testing.assert_array_equal(host(d_lut), luts)
    out16 = lutc.apply_u16(d_raw, d_lut, bits)
    ref16 = np.stack([oracle.apply_u16(raw[b], luts[b], bits) for b in range(2)])
    np.testing.assert_array_equal(host(out16), ref16)
    # the plain per-call chain (H) -> (S) -> (C) -> (A)
    hist = lutc.hist(d_raw, dev(A), dev(G), dev(O), bits)
    ref_hist = np.stack([oracle.hist(raw[b], luts[b], bits) for b in range(2)])
    np.testing.assert_array_equal(host(hist), ref_hist)
    S, lohi = lutc.stretch(hist, bits)
    for b in range(2):
        rS, lo, hi = oracle.stretch(ref_hist[b], bits)
        np.testing.assert_array_equal(host(S[b]), rS)
        assert tuple(host(lohi[b])) == (lo, hi)
    clut = torch.empty((2, 1029, 1 << bits), dtype=torch.uint8, device="cuda")
    for b in range(2):
        lutc.compose(d_lut[b], S[b], bits, out=clut[b])
    ref_clut = np.stack([oracle.compose(luts[b], host(S[b]), bits) for b in range(2)])
    np.testing.assert_array_equal(host(clut), ref_clut)
    out8 = lutc.apply_u8(d_raw, clut, bits)
    ref8 = np.stack([oracle.apply_u8(raw[b], ref_clut[b], bits) for b in range(2)])
    np.testing.assert_array_equal(host(out8), ref8)
    np.testing.assert_array_equal(ref8, oracle.correct_image(raw, A, G, O, bits, stretch=True))


@pytest.mark.parametrize("bits", [8, 10, 12, 14, 16])
def test_hist_every_bit_depth(bits):
    raw, A, G, O = make_case(30 + bits, 2, 129, 4133, bits, sat=0.001)
    hist = lutc.hist(dev(raw), dev(A), dev(G), dev(O), bits)
    for b in range(2):
        lut = oracle.lutgen(A[b], G[b], O[b], bits)
        np.testing.assert_array_equal(host(hist[b]), oracle.hist(raw[b], lut, bits))
    assert int(host(hist).sum()) == 2 * 129 * 4133


@pytest.mark.parametrize("bits", list(range(8, 17)))
@pytest.mark.parametrize("offset", [0, 1])
def test_stretch_every_bit_depth_and_alignment(bits, offset):
    # offset 1: the histogram starts 8 bytes off a 16-byte boundary (bins read one by one)
    L = 1 << bits
    rng = np.random.default_rng(bits * 7 + offset)
    h = np.zeros((3, L), np.uint64)
    h[0] = rng.integers(0, 1000, L).astype(np.uint64)
    c = L // 3  # almost all mass in five bins: lo and hi inside one thread's run
    h[1, c:c + 5] = rng.integers(1, 10**6, 5).astype(np.uint64)
    h[1] += rng.integers(0, 2, L).astype(np.uint64)
    h[2] = (rng.random(L) ** 8 * 1e9).astype(np.uint64)  # long tail: thresholds far apart
    flat = np.zeros(3 * L + 1, np.uint64)
    flat[offset:offset + 3 * L] = h.ravel()
    hist = dev(flat)[offset:offset + 3 * L].view(3, L)
    S, lohi = lutc.stretch(hist, bits)
    for b in range(3):
        rS, lo, hi = oracle.stretch(h[b], bits)
        np.testing.assert_array_equal(host(S[b]), rS)
        assert tuple(host(lohi[b])) == (lo, hi)


def test_stretch_degenerate_histograms():
    bits = 12
    L = 1 << bits
    h = np.zeros((4, L), np.uint64)
    h[0, 777] = 1234  # constant band
    # h[1] empty
    h[2, 0] = 1
    h[2, L - 1] = 1
    h[3] = np.random.default_rng(0).integers(0, 1 << 40, L).astype(np.uint64)  # large counts
    S, lohi = lutc.stretch(dev(h), bits)
    for b in range(4):
        rS, lo, hi = oracle.stretch(h[b], bits)
        np.testing.assert_array_equal(host(S[b]), rS)
        assert tuple(host(lohi[b])) == (lo, hi)


# ----------------------------------------------------------------------------- fused correct_image

CASES = [
    # bands, h, w, bits, dead, sat, pad, off, extreme
    (1, 1, 1, 12, 0, 0, 0, 0, 0),
    (1, 5, 7, 12, 0, 0, 0, 0, 0),
    (2, 33, 8, 10, 0, 0, 0, 0, 0),
    (1, 17, 9, 12, 0, 0, 0, 0, 0),
    (3, 257, 2051, 12, 0, 0, 0, 0, 0),
    (2, 129, 4133, 14, 0.01, 0.001, 0, 0, 0),
    (2, 100, 1000, 8, 0, 0, 0, 0, 0),
    (1, 300, 700, 15, 0, 0, 0, 0, 0),
    (1, 200, 600, 16, 0, 0, 0, 0, 0),
    (2, 77, 1500, 12, 0, 0, 3, 0, 0),     # rows not 16-byte aligned
    (2, 77, 1500, 12, 0, 0, 8, 1, 0),     # base not 16-byte aligned
    (2, 90, 3000, 12, 0, 0, 0, 0, 40),    # columns needing int64
    (4, 64, 520, 14, 0.2, 0.01, 0, 0, 3),
    (8, 3, 600, 12, 0, 0, 0, 0, 0),       # many band changes per block
    (3, 1000, 300, 10, 0, 0, 0, 0, 0),    # one narrow strip per band
    (2, 500, 4100, 12, 0, 0, 8, 0, 0),    # pitched rows, 16-byte aligned
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "b%d_h%d_w%d_bits%d" % c[:4] + ("_pad%d_off%d" % c[6:8]) + ("_x%d" % c[8]))
def test_correct_image(case):
    bands, h, w, bits, dead, sat, pad, off, extreme = case
    raw, A, G, O = make_case(1000 + h + w + bits, bands, h, w, bits, dead=dead, sat=sat, extreme_cols=extreme)
    if h * w > 4:
        raw[0, h // 2, :3] = [65535, min(65535, 1 << bits), (1 << bits) - 1]  # DN above M
    d_raw = pitched_device_raster(raw, pad, off) if (pad or off) else dev(raw)
    dA, dG, dO = dev(A), dev(G), dev(O)
    out, (hist, S, lohi) = lutc.correct_image(d_raw, dA, dG, dO, bits, stretch=True, with_tables=True)
    ref, (rh, rS, rl) = oracle.correct_image(raw, A, G, O, bits, stretch=True, with_tables=True)
    np.testing.assert_array_equal(host(hist), rh)
    np.testing.assert_array_equal(host(lohi), rl)
    np.testing.assert_array_equal(host(S), rS)
    np.testing.assert_array_equal(host(out), ref)
    out16 = lutc.correct_image(d_raw, dA, dG, dO, bits, stretch=False)
    np.testing.assert_array_equal(host(out16), oracle.correct_image(raw, A, G, O, bits, stretch=False))


def test_correct_image_pitched_output_and_canaries():
    bands, h, w, bits = 2, 61, 999, 12
    raw, A, G, O = make_case(77, bands, h, w, bits)
    pitch = w + 13
    buf = torch.full((bands * h * pitch + 64,), 0xA5, dtype=torch.uint8, device="cuda")
    out = buf[:bands * h * pitch].view(bands, h, pitch)[:, :, :w]
    lutc.correct_image(dev(raw), dev(A), dev(G), dev(O), bits, out=out)
    full = host(buf)
    assert np.all(full[bands * h * pitch:] == 0xA5)
    assert np.all(full[:bands * h * pitch].reshape(bands, h, pitch)[:, :, w:] == 0xA5)
    np.testing.assert_array_equal(host(out), oracle.correct_image(raw, A, G, O, bits))


def test_constant_band_maps_to_zero():
    bits = 12
    raw = np.full((1, 40, 300), 1234, np.uint16)
    A = np.zeros((1, 300), np.int32)
    G = np.full((1, 300), 65536, np.int32)
    O = np.zeros((1, 300), np.int32)
    out, (hist, S, lohi) = lutc.correct_image(dev(raw), dev(A), dev(G), dev(O), bits, with_tables=True)
    assert tuple(host(lohi[0])) == (1234, 1234)
    assert not host(out).any() and not host(S).any()


def test_empty_raster_defines_tables():
    bits = 10
    raw = torch.empty((2, 0, 16), dtype=torch.uint16, device="cuda")
    A = torch.zeros((2, 16), dtype=torch.int32, device="cuda")
    ws = torch.full((lutc.correct_image_workspace(lutc.raster_desc(raw, bits)),), 7, dtype=torch.uint8, device="cuda")
    out, (hist, S, lohi) = lutc.correct_image(raw, A, A, A, bits, workspace=ws, with_tables=True)
    assert out.numel() == 0
    assert not host(hist).any() and not host(S).any() and not host(lohi).any()


def test_repeated_calls_and_side_stream_agree():
    bits = 12
    raw, A, G, O = make_case(5, 2, 300, 2500, bits)
    dr, dA, dG, dO = dev(raw), dev(A), dev(G), dev(O)
    ws = torch.empty(lutc.correct_image_workspace(lutc.raster_desc(dr, bits)), dtype=torch.uint8, device="cuda")
    first = lutc.correct_image(dr, dA, dG, dO, bits, workspace=ws).clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        second = lutc.correct_image(dr, dA, dG, dO, bits, workspace=ws, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(first), host(second))
    np.testing.assert_array_equal(host(first), oracle.correct_image(raw, A, G, O, bits))


def test_fused_equals_plain_chain_on_device():
    bits = 14
    raw, A, G, O = make_case(9, 3, 150, 3100, bits, dead=0.01, sat=0.001)
    dr, dA, dG, dO = dev(raw), dev(A), dev(G), dev(O)
    fused = lutc.correct_image(dr, dA, dG, dO, bits)
    hist = lutc.hist(dr, dA, dG, dO, bits)
    S, _ = lutc.stretch(hist, bits)
    clut = torch.empty((3, 3100, 1 << bits), dtype=torch.uint8, device="cuda")
    for b in range(3):
        lutc.compose(lutc.lutgen(dA[b], dG[b], dO[b], bits), S[b], bits, out=clut[b])
    plain = lutc.apply_u8(dr, clut, bits)
    np.testing.assert_array_equal(host(fused), host(plain))


def test_no_kernel_recorded_a_device_error():
    import ctypes
    raw, A, G, O = make_case(6, 2, 200, 3000, 12)
    lutc.correct_image(dev(raw), dev(A), dev(G), dev(O), 12)
    status = ctypes.c_int(-99)
    rc = lutc.lib().lutc_device_status(ctypes.byref(status), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0 and status.value == 0


def test_status_errors_surface_as_exceptions():
    raw = torch.zeros((1, 4, 4), dtype=torch.uint16, device="cuda")
    A = torch.zeros((1, 5), dtype=torch.int32, device="cuda")  # wrong width
    with pytest.raises(lutc.LutcError):
        lutc.correct_image(raw, A, A, A, 12)
    with pytest.raises(lutc.LutcError):
        lutc.correct_image(raw, A[:, :4], A[:, :4], A[:, :4], 12, workspace=torch.empty(8, dtype=torch.uint8, device="cuda"))


# ----------------------------------------------------------------------------- named workloads

def test_tiny_workload_detector_only():
    wl = synth.WORKLOADS["tiny"]
    raw = synth.raster(wl.seed, wl.bands, wl.height, wl.width, wl.bits)
    A, G, O = synth.coeff_set(wl.seed, wl.bands, wl.width)
    out = lutc.correct_image(dev(raw), dev(A), dev(G), dev(O), wl.bits, stretch=False)
    ref = oracle.correct_image(raw, A, G, O, wl.bits, stretch=False)
    np.testing.assert_array_equal(host(out), ref)
    # the per-call path with a materialised LUT gives the same raster
    lut = lutc.lutgen(dev(A[0]), dev(G[0]), dev(O[0]), wl.bits).unsqueeze(0)
    np.testing.assert_array_equal(host(lutc.apply_u16(dev(raw), lut, wl.bits)), ref)


@pytest.mark.parametrize("name", ["scene", "large14"])
def test_full_size_workload(name):
    """The full-size single-scene workloads, in the launch configuration the benchmark times, every pixel."""
    wl = synth.WORKLOADS[name]
    raw = synth.raster(wl.seed, wl.bands, wl.height, wl.width, wl.bits, dead_frac=wl.dead_frac, sat_frac=wl.sat_frac)
    A, G, O = synth.coeff_set(wl.seed, wl.bands, wl.width)
    out, (hist, S, lohi) = lutc.correct_image(dev(raw), dev(A), dev(G), dev(O), wl.bits, with_tables=True)
    got = host(out)
    got_hist, got_lohi, got_S = host(hist), host(lohi), host(S)
    del out
    torch.cuda.empty_cache()
    assert [int(x) for x in got_hist.sum(axis=1)] == [wl.height * wl.width] * wl.bands
    for b in range(wl.bands):  # one band at a time keeps host memory bounded
        ref, (rh, rS, rl) = oracle.correct_image(raw[b:b + 1], A[b:b + 1], G[b:b + 1], O[b:b + 1], wl.bits,
                                                 with_tables=True)
        np.testing.assert_array_equal(got_hist[b], rh[0])
        np.testing.assert_array_equal(got_lohi[b], rl[0])
        np.testing.assert_array_equal(got_S[b], rS[0])
        np.testing.assert_array_equal(got[b], ref[0])


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("column_threads", [64, 128, 256])
def test_every_launch_configuration_is_exact(path, column_threads):
    """Both kernel families and every strip width give the oracle's result (speed is all tuning may change)."""
    cases = [(3, 130, 2600, 12), (2, 97, 777, 14), (2, 64, 1500, 10)]
    try:
        for bands, h, w, bits in cases:
            lutc.set_tuning(bits, path=path, column_threads=column_threads, blocks_per_sm=2 if path == 1 else 0)
            raw, A, G, O = make_case(900 + w, bands, h, w, bits, sat=0.001)
            dr, dA, dG, dO = dev(raw), dev(A), dev(G), dev(O)
            out, (hist, S, lohi) = lutc.correct_image(dr, dA, dG, dO, bits, with_tables=True)
            ref, (rh, rS, rl) = oracle.correct_image(raw, A, G, O, bits, with_tables=True)
            np.testing.assert_array_equal(host(hist), rh)
            np.testing.assert_array_equal(host(out), ref)
            np.testing.assert_array_equal(host(lutc.correct_image(dr, dA, dG, dO, bits, stretch=False)),
                                          oracle.correct_image(raw, A, G, O, bits, stretch=False))
            np.testing.assert_array_equal(host(lutc.apply_stretch(dr, dA, dG, dO, bits, S)), ref)
    finally:
        for bits in (10, 12, 14):
            lutc.reset_tuning(bits)


@pytest.mark.parametrize("column_threads", [64, 128, 256])
def test_rasters_with_fewer_tiles_than_a_wave(column_threads):
    """TMA passes on rasters with fewer tiles of work than one wave of blocks: the grid shrinks to the
    tiles (one tile of rows per block, the last share ragged), down to a single block; every result
    equals the oracle's."""
    cases = [(1, 1, 256, 12), (1, 5, 1024, 12), (2, 3, 2048, 10), (3, 17, 4096, 14), (1, 9, 16384, 12),
             (4, 33, 800, 12), (1, 64, 520, 13)]
    try:
        for bands, h, w, bits in cases:
            lutc.set_tuning(bits, path=1, column_threads=column_threads)
            raw, A, G, O = make_case(1700 + h * w + column_threads, bands, h, w, bits, sat=0.01)
            dr, dA, dG, dO = dev(raw), dev(A), dev(G), dev(O)
            out, (hist, S, lohi) = lutc.correct_image(dr, dA, dG, dO, bits, with_tables=True)
            assert lutc.last_path() == _lib.LUTC_PATH_TMA
            ref, (rh, rS, rl) = oracle.correct_image(raw, A, G, O, bits, with_tables=True)
            np.testing.assert_array_equal(host(hist), rh, err_msg=str((bands, h, w, bits)))
            np.testing.assert_array_equal(host(lohi), rl)
            np.testing.assert_array_equal(host(out), ref, err_msg=str((bands, h, w, bits)))
            np.testing.assert_array_equal(host(lutc.correct_image(dr, dA, dG, dO, bits, stretch=False)),
                                          oracle.correct_image(raw, A, G, O, bits, stretch=False))
    finally:
        for bits in (10, 12, 13, 14):
            lutc.reset_tuning(bits)


def test_a_wait_that_runs_out_is_reported_and_the_device_stays_usable():
    # a barrier nobody completes, with a limit of 2 M cycles (~1 ms): the wait gives up, records
    # LUTC_ETIMEOUT in the status word and the block returns
    lib = lutc.lib()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = ctypes.c_int(-99)
    assert lib.lutc_device_status(ctypes.byref(status), st) == 0 and status.value == 0
    assert lib.lutc_selftest_wait_timeout(2_000_000, st) == 0
    assert lib.lutc_device_status(ctypes.byref(status), st) == 0 and status.value == _lib.LUTC_ETIMEOUT
    # read-and-clear: the next read is clean, and the device still runs work exactly
    assert lib.lutc_device_status(ctypes.byref(status), st) == 0 and status.value == 0
    raw = synth.raster(3, 1, 64, 300, 12)
    A, G, O = synth.coeff_set(3, 1, 300)
    d = [torch.from_numpy(a).cuda() for a in (raw, A, G, O)]
    np.testing.assert_array_equal(lutc.correct_image(*d, 12).cpu().numpy(), oracle.correct_image(raw, A, G, O, 12))
    assert lib.lutc_selftest_wait_timeout(0, st) == _lib.LUTC_EINVAL
