"""The request loop on the GPU: results identical alone and in a mix, and equal to the oracle (GPU).

Tolerance zero: the arithmetic is integer.  A request's output must not
depend on which batch carried it, how full that batch was, or what else
was in flight on other streams.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

import paper_1505_05655_gb300 as lutc  # noqa: E402
from paper_1505_05655_gb300 import _lib  # noqa: E402

SENSORS = [(0, 700, 1, 12), (1, 1500, 3, 10), (2, 517, 4, 14), (3, 2100, 1, 12), (4, 999, 3, 12)]


def _setup(server, host=False):
    pool = {}
    for sid, w, bands, bits in SENSORS:
        A, G, O = synth.coeff_set(5000 + sid, bands, w)
        server.register_sensor(sid, w, bands, bits, A, G, O)
        raw = synth.raster(5000 + sid, bands, 400, w, bits, sat_frac=0.001)
        pool[sid] = dict(raw=raw, A=A, G=G, O=O, bits=bits, w=w, bands=bands,
                         draw=torch.from_numpy(raw).cuda())
    return pool


def _expected(p, h):
    return oracle.correct_image(np.ascontiguousarray(p["raw"][:, :h]), p["A"], p["G"], p["O"], p["bits"])


def test_result_is_the_same_alone_and_in_a_mix():
    # batches wait out their window even on an idle device, so that the target lands in a mix
    server = lutc.Server(budget_bytes=2 << 30, max_batch=8, max_wait_us=3000, streams=3, hold_when_idle=True)
    pool = _setup(server)
    target = (2, 333)  # sensor, rows
    p = pool[target[0]]
    alone = torch.empty((p["bands"], target[1], p["w"]), dtype=torch.uint8, device="cuda")
    # a request's bands are stacked at rows x pitch: submit contiguous copies of the first rows
    req = p["draw"][:, :target[1]].contiguous()
    info = server.wait(server.submit(target[0], req, alone))
    assert info.status == 0 and info.batch_size == 1
    # the same request among many others, several batches in flight
    rng = np.random.default_rng(1)
    others = []
    mixed = torch.empty_like(alone)
    tickets = []
    for k in range(40):
        if k == 21:
            tickets.append(("target", server.submit(target[0], req, mixed)))
        sid = int(rng.integers(0, len(SENSORS)))
        h = int(rng.integers(1, 400))
        q = pool[sid]
        out = torch.empty((q["bands"], h, q["w"]), dtype=torch.uint8, device="cuda")
        others.append((sid, h, out))
        tickets.append((len(others) - 1, server.submit(sid, q["draw"][:, :h].contiguous(), out)))
    infos = {}
    for key, t in tickets:
        infos[key] = server.wait(t)
    assert all(i.status == 0 for i in infos.values())
    assert infos["target"].batch_size > 1
    torch.cuda.synchronize()
    np.testing.assert_array_equal(mixed.cpu().numpy(), alone.cpu().numpy())
    np.testing.assert_array_equal(alone.cpu().numpy(), _expected(p, target[1]))
    for sid, h, out in others[::5]:
        np.testing.assert_array_equal(out.cpu().numpy(), _expected(pool[sid], h))
    st = server.stats()
    assert st["largest_batch"] <= 8 and st["completed"] == 42
    server.close()


def test_host_requests_copy_in_and_out():
    server = lutc.Server(budget_bytes=1 << 30, max_batch=4, max_wait_us=500, streams=2)
    pool = _setup(server)
    reqs = []
    for k, (sid, w, bands, bits) in enumerate(SENSORS * 2):
        h = 50 + 37 * k
        raw = torch.from_numpy(np.ascontiguousarray(pool[sid]["raw"][:, :h])).pin_memory()
        out = torch.zeros((bands, h, w), dtype=torch.uint8).pin_memory()
        reqs.append((sid, h, out, server.submit(sid, raw.numpy(), out.numpy(), host=True, keep=raw)))
    for sid, h, out, t in reqs:
        assert server.wait(t).status == 0
        np.testing.assert_array_equal(out.numpy(), _expected(pool[sid], h))
    server.close()


def test_small_budget_admits_in_turn_and_stays_exact():
    # each host request stages ~1-3 MB; a 6 MiB budget forces requests to wait for memory
    budget = 6 << 20
    server = lutc.Server(budget_bytes=budget, max_batch=8, max_wait_us=200, streams=3)
    pool = _setup(server)
    reqs = []
    for k in range(30):
        sid = k % len(SENSORS)
        p = pool[sid]
        h = 200
        out = np.zeros((p["bands"], h, p["w"]), np.uint8)
        raw = np.ascontiguousarray(p["raw"][:, :h])
        reqs.append((sid, out, server.submit(sid, raw, out, host=True, keep=raw)))
    for sid, out, t in reqs:
        info = server.wait(t)
        assert info.status == 0
        np.testing.assert_array_equal(out, _expected(pool[sid], 200))
    assert server.stats()["completed"] == 30
    server.close()


def test_device_budget_that_cannot_be_allocated_is_refused():
    # a petabyte budget: the server's one device allocation fails, creation reports LUTC_ENOMEM and
    # the device stays usable
    with pytest.raises(lutc.LutcError) as e:
        lutc.Server(budget_bytes=1 << 50)
    assert e.value.status == _lib.LUTC_ENOMEM
    x = torch.ones(1024, device="cuda")
    assert float(x.sum()) == 1024.0


def test_replayed_schedule_on_the_device_equals_the_oracle():
    # lutc_server_replay drives the real server: an open-loop schedule at a rate high enough to batch,
    # every request's output equal to the oracle, the schedule kept, latency counted from the schedule
    # every batch waits out a 1 ms window, so that requests share batches whatever the device's pace
    server = lutc.Server(budget_bytes=4 << 30, max_batch=8, max_wait_us=1000, streams=3, hold_when_idle=True)
    pool = _setup(server)
    rng = np.random.default_rng(7)
    n = 120
    at = np.cumsum(rng.exponential(1 / 3000.0, n))
    reqs, expect = [], []
    for i in range(n):
        sid = int(rng.integers(0, len(SENSORS)))
        h = int(rng.integers(1, 400))
        p = pool[sid]
        raw = p["draw"][:, :h].contiguous()
        out = torch.full((p["bands"], h, p["w"]), 0xA5, dtype=torch.uint8, device="cuda")
        reqs.append((float(at[i]), sid, raw, out, False))
        expect.append((sid, h))
    r = server.replay(reqs)
    torch.cuda.synchronize()
    assert (r["status"] == 0).all()
    assert np.all(r["done_s"] >= r["scheduled_s"]) and np.all(np.diff(r["scheduled_s"]) >= 0)
    assert r["batch_size"].max() > 1
    for (sid, h), (_, _, _, out, _) in zip(expect, reqs):
        np.testing.assert_array_equal(out.cpu().numpy(), _expected(pool[sid], h))
    server.close()


def test_fp64_probe_runs_and_counts_its_work():
    import ctypes
    lib = _lib.lib()
    blocks, iters = 16, 64
    sink = torch.zeros(blocks * 256, dtype=torch.float64, device="cuda")
    fmas = ctypes.c_longlong(0)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.lutc_probe_fp64_fma(blocks, iters, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(fmas), st) == 0
    torch.cuda.synchronize()
    assert fmas.value == blocks * 256 * 8 * iters
    v = sink.cpu().numpy()
    assert np.isfinite(v).all() and (v > 0).all()  # every thread wrote its chains' sum
