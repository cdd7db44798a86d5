"""Host logic of the request loop, with the fake executor (CPU only, no CUDA call is made).

The fake executor runs no kernel: a batch "completes" fake_latency_us after
its launch.  Everything else is the real server: the pending queue, the
batch window (max_batch / max_wait_us), admission against the device-memory
budget (an allocator over offsets), the streams in flight, tickets, timeouts,
host-injected batch failures (fail_every) and shutdown.
"""
import threading
import time

import numpy as np
import pytest

import paper_1505_05655_gb300 as lutc
from paper_1505_05655_gb300 import _lib

W, BANDS, BITS = 300, 2, 12


def _server(**kw):
    s = lutc.Server(fake_device=True, **kw)
    z = np.zeros((BANDS, W), np.int32)
    for sid in range(4):
        s.register_sensor(sid, W, BANDS, BITS, z, z, z)
    return s


def _bufs(h):
    return np.zeros((BANDS, h, W), np.uint16), np.zeros((BANDS, h, W), np.uint8)


def test_requests_complete_and_batch_up():
    s = _server(max_batch=8, max_wait_us=20000, fake_latency_us=2000)
    tickets = []
    keep = []
    for i in range(40):
        raw, out = _bufs(16)
        keep.append((raw, out))
        tickets.append(s.submit(i % 4, raw, out))
    infos = [s.wait(t) for t in tickets]
    assert all(i.status == 0 for i in infos)
    assert max(i.batch_size for i in infos) == 8
    st = s.stats()
    assert st["completed"] == 40 and st["largest_batch"] == 8 and 5 <= st["batches"] <= 40
    assert st["budget_in_use"] < 64 * 1024  # only the cached coefficients remain
    s.close()


def test_window_holds_a_lone_request_then_launches_it():
    s = _server(max_batch=32, max_wait_us=60000, fake_latency_us=100, hold_when_idle=True)
    raw, out = _bufs(8)
    t0 = time.perf_counter()
    info = s.wait(s.submit(0, raw, out))
    waited = info.start_s - info.submit_s
    assert info.status == 0 and info.batch_size == 1
    assert 0.05 <= waited < 1.0, waited
    assert time.perf_counter() - t0 >= 0.05
    # a full batch does not wait for the window
    ts = [s.submit(1, *_bufs(8)) for _ in range(32)]
    infos = [s.wait(t) for t in ts]
    assert max(i.start_s - i.submit_s for i in infos) < 0.05
    s.close()


def test_idle_device_launches_a_lone_request_at_once():
    s = _server(max_batch=32, max_wait_us=200000, fake_latency_us=100)
    for _ in range(3):
        info = s.wait(s.submit(0, *_bufs(8)))
        assert info.status == 0 and info.batch_size == 1
        assert info.start_s - info.submit_s < 0.05  # far inside the 200 ms window
    s.close()


def test_requests_accumulate_while_a_batch_runs_and_launch_when_it_ends():
    # the first request launches at once (idle device) and runs 150 ms; the next ones wait for it
    # to finish, not for their 2 s window, and go as one batch
    s = _server(max_batch=32, max_wait_us=2000000, fake_latency_us=150000, streams=3)
    first = s.submit(0, *_bufs(8))
    time.sleep(0.02)
    rest = [s.submit(k % 4, *_bufs(8)) for k in range(6)]
    i0 = s.wait(first)
    infos = [s.wait(t) for t in rest]
    assert i0.batch_size == 1 and all(i.status == 0 for i in infos)
    assert all(i.batch_size == 6 for i in infos)
    assert min(i.start_s for i in infos) >= i0.done_s - 0.005  # formed when the device went idle
    assert max(i.start_s - i.submit_s for i in infos) < 1.0  # well before the window's end
    assert s.stats()["batches"] == 2
    s.close()


def test_server_config_is_checked():
    with pytest.raises(lutc.LutcError):
        lutc.Server(fake_device=True, hold_when_idle=2)
    with pytest.raises(lutc.LutcError):
        lutc.Server(fake_device=True, streams=65)


def test_queued_requests_can_be_withdrawn():
    # one stream, one request per batch, 200 ms per batch: the first request runs, the rest queue
    s = _server(max_batch=1, max_wait_us=1, streams=1, fake_latency_us=200000)
    first = s.submit(0, *_bufs(4))
    time.sleep(0.02)
    queued = [s.submit(k % 4, *_bufs(4)) for k in range(5)]
    assert s.cancel(first) is False  # already in a batch: runs to completion
    t0 = time.perf_counter()
    assert all(s.cancel(t) for t in queued[1::2])
    for t in queued[1::2]:
        info = s.wait(t)
        assert info.status == _lib.LUTC_ECANCELED and info.batch_size == 0
    assert time.perf_counter() - t0 < 0.15  # completed at once, not after the running batch
    assert s.wait(first).status == 0
    for t in queued[0::2]:
        assert s.wait(t).status == 0
    with pytest.raises(lutc.LutcError):
        s.cancel(first)  # forgotten after its wait
    assert s.stats()["completed"] == 4
    s.close()


def test_withdrawing_every_queued_request_leaves_the_loop_working():
    # requests held in a long window on an idle device, all withdrawn while the batcher waits
    s = _server(max_batch=32, max_wait_us=300000, fake_latency_us=1000, hold_when_idle=True)
    ts = [s.submit(k % 4, *_bufs(4)) for k in range(3)]
    assert all(s.cancel(t) for t in ts)
    assert all(s.wait(t).status == _lib.LUTC_ECANCELED for t in ts)
    time.sleep(0.35)  # past the window the batcher had armed for the first of them
    info = s.wait(s.submit(1, *_bufs(4)))
    assert info.status == 0 and info.batch_size == 1
    assert s.stats()["batches"] == 1
    s.close()


def test_first_request_of_a_sensor_is_the_cache_miss():
    s = _server(max_batch=1, max_wait_us=1, fake_latency_us=100)
    infos = [s.wait(s.submit(2, *_bufs(4))) for _ in range(3)]
    assert [i.cache_miss for i in infos] == [1, 0, 0]
    s.close()


def test_admission_never_exceeds_the_budget():
    # host requests need staging: 2 bands x 100 rows x (608 + 304) bytes = 182 KB each;
    # a 1 MiB budget admits only a few at a time, the rest wait in the queue
    budget = 1 << 20
    s = _server(budget_bytes=budget, max_batch=16, max_wait_us=1000, fake_latency_us=20000, streams=4)
    peak = [0]
    stop = threading.Event()

    def watch():
        while not stop.is_set():
            peak[0] = max(peak[0], s.stats()["budget_in_use"])
            time.sleep(0.001)

    th = threading.Thread(target=watch)
    th.start()
    ts = [s.submit(i % 4, *_bufs(100), host=True) for i in range(24)]
    infos = [s.wait(t) for t in ts]
    stop.set()
    th.join()
    assert all(i.status == 0 for i in infos)
    assert 0 < peak[0] <= budget
    assert max(i.batch_size for i in infos) < 16  # memory, not max_batch, bounded the batches
    s.close()


def test_request_larger_than_the_budget_is_refused():
    s = _server(budget_bytes=256 << 10, fake_latency_us=10)
    with pytest.raises(lutc.LutcError) as e:
        s.submit(0, *_bufs(2000), host=True)
    assert e.value.status == _lib.LUTC_EBUSY
    s.close()


def test_full_queue_refuses():
    s = _server(max_queue=4, max_batch=1, max_wait_us=1, streams=1, fake_latency_us=200000)
    codes = [s.try_submit(0, *_bufs(4))[0] for _ in range(12)]
    assert _lib.LUTC_EBUSY in codes and codes[0] == 0
    s.close()


def test_wait_times_out_while_running():
    s = _server(max_batch=1, max_wait_us=1, fake_latency_us=300000)
    t = s.submit(0, *_bufs(4))
    assert s.wait(t, timeout_us=1000) is None  # still running: the ticket stays valid
    info = s.wait(t)
    assert info.status == 0
    with pytest.raises(lutc.LutcError):
        s.wait(t)  # forgotten after completion
    s.close()


def test_injected_batch_failures_are_reported_per_request():
    s = _server(max_batch=1, max_wait_us=1, fake_latency_us=100, fail_every=3)
    infos = [s.wait(s.submit(0, *_bufs(4))) for _ in range(9)]
    failed = [i.status for i in infos]
    assert failed.count(_lib.LUTC_ECUDA) == 3 and failed.count(0) == 6
    s.close()


def test_unknown_sensor_and_bad_arguments():
    s = _server()
    with pytest.raises(lutc.LutcError):
        s.submit(99, *_bufs(4))
    with pytest.raises(lutc.LutcError):
        s.register_sensor(0, W, BANDS, BITS, np.zeros((BANDS, W)), np.zeros((BANDS, W)), np.zeros((BANDS, W)))
    s.close()


def test_shutdown_with_work_pending_does_not_hang():
    s = _server(max_batch=2, max_wait_us=1, streams=1, fake_latency_us=50000)
    for _ in range(20):
        s.submit(0, *_bufs(4))
    t0 = time.perf_counter()
    s.close()  # in-flight batch drains, pending requests end with LUTC_ESHUTDOWN
    assert time.perf_counter() - t0 < 5


def test_concurrent_submitters():
    s = _server(max_batch=16, max_wait_us=500, fake_latency_us=500, streams=3)
    results = []
    lock = threading.Lock()

    def client(k):
        for _ in range(25):
            info = s.wait(s.submit(k % 4, *_bufs(8)))
            with lock:
                results.append(info.status)

    ths = [threading.Thread(target=client, args=(k,)) for k in range(6)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert len(results) == 150 and all(r == 0 for r in results)
    assert s.stats()["completed"] == 150
    s.close()


def test_replay_keeps_its_schedule_and_collects_every_request():
    # lutc_server_replay: requests handed over by a native thread at their scheduled times; the
    # latency is counted from the scheduled time, so lateness of the hand-over would show
    s = _server(max_batch=8, max_wait_us=1000, fake_latency_us=300, hold_when_idle=True)
    bufs = [_bufs(8) for _ in range(16)]
    rng = np.random.default_rng(7)
    at = np.cumsum(rng.exponential(1 / 4000.0, 800))  # Poisson arrivals at 4000 requests per second
    sched = [(float(t), i % 4, *bufs[i % 16], False) for i, t in enumerate(at)]
    r = s.replay(sched)
    assert (r["status"] == 0).all()
    assert np.all(np.diff(r["scheduled_s"]) >= 0)
    np.testing.assert_allclose(r["scheduled_s"] - r["scheduled_s"][0], at - at[0], atol=1e-9)
    lag = r["submit_s"] - r["scheduled_s"]
    assert lag.min() >= 0 and np.median(lag) < 1e-3, np.median(lag)
    lat = r["done_s"] - r["scheduled_s"]
    assert lat.min() >= 300e-6  # at least the fake device's latency
    assert r["batch_size"].max() > 1  # a 1 ms window at 4000 requests per second fills batches
    assert s.stats()["completed"] == 800
    s.close()


def test_replay_closed_burst_rides_out_a_full_queue():
    # a burst larger than the queue: refused submissions (LUTC_EBUSY) are retried until admitted
    s = _server(max_batch=4, max_wait_us=100, fake_latency_us=200, max_queue=16)
    raw, out = _bufs(8)
    r = s.replay([(0.0, i % 4, raw, out, False) for i in range(200)])
    assert (r["status"] == 0).all() and s.stats()["completed"] == 200
    s.close()


def test_replay_rejects_a_bad_schedule_before_submitting():
    s = _server()
    raw, out = _bufs(8)
    for bad in ([(0.01, 0, raw, out, False), (0.0, 0, raw, out, False)], [(-1.0, 0, raw, out, False)],
                [(float("nan"), 0, raw, out, False)]):
        with pytest.raises(lutc.LutcError) as e:
            s.replay(bad)
        assert e.value.status == _lib.LUTC_EINVAL
    assert s.stats()["completed"] == 0
    # an unknown sensor stops the schedule at that request; the ones before it complete
    r = None
    with pytest.raises(lutc.LutcError):
        s.replay([(0.0, 0, raw, out, False), (0.0, 99, raw, out, False), (0.0, 1, raw, out, False)])
    assert s.stats()["completed"] == 1
    s.close()
