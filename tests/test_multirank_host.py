"""Host logic of the multi-rank paths on CPU ranks over gloo (world size 2).

(1) The benchmark's weak scaling: every rank corrects its own scene (inputs
seeded by rank), the step time is the slowest rank's and the job's rate
counts every rank's pixels.  (2) Bands split by rows: the only exchange is the
sum of the per-band histograms, after which each rank's rows are corrected
exactly as a single device would.  The library's GPU steps are replaced by
the CPU oracle here; on GPUs the same code runs them over NCCL.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_1505_05655_gb300 import sharded


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _oracle_steps():
    def hist(raw, A, G, O, bits):
        r = raw.numpy()
        return torch.from_numpy(np.stack([oracle.hist(np.ascontiguousarray(r[b]),
                                                      oracle.lutgen(A[b].numpy(), G[b].numpy(), O[b].numpy(), bits),
                                                      bits) for b in range(r.shape[0])]))

    def stretch(h, bits):
        return torch.from_numpy(np.stack([oracle.stretch(h[b].numpy(), bits)[0] for b in range(h.shape[0])]))

    def apply(raw, A, G, O, bits, S):
        r = raw.numpy()
        out = []
        for b in range(r.shape[0]):
            lut = oracle.lutgen(A[b].numpy(), G[b].numpy(), O[b].numpy(), bits)
            out.append(oracle.apply_u8(np.ascontiguousarray(r[b]), oracle.compose(lut, S[b].numpy(), bits), bits))
        return torch.from_numpy(np.stack(out))

    return hist, stretch, apply


def _run(rank, world, port, fn, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, fn(rank, world)))
    except Exception as e:  # reported by the parent
        q.put((rank, e))
    finally:
        dist.destroy_process_group()


def _spawn(fn, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_run, args=(r, world, port, fn, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
    for r, v in res.items():
        if isinstance(v, Exception):
            raise v
    return res


def _band_split(rank, world):
    bands, h, w, bits = 2, 97, 300, 12
    raw = synth.raster(41, bands, h, w, bits, sat_frac=0.01)
    A, G, O = (torch.from_numpy(a) for a in synth.coeff_set(41, bands, w))
    r0, r1 = sharded.row_range(h, world, rank)
    out = sharded.correct_rows(torch.from_numpy(np.ascontiguousarray(raw[:, r0:r1])), A, G, O, bits,
                               steps=_oracle_steps())
    return r0, r1, out.numpy()


def test_rows_split_across_two_ranks_equal_the_single_device_result():
    res = _spawn(_band_split)
    bands, h, w, bits = 2, 97, 300, 12
    raw = synth.raster(41, bands, h, w, bits, sat_frac=0.01)
    A, G, O = synth.coeff_set(41, bands, w)
    full = oracle.correct_image(raw, A, G, O, bits)
    got = np.concatenate([res[r][2] for r in sorted(res)], axis=1)
    assert [res[r][:2] for r in sorted(res)] == [(0, 48), (48, 97)]
    np.testing.assert_array_equal(got, full)
    # without the exchange each half would be stretched on its own histogram: the outputs differ
    alone = oracle.correct_image(np.ascontiguousarray(raw[:, :48]), A, G, O, bits)
    assert not np.array_equal(alone, full[:, :48])


def _weak_scaling(rank, world):
    import bench
    wl = synth.WORKLOADS["tiny"]
    raw, A, G, O = bench.gen_inputs(wl, rank)
    local_ms = [10.0 + rank, 20.0 - rank]
    slowest = bench.max_over_ranks(local_ms, torch.device("cpu"))
    return slowest, bench.whole_job_rate(wl.pixels, world, 5, slowest[0]), int(raw.astype(np.int64).sum())


def test_weak_scaling_takes_the_slowest_rank_and_counts_every_rank():
    res = _spawn(_weak_scaling)
    assert res[0][0] == res[1][0] == [11.0, 20.0]
    wl = synth.WORKLOADS["tiny"]
    assert res[0][1] == pytest.approx(wl.pixels * 2 * 5 / 11e-3 / 1e9)
    assert res[0][2] != res[1][2]  # each rank corrects its own scene


def test_row_range_covers_every_row_once():
    for h in (0, 1, 7, 97, 12000):
        for world in (1, 2, 3, 8):
            spans = [sharded.row_range(h, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == h
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1
    with pytest.raises(ValueError):
        sharded.row_range(10, 2, 2)
