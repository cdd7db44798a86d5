"""Benchmark of the fused LUT correction on GB300.

One step = one ``lutc_correct_image`` (detector LUT evaluation, per-band
histogram, 2/98 % stretch, composed uint8 gather) over the whole "scene"
workload: 4 bands of 12000 x 12000 uint16 12-bit pixels, resident in HBM
(1.15 GB in, 576 MB out per step: larger than the 129 MB L2, so no flush is
needed between steps).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload scene|large14|tiny]
  python bench.py --impl reference ...   # the CPU oracle, timed on a bounded sample

With N > 1 (torchrun) every rank corrects its own scene (weak scaling, no
data-path collective); the step time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import datetime
import gc
import glob
import hashlib
import json
import os
import shutil
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Gpixel/s & % HBM peak (fused/batched vs plain); p50/p99 served latency"
UNIT = "Gpixel/s"
E2E_REPEATS = 9  # interleaved runs of each end-to-end variant; the median is reported
FALLBACK_HBM_GBS = 6800.0


# ----------------------------------------------------------------------------- helpers

def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# sources whose change invalidates a committed DRAM-traffic figure, per workload
TRAFFIC_SOURCES = {
    "scene": ["csrc/lutc_tma.cu", "csrc/lutc_ptx.cuh", "csrc/lutc_internal.cuh", "csrc/lutc_correct.cu", "_build.py"],
    "large14": ["csrc/lutc_tma.cu", "csrc/lutc_ptx.cuh", "csrc/lutc_internal.cuh", "csrc/lutc_correct.cu", "_build.py"],
    "batch": ["csrc/lutc_tma.cu", "csrc/lutc_ptx.cuh", "csrc/lutc_internal.cuh", "csrc/lutc_batch.cu", "_build.py"],
}


def _code_only(text: str) -> str:
    """Source text without comments and with whitespace collapsed: what a capture depends on.
    Preprocessor lines stay lines of their own (a directive ends at its line's end)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    out = []
    for line in text.splitlines():
        s = " ".join(line.split())
        if s:
            out.append("\n" + s + "\n" if s.startswith("#") else s)
    return " ".join(out)


def csrc_hash(workload: str) -> str:
    """Hash of the code (comments and layout aside) of the sources a workload's kernels are built from."""
    h = hashlib.sha256()
    for rel in TRAFFIC_SOURCES[workload.split("/")[0]]:
        with open(os.path.join(ROOT, "paper_1505_05655_gb300", rel), encoding="utf-8") as f:
            h.update(rel.encode())
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def ncu_l1tex_busy(kernel: str, workload: str):
    """L1TEX / shared-memory pipe utilisation of `kernel` from the committed ncu capture, if it was
    taken on this source (the pipe that bounds a kernel whose DRAM fraction is low)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            e = json.load(f)[workload][kernel]
        if e.get("l1tex_csrc", e.get("csrc")) != csrc_hash(workload) or "l1tex_busy" not in e:
            return None
        return {"busy": float(e["l1tex_busy"]), "source": e.get("l1tex_capture"), "kind": "ncu, cold launch"}
    except Exception:
        return None


def ncu_traffic(kernel: str, workload: str, units: float | None = None):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was taken on this source.

    Entries with "bytes_per_px" were captured on a smaller case of the same kernel and are
    scaled to `units` pixels per launch (traffic grows in proportion to the pixels).
    """
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        e = t[workload][kernel]
        if e.get("csrc") != csrc_hash(workload):
            return None
        if "bytes_per_px" in e:
            return float(e["bytes_per_px"]) * units
        return float(e["bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms in the background."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str | None):
        self.proc = None
        self.path = None
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        self.path = os.path.join("/tmp", "lutc_clocks_%d.csv" % os.getpid())
        cmd = [exe, "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100"]
        if device_id:
            cmd += ["-i", device_id]
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, t0: float, t1: float):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    rows.append((ts, float(parts[1]), float(parts[2]), parts[3:]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        inside = [r for r in rows if t0 - 0.15 <= r[0] <= t1 + 0.15]
        if not inside:
            inside = sorted(rows, key=lambda r: min(abs(r[0] - t0), abs(r[0] - t1)))[:2]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in inside for n, v in zip(names, r[3][2:6]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(values, device):
    """Element-wise maximum of per-rank timings over the process group (the slowest rank sets the time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_rate(pixels_per_rank: int, world: int, steps: int, ms: float) -> float:
    """Gpixel/s of the whole job: every rank's pixels over the slowest rank's time."""
    return pixels_per_rank * world * steps / (ms * 1e-3) / 1e9


def workload_config(wl) -> dict:
    what = "full pipeline: detector LUT, 2/98 % stretch, uint8 out" if wl.stretch else "detector LUT only, uint16 out"
    in_bytes = wl.pixels * 2
    return {"workload": "%s: %d bands x %d x %d uint16, %d-bit, %s" % (wl.name, wl.bands, wl.height, wl.width,
                                                                      wl.bits, what),
            "bands": wl.bands, "height": wl.height, "width": wl.width, "bits": wl.bits,
            "pixels_per_step": wl.pixels,
            "l2": ("inputs larger than L2 (%.2f GB read per step)" % (in_bytes / 1e9)) if in_bytes > 129e6
            else "inputs smaller than L2 (%.1f MB); L2 not flushed" % (in_bytes / 1e6)}


def gen_inputs(wl, seed_offset: int, raw_out=None):
    import synth
    raw = synth.raster(wl.seed + seed_offset, wl.bands, wl.height, wl.width, wl.bits, dead_frac=wl.dead_frac,
                       sat_frac=wl.sat_frac, out=raw_out)
    A, G, O = synth.coeff_set(wl.seed + seed_offset, wl.bands, wl.width)
    return raw, A, G, O


# ----------------------------------------------------------------------------- reference arm (the CPU oracle)

def run_reference(args, wl):
    """The oracle as the reference arm: its own steps on all host threads (row ranges, per-thread
    histograms summed), each step a bounded sample of the workload's rows (all bands)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import synth
    threads = max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1))
    A, G, O = synth.coeff_set(wl.seed, wl.bands, wl.width)

    def sample(rows):
        return synth.raster(wl.seed, wl.bands, rows, wl.width, wl.bits, dead_frac=wl.dead_frac, sat_frac=wl.sat_frac)

    # size each step so that warm-up + timed steps take about two minutes in all
    probe_rows = min(wl.height, 512)
    probe = sample(probe_rows)
    cpu_baseline_threads(wl, probe, A, G, O, threads)  # first call: tables built, threads started
    t = time.perf_counter()
    cpu_baseline_threads(wl, probe, A, G, O, threads)
    rate = wl.bands * probe_rows * wl.width / max(time.perf_counter() - t, 1e-6)
    per_step = 120.0 / max(1, args.steps + args.warmup)
    rows = int(max(1, min(wl.height, per_step * rate / (wl.bands * wl.width))))
    raw = sample(rows)
    for _ in range(args.warmup):
        cpu_baseline_threads(wl, raw, A, G, O, threads)
    t = time.perf_counter()
    for _ in range(args.steps):
        cpu_baseline_threads(wl, raw, A, G, O, threads)
    dt = time.perf_counter() - t
    px = wl.bands * rows * wl.width
    value = px * args.steps / dt / 1e9
    desc = ("rows 0-%d of all %d bands (%d px) of the %s workload per step; the oracle's steps (lutgen, hist, "
            "stretch, compose, apply) on %d threads" % (rows - 1, wl.bands, px, wl.name, threads))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": workload_config(wl),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- the CUDA path

def ncu_entry(workload: str, kernel: str, hash_key: str = "csrc"):
    """The committed ncu summary entry of `kernel` on `workload`, if it was taken on this source."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            e = json.load(f)[workload][kernel]
        return e if e.get(hash_key) == csrc_hash(workload) else None
    except Exception:
        return None


def smem_pipe(workload: str, kernel: str, pixels: int, measured_ms: float, sm_mhz: float | None, sms: int):
    """The shared-memory pipe floor of a pass: its LSU shared-memory wavefronts per launch (committed ncu
    capture on this source, scaled by pixels when captured on a smaller case) at one wavefront per SM
    clock on every SM, against the measured duration."""
    e = ncu_entry(workload, kernel, "smem_csrc")
    if not e or not sm_mhz:
        return None
    wf = float(e["smem_wavefronts"]) / float(e["smem_captured_pixels"]) * pixels
    floor_ms = wf / (sms * sm_mhz * 1e6) * 1e3
    return {"wavefronts_per_launch": wf, "wavefronts_per_px": wf / pixels,
            "floor_ms": floor_ms, "measured_ms": measured_ms, "frac_smem": floor_ms / measured_ms,
            "rate": "1 wavefront per SM clock, %d SMs at the sampled median %.0f MHz" % (sms, sm_mhz),
            "capture": e.get("smem_capture")}


def fused_leg(lib, lutc, wl, raw, cd, out, wsb, device, steps: int, warmup: int, ws: int = 1):
    """One lutc_correct_image step timed as CUDA-graph replays (clocks sampled meanwhile), as direct
    C-ABI calls, and per phase from traced direct calls; returns the timings and the kernel family."""
    import torch
    import torch.distributed as dist
    from paper_1505_05655_gb300._lib import LUTC_STRETCH

    stream = torch.cuda.current_stream(device)
    st = ctypes.c_void_p(stream.cuda_stream)
    desc = lutc.raster_desc(raw, wl.bits)
    flags = LUTC_STRETCH if wl.stretch else 0
    pitch = out.stride(1) * out.element_size()

    def call(s=st):
        rc = lib.lutc_correct_image(ctypes.byref(desc), cd, flags, ctypes.c_void_p(out.data_ptr()), pitch,
                                    ctypes.c_void_p(wsb.data_ptr()), wsb.numel(), s)
        if rc:
            raise RuntimeError("lutc_correct_image failed: %d" % rc)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(device)

    dev_id = None
    try:
        dev_id = str(torch.cuda.get_device_properties(device).uuid)
        dev_id = dev_id if dev_id.startswith("GPU-") else "GPU-" + dev_id
    except Exception:
        dev_id = None
    sampler = ClockSampler(dev_id)
    for _ in range(max(3, warmup)):
        call()
    path = lutc.last_path()
    barrier()
    # One step captured in a CUDA graph (histogram clear, pass 1, scan, pass 2): replaying it keeps
    # host launch latency out of the timed loop.  Every replay does the whole step's work.
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        call(ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream))
    for _ in range(3):
        graph.replay()

    def timed(fn, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1)

    wall0 = time.time()
    ms = timed(graph.replay, steps)
    wall1 = time.time()
    clocks = sampler.stop(wall0, wall1)
    direct_ms = timed(call, steps)
    phases = []
    if wl.stretch:
        k = min(steps, 200)
        lutc.trace_enable(k)
        timed(call, k)
        phases = lutc.trace_read(k)
        lutc.trace_enable(0)
    del graph
    return {"ms": ms, "direct_ms": direct_ms, "phases": phases, "path": path, "clocks": clocks, "steps": steps}


def fused_roofline(wl, workload: str, phases, path: int, clocks, peak: float, peak_src: str, sms: int):
    """Roofline of the dominant pass (HBM, algorithmic bytes over the traced mean duration) with the
    shared-memory pipe floor of both passes beside it; (roofline, phases_ms)."""
    from paper_1505_05655_gb300._lib import LUTC_PATH_TMA
    avg = [statistics.fmean(p[i] for p in phases) for i in range(3)]
    tma = path == LUTC_PATH_TMA
    kern = ("k_tma_strip<hist>", "k_stretch", "k_tma_strip<apply>") if tma else \
        ("k_strip_hist", "k_stretch", "k_strip_apply")
    keys = ("pass1", "scan", "pass2")
    alg = [2 * wl.pixels, 8 * wl.bands * (1 << wl.bits), 3 * wl.pixels]
    dom = max(range(3), key=lambda i: avg[i])
    ach = alg[dom] / (avg[dom] * 1e-3) / 1e9
    mhz = clocks["sm_mhz"] if clocks else None
    pipe = {k: smem_pipe(workload, k, wl.pixels, avg[i], mhz, sms) if tma else None
            for i, k in ((0, "pass1"), (2, "pass2"))}
    tr = ncu_traffic(keys[dom], workload, wl.pixels) if tma else None
    roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": tr, "kernel": "%s %s" % (keys[dom], kern[dom]),
            "kernel_family": "tma" if tma else "strip (lutc_last_path)",
            "l1tex": ncu_l1tex_busy(keys[dom], workload) if tma else None,
            "peak_source": peak_src + " (copy bandwidth)", "alg_bytes_per_launch": alg[dom],
            "traffic_GBs": tr / (avg[dom] * 1e-3) / 1e9 if tr else None,
            "smem_pipe": pipe}
    ph = {"pass1_hist": avg[0], "scan": avg[1], "pass2_apply": avg[2],
          "pass1_GBs": alg[0] / (avg[0] * 1e-3) / 1e9, "pass2_GBs": alg[2] / (avg[2] * 1e-3) / 1e9,
          "pass1_hbm_frac": alg[0] / (avg[0] * 1e-3) / 1e9 / peak,
          "pass2_hbm_frac": alg[2] / (avg[2] * 1e-3) / 1e9 / peak}
    return roof, ph


def run_lutc(args, wl):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)

    import paper_1505_05655_gb300 as lutc
    from paper_1505_05655_gb300._lib import LUTC_STRETCH

    lib = lutc.lib()
    n_sm = torch.cuda.get_device_properties(device).multi_processor_count
    # inputs: generated straight into pinned host memory (the end-to-end leg copies from there)
    shape = (wl.bands, wl.height, wl.width)
    raw_h = torch.empty(shape, dtype=torch.uint16, pin_memory=True)
    _, A, G, O = gen_inputs(wl, rank, raw_out=raw_h.numpy())
    out_dtype = torch.uint8 if wl.stretch else torch.uint16
    out_h = torch.empty(shape, dtype=out_dtype, pin_memory=True)
    raw = raw_h.to(device)
    dA, dG, dO = (torch.from_numpy(a).to(device) for a in (A, G, O))
    out = torch.empty(shape, dtype=out_dtype, device=device)
    desc = lutc.raster_desc(raw, wl.bits)
    cd = lutc.coeff_descs(dA, dG, dO)
    wsb = torch.empty(max(256, lutc.correct_image_workspace(desc)), dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream(device)
    st = ctypes.c_void_p(stream.cuda_stream)
    flags = LUTC_STRETCH if wl.stretch else 0
    pitch = out.stride(1) * out.element_size()

    def check(rc):
        if rc:
            raise RuntimeError("lutc_correct_image failed: %d" % rc)

    call = lambda: check(lib.lutc_correct_image(ctypes.byref(desc), cd, flags, ctypes.c_void_p(out.data_ptr()), pitch,
                                                ctypes.c_void_p(wsb.data_ptr()), wsb.numel(), st))

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(device)

    leg = fused_leg(lib, lutc, wl, raw, cd, out, wsb, device, args.steps, args.warmup, ws)
    ms, direct_ms = max_over_ranks([leg["ms"], leg["direct_ms"]], device)
    ms_step = ms / args.steps
    value = whole_job_rate(wl.pixels, ws, args.steps, ms)

    # keep this step's output for the parity check against the oracle below
    out_h.copy_(out)

    peak, peak_src = peaks()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic", "config": workload_config(wl)}
    bytes_per_px = 5 if wl.stretch else 4
    line["hbm_frac_step"] = wl.pixels * bytes_per_px / (ms_step * 1e-3) / 1e9 / peak
    line["timing"] = ("CUDA events around %d replays of a CUDA graph holding one lutc_correct_image step; "
                      "direct_calls: the same steps as C-ABI calls" % args.steps)
    line["direct_calls"] = {"value": wl.pixels * ws * args.steps / (direct_ms * 1e-3) / 1e9, "unit": UNIT,
                            "ms_per_step": direct_ms / args.steps}
    if leg["phases"]:
        line["roofline"], line["phases_ms"] = fused_roofline(wl, wl.name, leg["phases"], leg["path"], leg["clocks"],
                                                             peak, peak_src, n_sm)
    else:
        ach = wl.pixels * 4 / (ms_step * 1e-3) / 1e9
        line["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                            "traffic": ncu_traffic("pass2", wl.name), "kernel": "detector-only apply",
                            "kernel_family": {1: "tma", 2: "strip"}.get(leg["path"], "none"),
                            "peak_source": peak_src + " (copy bandwidth)", "alg_bytes_per_launch": 4 * wl.pixels}
    line["clocks"] = leg["clocks"]
    line["gpu_launches"] = (3 if wl.stretch else 1) * args.steps  # in the graph: pass 1, scan, pass 2
    status = ctypes.c_int(-1)
    lib.lutc_device_status(ctypes.byref(status), st)
    line["device_status"] = status.value

    # the plain per-call path with materialised tables, for comparison
    if wl.stretch and not args.no_plain:
        line["plain"] = run_plain(lutc, raw, dA, dG, dO, wl, device, stream, steps=max(3, min(args.steps, 20)))

    if args.no_e2e:
        del raw, out, wsb
        return finish_lutc(args, line, wl, rank, ws, raw_h, out_h, A, G, O, value)
    # end to end through the C ABI with HOST buffers: lutc_correct_image_host pipelines the pinned
    # host raster in, both passes and the result out (chunks of rows, copy engines both ways)
    e2e_steps = max(3, min(args.steps, 10))
    hdesc = lutc.Raster(raw_h.data_ptr(), raw_h.stride(1) * 2, wl.width, wl.height, wl.bands, wl.bits)
    hws = torch.empty(max(256, lib.lutc_correct_image_host_workspace(ctypes.byref(hdesc), flags)), dtype=torch.uint8,
                      device=device)
    hcall = lambda: lib.lutc_correct_image_host(ctypes.byref(hdesc), cd, flags, ctypes.c_void_p(out_h.data_ptr()),
                                                out_h.stride(1) * out_h.element_size(), ctypes.c_void_p(hws.data_ptr()),
                                                hws.numel(), st)
    # the same steps as one frame sequence (lutc_correct_frames_host): step k + 1's copies in overlap
    # step k's pass 2 and copies out (two workspace halves); each step reads its pinned raster and
    # writes its pinned result
    outs_h = [out_h, torch.empty_like(out_h).pin_memory()]
    fws = torch.empty(max(256, lib.lutc_correct_frames_host_workspace(ctypes.byref(hdesc), flags, e2e_steps)),
                      dtype=torch.uint8, device=device)
    fin = (ctypes.c_void_p * e2e_steps)(*([raw_h.data_ptr()] * e2e_steps))
    fout = (ctypes.c_void_p * e2e_steps)(*[outs_h[k % 2].data_ptr() for k in range(e2e_steps)])
    fcall = lambda: lib.lutc_correct_frames_host(ctypes.byref(hdesc), fin, e2e_steps, cd, flags, fout,
                                                 out_h.stride(1) * out_h.element_size(),
                                                 ctypes.c_void_p(fws.data_ptr()), fws.numel(), st)

    def single_steps():
        for _ in range(e2e_steps):
            check(hcall())

    def frame_steps():
        check(fcall())

    def copy_steps():  # separate whole-raster copies around the device call (no overlap), for comparison
        for _ in range(e2e_steps):
            raw.copy_(raw_h, non_blocking=True)
            check(call())
            out_h.copy_(out, non_blocking=True)

    check(hcall())
    check(fcall())
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # every variant timed E2E_REPEATS times, interleaved, and the median kept: the host link and host
    # memory are shared with the machine's other work, and one slow window must not decide a number
    samples = {"frames": [], "single": [], "copies": []}
    for _ in range(E2E_REPEATS):
        for name, fn in (("frames", frame_steps), ("single", single_steps), ("copies", copy_steps)):
            e0.record(stream)
            fn()
            e1.record(stream)
            barrier()
            samples[name].append(e0.elapsed_time(e1))
    ems, ems_single, sms = (statistics.median(samples[k]) for k in ("frames", "single", "copies"))
    # each host-path variant once more into cleared buffers, against the device path's result
    ref_out = out.cpu()
    out_h.zero_()
    outs_h[1].zero_()
    frame_steps()
    barrier()
    host_same = bool(torch.equal(outs_h[0], ref_out)) and bool(torch.equal(outs_h[1], ref_out))
    out_h.zero_()
    single_steps()
    barrier()
    host_same = host_same and bool(torch.equal(out_h, ref_out))
    ems, ems_single, sms = max_over_ranks([ems, ems_single, sms], device)
    line["e2e"] = {"value": wl.pixels * ws * e2e_steps / (ems * 1e-3) / 1e9, "unit": UNIT,
                   "h2d_bytes_per_step": raw_h.numel() * raw_h.element_size(),
                   "d2h_bytes_per_step": out_h.numel() * out_h.element_size(), "steps": e2e_steps,
                   "path": "lutc_correct_frames_host over the steps: each step's pinned raster in and result out, "
                           "chunked copies overlapped with both passes and with the neighbouring steps",
                   "host_GBs": (raw_h.numel() * 2 + out_h.numel() * out_h.element_size()) * e2e_steps / (ems * 1e-3)
                   / 1e9,
                   "output_equals_device_path": host_same,
                   "timing": "median of %d interleaved runs of each variant" % E2E_REPEATS,
                   "samples_gpx_s": [round(wl.pixels * ws * e2e_steps / (t * 1e-3) / 1e9, 1) for t in samples["frames"]],
                   "single_calls": {"value": wl.pixels * ws * e2e_steps / (ems_single * 1e-3) / 1e9, "unit": UNIT,
                                    "path": "one lutc_correct_image_host call per step",
                                    "samples_gpx_s": [round(wl.pixels * ws * e2e_steps / (t * 1e-3) / 1e9, 1)
                                                      for t in samples["single"]]},
                   "serial_copies": {"value": wl.pixels * ws * e2e_steps / (sms * 1e-3) / 1e9, "unit": UNIT,
                                     "path": "whole-raster copy in, lutc_correct_image, whole-raster copy out",
                                     "samples_gpx_s": [round(wl.pixels * ws * e2e_steps / (t * 1e-3) / 1e9, 1)
                                                       for t in samples["copies"]]}}

    # the device buffers of this leg are not needed by what follows (large14, the batch)
    del raw, out, wsb, hws, fws, outs_h
    gc.collect()
    torch.cuda.empty_cache()
    return finish_lutc(args, line, wl, rank, ws, raw_h, out_h, A, G, O, value)


def finish_lutc(args, line, wl, rank, ws, raw_h, out_h, A, G, O, value):
    """Oracle parity and CPU baseline, the sub-objects of the default line, and the line itself."""
    import torch
    import torch.distributed as dist
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], line["parity"] = cpu_baseline(wl, raw_h.numpy(), A, G, O, out_h.numpy())
    if ws > 1:
        dist.destroy_process_group()
    if rank == 0 and ws == 1 and wl.name == "scene" and not args.quick and not (args.height or args.width):
        # the metric also names the batched and the served paths: summaries of both
        import copy
        sub = copy.copy(args)
        sub._return = True
        sub.steps, sub.warmup, sub.no_tune, sub.batch_images = 20, 3, False, 256
        del raw_h, out_h
        gc.collect()
        torch.cuda.empty_cache()
        # the large 14-bit scene on the same kernels, timed and checked against the oracle in full
        line["large14"] = run_large14(sub)
        line["tiny"] = run_tiny(sub)
        gc.collect()
        torch.cuda.empty_cache()
        b = run_batch(sub)
        line["batched"] = {"value": b["value"], "unit": UNIT, "ms_per_step": b["ms_per_step"],
                           "images": b["config"]["images"], "pixels_per_step": b["config"]["pixels_per_step"],
                           "hbm_frac_step": b["hbm_frac_step"], "vs_fused_single": b["value"] / value,
                           "sequential_calls": b["sequential_calls"]["value"], "autotuned": b["config"]["autotuned"],
                           "parity": b.get("parity"), "phases_ms": b["phases_ms"], "roofline": b["roofline"],
                           "clocks": b["clocks"], "cpu_baseline": b.get("cpu_baseline")}
        gc.collect()
        torch.cuda.empty_cache()
        v = serve_in_child(args, value)
        line["served"] = served_summary(v, value)
        line["fit"] = run_fit(sub)
        line["demosaic"] = run_demosaic(sub)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_large14(args):
    """The large 14-bit scene (3 x 24000 x 24000, dead columns, saturated pixels) on the fused path:
    graph-timed steps, phases, both passes against HBM and the shared-memory pipe, clocks during its
    own timed region, and every output pixel against the oracle (all host threads)."""
    import torch
    import synth
    import paper_1505_05655_gb300 as lutc

    wl = synth.WORKLOADS["large14"]
    device = torch.device("cuda", torch.cuda.current_device())
    lib = lutc.lib()
    n_sm = torch.cuda.get_device_properties(device).multi_processor_count
    t = time.perf_counter()
    raw_np, A, G, O = gen_inputs(wl, 0)
    gen_s = time.perf_counter() - t
    raw = torch.from_numpy(raw_np).to(device)
    dA, dG, dO = (torch.from_numpy(a).to(device) for a in (A, G, O))
    out = torch.empty(raw.shape, dtype=torch.uint8, device=device)
    desc = lutc.raster_desc(raw, wl.bits)
    cd = lutc.coeff_descs(dA, dG, dO)
    wsb = torch.empty(max(256, lutc.correct_image_workspace(desc)), dtype=torch.uint8, device=device)
    steps = max(20, args.steps)
    leg = fused_leg(lib, lutc, wl, raw, cd, out, wsb, device, steps, 3)
    ms_step = leg["ms"] / steps
    peak, peak_src = peaks()
    roof, ph = fused_roofline(wl, wl.name, leg["phases"], leg["path"], leg["clocks"], peak, peak_src, n_sm)
    res = {"config": workload_config(wl), "steps": steps, "ms_per_step": ms_step,
           "value": wl.pixels / (ms_step * 1e-3) / 1e9, "unit": UNIT,
           "hbm_frac_step": wl.pixels * 5 / (ms_step * 1e-3) / 1e9 / peak,
           "direct_calls": {"value": wl.pixels * steps / (leg["direct_ms"] * 1e-3) / 1e9,
                            "ms_per_step": leg["direct_ms"] / steps},
           "phases_ms": ph, "roofline": roof, "clocks": leg["clocks"],
           "timing": "CUDA events around %d replays of a CUDA graph holding one step; inputs larger than L2" % steps}
    if not args.no_cpu_baseline:
        got = out.cpu().numpy()
        threads = max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1))
        t = time.perf_counter()
        ref = cpu_baseline_threads(wl, raw_np, A, G, O, threads)
        dt = time.perf_counter() - t
        res["parity"] = {"bit_exact_vs_oracle": bool(np.array_equal(ref, got)), "pixels_compared": int(ref.size)}
        res["cpu_baseline"] = {"value": wl.pixels / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": "the whole large14 workload on %d threads, %.1f s (inputs generated in "
                                         "%.1f s)" % (threads, dt, gen_s)}
    del raw, out, wsb
    return res


def run_tiny(args):
    """The tiny detector-only configuration (1 x 1024 x 1024, 12-bit, uint16 out): graph-timed steps and
    the output against the oracle."""
    import torch
    import synth
    import paper_1505_05655_gb300 as lutc
    import oracle

    wl = synth.WORKLOADS["tiny"]
    device = torch.device("cuda", torch.cuda.current_device())
    lib = lutc.lib()
    raw_np, A, G, O = gen_inputs(wl, 0)
    raw = torch.from_numpy(raw_np).to(device)
    dA, dG, dO = (torch.from_numpy(a).to(device) for a in (A, G, O))
    out = torch.empty(raw.shape, dtype=torch.uint16, device=device)
    desc = lutc.raster_desc(raw, wl.bits)
    cd = lutc.coeff_descs(dA, dG, dO)
    wsb = torch.empty(256, dtype=torch.uint8, device=device)
    steps = 2000
    leg = fused_leg(lib, lutc, wl, raw, cd, out, wsb, device, steps, 10)
    ms_step = leg["ms"] / steps
    # a stream of such frames: a graph of `per_graph` calls, each a whole step, replayed `reps` times
    from paper_1505_05655_gb300._lib import LUTC_STRETCH
    per_graph, reps = 20, 100
    stream = torch.cuda.current_stream(device)
    pitch = out.stride(1) * out.element_size()

    def call(s):
        rc = lib.lutc_correct_image(ctypes.byref(desc), cd, LUTC_STRETCH if wl.stretch else 0,
                                    ctypes.c_void_p(out.data_ptr()), pitch, ctypes.c_void_p(wsb.data_ptr()), wsb.numel(),
                                    ctypes.c_void_p(s.cuda_stream))
        if rc:
            raise RuntimeError("lutc_correct_image failed: %d" % rc)

    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for _ in range(per_graph):
            call(torch.cuda.current_stream(device))
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize(device)
    us_call = e0.elapsed_time(e1) * 1e3 / (reps * per_graph)
    res = {"config": workload_config(wl), "steps": reps * per_graph, "us_per_step": us_call,
           "value": wl.pixels / (us_call * 1e-6) / 1e9, "unit": UNIT,
           "kernel_family": {1: "tma", 2: "strip"}.get(leg["path"], "none"),
           "timing": "CUDA events around %d replays of a CUDA graph holding %d calls, each a whole step; 4 MB in "
                     "and out, inside L2 (launch-bound: reported, not held against the HBM roofline)" % (reps, per_graph),
           "one_call_graph": {"us_per_step": ms_step * 1e3, "steps": steps,
                              "timing": "CUDA events around %d replays of a CUDA graph holding one call (mostly "
                                        "the graph launch)" % steps}}
    if not args.no_cpu_baseline:
        ref = oracle.correct_image(raw_np, A, G, O, wl.bits, stretch=False)
        res["parity"] = {"bit_exact_vs_oracle": bool(np.array_equal(ref, out.cpu().numpy())),
                         "pixels_compared": int(ref.size)}
    return res


def served_summary(v, fused_value: float) -> dict:
    """The bench line's summary of the serving run (`--workload serve`)."""
    keep = ("p50_ms", "p99_ms", "gpx_s", "req_s", "offered_req_s", "mean_batch", "requests", "failed", "tail",
            "cache_misses")
    sat = v["saturation"]
    return {"saturation_gpx_s": sat["gpx_s"], "vs_fused_single": sat["gpx_s"] / fused_value,
            "saturation": {k: sat.get(k) for k in keep},
            "latency_ms": {r: {k: d.get(k) for k in keep} for r, d in v["latency"].items()},
            "outputs_equal_single_calls": v["outputs_equal_single_calls"],
            "host_requests": {"saturation_gpx_s": v["host_requests"]["saturation"]["gpx_s"],
                              "saturation": {k: v["host_requests"]["saturation"].get(k) for k in keep},
                              "latency_200": {k: v["host_requests"]["latency_200"].get(k) for k in keep},
                              "outputs_equal_single_calls": v["host_requests"]["outputs_equal_single_calls"]},
            "first_requests": {k: v["warmup_with_cache_misses"].get(k) for k in keep},
            "load_generator": v["config"].get("load_generator"), "config": v["config"]["workload"]}


def run_plain(lutc, raw, dA, dG, dO, wl, device, stream, steps):
    """lutgen -> hist -> stretch -> compose -> apply_u8 as separate calls, tables materialised."""
    import torch
    L = 1 << wl.bits
    lut = torch.empty((wl.bands, wl.width, L), dtype=torch.uint16, device=device)
    clut = torch.empty((wl.bands, wl.width, L), dtype=torch.uint8, device=device)
    hist = torch.empty((wl.bands, L), dtype=torch.uint64, device=device)
    S = torch.empty((wl.bands, L), dtype=torch.uint8, device=device)
    lohi = torch.empty((wl.bands, 2), dtype=torch.int32, device=device)
    out = torch.empty(raw.shape, dtype=torch.uint8, device=device)

    def step():
        for b in range(wl.bands):
            lutc.lutgen(dA[b], dG[b], dO[b], wl.bits, out=lut[b], stream=stream)
        lutc.hist(raw, dA, dG, dO, wl.bits, out=hist, stream=stream)
        lutc.stretch(hist, wl.bits, S=S, lohi=lohi, stream=stream)
        for b in range(wl.bands):
            lutc.compose(lut[b], S[b], wl.bits, out=clut[b], stream=stream)
        lutc.apply_u8(raw, clut, wl.bits, out=out, stream=stream)

    for _ in range(3):
        step()
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(device)
    ms = e0.elapsed_time(e1) / steps
    return {"value": wl.pixels / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "path": "lutgen, hist, stretch, compose, apply_u8 as separate calls (%d launches)" % (2 * wl.bands + 3)}


def cpu_baseline_threads(wl, raw, A, G, O, threads: int):
    """The oracle's steps on all host cores: row ranges for hist and apply (per-thread histograms
    summed), column ranges for lutgen and compose.  ctypes releases the GIL inside each oracle call."""
    import concurrent.futures as cf
    import oracle
    bands, H, W = raw.shape
    rows = [(r * H // threads, (r + 1) * H // threads) for r in range(threads)]
    cols = [(c * W // threads, (c + 1) * W // threads) for c in range(threads)]
    out = np.empty((bands, H, W), np.uint8 if wl.stretch else np.uint16)
    with cf.ThreadPoolExecutor(threads) as ex:
        for b in range(bands):
            D = np.concatenate(list(ex.map(lambda c: oracle.lutgen(A[b, c[0]:c[1]], G[b, c[0]:c[1]],
                                                                   O[b, c[0]:c[1]], wl.bits), cols)))
            if not wl.stretch:
                list(ex.map(lambda r: out[b, r[0]:r[1]].__setitem__(
                    slice(None), oracle.apply_u16(raw[b, r[0]:r[1]], D, wl.bits)), rows))
                continue
            h = sum(ex.map(lambda r: oracle.hist(raw[b, r[0]:r[1]], D, wl.bits), rows))
            S = oracle.stretch(h, wl.bits)[0]
            C = np.concatenate(list(ex.map(lambda c: oracle.compose(D[c[0]:c[1]], S, wl.bits), cols)))
            list(ex.map(lambda r: out[b, r[0]:r[1]].__setitem__(
                slice(None), oracle.apply_u8(raw[b, r[0]:r[1]], C, wl.bits)), rows))
    return out


def cpu_baseline(wl, raw, A, G, O, gpu_out):
    """The oracle on the same host raster, on all host cores and on one; also checks the GPU result bit for bit."""
    import oracle
    threads = max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1))
    t = time.perf_counter()
    ref_mt = cpu_baseline_threads(wl, raw, A, G, O, threads)
    dt_mt = time.perf_counter() - t
    t = time.perf_counter()
    ref = oracle.correct_image(raw, A, G, O, wl.bits, stretch=wl.stretch)
    dt = time.perf_counter() - t
    base = {"value": wl.pixels / dt_mt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "the whole %s workload (%d px): the oracle's steps (lutgen, hist, stretch, compose, apply) "
                      "on %d threads, row ranges with per-thread histograms summed, %.2f s"
                      % (wl.name, wl.pixels, threads, dt_mt),
            "single_core": {"value": wl.pixels / dt / 1e9, "unit": UNIT, "cores": 1,
                            "sample": "oracle correct_image, single-threaded C, %.1f s" % dt}}
    same = bool(np.array_equal(ref, gpu_out)) and bool(np.array_equal(ref_mt, gpu_out))
    return base, {"bit_exact_vs_oracle": same, "pixels_compared": int(ref.size)}


def run_batch(args):
    """The 256-image mixed batch: one autotuned persistent launch per phase, replayed from a CUDA graph."""
    import torch
    import oracle
    import synth
    import paper_1505_05655_gb300 as lutc

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    align = args.row_align  # bytes; rows of every input (uint16) and output (uint8) padded to a multiple
    ims = synth.batch_images(synth.BATCH_SEED + 7 * rank, n=args.batch_images, pitch_multiple=align // 2)
    pixels = sum(im["bands"] * im["height"] * im["width"] for im in ims)
    host_in = [torch.from_numpy(im["raw"]).pin_memory() for im in ims]
    dev_in = [h.to(device) for h in host_in]
    images = []
    for im, d in zip(ims, dev_in):
        A, G, O = (torch.from_numpy(a).to(device) for a in (im["A"], im["G"], im["O"]))
        # output rows padded like the input rows, so every row takes vector stores
        opitch = -(-im["width"] // align) * align
        out = torch.empty((im["bands"], im["height"], opitch), dtype=torch.uint8, device=device)[:, :, :im["width"]]
        images.append((d[:, :, :im["width"]], A, G, O, im["bits"], out, True))
    stream = torch.cuda.current_stream(device)
    if args.no_tune:
        from paper_1505_05655_gb300._lib import BatchConfig
        cfg, tune_ms = BatchConfig(0, 0, 1), None
    else:
        cfg, tune_ms = lutc.batch_autotune(images, reps=3)
    batch = lutc.Batch(images, config=cfg)

    def timed(fn, steps):
        torch.cuda.synchronize(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(device)
        return e0.elapsed_time(e1) / steps

    for _ in range(max(3, args.warmup)):
        batch.run()
    sampler = ClockSampler(None)
    wall0 = time.time()
    ms = timed(batch.run, args.steps)
    wall1 = time.time()
    clocks = sampler.stop(wall0, wall1)
    value = pixels / (ms * 1e-3) / 1e9

    # phase times from traced runs of the same batch without the graph
    nograph = lutc.Batch(images, column_threads=cfg.column_threads, blocks_per_sm=cfg.blocks_per_sm,
                         use_graph=False)
    nograph.run()
    k = max(3, min(args.steps, 20))
    lutc.trace_enable(k)
    timed(nograph.run, k)
    phases = lutc.trace_read(k)
    lutc.trace_enable(0)
    nograph.close()
    avg = [statistics.fmean(p[i] for p in phases) for i in range(3)]
    alg = [2 * pixels, 0, 3 * pixels]
    dom = 0 if avg[0] > avg[2] else 2
    peak, peak_src = peaks()
    ach = alg[dom] / (avg[dom] * 1e-3) / 1e9

    def sequential():
        for (raw, A, G, O, bits, out, _) in images:
            lutc.correct_image(raw, A, G, O, bits, out=out)

    seq_ms = timed(sequential, 3)

    def e2e():
        for h, d in zip(host_in, dev_in):
            d.copy_(h, non_blocking=True)
        batch.run()
        for h, t in zip(out_host, images):
            h.copy_(t[5], non_blocking=True)

    out_host = [torch.empty(t[5].shape, dtype=torch.uint8, pin_memory=True) for t in images]
    # (the device outputs are row-pitched views; their D2H copies go through torch's strided copy)
    e2e_ms = timed(e2e, 3)

    # kernels one batch step launches (every image here takes the TMA kernels): the reset of histograms
    # and runs, pass 1 split into the images of <= 12 bits and the deeper ones, the scan, pass 2
    batch_launches = 1 + int(any(im["bits"] <= 12 for im in ims)) + int(any(im["bits"] > 12 for im in ims)) + 2
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "batch: %d images, W log-uniform 512-8192, H log-uniform 256-8192, bits "
                                   "{10,12,14}, bands {1,3,4}, full pipeline, uint8 out" % len(ims),
                       "images": len(ims), "pixels_per_step": pixels, "row_align_bytes": align,
                       "l2": "inputs larger than L2 (%.2f GB read per step)" % (2 * pixels / 1e9),
                       "autotuned": {"column_threads": cfg.column_threads, "blocks_per_sm": cfg.blocks_per_sm,
                                     "graph": True, "tuning_ms": tune_ms}},
            "hbm_frac_step": 5 * pixels / (ms * 1e-3) / 1e9 / peak,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "traffic": ncu_traffic(["pass1", "", "pass2"][dom],
                                                "batch" if align == 16 else "batch/align%d" % align, pixels),
                         "kernel": ["pass1 k_tma_strip<hist, batch>", "", "pass2 k_tma_strip<apply, batch>"][dom],
                         "peak_source": peak_src + " (copy bandwidth)", "alg_bytes_per_launch": alg[dom]},
            "phases_ms": {"pass1_hist": avg[0], "scan": avg[1], "pass2_apply": avg[2]},
            "sequential_calls": {"value": pixels / (seq_ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": seq_ms,
                                 "path": "%d lutc_correct_image calls, one per image" % len(ims)},
            "clocks": clocks, "gpu_launches": batch_launches * args.steps,
            "e2e": {"value": pixels / (e2e_ms * 1e-3) / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": sum(h.numel() * 2 for h in host_in),
                    "d2h_bytes_per_step": sum(h.numel() for h in out_host), "steps": 3}}
    tr = line["roofline"]["traffic"]
    line["roofline"]["traffic_GBs"] = tr / (avg[dom] * 1e-3) / 1e9 if tr else None
    n_sm = torch.cuda.get_device_properties(device).multi_processor_count
    key = "batch" if align == 16 else "batch/align%d" % align
    mhz = clocks["sm_mhz"] if clocks else None
    line["roofline"]["smem_pipe"] = {"pass1": smem_pipe(key, "pass1", pixels, avg[0], mhz, n_sm),
                                     "pass2": smem_pipe(key, "pass2", pixels, avg[2], mhz, n_sm)}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # every image against the oracle, one image per host thread at a time
        import concurrent.futures as cf
        threads = max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1))
        got = [t[5].cpu().numpy() for t in images]

        def same_as_oracle(i):
            im = ims[i]
            ref = oracle.correct_image(im["raw"][:, :, :im["width"]], im["A"], im["G"], im["O"], im["bits"])
            return bool(np.array_equal(ref, got[i])), ref.size

        t = time.perf_counter()
        with cf.ThreadPoolExecutor(threads) as ex:
            res = list(ex.map(same_as_oracle, range(len(ims))))
        dt = time.perf_counter() - t
        px = sum(n for _, n in res)
        line["cpu_baseline"] = {"value": px / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": "every image of the batch (%d px), the oracle's correct_image, one image "
                                          "per thread on %d threads, %.1f s" % (px, threads, dt)}
        line["parity"] = {"bit_exact_vs_oracle": all(ok for ok, _ in res), "pixels_compared": px,
                          "images_compared": len(res)}
        del got
    batch.close()
    if getattr(args, "_return", False):
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_serve(args):
    """Open-loop Poisson loads on the request loop, driven by the library's native replay thread
    (lutc_server_replay): p50/p99 latency per load, saturation throughput and its latency, loads at
    fractions of the saturated request rate, and host-memory requests."""
    import torch
    import synth
    import paper_1505_05655_gb300 as lutc

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    nsens = synth.SERVE_SENSORS
    w, _, bits, bands = synth.batch_spec(synth.SERVE_SEED, nsens)
    pool_per_sensor = 4
    server = lutc.Server(budget_bytes=40 << 30, max_batch=32, max_wait_us=2000, streams=4)
    pool = []  # (sensor, raster on device, output on device, pixels)
    pool_host = []  # (sensor, raster in pinned host memory, output in pinned host memory, pixels, keep, keep)
    for sid in range(nsens):
        W, B, Bt = int(w[sid]), int(bands[sid]), int(bits[sid])
        A, G, O = synth.coeff_set(synth.batch_image_seed(synth.SERVE_SEED, sid), B, W)
        server.register_sensor(sid, W, B, Bt, A, G, O)
        _, hs, _, _ = synth.batch_spec(synth.SERVE_SEED + 1 + sid, pool_per_sensor)
        for k in range(pool_per_sensor):
            H = int(hs[k])
            # rows padded to args.row_align bytes (at least the TMA path's 16), bands stacked at H x pitch
            pitch = -(-W // (args.row_align // 2)) * (args.row_align // 2)
            host = np.zeros((B, H, pitch), np.uint16)
            synth.raster(synth.batch_image_seed(synth.SERVE_SEED + 100 + sid, k), B, H, W, Bt, out=host[:, :, :W])
            raw = torch.from_numpy(host).to(device)[:, :, :W]
            opitch = -(-W // args.row_align) * args.row_align
            out = torch.empty((B, H, opitch), dtype=torch.uint8, device=device)[:, :, :W]
            pool.append((sid, raw, out, B * H * W))
            if (sid * pool_per_sensor + k) % 16 == 0:
                # every 16th raster also from pinned host memory (the server stages it in and out); a small
                # set of reused host buffers, like a receiver's: a 10 GB page-locked working set slows
                # every host access down (address translation), whichever engine copies
                raw_h = torch.from_numpy(host).pin_memory()
                out_h = torch.empty((B, H, opitch), dtype=torch.uint8).pin_memory()
                pool_host.append((sid, raw_h[:, :, :W].numpy(), out_h[:, :, :W].numpy(), B * H * W, raw_h, out_h))
    rng = np.random.default_rng(synth.SERVE_SEED)
    used_dev, used_host = set(), set()
    mean_px = float(np.mean([p[3] for p in pool]))

    def drive(rate, n, closed=False, host=False):
        gc.collect()  # nothing of the earlier loads is left for the collector to find during this one
        used = used_host if host else used_dev
        src = pool_host if host else pool
        picks = rng.integers(0, len(src), n)
        at = np.zeros(n) if closed else np.cumsum(rng.exponential(1.0 / rate, n))
        r = server.replay([(float(at[i]), src[j][0], src[j][1], src[j][2], host) for i, j in enumerate(picks)])
        used.update(int(j) for j in picks)
        # closed burst: latency from each request's own submission; open loop: from its scheduled arrival,
        # so any lateness of the hand-over (submit_lag) counts against the request
        t_from = r["submit_s"] if closed else r["scheduled_s"]
        lat = r["done_s"] - t_from
        px = sum(src[j][3] for j in picks)
        span = r["done_s"].max() - r["submit_s"].min()
        prep = r["launched_s"] - r["start_s"]
        run = r["done_s"] - r["launched_s"]
        lag = r["submit_s"] - r["scheduled_s"]
        # where the slowest 1 % spent their time: late hand-over by the load generator, the batch window
        # and admission (submit -> start), batch preparation (start -> launched), the device
        p99 = float(np.percentile(lat, 99))
        slow = lat >= p99
        stage = lambda xs: round(float(np.median(xs)) * 1e3, 3)
        tail = dict(requests=int(slow.sum()), max_ms=round(float(lat.max()) * 1e3, 3),
                    submit_lag_ms=0.0 if closed else stage(lag[slow]),
                    submit_lag_max_ms=0.0 if closed else round(float(lag.max()) * 1e3, 3),
                    queue_ms=stage((r["start_s"] - r["submit_s"])[slow]), prep_ms=stage(prep[slow]),
                    launch_to_done_ms=stage(run[slow]), cache_misses=int(r["cache_miss"][slow].sum()))
        miss = r["cache_miss"] == 1  # requests that uploaded their sensor's coefficients
        misses = dict(requests=int(miss.sum()),
                      p50_ms=float(np.percentile(lat[miss], 50) * 1e3) if miss.any() else None,
                      max_ms=float(lat[miss].max() * 1e3) if miss.any() else None)
        return dict(p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=p99 * 1e3, gpx_s=px / span / 1e9,
                    cache_misses=misses,
                    req_s=n / span, offered_req_s=None if closed else rate,
                    offered_gpx_s=None if closed else mean_px * rate / 1e9,
                    mean_batch=float(np.mean(r["batch_size"])), requests=n, failed=int((r["status"] != 0).sum()),
                    batch_prep_ms=float(np.median(prep) * 1e3), launch_to_done_ms=float(np.median(run) * 1e3),
                    latency_from="submission" if closed else "scheduled arrival", tail=tail)

    warm = drive(400, 200)  # first requests of every sensor upload its coefficients
    sat = drive(0, max(2000, 2 * args.steps), closed=True)
    loads = {}
    # the configured open-loop loads, at least 2000 requests each (40 s at 50 req/s)
    # (`--cases` keeps only the loads whose names contain one of its words; saturation always runs)
    for rate, n in ((50, max(2000, args.steps // 4)), (200, max(2000, args.steps)), (800, max(2000, 2 * args.steps))):
        if _selected(args, str(rate)):
            loads[str(rate)] = drive(rate, n)
    # loads high enough to batch for real: fractions of the saturated request rate, ~1 s each
    for frac in (0.25, 0.5, 0.75, 0.9):
        rate, name = frac * sat["req_s"], "%d%% of saturation" % round(100 * frac)
        if _selected(args, name):
            loads[name] = drive(rate, int(max(2000, min(60000, rate))))
    # the metric's own target: an offered load of 80 % of the fused single-scene rate, when it is known
    if args.fused_gpx and _selected(args, "80% of the fused scene"):
        rate = 0.8 * args.fused_gpx * 1e9 / mean_px
        loads["80% of the fused scene"] = drive(rate, int(max(2000, min(60000, rate))))
    # requests from pinned host memory: staged in and out by the server (copies inside each request's latency)
    empty = dict(p50_ms=None, p99_ms=None, gpx_s=None, tail=None)
    host = _selected(args, "host")
    host_sat = drive(0, max(300, args.steps), closed=True, host=True) if host else empty
    host_200 = drive(200, max(300, args.steps // 2), host=True) if host else empty
    host_exact = True
    for k in sorted(used_host)[::9]:  # entries some request wrote
        sid, raw_np, out_np = pool_host[k][:3]
        b = raw_np.shape[0]
        A, G, O = synth.coeff_set(synth.batch_image_seed(synth.SERVE_SEED, sid), b, raw_np.shape[2])
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        ref = lutc.correct_image(d(raw_np), d(A), d(G), d(O), int(bits[sid])).cpu().numpy()
        host_exact = host_exact and bool(np.array_equal(ref, out_np))
    # each pool raster's output must equal a single call on it
    exact = True
    for k in sorted(used_dev)[::9]:
        sid, raw, out, _ = pool[k]
        b = raw.shape[0]
        A, G, O = synth.coeff_set(synth.batch_image_seed(synth.SERVE_SEED, sid), b, raw.shape[2])
        d = lambda a: torch.from_numpy(a).to(device)
        exact = exact and bool(torch.equal(lutc.correct_image(raw, d(A), d(G), d(O), int(bits[sid])), out))
    st = server.stats()
    server.close()
    line = {"metric": METRIC, "value": sat["gpx_s"], "unit": UNIT, "n_gpus": ws, "steps": sat["requests"],
            "warmup": warm["requests"], "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "serve: %d sensors from the batch mixture, %d pool rasters each, device-resident; "
                                   "Poisson arrivals 50/200/800 req/s, 25/50/75/90 %% of the saturated request "
                                   "rate and 80 %% of the fused single-scene rate; budget 40 GiB; a request launches at once on an idle device, else batches "
                                   "<= 32 requests or 2 ms, 4 streams" % (nsens, pool_per_sensor),
                       "row_align_bytes": args.row_align, "mean_request_px": mean_px,
                       "load_generator": "lutc_server_replay: arrival times drawn up front, submitted on schedule "
                                         "by a native thread, collected by the calling thread",
                       "l2": "inputs larger than L2 (pool %.1f GB)" % (sum(p_[3] for p_ in pool) * 2 / 1e9)},
            "latency": loads, "saturation": sat, "warmup_with_cache_misses": warm, "server": st,
            "outputs_equal_single_calls": exact,
            "host_requests": {"saturation": host_sat, "latency_200": host_200, "outputs_equal_single_calls": host_exact,
                              "path": "LUTC_REQ_HOST: rasters and outputs in pinned host memory (16 reused buffers), staged by "
                                      "the server with SM-driven row copies"}}
    if getattr(args, "_return", False):
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)


def serve_in_child(args, fused_gpx: float | None = None):
    """The serving summary from a fresh process (`--workload serve`): its latency tails measure the
    server, not the many GB this process has allocated and freed by then."""
    cmd = [sys.executable, os.path.abspath(__file__), "--workload", "serve", "--steps", "1000",
           "--row-align", str(args.row_align)] + (["--fused-gpx", "%.3f" % fused_gpx] if fused_gpx else [])
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "LOCAL_WORLD_SIZE")}
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=ROOT, timeout=900)
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    if r.returncode != 0 or not lines:
        raise RuntimeError("serving run failed (%d): %s" % (r.returncode, (r.stderr or r.stdout)[-2000:]))
    return json.loads(lines[-1])


def _selected(args, name: str) -> bool:
    words = [w.replace("_", " ") for w in getattr(args, "cases", "").split(",") if w]
    return not words or any(w in name for w in words)


def fp64_peak_tflops(device) -> tuple[float, str]:
    """fp64 FMA-pipe peak derived from the unit count: SMs x 2 fp64 FMA per clock x 2 flops x maximum SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz = 2070.0
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits",
                              "-i", str(device.index or 0)], capture_output=True, text=True, timeout=20).stdout
        mhz = float(out.strip().splitlines()[0])
    except Exception:
        pass
    return sms * 2 * 2 * mhz * 1e6 / 1e12, "%d SMs x 2 fp64 FMA/clk x 2 flop x %.0f MHz" % (sms, mhz)


def fp64_peak_measured(device) -> dict:
    """The fp64 FMA rate measured on this device: lutc_probe_fp64_fma (register-only FMA chains, 8 blocks
    of 256 threads per SM), timed with CUDA events over 5 launches after 2 warm-ups, clocks sampled."""
    import torch
    import paper_1505_05655_gb300 as lutc
    lib = lutc.lib()
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    stream = torch.cuda.current_stream(device)
    st = ctypes.c_void_p(stream.cuda_stream)
    blocks, iters = sms * 8, 1 << 14
    sink = torch.empty(blocks * 256, dtype=torch.float64, device=device)
    fmas = ctypes.c_longlong(0)
    launch = lambda: lutc.check(lib.lutc_probe_fp64_fma(blocks, iters, ctypes.c_void_p(sink.data_ptr()),
                                                        ctypes.byref(fmas), st), "lutc_probe_fp64_fma")
    for _ in range(2):
        launch()
    torch.cuda.synchronize(device)
    sampler = ClockSampler(None)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    wall0 = time.time()
    e0.record(stream)
    for _ in range(5):
        launch()
    e1.record(stream)
    torch.cuda.synchronize(device)
    wall1 = time.time()
    clocks = sampler.stop(wall0, wall1)
    ms = e0.elapsed_time(e1) / 5
    tflops = 2 * fmas.value / (ms * 1e-3) / 1e12
    mhz = clocks["sm_mhz"] if clocks else None
    return {"tflops": tflops, "ms_per_launch": ms, "fmas_per_launch": fmas.value, "clocks": clocks,
            "fma_per_sm_per_clock": fmas.value / (ms * 1e-3) / (sms * mhz * 1e6) if mhz else None,
            "how": "lutc_probe_fp64_fma: %d blocks x 256 threads x 8 chains x %d FMAs on registers" % (blocks, iters)}


def run_fit(args):
    """Per-detector least-squares fit: the paper's shape (6 lines x 6000 detectors) and a large calibration."""
    import torch
    import synth
    import paper_1505_05655_gb300 as lutc

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    stream = torch.cuda.current_stream(device)
    derived, derived_how = fp64_peak_tflops(device)
    probe = fp64_peak_measured(device)
    peak, peak_how = probe["tflops"], "measured: " + probe["how"]

    def timed(fn, steps):
        torch.cuda.synchronize(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(device)
        return e0.elapsed_time(e1) / steps

    shapes = {"paper": (6, 6000, 12), "large": (1024, 65536, 14)}
    res = {}
    for name, (n, ncols, bits) in shapes.items():
        if not _selected(args, name):
            continue
        x, y = synth.calib(synth.CALIB_SEED + rank, n, ncols, bits, dead_frac=0.01)
        xd, yd = torch.from_numpy(x).to(device), torch.from_numpy(y).to(device)
        per = {}
        for order in (1, 2, 3):
            coef = torch.empty((ncols, order + 1), dtype=torch.float64, device=device)
            st = torch.empty(ncols, dtype=torch.int32, device=device)
            call = lambda: lutc.fit(xd, yd, order, coef=coef, status=st, stream=stream)
            for _ in range(5):
                call()
            steps = 200 if name == "paper" else 20
            ms = timed(call, steps)
            # kernel time without host overhead: many calls captured in one graph, replayed
            per_graph = 100 if name == "paper" else 5
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                cs = torch.cuda.current_stream(device)
                for _ in range(per_graph):
                    lutc.fit(xd, yd, order, coef=coef, status=st, stream=cs)
            graph.replay()
            reps = 10 if name == "paper" else 4
            gms = timed(graph.replay, reps) / per_graph
            # fp64 work the method cannot avoid: the moments Q_j = sum x^j y (one multiply-add per j);
            # the power sums P_k are exact integer sums.  Issued fp64 instructions per sample: one
            # conversion of x, m - 1 products x^j, m + 1 moment updates.
            flops = n * ncols * 2 * (order + 1)
            issue = n * ncols * (2 * order + 1)
            per[str(order)] = {"us_per_kernel": gms * 1e3, "us_per_call_from_python": ms * 1e3,
                               "detectors_per_s": ncols / (gms * 1e-3),
                               "roofline": {"bound": "alu", "achieved": flops / (gms * 1e-3) / 1e12, "peak": peak,
                                            "unit": "TFLOP/s (fp64)", "frac": flops / (gms * 1e-3) / 1e12 / peak,
                                            "flops_per_sample": 2 * (order + 1), "peak_source": peak_how,
                                            "frac_of_derived_peak": flops / (gms * 1e-3) / 1e12 / derived,
                                            "fp64_issue_frac": issue / (gms * 1e-3) / 1e12 / (peak / 2)}}
            if name == "paper" and rank == 0 and not args.no_cpu_baseline:
                import oracle
                t = time.perf_counter()
                reps = 0
                while time.perf_counter() - t < 0.5:
                    rc, rs = oracle.polyfit(x, y, order)
                    reps += 1
                dt = (time.perf_counter() - t) / reps
                same_status = bool(np.array_equal(rs, st.cpu().numpy()))
                ok = rs == 0
                sc = float(1 << bits) ** np.arange(order + 1)
                rel = np.abs(coef.cpu().numpy()[ok] - rc[ok]) * sc / np.maximum(np.abs(rc[ok] * sc).max(axis=1,
                                                                                                    keepdims=True), 1)
                per[str(order)]["cpu_baseline"] = {"us_per_call": dt * 1e6, "cores": 1, "kind": "oracle",
                                                   "sample": "the whole %d x %d calibration" % (n, ncols)}
                per[str(order)]["parity"] = {"status_equal": same_status,
                                             "max_rel_diff_scaled_coef": float(rel.max()) if rel.size else 0.0}
        res[name] = {"lines": n, "detectors": ncols, "bits": bits, "orders": per,
                     "x_bytes": n * ncols * 2}
    res["fp64_peak"] = dict(probe, derived_tflops=derived, derived_how=derived_how)
    return res


def run_demosaic(args):
    """Bilinear demosaic: the paper's 2048 x 2048 16-bit frame, and a frame larger than L2, raw and
    fused with the detector correction."""
    import torch
    import synth
    import paper_1505_05655_gb300 as lutc

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    stream = torch.cuda.current_stream(device)
    peak, peak_src = peaks()

    def timed(fn, steps):
        torch.cuda.synchronize(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(device)
        return e0.elapsed_time(e1) / steps

    cases = [("paper 2048x2048 16-bit, raw", 2048, 2048, 16, False),
             ("paper 2048x2048 12-bit, fused detector correction", 2048, 2048, 12, True),
             ("large 16384x16384 16-bit, raw", 16384, 16384, 16, False),
             ("large 16384x16384 12-bit, fused detector correction", 16384, 16384, 12, True)]
    res = {}
    for name, h, w, bits, correct in cases:
        if not _selected(args, name):
            continue
        img = synth.raster(synth.CALIB_SEED + 7 + rank, 1, h, w, bits)[0]
        raw = torch.from_numpy(img).to(device)
        kw = {}
        if correct:
            A, G, O = synth.coeffs(synth.CALIB_SEED + 7 + rank, 0, w)
            kw = {k: torch.from_numpy(v).to(device) for k, v in (("A", A), ("G", G), ("O", O))}
        out = torch.empty((3, h, w), dtype=torch.uint16, device=device)
        call = lambda: lutc.demosaic(raw, "rggb", bits, out=out, stream=stream, **kw)
        for _ in range(3):
            call()
        per_graph = 50 if h <= 2048 else 5
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            cs = torch.cuda.current_stream(device)
            for _ in range(per_graph):
                lutc.demosaic(raw, "rggb", bits, out=out, stream=cs, **kw)
        graph.replay()
        ms = timed(graph.replay, 10) / per_graph
        px = h * w
        alg = 8 * px
        ach = alg / (ms * 1e-3) / 1e9
        entry = {"us_per_frame": ms * 1e3, "gpx_s": px / (ms * 1e-3) / 1e9,
                 "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                              "alg_bytes_per_px": 8, "peak_source": peak_src + " (copy bandwidth)"},
                 "l2": "frame %s L2 (%.0f MB in, %.0f MB out)" % ("inside" if 8 * px < 129e6 else "larger than",
                                                                  2 * px / 1e6, 6 * px / 1e6)}
        if h <= 2048 and rank == 0 and not args.no_cpu_baseline:
            import oracle
            lut = oracle.lutgen(A, G, O, bits) if correct else None
            t = time.perf_counter()
            ref = oracle.demosaic(img, "rggb", lut=lut, bits=bits)
            dt = time.perf_counter() - t
            entry["cpu_baseline"] = {"value": px / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                                     "sample": "the whole frame, single-threaded C oracle, %.2f s" % dt}
            entry["bit_exact_vs_oracle"] = bool(np.array_equal(ref, out.cpu().numpy()))
        res[name] = entry
        del raw, out, kw
        torch.cuda.empty_cache()
    return res


def main():
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="lutc", choices=["lutc", "reference"])
    ap.add_argument("--workload", default="scene", choices=sorted(synth.WORKLOADS) + ["batch", "serve", "fit", "demosaic"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--batch-images", type=int, default=256, help="images in the batch workload")
    ap.add_argument("--no-tune", action="store_true", help="batch workload: automatic configuration, no autotuner")
    ap.add_argument("--row-align", type=int, default=128, choices=[16, 32, 64, 128, 256, 512],
                    help="batch and serve workloads: bytes every image row is padded to (input and output)")
    ap.add_argument("--quick", action="store_true", help="scene line only (no batch and serving summaries)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffers) leg")
    ap.add_argument("--fused-gpx", type=float, default=0.0, help="serve workload: the fused single-scene rate "
                                                                 "(Gpixel/s); adds a load offered at 80 %% of it")
    ap.add_argument("--height", type=int, default=0, help="single-image workloads: rows per band instead of the "
                                                          "workload's (a smaller case of it, e.g. for a profile)")
    ap.add_argument("--width", type=int, default=0, help="single-image workloads: columns instead of the workload's")
    ap.add_argument("--cases", default="", help="fit / demosaic / serve workloads: run only the cases whose name contains "
                                                  "one of these comma-separated words ('_' stands for a space)")
    args = ap.parse_args()
    if args.workload == "batch" and args.impl != "reference":
        run_batch(args)
        return
    if args.workload == "serve" and args.impl != "reference":
        run_serve(args)
        return
    if args.workload == "demosaic" and args.impl != "reference":
        print(json.dumps({"workload": "demosaic", "demosaic": run_demosaic(args)}), flush=True)
        return
    if args.workload == "fit" and args.impl != "reference":
        print(json.dumps({"workload": "fit", "fit": run_fit(args)}), flush=True)
        return
    wl = synth.WORKLOADS[args.workload if args.workload in synth.WORKLOADS else "scene"]
    if args.height or args.width:
        import dataclasses
        wl = dataclasses.replace(wl, height=args.height or wl.height, width=args.width or wl.width)
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_lutc(args, wl)


if __name__ == "__main__":
    main()
