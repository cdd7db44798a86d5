"""Host-side pieces of bench.py (CPU only).

A stored ncu figure (DRAM bytes per launch, shared-memory pipe utilisation) is
reported only while the sources its kernels are built from are the ones it
was captured on; the key is a hash of their code with comments and layout
removed, so that editing a comment keeps the figure and editing code drops it.
"""
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_code_hash_ignores_comments_and_layout_but_not_code():
    src = open(os.path.join(ROOT, "paper_1505_05655_gb300", "csrc", "lutc_tma.cu")).read()
    base = bench._code_only(src)
    commented = src.replace("namespace lutc {", "// a new comment line\nnamespace lutc {  /* and a block */", 1)
    reflowed = src.replace("constexpr int kConsumers = 256;", "constexpr  int   kConsumers =\n  256;", 1)
    assert bench._code_only(commented) == base
    assert bench._code_only(reflowed) == base
    assert bench._code_only(src.replace("constexpr int kConsumers = 256;", "constexpr int kConsumers = 128;", 1)) != base
    # preprocessor lines stay lines: joining a define with the next statement would change the code
    assert bench._code_only("#define A 1\nint x;") != bench._code_only("#define A 1 int x;")



def test_smem_pipe_floor_scales_a_capture_and_drops_a_stale_one(monkeypatch):
    # the floor is the captured wavefronts (per pixel, scaled to the launch) at one per SM clock on
    # every SM; a capture of other sources gives nothing
    entry = {"smem_wavefronts": 78.4e6, "smem_captured_pixels": 576e6, "smem_csrc": bench.csrc_hash("scene"),
             "smem_capture": "profiles/x.md"}
    monkeypatch.setattr(bench, "ncu_entry", lambda w, k, key="csrc": entry if entry[key] == bench.csrc_hash(w) else None)
    p = bench.smem_pipe("scene", "pass1", 1152e6, 0.60, 2070.0, 152)
    assert abs(p["wavefronts_per_launch"] - 156.8e6) < 1
    assert abs(p["floor_ms"] - 156.8e6 / (152 * 2070e6) * 1e3) < 1e-9
    assert abs(p["frac_smem"] - p["floor_ms"] / 0.60) < 1e-12
    assert bench.smem_pipe("scene", "pass1", 1152e6, 0.60, None, 152) is None  # no clock sample
    entry["smem_csrc"] = "0" * 16
    assert bench.smem_pipe("scene", "pass1", 1152e6, 0.60, 2070.0, 152) is None


def test_served_summary_keeps_latency_beside_every_throughput():
    load = dict(p50_ms=0.3, p99_ms=0.5, gpx_s=10.0, req_s=600.0, offered_req_s=600.0, mean_batch=1.2, requests=2000,
                failed=0, tail=dict(submit_lag_ms=0.01), batch_prep_ms=0.1)
    v = {"saturation": dict(load, gpx_s=900.0, offered_req_s=None), "latency": {"50": load, "75% of saturation": load},
         "outputs_equal_single_calls": True,
         "host_requests": {"saturation": dict(load, gpx_s=50.0), "latency_200": load, "outputs_equal_single_calls": True},
         "warmup_with_cache_misses": dict(load, tail=dict(cache_misses=3)),
         "config": {"workload": "serve", "load_generator": "native"}}
    s = bench.served_summary(v, 1000.0)
    assert s["saturation_gpx_s"] == 900.0 and abs(s["vs_fused_single"] - 0.9) < 1e-12
    for entry in [s["saturation"], *s["latency_ms"].values(), s["host_requests"]["latency_200"]]:
        assert entry["p50_ms"] is not None and entry["p99_ms"] is not None and entry["gpx_s"] is not None
