"""The bench's roofline object on CPU: achieved = algorithmic work per launch / mean launch time,
the peak it is measured against, and the DRAM traffic of profiles/traffic.json used only while the
sources it was captured from are unchanged."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _prof(ms, launches, flops, nbytes):
    return {"phases": {"pcg": {"ms": ms, "launches": launches, "flops": flops, "bytes": nbytes}}}


def test_fp64_roofline_is_flops_over_launch_time():
    clocks = {"sm_max_mhz": 2070.0}
    r = bench.roofline(_prof(10.0, 20, 4.0e9, 0.0), clocks, "fp64", "k_pcg64_res")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    # 2e8 FLOP per launch in 0.5 ms
    assert abs(r["achieved"] - 0.4) < 1e-12
    assert abs(r["peak"] - 4.0 * 152 * 2070.0e6 / 1e12) < 1e-12
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r


def test_mixed_roofline_is_bytes_over_launch_time_against_measured_copy():
    r = bench.roofline(_prof(4.0, 8, 0.0, 8.0e9), {}, "mixed", "k_pcg_mixed_pool")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 2000.0) < 1e-9  # 1e9 B per launch in 0.5 ms
    pk = bench.measured_peaks().get("hbm_gbs")
    assert r["peak"] == (float(pk) if pk else 6800.0)


def test_traffic_follows_the_source_hash():
    path = os.path.join(ROOT, "profiles", "traffic.json")
    t = json.load(open(path))
    assert t, "no traffic entries"
    for kernel, e in t.items():
        r = bench.roofline(_prof(1.0, 1, 1.0, 1.0), {}, "fp64", kernel)
        current = bench.source_hash(e["files"]) == e["source_hash"]
        assert r["traffic"] == (e["bytes_per_launch"] if current else None), kernel
        assert os.path.exists(os.path.join(ROOT, "profiles", e["capture"]))


def test_iteration_histogram_counts_every_step():
    st = [{"newton_iters": n, "pcg_iters": p} for n, p in [(3, 50), (25, 700), (52, 1200), (300, 10650), (25, 800)]]
    h = bench.iteration_histogram(st)
    for name in ("newton", "pcg"):
        assert sum(b["steps"] for b in h[name]["bins"]) == len(st)
    assert h["newton"]["p50"] == 25.0 and h["newton"]["max"] == 300.0
    assert h["pcg"]["bins"][-1] == {"from": 10000, "to": None, "steps": 1}
    assert bench.iteration_histogram([]) is None
