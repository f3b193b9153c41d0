"""The benchmark's JSON line on a GPU: one line from a short run of the
headline workload, with every key of the output contract and values that
hold together (device-timed rate from the step time, a roofline fraction
against a measured peak, the end-to-end arm through host buffers, clocks
sampled during the timed region)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_has_the_contract_keys():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--samples", "16", "--steps", "3", "--warmup", "3",
           "--no-cpu-baseline", "--side-steps", "1", "--serving-chains", "8"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
                "gpu_launches", "clocks"):
        assert key in d, key
    assert d["unit"] == "samples/s" and d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3
    assert d["dtype"] == "f64" and d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["config"]["mode"] == "fp64" and d["roofline"]["kernel"] == "walk_fp64_minors_kernel"
    side = d["other_forms"]
    assert set(side) == {"mixed", "df"}
    for name, f in side.items():
        assert f["samples_per_s"] > 0 and 0 <= f["samples_equal_to_headline_run"] <= 1, name
    assert d["df_kernels_k30"]["minors"]["speedup_over_fp64"] > 1
    srv = d["serving"]
    for name in ("served_fp64", "served_mixed", "one_call_per_sample_fp64"):
        assert srv[name]["requests"] == 8 and srv[name]["samples_per_s"] > 0, name
        assert srv[name]["p99_ms"] >= srv[name]["p50_ms"] > 0, name
    assert srv["served_fp64_equal_to_calls"] == 1.0
    assert d["latency_ms"]["max"] >= d["latency_ms"]["p50"] > 0
    assert d["config"]["workload"] == "cc_sampling_n30_m60" and d["config"]["samples_per_step"] == 16
    assert abs(d["value"] - 16 / (d["ms_per_step"] / 1000.0)) <= 1e-6 * d["value"]
    roof = d["roofline"]
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert 0 < roof["frac"] < 1.2 and abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-9
    assert 0 < roof["frac_of_nominal"] < 1.2 and roof["peak_nominal"] > 0
    e2e = d["e2e"]
    assert e2e["value"] > 0 and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] > 0
    assert d["clocks"] is None or d["clocks"]["sm_mhz"] > 0
    k30 = d["fp64_kernels_k30"]
    for kind in ("perm", "minors"):
        assert 0 < k30[kind]["frac_of_fp64_peak"] < k30[kind]["frac_of_fp64_pipe"] < 1.2
