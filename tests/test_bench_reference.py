"""The benchmark's reference arm (the oracle on the host cores) on CPU: one
JSON line from rank 0 with the contract's keys, nothing from other ranks."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CMD = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0",
       "--cpu-seconds", "0.5"]


def _run(rank):
    env = dict(os.environ, RANK=str(rank))
    return subprocess.run(CMD, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)


def test_reference_arm_prints_one_line():
    r = _run(0)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "samples/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "samples/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "cc_sampling_n30_m60"


def test_reference_arm_other_ranks_are_silent():
    r = _run(1)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_bench_addend_count_matches_the_planner():
    """The addend count the benchmark reports (bench.addend_count) is the
    planner's: one copy of a smallest-multiplicity row pinned, the others
    digits of radix M + 1."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import paper_2309_07027_gb300 as bs
    g = np.random.default_rng(77)
    for _ in range(40):
        R = int(g.integers(1, 8))
        M = g.integers(0, 4, size=R).astype(np.int32)
        if M.sum() == 0:
            M[0] = 1
        n = int(M.sum())
        plan = bs.debug_plan(M, np.ones(n, np.int32))
        assert not plan["transposed"]
        assert bench.addend_count(M) == plan["C"], (M, plan)
    assert bench.addend_count([3, 2, 2, 1, 1, 1, 1, 1]) == 576


def test_headline_cpu_baseline_has_the_plain_fp64_row():
    """The headline line's cpu_baseline (host cores, no GPU): the
    double-double oracle's rate with its one-core figure, and beside it the
    plain-FP64 row (the oracle's plain-double Gray walk on the same
    matrix sizes), which must be the faster of the two."""
    sys.path.insert(0, ROOT)
    import bench
    cb = bench.oracle_baseline(1.0)
    assert cb["kind"] == "oracle" and cb["unit"] == "samples/s" and cb["cores"] >= 1
    assert cb["value"] > 0 and cb["one_core"]["value"] > 0
    p = cb["plain_fp64"]
    assert p["value"] > 0 and p["one_core"]["value"] > cb["one_core"]["value"]
    assert "what" in p and "sample" in p
