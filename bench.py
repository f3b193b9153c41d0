#!/usr/bin/env python3
"""Benchmark: Clifford & Clifford boson sampling, n = 30 photons in m = 60
modes (seeded Haar-random interferometer, inputs in modes 0..29), through the
library's C ABI.

One step = one batch of ``--samples`` (default 200) samples drawn with every
hot-path stage on the GPU: per-chain planning, Gray decode / re-seed, the
incremental column-sum walk, the per-addend products, the fused Laplace
minors, compensated accumulation and the weighted draw.  The headline runs
the FP64 form (``--mode fp64``: column sums, products and weights in double
precision, double-double partial sums); the MIXED form is reported beside it.

  value     samples/s with U resident on the device (bs_sample_dev), CUDA
            events around every step, L2 flushed (256 MiB write) between steps
  e2e       samples/s through bs_sample with host U / host counts (copies
            inside the timed region), on the first timed steps' seeds, after
            one warm-up call through that API
  roofline  the fused-minors walk kernel of the run's precision: algorithmic
            flops (per-addend count 22K - 22, K columns) / summed kernel time
            (CUDA events on the launching stream, over --profile-steps steps
            of the same seeds) vs 2 x the FMA rate of that pipe measured on
            this GPU
  cpu_baseline  the oracle (double-double C, minors computed separately, one
            process per host core) on a bounded prefix of one chain per core,
            scaled to samples/s by its own operation count; the one-core
            figure beside it

``--impl reference`` runs the oracle as the reference arm (CPU only).
Multi-GPU: samples are independent, so ranks draw disjoint sample sets
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gray-code addends/s vs FP64 peak; C&C samples/s & p99 latency, n=30 m=60"
UNIT = "samples/s"
N_PHOTONS, M_MODES, SEED = 30, 60, 3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--samples", type=int, default=200)
    ap.add_argument("--mode", default="fp64", choices=["fp64", "mixed", "df"])
    ap.add_argument("--side-steps", type=int, default=3,
                    help="steps of the other precision's side measurement (0: skip)")
    ap.add_argument("--profile-steps", type=int, default=2, help="steps of the per-walk profiled pass")
    ap.add_argument("--e2e-steps", type=int, default=3, help="steps of the end-to-end pass")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="cc", choices=["cc", "single", "batch", "serving", "lossy", "formulas"],
                    help="cc: the headline line; the others print their own line for the other configs")
    ap.add_argument("--chains", type=int, default=64)
    ap.add_argument("--serving-rates", default="50,200,1000,inf",
                    help="Poisson arrival rates (Hz) of --workload serving, comma-separated (inf: all at once)")
    ap.add_argument("--serving-chains", type=int, default=64,
                    help="chains of the serving side measurement on the headline line (0: skip)")
    ap.add_argument("--lossy-samples", type=int, default=20, help="samples of the lossy workload")
    ap.add_argument("--lossy-modes", default="mixed,df", help="modes of the lossy workload, comma-separated")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def start_clocks(device):
    path = tempfile.mktemp(prefix="bs_clocks_", suffix=".csv")
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", "-i", str(device), "--query-gpu=" + CLOCK_FIELDS,
                              "--format=csv,noheader,nounits", "-lms", "200"], stdout=f, stderr=subprocess.DEVNULL)
        return p, f, path
    except (OSError, FileNotFoundError):
        return None, None, path


def stop_clocks(handle):
    p, f, path = handle
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
    f.close()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    with open(path) as fh:
        for line in fh:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
    os.unlink(path)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


# ---------------------------------------------------------------- oracle baseline
def full_sample_ops(n):
    # operations the oracle's sampler spends on a collision-free sample:
    # step k computes k minors, each a (k-1)x(k-1) Gray walk of 2^(k-2)
    # addends over k-1 columns
    return sum(k * (k - 1) * 2.0 ** (k - 2) for k in range(2, n + 1))


# bound on any wait for the host-core oracle processes (a worker that cannot
# start would otherwise leave the pool waiting forever)
POOL_TIMEOUT_S = 600


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_chain_prefix(job):
    """One oracle chain prefix (pool worker; module-level so that a spawned
    process can import it): returns (addend-column ops, seconds)."""
    steps, seed = job
    import oracle
    import synthetic as S
    u, occ = S.config_cc(N_PHOTONS, M_MODES, SEED)
    t0 = time.perf_counter()
    _, _, ops = oracle.cc_sample(u, occ, 1, seed=seed, max_steps=steps)
    return ops, time.perf_counter() - t0


def _oracle_fp64_prefix(job):
    """The plain-FP64 CPU form on the same work (pool worker): steps 2..s of
    a chain, each step's k minors computed separately by the oracle's
    plain-double Gray walk over the (k-1) x (k-1) matrices.  The oracle's
    sampler expands repeated rows, so a step's cost does not depend on the
    rows drawn: they are drawn uniformly here (seeded).  Returns
    (addend-column ops, seconds)."""
    steps, seed = job
    import numpy as np
    import oracle
    import synthetic as S
    u, occ = S.config_cc(N_PHOTONS, M_MODES, SEED)
    cols = np.repeat(np.arange(M_MODES), occ)
    rows = S.rng(seed).integers(0, M_MODES, size=N_PHOTONS)
    ops = 0.0
    t0 = time.perf_counter()
    for k in range(2, steps + 1):
        a = u[np.ix_(rows[:k - 1], cols[:k])]
        oracle.minors_fp64(a, np.ones(k - 1, np.int32), np.ones(k, np.int32))
        ops += k * (k - 1) * 2.0 ** (k - 2)
    return ops, time.perf_counter() - t0


def calibrate_prefix(target_s, fn=_oracle_chain_prefix):
    """Longest chain prefix (steps 1..s, s >= 12) whose single-threaded
    oracle run stays under about target_s; returns (s, ops, seconds)."""
    steps, last = 12, None
    while steps <= N_PHOTONS:
        ops, dt = fn((steps, 7))
        last = (steps, ops, dt)
        if dt > target_s:
            break
        steps += 1
    return last


class OraclePool:
    """One single-threaded oracle process per host core, started with spawn
    (never fork a process that has touched the GPU).  Each run draws one
    chain prefix per process with its own seed and reports the total
    operations over the wall time of the whole run."""

    def __init__(self, procs):
        import multiprocessing as mp
        self.procs = procs
        self.pool = mp.get_context("spawn").Pool(procs)
        self.pool.map_async(_oracle_chain_prefix, [(2, 7 + i) for i in range(procs)],
                            chunksize=1).get(timeout=POOL_TIMEOUT_S)  # imports

    def run(self, steps, fn=_oracle_chain_prefix):
        t0 = time.perf_counter()
        res = self.pool.map_async(fn, [(steps, 7 + i) for i in range(self.procs)],
                                  chunksize=1).get(timeout=POOL_TIMEOUT_S)
        return sum(r[0] for r in res), time.perf_counter() - t0

    def close(self):
        self.pool.terminate()
        self.pool.join()


def oracle_baseline(budget_s):
    """The oracle on the host: one core on a chain prefix calibrated to about
    budget_s / 3, then every core at once on the same prefix length (one
    chain per core).  samples/s = (ops/s) / (ops of a full sample)."""
    steps, ops1, dt1 = calibrate_prefix(budget_s / 3)
    full = full_sample_ops(N_PHOTONS)
    one = {"value": ops1 / dt1 / full, "cores": 1}
    fsteps, fops1, fdt1 = calibrate_prefix(budget_s / 6, _oracle_fp64_prefix)
    procs = host_cores()
    pool = OraclePool(procs)
    try:
        ops, wall = pool.run(steps)
        fops, fwall = pool.run(fsteps, _oracle_fp64_prefix)
    finally:
        pool.close()
    plain = {"value": fops / fwall / full, "cores": procs, "one_core": {"value": fops1 / fdt1 / full, "cores": 1},
             "what": ("the oracle's plain-double Gray walk (no compensation), each of a step's k minors computed "
                      "separately, on the same matrix sizes"),
             "sample": f"steps 2..{fsteps} of one chain per core, {procs} cores in parallel: {fops:.3g} ops in "
                       f"{fwall:.2f} s"}
    return {"value": ops / wall / full, "unit": UNIT, "cores": procs, "kind": "oracle",
            "one_core": one, "plain_fp64": plain,
            "what": ("the double-double oracle, each of a step's k minors computed separately as its own "
                     "(k-1) x (k-1) Gray BB/FG permanent (k times the work of the fused walk), not a tuned CPU "
                     "code"),
            "sample": (f"steps 1..{steps} of one n=30 m=60 chain per core, {procs} cores in parallel (double-double "
                       f"C oracle, minors computed separately): {ops:.3g} addend-column ops in "
                       f"{wall:.2f} s; scaled by the {full:.3g} ops of a full collision-free sample")}


def run_reference(args):
    """Reference arm: the oracle on every host core.  Warm-up calibrates a
    chain prefix that takes about --cpu-seconds / 4 on one core; each timed
    step runs that prefix on every core at once (one chain per core)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    steps, _, _ = calibrate_prefix(max(args.cpu_seconds, 2.0) / 4)
    procs = host_cores()
    pool = OraclePool(procs)
    times, ops_sum = [], 0.0
    try:
        for _ in range(max(args.warmup, 0)):
            pool.run(steps)
        for _ in range(max(args.steps, 1)):
            ops, wall = pool.run(steps)
            times.append(wall)
            ops_sum += ops
    finally:
        pool.close()
    full = full_sample_ops(N_PHOTONS)
    value = ops_sum / sum(times) / full
    cb = {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
          "sample": (f"steps 1..{steps} of one n=30 m=60 chain per core and step, {procs} cores in parallel "
                     f"({ops_sum / len(times):.3g} addend-column ops per step), scaled by the {full:.3g} ops of a "
                     f"full collision-free sample")}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "dtype_detail": "double-double (pairs of f64) throughout",
            "data": "synthetic (seeded Haar-random 60-mode unitary)",
            "config": {"workload": "cc_sampling_n30_m60", "n": N_PHOTONS, "m": M_MODES,
                       "samples_per_step": f"bounded chain prefix per host core (oracle, {procs} cores)"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- multi-rank helpers
def paper_model(samples_per_s, n=N_PHOTONS, m=M_MODES):
    """The portable figure of the paper's performance model (Sec. 4, Eq.
    performance): T_sampling = T0 [n (m + n) / m C(2m + n, n + 1) / C(m + n,
    n + 1) + n^2 m]; T0 of this run (one GPU) beside the paper's fit for its
    4-FPGA system, as context."""
    from math import comb
    bracket = n * (m + n) / m * comb(2 * m + n, n + 1) / comb(m + n, n + 1) + n * n * m
    return {"T0_s": 1.0 / samples_per_s / bracket, "paper_T0_s_4_fpga": 7.5e-11, "bracket": bracket}


def rank_seed_base(rank):
    """Seed of a rank's sample stream: ranks draw disjoint, independent
    sample sets (the samples of Sec. 4 are independent; no collective on the
    data path)."""
    return 1000003 * (rank + 1)


def max_over_ranks(seconds, dist):
    """The job time is the slowest rank's (all_reduce MAX); works on gloo
    (CPU tensor) and NCCL (CUDA tensor)."""
    if dist is None:
        return seconds
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, units_per_rank, seconds):
    """Whole-job rate: units processed by all ranks / the slowest rank's time."""
    return world * units_per_rank / seconds


# ---------------------------------------------------------------- GPU arm
# Arithmetic of each form (the headline's dtype and the side forms').
DTYPES = {"fp64": "f64", "mixed": "f32", "df": "f32x2"}
DTYPE_DETAIL = {
    "fp64": ("f64 column sums, products and weights; per-lane double runs folded into double-double, "
             "double-double task partials (Sum2 reduce)"),
    "mixed": ("f32 column sums and products where the MIXED rule predicts an error below 1e-6 prod ||a_j|| "
              "(column sums re-seeded every 2^8 steps where only their drift would exceed it; the rule is "
              "oracle-checked in tests/test_gpu_widths.py), double-float otherwise; float-float runs folded into "
              "double-double partials"),
    "df": ("double-float: each value a pair of f32 (about 48 significant bits) on the FP32 pipe; exact "
           "fixed-point column sums, FMA-based exact products, Sum2 runs, double-double partials; within the FP64 "
           "tolerance 1e-10 prod ||a_j||, with errors against the oracle about 100x the FP64 kernels' "
           "(tests/test_gpu_parity.py, tests/test_gpu_widths.py)"),
}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k = 30
# fused-minor launch of this workload under ncu, and the chains it ran; by
# precision [FP64, FP32, double-float].  The traffic does not grow in
# proportion to the chains (the task partials stay in L2 for a few chains
# and spill from it at 200: FP64 0.69 MB at 8 chains, 1.36 MB at 32, 80.1 MB
# at 200), so only a capture of the full 200-chain launch is used; None where
# there is none, or where the kernel changed since the capture.
TRAFFIC_K30 = [{"bytes": 80.08e6, "chains": 200}, None, None]
# The bounding pipe's busy fraction in the same captures
# (sm__pipe_fp64_cycles_active / sm__pipe_fma_cycles_active, pct of peak
# sustained active): FP64 pipe for the FP64 kernel, FMA pipe for the others.
PIPE_K30 = [{"pipe": "fp64", "active": 0.928}, {"pipe": "fma", "active": 0.709}, {"pipe": "fma", "active": 0.788}]

def run_mine(args):
    import numpy as np
    import torch

    import paper_2309_07027_gb300 as bs
    import synthetic as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    modes = {"fp64": bs.BS_FP64, "mixed": bs.BS_MIXED, "df": bs.BS_DF64}
    mode = modes[args.mode]
    u, occ = S.config_cc(N_PHOTONS, M_MODES, SEED)
    ctx = bs.Context(local)
    # a dedicated stream: on the legacy default stream the sampler cannot
    # replay its captured graph and launches eagerly
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx.set_stream(stream)
    fp64_rate, fp32_rate = ctx.measure_fma_rates()
    u_dev = torch.from_numpy(u).to("cuda")
    S_ = args.samples
    out_dev = torch.zeros((S_, M_MODES), dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    seed_base = rank_seed_base(rank)

    for w in range(args.warmup):
        ctx.sample_dev(u_dev, occ, S_, seed_base + w, out_dev, mode=mode)
        ctx.sync()

    def timed_steps(steps, profile, md, out):
        """`steps` sampler steps (seeds fixed per step), each between CUDA
        events on the stream, the L2 flushed before each; returns the step
        times (ms)."""
        ctx.set_profiling(profile)
        evs = []
        for i in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.sample_dev(u_dev, occ, S_, seed_base + 100 + i, out, mode=md)
            e1.record(stream)
            evs.append((e0, e1))
            if profile:
                # a profiled graph replay is read back before the next one
                # starts: wait here, outside the timed events
                stream.synchronize()
        torch.cuda.synchronize()
        ctx.set_profiling(False)
        return [a.elapsed_time(b) for a, b in evs]

    # timed region: the production path (graph replay, no per-walk events)
    ctx.reset_stats()
    clocks = start_clocks(local)
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    step_ms = timed_steps(args.steps, False, mode, out_dev)
    barrier()
    wall = time.perf_counter() - wall0
    clk = stop_clocks(clocks)
    ctx.sync()
    launches = int(ctx.stats()["kernel_launches"])
    counts = out_dev.cpu().numpy()  # the last timed step (seed seed_base + 100 + steps - 1)
    assert np.all(counts.sum(axis=1) == N_PHOTONS), "sampler returned a wrong photon count"
    t_max = max_over_ranks(sum(step_ms) / 1000.0, dist)
    value = aggregate_rate(world, S_ * args.steps, t_max)
    # the first steps again with CUDA events around every walk launch (on the
    # launching stream, inside the replayed graph): kernel times for the
    # roofline; the events add about 3 % to a step
    ctx.reset_stats()
    psteps = max(1, min(args.profile_steps, args.steps))
    prof_step_ms = timed_steps(psteps, True, mode, out_dev)
    st = ctx.stats()

    # roofline of the dominant walk kernel: the fused minors of the run's
    # precision (MIXED sends heavy-collision chains to the FP64 kernel, whose
    # time and work are reported beside)
    p = {bs.BS_FP64: 0, bs.BS_MIXED: 1, bs.BS_DF64: 2}[mode]
    walk_s = st["walk_ms"][p] / 1000.0
    fl = st["addend_flops"][p]
    # (the double-float form's algorithmic flops are FP64-equivalent ones,
    # set against the FP64 pipe's peak: its fraction exceeds 1 by design)
    peak = 2.0 * (fp32_rate if p == 1 else fp64_rate) / 1e12
    achieved = fl / walk_s / 1e12 if walk_s > 0 else 0.0
    # DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the k = 30
    # fused-minor launch, from an ncu capture of that launch with the same
    # number of chains (null for other chain counts: the task partials' share
    # of the traffic depends on whether they fit L2).  The kernels are
    # compute-bound; the figure shows that they re-read nothing.
    cap = TRAFFIC_K30[p]
    traffic = cap["bytes"] if cap and cap["chains"] == S_ else None
    # nominal peak from unit counts and clocks: FMA lanes per SM per clock
    # (128 FP32, 2 FP64 on this part) x SMs x maximum SM clock x 2 flops
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    max_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    lanes = 128 if p == 1 else 2
    peak_nominal = 2.0 * lanes * sms * max_mhz * 1e6 / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if peak else None, "traffic": traffic,
            "traffic_launch": (f"the k = 30 launch of {S_} chains (ncu dram__bytes_read.sum + dram__bytes_write.sum)"
                               if traffic is not None else None),
            "ncu_pipe_active_k30": PIPE_K30[p],
            "kernel": ("walk_fp64_minors_kernel", "walk_fp32_minors_kernel", "walk_df_minors_kernel")[p],
            "peak_source": ("measured on this GPU by bs_measure_fma_rates (2 flops per lane-FMA), "
                            + ("FP32 FMA pipe" if p == 1 else "FP64 pipe")),
            "peak_nominal": peak_nominal, "frac_of_nominal": achieved / peak_nominal,
            "peak_nominal_source": f"{lanes} FMA lanes / SM / clock x {sms} SMs x {max_mhz:.0f} MHz x 2",
            "walk_ms_per_step": st["walk_ms"][p] / psteps, "walk_launches": int(st["timed_launches"][p]),
            "walk_share_of_step": st["walk_ms"][p] / sum(prof_step_ms) if sum(prof_step_ms) else None,
            "measured_over": f"{psteps} profiled steps on the first timed steps' seeds, right after the timed "
                             f"pass ({statistics.mean(prof_step_ms):.1f} ms per profiled step)",
            "addends_per_s": st["addends"][p] / walk_s if walk_s > 0 else 0.0,
            "other_kernels": {name: {"walk_ms_per_step": st["walk_ms"][q] / psteps, "addends": st["addends"][q]}
                              for q, name in enumerate(("fp64", "fp32", "df")) if q != p}}

    # end to end through the host API (U from host memory, counts back), on
    # the first timed steps' seeds, hence the same samples and work; the L2
    # flush before each step stays outside the timed interval
    e2e = None
    if not args.no_e2e:
        ctx.set_stream(None)
        ctx.sample(u, occ, S_, seed_base + 90, mode=mode)  # the host path captures its own graph on first use
        esteps = max(1, min(args.e2e_steps, args.steps))
        e2e_t = 0.0
        for i in range(esteps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.sample(u, occ, S_, seed_base + 100 + i, mode=mode)
            e2e_t += time.perf_counter() - t0
        e2e_t = max_over_ranks(e2e_t, dist)  # the slowest rank, as for the device-timed value
        # the device-timed rate of the same seeds (the first timed steps),
        # so that the two numbers compare the same work
        dev_same = max_over_ranks(sum(step_ms[:esteps]) / 1000.0, dist)
        e2e = {"value": world * S_ * esteps / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(u.nbytes),
               "d2h_bytes_per_step": int(S_ * M_MODES * 4), "steps": esteps,
               "device_timed_same_steps": world * S_ * esteps / dev_same}
        ctx.set_stream(stream)

    # the other forms on the same workload: samples/s over a few steps and,
    # on the last timed step's seeds, how many of their samples equal the
    # headline run's (the oracle comparisons of every form are in tests/)
    side = {}
    if args.side_steps > 0:
        for name in ("df", "mixed", "fp64"):
            other = modes[name]
            if other == mode:
                continue
            out2 = torch.zeros((S_, M_MODES), dtype=torch.int32, device="cuda")
            ctx.sample_dev(u_dev, occ, S_, seed_base + 98, out2, mode=other)  # warm-up / capture
            ctx.sync()
            sms_ = timed_steps(min(args.side_steps, args.steps), False, other, out2)
            ctx.sample_dev(u_dev, occ, S_, seed_base + 100 + args.steps - 1, out2, mode=other)
            ctx.sync()
            same = float(np.mean(np.all(out2.cpu().numpy() == counts, axis=1)))
            side[name] = {"samples_per_s": S_ * len(sms_) / (sum(sms_) / 1000.0), "steps": len(sms_),
                          "dtype": DTYPES[name], "dtype_detail": DTYPE_DETAIL[name],
                          "samples_equal_to_headline_run": same}

    # the plain FP64 kernels on single k = 30 jobs, as fractions of the FP64
    # peak (the FP64 form is meant to keep the FP64 pipe >= 60 % busy for
    # k >= 30): permanent 30 x 30, minors 29 x 30
    fp64_k30, df_k30 = {}, {}
    ctx.set_profiling(True)
    u60 = S.haar_unitary(60, 77)
    for kind, rows in (("perm", 30), ("minors", 29)):
        a = u60[:rows, :30]
        M, N = np.ones(rows, np.int32), np.ones(30, np.int32)
        res = {}
        for md, p in ((bs.BS_FP64, 0), (bs.BS_DF64, 2)):
            for rep in range(2):
                ctx.reset_stats()
                if kind == "perm":
                    v = ctx.perm(a, M, N, mode=md)
                else:
                    v = ctx.laplace_minors(a, M, N, mode=md)
                s2 = ctx.stats()
            res[p] = (np.atleast_1d(v), s2["walk_ms"][p] / 1000.0, s2["addends"][p], s2["addend_flops"][p])
        _, secs, adds, flops = res[0]
        rate = adds / secs
        # FP64-pipe operations the walk needs per addend at K = 30 columns:
        # permanent 2K (update) + 4(K - 1) (product) + 2 (weighted sum);
        # lane-pair minors about 14K (each lane: update K, suffix and prefix
        # chains 2K - 4 each, accumulate 2K, exchange and weight about 6)
        ops = 6 * 30 - 2 if kind == "perm" else 14 * 30
        fp64_k30[kind] = {"addends_per_s": rate,
                          "frac_of_fp64_peak": flops / secs / (2.0 * fp64_rate),
                          "fp64_pipe_ops_per_addend": ops,
                          "frac_of_fp64_pipe": rate * ops / fp64_rate}
        vd, secs_d, adds_d, flops_d = res[2]
        norms = np.sqrt((np.abs(a) ** 2).sum(axis=0))
        scale = float(np.prod(norms)) / (float(norms.max()) if kind == "minors" else 1.0)
        df_k30[kind] = {"addends_per_s": adds_d / secs_d, "speedup_over_fp64": secs / secs_d,
                        "fp64_equivalent_tflops": flops_d / secs_d / 1e12,
                        "max_diff_from_fp64_over_prod_norms": float(np.max(np.abs(vd - res[0][0]))) / scale}
    ctx.set_profiling(False)
    serving_c4 = serving_measure(args.serving_chains) if rank == 0 and args.serving_chains > 0 else None
    if rank != 0:
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.mode], "dtype_detail": DTYPE_DETAIL[args.mode],
        "data": "synthetic (seeded Haar-random 60-mode unitary)",
        "config": {"workload": "cc_sampling_n30_m60", "n": N_PHOTONS, "m": M_MODES, "samples_per_step": S_,
                   "mode": args.mode, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{world} (independent samples)"},
        "latency_ms": {"p50": statistics.median(step_ms), "max": max(step_ms), "steps": len(step_ms),
                       "what": ("per batch of samples (all chains of a batch finish together), over the timed "
                                "steps; per-request p50 / p99 come from the serving workload")},
        "paper_model": paper_model(value / world),
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clk, "other_forms": side, "fp64_kernels_k30": fp64_k30, "df_kernels_k30": df_k30,
        "serving": serving_c4, "wall_s": wall,
        "fma_rates_measured": {"fp64_per_s": fp64_rate, "fp32_per_s": fp32_rate},
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- other configs
def oracle_work(M, N):
    """Inner operations of the oracle's term-by-term walk for one item: its
    term count (row 0 pinned, the rest of its copies a digit) x formula rows
    x product columns (each term rebuilds every column sum)."""
    occ = [int(m) for m in M if m > 0]
    if not occ:
        return 1
    terms = occ[0] if occ[0] > 1 else 1
    for m in occ[1:]:
        terms *= m + 1
    rows = len(occ) + (1 if occ[0] > 1 else 0)
    cols = sum(1 for x in N if x > 0)
    return terms * rows * cols


def _oracle_item(job):
    """Pool worker (module level, for spawn): time one item with the oracle
    in double-double (plain=False) or in plain double (plain=True)."""
    a, M, N, plain = job
    import oracle
    t0 = time.perf_counter()
    if plain:
        oracle.perm_mult_fp64(a, M, N)
    else:
        oracle.perm_mult(a, M, N)
    return time.perf_counter() - t0


def oracle_batch_timing(items, budget_s):
    """The oracle on a seeded subset of the batch: items in a seeded order,
    each predicted (from a calibration on the cheapest items) to take at
    most budget_s / 8, until about budget_s of one-core work.  The time per
    inner operation, tau, fitted on the subset, projects the whole batch;
    the same subset then runs on every host core at once (spawned processes,
    the subset once per core, items handed out one at a time) and in plain
    double on one core."""
    import numpy as np
    work = np.array([oracle_work(M, N) for _, M, N in items], dtype=np.float64)
    by_work = np.argsort(work)
    cheap = by_work[len(items) // 20: len(items) // 20 + 8]   # small but not call-overhead bound
    t_cal = sum(_oracle_item((*items[i], False)) for i in cheap)
    tau0 = t_cal / work[cheap].sum()
    order = np.random.default_rng(2024).permutation(len(items))
    subset, spent = [], 0.0
    for i in order:
        pred = tau0 * work[i]
        if pred > budget_s / 8:
            continue
        subset.append(int(i))
        spent += pred
        if spent >= budget_s:
            break
    w_sub = work[subset].sum()
    t1 = sum(_oracle_item((*items[i], False)) for i in subset)
    tf = sum(_oracle_item((*items[i], True)) for i in subset)
    procs = host_cores()
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map_async(_oracle_item, [(*items[i], False) for i in cheap[:procs]],
                       chunksize=1).get(timeout=POOL_TIMEOUT_S)  # imports
        t0 = time.perf_counter()
        jobs = [(*items[i], False) for i in subset for _ in range(procs)]   # a full share per core
        pool.map_async(_oracle_item, jobs, chunksize=1).get(timeout=POOL_TIMEOUT_S)
        tall = (time.perf_counter() - t0) / procs
    total = work.sum()
    return {"subset_items": len(subset), "subset_work_fraction": float(w_sub / total),
            "one_core": {"tau_s_per_op": t1 / w_sub, "projected_batch_s": t1 / w_sub * total,
                         "permanents_per_s": len(items) / (t1 / w_sub * total)},
            "all_cores": {"cores": procs, "projected_batch_s": tall / w_sub * total,
                          "permanents_per_s": len(items) / (tall / w_sub * total)},
            "plain_fp64_one_core": {"projected_batch_s": tf / w_sub * total,
                                    "permanents_per_s": len(items) / (tf / w_sub * total)},
            "what": ("oracle: Eq. bbfgrepeated term by term in double-double; plain FP64: the same walk in "
                     "double; projected over the whole batch by inner operations (terms x rows x columns)")}


def run_batch(args):
    """4096 uneven permanents (k ~ U[10, 28], binomially collapsed outputs):
    FP64 and MIXED throughput, MIXED error against FP64 on every item and
    both against the oracle on the 16 cheapest items."""
    import numpy as np
    import torch
    import oracle
    import paper_2309_07027_gb300 as bs
    import synthetic as S
    items = S.config_batch(count=4096, seed=2)
    ctx = bs.Context(0)
    packed, offs, rows, cols, mults, roff, coff = ctx.pack_batch(items)
    dev = torch.from_numpy(packed).cuda()
    out = {}
    res = {}
    for mode, name in ((bs.BS_FP64, "fp64"), (bs.BS_MIXED, "mixed"), (bs.BS_DF64, "df")):
        o = torch.zeros(len(items), dtype=torch.complex128, device="cuda")
        ctx.set_stream(torch.cuda.current_stream())
        for w in range(args.warmup):
            ctx.perm_batch_dev(dev, offs, rows, cols, mults, roff, coff, mode, o)
        ctx.sync()
        ctx.reset_stats()
        ctx.set_profiling(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for s in range(args.steps):
            ctx.perm_batch_dev(dev, offs, rows, cols, mults, roff, coff, mode, o)
        e1.record()
        ctx.sync()
        st = ctx.stats()
        ctx.set_profiling(False)
        ms = e0.elapsed_time(e1) / args.steps
        res[name] = o.cpu().numpy()
        p = {bs.BS_FP64: 0, bs.BS_MIXED: 1, bs.BS_DF64: 2}[mode]
        rates = ctx.measure_fma_rates()
        out[name] = {"permanents_per_s": len(items) / (ms / 1000), "ms_per_batch": ms,
                     "addends_per_s": sum(st["addends"]) / (ms / 1000) / args.steps,
                     # FP64 and double-float against the FP64 pipe (FP64-equivalent flops), FP32 against its own
                     "walk_kernel_frac_of_peak": (st["addend_flops"][p] / (st["walk_ms"][p] / 1000) /
                                                  (2 * rates[1 if p == 1 else 0])) if st["walk_ms"][p] else None}
    sc = np.array([np.prod(np.sqrt((np.abs(a) ** 2 * M[:, None]).sum(0)) ** N) for a, M, N in items])
    rel = np.abs(res["mixed"] - res["fp64"]) / sc
    rel_df = np.abs(res["df"] - res["fp64"]) / sc
    costs = np.argsort([int(np.prod(np.asarray(M) + 1)) for _, M, _ in items])[:16]
    orc = {"fp64_max": 0.0, "mixed_max": 0.0}
    for b_ in costs:
        a, M, N = items[b_]
        v, t = oracle.perm_mult(a, M, N)
        orc["fp64_max"] = max(orc["fp64_max"], abs(res["fp64"][b_] - (v + t)) / sc[b_])
        orc["mixed_max"] = max(orc["mixed_max"], abs(res["mixed"][b_] - (v + t)) / sc[b_])
    # a small batch, where host planning and launches dominate: per-call time
    # with the captured graph replayed vs planned and launched every call
    small = S.config_batch(count=64, seed=12, kmin=10, kmax=16)
    sp, soffs, srows, scols, smults, sroff, scoff = ctx.pack_batch(small)
    sdev = torch.from_numpy(sp).cuda()
    so = torch.zeros(len(small), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.Stream()
    ctx.set_stream(stream)
    small_us = {}
    for graphs in (True, False):
        ctx.set_graphs(graphs)
        for w in range(3):
            ctx.perm_batch_dev(sdev, soffs, srows, scols, smults, sroff, scoff, bs.BS_MIXED, so)
        ctx.sync()
        reps = 50
        t0 = time.perf_counter()
        for r in range(reps):
            ctx.perm_batch_dev(sdev, soffs, srows, scols, smults, sroff, scoff, bs.BS_MIXED, so)
        ctx.sync()
        small_us["graph" if graphs else "eager"] = (time.perf_counter() - t0) / reps * 1e6
    ctx.set_graphs(True)
    ctx.set_stream(None)
    line = {"workload": "batch_4096_k10_28", "metric": "permanents/s", "fp64": out["fp64"], "mixed": out["mixed"],
            "df": out["df"],
            "mixed_vs_fp64_err_over_prod_norms": {"max": float(rel.max()), "p99": float(np.percentile(rel, 99))},
            "df_vs_fp64_err_over_prod_norms": {"max": float(rel_df.max()), "p99": float(np.percentile(rel_df, 99))},
            "err_vs_oracle_over_prod_norms_16_cheapest": orc,
            "small_batch_64_k10_16_mixed_us_per_call": small_us,
            "cpu_oracle": None if args.no_cpu_baseline else oracle_batch_timing(items, args.cpu_seconds)}
    print(json.dumps(line), flush=True)
    return 0


def serving_measure(chains, modes=("fp64", "mixed"), rate_hz=200.0, baseline=True):
    """Serving workload (C4): ``chains`` C&C samples, each with its own Haar
    60 x 60 unitary and n ~ U[16, 34], Poisson arrivals at ``rate_hz``
    (inf: all at once), served by the continuous-batching engine (every
    chain on the device) in each of ``modes``, and the same requests
    answered by one sample_ex call each in FP64 (one walk launch per minors
    job).  Samples/s over the wall time and per-request latency (arrival to
    counts)."""
    import numpy as np
    import paper_2309_07027_gb300 as bs
    from paper_2309_07027_gb300 import serving
    import synthetic as S
    cfg = S.config_serving(chains=chains, rate_hz=rate_hz)
    mode_of = {"fp64": bs.BS_FP64, "mixed": bs.BS_MIXED, "df": bs.BS_DF64}
    rate_name = "all_at_once" if rate_hz == float("inf") else f"poisson{rate_hz:g}hz"
    out = {"workload": f"serving_{chains}_chains_n16_34_m60_{rate_name}",
           "latency_what": "per request: arrival (submission) to counts available"}
    ref = None
    for name in modes:
        with bs.Server(0, mem_budget_bytes=40 << 30, max_active=64, tick_tasks=8192, mode=mode_of[name]) as srv:
            wall, lat, counts = serving.run_served(cfg, srv)
            st = srv.stats()
        r = serving.summarize(wall, lat, len(cfg))
        r["server"] = {k: st[k] for k in ("ticks", "walk_launches", "max_resident", "mem_peak_bytes")}
        out[f"served_{name}"] = r
        if name == "fp64":
            ref = counts
    if baseline:
        ctx = bs.Context(0)
        ctx.sample_ex(cfg[0]["unitary"], cfg[0]["occupation"], 1, 1)  # load and warm the kernels
        wall, lat, counts = serving.run_one_call_per_sample(cfg, ctx, mode=bs.BS_FP64)
        ctx.close()
        out["one_call_per_sample_fp64"] = serving.summarize(wall, lat, len(cfg))
        if ref is not None:
            out["served_fp64_equal_to_calls"] = float(np.mean([np.array_equal(a, b) for a, b in zip(ref, counts)]))
    return out


def run_serving(args):
    """C4 with the arrival rate swept to saturation: one JSON line per rate."""
    for rate in (float(x) for x in args.serving_rates.split(",")):
        print(json.dumps(serving_measure(args.chains, ("fp64", "mixed", "df"), rate_hz=rate)), flush=True)
    return 0


def run_lossy(args):
    """n = 40 photons, m = 60, eta = 0.5: the 100 x 40 isometry, only the
    first 60 outputs counted; seconds per sample in each of --lossy-modes
    (every chain draws all 40 photons, loss modes included)."""
    import numpy as np
    import paper_2309_07027_gb300 as bs
    import synthetic as S
    v, mdet = S.config_lossy()
    ctx = bs.Context(0)
    ns = max(1, args.lossy_samples)
    mode_of = {"fp64": bs.BS_FP64, "mixed": bs.BS_MIXED, "df": bs.BS_DF64}
    res = {}
    for name in args.lossy_modes.split(","):
        t0 = time.perf_counter()
        counts = ctx.sample_ex(v, np.ones(v.shape[1], np.int32), ns, seed=5, m_detected=mdet, mode=mode_of[name])
        dt = time.perf_counter() - t0
        res[name] = {"s_per_sample": dt / ns, "samples": ns, "detected_mean": float(counts.sum(1).mean()),
                     "counts": counts.tolist() if ns <= 4 else None}
    same = None
    if "mixed" in res and "df" in res and res["mixed"]["counts"] is not None and res["df"]["counts"] is not None:
        same = float(np.mean([a == b for a, b in zip(res["mixed"]["counts"], res["df"]["counts"])]))
    for r in res.values():
        r.pop("counts")
    print(json.dumps({"workload": "lossy_n40_m60_eta0.5", "metric": "s/sample", "modes": res,
                      "samples_equal_mixed_df": same,
                      "paper_context_s_per_sample": {"ideal_4_fpga": 80, "lossy_4_fpga": 360}}), flush=True)
    return 0


def run_formulas(args):
    """The comparison of Sec. 3.2 on this GPU: relative error (against the
    double-double oracle) of the FP64 Gray walks of Eq. bbfg, Eq. ryser and
    its Nijenhuis-Wilf form, plus MIXED BB/FG, on Haar-random n x n unitaries
    (Fig. accuracy's inputs), and each formula's speed on one 30 x 30
    permanent."""
    import numpy as np
    import oracle
    import paper_2309_07027_gb300 as bs
    import synthetic as S
    ctx = bs.Context(0)
    fp64_rate = ctx.measure_fma_rates()[0]
    acc = {}
    for n in (8, 12, 16, 20, 24):
        worst = {"bbfg": 0.0, "ryser": 0.0, "nw": 0.0, "bbfg_mixed": 0.0}
        for r in range(2):
            a = S.haar_unitary(n, 1000 + 10 * n + r)
            v, t = oracle.bbfg_gray(a)
            ref = v + t
            for f in ("bbfg", "ryser", "nw"):
                worst[f] = max(worst[f], abs(ctx.perm_formula(a, f) - ref) / abs(ref))
            worst["bbfg_mixed"] = max(worst["bbfg_mixed"], abs(ctx.perm(a, mode=bs.BS_MIXED) - ref) / abs(ref))
        acc[str(n)] = worst
    speed = {}
    a = S.haar_unitary(30, 1030)
    ctx.set_profiling(True)
    for f in ("bbfg", "ryser", "nw"):
        ctx.perm_formula(a, f)  # warm-up
        ctx.reset_stats()
        t0 = time.perf_counter()
        ctx.perm_formula(a, f)
        wall = time.perf_counter() - t0
        st = ctx.stats()
        secs = st["walk_ms"][0] / 1000.0
        speed[f] = {"addends": int(st["addends"][0]), "walk_s": secs, "call_s": wall,
                    "addends_per_s": st["addends"][0] / secs,
                    "frac_of_fp64_peak": st["addend_flops"][0] / secs / (2.0 * fp64_rate)}
    ctx.set_profiling(False)
    print(json.dumps({"workload": "formulas_haar_n8_24_and_n30", "metric": "relative error; addends/s",
                      "relative_error_max_of_2": acc, "speed_n30_fp64": speed,
                      "reference": "oracle double-double BB/FG (Eq. bbfg)"}), flush=True)
    return 0


def addend_count(M):
    """Addends of Eq. bbfgrepeated with one copy of a smallest-multiplicity
    row pinned: prod over the other rows of (M + 1), times M_p for the M_p - 1
    remaining copies of the pinned row."""
    ms = sorted(int(m) for m in M if m > 0)
    if not ms:
        return 1
    c = ms[0] if ms[0] > 1 else 1
    for m in ms[1:]:
        c *= m + 1
    return c


def _time_calls(fn, reps):
    """Median wall time of reps calls (each returns host results, so the
    call includes the copies and the synchronisation)."""
    fn()
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        ts.append(time.perf_counter() - t0)
    return statistics.median(ts)


def run_single(args):
    """The 12-photon configuration: A = 8 distinct output rows (multiplicities
    3,2,2,1,1,1,1,1) x 12 input columns of a Haar 24 x 24 unitary; its
    permanent and the 12 Laplace minors of the 11 x 12 matrix left after one
    copy of the last row is removed.  GPU call latency per mode and error
    against the double-double oracle, beside the oracle's own times (double-
    double and plain FP64, one host core)."""
    import numpy as np
    import oracle
    import paper_2309_07027_gb300 as bs
    import synthetic as S
    a, M, N, _, _ = S.config_single(seed=1)
    M2 = M.copy()
    M2[-1] -= 1
    ref = sum(oracle.perm_mult(a, M, N))
    mv, mt = oracle.minors(a, M2, N)
    ref_minors = mv + mt
    norms = np.sqrt((np.abs(a) ** 2 * M[:, None]).sum(axis=0))
    scale = float(np.prod(norms ** N))
    ctx = bs.Context(0)
    reps = max(args.steps, 1) * 20
    out = {}
    for mode, name in ((bs.BS_FP64, "fp64"), (bs.BS_MIXED, "mixed")):
        p = ctx.perm(a, M, N, mode=mode)
        mi = ctx.laplace_minors(a, M2, N, mode=mode)
        out[name] = {"perm_us": 1e6 * _time_calls(lambda: ctx.perm(a, M, N, mode=mode), reps),
                     "minors_us": 1e6 * _time_calls(lambda: ctx.laplace_minors(a, M2, N, mode=mode), reps),
                     "perm_err_over_prod_norms": abs(p - ref) / scale,
                     "minors_max_err_over_prod_norms": float(np.max(np.abs(mi - ref_minors))) / scale}
    ctx.close()
    cpu = {"cores": 1,
           "perm_dd_us": 1e6 * _time_calls(lambda: oracle.perm_mult(a, M, N), 5),
           "minors_dd_us": 1e6 * _time_calls(lambda: oracle.minors(a, M2, N), 3),
           "perm_fp64_us": 1e6 * _time_calls(lambda: oracle.perm_mult_fp64(a, M, N), 5),
           "what": ("oracle: Eq. bbfgrepeated term by term in double-double (perm) and the expanded-matrix "
                    "Gray walk per minor; plain FP64: the same term-by-term walk in double")}
    print(json.dumps({"workload": "single_12_photons_rows_3_2_2_1_1_1_1_1", "metric": "us per call",
                      "addends": addend_count(M),
                      "gpu": out, "cpu_oracle": cpu,
                      "calls_timed": reps, "timing": "median wall time per call, host inputs and outputs"}),
          flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    from paper_2309_07027_gb300 import _build
    _build.build()
    if args.workload == "single":
        return run_single(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "lossy":
        return run_lossy(args)
    if args.workload == "formulas":
        return run_formulas(args)
    return run_mine(args)


if __name__ == "__main__":
    sys.exit(main())
