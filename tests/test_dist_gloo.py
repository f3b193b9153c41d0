"""Multi-rank path of the benchmark, on CPU with the gloo backend and two
ranks: every rank gets its own sample stream, the job time is the slowest
rank's, and the rate counts the work of all ranks."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import bench
    seed = bench.rank_seed_base(rank)
    t = bench.max_over_ranks(0.25 + rank, dist)
    rate = bench.aggregate_rate(world, 100, t)
    seeds = [None] * world
    dist.all_gather_object(seeds, seed)
    out[rank] = (seed, t, rate, tuple(seeds))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    (s0, t0, r0, seeds0), (s1, t1, r1, seeds1) = res[0], res[1]
    assert s0 != s1 and seeds0 == seeds1 == (s0, s1)
    assert t0 == t1 == 1.25          # the slowest rank decides
    assert r0 == r1 == pytest.approx(2 * 100 / 1.25)
