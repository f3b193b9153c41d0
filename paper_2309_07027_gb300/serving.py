"""Clifford & Clifford sampling chains as clients of the serving engine.

Each chain samples one output pattern (Sec. 4; algorithm B of Clifford &
Clifford): it permutes its input photons, and for k = 1..n asks for the
Laplace minors of the (k-1) x k matrix of rows drawn so far (row
multiplicities = collisions) and the first k permuted input columns, then
draws row k with probability |sum_l U[i, col_l] minor_l|^2.  The minors come
from the library -- either from a ``Server`` (continuous batching across
all chains) or from one ``Context.laplace_minors`` call per request (the
one-launch-per-permanent form).  Only the draw (m weights of k terms) runs
on the host.

Every request records its latency (request issued -> result available).
"""
from __future__ import annotations

import threading
import time

import numpy as np

from . import BS_FP64, Context, Server


class Chain:
    def __init__(self, unitary, occupation, seed):
        self.u = np.ascontiguousarray(unitary, dtype=np.complex128)
        occ = np.asarray(occupation, dtype=np.int64)
        inputs = np.repeat(np.arange(len(occ)), occ)
        self.rng = np.random.Generator(np.random.PCG64(seed))
        self.cols = self.rng.permutation(inputs)
        self.n = len(inputs)
        self.rows = []

    @property
    def done(self):
        return len(self.rows) == self.n

    def request(self):
        """(A, row_mult, col_mult) of the next step's minors, or None at k = 1."""
        k = len(self.rows) + 1
        if k == 1:
            return None
        modes, counts = np.unique(np.asarray(self.rows), return_counts=True)
        a = self.u[np.ix_(modes, self.cols[:k])]
        return a, counts.astype(np.int32), np.ones(k, dtype=np.int32)

    def advance(self, minors):
        k = len(self.rows) + 1
        amp = self.u[:, self.cols[:k]] @ (np.ones(1) if minors is None else minors)
        w = np.abs(amp) ** 2
        self.rows.append(int(self.rng.choice(len(w), p=w / w.sum())))

    def occupation(self):
        out = np.zeros(self.u.shape[0], dtype=np.int32)
        for r in self.rows:
            out[r] += 1
        return out


def _run(chains, arrivals, answer):
    """Runs every chain in its own thread, starting at its arrival offset;
    answer(chain, request) -> minors.  Returns (wall seconds, latencies)."""
    lat = []
    lock = threading.Lock()
    t0 = time.perf_counter()

    def worker(ch, at):
        delay = t0 + at - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        mine = []
        while not ch.done:
            req = ch.request()
            if req is None:
                ch.advance(None)
                continue
            ts = time.perf_counter()
            minors = answer(ch, req)
            mine.append(time.perf_counter() - ts)
            ch.advance(minors)
        with lock:
            lat.extend(mine)

    th = [threading.Thread(target=worker, args=(c, a)) for c, a in zip(chains, arrivals)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return time.perf_counter() - t0, lat


def run_served(chains, arrivals, server: Server):
    def answer(ch, req):
        a, M, N = req
        out, _ = server.wait(server.submit(1, a, M, N))
        return out
    return _run(chains, arrivals, answer)


def run_one_call_per_permanent(chains, arrivals, ctx: Context, mode=BS_FP64):
    """Baseline: every request is one bs_laplace_minors call (its own
    launches); calls are serialised on the context."""
    lock = threading.Lock()

    def answer(ch, req):
        a, M, N = req
        with lock:
            return ctx.laplace_minors(a, M, N, mode=mode)
    return _run(chains, arrivals, answer)


def summarize(wall, lat, nsamples):
    lat_ms = np.sort(np.asarray(lat) * 1e3) if lat else np.zeros(1)
    return {"samples_per_s": nsamples / wall, "wall_s": wall, "requests": len(lat),
            "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
            "max_ms": float(lat_ms[-1])}
