"""Clifford & Clifford samples served by the continuous-batching engine.

Each request is one sample (Sec. 4; algorithm B of Clifford & Clifford): the
engine keeps the chain's interferometer, permuted inputs and drawn rows on
the device, plans each step's Laplace-minors job there, walks it in the
shared launches of the next ticks together with every other resident
request, and draws the step's row on the device with the counter-based
random numbers of ``bs_sample`` -- nothing of a chain runs on the host.  The
baseline answers the same requests with one ``Context.sample_ex`` call per
sample (all of that sample's launches, calls serialised on one context).

Latency of a request: its arrival (submission) until its counts are
available.
"""
from __future__ import annotations

import threading
import time

import numpy as np

from . import BS_FP64, Context, Server


def _arrive(t0, at):
    delay = t0 + at - time.perf_counter()
    if delay > 0:
        time.sleep(delay)


def run_served(requests, server: Server, m_detected: int = 0):
    """requests: dicts with ``unitary``, ``occupation``, ``seed``, ``sample``
    (optional, default 0) and ``arrival_s``.  One submitter thread submits at
    the arrival offsets; the engine's own clock gives each latency.  Returns
    (wall seconds, latencies, counts per request)."""
    tickets = [None] * len(requests)
    t0 = time.perf_counter()

    def submitter():
        for i, r in enumerate(requests):
            _arrive(t0, r["arrival_s"])
            tickets[i] = server.submit_sample(r["unitary"], r["occupation"], r["seed"], r.get("sample", 0),
                                              m_detected)

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    lat, counts = [], []
    for t in tickets:
        c, l = server.wait_sample(t)
        counts.append(c)
        lat.append(l)
    return time.perf_counter() - t0, lat, counts


def run_one_call_per_sample(requests, ctx: Context, mode=BS_FP64, m_detected: int = 0):
    """Baseline: every request is one sample_ex call with n_samples = 1,
    issued at its arrival; calls are serialised on the context, so a request
    that arrives while another runs waits for it.  Returns (wall seconds,
    latencies, counts)."""
    lat, counts = [], []
    t0 = time.perf_counter()
    for r in requests:
        _arrive(t0, r["arrival_s"])
        if r.get("sample", 0) != 0:
            raise ValueError("the one-call baseline draws sample 0 of each seed")
        c = ctx.sample_ex(r["unitary"], r["occupation"], 1, r["seed"], m_detected=m_detected, mode=mode)[0]
        counts.append(c)
        lat.append(time.perf_counter() - (t0 + r["arrival_s"]))
    return time.perf_counter() - t0, lat, counts


def summarize(wall, lat, nsamples):
    lat_ms = np.sort(np.asarray(lat) * 1e3) if lat else np.zeros(1)
    return {"samples_per_s": nsamples / wall, "wall_s": wall, "requests": len(lat),
            "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
            "max_ms": float(lat_ms[-1])}
