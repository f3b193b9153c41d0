"""Serving engine (continuous batching): results are bit-identical alone and
in the mix, admission respects slots and the memory budget, and requests
that arrive while long ones run are served at the next tick."""
import threading
import time

import numpy as np
import pytest

import oracle
import synthetic as S

pytestmark = pytest.mark.gpu


def _mixed_requests(seed, count, kmin, kmax):
    g = S.rng(seed)
    reqs = []
    u = S.haar_unitary(60, seed)
    for i in range(count):
        k = int(g.integers(kmin, kmax + 1))
        cols = np.sort(g.choice(60, size=k, replace=False))
        rows, mult = S.collapse_modes(k - (i % 2), 60, g)
        a = u[np.ix_(rows, cols)]
        N = np.ones(k, dtype=np.int32)
        reqs.append((i % 2, a, mult, N))   # even: permanent, odd: minors
    return reqs


@pytest.mark.parametrize("mode", [0, 1])
def test_server_results_identical_alone_and_mixed(ctx, bslib, mode):
    """Each request gives the same bits when it is the only one on the server
    and when it runs mixed with 39 others (the server's chunking depends only
    on the request); every result is also within the parity tolerance of the
    direct entry points and of the oracle."""
    reqs = _mixed_requests(5, 40, 6, 20)
    with bslib.Server(0, mem_budget_bytes=256 << 20, max_active=16, tick_tasks=512, mode=mode) as srv:
        tickets = [srv.submit(kind, a, M, N) for kind, a, M, N in reqs]
        mixed = [srv.wait(t)[0] for t in tickets]
        st = srv.stats()
        alone = [srv.wait(srv.submit(kind, a, M, N))[0] for kind, a, M, N in reqs]
    assert st["completed"] == len(reqs) and st["max_resident"] > 1
    tol = 1e-10 if mode == 0 else 1e-6
    for (kind, a, M, N), got, ref in zip(reqs, mixed, alone):
        assert np.array_equal(got, ref)
        direct = ctx.perm(a, M, N, mode=mode) if kind == 0 else ctx.laplace_minors(a, M, N, mode=mode)
        norms = np.sqrt((np.abs(a) ** 2 * M[:, None]).sum(axis=0))
        assert np.all(np.abs(np.atleast_1d(direct) - got) <= 10 * tol * np.prod(norms ** N))
    kind, a, M, N = reqs[0]
    v, t = oracle.perm_mult(a, M, N)
    norms = np.sqrt((np.abs(a) ** 2 * M[:, None]).sum(axis=0))
    assert abs(mixed[0][0] - (v + t)) <= tol * np.prod(norms ** N)


def test_server_admission_by_memory_and_too_large(bslib):
    u = S.haar_unitary(48, 3)
    a = u[:24, :24]
    ones = np.ones(24, dtype=np.int32)
    # a 24x24 permanent needs ~150 KB (4096 task partials + matrices); a
    # 512 KiB budget holds three at a time, the rest wait for memory
    with bslib.Server(0, mem_budget_bytes=512 << 10, max_active=64, tick_tasks=256, mode=0) as srv:
        tickets = [srv.submit(0, a, ones, ones) for _ in range(12)]
        vals = [srv.wait(t)[0][0] for t in tickets]
        st = srv.stats()
        assert st["mem_peak_bytes"] <= 512 << 10 and 1 <= st["max_resident"] < 12
        assert all(v == vals[0] for v in vals)
        # 40x40 needs 2^22 task partials (128 MiB): it can never be admitted
        big = u[:40, :40]
        t = srv.submit(0, big, np.ones(40, np.int32), np.ones(40, np.int32))
        with pytest.raises(bslib.BsError) as e:
            srv.wait(t)
        assert e.value.code == bslib.BS_ENOMEM


def test_server_short_requests_overtake_a_long_one(bslib):
    u = S.haar_unitary(40, 4)
    big = u[:29, :29]
    ones29 = np.ones(29, dtype=np.int32)
    small = u[:10, :10]
    ones10 = np.ones(10, dtype=np.int32)
    # small ticks: the long request (2048 tasks) spans many of them
    with bslib.Server(0, mem_budget_bytes=1 << 30, max_active=16, tick_tasks=128, mode=0) as srv:
        long_t = srv.submit(0, big, ones29, ones29)
        time.sleep(0.05)                    # the long request is already running
        shorts = [srv.submit(0, small, ones10, ones10) for _ in range(8)]
        short_done = []
        for t in shorts:
            _, lat = srv.wait(t)
            short_done.append(time.perf_counter())
        _, long_lat = srv.wait(long_t)
        long_done = time.perf_counter()
    assert max(short_done) < long_done
    assert long_lat > 0


def test_server_many_client_threads(bslib):
    reqs = _mixed_requests(9, 48, 8, 18)
    out = [None] * len(reqs)
    with bslib.Server(0, mem_budget_bytes=512 << 20, max_active=32, tick_tasks=1024, mode=1) as srv:
        def client(idx):
            for i in range(idx, len(reqs), 8):
                kind, a, M, N = reqs[i]
                out[i] = srv.wait(srv.submit(kind, a, M, N))[0]
        th = [threading.Thread(target=client, args=(c,)) for c in range(8)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        st = srv.stats()
    assert all(o is not None for o in out) and st["completed"] == len(reqs)
