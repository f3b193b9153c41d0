"""Clifford & Clifford samples served by the engine (Sec. 4): every step of a
served chain -- the row draw, the planning and packing of the next minors
job -- runs on the device, interleaved with the other resident requests.
A served sample equals the oracle's chain seed for seed (FP64), equals the
library sampler's sample exactly (every mode), follows the Boson-sampling
distribution (MIXED, chi-square), and can be cancelled."""
import itertools
import time

import numpy as np
import pytest

import oracle
import synthetic as S

pytestmark = pytest.mark.gpu


def _serve(bslib, mode, u, occ, seed, samples, m_detected=0, **kw):
    opts = dict(mem_budget_bytes=512 << 20, max_active=64, tick_tasks=1024)
    opts.update(kw)
    with bslib.Server(0, mode=mode, **opts) as srv:
        tickets = [srv.submit_sample(u, occ, seed, s, m_detected) for s in samples]
        got = [srv.wait_sample(t) for t in tickets]
        st = srv.stats()
    return np.array([g[0] for g in got]), [g[1] for g in got], st


@pytest.mark.parametrize("mode", [0, 2])
def test_served_chains_equal_oracle_sampler(bslib, mode):
    """Served samples 0..99 of one seed draw the oracle's rows, seed for seed,
    except a draw within 1e-9 of a CDF boundary (FP64 and double-float)."""
    u, occ = S.config_cc(n=6, m=12, seed=3)
    ns = 100
    got, lat, st = _serve(bslib, mode, u, occ, 2024, range(ns))
    ref, margin, _ = oracle.cc_sample(u, occ, ns, seed=2024)
    mismatch = [s for s in range(ns) if not np.array_equal(got[s], ref[s])]
    assert all(margin[s] < 1e-9 for s in mismatch), (mismatch, margin[mismatch])
    assert len(mismatch) <= 1
    assert np.all(got.sum(axis=1) == 6)
    assert st["completed"] == ns and st["max_resident"] > 1 and all(x > 0 for x in lat)
    assert st["mem_in_use_bytes"] == 0 and st["resident"] == 0


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_served_chains_equal_library_sampler(ctx, bslib, mode):
    """Served samples plan every step as bs_sample does (same rule, same
    chunking) and draw with the same counters: the counts are identical,
    sample for sample, whatever else shares the ticks.  Collisions (n = 12
    photons in 14 modes) give multi-digit steps."""
    u, occ = S.config_cc(n=12, m=14, seed=17)
    ns = 48
    ref = ctx.sample(u, occ, ns, seed=77, mode=mode)
    got, _, st = _serve(bslib, mode, u, occ, 77, range(ns), tick_tasks=64)
    assert np.array_equal(got, ref)
    assert st["ticks"] > 12
    # out of order and interleaved with another seed's chains
    order = list(range(ns))[::-1]
    with bslib.Server(0, mem_budget_bytes=512 << 20, max_active=16, tick_tasks=256, mode=mode) as srv:
        t = []
        for s in order:
            t.append(srv.submit_sample(u, occ, 77, s))
            srv.submit_sample(u, occ, 5, s)  # released unread when the server closes
        got2 = np.array([srv.wait_sample(x)[0] for x in t])
    assert np.array_equal(got2, ref[order])


@pytest.mark.parametrize("mode", [0, 1])
def test_served_lossy_chains_equal_library_sampler(ctx, bslib, mode):
    """Lossy isometry ((m + n) x n, only the first m rows counted): served
    counts equal sample_ex's."""
    v, mdet = S.config_lossy(n=8, m=16, eta=0.5, seed=48)
    occ = np.ones(8, dtype=np.int32)
    ref = ctx.sample_ex(v, occ, 40, seed=4048, m_detected=mdet, mode=mode)
    got, _, _ = _serve(bslib, mode, v, occ, 4048, range(40), m_detected=mdet)
    assert got.shape == (40, mdet)
    assert np.array_equal(got, ref)


def test_served_mixed_chi_square(bslib):
    """n = 3 photons in m = 5 modes: 6000 served MIXED samples against the
    exact pattern probabilities |per(U_ST)|^2 / prod s! t! (oracle)."""
    st = pytest.importorskip("scipy.stats")
    n, m = 3, 5
    u = S.haar_unitary(m, 31)
    s = np.zeros(m, dtype=np.int32)
    s[:n] = 1
    pats = []
    for c in itertools.combinations_with_replacement(range(m), n):
        t = np.zeros(m, dtype=np.int32)
        for i in c:
            t[i] += 1
        pats.append(t)
    probs = np.array([oracle.bs_probability(u, s, t) for t in pats])
    counts, _, stats = _serve(bslib, 1, u, s, 99, range(6000), max_active=256, tick_tasks=4096)
    assert stats["completed"] == 6000
    index = {tuple(t): i for i, t in enumerate(pats)}
    obs = np.zeros(len(pats))
    for row in counts:
        obs[index[tuple(row)]] += 1
    exp = probs * len(counts)
    keep = exp >= 5
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    chi2 = float(np.sum((o - e) ** 2 / np.maximum(e, 1e-300)))
    assert st.chi2.sf(chi2, len(o) - 1) > 1e-3, chi2


def test_served_degenerate_chains(ctx, bslib):
    """No photons: the empty pattern at once.  One photon: one draw from
    |U_i,c|^2.  Bad arguments are refused."""
    u = S.haar_unitary(6, 2)
    with bslib.Server(0, mem_budget_bytes=64 << 20, max_active=4, tick_tasks=64, mode=0) as srv:
        c, _ = srv.wait_sample(srv.submit_sample(u, np.zeros(6, np.int32), 1, 0))
        assert np.array_equal(c, np.zeros(6, np.int32))
        one = np.zeros(6, np.int32)
        one[4] = 1
        got = np.array([srv.wait_sample(srv.submit_sample(u, one, 8, s))[0] for s in range(20)])
        assert np.array_equal(got, ctx.sample(u, one, 20, seed=8, mode=0))
        with pytest.raises(bslib.BsError) as e:
            srv.submit_sample(u, np.array([1, -1, 0, 0, 0, 0]), 1, 0)
        assert e.value.code == bslib.BS_EINVAL
        t = srv.submit(0, u[:3, :3], np.ones(3), np.ones(3))
        with pytest.raises(bslib.BsError):
            srv.wait_sample(t)  # a permanent's ticket is not a sampling ticket
        srv.wait(t)


def test_server_cancel(ctx, bslib):
    """A waiting request is dropped at once; a running chain is released after
    its current tick (its waiter gets BS_ECANCELED, its memory returns);
    finished tickets cannot be cancelled; the others' results are unchanged."""
    u, occ = S.config_cc(n=34, m=60, seed=3)   # seconds per chain: last steps up to 2^32 addends
    small_u, small_occ = S.config_cc(n=8, m=16, seed=9)
    ref = ctx.sample(small_u, small_occ, 8, seed=3, mode=0)
    with bslib.Server(0, mem_budget_bytes=1 << 30, max_active=2, tick_tasks=256, mode=0) as srv:
        long_t = srv.submit_sample(u, occ, 1, 0)
        long2 = srv.submit_sample(u, occ, 1, 1)
        queued = srv.submit_sample(u, occ, 1, 2)            # waits: two slots
        time.sleep(0.2)
        assert srv.stats()["waiting"] >= 1
        srv.cancel(queued)
        with pytest.raises(bslib.BsError) as e:
            srv.wait_sample(queued)
        assert e.value.code == bslib.BS_ECANCELED
        t0 = time.perf_counter()
        srv.cancel(long_t)
        srv.cancel(long2)
        for t in (long_t, long2):
            with pytest.raises(bslib.BsError) as e:
                srv.wait_sample(t)
            assert e.value.code == bslib.BS_ECANCELED
        assert time.perf_counter() - t0 < 2.0             # a few ticks, not the chains' remaining steps
        st = srv.stats()
        assert st["cancelled"] == 3 and st["resident"] == 0 and st["mem_in_use_bytes"] == 0
        got = np.array([srv.wait_sample(srv.submit_sample(small_u, small_occ, 3, s))[0] for s in range(8)])
        assert np.array_equal(got, ref)
        done = srv.submit(0, u[:4, :4], np.ones(4), np.ones(4))
        srv.wait(done)
        with pytest.raises(bslib.BsError) as e:
            srv.cancel(done)                                # released: unknown ticket
        assert e.value.code == bslib.BS_EINVAL


def test_served_mixed_chains_switch_precision_as_the_sampler_does(ctx, bslib):
    """MIXED at a size where the rule sends some steps to FP32 and others to
    the double-float kernels (n = 24 photons in 10 modes, two or three per
    input mode, so late steps have heavily repeated rows): the served
    samples equal the direct sampler's, so every step took the same
    precision in both."""
    u = S.haar_unitary(10, 19)
    occ = np.array([3, 3, 3, 3, 2, 2, 2, 2, 2, 2], dtype=np.int32)
    ctx.reset_stats()
    ref = ctx.sample(u, occ, 12, seed=9, mode=1)
    st = ctx.stats()
    assert st["addends"][1] > 0 and st["addends"][2] > 0, st["addends"]
    got, _, _ = _serve(bslib, 1, u, occ, 9, range(12), tick_tasks=2048)
    assert np.array_equal(got, ref)


def test_served_mixed_chains_with_reseeded_fp32_steps(ctx, bslib):
    """Late steps of n = 28 chains in m = 40 modes are long FP32 walks (chunks
    of 2^12) that the MIXED rule may keep in FP32 only with in-chunk
    re-seeding, or send to double-float: served samples still equal the
    direct sampler's, step for step."""
    u, occ = S.config_cc(n=28, m=40, seed=23)
    ref = ctx.sample(u, occ, 16, seed=12, mode=1)
    got, _, _ = _serve(bslib, 1, u, occ, 12, range(16), tick_tasks=4096)
    assert np.array_equal(got, ref)
