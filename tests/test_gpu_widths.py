"""GPU parity of the MIXED (FP32) kernels at the widths the sampling and
batch workloads run them, against the oracle; the sampler's drawn rows at
the n = 30, m = 60 workload size against the oracle's chains; the
power-of-two column normalisation at extreme ranges; and the lossy sampler
against binomial thinning of the ideal one (Sec. 4 loss model).

Oracle references:
  * dense matrices: oracle.perm_mult of the matrix with one column removed
    (Eq. bbfgrepeated term by term), for a few minors per width -- the oracle
    evaluates about 4e4 addends per second per core, and the cheapest
    patterns the MIXED rule keeps in FP32 grow from 9e4 addends at K = 24 to
    4e7 at K = 36, so dense MIXED cases stop at K = 29 (bucket 32);
  * block-diagonal matrices (FP64, every width up to 48): the expanded matrix is
    block diagonal, so its permanent is the product of the block permanents
    and a minor is the deficit block's minor times the other blocks'
    permanents (zero when the removed column lies in a square block); each
    block is a small oracle call.

Tolerances as in test_gpu_parity: |err| <= 1e-10 (FP64) / 1e-6 (MIXED) times
prod_j ||a_j||^{N_j} with column norms over the rows repeated by their
multiplicities.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic as S

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-6, 2: 1e-10}  # FP64, MIXED, double-float


def scale(a, M, N):
    norms = np.sqrt((np.abs(np.asarray(a)) ** 2 * np.asarray(M)[:, None]).sum(axis=0))
    return float(np.prod(norms ** np.asarray(N)))


def minor_scale(a, M, N, l):
    N2 = np.array(N).copy()
    N2[l] -= 1
    return scale(a, M, N2)


def keeps_fp32(bslib, M, K, kind):
    """The library's MIXED rule for the problem planned alone (host-only
    helper): True when the default tolerance keeps it in the FP32 kernels."""
    return bslib.debug_mixed_error(np.asarray(M, np.int32), np.ones(K, np.int32), kind)[2]


def block_reference(a, M, N, groups, kind):
    """Oracle values of a block-diagonal problem: (perm,) or minors[K]."""
    vals = []
    for rows, cols in groups:
        blk = a[np.ix_(rows, cols)]
        Mb, Nb = M[rows], N[cols]
        if int(Mb.sum()) == int(Nb.sum()):
            v, t = oracle.perm_mult(blk, Mb, Nb)
            vals.append(("perm", cols, v + t))
        else:
            v, t = oracle.minors(blk, Mb, Nb)
            vals.append(("minors", cols, v + t))
    if kind == 0:
        return np.prod([x for tag, _, x in vals])
    K = a.shape[1]
    out = np.zeros(K, dtype=np.complex128)
    others = np.prod([x for tag, _, x in vals if tag == "perm"])
    for tag, cols, x in vals:
        if tag == "minors":
            out[cols] = x * others
    return out


def run_checked(ctx, fn, mode, want_fp32):
    ctx.reset_stats()
    got = fn()
    st = ctx.stats()
    if mode == 1 and want_fp32:
        assert st["addends"][1] > 0 and st["addends"][0] == 0, "expected the FP32 kernel"
    return got


# ---------------------------------------------------------------- dense, direct oracle
# (K, row multiplicities): the cheapest patterns the MIXED rule keeps in FP32
# at these widths (buckets 24, 28, 32), 9e4 - 1.1e6 addends per minor; the
# oracle's minors run in spawned processes, one per minor.
DENSE_MINORS = [
    (24, [3, 3, 3] + [2] * 6 + [1] * 2, (0, 12, 23)),
    (26, [3, 3, 3] + [2] * 7 + [1] * 2, (0, 25)),
    (28, [3, 3, 3, 3] + [2] * 6 + [1] * 3, (0, 27)),
    (29, [3, 3, 3, 3] + [2] * 7 + [1] * 2, (14,)),
]


def _dense_case(K, M):
    M = np.array(M, dtype=np.int32)
    g = S.rng(4200 + K)
    u = S.haar_unitary(64, 4300 + K)
    a = u[g.permutation(64)[: len(M)]][:, g.permutation(64)[:K]]
    return a, M, np.ones(K, dtype=np.int32)


def _oracle_minor(job):
    """One oracle minor (pool worker, importable by a spawned process)."""
    K, M, l = job
    a, M, N = _dense_case(K, M)
    keep = [j for j in range(K) if j != l]
    v, t = oracle.perm_mult(a[:, keep], M, N[keep])
    return K, l, v + t


@pytest.fixture(scope="module")
def dense_oracle_minors():
    import multiprocessing as mp
    import os
    jobs = [(K, M, l) for K, M, ls in DENSE_MINORS for l in ls]
    procs = max(1, min(len(jobs), len(os.sched_getaffinity(0))))
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map_async(_oracle_minor, jobs, chunksize=1).get(timeout=1200)
    return {(K, l): v for K, l, v in res}


@pytest.mark.parametrize("K,M,ls", DENSE_MINORS)
def test_fp32_minors_dense_against_oracle(ctx, bslib, dense_oracle_minors, K, M, ls):
    """MIXED fused minors in the FP32 kernels (checked from the statistics)
    on a dense Haar block at the headline kernel widths, against the oracle's
    permanent of the column-deleted matrix, within the MIXED tolerance."""
    a, M, N = _dense_case(K, M)
    assert int(M.sum()) == K - 1 and keeps_fp32(bslib, M, K, 1)
    got = run_checked(ctx, lambda: ctx.laplace_minors(a, M, N, mode=1), 1, True)
    for l in ls:
        ref = dense_oracle_minors[(K, l)]
        assert abs(got[l] - ref) <= TOL[1] * minor_scale(a, M, N, l), (K, l, got[l], ref)


def test_fp32_perm_dense_against_oracle(ctx, bslib):
    """MIXED permanent of a dense 24-column Haar block in the FP32 kernel."""
    K = 24
    M = np.array([3, 3, 3] + [2] * 6 + [1] * 3, dtype=np.int32)
    assert keeps_fp32(bslib, M, K, 0)
    g = S.rng(4400)
    u = S.haar_unitary(64, 4401)
    a = u[g.permutation(64)[: len(M)]][:, g.permutation(64)[:K]]
    N = np.ones(K, dtype=np.int32)
    got = run_checked(ctx, lambda: ctx.perm(a, M, N, mode=1), 1, True)
    v, t = oracle.perm_mult(a, M, N)
    assert abs(got - (v + t)) <= TOL[1] * scale(a, M, N), (got, v)


# ---------------------------------------------------------------- block diagonal, every width
# Block-diagonal inputs cancel far more than unstructured ones (the modulus-
# sum of the addends exceeds the permanent by up to 6e6 at K = 48), so they
# pin the FP64 and double-float kernels at every width, not the FP32 ones.
BLOCK_WIDTHS = [13, 17, 21, 24, 25, 28, 29, 30, 32, 33, 36, 37, 40, 41, 44, 45, 48]


def block_case(K, n, seed):
    mult = 3 if K >= 25 else 2
    return S.block_diagonal(K, n, seed, width=12, mult=mult)


@pytest.mark.parametrize("mode", [0, 2])
@pytest.mark.parametrize("K", BLOCK_WIDTHS)
def test_minors_block_diagonal_every_width(ctx, mode, K):
    a, M, N, groups = block_case(K, K - 1, 4500 + K)
    got = ctx.laplace_minors(a, M, N, mode=mode)
    ref = block_reference(a, M, N, groups, 1)
    for l in range(K):
        assert abs(got[l] - ref[l]) <= TOL[mode] * minor_scale(a, M, N, l), (K, l, got[l], ref[l])


@pytest.mark.parametrize("mode", [0, 2])
@pytest.mark.parametrize("K", BLOCK_WIDTHS)
def test_perm_block_diagonal_every_width(ctx, mode, K):
    a, M, N, groups = block_case(K, K, 4600 + K)
    got = ctx.perm(a, M, N, mode=mode)
    ref = block_reference(a, M, N, groups, 0)
    assert abs(got - ref) <= TOL[mode] * scale(a, M, N), (K, got, ref)


# ---------------------------------------------------------------- FP32 re-seeding inside chunks
def test_mixed_reseeded_fp32_meets_the_drift_free_prediction(ctx, bslib):
    """A 29 x 30 minors job (2^28 addends) is walked by the FP32 kernel in
    chunks of 2^11 addends.  With the MIXED tolerance set between the rule's
    prediction without and with its drift term, the rule keeps the job in
    FP32 and has the kernel re-seed its column sums every 2^8 steps; the
    error (against the FP64 kernel, itself checked against the oracle at
    this width) then stays below the drift-free prediction, the bound of
    chunks of 2^8 addends."""
    K = 30
    a = S.haar_unitary(64, 4900)[:K - 1, :K]
    M = np.ones(K - 1, dtype=np.int32)
    N = np.ones(K, dtype=np.int32)
    e, L, _ = bslib.debug_mixed_error(M, N, 1)
    e8, _, _ = bslib.debug_mixed_error(M, N, 1, chunk_log2=8)
    assert L > 8 and e - e8 == pytest.approx(0.5 * (L - 8), abs=1e-4)
    ref = ctx.laplace_minors(a, M, N, mode=0)
    try:
        ctx.set_mixed_tolerance(2.0 ** ((e + e8) / 2))
        got = run_checked(ctx, lambda: ctx.laplace_minors(a, M, N, mode=1), 1, True)
    finally:
        ctx.set_mixed_tolerance(1e-6)
    err = max(abs(got[l] - ref[l]) / minor_scale(a, M, N, l) for l in range(K))
    assert 0 < err <= 2.0 ** e8, (err, 2.0 ** e8)


def test_mixed_reseeded_fp32_sweep(ctx, bslib):
    """Ten long-chunk FP32 jobs (K = 27..32, up to three repeated rows,
    permanents and minors), each run with the MIXED tolerance between its
    two predictions: every one runs in FP32 with in-chunk re-seeding and
    stays below its drift-free prediction (errors against the FP64
    kernels)."""
    g = np.random.default_rng(2719)
    done = 0
    for trial in range(40):
        if done == 10:
            break
        kind = trial % 2
        K = int(g.integers(27, 33))
        n = K - kind
        nrep = int(g.integers(0, 4))
        M = np.ones(n - nrep, np.int32)
        for _ in range(nrep):
            M[int(g.integers(0, len(M)))] += 1
        N = np.ones(K, np.int32)
        e, L, _ = bslib.debug_mixed_error(M, N, kind)
        e8, _, _ = bslib.debug_mixed_error(M, N, kind, chunk_log2=8)
        if L <= 8:
            continue
        u = S.haar_unitary(80, 9100 + trial)
        a = u[g.permutation(80)[:len(M)]][:, g.permutation(80)[:K]]
        call = (lambda md: ctx.perm(a, M, N, mode=md)) if kind == 0 else \
            (lambda md: ctx.laplace_minors(a, M, N, mode=md))
        ref = np.atleast_1d(call(0))
        try:
            ctx.set_mixed_tolerance(2.0 ** ((e + e8) / 2))
            got = np.atleast_1d(run_checked(ctx, lambda: call(1), 1, True))
        finally:
            ctx.set_mixed_tolerance(1e-6)
        if kind == 0:
            err = abs(got[0] - ref[0]) / scale(a, M, N)
        else:
            err = max(abs(got[l] - ref[l]) / minor_scale(a, M, N, l) for l in range(K))
        assert err <= 2.0 ** e8, (K, M.tolist(), L, err, 2.0 ** e8)
        done += 1
    assert done == 10


def test_mixed_reseeded_fp32_permanent(ctx, bslib):
    """The permanent kernel's re-seed segments: a 30 x 30 permanent (2^29
    addends, FP32 chunks of 2^11) with the tolerance between the rule's two
    predictions runs in FP32 re-seeded every 2^8 steps and stays below the
    drift-free prediction (against the FP64 kernel)."""
    n = 30
    a = S.haar_unitary(64, 4950)[:n, :n]
    ones = np.ones(n, dtype=np.int32)
    e, L, _ = bslib.debug_mixed_error(ones, ones, 0)
    e8, _, _ = bslib.debug_mixed_error(ones, ones, 0, chunk_log2=8)
    assert L > 8
    ref = ctx.perm(a, ones, ones, mode=0)
    try:
        ctx.set_mixed_tolerance(2.0 ** ((e + e8) / 2))
        got = run_checked(ctx, lambda: ctx.perm(a, ones, ones, mode=1), 1, True)
    finally:
        ctx.set_mixed_tolerance(1e-6)
    err = abs(got - ref) / scale(a, ones, ones)
    assert 0 < err <= 2.0 ** e8, (err, 2.0 ** e8)


# ---------------------------------------------------------------- power-of-two column normalisation
@pytest.mark.parametrize("kind", ["pow2", "decimal"])
def test_mixed_column_normalisation_extreme_ranges(ctx, bslib, kind):
    """FP32 column sums cover about 1e-38..3e38.  Columns scaled by 2^+-100
    or 1e+-30 would overflow or underflow unscaled FP32 products; the pack
    kernel scales every FP32 column by a power of two (Appendix A.5
    normalises for the same reason).  Checked against the oracle: for 2^+-100
    the exact rescaled oracle value of the unscaled matrix, for 1e+-30 the
    oracle on the scaled matrix itself."""
    K = 16
    u = S.haar_unitary(32, 4700)
    M = np.array([2, 2, 2] + [1] * 10, dtype=np.int32)
    a0 = u[:13, :K]
    N = np.ones(K, dtype=np.int32)
    assert keeps_fp32(bslib, M, K, 0)
    if kind == "pow2":
        ex = np.array([100 if j % 2 == 0 else -100 for j in range(K)])
        a = a0 * np.ldexp(1.0, ex)[None, :]
        v, t = oracle.perm_mult(a0, M, N)
        ref = (v + t) * math.ldexp(1.0, int(ex.sum()))
        sc = scale(a0, M, N) * math.ldexp(1.0, int(ex.sum()))
    else:
        f = np.array([1e30 if j % 2 == 0 else 1e-30 for j in range(K)])
        a = a0 * f[None, :]
        v, t = oracle.perm_mult(a, M, N)
        ref = v + t
        sc = scale(a, M, N)
    got = run_checked(ctx, lambda: ctx.perm(a, M, N, mode=1), 1, True)
    assert np.isfinite(got) and abs(got - ref) <= TOL[1] * sc, (kind, got, ref)
    # minors of the same matrix with one photon fewer in the first row
    M2 = M.copy()
    M2[0] -= 1
    got_m = run_checked(ctx, lambda: ctx.laplace_minors(a, M2, N, mode=1), 1, True)
    for l in (0, 1, K - 1):
        keep = [j for j in range(K) if j != l]
        v, t = oracle.perm_mult(a[:, keep], M2, N[keep])
        assert abs(got_m[l] - (v + t)) <= TOL[1] * minor_scale(a, M2, N, l), (kind, l)


# ---------------------------------------------------------------- sampler rows at the workload size
# draw margins below which a row may legitimately differ from the oracle's:
# the mode's error in the CDF (FP64 ~1e-13 relative; MIXED minors ~1e-10
# prod ||a_j||, i.e. ~1e-7 of a k <= 18 weight, with headroom)
MARGIN = {0: 1e-9, 1: 1e-5, 2: 1e-9}
TRACE_STEPS, TRACE_SAMPLES = 18, 8


@pytest.fixture(scope="module")
def oracle_trace():
    u, occ = S.config_cc(n=30, m=60, seed=3)
    _, _, _, rows, smargin = oracle.cc_sample(u, occ, TRACE_SAMPLES, seed=7, max_steps=TRACE_STEPS, trace=True)
    return u, occ, rows, smargin


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_sampler_rows_match_oracle_at_workload_size(ctx, oracle_trace, mode):
    """n = 30 photons, m = 60 modes (the sampling workload): the drawn row
    r_k of every step k <= 18 of every chain equals the oracle chain's, seed
    for seed.  A chain may leave the oracle's path only at a step whose
    oracle draw lies within the mode's error margin of a CDF boundary (after
    that the chains condition on different rows); such departures are
    counted and capped at one."""
    u, occ, ref_rows, ref_margin = oracle_trace
    counts, rows = ctx.sample_trace(u, occ, TRACE_SAMPLES, seed=7, mode=mode)
    assert rows.shape == (TRACE_SAMPLES, 30)
    for s in range(TRACE_SAMPLES):
        assert np.array_equal(np.bincount(rows[s], minlength=60), counts[s])
    departures = 0
    for s in range(TRACE_SAMPLES):
        diff = np.nonzero(rows[s, :TRACE_STEPS] != ref_rows[s])[0]
        if len(diff) == 0:
            continue
        k = int(diff[0])
        assert ref_margin[s, k] < MARGIN[mode], (mode, s, k, rows[s, :k + 1], ref_rows[s, :k + 1],
                                                 ref_margin[s, k])
        departures += 1
    assert departures <= 1, departures


def _check_rows(rows, ref_rows, ref_margin, steps, margin, max_departures):
    departures = 0
    for s in range(len(ref_rows)):
        diff = np.nonzero(rows[s, :steps] != ref_rows[s, :steps])[0]
        if len(diff) == 0:
            continue
        k = int(diff[0])
        assert ref_margin[s, k] < margin, (s, k, rows[s, :k + 1], ref_rows[s, :k + 1], ref_margin[s, k])
        departures += 1
    assert departures <= max_departures, departures


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_sampler_rows_match_oracle_in_the_bench_launch(ctx, oracle_trace, mode):
    """The benchmark's launch configuration: 200 chains of the n = 30, m = 60
    workload advance together (one walk launch per precision and step for
    all of them).  A chain's random numbers depend only on (seed, sample
    index), so chains 0..7 of the 200 are the oracle's chains 0..7: their
    first 18 rows match, with the same departure rule."""
    u, occ, ref_rows, ref_margin = oracle_trace
    counts, rows = ctx.sample_trace(u, occ, 200, seed=7, mode=mode)
    assert rows.shape == (200, 30) and np.all(counts.sum(axis=1) == 30)
    _check_rows(rows[:TRACE_SAMPLES], ref_rows, ref_margin, TRACE_STEPS, MARGIN[mode], 1)


def test_lossy_sampler_rows_match_oracle_at_workload_size(ctx):
    """The lossy workload at full size (n = 40 photons, m = 60 modes,
    eta = 0.5, the 100 x 40 isometry, MIXED as the lossy benchmark runs it):
    the first 16 rows of four chains equal the oracle's lossy chains (loss
    modes included), with the same departure rule."""
    v, mdet = S.config_lossy()
    occ = np.ones(v.shape[1], dtype=np.int32)
    steps, ns = 16, 4
    _, _, _, ref_rows, ref_margin = oracle.cc_sample(v, occ, ns, seed=41, m_detected=mdet, max_steps=steps,
                                                     trace=True)
    counts, rows = ctx.sample_trace(v, occ, ns, seed=41, m_detected=mdet, mode=1)
    assert rows.shape == (ns, 40) and counts.shape == (ns, mdet)
    for s in range(ns):
        assert np.array_equal(np.bincount(rows[s][rows[s] < mdet], minlength=mdet), counts[s])
    _check_rows(rows, ref_rows, ref_margin, steps, MARGIN[1], 0)


def test_sampler_trace_equals_plain_sampler(ctx):
    """bs_sample_trace draws exactly what bs_sample_ex draws."""
    u, occ = S.config_cc(n=10, m=20, seed=8)
    for mode in (0, 1):
        counts, rows = ctx.sample_trace(u, occ, 32, seed=21, mode=mode)
        assert np.array_equal(counts, ctx.sample_ex(u, occ, 32, seed=21, mode=mode))
        assert rows.shape == (32, 10) and np.all(rows >= 0) and np.all(rows < 20)


# ---------------------------------------------------------------- lossy sampler vs thinning
def _patterns(m, nmax):
    import itertools
    pats = [np.zeros(m, dtype=np.int32)]
    for k in range(1, nmax + 1):
        for c in itertools.combinations_with_replacement(range(m), k):
            t = np.zeros(m, dtype=np.int32)
            for i in c:
                t[i] += 1
            pats.append(t)
    return pats


def test_lossy_sampler_matches_binomial_thinning(ctx):
    """Uniform loss commutes with the interferometer, so lossy sampling with
    transmissivity eta equals ideal sampling followed by losing each output
    photon independently with probability 1 - eta (the loss model of Sec. 4).
    (1) The exact detected-pattern distribution, from the oracle's ideal
    probabilities thinned binomially, against bs_sample_ex on the lossy
    isometry (chi-square); (2) the GPU's ideal samples thinned on the host
    against the GPU's lossy samples (two-sample chi-square)."""
    st = pytest.importorskip("scipy.stats")
    n, m, eta = 4, 6, 0.5
    u = S.haar_unitary(m, 4800)
    occ = np.zeros(m, dtype=np.int32)
    occ[:n] = 1
    pats = _patterns(m, n)
    index = {tuple(t): i for i, t in enumerate(pats)}
    ideal = [t for t in pats if t.sum() == n]
    p_ideal = np.array([oracle.bs_probability(u, occ, t) for t in ideal])
    assert abs(p_ideal.sum() - 1.0) < 1e-12
    # exact thinned distribution: P(d) = sum_t p(t) prod_i C(t_i, d_i) eta^|d| (1-eta)^(n-|d|)
    p_det = np.zeros(len(pats))
    import itertools
    for t, p in zip(ideal, p_ideal):
        for d in itertools.product(*[range(int(x) + 1) for x in t]):
            d = np.array(d, dtype=np.int32)
            w = np.prod([math.comb(int(a), int(b)) for a, b in zip(t, d)])
            p_det[index[tuple(d)]] += p * w * eta ** int(d.sum()) * (1 - eta) ** int(n - d.sum())
    assert abs(p_det.sum() - 1.0) < 1e-12
    v = S.lossy_isometry(u, np.arange(n), eta)
    ns = 40000
    lossy = ctx.sample_ex(v, np.ones(n, np.int32), ns, seed=4801, m_detected=m, mode=0)
    obs = np.zeros(len(pats))
    for row in lossy:
        obs[index[tuple(row)]] += 1
    exp = p_det * ns
    keep = exp >= 5
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    chi2 = float(np.sum((o - e) ** 2 / np.maximum(e, 1e-300)))
    assert st.chi2.sf(chi2, len(o) - 1) > 1e-3, chi2
    # (2) thinning of the GPU's ideal samples, two-sample test
    ideal_s = ctx.sample(u, occ, ns, seed=4802, mode=0)
    g = S.rng(4803)
    thinned = g.binomial(ideal_s, eta)
    obs2 = np.zeros(len(pats))
    for row in thinned:
        obs2[index[tuple(row)]] += 1
    table = np.vstack([obs[keep], obs2[keep]])
    table = np.hstack([table, [[obs[~keep].sum()], [obs2[~keep].sum()]]])
    table = table[:, table.sum(axis=0) > 0]
    _, pval, _, _ = st.chi2_contingency(table)
    assert pval > 1e-3, pval


def test_mixed_sampler_agrees_with_fp64_at_workload_size(ctx):
    """The sampling workload in full (n = 30, m = 60, 200 samples, all 30
    steps, including the late steps whose FP32 jobs are re-seeded inside
    their chunks and those the rule sends to the double-float kernels): a
    MIXED chain leaves the FP64 chain's rows only at a draw that falls within
    MIXED's error of a CDF boundary, so almost every sample is identical."""
    u, occ = S.config_cc(n=30, m=60, seed=3)
    _, r64 = ctx.sample_trace(u, occ, 200, seed=61, mode=0)
    ctx.reset_stats()
    _, rmx = ctx.sample_trace(u, occ, 200, seed=61, mode=1)
    st = ctx.stats()
    assert st["addends"][1] > 0 and st["addends"][2] > 0, st["addends"]
    same = float(np.mean(np.all(r64 == rmx, axis=1)))
    assert same >= 0.9, same


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_sampler_under_a_small_budget_runs_in_passes(ctx, bslib, mode):
    """A context with a 16 MiB device budget cannot hold the partial slots of
    200 chains of n = 20 photons at once (about 80 KB each), so bs_sample
    runs them in passes of a few dozen chains: every sample equals the one
    drawn by an unbounded context (chains depend only on seed and index)."""
    u, occ = S.config_cc(n=20, m=40, seed=13)
    ref = ctx.sample(u, occ, 200, seed=31, mode=mode)
    small = bslib.Context(0, mem_budget_bytes=16 << 20)
    try:
        got = small.sample(u, occ, 200, seed=31, mode=mode)
    finally:
        small.close()
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_sampler_at_the_largest_output_mode_count(ctx, bslib, mode):
    """m = 8192 output modes (the largest supported; the draw's weights then
    need more than 48 KB of shared memory): an isometry with 6 input columns,
    sampled by bs_sample_ex and by a server, equals the oracle's chains seed
    for seed (up to a draw within the mode's margin of a CDF boundary)."""
    g = S.rng(8192)
    q, _ = np.linalg.qr(g.standard_normal((8192, 6)) + 1j * g.standard_normal((8192, 6)))
    v = np.ascontiguousarray(q)
    occ = np.ones(6, dtype=np.int32)
    ns = 16
    ref, margin, _ = oracle.cc_sample(v, occ, ns, seed=88)
    got = ctx.sample_ex(v, occ, ns, seed=88, mode=mode)
    bad = [s for s in range(ns) if not np.array_equal(got[s], ref[s])]
    assert all(margin[s] < MARGIN[mode] for s in bad) and len(bad) <= 1, (bad, margin[bad])
    with bslib.Server(0, mem_budget_bytes=512 << 20, max_active=8, tick_tasks=256, mode=mode) as srv:
        served = np.array([srv.wait_sample(t)[0] for t in [srv.submit_sample(v, occ, 88, s) for s in range(4)]])
    assert np.array_equal(served, got[:4])
