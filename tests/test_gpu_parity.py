"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (from the accuracy targets of the method, Sec. 3.2):
  FP64 and double-float modes
              |perm_gpu - perm_oracle| <= 1e-10 * prod_j ||a_j||_2^{N_j}
  MIXED mode  |perm_gpu - perm_oracle| <= 1e-6  * prod_j ||a_j||_2^{N_j}
with ||a_j|| the 2-norm of column j over the rows repeated by their
multiplicities (a Hadamard-type scale of the permanent).  Heavily repeated
rows make the addends cancel far below that scale; there the rounding
error is bounded by the modulus-sum of the addends S_abs (oracle
perm_mult_abs): each addend carries a relative error of about K u, so
|error| <= TOL_L1 * S_abs with TOL_L1 = 1e-12 (FP64; K <= 48, u = 2^-53,
plus the re-seeded column-sum drift).  MIXED mode sends such jobs to the
FP64 kernels, so the same bound applies to them.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic as S

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-6, 2: 1e-10}  # FP64, MIXED, double-float
TOL_L1 = 1e-12


def scale(a, M, N):
    a = np.asarray(a)
    M = np.asarray(M)
    N = np.asarray(N)
    norms = np.sqrt((np.abs(a) ** 2 * M[:, None]).sum(axis=0))
    return float(np.prod(norms ** N))


def minor_scale(a, M, N, l):
    N2 = np.array(N).copy()
    N2[l] -= 1
    return scale(a, M, N2)


def ref_perm(a, M, N):
    v, t = oracle.perm_mult(a, M, N)
    return v + t


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_config_single_perm(ctx, mode):
    a, M, N, _, _ = S.config_single(seed=1)
    got = ctx.perm(a, M, N, mode=mode)
    ref = ref_perm(a, M, N)
    assert abs(got - ref) <= TOL[mode] * scale(a, M, N), (got, ref)
    if mode == 0:
        got2, tail = ctx.perm(a, M, N, mode=0, with_tail=True)
        assert abs((got2 + tail) - ref) <= 1e-13 * scale(a, M, N)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_config_single_minors(ctx, mode):
    a, M, N, _, _ = S.config_single(seed=1)
    # remove one photon from the last multiplicity-1 row: 11 rows x 12 columns
    M2 = M.copy()
    M2[-1] -= 1
    got = ctx.laplace_minors(a, M2, N, mode=mode)
    ref, tail = oracle.minors(a, M2, N)
    for l in range(len(N)):
        assert abs(got[l] - (ref[l] + tail[l])) <= TOL[mode] * minor_scale(a, M2, N, l), l
    # Laplace identity: sum_l N_l a_{r,l} minor_l = perm with row r restored
    full = ref_perm(a, M, N)
    lap = np.sum(N * a[-1] * got)
    assert abs(lap - full) <= 10 * TOL[mode] * scale(a, M, N)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 9, 12, 13, 16, 17, 20, 21])
def test_distinct_sizes(ctx, mode, n):
    """Distinct rows and columns: C = 2^(n-1) addends, spanning many chunks
    and tasks with a ragged last task."""
    u = S.haar_unitary(48, 100 + n)
    a = u[:n, 10:10 + n]
    ones = np.ones(n, dtype=np.int32)
    got = ctx.perm(a, ones, ones, mode=mode)
    v, t = oracle.bbfg_gray(a)
    assert abs(got - (v + t)) <= TOL[mode] * scale(a, ones, ones), (n, got, v)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("K", [4, 6, 11, 15, 19, 24, 27, 30, 32, 33, 36, 38, 41, 44, 45, 48])
def test_every_column_bucket(ctx, mode, K):
    """Few distinct rows with large multiplicities: every K bucket (up to 48
    product columns) with an addend count the oracle finishes quickly."""
    g = S.rng(2000 + K)
    R = 3 if K > 30 else 4
    M = np.full(R, K // R, dtype=np.int32)
    M[: K - M.sum()] += 1
    u = S.haar_unitary(64, 300 + K)
    a = u[g.permutation(64)[:R]][:, g.permutation(64)[:K]]
    N = np.ones(K, dtype=np.int32)
    got = ctx.perm(a, M, N, mode=mode)
    ref = ref_perm(a, M, N)
    bound = TOL[mode] * scale(a, M, N) + TOL_L1 * oracle.perm_mult_abs(a, M, N)
    assert abs(got - ref) <= bound, (K, got, ref, bound)


def test_mixed_routes_heavy_collisions_to_double_float(ctx):
    """The MIXED rule sends heavily repeated rows (here 7, 7, 6: predicted
    FP32 error 2^-7.9 of prod ||a_j||) to the double-float kernels, which give
    exactly the double-float-mode result; light repeats (2, 2, 2 and distinct
    rows: 2^-23.8) stay in FP32."""
    u = S.haar_unitary(40, 9)
    a = u[:3, :20]
    M = np.array([7, 7, 6], dtype=np.int32)
    N = np.ones(20, dtype=np.int32)
    ctx.reset_stats()
    got = ctx.perm(a, M, N, mode=1)
    st = ctx.stats()
    assert st["addends"][2] > 0 and st["addends"][1] == 0 and st["addends"][0] == 0
    assert got == ctx.perm(a, M, N, mode=2)
    assert abs(got - ref_perm(a, M, N)) <= TOL[0] * scale(a, M, N) + TOL_L1 * oracle.perm_mult_abs(a, M, N)
    b = u[:12, :14]
    Mb = np.array([2, 2, 2] + [1] * 9, dtype=np.int32)
    Nb = np.ones(14, dtype=np.int32)
    Nb[0] += 1                                    # sum M = 15 = sum N
    r64, r32 = ctx.perm(b, Mb, Nb, mode=0), ctx.perm(b, Mb, Nb, mode=1)
    assert r64 != r32
    assert abs(r32 - ref_perm(b, Mb, Nb)) <= TOL[1] * scale(b, Mb, Nb)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_edge_cases(ctx, mode):
    # n = 0: the empty permanent
    assert ctx.perm(np.zeros((2, 2)), [0, 0], [0, 0], mode=mode) == 1
    # n = 1
    a = np.array([[0.3 - 0.7j]])
    assert abs(ctx.perm(a, [1], [1], mode=mode) - a[0, 0]) <= TOL[mode] * abs(a[0, 0])
    # a single row and column repeated n times: perm = n! a^n
    for n in (2, 5, 9):
        got = ctx.perm(a, [n], [n], mode=mode)
        ref = math.factorial(n) * a[0, 0] ** n
        assert abs(got - ref) <= TOL[mode] * abs(ref) * 10
    # zero multiplicities, repeated first row, column multiplicities
    b = S.random_complex(4, 5, 77)
    M = np.array([3, 0, 2, 1])
    N = np.array([2, 1, 0, 2, 1])
    got = ctx.perm(b, M, N, mode=mode)
    assert abs(got - ref_perm(b, M, N)) <= TOL[mode] * scale(b, M, N)
    # transposed orientation chosen (columns repeated more than rows)
    c = S.random_complex(6, 2, 78)
    got = ctx.perm(c, np.ones(6, np.int32), [3, 3], mode=mode)
    assert abs(got - ref_perm(c, np.ones(6), [3, 3])) <= TOL[mode] * scale(c, np.ones(6), [3, 3])
    # all rows repeated (no binary digit besides the split pinned row)
    d = S.random_complex(3, 6, 79)
    got = ctx.perm(d, [2, 2, 2], np.ones(6, np.int32), mode=mode)
    assert abs(got - ref_perm(d, [2, 2, 2], np.ones(6))) <= TOL[mode] * scale(d, [2, 2, 2], np.ones(6))


def test_invalid_arguments(ctx, bslib):
    with pytest.raises(bslib.BsError) as e:
        ctx.perm(np.ones((2, 2)), [1, 1], [1, 2])
    assert e.value.code == bslib.BS_EINVAL
    with pytest.raises(bslib.BsError):
        ctx.perm(np.ones((2, 2)), [-1, 3], [1, 1])
    with pytest.raises(bslib.BsError):
        ctx.perm(np.ones((1, 1)), [49], [49])
    # the context still works afterwards
    assert abs(ctx.perm(np.array([[2.0]]), [1], [1]) - 2.0) < 1e-15


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_minors_with_repeats_and_empty(ctx, mode):
    g = S.rng(55)
    for trial in range(6):
        R, K = int(g.integers(1, 5)), int(g.integers(2, 7))
        a = S.random_complex(R, K, 900 + trial)
        N = np.ones(K, dtype=np.int32)
        N[g.integers(0, K)] += 1
        n = int(N.sum()) - 1
        M = np.zeros(R, dtype=np.int32)
        for _ in range(n):
            M[g.integers(0, R)] += 1
        got = ctx.laplace_minors(a, M, N, mode=mode)
        ref, tail = oracle.minors(a, M, N)
        for l in range(K):
            assert abs(got[l] - (ref[l] + tail[l])) <= TOL[mode] * max(minor_scale(a, M, N, l), 1e-300) * 10
    # zero rows: the single minor is per(0x0) = 1
    got = ctx.laplace_minors(np.zeros((1, 1)), [0], [1], mode=mode)
    assert got[0] == 1


# (row multiplicities, binary digits after pinning one M = 1 row): binary
# digit counts 1..6 with chunks of 64 addends, so the FP32 minors walk ends
# its branch-free blocks every 2^nbin steps (nbin < 7) or at every fold
# point, takes the mixed-radix step at each block end, and (C not a multiple
# of 64) lets a lane run past the end of a short last chunk inside a block.
# Each case stays in FP32 under the MIXED rule (checked from the statistics
# of every call).
BLOCK_CASES = [
    ([1, 1] + [2] * 7, 1),
    ([1] * 3 + [2] * 6, 2),
    ([1] * 4 + [2] * 5, 3),
    ([1] * 5 + [2] * 4, 4),
    ([1] * 6 + [2] * 3, 5),
    ([1] * 7, 6),
    ([1, 1] + [2] * 6 + [3], 1),
    ([1] * 3 + [2] * 6 + [3], 2),
    ([1] * 4 + [2] * 5 + [3], 3),
    ([1] * 7 + [2, 2, 3], 6),
]


@pytest.mark.parametrize("M,nbin", BLOCK_CASES)
def test_fp32_minors_block_schedule(ctx, M, nbin):
    """MIXED fused minors in the FP32 kernel (checked from the statistics)
    against the oracle's permanent of each column-deleted matrix."""
    M = np.array(M, dtype=np.int32)
    K = int(M.sum()) + 1
    ones = int((M == 1).sum())
    assert nbin == ones - 1
    u = S.haar_unitary(32, 700 + nbin)
    g = S.rng(710 + nbin)
    a = u[g.permutation(32)[: len(M)]][:, g.permutation(32)[:K]]
    N = np.ones(K, dtype=np.int32)
    ctx.reset_stats()
    got = ctx.laplace_minors(a, M, N, mode=1)
    st = ctx.stats()
    assert st["addends"][1] > 0 and st["addends"][0] == 0, "expected the FP32 kernel"
    for l in range(K):
        keep = [j for j in range(K) if j != l]
        ref = ref_perm(a[:, keep], M, N[keep])
        assert abs(got[l] - ref) <= TOL[1] * minor_scale(a, M, N, l), (nbin, l, got[l], ref)


MINOR_WIDTHS = [13, 17, 20, 21, 24, 25, 26, 28, 29, 31, 32, 33, 36, 37, 40, 41, 44, 45, 48]


@pytest.mark.parametrize("mode", [0, 2])
@pytest.mark.parametrize("K", MINOR_WIDTHS)
def test_fp64_minors_every_width_against_oracle(ctx, mode, K):
    """FP64 fused minors of a (K-1)-photon row set over K columns, for every
    column width up to 48: three distinct rows with large multiplicities keep
    the oracle's term-by-term formula cheap; every minor is checked against
    the oracle's permanent of the matrix with that column removed."""
    g = S.rng(4000 + K)
    R = 3
    M = np.full(R, (K - 1) // R, dtype=np.int32)
    M[: K - 1 - M.sum()] += 1
    u = S.haar_unitary(64, 500 + K)
    a = u[g.permutation(64)[:R]][:, g.permutation(64)[:K]]
    N = np.ones(K, dtype=np.int32)
    got = ctx.laplace_minors(a, M, N, mode=mode)
    for l in range(K):
        keep = [j for j in range(K) if j != l]
        ref = ref_perm(a[:, keep], M, N[keep])
        bound = TOL[mode] * minor_scale(a, M, N, l) + TOL_L1 * oracle.perm_mult_abs(a[:, keep], M, N[keep])
        assert abs(got[l] - ref) <= bound, (K, l, got[l], ref, bound)


def _rows_for(total):
    """Row multiplicities summing to `total`: two rows of multiplicity 1
    (binary Gray digits, one of them pinned) and two of large multiplicity
    (n-ary digits), so the oracle's term-by-term sum stays small."""
    if total <= 2:
        return np.ones(total, dtype=np.int32)
    rest = total - 2
    return np.array([1, 1, (rest + 1) // 2, rest // 2], dtype=np.int32)[: 4 if rest > 1 else 3]


@pytest.mark.parametrize("K", range(1, 49))
def test_fp64_every_column_count_against_oracle(ctx, K):
    """The FP64 kernels run a separately compiled walk for each exact column
    count (permanents) and each owned-column count of a lane pair (minors),
    so every K from 1 to 48 is its own instance: the permanent of a K-column
    problem and, for K >= 2, the K minors of a (K-1)-photon row set, each
    against the oracle (Eq. bbfgrepeated term by term)."""
    g = S.rng(7000 + K)
    u = S.haar_unitary(64, 700 + K)
    N = np.ones(K, dtype=np.int32)
    M = _rows_for(K)
    a = u[g.permutation(64)[: len(M)]][:, g.permutation(64)[:K]]
    got = ctx.perm(a, M, N, mode=0)
    ref = ref_perm(a, M, N)
    bound = TOL[0] * scale(a, M, N) + TOL_L1 * oracle.perm_mult_abs(a, M, N)
    assert abs(got - ref) <= bound, (K, got, ref, bound)
    if K < 2:
        return
    M = _rows_for(K - 1)
    a = u[g.permutation(64)[: len(M)]][:, g.permutation(64)[:K]]
    got = ctx.laplace_minors(a, M, N, mode=0)
    for l in range(K):
        keep = [j for j in range(K) if j != l]
        ref = ref_perm(a[:, keep], M, N[keep])
        bound = TOL[0] * minor_scale(a, M, N, l) + TOL_L1 * oracle.perm_mult_abs(a[:, keep], M, N[keep])
        assert abs(got[l] - ref) <= bound, (K, l, got[l], ref, bound)


@pytest.mark.parametrize("K", MINOR_WIDTHS)
def test_fp32_minors_every_width(ctx, bslib, K):
    """The FP32 fused minors at every column width, forced to FP32 with the
    MIXED tolerance knob (rows of multiplicity 3, which the default rule
    sends to FP64 from width 24 on): every minor against the FP64 kernel
    within the error the precision rule predicts for the job
    (2^log2_err prod ||a_j||), and the Laplace identity
    sum_l v_l minor_l = per([A; v]) against the FP64 permanent.  The FP64
    kernels are pinned to the oracle at these widths (test_gpu_widths), and
    the FP32 kernels at their default-tolerance widths by dense oracle cases
    there."""
    g = S.rng(4100 + K)
    n = K - 1
    m = 3 if K >= 24 else (2 if K >= 17 else 1)
    R = min(n, max(2, -(-n // m)))
    M = np.full(R, n // R, dtype=np.int32)
    M[: n - M.sum()] += 1
    u = S.haar_unitary(64, 600 + K)
    rows = g.permutation(64)[: R + 1]
    cols = g.permutation(64)[:K]
    a = u[rows[:R]][:, cols]
    v = u[rows[R], cols]
    N = np.ones(K, dtype=np.int32)
    log2_err, _, _ = bslib.debug_mixed_error(M, N, 1)
    bound = 2.0 ** log2_err
    ctx.set_mixed_tolerance(1e300)
    try:
        ctx.reset_stats()
        got = ctx.laplace_minors(a, M, N, mode=1)
        st = ctx.stats()
    finally:
        ctx.set_mixed_tolerance(1e-6)
    assert st["addends"][1] > 0 and st["addends"][0] == 0, "expected the FP32 kernel"
    ref = ctx.laplace_minors(a, M, N, mode=0)
    for l in range(K):
        assert abs(got[l] - ref[l]) <= bound * minor_scale(a, M, N, l), (K, l, got[l], ref[l], log2_err)
    full = ctx.perm(np.vstack([a, v]), np.append(M, 1), N, mode=0)
    lap = np.sum(v * got)
    assert abs(lap - full) <= 10 * bound * scale(np.vstack([a, v]), np.append(M, 1), N), (K, lap, full)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batch_matches_oracle_and_single_calls(ctx, mode):
    items = S.config_batch(count=48, seed=7, kmin=6, kmax=18, m=60, group=16)
    items.append((np.zeros((1, 1)), np.array([0]), np.array([0])))       # trivial item
    got = ctx.perm_batch(items, mode=mode)
    for b, (a, M, N) in enumerate(items):
        ref = ref_perm(a, M, N)
        assert abs(got[b] - ref) <= TOL[mode] * scale(a, M, N) + (0 if np.sum(M) else 1e-300), b
        # each result is bit-identical whether computed alone or in the batch
        alone = ctx.perm(a, M, N, mode=mode)
        assert alone == got[b], (b, alone, got[b])


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_full_batch_config_sampled(ctx, mode):
    """4096 uneven permanents (k in [10, 28]) in one call; the oracle checks
    the cheapest items one by one, and FP64 / MIXED agree on every item."""
    items = S.config_batch(count=4096, seed=2)
    got = ctx.perm_batch(items, mode=mode)
    costs = [int(np.prod(np.asarray(M) + 1)) for _, M, _ in items]
    order = np.argsort(costs)
    for b in list(order[:12]) + list(order[2048:2051]):
        a, M, N = items[b]
        assert abs(got[b] - ref_perm(a, M, N)) <= TOL[mode] * scale(a, M, N), b
    if mode == 1:
        ref64 = ctx.perm_batch(items, mode=0)
        sc = np.array([scale(a, M, N) for a, M, N in items])
        assert np.all(np.abs(got - ref64) <= 1e-6 * sc)


def test_batch_device_pointers(ctx):
    import torch
    items = S.config_batch(count=32, seed=9, kmin=8, kmax=14)
    packed, offs, rows, cols, mults, roff, coff = ctx.pack_batch(items)
    dev = torch.from_numpy(packed).cuda()
    out = torch.zeros(len(items), dtype=torch.complex128, device="cuda")
    ctx.set_stream(torch.cuda.current_stream())
    try:
        ctx.perm_batch_dev(dev, offs, rows, cols, mults, roff, coff, 0, out)
        ctx.sync()
    finally:
        ctx.set_stream(None)
    host = ctx.perm_batch(items, mode=0)
    assert np.array_equal(out.cpu().numpy(), host)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batch_graph_replay(ctx, mode):
    """A repeated batch replays its captured device sequence: the results
    equal the eager launches bit for bit, new matrix data in the same buffer
    is read at replay, and a call that rewrites the context buffers in
    between forces a fresh capture (same results again)."""
    import torch
    items = S.config_batch(count=48, seed=21, kmin=8, kmax=18)
    packed, offs, rows, cols, mults, roff, coff = ctx.pack_batch(items)
    phase = np.exp(0.3j)
    orig = torch.from_numpy(packed).cuda()
    dev = orig.clone()
    torch.cuda.synchronize()
    out = torch.zeros(len(items), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.Stream()
    ctx.set_stream(stream)

    def run():
        ctx.perm_batch_dev(dev, offs, rows, cols, mults, roff, coff, mode, out)
        ctx.sync()
        return out.cpu().numpy().copy()

    try:
        ctx.set_graphs(False)
        eager = run()
        dev.mul_(phase)
        torch.cuda.synchronize()
        eager_phase = run()
        dev.copy_(orig)
        torch.cuda.synchronize()
        ctx.set_graphs(True)
        first = run()  # capture
        k0 = ctx.stats()["kernel_launches"]
        second = run()  # replay
        assert ctx.stats()["kernel_launches"] > k0
        assert np.array_equal(first, eager) and np.array_equal(second, eager)
        dev.mul_(phase)
        torch.cuda.synchronize()
        assert np.array_equal(run(), eager_phase)  # replay reads the new data
        dev.copy_(orig)
        torch.cuda.synchronize()
        ctx.perm(items[0][0], items[0][1], items[0][2], mode=mode)  # rewrites the job buffers
        assert np.array_equal(run(), eager)
    finally:
        ctx.set_graphs(True)
        ctx.set_stream(None)
    host = ctx.perm_batch(items, mode=mode)
    assert np.array_equal(host, eager)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_single_call_graph_replay(ctx, mode):
    """Repeated single calls of one plan replay a captured graph (from the
    second call on): permanents with their double-double tails and minors
    equal the eager launches bit for bit, each call reads its own matrix, and
    a call of another plan in between runs eagerly and leaves the results
    unchanged."""
    u = S.haar_unitary(40, 31)
    mats = [u[:14, :14], u[14:28, :14], u[20:34, 2:16]]
    M = np.array([2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1], np.int32)
    N = np.ones(14, np.int32)
    a_rows = [m[:13] for m in mats]
    M2 = M.copy()
    M2[0] -= 1
    stream = None

    def calls():
        out = []
        for a in a_rows:
            out.append(ctx.perm(a, M, N, mode=mode, with_tail=True))
        for a in a_rows:
            out.append(tuple(ctx.laplace_minors(a, M2, N, mode=mode)))
        return out

    try:
        ctx.set_graphs(False)
        eager = calls()
        ctx.set_graphs(True)
        first = calls()   # eager on first sight, captured on the second call
        k0 = ctx.stats()["kernel_launches"]
        second = calls()  # replays
        assert ctx.stats()["kernel_launches"] > k0
        assert first == eager and second == eager
        ctx.perm(np.ones((3, 3)), [1, 1, 1], [1, 1, 1], mode=mode)  # another plan in between
        assert calls() == eager
    finally:
        ctx.set_graphs(True)
        ctx.set_stream(stream)


def test_autotuner_picks_a_valid_chunk_and_results_stay_exact(ctx, bslib):
    saved = (ctx.chunk_log2(0), ctx.chunk_log2(1))
    try:
        for mode in (0, 1):
            best, rate = ctx.tune(mode, kind=1, K=20)
            assert best in (8, 10, 12, 14) and ctx.chunk_log2(mode) == best and rate > 0
            a, M, N, _, _ = S.config_single(seed=1)
            assert abs(ctx.perm(a, M, N, mode=mode) - ref_perm(a, M, N)) <= TOL[mode] * scale(a, M, N)
    finally:
        ctx.set_chunk_log2(0, saved[0])
        ctx.set_chunk_log2(1, saved[1])


def test_deadline_returns_timeout_and_context_survives(ctx, bslib):
    u = S.haar_unitary(40, 5)
    a = u[:30, :30]
    ones = np.ones(30, dtype=np.int32)
    ctx.set_deadline(1e-6)
    try:
        with pytest.raises(bslib.BsError) as e:
            ctx.perm(a, ones, ones, mode=0)
        assert e.value.code == bslib.BS_ETIMEOUT
    finally:
        ctx.set_deadline(0.0)
    b = u[:6, :6]
    v, t = oracle.bbfg_gray(b)
    assert abs(ctx.perm(b, np.ones(6), np.ones(6)) - (v + t)) <= 1e-10 * scale(b, np.ones(6), np.ones(6))


# ---------------------------------------------------------------- sampling
@pytest.mark.parametrize("mode", [0, 2])
def test_sampler_matches_oracle_sampler_fp64(ctx, mode):
    """Same seed, same Philox counters: the GPU chain (FP64 or double-float)
    and the oracle chain draw the same rows, except a draw that lands within
    1e-9 of a CDF boundary."""
    u, occ = S.config_cc(n=6, m=12, seed=3)
    ns = 200
    got = ctx.sample(u, occ, ns, seed=2024, mode=mode)
    ref, margin, _ = oracle.cc_sample(u, occ, ns, seed=2024)
    mismatch = [s for s in range(ns) if not np.array_equal(got[s], ref[s])]
    assert all(margin[s] < 1e-9 for s in mismatch), (mismatch, margin[mismatch])
    assert len(mismatch) <= 1
    assert np.all(got.sum(axis=1) == 6)


@pytest.mark.parametrize("mode", [0, 2])
@pytest.mark.parametrize("n,m", [(6, 12), (8, 16)])
def test_lossy_sampler_matches_oracle_sampler_fp64(ctx, n, m, mode):
    """Lossy sampling (one loss mode per photon, transmissivity 0.5): the GPU
    chains and the oracle's draw the same rows, seed for seed, only modes
    below m counted, except a draw within 1e-9 of a CDF boundary."""
    v, mdet = S.config_lossy(n=n, m=m, eta=0.5, seed=40 + n)
    ns = 120
    occ = np.ones(n, dtype=np.int32)
    got = ctx.sample_ex(v, occ, ns, seed=4040 + n, m_detected=mdet, mode=mode)
    ref, margin, _ = oracle.cc_sample(v, occ, ns, seed=4040 + n, m_detected=mdet)
    assert got.shape == ref.shape == (ns, m)
    mismatch = [s_ for s_ in range(ns) if not np.array_equal(got[s_], ref[s_])]
    assert all(margin[s_] < 1e-9 for s_ in mismatch), (mismatch, margin[mismatch])
    assert len(mismatch) <= 1
    assert np.all(got.sum(axis=1) <= n) and got.sum() < n * ns


def test_sampler_graph_replay_equals_eager(ctx):
    """The captured step loop, replayed for new seeds, draws exactly what the
    directly launched kernels draw."""
    u, occ = S.config_cc(n=10, m=20, seed=8)
    ctx.set_graphs(False)
    try:
        eager = [ctx.sample(u, occ, 64, seed=s, mode=m) for s, m in ((1, 0), (2, 0), (3, 1))]
    finally:
        ctx.set_graphs(True)
    for rep in range(2):
        graph = [ctx.sample(u, occ, 64, seed=s, mode=m) for s, m in ((1, 0), (2, 0), (3, 1))]
        for e, g in zip(eager, graph):
            assert np.array_equal(e, g)


def test_profiled_sampler_graph_times_every_walk(ctx):
    """With profiling on, the replayed sampler graph carries the walk timing
    events: every walk of every replay is timed, the draws equal the eager
    ones, and a context call after it sees no stale error."""
    import torch
    u, occ = S.config_cc(n=10, m=20, seed=8)
    n = int(np.sum(occ))
    stream = torch.cuda.Stream()
    ctx.set_stream(stream)
    try:
        ctx.set_graphs(False)
        eager = ctx.sample(u, occ, 32, seed=5, mode=1)
        ctx.set_graphs(True)
        ctx.set_profiling(True)
        ctx.walk_times()
        got = []
        for rep in range(3):
            got.append(ctx.sample(u, occ, 32, seed=5, mode=1))
            t = ctx.walk_times()
            assert len(t) == 2 * (n - 1), (rep, len(t))  # FP32 and double-float walk per step k = 2..n
            assert np.all(t >= 0) and np.sum(t) > 0
        for g in got:
            assert np.array_equal(g, eager)
    finally:
        ctx.set_profiling(False)
        ctx.set_graphs(True)
        ctx.set_stream(None)
    assert np.array_equal(ctx.sample(u, occ, 32, seed=5, mode=1), eager)


def test_sampler_seed_and_batch_independence(ctx):
    u, occ = S.config_cc(n=8, m=16, seed=4)
    a = ctx.sample(u, occ, 40, seed=11, mode=0)
    b = ctx.sample(u, occ, 40, seed=11, mode=0)
    c = ctx.sample(u, occ, 10, seed=11, mode=0)
    assert np.array_equal(a, b)
    assert np.array_equal(a[:10], c)


def test_sampler_mixed_chi_square(ctx):
    st = pytest.importorskip("scipy.stats")
    import itertools
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
    counts = ctx.sample(u, s, 20000, seed=99, mode=1)
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


def test_sampler_marginals_and_lossy(ctx):
    u, occ = S.config_cc(n=6, m=12, seed=26)
    counts = ctx.sample(u, occ, 4000, seed=5, mode=1)
    ref = (np.abs(u) ** 2) @ occ
    mean = counts.mean(axis=0)
    sd = counts.std(axis=0) / np.sqrt(len(counts))
    assert np.all(np.abs(mean - ref) < 5 * sd + 1e-3)
    # lossy isometry: detected photon number ~ Binomial(n, eta)
    v, mdet = S.config_lossy(n=6, m=12, eta=0.5, seed=5)
    lc = ctx.sample_ex(v, np.ones(6, dtype=np.int32), 4000, seed=6, m_detected=mdet, mode=1)
    det = lc.sum(axis=1)
    assert det.max() <= 6
    assert abs(det.mean() - 3.0) < 5 * math.sqrt(6 * 0.25 / 4000)
