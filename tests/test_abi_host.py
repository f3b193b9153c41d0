"""Host-side checks of libbs.so that need no GPU: every symbol declared in
include/bs.h is exported, the n-ary reflected Gray counter used by the
kernels (compiled for the host from the same header) has the Gray
properties of Sec. 2.2, the planner's canonicalisation decisions, and that
compute calls fail loudly without a device."""
import ctypes
import itertools
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(bs_[a-z0-9_]+)\s*\(", src, flags=re.M)))


def test_all_declared_symbols_exported(bslib):
    names = declared_functions()
    assert len(names) >= 20
    lib = ctypes.CDLL(bslib.library_path())
    for n in names:
        assert hasattr(lib, n), n


def _reference_gray(radix):
    """Reflected mixed-radix Gray code by its recursive definition: the code
    for digits 0..j is the code for digits 0..j-1 traversed forward for even
    values of digit j and backward for odd values (digit 0 fastest)."""
    seq = [()]
    for r in radix:
        nxt = []
        for v in range(r):
            part = seq if v % 2 == 0 else seq[::-1]
            nxt.extend(code + (v,) for code in part)
        seq = nxt
    return [list(c) for c in seq]


@pytest.mark.parametrize("radix,nbin", [([2, 2, 2], 3), ([2, 2, 3], 2), ([3, 4, 2], 0), ([2, 3, 3, 5], 1),
                                        ([2] * 10, 10), ([2, 2, 2, 2, 4, 3], 4), ([5], 0), ([], 0)])
def test_gray_walk_is_reflected_gray_code(bslib, radix, nbin):
    C = int(np.prod(radix)) if radix else 1
    deltas, moved, w = bslib.debug_gray_walk(radix, nbin, 0, C)
    ref = _reference_gray(radix)
    assert [list(r) for r in deltas] == ref
    # one digit moves by +-1 per step, every code appears once
    for s in range(1, C):
        diff = deltas[s] - deltas[s - 1]
        assert np.count_nonzero(diff) == 1 and abs(diff[moved[s]]) == 1
    assert len({tuple(r) for r in deltas}) == C
    # weights = prod C(M_j, Delta_j) over digits (binary digits weigh 1)
    for s in range(C):
        want = 1
        for j, r in enumerate(radix):
            want *= math.comb(r - 1, int(deltas[s][j]))
        assert int(w[s]) == want


@pytest.mark.parametrize("radix,nbin", [([2, 2, 3, 4], 2), ([2] * 6 + [3, 3], 6), ([4, 5, 3], 0)])
def test_gray_decode_matches_stepping(bslib, radix, nbin):
    """Decoding any start index gives the state reached by stepping from 0
    (Sec. 2.2: constant-time decode enables independent chunks)."""
    C = int(np.prod(radix))
    full, _, wf = bslib.debug_gray_walk(radix, nbin, 0, C)
    for start in range(0, C, max(1, C // 17)):
        part, _, wp = bslib.debug_gray_walk(radix, nbin, start, C - start)
        assert np.array_equal(part, full[start:])
        assert np.array_equal(wp, wf[start:])


def test_gray_binary_matches_paper_table(bslib):
    from conftest import read_golden
    deltas, moved, _ = bslib.debug_gray_walk([2, 2, 2], 3, 0, 8)
    gold = read_golden("gray_code_3bit.txt")
    for (idx, code), row in zip(gold, deltas):
        # code string is written most significant bit first
        assert "".join(str(int(b)) for b in row[::-1]) == code


def test_gray_walk_rejects_bad_radix(bslib):
    with pytest.raises(bslib.BsError):
        bslib.debug_gray_walk([3, 2], 1, 0, 2)      # first digit must be binary
    with pytest.raises(bslib.BsError):
        bslib.debug_gray_walk([2, 2], 2, 3, 5)      # walk leaves [0, C)


def test_planner_addend_counts_and_orientation(bslib):
    # config 1: rows (3,2,2,1,1,1,1,1), 12 distinct columns -> 4*3*3*2^4 = 576
    p = bslib.debug_plan([3, 2, 2, 1, 1, 1, 1, 1], [1] * 12)
    assert p["C"] == 576 and p["K"] == 12 and not p["transposed"]
    assert p["nbin"] == 4 and p["nrows"] == 7
    # the orientation with repeated entries on the row side is chosen:
    # rows cost 1 * 2^5 = 32 addends, columns 3 * 4 = 12
    q = bslib.debug_plan([1] * 6, [3, 3])
    assert q["transposed"] and q["C"] == 12 and q["K"] == 6
    # rows (2,3) x one column of multiplicity 5: transposed, the single row
    # of multiplicity 5 splits into the pinned copy + a radix-5 digit
    r = bslib.debug_plan([2, 3], [5])
    assert r["transposed"] and r["C"] == 5 and r["nrows"] == 1 and r["K"] == 5
    # no row of multiplicity one and no cheaper transpose: the smallest
    # multiplicity is split (1 + (M-1)): digits radix 2 and 4
    t = bslib.debug_plan([2, 3], [1] * 5)
    assert not t["transposed"] and t["C"] == 8 and t["nrows"] == 2 and t["nbin"] == 1
    # zero multiplicities are dropped
    z = bslib.debug_plan([0, 1, 0, 1], [1, 0, 1])
    assert z["C"] == 2 and z["K"] == 2
    # minors: sum M = sum N - 1, never transposed, K = sum N
    m = bslib.debug_plan([1, 1], [1, 1, 1], kind=1)
    assert m["C"] == 2 and m["K"] == 3 and not m["transposed"]


def test_single_call_chunking(bslib):
    """Jobs planned one call at a time (FP64, chunk cap 2^11 by default):
    chunks of 2^6 to 2^11 addends aimed
    at 32768 warp tasks of 32 chunks; a job too small to give 256 tasks at
    2^6 gets chunks down to 2^3 until it does, or 2^1 for jobs of at most
    1024 addends (latency-bound jobs spread over more warps); jobs large
    enough keep 2^6 or longer."""
    def plan(n):
        return bslib.debug_plan([1] * n, [1] * n)
    for n in (3, 8, 11, 14, 17, 20, 23, 26, 29, 32, 36):
        p = plan(n)
        C, l, tasks = p["C"], p["log2L"], p["tasks"]
        assert C == 2 ** (n - 1) and 1 <= l <= 11
        assert tasks == -(-C // (32 << l))
        if l == 11:  # the re-seed interval caps the chunk
            assert tasks >= 32768
        elif l > 6:  # the large-job rule: about 32768 tasks
            assert 32768 <= tasks < 2 * 32768
        elif l == 6:
            assert tasks >= 256
        else:        # shortened only as far as needed to reach 256 tasks
            assert l == (1 if C <= 1024 else 3) or 256 <= tasks < 2 * 256
    assert [plan(n)["log2L"] for n in (17, 18, 19, 20, 23, 26, 29, 33)] == [3, 4, 5, 6, 6, 6, 8, 11]
    c1 = bslib.debug_plan([3, 2, 2, 1, 1, 1, 1, 1], [1] * 12)
    assert c1["log2L"] == 1 and c1["tasks"] == 9


def test_planner_rejects_invalid(bslib):
    for M, N, kind in [([1, 1], [1], 0), ([-1, 2], [1], 0), ([25, 25], [50], 0), ([1], [1], 1)]:
        with pytest.raises(bslib.BsError) as e:
            bslib.debug_plan(M, N, kind)
        assert e.value.code == bslib.BS_EINVAL


def test_no_gpu_fails_loudly(bslib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(bslib.BsError) as e:
        bslib.Context(0)
    assert "BS_ENODEV" in str(e.value)


def test_mixed_rule_sum_over_delta_matches_brute_force(bslib):
    """The MIXED precision rule's sum over Delta vectors (a dynamic program
    over Q = sum_k (M_k - 2 Delta_k)^2) against direct enumeration of every
    Delta vector: one copy of a smallest-multiplicity row pinned (coefficient
    M_p - 2D, weight C(M_p - 1, D)), every other row coefficient M_k - 2D with
    weight C(M_k, D).  The prediction is that sum's log2 RSS plus the
    rounding and drift terms, log2(K)/2 + max(0, log2L - 8)/2 - 21.02."""
    import itertools
    from math import comb, log2
    g = np.random.default_rng(5)
    for trial in range(40):
        R = int(g.integers(1, 6))
        M = g.integers(1, 5, size=R).astype(np.int32)
        n = int(M.sum())
        kind = int(g.integers(0, 2))
        K = n + kind
        order = sorted(range(R), key=lambda k: M[k])
        p = order[0]
        ranges = [range(M[k]) if k == p else range(M[k] + 1) for k in range(R)]
        total = 0.0
        for D in itertools.product(*ranges):
            w, q = 1.0, 0
            for k in range(R):
                if k == p:
                    w *= comb(int(M[k]) - 1, D[k]) ** 2
                    q += (int(M[k]) - 2 * D[k]) ** 2
                else:
                    w *= comb(int(M[k]), D[k]) ** 2
                    q += (int(M[k]) - 2 * D[k]) ** 2
            total += w * (q / n) ** K
        lrss = (1 - n) + 0.5 * log2(total)
        got, l32, _ = bslib.debug_mixed_error(M, np.ones(K, np.int32), kind)
        want = lrss + 0.5 * log2(K) + 0.5 * max(0, l32 - 8) - 21.02
        assert abs(got - want) < 1e-4, (M.tolist(), kind, got, want)


def test_mixed_rule_closed_form_for_distinct_rows(bslib):
    """Distinct rows (every M = 1): every coefficient is +-1, Q = n for all
    2^(n-1) addends, so RSS / prod ||a_j|| = 2^((1-n)/2) exactly."""
    from math import log2
    for n in (3, 10, 24, 30):
        got, l32, _ = bslib.debug_mixed_error(np.ones(n, np.int32), np.ones(n, np.int32), 0)
        want = (1 - n) / 2 + 0.5 * log2(n) + 0.5 * max(0, l32 - 8) - 21.02
        assert abs(got - want) < 1e-4, (n, got, want)


def test_mixed_plan_reseeds_where_only_the_drift_term_fails(bslib):
    """The three-way MIXED decision: FP32 when the prediction at the job's
    chunk length meets 1e-6; FP32 with the column sums re-seeded every 2^8
    steps when only the prediction without its drift term does (the drift
    term is (log2 L - 8) / 2 for chunks of 2^log2L addends); else the
    fallback kernels.  Checked over chunk lengths 2^3..2^12 on random
    multiplicity patterns, against the prediction itself."""
    tol = float(np.float32(-19.93))
    g = np.random.default_rng(404)
    seen = set()
    for trial in range(300):
        K = int(g.integers(8, 41))
        hits = g.integers(0, int(g.integers(K // 3 + 1, 3 * K)), size=K - 1)
        _, M = np.unique(hits, return_counts=True)
        M = M.astype(np.int32)
        for L in (3, 8, 10, 12):
            e, l, plan = bslib.debug_mixed_error(M, np.ones(K, np.int32), 1, chunk_log2=L)
            assert l == L
            e8, _, _ = bslib.debug_mixed_error(M, np.ones(K, np.int32), 1, chunk_log2=8)
            assert abs((e - e8) - 0.5 * max(0, L - 8)) < 1e-4
            want = 1 if e <= tol else (2 if L > 8 and e8 <= tol else 0)
            assert plan == want, (M.tolist(), L, e, e8, plan)
            seen.add(plan)
    assert seen == {0, 1, 2}
