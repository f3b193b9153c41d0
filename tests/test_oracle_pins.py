"""Pins for the CPU oracle: each test ties an oracle function to something
other than itself (the paper's printed values, closed forms, exact integer
arithmetic, brute force, textbook identities, an independent 50-digit
evaluation).  No GPU is involved.

A plausible slip in the oracle (dropped term, wrong sign, swapped index,
wrong binomial, wrong prefactor) fails at least one of these.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synthetic as S
from conftest import read_golden


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def py_perm(a):
    """Brute-force permanent in Python arithmetic (ints stay exact)."""
    n = len(a)
    tot = 0
    for p in itertools.permutations(range(n)):
        t = 1
        for i in range(n):
            t *= a[i][p[i]]
        tot += t
    return tot


# ---------------------------------------------------------------- Table "gray"
def test_gray_walk_matches_paper_table():
    gold = read_golden("gray_code_3bit.txt")
    seq = oracle.gray_sequence(3)
    assert len(seq) == len(gold)
    for (idx, code), g in zip(gold, seq):
        assert format(g, "03b") == code, (idx, code, g)
        # the closed form of Sec. 2.1: g_i = i xor (i >> 1)
        assert g == int(idx) ^ (int(idx) >> 1)


def test_gray_walk_properties():
    for bits in range(1, 13):
        seq = oracle.gray_sequence(bits)
        assert len(set(seq)) == 1 << bits
        for a, b in zip(seq, seq[1:]):
            assert bin(a ^ b).count("1") == 1


# ---------------------------------------------------------------- hand values
def test_textbook_small_permanents():
    assert oracle.perm_bruteforce(np.array([[1, 2], [3, 4]]))[0] == 10
    assert oracle.perm_bruteforce(np.arange(1, 10).reshape(3, 3))[0] == 450
    assert oracle.bbfg_gray(np.arange(1, 10).reshape(3, 3))[0] == 450
    assert oracle.ryser(np.arange(1, 10).reshape(3, 3))[0] == 450
    assert oracle.nw(np.arange(1, 10).reshape(3, 3))[0] == 450
    assert oracle.nw(np.array([[2.5 - 1j]]))[0] == 2.5 - 1j
    assert oracle.bbfg_gray(np.array([[2.5 - 1j]]))[0] == 2.5 - 1j
    # empty matrix: the permanent of the 0 x 0 matrix is 1
    assert oracle.bbfg_gray(np.zeros((0, 0)))[0] == 1
    assert oracle.ryser(np.zeros((0, 0)))[0] == 1
    assert oracle.nw(np.zeros((0, 0)))[0] == 1


def test_bruteforce_matches_python_bruteforce():
    g = S.rng(11)
    for n in range(1, 7):
        a = g.integers(-4, 5, size=(n, n)) + 1j * g.integers(-4, 5, size=(n, n))
        ref = py_perm([[complex(int(x.real), int(x.imag)) for x in row] for row in a])
        val, tail = oracle.perm_bruteforce(a)
        assert val == ref


# ---------------------------------------------------------------- formulas agree
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_four_formulas_agree(n):
    a = S.random_complex(n, n, 100 + n)
    ref = oracle.perm_bruteforce(a)
    for f in (oracle.bbfg_gray, oracle.bbfg_direct, oracle.ryser, oracle.nw):
        v = f(a)
        err = abs((v[0] - ref[0]) + (v[1] - ref[1]))
        assert err <= 1e-27 * max(1.0, abs(ref[0])) * math.factorial(n), (f.__name__, n, err)


def test_mpmath_50_digits():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    for n in (5, 7, 8):
        a = S.random_complex(n, n, 200 + n)
        am = [[mp.mpc(float(x.real), float(x.imag)) for x in row] for row in a]
        ref = mp.mpc(0)
        for p in itertools.permutations(range(n)):
            t = mp.mpc(1)
            for i in range(n):
                t *= am[i][p[i]]
            ref += t
        v, tail = oracle.bbfg_gray(a)
        got = mp.mpc(v.real, v.imag) + mp.mpc(tail.real, tail.imag)
        assert abs(got - ref) <= mp.mpf("1e-28") * abs(ref), n


def test_ones_matrix_is_factorial():
    for n in range(1, 17):
        j = np.ones((n, n))
        for f in (oracle.bbfg_gray, oracle.ryser, oracle.nw):
            v, tail = f(j)
            assert v.imag == 0 and tail.imag == 0
            assert int(Fraction(v.real) + Fraction(tail.real)) == math.factorial(n), (f.__name__, n)


def test_diagonal_is_product():
    for n in (3, 6, 10):
        d = S.random_complex(1, n, 300 + n)[0]
        v, tail = oracle.bbfg_gray(np.diag(d))
        assert rel(v + tail, np.prod(d)) < 1e-15
        v2, _ = oracle.ryser(np.diag(d))
        assert rel(v2, np.prod(d)) < 1e-15
        v3, _ = oracle.nw(np.diag(d))
        assert rel(v3, np.prod(d)) < 1e-15


def test_row_and_column_permutation_invariance():
    g = S.rng(5)
    for n in (5, 9, 12):
        a = S.random_complex(n, n, 400 + n)
        ref, _ = oracle.bbfg_gray(a)
        b = a[g.permutation(n)][:, g.permutation(n)]
        v, _ = oracle.bbfg_gray(b)
        assert rel(v, ref) < 1e-14
        v2, _ = oracle.bbfg_gray(a.T)
        assert rel(v2, ref) < 1e-14


def test_exact_gaussian_integer_permanents():
    for n in range(1, 12):
        a = S.gaussian_integer_matrix(n, 500 + n, bound=3)
        re, im = oracle.ryser_exact_gauss(a)
        if n <= 6:
            ref = py_perm([[complex(int(x.real), int(x.imag)) for x in row] for row in a])
            assert (re, im) == (int(ref.real), int(ref.imag))
        v, tail = oracle.bbfg_gray(a)
        got_re = Fraction(v.real) + Fraction(tail.real)
        got_im = Fraction(v.imag) + Fraction(tail.imag)
        assert got_re == re and got_im == im, n


def test_nijenhuis_wilf_exact_gaussian_integers():
    """The Nijenhuis-Wilf form (Sec. 2) in exact integers equals Ryser's
    formula and the permanent's definition; its double-double Gray walk
    gives the same integers."""
    for n in range(1, 12):
        a = S.gaussian_integer_matrix(n, 520 + n, bound=3)
        nw_exact = oracle.nw_exact_gauss(a)
        assert nw_exact == oracle.ryser_exact_gauss(a), n
        if n <= 6:
            ref = py_perm([[complex(int(x.real), int(x.imag)) for x in row] for row in a])
            assert nw_exact == (int(ref.real), int(ref.imag))
        v, tail = oracle.nw(a)
        assert Fraction(v.real) + Fraction(tail.real) == nw_exact[0], n
        assert Fraction(v.imag) + Fraction(tail.imag) == nw_exact[1], n


def test_formula_abs_closed_forms():
    """Modulus sums of the Ryser and Nijenhuis-Wilf addends: closed forms on
    J_n and on the identity, and the bound S_abs >= |perm|."""
    for n in range(1, 11):
        j = np.ones((n, n))
        ryser_abs = sum(math.comb(n, k) * k ** n for k in range(n + 1))
        nw_abs = 2 * sum(math.comb(n - 1, k) * abs(Fraction(2 - n, 2) + k) ** n for k in range(n))
        assert oracle.formula_abs("ryser", j) == pytest.approx(ryser_abs, rel=1e-13), n
        assert oracle.formula_abs("nw", j) == pytest.approx(float(nw_abs), rel=1e-13), n
        eye = np.eye(n)
        assert oracle.formula_abs("ryser", eye) == pytest.approx(1.0, rel=1e-15)
        assert oracle.formula_abs("nw", eye) == pytest.approx(1.0, rel=1e-15)
    for n in (6, 10, 14):
        a = S.haar_unitary(2 * n, 40 + n)[:n, :n]
        p = abs(oracle.bbfg_gray(a)[0])
        assert oracle.formula_abs("ryser", a) >= p
        assert oracle.formula_abs("nw", a) >= p


def test_ryser_and_bbfg_agree_on_unitary_submatrices():
    u = S.haar_unitary(40, 7)
    for n in (12, 16):
        a = u[:n, :n]
        v1, t1 = oracle.bbfg_gray(a)
        v2, t2 = oracle.ryser(a)
        scale = np.prod(np.linalg.norm(a, axis=0))
        assert abs((v1 - v2) + (t1 - t2)) < 1e-26 * scale


# ---------------------------------------------------------------- Sec. 3.2 zero test
@pytest.mark.parametrize("r,c", [(5, 3), (8, 6), (10, 3), (12, 10)])
def test_rectangular_bbfg_is_zero(r, c):
    """BB/FG on an r x c matrix with r >= c + 2 cancels exactly (Sec. 3.2)."""
    a = S.random_complex(r, c, 600 + r * c)
    v, tail = oracle.bbfg_gray(a)
    scale = np.prod(np.abs(a).sum(axis=0))  # bound on every addend
    assert abs(v) <= 1e-28 * scale
    # r = c + 1 does not cancel in general: the zero above is not vacuous
    a1 = S.random_complex(c + 1, c, 700 + c)
    v1, _ = oracle.bbfg_gray(a1)
    assert abs(v1) > 1e-6 * np.prod(np.linalg.norm(a1, axis=0))


# ---------------------------------------------------------------- Appendix A.1 padding
def test_padding_with_neutral_columns():
    """Embedding a 3x3 matrix into a 3x48 one whose extra columns are 1 in the
    first row and 0 elsewhere leaves BB/FG unchanged (Appendix A.1)."""
    a = S.random_complex(3, 3, 800)
    b = np.zeros((3, 48), dtype=np.complex128)
    b[:, :3] = a
    b[0, 3:] = 1.0
    ref, _ = oracle.perm_bruteforce(a)
    v, _ = oracle.bbfg_gray(b)
    assert rel(v, ref) < 1e-15


# ---------------------------------------------------------------- Eq. (bbfgrepeated)
def _random_mult_case(g, R, K, n, seed):
    a = S.random_complex(R, K, seed)
    M = np.zeros(R, dtype=np.int32)
    N = np.zeros(K, dtype=np.int32)
    for _ in range(n):
        M[g.integers(0, R)] += 1
        N[g.integers(0, K)] += 1
    return a, M, N


def test_multiplicity_formula_equals_expanded_permanent():
    g = S.rng(9)
    for trial in range(40):
        R = int(g.integers(1, 6))
        K = int(g.integers(1, 6))
        n = int(g.integers(1, 11))
        a, M, N = _random_mult_case(g, R, K, n, 900 + trial)
        v1, t1 = oracle.perm_mult(a, M, N)
        v2, t2 = oracle.perm_expanded(a, M, N)
        scale = np.prod(np.abs(a).sum(axis=0) ** N) + 1.0
        assert abs((v1 - v2) + (t1 - t2)) <= 1e-26 * scale, (trial, M, N, v1, v2)


def test_multiplicity_formula_first_row_repeated_and_zero_rows():
    a = S.random_complex(3, 3, 1000)
    # first row repeated 3 times, a zero-multiplicity row in the middle
    M = np.array([3, 0, 2])
    N = np.array([2, 1, 2])
    v1, _ = oracle.perm_mult(a, M, N)
    v2, _ = oracle.perm_expanded(a, M, N)
    assert rel(v1, v2) < 1e-25
    # row order does not matter (the pinned row choice is free)
    v3, _ = oracle.perm_mult(a[[2, 1, 0]], M[[2, 1, 0]], N)
    assert rel(v3, v2) < 1e-25
    # the expanded matrix built independently in Python
    rows = np.repeat(np.arange(3), M)
    cols = np.repeat(np.arange(3), N)
    ref = oracle.perm_bruteforce(a[np.ix_(rows, cols)])
    assert rel(v2, ref[0]) < 1e-25


def test_multiplicity_formula_exact_gaussian_integers():
    g = S.rng(12)
    for trial in range(10):
        R, K = 3, 4
        n = 8
        a = S.gaussian_integer_matrix(max(R, K), 1100 + trial)[:R, :K]
        M = np.zeros(R, dtype=np.int32)
        N = np.zeros(K, dtype=np.int32)
        for _ in range(n):
            M[g.integers(0, R)] += 1
            N[g.integers(0, K)] += 1
        rows = np.repeat(np.arange(R), M)
        cols = np.repeat(np.arange(K), N)
        re, im = oracle.ryser_exact_gauss(a[np.ix_(rows, cols)])
        v, tail = oracle.perm_mult(a, M, N)
        assert Fraction(v.real) + Fraction(tail.real) == re
        assert Fraction(v.imag) + Fraction(tail.imag) == im


def test_plain_fp64_walk_against_exact_and_double_double():
    """The plain-double twin of the multiplicity walk (the CPU timing
    baseline): exact on small Gaussian-integer cases (every sum and product
    is an exact double), within plain FP64 rounding of the double-double
    oracle on random cases, per(J_n) = n! and the empty permanent."""
    g = S.rng(13)
    for trial in range(10):
        R, K, n = 3, 4, 7
        a = S.gaussian_integer_matrix(max(R, K), 1200 + trial, bound=2)[:R, :K]
        M = np.zeros(R, dtype=np.int32)
        N = np.zeros(K, dtype=np.int32)
        for _ in range(n):
            M[g.integers(0, R)] += 1
            N[g.integers(0, K)] += 1
        rows = np.repeat(np.arange(R), M)
        cols = np.repeat(np.arange(K), N)
        re, im = oracle.ryser_exact_gauss(a[np.ix_(rows, cols)])
        got = oracle.perm_mult_fp64(a, M, N)
        assert (Fraction(got.real), Fraction(got.imag)) == (re, im), trial
    for trial in range(20):
        a, M, N = _random_mult_case(g, int(g.integers(1, 6)), int(g.integers(1, 6)), int(g.integers(1, 11)),
                                    1300 + trial)
        v, t = oracle.perm_mult(a, M, N)
        got = oracle.perm_mult_fp64(a, M, N)
        scale = oracle.perm_mult_abs(a, M, N)
        assert abs(got - (v + t)) <= 1e-13 * scale + 1e-300, (trial, M, N)
    for n in range(1, 13):
        assert oracle.perm_mult_fp64(np.ones((1, 1)), [n], [n]) == math.factorial(n)
    assert oracle.perm_mult_fp64(np.zeros((2, 2)), [0, 0], [0, 0]) == 1


def test_plain_fp64_gray_walk_and_minors():
    """The plain-double Gray walk and minors (the sampling workload's CPU
    timing baseline): exact on Gaussian-integer matrices (every column sum,
    product and partial sum is an exact double at these sizes), within
    plain FP64 rounding of the double-double oracle on Haar matrices, per(J_n)
    = n! exactly, the Laplace identity sum_l v_l minor_l = per([A; v]), and
    the empty cases."""
    for trial in range(8):
        n = 3 + trial
        a = S.gaussian_integer_matrix(n, 1400 + trial, bound=2)
        re, im = oracle.ryser_exact_gauss(a)
        got = oracle.bbfg_gray_fp64(a)
        assert (Fraction(got.real), Fraction(got.imag)) == (re, im), trial
    for n in range(1, 11):
        assert oracle.bbfg_gray_fp64(np.ones((n, n))) == math.factorial(n)
    for n in (8, 12, 16):
        a = S.haar_unitary(n + 4, 1500 + n)[:n, :n]
        v, t = oracle.bbfg_gray(a)
        scale = float(np.prod(np.sqrt((np.abs(a) ** 2).sum(axis=0))))  # Hadamard bound
        assert abs(oracle.bbfg_gray_fp64(a) - (v + t)) <= 1e-13 * scale, n
    assert oracle.bbfg_gray_fp64(np.zeros((0, 0))) == 1
    # minors: against the double-double minors and the Laplace identity
    u = S.haar_unitary(12, 1600)
    a = u[:6, :7]
    M = np.ones(6, dtype=np.int32)
    N = np.ones(7, dtype=np.int32)
    got = oracle.minors_fp64(a, M, N)
    mv, mt = oracle.minors(a, M, N)
    assert np.all(np.abs(got - (mv + mt)) <= 1e-14), np.abs(got - (mv + mt)).max()
    v = u[6, :7]
    pv, pt = oracle.bbfg_gray(np.vstack([a, v[None, :]]))
    assert abs(np.sum(v * got) - (pv + pt)) <= 1e-14
    M2 = np.array([2, 1, 1, 1, 1, 0], dtype=np.int32)   # a repeated row: expanded
    got2 = oracle.minors_fp64(a, M2, N)
    mv2, mt2 = oracle.minors(a, M2, N)
    assert np.all(np.abs(got2 - (mv2 + mt2)) <= 1e-14)


def test_mult_no_photons_and_bad_input():
    assert oracle.perm_mult(np.zeros((2, 2)), [0, 0], [0, 0])[0] == 1
    with pytest.raises(oracle.OracleError):
        oracle.perm_mult(np.ones((2, 2)), [1, 1], [1, 2])   # sum M != sum N
    with pytest.raises(oracle.OracleError):
        oracle.perm_mult(np.ones((2, 2)), [-1, 3], [1, 1])


# ---------------------------------------------------------------- Appendix A.5
def test_all_ones_partial_sum_matches_paper():
    """The positive addends of the normalized all-ones 40x40 matrix sum to the
    worst partial sum the paper prints (about +-27, 6 integer bits)."""
    (n, printed, bits), = read_golden("all_ones_partial_sum.txt")
    n, printed, bits = int(n), int(printed), int(bits)
    a = np.full((1, 1), 1.0 / n)
    pos, neg = oracle.mult_extremes(a, [n], [n])
    worst = max(pos, -neg)
    assert round(worst) == printed
    assert math.ceil(math.log2(worst)) + 1 == bits
    # exact rational evaluation of the same addend classes (independent of C)
    ex_pos = sum(Fraction(math.comb(n - 1, j)) * Fraction(n - 2 * j, n) ** n
                 for j in range(0, n) if j % 2 == 0)
    ex_neg = -sum(Fraction(math.comb(n - 1, j)) * Fraction(n - 2 * j, n) ** n
                  for j in range(0, n) if j % 2 == 1)
    assert abs(pos - float(ex_pos)) < 1e-12 * float(ex_pos)
    assert abs(neg - float(ex_neg)) < 1e-12 * abs(float(ex_neg))
    # and the whole sum is 2^(n-1) per(J/n) = 2^(n-1) n!/n^n
    total = Fraction(2) ** (n - 1) * math.factorial(n) / Fraction(n) ** n
    assert abs((pos + neg) - float(total)) < 1e-12 * worst


def test_abs_sum_bounds_and_closed_form():
    """S_abs >= |perm| (triangle inequality); for the n x n all-ones matrix
    (one row of multiplicity n, one column of multiplicity n) the addends are
    C(n-1, j) |n - 2j|^n, so S_abs = 2^(1-n) sum_j C(n-1, j) |n-2j|^n; a single
    column (K = 1) with one row gives |a|."""
    g = S.rng(21)
    for trial in range(15):
        a, M, N = _random_mult_case(g, 3, 4, int(g.integers(1, 9)), 1400 + trial)
        v, t = oracle.perm_mult(a, M, N)
        assert oracle.perm_mult_abs(a, M, N) >= abs(v + t) * (1 - 1e-14)
    for n in (3, 10, 25):
        ref = sum(math.comb(n - 1, j) * abs(n - 2 * j) ** n for j in range(n)) / 2 ** (n - 1)
        assert abs(oracle.perm_mult_abs(np.ones((1, 1)), [n], [n]) - ref) <= 1e-13 * ref
    assert abs(oracle.perm_mult_abs(np.array([[0.6 - 0.8j]]), [1], [1]) - 1.0) < 1e-15


# ---------------------------------------------------------------- minors
def test_laplace_identity():
    g = S.rng(13)
    for trial in range(20):
        R = int(g.integers(1, 5))
        K = int(g.integers(2, 6))
        n = int(g.integers(2, 9))
        a, M, N = _random_mult_case(g, R, K, n, 1200 + trial)
        # remove one photon from the rows: minors need sum M = sum N - 1
        k = int(np.nonzero(M)[0][0])
        M[k] -= 1
        row = S.random_complex(1, K, 1300 + trial)[0]
        mv, mt = oracle.minors(a, M, N)
        lap = np.sum(N * row * (mv + mt))
        full = np.vstack([a, row[None, :]])
        v, t = oracle.perm_expanded(full, np.append(M, 1), N)
        scale = np.prod(np.abs(full).sum(axis=0) ** N)
        assert abs(lap - (v + t)) <= 1e-14 * scale, trial
        # a column with N_l = 0 gets a zero minor
        for l in np.nonzero(N == 0)[0]:
            assert mv[l] == 0


def test_minors_of_empty_row_set():
    # 0 rows, 1 column with multiplicity 1: the single minor is per(0x0) = 1
    mv, _ = oracle.minors(np.zeros((0, 1)), np.zeros(0, dtype=np.int32), [1])
    assert mv[0] == 1


# ---------------------------------------------------------------- Eq. (bs_p)
def _patterns(n, m):
    for c in itertools.combinations_with_replacement(range(m), n):
        t = np.zeros(m, dtype=np.int32)
        for i in c:
            t[i] += 1
        yield t


@pytest.mark.parametrize("n,m", [(3, 5), (6, 12)])
def test_bs_distribution_sums_to_one(n, m):
    u = S.haar_unitary(m, 20 + n)
    s = np.zeros(m, dtype=np.int32)
    s[:n] = 1
    tot = 0.0
    mean = np.zeros(m)
    count = 0
    for t in _patterns(n, m):
        p = oracle.bs_probability(u, s, t)
        assert -1e-15 <= p <= 1.0 + 1e-12
        tot += p
        mean += p * t
        count += 1
    assert count == math.comb(m + n - 1, n)
    assert abs(tot - 1.0) < 1e-12
    # closed form of the mean occupation: E[t_i] = sum_j s_j |U_ij|^2
    ref = (np.abs(u) ** 2) @ s
    assert np.max(np.abs(mean - ref)) < 1e-12


def test_bs_probability_bosonic_bunching_two_photons():
    """Hong-Ou-Mandel: a balanced beam splitter never gives one photon per
    output port (textbook closed form, probability 0 for (1,1))."""
    u = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2)
    assert oracle.bs_probability(u, [1, 1], [1, 1]) < 1e-30
    assert abs(oracle.bs_probability(u, [1, 1], [2, 0]) - 0.5) < 1e-15


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    for row in read_golden("philox4x32_10_kat.txt"):
        vals = [int(x, 16) for x in row]
        assert oracle.philox4x32_10(vals[0:4], vals[4:6]) == vals[6:10]


# ---------------------------------------------------------------- C&C sampler
def test_cc_sampler_chi_square_tiny():
    scipy_stats = pytest.importorskip("scipy.stats")
    n, m = 3, 5
    u = S.haar_unitary(m, 31)
    s = np.zeros(m, dtype=np.int32)
    s[:n] = 1
    pats = list(_patterns(n, m))
    probs = np.array([oracle.bs_probability(u, s, t) for t in pats])
    counts, margin, _ = oracle.cc_sample(u, s, 4000, seed=12345)
    assert np.all(counts.sum(axis=1) == n)
    index = {tuple(t): i for i, t in enumerate(pats)}
    obs = np.zeros(len(pats))
    for row in counts:
        obs[index[tuple(row)]] += 1
    exp = probs * len(counts)
    keep = exp >= 5
    other_obs = obs[~keep].sum()
    other_exp = exp[~keep].sum()
    o = np.append(obs[keep], other_obs)
    e = np.append(exp[keep], other_exp)
    chi2 = float(np.sum((o - e) ** 2 / np.maximum(e, 1e-300)))
    pval = scipy_stats.chi2.sf(chi2, len(o) - 1)
    assert pval > 1e-3, (chi2, pval)


def test_cc_sampler_lossy_closed_forms():
    """Uniform loss (one loss mode per input photon, transmissivity eta):
    the detected photon number is Binomial(n, eta) exactly, and the mean
    occupation of detected mode i is eta * sum_j |U_ij|^2 over the occupied
    inputs j -- both checked on the oracle's lossy chains."""
    scipy_stats = pytest.importorskip("scipy.stats")
    n, m, eta, ns = 4, 6, 0.5, 3000
    v, mdet = S.config_lossy(n=n, m=m, eta=eta, seed=61)
    counts, _, _ = oracle.cc_sample(v, np.ones(n, np.int32), ns, seed=62, m_detected=mdet)
    assert counts.shape == (ns, m)
    det = counts.sum(axis=1)
    o = np.bincount(det, minlength=n + 1)[: n + 1]
    e = ns * scipy_stats.binom.pmf(np.arange(n + 1), n, eta)
    chi2 = float(np.sum((o - e) ** 2 / e))
    assert scipy_stats.chi2.sf(chi2, n) > 1e-3, (o, e)
    u = S.haar_unitary(m, 61)
    ref = eta * (np.abs(u[:, :n]) ** 2).sum(axis=1)
    mean = counts.mean(axis=0)
    sd = counts.std(axis=0) / np.sqrt(ns)
    assert np.all(np.abs(mean - ref) < 5 * sd + 1e-3), (mean, ref)


def test_cc_sampler_marginals_n6_m12():
    n, m = 6, 12
    u = S.haar_unitary(m, 26)
    s = np.zeros(m, dtype=np.int32)
    s[:n] = 1
    counts, _, _ = oracle.cc_sample(u, s, 3000, seed=777)
    ref = (np.abs(u) ** 2) @ s
    mean = counts.mean(axis=0)
    std = counts.std(axis=0) / np.sqrt(len(counts))
    assert np.all(np.abs(mean - ref) < 5 * std + 1e-3)


def test_cc_sampler_deterministic_in_seed():
    u, occ = S.config_cc(n=5, m=10, seed=3)
    a, _, _ = oracle.cc_sample(u, occ, 20, seed=99)
    b, _, _ = oracle.cc_sample(u, occ, 20, seed=99)
    c, _, _ = oracle.cc_sample(u, occ, 20, seed=100)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def test_cc_sampler_trace_is_consistent_and_first_draw_law():
    """The drawn-row trace: its histogram is the returned occupation, a
    max_steps run is a prefix of the full run, the smallest step margin is the
    sample's margin, and the first draw follows the closed form of C&C's first
    step: after the uniform column permutation, P(r_1 = i) = (1/n) sum_j s_j
    |U_ij|^2 (the first weight is |U_i,col_1|^2)."""
    scipy_stats = pytest.importorskip("scipy.stats")
    u, occ = S.config_cc(n=5, m=10, seed=3)
    counts, margin, _, rows, sm = oracle.cc_sample(u, occ, 30, seed=5, trace=True)
    assert rows.shape == (30, 5) and sm.shape == (30, 5)
    for s in range(30):
        assert np.array_equal(np.bincount(rows[s], minlength=10), counts[s])
        assert sm[s].min() == margin[s]
    _, _, _, rows3, _ = oracle.cc_sample(u, occ, 30, seed=5, max_steps=3, trace=True)
    assert np.array_equal(rows3, rows[:, :3])
    ns = 20000
    _, _, _, first, _ = oracle.cc_sample(u, occ, ns, seed=6, max_steps=1, trace=True)
    p = (np.abs(u) ** 2) @ occ / occ.sum()
    o = np.bincount(first[:, 0], minlength=10)
    e = ns * p
    chi2 = float(np.sum((o - e) ** 2 / e))
    assert scipy_stats.chi2.sf(chi2, 9) > 1e-3, (o, e)
