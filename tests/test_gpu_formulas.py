"""Ryser's formula and its Nijenhuis-Wilf form on the GPU (bs_perm_formula),
the comparison of Sec. 3.2, against the oracle.

Tolerance: every formula is walked in FP64 with re-seeded sums and
double-double partials, so its rounding error is a small multiple of
n * 2^-53 times the modulus sum of its addends (S_abs, computed by the
oracle); 1e-12 * S_abs leaves a margin of about 50 at n = 18.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic as S

pytestmark = pytest.mark.gpu

FORMULAS = ("bbfg", "ryser", "nw")


def _s_abs(formula, a):
    n = a.shape[0]
    if formula == "bbfg":
        return oracle.perm_mult_abs(a, np.ones(n, np.int32), np.ones(n, np.int32))
    return oracle.formula_abs(formula, a)


@pytest.mark.parametrize("formula", FORMULAS)
def test_formula_matches_oracle_on_unitary_blocks(ctx, formula):
    for n in (1, 2, 3, 5, 8, 11, 14, 18):
        a = S.haar_unitary(2 * n, 900 + n)[:n, :n]
        got, tail = ctx.perm_formula(a, formula, with_tail=True)
        ref, ref_tail = oracle.bbfg_gray(a)
        err = abs((got - ref) + (tail - ref_tail))
        assert err <= 1e-12 * _s_abs(formula, a), (formula, n, err)


@pytest.mark.parametrize("formula", FORMULAS)
def test_formula_exact_on_gaussian_integers(ctx, formula):
    """Small Gaussian-integer matrices: every sum and product is an exact
    double (halves included for Nijenhuis-Wilf), so the result is the exact
    integer permanent."""
    for n in range(1, 9):
        a = S.gaussian_integer_matrix(n, 940 + n, bound=3)
        re, im = oracle.ryser_exact_gauss(a)
        got, tail = ctx.perm_formula(a.astype(np.complex128), formula, with_tail=True)
        assert (got.real + tail.real, got.imag + tail.imag) == (float(re), float(im)), (formula, n)


@pytest.mark.parametrize("formula", FORMULAS)
def test_formula_closed_forms(ctx, formula):
    for n in range(1, 13):
        got = ctx.perm_formula(np.ones((n, n)), formula)
        assert got == complex(math.factorial(n)), (formula, n)
    d = S.random_complex(1, 9, 960)[0]
    got = ctx.perm_formula(np.diag(d), formula)
    assert abs(got - np.prod(d)) <= 1e-14 * abs(np.prod(d))
    assert ctx.perm_formula(np.zeros((0, 0)), formula) == 1


def test_formula_bbfg_equals_bs_perm(ctx):
    a = S.haar_unitary(40, 970)[:20, :20]
    assert ctx.perm_formula(a, "bbfg") == ctx.perm(a)


def test_formula_invalid_arguments(ctx):
    import paper_2309_07027_gb300 as bs
    lib = bs.load()
    out = np.zeros(1, np.complex128)
    a = np.eye(3, dtype=np.complex128)
    assert lib.bs_perm_formula(ctx._p, a.ctypes.data, 3, 3, 7, out.ctypes.data, None) == bs.BS_EINVAL
    assert lib.bs_perm_formula(ctx._p, a.ctypes.data, 3, 2, 1, out.ctypes.data, None) == bs.BS_EINVAL
    assert lib.bs_perm_formula(ctx._p, a.ctypes.data, 49, 49, 1, out.ctypes.data, None) == bs.BS_EINVAL
    assert lib.bs_perm_formula(ctx._p, a.ctypes.data, -1, 3, 2, out.ctypes.data, None) == bs.BS_EINVAL
    assert lib.bs_perm_formula(ctx._p, a.ctypes.data, 3, 3, 2, None, None) == bs.BS_EINVAL
