"""CPU oracle for the generalized BB/FG permanent (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it and
shares no code with it.  The arithmetic lives in ``oracle.c`` (complex
double-double); this module marshals numpy arrays through ctypes.

Every function returns complex results as ``(value, tail)`` pairs where
``value`` is the double-double rounded to complex128 and ``tail`` is the low
part (so value + tail carries ~106 bits) -- except ``perm_mult_fp64``, the
same term-by-term walk in plain double (a timing baseline), which returns
one complex128.
"""
from __future__ import annotations

import ctypes as C
import numpy as np

from .build import build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        for name in ("orc_perm_bruteforce", "orc_ryser_gray"):
            getattr(L, name).argtypes = [C.c_int, dp, C.c_int, dp]
        for name in ("orc_bbfg_gray", "orc_bbfg_direct", "orc_bbfg_gray_fp64"):
            getattr(L, name).argtypes = [C.c_int, C.c_int, dp, C.c_int, dp]
        for name in ("orc_perm_mult", "orc_perm_expanded", "orc_minors", "orc_bbfg_mult_extremes",
                     "orc_perm_mult_abs", "orc_perm_mult_fp64", "orc_minors_fp64"):
            getattr(L, name).argtypes = [C.c_int, C.c_int, dp, C.c_int, ip, ip, dp]
        L.orc_gray_sequence.argtypes = [C.c_int, C.POINTER(C.c_uint64)]
        L.orc_ryser_exact_gauss.argtypes = [C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.orc_philox4x32_10.restype = None
        L.orc_cc_sample.argtypes = [C.c_int, C.c_int, dp, C.c_int, ip, C.c_int, C.c_uint64, C.c_int,
                                    C.c_int, ip, dp, dp, ip, dp]
        _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _mat(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    if a.ndim != 2:
        raise ValueError("matrix must be 2-D")
    return a


def _dp(x):
    return x.ctypes.data_as(C.POINTER(C.c_double))


def _ip(x):
    return x.ctypes.data_as(C.POINTER(C.c_int))


def _chk(rc, name):
    if rc != 0:
        raise OracleError(f"{name} failed with code {rc}")


def _zdd(out):
    return complex(out[0], out[2]), complex(out[1], out[3])


def _dd_value(out):
    """Return the double-double as a (value, tail) complex pair."""
    return _zdd(out)


def perm_bruteforce(a):
    """Eq. (perm_def): sum over all permutations (n <= 10)."""
    a = _mat(a)
    n = a.shape[0]
    assert a.shape == (n, n)
    out = np.zeros(4)
    _chk(lib().orc_perm_bruteforce(n, _dp(a.view(np.float64)), n, _dp(out)), "perm_bruteforce")
    return _dd_value(out)


def bbfg_gray(a):
    """Eq. (bbfg), delta_1=+1, binary reflected Gray walk; r x c allowed."""
    a = _mat(a)
    r, c = a.shape
    out = np.zeros(4)
    _chk(lib().orc_bbfg_gray(r, c, _dp(a.view(np.float64)), c, _dp(out)), "bbfg_gray")
    return _dd_value(out)


def bbfg_gray_fp64(a):
    """The bbfg_gray walk in plain double arithmetic (the plain-FP64 CPU
    form of Eq. (bbfg), a timing baseline)."""
    a = _mat(a)
    r, c = a.shape
    out = np.zeros(2)
    _chk(lib().orc_bbfg_gray_fp64(r, c, _dp(a.view(np.float64)), c, _dp(out)), "bbfg_gray_fp64")
    return complex(out[0], out[1])


def gray_sequence(bits):
    """Gray codes visited by the bbfg_gray walk (bit t <-> delta_{t+2} = -1)."""
    out = np.zeros(1 << bits, dtype=np.uint64)
    _chk(lib().orc_gray_sequence(bits, out.ctypes.data_as(C.POINTER(C.c_uint64))), "gray_sequence")
    return [int(x) for x in out]


def bbfg_direct(a):
    """Eq. (bbfg) with column sums recomputed for each delta (no Gray reuse)."""
    a = _mat(a)
    r, c = a.shape
    out = np.zeros(4)
    _chk(lib().orc_bbfg_direct(r, c, _dp(a.view(np.float64)), c, _dp(out)), "bbfg_direct")
    return _dd_value(out)


def ryser(a):
    """Eq. (ryser), Gray-ordered subsets."""
    a = _mat(a)
    n = a.shape[0]
    assert a.shape == (n, n)
    out = np.zeros(4)
    _chk(lib().orc_ryser_gray(n, _dp(a.view(np.float64)), n, _dp(out)), "ryser_gray")
    return _dd_value(out)


def _exact_gauss_call(name, a_int):
    a = np.asarray(a_int)
    n = a.shape[0]
    buf = np.zeros((n, n, 2), dtype=np.int64)
    buf[..., 0] = np.real(a).astype(np.int64)
    buf[..., 1] = np.imag(a).astype(np.int64)
    buf = np.ascontiguousarray(buf)
    out = np.zeros(4, dtype=np.int64)
    _chk(getattr(lib(), name)(n, buf.ctypes.data_as(C.POINTER(C.c_int64)),
                              out.ctypes.data_as(C.POINTER(C.c_int64))), name)

    def join(hi, lo):
        return (int(hi) << 64) + (int(lo) & ((1 << 64) - 1))
    return join(out[0], out[1]), join(out[2], out[3])


def ryser_exact_gauss(a_int):
    """Exact Ryser for Gaussian-integer matrices; returns a Python complex of ints
    as a (re, im) tuple of Python ints."""
    return _exact_gauss_call("orc_ryser_exact_gauss", a_int)


def nw(a):
    """Nijenhuis-Wilf form of Eq. (ryser) (Sec. 2), Gray-ordered subsets."""
    a = _mat(a)
    n = a.shape[0]
    assert a.shape == (n, n)
    out = np.zeros(4)
    _chk(lib().orc_nw_gray(n, _dp(a.view(np.float64)), n, _dp(out)), "nw_gray")
    return _dd_value(out)


def nw_exact_gauss(a_int):
    """Exact Nijenhuis-Wilf for Gaussian-integer matrices; (re, im) Python ints."""
    return _exact_gauss_call("orc_nw_exact_gauss", a_int)


def formula_abs(which, a):
    """Modulus-sum of the addends of Eq. (ryser) (which='ryser') or of the
    Nijenhuis-Wilf form (which='nw'), times the prefactor's modulus."""
    a = _mat(a)
    n = a.shape[0]
    out = np.zeros(1)
    code = {"ryser": 1, "nw": 2}[which]
    _chk(lib().orc_formula_abs(code, n, _dp(a.view(np.float64)), n, _dp(out)), "formula_abs")
    return float(out[0])


def _mult_call(name, a, row_mult, col_mult, nout):
    a = _mat(a)
    R, K = a.shape
    M = np.ascontiguousarray(np.asarray(row_mult, dtype=np.int32))
    N = np.ascontiguousarray(np.asarray(col_mult, dtype=np.int32))
    assert M.shape == (R,) and N.shape == (K,)
    out = np.zeros(nout)
    _chk(getattr(lib(), name)(R, K, _dp(a.view(np.float64)), K, _ip(M), _ip(N), _dp(out)), name)
    return out


def perm_mult(a, row_mult, col_mult):
    """Eq. (bbfgrepeated) term by term (plain odometer order, direct binomials)."""
    return _dd_value(_mult_call("orc_perm_mult", a, row_mult, col_mult, 4))


def perm_expanded(a, row_mult, col_mult):
    """per() of the matrix expanded by the multiplicities, via bbfg_gray."""
    return _dd_value(_mult_call("orc_perm_expanded", a, row_mult, col_mult, 4))


def minors(a, row_mult, col_mult):
    """Laplace minors: per(expanded a with one copy of column l removed)."""
    K = np.asarray(a).shape[1]
    out = _mult_call("orc_minors", a, row_mult, col_mult, 4 * K).reshape(K, 4)
    val = out[:, 0] + 1j * out[:, 2]
    tail = out[:, 1] + 1j * out[:, 3]
    return val, tail


def minors_fp64(a, row_mult, col_mult):
    """Laplace minors as minors(), each by the plain-double Gray walk
    (timing baseline)."""
    K = np.asarray(a).shape[1]
    out = _mult_call("orc_minors_fp64", a, row_mult, col_mult, 2 * K).reshape(K, 2)
    return out[:, 0] + 1j * out[:, 1]


def perm_mult_fp64(a, row_mult, col_mult):
    """Eq. (bbfgrepeated) term by term in plain double arithmetic: the
    plain-FP64 CPU form of the method (a timing baseline)."""
    out = _mult_call("orc_perm_mult_fp64", a, row_mult, col_mult, 2)
    return complex(out[0], out[1])


def perm_mult_abs(a, row_mult, col_mult):
    """Modulus-sum S_abs of the addends of Eq. (bbfgrepeated) (with 2^(1-n))."""
    return float(_mult_call("orc_perm_mult_abs", a, row_mult, col_mult, 1)[0])


def mult_extremes(a, row_mult, col_mult):
    """(sum of positive, sum of negative) real addends of Eq. (bbfgrepeated)."""
    out = _mult_call("orc_bbfg_mult_extremes", a, row_mult, col_mult, 2)
    return float(out[0]), float(out[1])


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(o[i]) for i in range(4)]


def cc_sample(u, occupation, n_samples, seed, m_detected=0, max_steps=0, trace=False):
    """Clifford & Clifford sampler.  ``u`` is m x m' (rows = output modes),
    ``occupation`` has length m'.  Returns (counts[n_samples, m_det],
    margin[n_samples], addend_ops) where margin is the smallest relative
    distance of a draw to a CDF boundary in each sample.  With trace=True
    two more arrays follow: rows[n_samples, steps], the drawn row of every
    step in draw order, and step_margin[n_samples, steps], the margin of
    each draw alone (steps = max_steps, or n when max_steps <= 0)."""
    u = _mat(u)
    m, mc = u.shape
    occ = np.ascontiguousarray(np.asarray(occupation, dtype=np.int32))
    assert occ.shape == (mc,)
    mdet = m if m_detected <= 0 else int(m_detected)
    n = int(occ.sum())
    steps = n if max_steps <= 0 or max_steps > n else int(max_steps)
    out = np.zeros((n_samples, mdet), dtype=np.int32)
    margin = np.zeros(max(n_samples, 1))
    ops = np.zeros(1)
    rows = np.zeros((max(n_samples, 1), max(steps, 1)), dtype=np.int32)
    smargin = np.zeros((max(n_samples, 1), max(steps, 1)))
    _chk(lib().orc_cc_sample(m, mc, _dp(u.view(np.float64)), mc, _ip(occ), int(n_samples),
                             C.c_uint64(int(seed) & ((1 << 64) - 1)), int(mdet), int(max_steps),
                             _ip(out), _dp(margin), _dp(ops),
                             _ip(rows) if trace else None, _dp(smargin) if trace else None), "cc_sample")
    if trace:
        return out, margin[:n_samples], float(ops[0]), rows[:n_samples, :steps], smargin[:n_samples, :steps]
    return out, margin[:n_samples], float(ops[0])


def bs_probability(u, s, t):
    """Eq. (bs_p): |per(U_ST)|^2 / prod s_i! t_i!, U_ST built by repeating
    column i s_i times and row j t_j times; per() by perm_expanded."""
    from math import factorial
    u = _mat(u)
    s = np.asarray(s, dtype=np.int32)
    t = np.asarray(t, dtype=np.int32)
    rows = np.nonzero(t)[0]
    cols = np.nonzero(s)[0]
    if len(rows) == 0 and len(cols) == 0:
        return 1.0
    sub = u[np.ix_(rows, cols)]
    val, tail = perm_expanded(sub, t[rows], s[cols])
    den = 1
    for x in s:
        den *= factorial(int(x))
    for x in t:
        den *= factorial(int(x))
    p = abs(val) ** 2 + 2 * (val.real * tail.real + val.imag * tail.imag)
    return p / den
