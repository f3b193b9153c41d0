"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the permanent method itself: it only draws
random matrices and multiplicity patterns with numpy's PCG64 generator, in the
shapes of the paper's workloads (random unitary interferometers with random
row/column multiplicities, Sec. 3.1 and Sec. 4).

Workloads (sizes as named in the docstrings of each generator):
  * ``config_single``  - one 12-photon permanent from a 24-mode Haar unitary,
                         output multiplicities (3,2,2,1,1,1,1,1), 12 inputs.
  * ``config_batch``   - 4096 permanents of k ~ U[10,28] photons from 60-mode
                         Haar unitaries, outputs collapsed binomially.
  * ``config_cc``      - Clifford & Clifford sampling, n=30 photons, m=60.
  * ``config_serving`` - 64 sampling chains, n ~ U[16,34], m=60.
  * ``config_lossy``   - 40 photons, m=60, uniform transmissivity 0.5.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng", "haar_unitary", "random_complex", "gaussian_integer_matrix",
    "config_single", "config_batch", "config_cc", "config_serving", "config_lossy",
    "collapse_modes", "lossy_isometry", "block_diagonal",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def haar_unitary(m: int, seed: int) -> np.ndarray:
    """Haar-random m x m unitary: QR of a complex Ginibre matrix with the
    phases of R's diagonal moved into Q (Mezzadri, Notices AMS 54 (2007))."""
    g = rng(seed)
    z = (g.standard_normal((m, m)) + 1j * g.standard_normal((m, m))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    ph = d / np.abs(d)
    return np.ascontiguousarray(q * ph[None, :], dtype=np.complex128)


def random_complex(rows: int, cols: int, seed: int, scale: float = 1.0) -> np.ndarray:
    g = rng(seed)
    a = (g.standard_normal((rows, cols)) + 1j * g.standard_normal((rows, cols))) * scale
    return np.ascontiguousarray(a, dtype=np.complex128)


def gaussian_integer_matrix(n: int, seed: int, bound: int = 3) -> np.ndarray:
    """Entries a+bi with integers |a|,|b| <= bound (exactly representable)."""
    g = rng(seed)
    re = g.integers(-bound, bound + 1, size=(n, n))
    im = g.integers(-bound, bound + 1, size=(n, n))
    return np.ascontiguousarray(re + 1j * im, dtype=np.complex128)


def collapse_modes(k: int, m: int, g: np.random.Generator):
    """Throw k photons uniformly (with replacement) into m modes; return the
    occupied modes (ascending) and their occupation counts."""
    hits = g.integers(0, m, size=k)
    modes, counts = np.unique(hits, return_counts=True)
    return modes.astype(np.int64), counts.astype(np.int32)


def config_single(seed: int = 1):
    """12-photon permanent with row multiplicities (3,2,2,1,1,1,1,1).

    Haar 24x24 unitary from ``seed``; inputs are modes 0..11 with one photon
    each (columns); the output uses the first 8 modes of a seeded permutation
    of the 24 modes (rows).  Returns (A[8,12], row_mult[8], col_mult[12], U,
    row_modes)."""
    u = haar_unitary(24, seed)
    g = rng(seed + 1000)
    rows = g.permutation(24)[:8]
    mult = np.array([3, 2, 2, 1, 1, 1, 1, 1], dtype=np.int32)
    a = np.ascontiguousarray(u[np.ix_(rows, np.arange(12))])
    return a, mult, np.ones(12, dtype=np.int32), u, rows


def config_batch(count: int = 4096, seed: int = 2, kmin: int = 10, kmax: int = 28,
                 m: int = 60, group: int = 64):
    """Batch of ``count`` permanents with k ~ U[kmin,kmax] photons each.

    Items are grouped by ``group`` and each group shares one Haar m x m
    unitary.  Per item: k distinct input modes (columns, multiplicity 1) drawn
    without replacement; k output photons thrown uniformly with replacement
    into the m output modes (rows, multiplicities = collision counts, so
    P(repeat) ~ k^2/2m).  Returns a list of (A, row_mult, col_mult)."""
    g = rng(seed)
    items = []
    u = None
    for t in range(count):
        if t % group == 0:
            u = haar_unitary(m, seed * 100003 + t // group)
        k = int(g.integers(kmin, kmax + 1))
        cols = np.sort(g.choice(m, size=k, replace=False))
        rows, rmult = collapse_modes(k, m, g)
        a = np.ascontiguousarray(u[np.ix_(rows, cols)])
        items.append((a, rmult, np.ones(k, dtype=np.int32)))
    return items


def config_cc(n: int = 30, m: int = 60, seed: int = 3):
    """Clifford & Clifford workload: Haar m x m unitary, one photon in each of
    modes 0..n-1.  Returns (U, input_occupation[m])."""
    u = haar_unitary(m, seed)
    occ = np.zeros(m, dtype=np.int32)
    occ[:n] = 1
    return u, occ


def config_serving(chains: int = 64, nmin: int = 16, nmax: int = 34, m: int = 60,
                   seed: int = 4, rate_hz: float = 200.0):
    """Serving workload: ``chains`` sampling chains, each with its own Haar
    m x m unitary and photon number n ~ U[nmin, nmax] (one photon in modes
    0..n-1); Poisson arrival offsets (seconds) at ``rate_hz`` (inf: all at
    time 0).  The unitaries and photon numbers do not depend on the rate."""
    g = rng(seed)
    out = []
    t = 0.0
    for c in range(chains):
        n = int(g.integers(nmin, nmax + 1))
        t += float(g.exponential(1.0)) / rate_hz  # inf: 0
        occ = np.zeros(m, dtype=np.int32)
        occ[:n] = 1
        out.append(dict(unitary=haar_unitary(m, seed * 7919 + c), occupation=occ,
                        arrival_s=t, seed=seed * 1000 + c))
    return out


def lossy_isometry(u: np.ndarray, inputs: np.ndarray, eta: float) -> np.ndarray:
    """(m + n) x n isometry for uniform transmissivity ``eta``: the columns of
    U for the input modes scaled by sqrt(eta), stacked on sqrt(1-eta) times the
    n x n identity (one loss mode per photon)."""
    a = np.sqrt(eta) * u[:, inputs]
    loss = np.sqrt(1.0 - eta) * np.eye(len(inputs), dtype=np.complex128)
    return np.ascontiguousarray(np.vstack([a, loss]))


def config_lossy(n: int = 40, m: int = 60, eta: float = 0.5, seed: int = 5):
    """Lossy sampling workload: Haar m x m unitary, one photon in modes
    0..n-1, loss modelled by ``lossy_isometry``.  Returns (V[(m+n) x n],
    m_detected)."""
    u = haar_unitary(m, seed)
    v = lossy_isometry(u, np.arange(n), eta)
    return v, m


def block_diagonal(K: int, n: int, seed: int, width: int = 12, mult: int = 3):
    """Block-diagonal problem with K distinct columns (multiplicity 1) and n
    photons (n = K for a permanent, K - 1 for Laplace minors).

    The columns are split into ceil(K / width) nearly equal consecutive
    groups; group g gets its own distinct rows, as many of multiplicity
    ``mult`` as fit and the rest of multiplicity 1, whose multiplicities sum
    to the group's column count -- except the last group, which gets one
    photon less when n = K - 1.  The entries of each block are a block of one
    Haar 64 x 64 unitary (disjoint rows and columns); every entry outside the
    blocks is zero.  Returns (A[R, K], row_mult[R], col_mult[K], groups) with
    groups = [(row indices, column indices), ...] into A."""
    assert n in (K, K - 1) and K >= 1
    u = haar_unitary(64, seed)
    g = rng(seed + 17)
    ngroups = -(-K // width)
    bounds = [K * i // ngroups for i in range(ngroups + 1)]
    rows_m, groups = [], []
    for gi in range(ngroups):
        kc = bounds[gi + 1] - bounds[gi]
        photons = kc - (1 if (n == K - 1 and gi == ngroups - 1) else 0)
        ms = [mult] * (photons // mult) + [1] * (photons % mult)
        first = len(rows_m)
        rows_m.extend(ms)
        groups.append((list(range(first, len(rows_m))), list(range(bounds[gi], bounds[gi + 1]))))
    R = len(rows_m)
    src_rows = g.permutation(64)[:R]
    src_cols = g.permutation(64)[:K]
    a = np.zeros((R, K), dtype=np.complex128)
    for rows, cols in groups:
        a[np.ix_(rows, cols)] = u[np.ix_(src_rows[rows], src_cols[cols])]
    return a, np.array(rows_m, dtype=np.int32), np.ones(K, dtype=np.int32), groups
