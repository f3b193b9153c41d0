"""GB300 (sm_103a) boson-sampling permanents: Python binding of libbs.so.

This module only marshals arguments for the C ABI declared in
``include/bs.h``; every step of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: if ``libbs.so`` is missing or cannot be
loaded an ``ImportError``-style ``RuntimeError`` is raised, and compute calls
on a machine without a GPU raise ``BsError`` (BS_ENODEV).

Entry points (names follow the C ABI):
  Context.perm(A, row_mult, col_mult, mode)            -> complex
  Context.perm_batch(items, mode)                      -> complex array
  Context.perm_batch_dev(A_packed_dev, ..., out_dev)   (torch CUDA tensors)
  Context.laplace_minors(A, row_mult, col_mult, mode)  -> complex array
  Context.sample(U, occupation, n_samples, seed, mode) -> int array
  Context.sample_ex / sample_dev                        (general / device forms)
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = ["BS_FP64", "BS_MIXED", "BS_DF64", "BsError", "Context", "Server", "library_path", "load", "debug_gray_walk",
           "debug_plan", "perm_noalloc", "MAX_N"]

BS_FP64 = 0
BS_MIXED = 1
BS_DF64 = 2  # double-float: FP64-class results on the FP32 pipe
# statistics slots by kernel family: FP64, FP32, double-float
PRECISIONS = ("fp64", "fp32", "df")
# formulas of bs_perm_formula (bs_formula)
FORMULAS = {"bbfg": 0, "ryser": 1, "nw": 2}
MAX_N = 48

BS_OK, BS_EINVAL, BS_ENOMEM, BS_ECUDA, BS_ETIMEOUT, BS_ENODEV, BS_ECANCELED = 0, -1, -2, -3, -4, -5, -6  # noqa: E501
_CODES = {BS_EINVAL: "BS_EINVAL", BS_ENOMEM: "BS_ENOMEM", BS_ECUDA: "BS_ECUDA", BS_ETIMEOUT: "BS_ETIMEOUT",
          BS_ENODEV: "BS_ENODEV", BS_ECANCELED: "BS_ECANCELED"}

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_HERE, "libbs.so")


class BsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_CODES.get(code, code)}: {msg}")
        self.code = code


class _Stats(C.Structure):
    # index 0: FP64 walk kernels, 1: FP32 walk kernels, 2: double-float walk kernels
    _fields_ = [("walk_launches", C.c_uint64), ("kernel_launches", C.c_uint64), ("addends", C.c_uint64 * 3),
                ("addend_flops", C.c_uint64 * 3), ("walk_ms", C.c_double * 3), ("timed_launches", C.c_uint64 * 3)]


class _ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("ticks", C.c_uint64),
                ("walk_launches", C.c_uint64), ("busy_s", C.c_double), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("max_ms", C.c_double), ("max_resident", C.c_int),
                ("mem_peak_bytes", C.c_size_t), ("mem_in_use_bytes", C.c_size_t), ("resident", C.c_int),
                ("waiting", C.c_int), ("cancelled", C.c_uint64)]


_lib = None


def load():
    """Load libbs.so (built by ``__graft_entry__.build()`` / ``_build.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libbs.so not found at {path}: build it with "
                           f"`python -m paper_2309_07027_gb300._build` (needs nvcc); there is no fallback")
    L = C.CDLL(path)
    vp, ip, dp, i64p = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_int64)
    sig = {
        "bs_ctx_create": ([C.POINTER(C.c_void_p), C.c_int, C.c_size_t], C.c_int),
        "bs_ctx_destroy": ([vp], None),
        "bs_last_error": ([vp], C.c_char_p),
        "bs_ctx_set_stream": ([vp, vp], C.c_int),
        "bs_ctx_use_own_stream": ([vp], C.c_int),
        "bs_ctx_sync": ([vp], C.c_int),
        "bs_ctx_set_deadline": ([vp, C.c_double], C.c_int),
        "bs_ctx_set_chunk_log2": ([vp, C.c_int, C.c_int], C.c_int),
        "bs_ctx_get_chunk_log2": ([vp, C.c_int], C.c_int),
        "bs_ctx_set_mixed_tolerance": ([vp, C.c_double], C.c_int),
        "bs_tune": ([vp, C.c_int, C.c_int, C.c_int, ip, dp], C.c_int),
        "bs_perm": ([vp, vp, C.c_int, C.c_int, C.c_int, ip, ip, C.c_int, vp, vp], C.c_int),
        "bs_perm_formula": ([vp, vp, C.c_int, C.c_int, C.c_int, vp, vp], C.c_int),
        "bs_perm_batch": ([vp, C.c_int, vp, i64p, ip, ip, ip, i64p, i64p, C.c_int, vp], C.c_int),
        "bs_perm_batch_dev": ([vp, C.c_int, vp, i64p, ip, ip, ip, i64p, i64p, C.c_int, vp], C.c_int),
        "bs_laplace_minors": ([vp, vp, C.c_int, C.c_int, C.c_int, ip, ip, C.c_int, vp], C.c_int),
        "bs_sample": ([vp, vp, C.c_int, ip, C.c_int, C.c_uint64, C.c_int, ip], C.c_int),
        "bs_sample_ex": ([vp, vp, C.c_int, C.c_int, C.c_int, ip, C.c_int, C.c_uint64, C.c_int, C.c_int, ip],
                         C.c_int),
        "bs_sample_dev": ([vp, vp, C.c_int, C.c_int, C.c_int, ip, C.c_int, C.c_uint64, C.c_int, C.c_int, vp],
                          C.c_int),
        "bs_sample_trace": ([vp, vp, C.c_int, C.c_int, C.c_int, ip, C.c_int, C.c_uint64, C.c_int, C.c_int, ip,
                             ip], C.c_int),
        "bs_ctx_set_profiling": ([vp, C.c_int], C.c_int),
        "bs_ctx_set_graphs": ([vp, C.c_int], C.c_int),
        "bs_ctx_get_stats": ([vp, C.POINTER(_Stats)], C.c_int),
        "bs_ctx_get_walk_times": ([vp, dp, C.c_int], C.c_int),
        "bs_ctx_reset_stats": ([vp], C.c_int),
        "bs_measure_fma_rates": ([vp, dp, dp], C.c_int),
        "bs_debug_gray_walk": ([C.c_int, C.c_int, ip, C.c_uint64, C.c_int, ip, ip, C.POINTER(C.c_uint64)],
                               C.c_int),
        "bs_debug_plan": ([C.c_int, C.c_int, ip, ip, C.c_int, i64p], C.c_int),
        "bs_debug_mixed_error": ([C.c_int, C.c_int, ip, ip, C.c_int, C.c_int, dp, ip, ip], C.c_int),
        "bs_perm_noalloc": ([vp, C.c_int, C.c_int, C.c_int, ip, ip, C.c_int, vp, vp, vp], C.c_int),
        "bs_server_create": ([C.POINTER(C.c_void_p), C.c_int, C.c_size_t, C.c_int, C.c_int, C.c_int], C.c_int),
        "bs_server_destroy": ([vp], None),
        "bs_server_submit": ([vp, C.c_int, vp, C.c_int, C.c_int, C.c_int, ip, ip], C.c_int64),
        "bs_server_poll": ([vp, C.c_int64, vp, C.c_int, dp], C.c_int),
        "bs_server_wait": ([vp, C.c_int64, vp, C.c_int, dp], C.c_int),
        "bs_server_submit_sample": ([vp, vp, C.c_int, C.c_int, C.c_int, ip, C.c_uint64, C.c_uint64, C.c_int],
                                    C.c_int64),
        "bs_server_poll_sample": ([vp, C.c_int64, ip, C.c_int, dp], C.c_int),
        "bs_server_wait_sample": ([vp, C.c_int64, ip, C.c_int, dp], C.c_int),
        "bs_server_cancel": ([vp, C.c_int64], C.c_int),
        "bs_server_get_stats": ([vp, C.POINTER(_ServerStats)], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _err(ctx_ptr):
    return load().bs_last_error(ctx_ptr).decode()


def _check(rc, ctx_ptr=None):
    if rc != BS_OK:
        raise BsError(rc, _err(ctx_ptr))


def _c128(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    if a.ndim != 2:
        raise ValueError("matrix must be 2-D")
    return a


def _i32(x, n=None):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.int32))
    if n is not None and x.shape != (n,):
        raise ValueError(f"expected {n} multiplicities, got shape {x.shape}")
    return x


def _ip(x):
    return x.ctypes.data_as(C.POINTER(C.c_int))


def _i64p(x):
    return x.ctypes.data_as(C.POINTER(C.c_int64))


class Context:
    """One GPU context (stream, device buffers, memory budget)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        L = load()
        p = C.c_void_p()
        _check(L.bs_ctx_create(C.byref(p), int(device), int(mem_budget_bytes)))
        self._p = p
        self._L = L

    def close(self):
        if getattr(self, "_p", None):
            self._L.bs_ctx_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------- control
    def set_stream(self, stream):
        """Use a ``torch.cuda.Stream`` (or a raw cudaStream_t handle; 0 is the
        legacy default stream) for later work; ``None`` returns to the
        context's own stream."""
        if stream is None:
            _check(self._L.bs_ctx_use_own_stream(self._p), self._p)
            return
        handle = int(getattr(stream, "cuda_stream", stream))
        _check(self._L.bs_ctx_set_stream(self._p, C.c_void_p(handle)), self._p)

    def sync(self):
        _check(self._L.bs_ctx_sync(self._p), self._p)

    def set_deadline(self, seconds: float):
        _check(self._L.bs_ctx_set_deadline(self._p, float(seconds)), self._p)

    def set_chunk_log2(self, mode: int, log2_chunk_max: int):
        _check(self._L.bs_ctx_set_chunk_log2(self._p, int(mode), int(log2_chunk_max)), self._p)

    def chunk_log2(self, mode: int) -> int:
        return int(self._L.bs_ctx_get_chunk_log2(self._p, int(mode)))

    def set_mixed_tolerance(self, tol: float = 1e-6):
        """MIXED accuracy target (bs_ctx_set_mixed_tolerance); >= 1e300 forces FP32."""
        _check(self._L.bs_ctx_set_mixed_tolerance(self._p, float(tol)), self._p)

    def set_graphs(self, on: bool):
        """Replay the sampler's step loop from a captured CUDA graph (default)."""
        _check(self._L.bs_ctx_set_graphs(self._p, 1 if on else 0), self._p)

    def tune(self, mode: int, kind: int = 1, K: int = 28):
        """Autotune the chunk-length cap for ``mode``; returns (log2, addends/s)."""
        b = C.c_int()
        r = C.c_double()
        _check(self._L.bs_tune(self._p, int(mode), int(kind), int(K), C.byref(b), C.byref(r)), self._p)
        return b.value, r.value

    def set_profiling(self, on: bool):
        _check(self._L.bs_ctx_set_profiling(self._p, 1 if on else 0), self._p)

    def stats(self) -> dict:
        s = _Stats()
        _check(self._L.bs_ctx_get_stats(self._p, C.byref(s)), self._p)
        out = {}
        for f, _ in _Stats._fields_:
            v = getattr(s, f)
            out[f] = list(v) if hasattr(v, "__len__") else v
        return out

    def walk_times(self, max_entries: int = 4096):
        """Per-launch walk durations (ms) timed since the last call."""
        buf = np.zeros(max_entries, dtype=np.float64)
        n = self._L.bs_ctx_get_walk_times(self._p, buf.ctypes.data_as(C.POINTER(C.c_double)), max_entries)
        if n < 0:
            _check(n, self._p)
        return buf[:min(n, max_entries)].copy()

    def reset_stats(self):
        _check(self._L.bs_ctx_reset_stats(self._p), self._p)

    def measure_fma_rates(self):
        """(fp64, fp32) lane-FMA/s measured on this device."""
        a, b = C.c_double(), C.c_double()
        _check(self._L.bs_measure_fma_rates(self._p, C.byref(a), C.byref(b)), self._p)
        return a.value, b.value

    # ---------------------------------------------------------- permanents
    def perm(self, a, row_mult=None, col_mult=None, mode: int = BS_FP64, with_tail: bool = False):
        a = _c128(a)
        R, K = a.shape
        M = _i32(np.ones(R) if row_mult is None else row_mult, R)
        N = _i32(np.ones(K) if col_mult is None else col_mult, K)
        out = np.zeros(1, dtype=np.complex128)
        lo = np.zeros(1, dtype=np.complex128)
        _check(self._L.bs_perm(self._p, a.ctypes.data, R, K, K, _ip(M), _ip(N), int(mode), out.ctypes.data,
                               lo.ctypes.data), self._p)
        return (complex(out[0]), complex(lo[0])) if with_tail else complex(out[0])

    def perm_formula(self, a, formula: str = "bbfg", with_tail: bool = False):
        """Permanent of a square matrix by Eq. bbfg ("bbfg"), Eq. ryser
        ("ryser") or its Nijenhuis-Wilf form ("nw"), in FP64 (Sec. 3.2's
        accuracy comparison)."""
        a = _c128(a)
        n = a.shape[0]
        if a.shape != (n, n):
            raise ValueError("perm_formula needs a square matrix")
        out = np.zeros(1, dtype=np.complex128)
        lo = np.zeros(1, dtype=np.complex128)
        _check(self._L.bs_perm_formula(self._p, a.ctypes.data, n, n, FORMULAS[formula], out.ctypes.data,
                                       lo.ctypes.data), self._p)
        return (complex(out[0]), complex(lo[0])) if with_tail else complex(out[0])

    def laplace_minors(self, a, row_mult=None, col_mult=None, mode: int = BS_FP64):
        a = _c128(a)
        R, K = a.shape
        M = _i32(np.ones(R) if row_mult is None else row_mult, R)
        N = _i32(np.ones(K) if col_mult is None else col_mult, K)
        out = np.zeros(K, dtype=np.complex128)
        _check(self._L.bs_laplace_minors(self._p, a.ctypes.data, R, K, K, _ip(M), _ip(N), int(mode),
                                         out.ctypes.data), self._p)
        return out

    @staticmethod
    def pack_batch(items):
        """Pack [(A, row_mult, col_mult), ...] into the batch layout."""
        offs, rows, cols, mults, roff, coff = [], [], [], [], [], []
        mats = []
        at = 0
        m_at = 0
        for a, M, N in items:
            a = _c128(a)
            R, K = a.shape
            offs.append(at)
            rows.append(R)
            cols.append(K)
            mats.append(a.reshape(-1))
            at += R * K
            roff.append(m_at)
            mults.extend(list(np.asarray(M, dtype=np.int32).reshape(R)))
            m_at += R
            coff.append(m_at)
            mults.extend(list(np.asarray(N, dtype=np.int32).reshape(K)))
            m_at += K
        packed = np.ascontiguousarray(np.concatenate(mats) if mats else np.zeros(1, np.complex128))
        return (packed, np.asarray(offs, np.int64), np.asarray(rows, np.int32), np.asarray(cols, np.int32),
                np.asarray(mults if mults else [0], np.int32), np.asarray(roff, np.int64),
                np.asarray(coff, np.int64))

    def perm_batch(self, items, mode: int = BS_FP64):
        packed, offs, rows, cols, mults, roff, coff = self.pack_batch(items)
        out = np.zeros(len(items), dtype=np.complex128)
        _check(self._L.bs_perm_batch(self._p, len(items), packed.ctypes.data, _i64p(offs), _ip(rows), _ip(cols),
                                     _ip(mults), _i64p(roff), _i64p(coff), int(mode), out.ctypes.data), self._p)
        return out

    def perm_batch_dev(self, packed_dev, offs, rows, cols, mults, roff, coff, mode, out_dev):
        """Device form: ``packed_dev`` / ``out_dev`` are CUDA complex128 tensors,
        the rest host arrays from ``pack_batch``.  Asynchronous: call sync()."""
        offs = np.ascontiguousarray(offs, np.int64)
        rows = _i32(rows)
        cols = _i32(cols)
        mults = _i32(mults)
        roff = np.ascontiguousarray(roff, np.int64)
        coff = np.ascontiguousarray(coff, np.int64)
        _check(self._L.bs_perm_batch_dev(self._p, len(rows), C.c_void_p(packed_dev.data_ptr()), _i64p(offs),
                                         _ip(rows), _ip(cols), _ip(mults), _i64p(roff), _i64p(coff), int(mode),
                                         C.c_void_p(out_dev.data_ptr())), self._p)

    # ---------------------------------------------------------- sampling
    def sample(self, u, occupation, n_samples: int, seed: int, mode: int = BS_FP64):
        u = _c128(u)
        m = u.shape[0]
        assert u.shape == (m, m), "bs_sample takes a square interferometer; use sample_ex"
        occ = _i32(occupation, m)
        out = np.zeros((max(n_samples, 0), m), dtype=np.int32)
        _check(self._L.bs_sample(self._p, u.ctypes.data, m, _ip(occ), int(n_samples),
                                 C.c_uint64(int(seed) & ((1 << 64) - 1)), int(mode), _ip(out)), self._p)
        return out

    def sample_ex(self, u, occupation, n_samples: int, seed: int, m_detected: int = 0, mode: int = BS_FP64):
        u = _c128(u)
        mr, mc = u.shape
        occ = _i32(occupation, mc)
        mdet = mr if m_detected <= 0 or m_detected > mr else int(m_detected)
        out = np.zeros((max(n_samples, 0), mdet), dtype=np.int32)
        _check(self._L.bs_sample_ex(self._p, u.ctypes.data, mr, mc, mc, _ip(occ), int(n_samples),
                                    C.c_uint64(int(seed) & ((1 << 64) - 1)), int(mdet), int(mode), _ip(out)),
               self._p)
        return out

    def sample_trace(self, u, occupation, n_samples: int, seed: int, m_detected: int = 0, mode: int = BS_FP64):
        """bs_sample_trace: (counts[n_samples, m_detected], rows[n_samples, n]),
        rows holding the drawn row of every step in draw order."""
        u = _c128(u)
        mr, mc = u.shape
        occ = _i32(occupation, mc)
        n = int(occ.sum())
        mdet = mr if m_detected <= 0 or m_detected > mr else int(m_detected)
        out = np.zeros((max(n_samples, 0), mdet), dtype=np.int32)
        rows = np.zeros((max(n_samples, 0), n), dtype=np.int32)
        _check(self._L.bs_sample_trace(self._p, u.ctypes.data, mr, mc, mc, _ip(occ), int(n_samples),
                                       C.c_uint64(int(seed) & ((1 << 64) - 1)), int(mdet), int(mode), _ip(out),
                                       _ip(rows)), self._p)
        return out, rows

    def sample_dev(self, u_dev, occupation, n_samples: int, seed: int, out_dev, m_detected: int = 0,
                   mode: int = BS_FP64):
        """Device form: ``u_dev`` is a CUDA complex128 (m_rows x m_cols) tensor,
        ``out_dev`` a CUDA int32 (n_samples x m_detected) tensor.  Async."""
        mr, mc = int(u_dev.shape[0]), int(u_dev.shape[1])
        occ = _i32(occupation, mc)
        ld = int(u_dev.stride(0))
        _check(self._L.bs_sample_dev(self._p, C.c_void_p(u_dev.data_ptr()), mr, mc, ld, _ip(occ), int(n_samples),
                                     C.c_uint64(int(seed) & ((1 << 64) - 1)), int(m_detected), int(mode),
                                     C.c_void_p(out_dev.data_ptr())), self._p)


# ------------------------------------------------------------------ serving
class Server:
    """Continuous-batching server (bs_server_*): requests from many client
    threads are admitted by slots and device memory and walked together,
    tick by tick, on one stream."""

    def __init__(self, device=0, mem_budget_bytes=1 << 30, max_active=64, tick_tasks=8192, mode=BS_MIXED):
        L = load()
        p = C.c_void_p()
        _check(L.bs_server_create(C.byref(p), int(device), int(mem_budget_bytes), int(max_active),
                                  int(tick_tasks), int(mode)))
        self._p = p
        self._L = L

    def close(self):
        if getattr(self, "_p", None):
            self._L.bs_server_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, kind, a, row_mult, col_mult):
        """kind 0: permanent, 1: Laplace minors.  Returns a ticket."""
        a = _c128(a)
        R, K = a.shape
        M = _i32(row_mult, R)
        N = _i32(col_mult, K)
        t = self._L.bs_server_submit(self._p, int(kind), a.ctypes.data, R, K, K, _ip(M), _ip(N))
        if t < 0:
            _check(int(t))
        return int(t), (1 if kind == 0 else K)

    def wait(self, ticket):
        """Blocks; returns (result array, latency seconds)."""
        t, n = ticket
        out = np.zeros(max(n, 1), dtype=np.complex128)
        lat = C.c_double()
        _check(self._L.bs_server_wait(self._p, t, out.ctypes.data, len(out), C.byref(lat)))
        return out[:n], lat.value

    def poll(self, ticket):
        """(done, result or None, latency or None)."""
        t, n = ticket
        out = np.zeros(max(n, 1), dtype=np.complex128)
        lat = C.c_double()
        rc = self._L.bs_server_poll(self._p, t, out.ctypes.data, len(out), C.byref(lat))
        if rc < 0:
            _check(rc)
        return (True, out[:n], lat.value) if rc == 1 else (False, None, None)

    def submit_sample(self, u, occupation, seed: int, sample: int = 0, m_detected: int = 0):
        """One Clifford & Clifford sample, run by the engine: the counts of
        sample ``sample`` of bs_sample_ex(u, occupation, seed) in the server's
        mode.  Returns a ticket for wait_sample / poll_sample / cancel."""
        u = _c128(u)
        mr, mc = u.shape
        occ = _i32(occupation, mc)
        mdet = mr if m_detected <= 0 or m_detected > mr else int(m_detected)
        t = self._L.bs_server_submit_sample(self._p, u.ctypes.data, mr, mc, mc, _ip(occ),
                                            C.c_uint64(int(seed) & ((1 << 64) - 1)),
                                            C.c_uint64(int(sample) & ((1 << 64) - 1)), int(mdet))
        if t < 0:
            _check(int(t))
        return int(t), -mdet  # negative width marks a sampling ticket

    def wait_sample(self, ticket):
        """Blocks; returns (counts[m_detected], latency seconds)."""
        t, w = ticket
        out = np.zeros(max(-w, 1), dtype=np.int32)
        lat = C.c_double()
        _check(self._L.bs_server_wait_sample(self._p, t, _ip(out), len(out), C.byref(lat)))
        return out[:-w], lat.value

    def poll_sample(self, ticket):
        """(done, counts or None, latency or None)."""
        t, w = ticket
        out = np.zeros(max(-w, 1), dtype=np.int32)
        lat = C.c_double()
        rc = self._L.bs_server_poll_sample(self._p, t, _ip(out), len(out), C.byref(lat))
        if rc < 0:
            _check(rc)
        return (True, out[:-w], lat.value) if rc == 1 else (False, None, None)

    def cancel(self, ticket):
        """Cancels a pending request; its waiter gets BsError(BS_ECANCELED)."""
        _check(self._L.bs_server_cancel(self._p, ticket[0]))

    def stats(self):
        s = _ServerStats()
        _check(self._L.bs_server_get_stats(self._p, C.byref(s)))
        return {f: getattr(s, f) for f, _ in _ServerStats._fields_}


# ------------------------------------------------------------------ allocation-free call
def perm_noalloc(a, row_mult=None, col_mult=None, mode: int = BS_FP64, stream=0, with_tail: bool = False):
    """bs_perm_noalloc: the permanent without any device allocation, for
    callers whose memory manager forbids allocations outside its own budget or
    that must not enter the CUDA allocator.  ``stream``: a torch.cuda.Stream,
    a raw handle, or 0; synchronised before the call returns.  Returns the
    value, or (value, tail) with with_tail=True."""
    L = load()
    a = _c128(a)
    R, K = a.shape
    M = _i32(np.ones(R) if row_mult is None else row_mult, R)
    N = _i32(np.ones(K) if col_mult is None else col_mult, K)
    out = np.zeros(1, dtype=np.complex128)
    lo = np.zeros(1, dtype=np.complex128)
    handle = int(getattr(stream, "cuda_stream", stream) or 0)
    _check(L.bs_perm_noalloc(a.ctypes.data, R, K, K, _ip(M), _ip(N), int(mode), C.c_void_p(handle),
                             out.ctypes.data, lo.ctypes.data))
    return (complex(out[0]), complex(lo[0])) if with_tail else complex(out[0])


# ------------------------------------------------------------------ host-only helpers
def debug_gray_walk(radix, nbin, start, steps):
    """Walk the n-ary reflected Gray counter of the kernels on the host.
    Returns (deltas[steps, ndigits], moved[steps], weights[steps])."""
    L = load()
    r = _i32(radix)
    nd = len(r)
    deltas = np.zeros((steps, max(nd, 1)), dtype=np.int32)
    moved = np.zeros(max(steps, 1), dtype=np.int32)
    w = np.zeros(max(steps, 1), dtype=np.uint64)
    _check(L.bs_debug_gray_walk(nd, int(nbin), _ip(r), C.c_uint64(int(start)), int(steps), _ip(deltas),
                                _ip(moved), w.ctypes.data_as(C.POINTER(C.c_uint64))))
    return deltas[:, :nd], moved[:steps], w[:steps]


def debug_mixed_error(row_mult, col_mult, kind=0, chunk_log2=0):
    """MIXED precision rule: (predicted log2 of the FP32 error relative to
    prod ||a_j||, FP32 chunk log2, decision at the default tolerance 1e-6:
    1 FP32, 2 FP32 re-seeded every 2^8 steps, 0 the fallback kernels).
    chunk_log2 <= 0: the chunk length of the problem planned alone."""
    L = load()
    M = _i32(row_mult)
    N = _i32(col_mult)
    e = C.c_double(0.0)
    l = C.c_int(0)
    plan = C.c_int(0)
    _check(L.bs_debug_mixed_error(len(M), len(N), _ip(M), _ip(N), int(kind), int(chunk_log2), C.byref(e),
                                  C.byref(l), C.byref(plan)))
    return float(e.value), int(l.value), int(plan.value)


def debug_plan(row_mult, col_mult, kind=0):
    """Planner summary: dict(C, nrows, nbin, K, transposed, pinned, log2L,
    tasks), the last two for the job run alone in FP64 mode."""
    L = load()
    M = _i32(row_mult)
    N = _i32(col_mult)
    info = np.zeros(8, dtype=np.int64)
    _check(L.bs_debug_plan(len(M), len(N), _ip(M), _ip(N), int(kind), _i64p(info)))
    return dict(C=int(info[0]), nrows=int(info[1]), nbin=int(info[2]), K=int(info[3]),
                transposed=bool(info[4]), pinned=int(info[5]), log2L=int(info[6]), tasks=int(info[7]))
