"""bs_perm_noalloc: the permanent for callers that may not allocate device
memory -- hosts whose memory manager owns a fixed device budget and forbids
allocations outside it, and real-time loops that must not enter the CUDA
allocator.  Its scratch is one fixed __device__ array shared by every call,
so this test calls it twice in a row, with the larger problem first, and
compares each result (value and double-double tail) with the allocating
entry point bs_perm under the parity tolerance of the GPU tests, on the
legacy default stream and on a caller's stream.  It also pins the stated
size limit: 2^34 addends fit the scratch, 2^35 are rejected.  It lives in a
file of its own that pytest collects last and must pass both alone in a
fresh process and after the other tests."""
import ctypes

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-6, 2: 1e-10}  # FP64, MIXED, double-float


def scale(a, M, N):
    norms = np.sqrt((np.abs(a) ** 2 * np.asarray(M)[:, None]).sum(axis=0))
    return float(np.prod(norms ** np.asarray(N)))


def noalloc_c_abi(lib, a, M, N, mode, stream=None):
    """Call bs_perm_noalloc directly through the C ABI (ctypes); returns
    (value, tail)."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    R, K = a.shape
    M = np.ascontiguousarray(M, dtype=np.int32)
    N = np.ascontiguousarray(N, dtype=np.int32)
    out = np.zeros(1, dtype=np.complex128)
    lo = np.zeros(1, dtype=np.complex128)
    fn = lib.bs_perm_noalloc
    ip = ctypes.POINTER(ctypes.c_int)
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    rc = fn(a.ctypes.data, R, K, K, M.ctypes.data_as(ip), N.ctypes.data_as(ip), int(mode), stream,
            out.ctypes.data, lo.ctypes.data)
    assert rc == 0, rc
    return complex(out[0]), complex(lo[0])


def problems():
    u = S.haar_unitary(40, 11)
    big = (u[:22, :22], np.ones(22, np.int32), np.ones(22, np.int32))      # 2^21 addends, many tasks
    a1, M1, N1, _, _ = S.config_single(seed=1)                              # 576 addends, 9 tasks
    return [big, (a1, M1, N1)]


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_noalloc_matches_bs_perm_on_two_calls(ctx, bslib, mode):
    lib = ctypes.CDLL(bslib.library_path())
    for a, M, N in problems():
        ref, ref_lo = ctx.perm(a, M, N, mode=mode, with_tail=True)
        got, lo = noalloc_c_abi(lib, a, M, N, mode)
        assert abs(got - ref) <= TOL[mode] * scale(a, M, N), (got, ref)
        if mode == 0:
            # same kernels, same chunking: the same double-double sum
            assert abs((got + lo) - (ref + ref_lo)) <= 1e-13 * scale(a, M, N), (got, lo, ref, ref_lo)


def test_noalloc_on_a_caller_stream(ctx, bslib):
    torch = pytest.importorskip("torch")
    lib = ctypes.CDLL(bslib.library_path())
    stream = torch.cuda.Stream()
    for a, M, N in problems():
        ref = ctx.perm(a, M, N, mode=0)
        got, _ = noalloc_c_abi(lib, a, M, N, 0, stream=stream.cuda_stream)
        assert abs(got - ref) <= TOL[0] * scale(a, M, N), (got, ref)


def test_noalloc_size_limit(ctx, bslib):
    """2^34 addends (35 distinct rows) fit the fixed scratch and give
    bs_perm's result; 2^35 (36 rows) are rejected before any work."""
    lib = ctypes.CDLL(bslib.library_path())
    u = S.haar_unitary(48, 12)
    a = u[:35, :35]
    ones = np.ones(35, np.int32)
    assert bslib.debug_plan(ones, ones)["C"] == 1 << 34
    ref = ctx.perm(a, ones, ones, mode=1)
    got, _ = noalloc_c_abi(lib, a, ones, ones, 1)
    assert abs(got - ref) <= TOL[1] * scale(a, ones, ones), (got, ref)
    b = u[:36, :36]
    ones = np.ones(36, np.int32)
    with pytest.raises(bslib.BsError) as e:
        bslib.perm_noalloc(b, ones, ones)
    assert e.value.code == bslib.BS_EINVAL and "scratch" in str(e.value)


def test_noalloc_rejects_jobs_beyond_its_scratch(bslib):
    u = S.haar_unitary(48, 12)
    a = u[:44, :44]
    with pytest.raises(bslib.BsError) as e:
        bslib.perm_noalloc(a, np.ones(44, np.int32), np.ones(44, np.int32))
    assert e.value.code == bslib.BS_EINVAL and "scratch" in str(e.value)
