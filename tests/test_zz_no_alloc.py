"""msp_solve_small_noalloc against msp_solve_all.

The allocation-free entry point serves callers that cannot allocate device
memory while solving (their device memory is owned by another allocator, or
a serving loop must not risk an allocation failure mid-request); it keeps
its intermediates in one static device array instead.  Its solution set must
equal the one msp_solve_all returns, on two calls in a row (the array keeps
the previous call's contents, so the second call checks that nothing stale
leaks into it).  The file sorts last so a run that stops at the first failure
has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

import msp_instances as mi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def msp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_05045_gb300 import build
    build.build()
    import paper_2507_05045_gb300 as m
    return m


def call_noalloc(lib, A, d, cap=1 << 16):
    A = np.ascontiguousarray(A, dtype=np.int32)
    d = np.ascontiguousarray(d, dtype=np.int32)
    m, n = A.shape
    out = np.zeros(cap, dtype=np.uint64)
    cnt = ctypes.c_size_t()
    rc = lib.msp_solve_small_noalloc(A.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     d.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), m, n,
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), cap,
                                     ctypes.byref(cnt), None)
    assert rc == 0, lib.msp_last_error().decode()
    return [(int(v),) for v in out[:cnt.value]]


CASES = [
    ("4_30_planted", lambda: mi.generate(4, 30, 1, planted=True, h=15)[:2]),
    ("5_40_planted", lambda: mi.generate(5, 40, 11, planted=True, h=20)[:2]),
    ("3_24_small_K", lambda: mi.generate(3, 24, 12, K=3, planted=True, h=12)[:2]),
    ("2_17_plain", lambda: mi.generate(2, 17, 13, K=5)[:2]),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_solve_all_twice(msp, name, make):
    A, d = make()
    lib = msp.load_library()
    want = msp.solve_all(A, d)
    first = call_noalloc(lib, A, d)
    second = call_noalloc(lib, A, d)
    assert first == want
    assert second == want


def test_noalloc_back_to_back_different_instances(msp):
    lib = msp.load_library()
    A1, d1, _ = mi.generate(3, 24, 21, K=3, planted=True, h=12)
    A2, d2, _ = mi.generate(4, 30, 22, planted=True, h=15)
    w1, w2 = msp.solve_all(A1, d1), msp.solve_all(A2, d2)
    assert call_noalloc(lib, A1, d1) == w1
    assert call_noalloc(lib, A2, d2) == w2


def test_noalloc_rejects_sizes_beyond_its_scratch(msp):
    lib = msp.load_library()
    A, d, _ = mi.generate(5, 41, 3)
    out = np.zeros(4, dtype=np.uint64)
    cnt = ctypes.c_size_t()
    rc = lib.msp_solve_small_noalloc(A.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     d.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 5, 41,
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), 4,
                                     ctypes.byref(cnt), None)
    assert rc == -2  # MSP_ERANGE
    assert b"40" in lib.msp_last_error()
