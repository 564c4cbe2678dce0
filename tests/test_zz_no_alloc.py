"""msp_solve_small_noalloc against msp_solve_all and the CPU oracle.

The allocation-free entry point serves callers that cannot allocate device
memory while solving (their device memory is owned by another allocator, or
a serving loop must not risk an allocation failure mid-request); it keeps
its intermediates in one static device array instead.  Its solution set must
equal the one msp_solve_all returns, and the oracle's, on two calls in a row
(the array keeps the previous call's contents, so the second call checks that
nothing stale leaks into it), and after calls on larger and smaller
instances.  The file sorts last so a run that stops at the first failure has
run every other test before it.
"""
import ctypes

import numpy as np
import pytest

import msp_instances as mi
import oracle

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


def oracle_set(A, d):
    A = np.asarray(A)
    return oracle.brute(A, d) if A.shape[1] <= 22 else oracle.mitm(A, d)


CASES = [
    ("4_30_planted", lambda: mi.generate(4, 30, 1, planted=True, h=15)[:2]),
    ("5_40_planted", lambda: mi.generate(5, 40, 11, planted=True, h=20)[:2]),
    ("3_24_small_K", lambda: mi.generate(3, 24, 12, K=3, planted=True, h=12)[:2]),
    ("2_17_plain", lambda: mi.generate(2, 17, 13, K=5)[:2]),
    # degenerate quarters: n < 4 or not a multiple of 4 (quarters of 0 or 1
    # columns, lists of one subset)
    ("1_1", lambda: mi.generate(2, 1, 14, K=3, planted=True, h=1)[:2]),
    ("2_2", lambda: mi.generate(2, 2, 15, K=3, planted=True, h=1)[:2]),
    ("3_3", lambda: mi.generate(3, 3, 16, K=2, planted=True, h=1)[:2]),
    ("2_5", lambda: mi.generate(2, 5, 17, K=3, planted=True, h=2)[:2]),
    # 16 rows and row sums up to 65512, just under the 16-bit field limit
    ("16_40_wide", lambda: mi.generate(16, 40, 205, K=2600, planted=True, h=20)[:2]),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_solve_all_twice(msp, name, make):
    A, d = make()
    lib = msp.load_library()
    want = oracle_set(A, d)
    assert msp.solve_all(A, d) == want
    first = call_noalloc(lib, A, d)
    second = call_noalloc(lib, A, d)
    assert first == want
    assert second == want


def test_noalloc_back_to_back_different_instances(msp):
    # small then large, then large then smaller: leftover bucket offsets,
    # counters and records of a larger layout sit under a smaller one
    lib = msp.load_library()
    order = [mi.generate(3, 24, 21, K=3, planted=True, h=12)[:2],
             mi.generate(4, 30, 22, planted=True, h=15)[:2],
             mi.generate(5, 40, 23, planted=True, h=20)[:2],
             mi.generate(2, 17, 24, K=5, planted=True, h=8)[:2],
             mi.generate(3, 24, 25, K=4, planted=True, h=12)[:2]]
    for A, d in order:
        want = oracle_set(A, d)
        assert msp.solve_all(A, d) == want
        assert call_noalloc(lib, A, d) == want


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
