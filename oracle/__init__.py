"""CPU oracle for the market split solution set.

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product path.  It
shares no code with the CUDA path: the C source in this folder is compiled
by :func:`build` into ``oracle/_build/liboracle.so`` and loaded through
ctypes.

Result convention: every solution x of A x = d (Section 1, eq. 1) as a tuple
of little-endian 64-bit words (bit j of word j // 64 is x_j); lists are
sorted ascending as unsigned integers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) if it is missing or stale."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = force or not os.path.exists(_LIB) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.msp_oracle_brute.restype = ctypes.c_int64
            lib.msp_oracle_brute.argtypes = [i32p, i32p, ctypes.c_int, ctypes.c_int, u64p, ctypes.c_int64]
            lib.msp_oracle_mitm.restype = ctypes.c_int64
            lib.msp_oracle_mitm.argtypes = [i32p, i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p,
                                            ctypes.c_int64]
            lib.msp_oracle_fourlist.restype = ctypes.c_int64
            lib.msp_oracle_fourlist.argtypes = [i32p, i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p,
                                                ctypes.c_int64, ctypes.c_int64, u64p, ctypes.c_int64, u64p,
                                                ctypes.POINTER(ctypes.c_double)]
            lib.msp_oracle_subset_count.restype = ctypes.c_int
            lib.msp_oracle_subset_count.argtypes = [i32p, ctypes.c_int, ctypes.c_int64, u64p]
            lib.msp_oracle_residue_hist.restype = ctypes.c_int
            lib.msp_oracle_residue_hist.argtypes = [i32p, ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int,
                                                    ctypes.c_int, i32p, u64p]
            _lib = lib
    return _lib


def _i32(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _masks(buf, count, words):
    arr = buf[: count * words].reshape(count, words)
    return [tuple(int(w) for w in row) for row in arr]


def _run(fn, A, d, m, n, *extra, _after=()):
    words = (n + 63) // 64
    a, ap = _i32(np.asarray(A).reshape(m, n))
    dd, dp = _i32(np.asarray(d).reshape(m))
    cap = 1024
    while True:
        out = np.zeros(cap * words, dtype=np.uint64)
        cnt = fn(ap, dp, m, n, *extra, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), cap, *_after)
        if cnt < 0:
            raise RuntimeError(f"oracle failed with status {cnt}")
        if cnt <= cap:
            return _masks(out, int(cnt), words)
        cap = int(cnt)


def brute(A, d):
    """Sol(A, d) by testing every x in {0,1}^n (n <= 40; practical n <= 26)."""
    A = np.asarray(A)
    m, n = A.shape
    return _run(_load().msp_oracle_brute, A, d, m, n)


def mitm(A, d, slices: int | None = None):
    """Sol(A, d) by the two-list meet in the middle on full vectors (n <= 80).

    ``slices`` splits the left half by the residue of its exact row-1 value
    so that one slice fits in memory; slices run in parallel (OpenMP).
    """
    A = np.asarray(A)
    m, n = A.shape
    if slices is None:
        half = n // 2
        slices = max(1, min(4096, (1 << max(0, half - 22))))
        slices = max(slices, os.cpu_count() or 1) if half >= 20 else slices
    return _run(_load().msp_oracle_mitm, A, d, m, n, int(slices))


def default_slicing(m: int, n: int) -> tuple[int, ...]:
    """Moduli of rows 1..4 for :func:`fourlist` giving slices of about 2^15
    left subsets, so that one slice's hash table stays in a core's cache.
    No modulus passes 2^7, well below the spread of a half's row sums in the
    (m, 10 (m - 1)) family, so the slices are close to equal; with fewer rows
    than needed the slices are simply larger."""
    bits = max(0, n // 2 - 15)
    t = max(1, min(m, 4))
    per = [min(7, bits // t + (1 if k < bits % t else 0)) for k in range(t)]
    return tuple(1 << b for b in per)


def fourlist(A, d, mods=None, slice_range=None, return_records: bool = False, timing: dict | None = None):
    """Sol(A, d) by the four-list meet in the middle over residue slices.

    ``mods`` are the moduli P_1..P_t (t <= 4) of rows 1..t whose residue
    tuple numbers the slices, s = r_1 + P_1 (r_2 + ...); ``slice_range``
    = (s_begin, s_end) enumerates only those slices (default: all), which
    gives exactly the solutions whose slice (:func:`slice_of`) lies in it.
    With ``return_records`` the result is (solutions, left subsets, right
    subsets enumerated).  A ``timing`` dict receives the seconds of the list
    build ("build") and of the slice joins ("join").
    """
    A = np.asarray(A)
    m, n = A.shape
    if mods is None:
        mods = default_slicing(m, n)
    md, mp = _i32(mods)
    S = int(np.prod(md)) if len(md) else 1
    s0, s1 = (0, S) if slice_range is None else (int(slice_range[0]), int(slice_range[1]))
    rec = np.zeros(2, dtype=np.uint64)
    recp = rec.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    sec = np.zeros(2, dtype=np.float64)
    secp = sec.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    sols = _run(_load().msp_oracle_fourlist, A, d, m, n, len(md), mp, s0, s1, _after=(recp, secp))
    if timing is not None:
        timing["build"], timing["join"] = float(sec[0]), float(sec[1])
    if return_records:
        return sols, int(rec[0]), int(rec[1])
    return sols


def slice_of(A, mask, mods) -> int:
    """The slice of a solution mask in :func:`fourlist`: the residue tuple of
    the row sums of its left half (columns 0 .. n/2 - 1) of rows 1..t."""
    A = np.asarray(A, dtype=np.int64)
    n = A.shape[1]
    v = sum(int(w) << (64 * k) for k, w in enumerate(mask))
    cols = [j for j in range(n // 2) if (v >> j) & 1]
    s, stride = 0, 1
    for k, P in enumerate(mods):
        s += (int(A[k, cols].sum()) % int(P)) * stride
        stride *= int(P)
    return s


def solve(A, d):
    """Sol(A, d): brute force for n <= 20, meet in the middle beyond."""
    n = np.asarray(A).shape[1]
    return brute(A, d) if n <= 20 else mitm(A, d)


def subset_count(weights, target) -> int:
    """Number of subsets of ``weights`` summing to ``target`` (exact, 128-bit)."""
    w, wp = _i32(weights)
    out = (ctypes.c_uint64 * 2)()
    rc = _load().msp_oracle_subset_count(wp, len(w), int(target), out)
    if rc < 0:
        raise RuntimeError(f"subset_count failed with status {rc}")
    return int(out[0]) | (int(out[1]) << 64)


def row1_candidates(A, d) -> int:
    """Row-1 candidate pairs of Algorithm 2: subsets x with a_1 . x = d_1.

    Every such x is one pair (left part, right part) whose row-1 sums add up
    to d_1, for any split of the columns into two halves, so the count does
    not depend on the split.
    """
    A = np.asarray(A)
    return subset_count(A[0], int(np.asarray(d)[0]))


def residue_hist(A, cols, mods):
    """Subsets of ``cols`` counted by (row_i sum mod mods[i]) for i < len(mods).

    Returned as a flat uint64 array indexed r_0 + mods[0] * (r_1 + ...).
    """
    A = np.asarray(A)
    m, n = A.shape
    a, ap = _i32(A)
    c, cp = _i32(cols)
    md, mp = _i32(mods)
    states = int(np.prod(md))
    out = np.zeros(states, dtype=np.uint64)
    rc = _load().msp_oracle_residue_hist(ap, m, n, cp, len(c), len(md), mp,
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    if rc < 0:
        raise RuntimeError(f"residue_hist failed with status {rc}")
    return out
