"""Seeded synthetic market-split instances (input construction only).

This module builds the inputs that both the CUDA path and the CPU oracle are
run on. It holds none of the solving method's arithmetic: it draws matrices,
right-hand sides and planted solution vectors, and nothing else.

Instance family (Section 1, the Cornuejols-Dawande construction): for a given
m, n = 10 (m - 1); every coefficient a_ij is drawn uniformly from [0, K)
(K = 100 gives the paper's range [0, 99]); the right-hand side of row i is
d_i = floor(sum_j a_ij / 2).  The paper's own test set (QOBLIB, Section 4) is
not available here; these seeded instances of the same shapes and
distribution stand in for it.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), seeded with ``seed``:
  * a_ij = draw mod K, filled row-major;
  * a planted instance then draws x* with exactly h ones by a partial
    Fisher-Yates shuffle of 0..n-1 from the same stream (position i swaps with
    i + draw mod (n - i)) and sets d = A x*.
"""
from __future__ import annotations

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 generator (64-bit state, golden-ratio increment)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)


def standard_n(m: int) -> int:
    """n = 10 (m - 1) for the (m, n) family of Section 1."""
    return 10 * (m - 1)


def generate(m: int, n: int | None = None, seed: int = 0, *, K: int = 100,
             planted: bool = False, h: int | None = None):
    """Return (A, d, xstar) for one seeded instance.

    A is int32 [m, n] row-major, d int32 [m].  xstar is a uint8 [n] 0/1 vector
    for planted instances (d = A xstar) and None for plain ones
    (d_i = floor(row sum_i / 2)).  ``h`` is the number of ones in xstar
    (default n // 2).
    """
    if n is None:
        n = standard_n(m)
    if m < 1 or n < 1 or K < 1:
        raise ValueError("m, n and K must be positive")
    rng = SplitMix64(seed)
    A = np.empty((m, n), dtype=np.int64)
    for i in range(m):
        for j in range(n):
            A[i, j] = rng.next() % K
    xstar = None
    if planted:
        if h is None:
            h = n // 2
        if not 0 <= h <= n:
            raise ValueError("h must lie in [0, n]")
        perm = list(range(n))
        for i in range(h):
            j = i + rng.next() % (n - i)
            perm[i], perm[j] = perm[j], perm[i]
        xstar = np.zeros(n, dtype=np.uint8)
        xstar[perm[:h]] = 1
        d = A @ xstar.astype(np.int64)
    else:
        d = A.sum(axis=1) // 2
    return A.astype(np.int32), d.astype(np.int32), xstar


def batch(m: int, n: int, count: int, seed0: int, *, K: int = 100,
          h: int | None = None):
    """``count`` independent instances with seeds seed0 .. seed0 + count - 1.

    The first half is plain and the second half planted (h ones), which is
    the mixed batch used for the many-small-instances workload.
    """
    out = []
    for k in range(count):
        planted = k >= count // 2
        out.append(generate(m, n, seed0 + k, K=K, planted=planted, h=h))
    return out


def mask_of(x) -> tuple[int, ...]:
    """Pack a 0/1 vector into little-endian 64-bit words (bit j = x_j)."""
    x = np.asarray(x).astype(np.uint8).ravel()
    words = (len(x) + 63) // 64
    out = [0] * words
    for j, v in enumerate(x):
        if v:
            out[j // 64] |= 1 << (j % 64)
    return tuple(out)


def restrict(A, d, fixed_cols, fixed_vals):
    """Sub-instance with the columns in ``fixed_cols`` fixed to ``fixed_vals``.

    Returns (A', d', free_cols): A' keeps the free columns in their original
    order and d' = d - sum of the fixed-to-one columns.  Every solution of the
    original instance that agrees with the fixed values restricts to a
    solution of (A', d'), and conversely.  d' may have negative entries, in
    which case the sub-instance has no solution.
    """
    A = np.asarray(A, dtype=np.int64)
    d = np.asarray(d, dtype=np.int64)
    fixed_cols = list(fixed_cols)
    fixed_set = set(fixed_cols)
    if len(fixed_set) != len(fixed_cols):
        raise ValueError("fixed columns must be distinct")
    free = [j for j in range(A.shape[1]) if j not in fixed_set]
    d2 = d.copy()
    for j, v in zip(fixed_cols, fixed_vals):
        if v:
            d2 = d2 - A[:, j]
    return A[:, free].astype(np.int32), d2, free
