"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test checks the oracle against something fixed independently of its
code: hand-derived solution sets, brute-force enumeration written in the
test (numpy, binary order), planted solutions, and invariants of
Sol(A, d) = {x in {0,1}^n : A x = d} (Section 1, eq. 1).
"""
import itertools
import json
import os

import numpy as np
import pytest

import msp_instances as mi
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def as_int(masks):
    return sorted(sum(w << (64 * k) for k, w in enumerate(t)) for t in masks)


def np_enumerate(A, d):
    """Every x in {0,1}^n, as a numpy bit matrix, filtered by A x == d."""
    A = np.asarray(A, dtype=np.int64)
    m, n = A.shape
    xs = ((np.arange(1 << n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int64)
    ok = np.all(xs @ A.T == np.asarray(d, dtype=np.int64)[None, :], axis=1)
    return sorted(int(v) for v in np.nonzero(ok)[0])


def test_hand_instances():
    g = json.load(open(os.path.join(GOLDEN, "hand_instances.json")))
    for inst in g["instances"]:
        A = np.array(inst["A"], dtype=np.int32)
        d = np.array(inst["d"], dtype=np.int32)
        assert as_int(oracle.brute(A, d)) == inst["solutions"], inst["name"]
        assert as_int(oracle.mitm(A, d)) == inst["solutions"], inst["name"]


def test_all_zero_matrix_gives_every_vector():
    A = np.zeros((3, 7), dtype=np.int32)
    d = np.zeros(3, dtype=np.int32)
    assert as_int(oracle.brute(A, d)) == list(range(128))
    assert as_int(oracle.mitm(A, d)) == list(range(128))
    assert oracle.mitm(A, np.array([0, 1, 0])) == []


@pytest.mark.parametrize("seed", range(60))
def test_brute_and_mitm_match_numpy_enumeration(seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 11))
    n = int(rng.integers(1, 15))
    K = int(rng.choice([2, 3, 5, 50, 100]))
    planted = bool(seed % 2)
    A, d, _ = mi.generate(m, n, 1000 + seed, K=K, planted=planted, h=n // 2)
    want = np_enumerate(A, d)
    assert as_int(oracle.brute(A, d)) == want
    for slices in (1, 3, 7):
        assert as_int(oracle.mitm(A, d, slices=slices)) == want


@pytest.mark.parametrize("seed", range(40))
def test_mitm_equals_brute_n_up_to_22(seed):
    rng = np.random.default_rng(10_000 + seed)
    m = int(rng.integers(1, 11))
    n = int(rng.integers(15, 23))
    K = int(rng.choice([2, 5, 50, 100]))
    A, d, _ = mi.generate(m, n, 2000 + seed, K=K, planted=bool(seed % 3), h=n // 2)
    b = oracle.brute(A, d)
    assert oracle.mitm(A, d, slices=1 + seed % 5) == b


@pytest.mark.parametrize("m", [3, 4, 5])
def test_planted_solution_found_standard_family(m):
    n = mi.standard_n(m)
    for seed in range(3):
        A, d, x = mi.generate(m, n, seed, planted=True, h=n // 2)
        sols = oracle.mitm(A, d)
        assert mi.mask_of(x) in sols


def _mask_to_x(mask, n):
    v = sum(w << (64 * k) for k, w in enumerate(mask))
    return np.array([(v >> j) & 1 for j in range(n)], dtype=np.int64)


@pytest.mark.parametrize("seed", range(12))
def test_every_reported_x_satisfies_ax_eq_d(seed):
    A, d, _ = mi.generate(4, 24, 300 + seed, K=[3, 10, 100][seed % 3], planted=True, h=12)
    for mask in oracle.mitm(A, d):
        x = _mask_to_x(mask, 24)
        assert np.array_equal(A.astype(np.int64) @ x, d.astype(np.int64))


@pytest.mark.parametrize("seed", range(12))
def test_complement_invariant(seed):
    # x solves A x = d  =>  1 - x solves A(1-x) = rowsum - d.  So the set is
    # closed under complement exactly when 2 d = rowsum (all rows).
    n = 18
    A, d, _ = mi.generate(3, n, 400 + seed, K=4, planted=True, h=9)
    rowsum = A.sum(axis=1)
    sols = set(as_int(oracle.mitm(A, d)))
    comp = set(as_int(oracle.mitm(A, rowsum - d)))
    full = (1 << n) - 1
    assert comp == {full ^ s for s in sols}
    d2 = rowsum // 2
    s2 = set(as_int(oracle.mitm(A, d2)))
    closed = s2 == {full ^ s for s in s2}
    if np.all(rowsum % 2 == 0):
        assert closed
    elif s2:
        assert not closed


@pytest.mark.parametrize("seed", range(10))
def test_column_permutation_maps_solution_set(seed):
    n = 20
    A, d, _ = mi.generate(3, n, 500 + seed, K=5, planted=True, h=10)
    perm = np.random.default_rng(seed).permutation(n)
    sols = as_int(oracle.mitm(A, d))
    sols_p = as_int(oracle.mitm(A[:, perm], d))
    # column k of the permuted matrix is column perm[k] of A
    mapped = sorted(sum(1 << k for k in range(n) if (s >> perm[k]) & 1) for s in sols)
    assert sols_p == mapped


@pytest.mark.parametrize("seed", range(10))
def test_row_permutation_and_duplicate_rows_leave_set_unchanged(seed):
    A, d, _ = mi.generate(4, 20, 600 + seed, K=6, planted=True, h=10)
    sols = oracle.mitm(A, d)
    perm = np.random.default_rng(seed).permutation(4)
    assert oracle.mitm(A[perm], d[perm]) == sols
    A2 = np.vstack([A, A[1:2]])
    d2 = np.concatenate([d, d[1:2]])
    assert oracle.mitm(A2, d2) == sols


@pytest.mark.parametrize("seed", range(8))
def test_surrogate_merge_of_rows_1_and_2_leaves_set_unchanged(seed):
    # eq. 2: rows 1 and 2 merged with weights 1 and nD, D > max a_ij.
    n = 18
    A, d, _ = mi.generate(3, n, 700 + seed, K=10, planted=True, h=9)
    D = int(A.max()) + 1
    w = n * D
    merged = A[0].astype(np.int64) + w * A[1].astype(np.int64)
    A2 = np.vstack([merged, A[2]]).astype(np.int32)
    d2 = np.array([int(d[0]) + w * int(d[1]), d[2]], dtype=np.int32)
    assert oracle.mitm(A2, d2) == oracle.mitm(A, d)


@pytest.mark.parametrize("seed", range(8))
def test_zero_column_doubles_solution_set(seed):
    n = 17
    A, d, _ = mi.generate(3, n, 800 + seed, K=5, planted=True, h=8)
    sols = as_int(oracle.mitm(A, d))
    A2 = np.hstack([A, np.zeros((3, 1), dtype=np.int32)])
    sols2 = as_int(oracle.mitm(A2, d))
    assert sols2 == sorted(sols + [s | (1 << n) for s in sols])


def test_subset_count_matches_enumeration():
    rng = np.random.default_rng(7)
    for _ in range(30):
        n = int(rng.integers(0, 13))
        w = rng.integers(0, 6, size=n).astype(np.int32)
        sums = [sum(int(w[j]) for j in range(n) if (x >> j) & 1) for x in range(1 << n)]
        for t in range(-1, int(w.sum()) + 2):
            assert oracle.subset_count(w, t) == sums.count(t)


def test_subset_count_closed_forms():
    # all-ones weights: C(n, t);  powers of two: exactly one subset per t.
    from math import comb
    for n in (10, 40, 100):
        for t in (0, 1, n // 3, n // 2, n):
            assert oracle.subset_count(np.ones(n, np.int32), t) == comb(n, t)
    assert oracle.subset_count(np.zeros(100, np.int32), 0) == 1 << 100
    w = np.array([1 << k for k in range(20)], dtype=np.int32)
    assert all(oracle.subset_count(w, t) == 1 for t in (0, 5, 12345, (1 << 20) - 1))


def test_row1_candidates_count_pairs_of_halves():
    A, d, _ = mi.generate(3, 16, 5)
    cnt = 0
    L = [sum(int(A[0, j]) for j in range(8) if (u >> j) & 1) for u in range(256)]
    R = [sum(int(A[0, 8 + j]) for j in range(8) if (w >> j) & 1) for w in range(256)]
    from collections import Counter
    cl, cr = Counter(L), Counter(R)
    cnt = sum(c * cr.get(int(d[0]) - v, 0) for v, c in cl.items())
    assert oracle.row1_candidates(A, d) == cnt


def test_residue_hist_matches_enumeration():
    A, _, _ = mi.generate(3, 12, 9)
    cols = [0, 2, 3, 5, 7, 8, 11]
    mods = [4, 3, 5]
    want = np.zeros(60, dtype=np.uint64)
    for bits in itertools.product([0, 1], repeat=len(cols)):
        s = [sum(int(A[i, c]) * b for c, b in zip(cols, bits)) for i in range(3)]
        idx = s[0] % 4 + 4 * (s[1] % 3 + 3 * (s[2] % 5))
        want[idx] += 1
    assert np.array_equal(oracle.residue_hist(A, cols, mods), want)


def test_generator_is_deterministic_and_in_range():
    A1, d1, _ = mi.generate(9, 80, 123)
    A2, d2, _ = mi.generate(9, 80, 123)
    assert np.array_equal(A1, A2) and np.array_equal(d1, d2)
    assert A1.min() >= 0 and A1.max() <= 99
    assert np.array_equal(d1, A1.sum(axis=1) // 2)
    A, d, x = mi.generate(6, 50, 3, planted=True, h=25)
    assert int(x.sum()) == 25 and np.array_equal(d, A @ x.astype(np.int64))
    # splitmix64 reference outputs for seed 0 (Steele, Lea, Flood 2014)
    g = mi.SplitMix64(0)
    assert [g.next() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


# ---- the four-list oracle (slices of residue tuples of the first rows) ----

def _random_mods(rng, m):
    t = int(rng.integers(0, min(4, m) + 1))
    return [int(x) for x in rng.integers(1, 8, size=t)]


@pytest.mark.parametrize("seed", range(80))
def test_fourlist_equals_numpy_enumeration(seed):
    # any moduli (powers of two or not, t = 0..4 rows), small K with long runs
    # of equal vectors, planted and plain right-hand sides
    rng = np.random.default_rng(30_000 + seed)
    m = int(rng.integers(1, 7))
    n = int(rng.integers(1, 15))
    K = int(rng.choice([2, 3, 5, 50, 100]))
    A, d, _ = mi.generate(m, n, 3000 + seed, K=K, planted=bool(seed % 2), h=n // 2)
    mods = _random_mods(rng, m)
    sols, rl, rr = oracle.fourlist(A, d, mods=mods, return_records=True)
    assert as_int(sols) == np_enumerate(A, d)
    # every left and right subset is enumerated exactly once over all slices
    assert (rl, rr) == (1 << (n // 2), 1 << (n - n // 2))


@pytest.mark.parametrize("seed", range(30))
def test_fourlist_equals_brute_n_up_to_24(seed):
    rng = np.random.default_rng(31_000 + seed)
    m = int(rng.integers(1, 11))
    n = int(rng.integers(15, 25))
    K = int(rng.choice([2, 5, 50, 100]))
    A, d, _ = mi.generate(m, n, 3100 + seed, K=K, planted=bool(seed % 3), h=n // 2)
    assert oracle.fourlist(A, d, mods=_random_mods(rng, m)) == oracle.brute(A, d)


@pytest.mark.parametrize("m,n,seed", [(4, 30, 1), (4, 30, 2), (5, 36, 3), (5, 40, 4), (3, 34, 5)])
def test_fourlist_equals_mitm(m, n, seed):
    # halves past the inner split (outer parts of several columns), default
    # slicing and a few others
    A, d, _ = mi.generate(m, n, 3200 + seed, planted=True, h=n // 2)
    want = oracle.mitm(A, d)
    assert oracle.fourlist(A, d) == want
    assert oracle.fourlist(A, d, mods=(3, 5)) == want
    assert oracle.fourlist(A, d, mods=(1,)) == want


@pytest.mark.parametrize("seed", range(12))
def test_fourlist_slice_ranges_partition_the_set(seed):
    # a range of slices gives exactly the solutions whose left-half residue
    # tuple lies in it; disjoint ranges covering all slices give the full set
    rng = np.random.default_rng(32_000 + seed)
    m = int(rng.integers(2, 6))
    n = int(rng.integers(12, 21))
    A, d, _ = mi.generate(m, n, 3300 + seed, K=int(rng.choice([3, 5, 20])), planted=True, h=n // 2)
    mods = [int(x) for x in rng.integers(2, 6, size=min(m, 3))]
    S = int(np.prod(mods))
    full = oracle.brute(A, d)
    cuts = sorted(set([0, S] + [int(x) for x in rng.integers(0, S, size=3)]))
    union, rec_l = [], 0
    for a, b in zip(cuts[:-1], cuts[1:]):
        part, rl, _ = oracle.fourlist(A, d, mods=mods, slice_range=(a, b), return_records=True)
        assert part == [x for x in full if a <= oracle.slice_of(A, x, mods) < b]
        union += part
        rec_l += rl
    assert sorted(union) == full
    assert rec_l == 1 << (n // 2)


def test_fourlist_slice_of_by_hand():
    # left half = columns 0, 1 of a 4-column instance; rows 1 and 2 mod (3, 2)
    A = np.array([[2, 5, 7, 1], [1, 1, 4, 4]], dtype=np.int32)
    # x = 0b0011: left sums (7, 2) -> residues (1, 0) -> slice 1
    assert oracle.slice_of(A, (0b0011,), (3, 2)) == 1
    # x = 0b0010: left sums (5, 1) -> (2, 1) -> 2 + 3 * 1 = 5
    assert oracle.slice_of(A, (0b0010,), (3, 2)) == 5
    # columns 2, 3 are the right half and never count
    assert oracle.slice_of(A, (0b1100,), (3, 2)) == 0


def test_fourlist_degenerate_inputs():
    A = np.zeros((3, 9), dtype=np.int32)
    assert as_int(oracle.fourlist(A, [0, 0, 0], mods=(2, 3))) == list(range(512))
    assert oracle.fourlist(A, [0, 1, 0]) == []
    A, d, _ = mi.generate(3, 16, 3)
    d2 = d.copy()
    d2[1] = A[1].sum() + 1
    assert oracle.fourlist(A, d2, mods=(4, 4)) == []
    assert oracle.fourlist(A, np.array([-1, 0, 0])) == []
    # n = 1 and n = 2 (empty or one-column halves)
    assert as_int(oracle.fourlist(np.array([[3]]), [3])) == [1]
    assert as_int(oracle.fourlist(np.array([[3, 0]]), [3])) == [1, 3]


@pytest.mark.parametrize("seed", range(4))
def test_fourlist_zero_column_and_row_permutation(seed):
    A, d, _ = mi.generate(4, 22, 3400 + seed, K=4, planted=True, h=11)
    sols = as_int(oracle.fourlist(A, d, mods=(4, 2)))
    A2 = np.hstack([A, np.zeros((4, 1), dtype=np.int32)])
    assert as_int(oracle.fourlist(A2, d, mods=(4, 2))) == sorted(sols + [s | (1 << 22) for s in sols])
    perm = np.array([2, 0, 3, 1])
    assert as_int(oracle.fourlist(A[perm], d[perm], mods=(3, 3))) == sols


def test_fourlist_planted_at_size():
    # the planted x* of a (6,50) instance is found with the default slicing,
    # and the enumeration covers both halves exactly
    A, d, x = mi.generate(6, 50, 21, planted=True, h=25)
    sols, rl, rr = oracle.fourlist(A, d, return_records=True)
    assert mi.mask_of(x) in sols
    assert (rl, rr) == (1 << 25, 1 << 25)
    for s in sols:
        xv = _mask_to_x(s, 50)
        assert np.array_equal(A.astype(np.int64) @ xv, d.astype(np.int64))
