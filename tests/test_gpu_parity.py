"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

The result of a solve is an exact set of integer bitmasks, so every
comparison here is bit-exact: the sorted solution list of libmsp must equal
the oracle's.  Inputs come from the seeded generator only.
"""
import json
import os

import numpy as np
import pytest

import msp_instances as mi
import oracle

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# the two enumeration paths of a solve: the direct pass (classes joined in
# shared memory) and the streaming / exact residue passes
PATHS = [pytest.param({"direct": 1}, id="direct"), pytest.param({"direct": 0}, id="streaming")]


def solve(msp, A, d, plan, expect_path=True):
    with msp.Instance(A, d, plan=plan) as inst:
        got = inst.solve_all()
        st = inst.stats()
    if expect_path and plan.get("direct") == 0:
        assert st["path"] == "streaming"
    return got, st


@pytest.fixture(scope="module")
def msp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_05045_gb300 import build
    build.build()
    import paper_2507_05045_gb300 as m
    return m


def load_golden(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated")
    g = json.load(open(path))
    out = []
    for e in g["instances"]:
        A, d, x = mi.generate(e["m"], e["n"], e["seed"], planted=e["planted"], h=e["h"])
        sols = [tuple(int(w, 16) for w in s) for s in e.get("solutions", [])]
        out.append((e, A, d, x, sols))
    return out


@pytest.mark.parametrize("plan", PATHS)
def test_hand_instances(msp, plan):
    g = json.load(open(os.path.join(GOLDEN, "hand_instances.json")))
    for inst in g["instances"]:
        got, _ = solve(msp, np.array(inst["A"]), np.array(inst["d"]), plan)
        assert [s[0] for s in got] == inst["solutions"], inst["name"]


@pytest.mark.parametrize("plan", PATHS)
@pytest.mark.parametrize("seed", range(40))
def test_random_small_vs_brute(msp, seed, plan):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 11))
    n = int(rng.integers(1, 23))
    K = int(rng.choice([2, 3, 5, 20, 100]))
    A, d, _ = mi.generate(m, n, 5000 + seed, K=K, planted=bool(seed % 2), h=n // 2)
    got, st = solve(msp, A, d, plan)
    assert got == oracle.brute(A, d)


@pytest.mark.parametrize("plan", PATHS)
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 9, 13])
def test_tiny_n_every_quarter_shape(msp, n, plan):
    for seed in range(3):
        A, d, _ = mi.generate(2, n, 90 + seed, K=3, planted=True, h=n // 2)
        assert solve(msp, A, d, plan)[0] == oracle.brute(A, d)


@pytest.mark.parametrize("plan", PATHS)
def test_sixteen_rows_and_wide_row_sums(msp, plan):
    # m = 16: four packed 16-bit words per vector; row sums near the 2^16
    # field limit with large coefficients
    for seed in range(3):
        A, d, _ = mi.generate(16, 20, 5 + seed, K=50, planted=True, h=10)
        assert solve(msp, A, d, plan)[0] == oracle.brute(A, d)
    A, d, _ = mi.generate(3, 21, 6, K=3100, planted=True, h=10)
    assert A.sum(axis=1).max() > 30000
    assert solve(msp, A, d, plan)[0] == oracle.brute(A, d)


@pytest.mark.parametrize("seed", range(24))
def test_random_sweep_all_paths(msp, seed):
    # random shapes and coefficient ranges: direct, streaming and exact passes
    # against the oracle
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 17))
    n = int(rng.integers(10, 31))
    K = int(rng.choice([2, 3, 7, 100, 1000]))
    A, d, _ = mi.generate(m, n, 20000 + seed, K=K, planted=bool(seed % 2), h=n // 2)
    want = oracle.brute(A, d) if n <= 20 else oracle.mitm(A, d)
    assert solve(msp, A, d, {"direct": 1})[0] == want
    assert solve(msp, A, d, {"direct": 0})[0] == want
    with msp.Instance(A, d, exact_path=True) as inst:
        assert inst.solve_all() == want


@pytest.mark.parametrize("plan", PATHS)
def test_degenerate_inputs(msp, plan):
    # all-zero matrix: every vector solves d = 0, none solves d != 0
    A = np.zeros((3, 12), np.int32)
    assert [s[0] for s in solve(msp, A, [0, 0, 0], plan)[0]] == list(range(1 << 12))
    assert solve(msp, A, [0, 1, 0], plan, False)[0] == []
    # right-hand side above a row sum
    A, d, _ = mi.generate(3, 16, 3)
    d2 = d.copy()
    d2[1] = A[1].sum() + 1
    assert solve(msp, A, d2, plan, False)[0] == []
    # d = 0 with positive entries: x = 0 only
    A = np.arange(1, 21, dtype=np.int32).reshape(2, 10)
    assert solve(msp, A, [0, 0], plan)[0] == [(0,)]
    # zero columns and duplicate rows
    A, d, _ = mi.generate(3, 18, 4, K=4, planted=True, h=9)
    A2 = np.hstack([A, np.zeros((3, 2), np.int32)])
    A2 = np.vstack([A2, A2[0:1]])
    d2 = np.concatenate([d, d[0:1]])
    assert solve(msp, A2, d2, plan)[0] == oracle.brute(A2, d2)


@pytest.mark.parametrize("plan", PATHS)
@pytest.mark.parametrize("seed", range(6))
def test_small_K_long_equal_key_runs(msp, seed, plan):
    # K = 2: many subsets share one vector, so keys repeat in long runs
    A, d, _ = mi.generate(2, 22, 6000 + seed, K=2, planted=True, h=11)
    assert solve(msp, A, d, plan)[0] == oracle.brute(A, d)


def test_config_4_30(msp):
    for e, A, d, x, sols in load_golden("sols_4_30.json"):
        got = msp.solve_all(A, d)
        assert got == sols
        if x is not None:
            assert mi.mask_of(x) in got


@pytest.mark.parametrize("plan", PATHS)
@pytest.mark.parametrize("seed", range(4))
def test_5_40_vs_mitm(msp, seed, plan):
    A, d, _ = mi.generate(5, 40, 7000 + seed, planted=bool(seed % 2), h=20)
    got, st = solve(msp, A, d, plan)
    assert got == oracle.mitm(A, d)
    if plan["direct"]:
        assert st["path"] == "direct"


@pytest.mark.parametrize("plan", PATHS)
def test_row1_candidate_count_matches_counting_dp(msp, plan):
    for (m, n, seed) in [(4, 30, 1), (5, 40, 2), (6, 50, 3), (3, 22, 4)]:
        A, d, _ = mi.generate(m, n, seed)
        _, st = solve(msp, A, d, plan)
        assert st["row1_candidates"] == oracle.row1_candidates(A, d)


@pytest.mark.parametrize("path", [-1, 1, 0])
def test_config_6_50_batch(msp, path):
    # one batched call over 64 instances: direct pass (default and forced)
    # and streaming pass
    entries = load_golden("sols_6_50_batch.json")
    got = msp.solve_batch([(A, d) for _, A, d, _, _ in entries], path=path)
    for (e, A, d, x, sols), g in zip(entries, got):
        assert g == sols, e["seed"]
        if x is not None:
            assert mi.mask_of(x) in g


def test_batch_mixed_feasibility_and_tags(msp):
    # infeasible right-hand sides, planted and plain instances and small-K
    # instances with many solutions in one batch: every instance keeps its
    # own solution set (match and solution tags carry the instance)
    insts = []
    for k in range(12):
        A, d, _ = mi.generate(4, 30, 300 + k, K=[100, 5, 3][k % 3], planted=bool(k % 2), h=15)
        if k % 4 == 3:
            d = d.copy()
            d[2] = A[2].sum() + 1
        insts.append((A, d))
    want = [oracle.mitm(A, d) for A, d in insts]
    # the heavy small-K instances may exceed the direct verification's
    # candidate lists, so the automatic choice may fall back to streaming
    for path in (-1, 0):
        assert msp.solve_batch(insts, path=path) == want
    light = [insts[k] for k in range(12) if k % 3 == 0]
    assert msp.solve_batch(light, path=1) == [want[k] for k in range(12) if k % 3 == 0]


@pytest.mark.parametrize("plan", PATHS)
def test_config_6_50_single(msp, plan):
    for e, A, d, x, sols in load_golden("sols_6_50_batch.json")[:8]:
        got, st = solve(msp, A, d, plan)
        assert got == sols
        if plan["direct"]:
            assert st["path"] == "direct"


def test_many_passes_same_result(msp):
    # a small budget forces many residue passes: the set must not change
    e, A, d, x, sols = load_golden("sols_6_50_batch.json")[40]
    with msp.Instance(A, d, memory_budget=400 << 20, plan={"direct": 0}) as inst:
        got = inst.solve_all()
        st = inst.stats()
    assert got == sols
    assert st["passes"] >= 1


@pytest.mark.parametrize("plan", PATHS)
@pytest.mark.parametrize("name", ["sols_7_60.json", "sols_7_60_planted.json", "sols_7_60_more.json"])
def test_config_7_60(msp, name, plan):
    for e, A, d, x, sols in load_golden(name):
        got, st = solve(msp, A, d, plan)
        assert got == sols
        assert st["row1_candidates"] == oracle.row1_candidates(A, d)
        if plan["direct"]:
            assert st["path"] == "direct"


def _check_solutions_exact(A, d, sols):
    A = np.asarray(A, dtype=np.int64)
    n = A.shape[1]
    for s in sols:
        v = sum(w << (64 * k) for k, w in enumerate(s))
        x = np.array([(v >> j) & 1 for j in range(n)], dtype=np.int64)
        assert np.array_equal(A @ x, np.asarray(d, dtype=np.int64))


def _subcube_parity(msp_sols, A, d, fixed_cols, fixed_vals):
    """GPU solutions agreeing with the fixed columns == oracle on the restriction."""
    A2, d2, free = mi.restrict(A, d, fixed_cols, fixed_vals)
    n = np.asarray(A).shape[1]
    if np.any(d2 < 0):
        want = []
    else:
        want = oracle.mitm(A2, d2.astype(np.int32))
    lifted = []
    for s in want:
        v = sum(w << (64 * k) for k, w in enumerate(s))
        full = sum(1 << fixed_cols[i] for i in range(len(fixed_cols)) if fixed_vals[i])
        full |= sum(1 << free[j] for j in range(len(free)) if (v >> j) & 1)
        lifted.append(full)
    got = []
    for s in msp_sols:
        v = sum(w << (64 * k) for k, w in enumerate(s))
        if all(((v >> c) & 1) == b for c, b in zip(fixed_cols, fixed_vals)):
            got.append(v)
    assert sorted(got) == sorted(lifted)


@pytest.mark.parametrize("plan", PATHS)
def test_config_8_70_full_solution_sets(msp, plan):
    # the plain and the planted (8,70) instance of seed 8: every solution,
    # compared with the four-list oracle's full enumeration (2^36 records)
    for e, A, d, x, sols in load_golden("sols_8_70.json"):
        got, st = solve(msp, A, d, plan)
        assert got == sols, (e["planted"], len(got), len(sols))
        assert st["row1_candidates"] == oracle.row1_candidates(A, d)
        if x is not None:
            assert mi.mask_of(x) in got


@pytest.mark.slow
def test_config_9_80_bench_instance_full_solution_set(msp):
    # the benchmark's plain (9,80) instance (seed 9080): every solution of the
    # exhaustive solve, compared with the four-list oracle's full enumeration
    # of all 2^41 half-subset records
    for e, A, d, x, sols in load_golden("sols_9_80.json"):
        with msp.Instance(A, d) as inst:
            got = inst.solve_all()
            st = inst.stats()
        assert st["path"] == "direct"
        assert got == sols
        assert e["records"] == [1 << 40, 1 << 40]


@pytest.mark.parametrize("plan", PATHS)
def test_config_8_70_planted_properties_and_subcube(msp, plan):
    A, d, x = mi.generate(8, 70, 8, planted=True, h=35)
    sols, st = solve(msp, A, d, plan)
    assert mi.mask_of(x) in sols
    _check_solutions_exact(A, d, sols)
    assert st["row1_candidates"] == oracle.row1_candidates(A, d)
    # 26 columns fixed to x*: the 44 free columns are solved by the oracle
    rng = np.random.default_rng(8)
    cols = sorted(int(c) for c in rng.choice(70, 26, replace=False))
    _subcube_parity(sols, A, d, cols, [int(x[c]) for c in cols])


@pytest.mark.slow
def test_config_9_80_planted_properties_and_subcube(msp):
    A, d, x = mi.generate(9, 80, 9, planted=True, h=40)
    with msp.Instance(A, d) as inst:
        sols = inst.solve_all()
        st = inst.stats()
    assert st["path"] == "direct"
    assert mi.mask_of(x) in sols
    _check_solutions_exact(A, d, sols)
    assert st["row1_candidates"] == oracle.row1_candidates(A, d)
    rng = np.random.default_rng(9)
    cols = sorted(int(c) for c in rng.choice(80, 34, replace=False))
    _subcube_parity(sols, A, d, cols, [int(x[c]) for c in cols])
    # the four-list oracle's full solution set of the same instance, when stored
    if os.path.exists(os.path.join(GOLDEN, "sols_9_80_planted.json")):
        (e, A2, d2, x2, want), = load_golden("sols_9_80_planted.json")
        assert np.array_equal(A2, A) and np.array_equal(d2, d)
        assert sols == want


def test_row_and_column_permutation_invariance(msp):
    A, d, x = mi.generate(6, 48, 77, K=20, planted=True, h=24)
    base = msp.solve_all(A, d)
    perm_r = np.array([3, 0, 5, 1, 4, 2])
    assert msp.solve_all(A[perm_r], d[perm_r]) == base
    perm_c = np.random.default_rng(1).permutation(48)
    got = msp.solve_all(A[:, perm_c], d)
    mapped = sorted(
        (sum(1 << k for k in range(48) if (s[0] >> perm_c[k]) & 1),) for s in base)
    assert got == mapped


def test_server_mixed_stream_matches_single_solves(msp):
    insts = []
    for k in range(24):
        m = [4, 5, 6][k % 3]
        A, d, _ = mi.generate(m, 10 * (m - 1), 8000 + k, planted=bool(k % 2), h=5 * (m - 1))
        insts.append((A, d))
    alone = [msp.solve_all(A, d) for A, d in insts]
    with msp.Server(max_inflight=4) as srv:
        ids = [srv.submit(A, d) for A, d in insts]
        results = {}
        import time
        t0 = time.time()
        while len(results) < len(ids) and time.time() - t0 < 300:
            for i in ids:
                if i not in results:
                    r = srv.poll(i)
                    if r is not None:
                        results[i] = r
            time.sleep(0.002)
    assert [results[i] for i in ids] == alone


@pytest.mark.parametrize("seed", range(8))
def test_exact_path_matches_streaming_path(msp, seed):
    # the streaming pass and the two-phase exact pass must give the same set
    rng = np.random.default_rng(900 + seed)
    m = int(rng.integers(2, 8))
    n = int(rng.integers(18, 41))
    K = int(rng.choice([3, 10, 100]))
    A, d, _ = mi.generate(m, n, 9000 + seed, K=K, planted=True, h=n // 2)
    want = oracle.brute(A, d) if n <= 22 else oracle.mitm(A, d)
    with msp.Instance(A, d, exact_path=True) as inst:
        assert inst.solve_all() == want
    assert solve(msp, A, d, {"direct": 0})[0] == want
    assert solve(msp, A, d, {"direct": 1})[0] == want


def test_degenerate_instance_falls_back_to_exact_passes(msp):
    # eight zero columns in Q1: every left key repeats 256 times, so the
    # partitions of the streaming pass overflow and the exact path re-runs them
    A, d, x = mi.generate(4, 36, 4242, planted=True, h=18)
    A = A.copy()
    A[:, :8] = 0
    d = (A.astype(np.int64) @ x.astype(np.int64)).astype(np.int32)
    want = oracle.mitm(A, d)
    got, st = solve(msp, A, d, {"direct": 0})
    assert got == want
    assert len(got) >= 256
    assert st["fast_passes_redone"] >= 1
    # the direct pass holds each repeated key once in its table
    assert solve(msp, A, d, {"direct": 1})[0] == want


@pytest.mark.parametrize("plan", PATHS)
def test_class_parts_partition_the_solution_set(msp, plan):
    # the solutions of the residue-class parts are disjoint and their union
    # is the full set; records_done adds up to all records
    A, d, x = mi.generate(6, 50, 4321, K=20, planted=True, h=25)
    full, st_full = solve(msp, A, d, plan)
    parts, union, recs = 4, [], 0
    for k in range(parts):
        with msp.Instance(A, d, class_part=(k, parts), plan=plan) as inst:
            got = inst.solve_all()
            st = inst.stats()
        assert set(got).isdisjoint(union)
        union += got
        recs += st["records_done"]
        assert st["classes_done"] * parts == st["classes_total"]
    assert sorted(union) == full
    assert recs == st_full["records_done"] == st_full["records_left"] + st_full["records_right"]
    assert mi.mask_of(x) in full


@pytest.mark.parametrize("plan", [
    {"class_bits": 3, "digit_bits": 2, "inner_bits": 3},
    {"class_bits": 6, "digit_bits": 4, "inner_bits": 6},
    {"class_bits": 0, "digit_bits": 0},     # one class, unsplit: exact-path passes
    {"class_bits": 9, "digit_bits": 0, "inner_bits": 0},
    {"inner_bits": 12},
])
def test_plan_choices_give_the_oracle_solutions(msp, plan):
    # every plan the autotuner may set splits the same work differently and
    # must return exactly the golden solution set
    for e, A, d, x, sols in load_golden("sols_6_50_batch.json")[:4]:
        with msp.Instance(A, d, plan=plan) as inst:
            got = inst.solve_all()
            st = inst.stats()
        assert got == sols, (plan, e["seed"])
        if "class_bits" in plan:
            assert st["class_bits"] == plan["class_bits"]
        if "digit_bits" in plan:
            assert st["digit_bits"] == plan["digit_bits"]


@pytest.mark.parametrize("tb", [12, 13, 15])
def test_direct_table_sizes_and_chunked_classes(msp, tb):
    # a 2^12-slot table holds 3072 left keys: the 2^13-record classes of
    # (6,50) are joined in three table fills, each probed by every right key
    for e, A, d, x, sols in load_golden("sols_6_50_batch.json")[:6]:
        got, st = solve(msp, A, d, {"direct": 1, "table_bits": tb})
        assert got == sols, (tb, e["seed"])
        assert st["path"] == "direct"
    for e, A, d, x, sols in load_golden("sols_7_60_planted.json"):
        assert solve(msp, A, d, {"direct": 1, "table_bits": tb})[0] == sols


def test_direct_pass_on_skewed_classes(msp):
    # K = 3 and zero columns: few distinct row vectors, classes of very
    # unequal size and long runs of equal keys; both paths give the oracle set
    A, _, x = mi.generate(5, 30, 31, K=3, planted=True, h=15)
    A = A.copy()
    A[:, 3:6] = 0
    d = (A.astype(np.int64) @ x.astype(np.int64)).astype(np.int32)
    want = oracle.mitm(A, d)
    assert len(want) > 1000
    for tb in (12, 14):
        got, st = solve(msp, A, d, {"direct": 1, "table_bits": tb})
        assert got == want
    assert solve(msp, A, d, {"direct": 0})[0] == want


def test_inner_list_window_past_the_stage(msp):
    # n = 46 splits 23/23 with 2^10 classes (keyed on rows 1-2) and inner
    # quarters of columns 9..22 and 32..45.  With rows 1 and 2 zero on the
    # left inner columns, all 2^14 left inner subsets fall into one class
    # (their keys, set by rows 3-5, stay distinct), so its window of classes
    # holds more subsets than the shared-memory stage and the list build
    # places them directly; the joins see classes of several table fills.
    A, _, x = mi.generate(5, 46, 4646, planted=True, h=16)
    A = A.copy()
    A[:2, 9:23] = 0
    d = (A.astype(np.int64) @ x.astype(np.int64)).astype(np.int32)
    want = oracle.mitm(A, d)
    assert mi.mask_of(x) in want
    got, st = solve(msp, A, d, {"direct": 1})
    assert st["path"] == "direct" and st["class_bits"] == 10 and st["direct_fallback"] == 0
    assert got == want


def test_streaming_pass_with_large_inner_quarters(msp):
    # the streaming pass with inner quarters of 27 columns (the shape the
    # (10,90) configuration takes), on the (10,70) restriction of a planted
    # (10,90) instance (20 seeded columns fixed to x*), against the oracle's
    # full solution set of that restriction
    for e, A, d, x, _ in load_golden("sols_10_70_subcube.json"):
        A2, d2, free = mi.restrict(A, d, e["fixed_cols"], e["fixed_vals"])
        want = [tuple(int(w, 16) for w in s) for s in e["solutions_restricted"]]
        plan = {"class_bits": 22, "digit_bits": 1, "inner_bits": 5, "direct": 0}
        got, st = solve(msp, A2, d2.astype(np.int32), plan)
        assert max(st["quarter"][2], st["quarter"][3]) == 27
        assert got == want
        # x* restricted to the free columns is among them
        xs = sum(1 << j for j, c in enumerate(free) if x[c])
        assert (xs,) in got or (xs & ((1 << 64) - 1), xs >> 64) in got
        assert solve(msp, A2, d2.astype(np.int32), {"direct": 1})[0] == want
        # the shape of the default (10,90) plan: 2^24 classes, inner quarters
        # of 29 columns (2^29-entry lists, buckets of about 32)
        plan = {"class_bits": 24, "digit_bits": 0, "inner_bits": 5, "direct": 0}
        got, st = solve(msp, A2, d2.astype(np.int32), plan)
        assert st["class_bits"] == 24 and max(st["quarter"][2], st["quarter"][3]) == 29
        assert got == want
        # the shape of the earlier (10,90) plan: 2^25 classes, buckets of 16
        plan = {"class_bits": 25, "digit_bits": 0, "inner_bits": 4, "direct": 0}
        got, st = solve(msp, A2, d2.astype(np.int32), plan)
        assert st["class_bits"] == 25 and max(st["quarter"][2], st["quarter"][3]) == 29
        assert got == want


@pytest.mark.slow
def test_streaming_pass_with_the_n100_plan_shape(msp):
    # the shape of the default (11,100) plan: 2^27 classes and inner quarters
    # of 30 columns (2^30-entry lists, about 120 GB), exact class sizes summed
    # over the outer elements, on the (10,70) restriction of the planted
    # (10,90) instance against the oracle's full set
    for e, A, d, x, _ in load_golden("sols_10_70_subcube.json"):
        A2, d2, free = mi.restrict(A, d, e["fixed_cols"], e["fixed_vals"])
        want = [tuple(int(w, 16) for w in s) for s in e["solutions_restricted"]]
        plan = {"class_bits": 27, "digit_bits": 0, "inner_bits": 4, "direct": 0}
        got, st = solve(msp, A2, d2.astype(np.int32), plan)
        assert st["class_bits"] == 27 and max(st["quarter"][2], st["quarter"][3]) == 30
        assert got == want


def test_streaming_pass_with_many_classes(msp):
    # the plans of n >= 96 take up to 2^27 residue classes, whose exact sizes
    # come from the outer elements (fewer than the classes); forced here on
    # the (8,70) instances (2^24 classes of 2^11 records) and a (6,50) one
    # (2^27 classes, most of them empty) against the oracle's full sets
    for e, A, d, x, sols in load_golden("sols_8_70.json"):
        got, st = solve(msp, A, d, {"class_bits": 24, "digit_bits": 0, "direct": 0})
        assert st["class_bits"] == 24 and st["classes_total"] == 1 << 24
        assert got == sols, e["planted"]
    for e, A, d, x, sols in load_golden("sols_6_50_batch.json")[32:34]:
        got, st = solve(msp, A, d, {"class_bits": 27, "digit_bits": 0, "direct": 0})
        assert st["class_bits"] == 27
        assert got == sols, e["seed"]


def test_first_solution_mode_streaming_pass(msp):
    # the streaming pass verifies after every residue pass and stops at the
    # first one that yields a solution: a nonempty subset of the oracle's set
    for e, A, d, x, sols in load_golden("sols_8_70.json"):
        with msp.Instance(A, d, plan={"direct": 0}, first=True, memory_budget=4 << 30) as inst:
            got = inst.solve_all()
            st = inst.stats()
        assert st["path"] == "streaming"
        assert got and set(got) <= set(sols), e["planted"]
        assert 0 < st["classes_done"] <= st["classes_total"]
    for e, A, d, x, sols in load_golden("sols_6_50_batch.json")[:3]:
        with msp.Instance(A, d, plan={"direct": 0}, first=True) as inst:
            got = inst.solve_all()
            st = inst.stats()
        if not sols:
            assert got == [] and st["classes_done"] == st["classes_total"]
        else:
            assert got and set(got) <= set(sols)


@pytest.mark.slow
def test_config_10_90_full_size_first_solution(msp):
    # the (10,90) configuration at full size on the streaming pass (2^24
    # classes, 29-column inner quarters, lists of about 17 GB): a planted
    # instance whose first solution lies in the first few percent of the
    # classes (seed 1093, x* with 45 ones) stops early, and every solution it
    # reports solves A x = d exactly
    A, d, x = mi.generate(10, 90, 1093, planted=True, h=45)
    with msp.Instance(A, d, first=True) as inst:
        got = inst.solve_all()
        st = inst.stats()
    assert st["path"] == "streaming" and st["class_bits"] == 24
    assert got
    _check_solutions_exact(A, d, got)
    assert 0 < st["classes_done"] < st["classes_total"]


def test_first_solution_mode(msp):
    # time-to-first: a nonempty subset of the oracle's full solution set,
    # found before all classes are joined; an instance without solutions is
    # searched to the end and returns none
    for e, A, d, x, sols in load_golden("sols_8_70.json"):
        with msp.Instance(A, d, plan={"direct": 1}) as inst:
            inst.solve_all()
            st_full = inst.stats()
        with msp.Instance(A, d, plan={"direct": 1}, first=True) as inst:
            got = inst.solve_all()
            st = inst.stats()
        assert got and set(got) <= set(sols), e["planted"]
        assert st["path"] == "direct"
        assert 0 < st["classes_done"] <= st["classes_total"] == st_full["classes_total"]
        assert st["records_done"] <= st_full["records_done"]
    for e, A, d, x, sols in load_golden("sols_6_50_batch.json")[:3]:
        with msp.Instance(A, d, plan={"direct": 1}, first=True) as inst:
            got = inst.solve_all()
            st = inst.stats()
        if not sols:
            assert got == [] and st["classes_done"] == st["classes_total"]
        else:
            assert got and set(got) <= set(sols)


def test_plan_options_are_validated(msp):
    A, d, _ = mi.generate(4, 30, 1)
    for bad in [{"class_bits": 28}, {"digit_bits": 13}, {"inner_bits": -2}, {"table_bits": 16},
                {"table_bits": 11}, {"direct": 2}]:
        with pytest.raises(msp.MspError) as e:
            msp.Instance(A, d, plan=bad)
        assert e.value.code == -2
    with pytest.raises(msp.MspError):
        msp.Instance(A, d, plan={"unknown": 1})


def test_autotune_picks_a_cached_plan_with_oracle_solutions(msp, tmp_path, monkeypatch):
    from paper_2507_05045_gb300 import autotune
    monkeypatch.setenv(autotune.CACHE_ENV, str(tmp_path / "tune.json"))
    res = autotune.autotune(6, 50, sample_records=2 ** 24)
    assert not res["cached"]
    assert len(res["table"]) >= 2
    assert res["projected_s"] <= res["default_projected_s"]
    again = autotune.autotune(6, 50)
    assert again["cached"] and again["plan"] == res["plan"]
    e, A, d, x, sols = load_golden("sols_6_50_batch.json")[1]
    with msp.Instance(A, d, plan="auto") as inst:
        assert inst.plan == res["plan"]
        assert inst.solve_all() == sols
