"""Host logic of the plan autotuner (no GPU): candidate plans and the cache."""
import json

import pytest

from paper_2507_05045_gb300 import autotune, msp


def test_candidates_start_with_the_formula_plan_and_are_distinct():
    base = {"class_bits": 19, "digit_bits": 9, "inner_bits": 4}
    cands = autotune.candidates(base, 40)
    # the direct pass (the formula's default) with its table sizes first
    assert cands[0] == {"direct": 1, "table_bits": 14}
    assert [c for c in cands if c["direct"] == 1] == cands[:3]
    assert {c["table_bits"] for c in cands[:3]} == {13, 14, 15}
    assert cands[3] == dict(base, direct=0)
    keys = [tuple(sorted(c.items())) for c in cands]
    assert len(keys) == len(set(keys))
    for c in cands[3:]:
        assert set(c) == set(autotune.STREAM_KEYS) | {"direct"} and c["direct"] == 0
        assert set(c) <= set(msp.PLAN_KEYS)
        assert 0 <= c["class_bits"] <= 27 and 0 <= c["digit_bits"] <= 12
        assert abs(c["class_bits"] - 19) <= 1
        # partitions of 2^11 .. 2^12 records: inside the streaming join's capacity
        if c is not cands[3]:
            assert 40 - c["class_bits"] - c["digit_bits"] in (11, 12)
    # an instance the direct pass does not fit gets streaming plans only
    assert all(c["direct"] == 0 for c in autotune.candidates(base, 45, direct=False))


def test_candidates_respect_the_bounds():
    for lg, B0, D0 in [(15, 0, 3), (50, 23, 12), (50, 27, 12), (1, 0, 0)]:
        for c in autotune.candidates({"class_bits": B0, "digit_bits": D0, "inner_bits": 4}, lg, False):
            assert 0 <= c["class_bits"] <= 27
            assert 0 <= c["digit_bits"] <= 12


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    assert autotune.cached_plan(9, 80, path, device="GPU-A") is None
    autotune.record_plan(9, 80, {"class_bits": 18, "digit_bits": 10, "inner_bits": 3, "bogus": 1},
                         {"projected_s": 1.5}, path, device="GPU-A")
    autotune.record_plan(8, 70, {"class_bits": 14}, None, path, device="GPU-A")
    autotune.record_plan(9, 80, {"class_bits": 20}, None, path, device="GPU-B")
    assert autotune.cached_plan(9, 80, path, device="GPU-A") == {
        "class_bits": 18, "digit_bits": 10, "inner_bits": 3}
    assert autotune.cached_plan(8, 70, path, device="GPU-A") == {"class_bits": 14}
    assert autotune.cached_plan(9, 80, path, device="GPU-B") == {"class_bits": 20}
    assert autotune.cached_plan(7, 60, path, device="GPU-A") is None
    data = json.load(open(path))
    assert data["GPU-A"]["9,80"]["projected_s"] == 1.5


def test_corrupt_cache_reads_as_empty(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    assert autotune.cached_plan(9, 80, str(path), device="X") is None


def test_cache_path_follows_the_environment(monkeypatch, tmp_path):
    monkeypatch.setenv(autotune.CACHE_ENV, str(tmp_path / "c.json"))
    assert autotune.cache_path() == str(tmp_path / "c.json")


def test_seeded_instance_shape_and_rhs():
    A, d = autotune._instance(6, 50, 7)
    assert A.shape == (6, 50) and A.dtype.name == "int32"
    assert ((A >= 0) & (A <= 99)).all()
    assert list(d) == [int(r.sum()) // 2 for r in A.astype("int64")]
