"""Resumable solves (class pieces with a checkpoint file), on the CPU.

The pieces are solved by a stand-in for ``Instance`` whose piece k returns a
fixed set of masks; the tests check the order of the calls, the file, a
crash between pieces and the refusal of another problem's checkpoint.
"""
import json

import numpy as np
import pytest

from paper_2507_05045_gb300 import checkpoint

A = np.arange(12, dtype=np.int32).reshape(2, 6)
D = np.array([7, 19], dtype=np.int32)


def piece_solutions(k, parts):
    # disjoint per piece, as the class pieces of a real solve are
    return [(k,), (1000 + k,)] if k % 3 != 1 else []


class FakeInstance:
    calls = []
    crash_at = None

    def __init__(self, A, d, class_part=None, plan=None):
        self.part, self.parts = class_part

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def solve_all(self):
        if self.part == FakeInstance.crash_at:
            raise RuntimeError("process lost")
        FakeInstance.calls.append(self.part)
        return piece_solutions(self.part, self.parts)


@pytest.fixture(autouse=True)
def reset():
    FakeInstance.calls = []
    FakeInstance.crash_at = None


def expected(parts):
    return sorted(s for k in range(parts) for s in piece_solutions(k, parts))


def test_all_pieces_once_and_union(tmp_path):
    path = str(tmp_path / "ck.json")
    got = checkpoint.solve_resumable(A, D, path, parts=8, instance=FakeInstance)
    assert got == expected(8)
    assert FakeInstance.calls == list(range(8))
    state = json.load(open(path))
    assert sorted(int(k) for k in state["done"]) == list(range(8))


def test_crash_then_resume_skips_done_pieces(tmp_path):
    path = str(tmp_path / "ck.json")
    FakeInstance.crash_at = 5
    with pytest.raises(RuntimeError):
        checkpoint.solve_resumable(A, D, path, parts=8, instance=FakeInstance)
    assert FakeInstance.calls == [0, 1, 2, 3, 4]
    state = json.load(open(path))
    assert sorted(int(k) for k in state["done"]) == [0, 1, 2, 3, 4]
    FakeInstance.calls = []
    FakeInstance.crash_at = None
    got = checkpoint.solve_resumable(A, D, path, parts=8, instance=FakeInstance)
    assert FakeInstance.calls == [5, 6, 7]
    assert got == expected(8)
    # a finished checkpoint solves nothing more
    FakeInstance.calls = []
    assert checkpoint.solve_resumable(A, D, path, parts=8, instance=FakeInstance) == expected(8)
    assert FakeInstance.calls == []


def test_checkpoint_of_another_problem_is_refused(tmp_path):
    path = str(tmp_path / "ck.json")
    checkpoint.solve_resumable(A, D, path, parts=4, instance=FakeInstance)
    with pytest.raises(ValueError):
        checkpoint.solve_resumable(A, D + 1, path, parts=4, instance=FakeInstance)
    with pytest.raises(ValueError):
        checkpoint.solve_resumable(A, D, path, parts=8, instance=FakeInstance)
    with pytest.raises(ValueError):
        checkpoint.solve_resumable(A, D, path, parts=4, plan={"direct": 0}, instance=FakeInstance)


def test_masks_round_trip_wide_words(tmp_path):
    # two-word masks (n > 64) survive the hex encoding of the file
    class Wide(FakeInstance):
        def solve_all(self):
            return [((1 << 64) - 1, self.part << 40)]
    path = str(tmp_path / "ck.json")
    got = checkpoint.solve_resumable(A, D, path, parts=3, instance=Wide)
    assert got == [((1 << 64) - 1, k << 40) for k in range(3)]
    assert checkpoint.solve_resumable(A, D, path, parts=3, instance=Wide) == got


def test_problem_id_depends_on_every_input():
    base = checkpoint.problem_id(A, D, 8)
    assert base == checkpoint.problem_id(A.copy(), D.copy(), 8)
    A2 = A.copy()
    A2[1, 5] += 1
    assert checkpoint.problem_id(A2, D, 8) != base
    assert checkpoint.problem_id(A.reshape(3, 4), D, 8) != base
    assert checkpoint.problem_id(A, D, 9) != base
    assert checkpoint.problem_id(A, D, 8, {"direct": 1}) != base
