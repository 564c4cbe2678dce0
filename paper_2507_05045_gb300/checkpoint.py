"""Resumable exhaustive solves.

A solve is split into ``parts`` disjoint pieces of the residue classes
(``MSP_OPT_CLASS_PART`` / ``MSP_OPT_CLASS_PARTS``): records of different
classes never match, so the solution set of the instance is the disjoint
union of the pieces' sets.  ``solve_resumable`` solves the pieces one after
another and, after each, rewrites a small JSON checkpoint with the pieces
done and their solutions (written to a temporary file, then renamed, so a
crash leaves the previous checkpoint intact).  Run again with the same
arguments, it skips the pieces the checkpoint holds.  All solving happens in
libmsp; this module only orders the calls and keeps the file.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

FORMAT = 1


def problem_id(A, d, parts: int, plan=None) -> str:
    """sha256 of (A, d, parts, plan): a checkpoint belongs to one problem."""
    A = np.ascontiguousarray(np.asarray(A), dtype=np.int32)
    d = np.ascontiguousarray(np.asarray(d).reshape(-1), dtype=np.int32)
    h = hashlib.sha256()
    h.update(np.asarray(A.shape, dtype=np.int64).tobytes())
    h.update(A.tobytes())
    h.update(d.tobytes())
    h.update(json.dumps({"parts": int(parts), "plan": plan or {}}, sort_keys=True).encode())
    return h.hexdigest()


def _load(path: str, pid: str, parts: int) -> dict:
    if not os.path.exists(path):
        return {"format": FORMAT, "problem": pid, "parts": parts, "done": {}}
    with open(path) as f:
        state = json.load(f)
    if state.get("format") != FORMAT or state.get("problem") != pid or state.get("parts") != parts:
        raise ValueError(f"checkpoint {path} belongs to another problem or split")
    return state


def _save(path: str, state: dict) -> None:
    tmp = f"{path}.tmp.{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(state, f)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def solve_resumable(A, d, path: str, parts: int = 64, plan=None, instance=None, **kwargs):
    """Every solution of A x = d, solved in ``parts`` class pieces with a
    checkpoint at ``path`` after each piece; pieces already in the
    checkpoint are not solved again.  Returns the sorted solution masks
    (tuples of 64-bit words, as ``Instance.solve_all``).  ``instance``
    replaces :class:`Instance` (same constructor); ``kwargs`` go to it."""
    if parts < 1:
        raise ValueError("parts must be at least 1")
    if instance is None:
        from .msp import Instance as instance
    pid = problem_id(A, d, parts, plan)
    state = _load(path, pid, parts)
    for part in range(parts):
        if str(part) in state["done"]:
            continue
        with instance(A, d, class_part=(part, parts), plan=plan, **kwargs) as inst:
            sols = inst.solve_all()
        state["done"][str(part)] = [[format(w, "x") for w in s] for s in sols]
        _save(path, state)
    out = set()
    for sols in state["done"].values():
        for s in sols:
            out.add(tuple(int(w, 16) for w in s))
    return sorted(out)
