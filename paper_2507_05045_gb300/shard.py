"""One exhaustive solve split across ranks by residue classes.

Records of different residue classes never match (the class of a left
half-pair fixes the class of every right half-pair it can pair with), so the
classes of an instance split into ``parts`` disjoint pieces
(``MSP_OPT_CLASS_PART`` / ``MSP_OPT_CLASS_PARTS``) whose solution sets are
disjoint and whose union is the full set.  Rank k of W solves pieces
k, k + W, k + 2W, ... on its own GPU; the only exchange is a gather of the
few solution masks at the end (a handful of 64-bit words per rank), which
goes through ``torch.distributed.all_gather_object``, so any backend
(NCCL between GPUs, gloo on the CPU) serves.  Nothing on the data path
touches another rank's device memory.
"""
from __future__ import annotations


def my_parts(rank: int, world: int, parts: int) -> list[int]:
    """The class pieces rank ``rank`` of ``world`` solves: rank, rank + world, ..."""
    if not (0 <= rank < world) or parts < 1:
        raise ValueError("need 0 <= rank < world and parts >= 1")
    return list(range(rank, parts, world))


def merge(per_rank: list[list[tuple]]) -> list[tuple]:
    """The sorted union of the ranks' solution lists.  The pieces partition
    the solution set, so a mask reported by two ranks means a fault."""
    out = [s for lst in per_rank for s in lst]
    key = (lambda t: tuple(reversed(t)))
    out.sort(key=key)
    for a, b in zip(out, out[1:]):
        if a == b:
            raise RuntimeError(f"solution {a} reported by two class pieces")
    return out


def solve_sharded(A, d, rank: int, world: int, parts: int | None = None, pg=None, solve_part=None,
                  **instance_kw) -> dict:
    """Solve the pieces of this rank and gather every rank's solutions.

    ``parts`` defaults to ``world``.  ``solve_part(k, parts)`` returns the
    sorted solutions of piece k; by default it is an ``msp.Instance`` solve
    with ``class_part=(k, parts)`` (plus ``instance_kw``) on this rank's
    current device.  ``pg`` is ``torch.distributed`` (or None for one rank).
    Returns ``{"solutions": all ranks' solutions (sorted), "mine": this
    rank's, "parts": the pieces it solved, "records": its records}``.
    """
    parts = world if parts is None else int(parts)
    mine_parts = my_parts(rank, world, parts)
    records = 0
    if solve_part is None:
        from . import msp

        def solve_part(k, p):  # noqa: E306
            nonlocal records
            with msp.Instance(A, d, class_part=(k, p), **instance_kw) as inst:
                got = inst.solve_all()
                records += inst.stats()["records_done"]
            return got
    mine = []
    for k in mine_parts:
        mine += solve_part(k, parts)
    mine = merge([mine])
    if pg is None or world == 1:
        everyone = [mine]
    else:
        everyone = [None] * world
        pg.all_gather_object(everyone, [list(s) for s in mine])
        everyone = [[tuple(s) for s in lst] for lst in everyone]
    return {"solutions": merge(everyone), "mine": mine, "parts": mine_parts, "records": records}
