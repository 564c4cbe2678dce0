"""Per-(m, n) plan autotuner.

A plan picks the enumeration path and its tile sizes.  The direct pass
(classes joined in shared memory) has one knob, the shared hash table of
2^table_bits slots.  The streaming pass has three: the residue modulus 2^B
(class bits), the radix digit width D (partitions of about |L| / 2^(B + D)
records) and the uneven quarter split (inner bits: an inner residue bucket
holds about 2^inner elements, the run one outer element expands to in the
scatter).  The library picks them by formula; this module times candidate
plans of both paths on a seeded sample of residue classes of an instance of
the shape and keeps the one with the smallest projected time to all
solutions.  Results are
cached in a JSON file keyed by the device name and (m, n); ``Instance(...,
plan="auto")`` reads the cache.

Every plan yields the same solution set: the tuner only changes how the work
is split, and the tests compare tuned solves with the oracle.
"""
from __future__ import annotations

import json
import os
import threading
import time

import numpy as np

from . import msp

CACHE_ENV = "MSP_AUTOTUNE_CACHE"
_lock = threading.Lock()

# kernels whose time grows with the number of classes solved (the rest build
# the quarter lists once per solve)
_PER_CLASS = ("gen_count", "offsets", "gen_scatter", "join", "join_big", "other", "direct", "recover",
              "verify")
_PER_SOLVE = ("gray", "bucket", "c1")
STREAM_KEYS = ("class_bits", "digit_bits", "inner_bits")
MAX_CLASS_BITS = 27  # MSP_OPT_CLASS_BITS range of the library


def cache_path() -> str:
    p = os.environ.get(CACHE_ENV)
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "msp_autotune.json")


def device_name() -> str:
    return msp.load_library().msp_device_name().decode() or "no-device"


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, data: dict) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def cached_plan(m: int, n: int, path: str | None = None, device: str | None = None) -> dict | None:
    """The cached plan for (m, n) on this device, or None."""
    data = _load(path or cache_path())
    ent = data.get(device or device_name(), {}).get(f"{m},{n}")
    if not ent:
        return None
    return {k: int(ent[k]) for k in msp.PLAN_KEYS if k in ent}


def record_plan(m: int, n: int, plan: dict, info: dict | None = None, path: str | None = None,
                device: str | None = None) -> None:
    """Store a plan for (m, n) on this device in the cache."""
    path = path or cache_path()
    with _lock:
        data = _load(path)
        ent = {k: int(v) for k, v in plan.items() if k in msp.PLAN_KEYS}
        ent.update(info or {})
        data.setdefault(device or device_name(), {})[f"{m},{n}"] = ent
        _store(path, data)


def candidates(base: dict, lg: int, direct: bool = True) -> list[dict]:
    """Candidate plans for sides of 2^lg records.  With ``direct`` (the
    instance fits the direct pass, the formula's default) the direct pass
    with tables of 2^14, 2^13 and 2^15 slots comes first.  Then the streaming
    pass around the formula's choice ``base`` (class_bits B0, digit_bits D0):
    B0 - 1 .. B0 + 1 classes, partitions of about 2^12 or 2^11 records (the
    streaming join holds at most 4608), inner buckets of about 2^3 .. 2^5
    elements, the formula's own streaming plan first."""
    B0, D0 = base["class_bits"], base["digit_bits"]
    out = [{"direct": 1, "table_bits": tb} for tb in (14, 13, 15)] if direct else []
    out.append(dict(base, direct=0))
    for B in (B0 - 1, B0, B0 + 1):
        if B < 0 or B > MAX_CLASS_BITS:
            continue
        for part_bits in (12, 11):
            D = lg - B - part_bits
            if D < 0 or D > 12:
                continue
            for inner in (3, 4, 5):
                c = {"class_bits": B, "digit_bits": D, "inner_bits": inner, "direct": 0}
                if c not in out:
                    out.append(c)
    return out


def _instance(m: int, n: int, seed: int):
    """A seeded instance of the shape: a_ij uniform in [0, 99], d = floor(row
    sum / 2) (the workload the paper's tables use)."""
    rng = np.random.default_rng(seed)
    A = rng.integers(0, 100, size=(m, n), dtype=np.int64).astype(np.int32)
    d = (A.astype(np.int64).sum(axis=1) // 2).astype(np.int32)
    return A, d


def measure(A, d, plan: dict | None, parts: int) -> dict:
    """Solve residue-class part 0 of ``parts`` of (A, d) under ``plan`` and
    project the time to all solutions from the kernels' CUDA-event times."""
    with msp.Instance(A, d, plan=plan, profiling=True, class_part=(0, parts)) as inst:
        t0 = time.perf_counter()
        inst.solve_all()
        wall = time.perf_counter() - t0
        st = inst.stats()
    k = st["kernels"]
    per_class = sum(k[x]["ms"] for x in _PER_CLASS if x in k)
    path = st["path"]
    per_solve = sum(k[x]["ms"] for x in _PER_SOLVE if x in k)
    total = st["records_left"] + st["records_right"]
    done = max(1, st["records_done"])
    proj_ms = per_class * total / done + per_solve
    return {"projected_s": proj_ms / 1e3, "sample_s": wall, "records_done": st["records_done"],
            "class_bits": st["class_bits"], "digit_bits": st["digit_bits"], "quarter": st["quarter"],
            "redone": st["fast_passes_redone"] + st["direct_fallback"], "path": path}


def _parts_for(A, d, plan, sample_records: float) -> int:
    """Class parts so that part 0 holds about ``sample_records`` records."""
    with msp.Instance(A, d, plan=plan, class_part=(0, 1 << 30)) as inst:
        inst.solve_all()  # at most one class: cheap, fills the plan's stats
        st = inst.stats()
    total = st["records_left"] + st["records_right"]
    classes = st["classes_total"]
    want = max(1.0, total / max(1.0, sample_records))
    return int(max(1, min(classes, round(want))))


def autotune(m: int, n: int, A=None, d=None, sample_records: float = 2 ** 33, seed: int = 12345,
             path: str | None = None, force: bool = False, verbose: bool = False) -> dict:
    """Pick the plan for (m, n) on this device (cached unless ``force``).

    Returns ``{"plan": {...}, "projected_s": t, "default_projected_s": t0,
    "table": [...]}``; the plan is also stored in the cache."""
    dev = device_name()
    if not force:
        hit = cached_plan(m, n, path, dev)
        if hit is not None:
            return {"plan": hit, "cached": True}
    if A is None:
        A, d = _instance(m, n, seed)
    A = np.asarray(A, dtype=np.int32)
    d = np.asarray(d, dtype=np.int32).reshape(-1)
    with msp.Instance(A, d, class_part=(0, 1 << 30)) as inst:
        inst.solve_all()  # no class: the formula's default path in the stats
        direct_ok = inst.stats()["path"] == "direct"
    with msp.Instance(A, d, class_part=(0, 1 << 30), plan={"direct": 0}) as inst:
        inst.solve_all()  # the formula's streaming plan
        st = inst.stats()
    q = st["quarter"]
    lg = max(q[0] + q[2], q[1] + q[3])
    # the formula's inner buckets: 2^(inner columns - B) elements (the inner
    # quarter may be capped below B + its target)
    inner0 = max(0, max(q[2], q[3]) - st["class_bits"])
    base = {"class_bits": st["class_bits"], "digit_bits": st["digit_bits"], "inner_bits": inner0}
    table = []
    best = None
    for plan in candidates(base, lg, direct_ok):
        r = measure(A, d, plan, _parts_for(A, d, plan, sample_records))
        r["plan"] = plan
        table.append(r)
        if verbose:
            print(f"autotune ({m},{n}) {plan}: projected {r['projected_s']:.3f} s", flush=True)
        if r["redone"] == 0 and (best is None or r["projected_s"] < best["projected_s"]):
            best = r
    if best is None:
        best = table[0]
    info = {"projected_s": best["projected_s"], "default_projected_s": table[0]["projected_s"],
            "sample_records": float(sample_records)}
    record_plan(m, n, best["plan"], info, path, dev)
    return {"plan": best["plan"], "projected_s": best["projected_s"],
            "default_projected_s": table[0]["projected_s"], "table": table, "cached": False}
