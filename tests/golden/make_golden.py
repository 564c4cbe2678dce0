"""Write the stored solution sets of the benchmark-shaped instances.

Calls only the CPU oracle (``oracle/``) and the instance generator
(``msp_instances``); nothing here touches the CUDA path.  Run from the
repository root:

    python tests/golden/make_golden.py [--big]

``--big`` also writes the (7,60) instance, which takes minutes of CPU.
``--only 8_70`` writes the (8,70) instance of seed 8, plain and planted, in
full with the four-list oracle (minutes of CPU); ``--only 9_80`` writes the
plain (9,80) instance of seed 9080 in full (the benchmark instance; about two
hours on 8 cores); ``--only 9_80_planted`` the planted (9,80) instance of
seed 9 (40 ones) likewise.  Those runs go slice range by slice range and keep their
progress in a state file beside the output (``--state``), so an interrupted
run resumes where it stopped.
Each output file holds, per instance, the generator arguments and the sorted
solution masks as hexadecimal strings (little-endian 64-bit words).
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import msp_instances as mi  # noqa: E402
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

SEED_4_30 = 1
SEED_BATCH_6_50 = 1000
SEED_7_60 = 7
SEED_8_70 = 8
SEED_9_80 = 9080
SEED_10_90 = 1090


def entry(m, n, seed, planted, h, slices=None):
    A, d, _ = mi.generate(m, n, seed, planted=planted, h=h)
    t0 = time.time()
    sols = oracle.mitm(A, d, slices=slices)
    dt = time.time() - t0
    print(f"  ({m},{n}) seed={seed} planted={planted}: {len(sols)} solutions, {dt:.1f}s", flush=True)
    return {"m": m, "n": n, "seed": seed, "planted": planted, "h": h,
            "solutions": [[f"{w:016x}" for w in s] for s in sols]}


def entry_fourlist(m, n, seed, planted, h, chunks, state_path):
    """Every solution by the four-list oracle, run over ``chunks`` equal
    slice ranges; finished ranges are kept in ``state_path``."""
    A, d, _ = mi.generate(m, n, seed, planted=planted, h=h)
    t0 = time.time()
    sols = _fourlist_chunks(A, d, chunks, state_path, f"{m}_{n}_{seed}_{int(planted)}")
    print(f"  ({m},{n}) seed={seed} planted={planted}: {len(sols)} solutions, "
          f"{time.time() - t0:.1f}s this run", flush=True)
    return {"m": m, "n": n, "seed": seed, "planted": planted, "h": h,
            "slicing": list(oracle.default_slicing(m, n)),
            "records": [1 << (n // 2), 1 << (n - n // 2)], "solutions": sols}


def entry_10_70_subcube(state_path):
    """A planted (10,90) instance with 20 seeded columns fixed to x*: the
    (10,70) restriction, solved in full by the four-list oracle."""
    import numpy as np
    A, d, x = mi.generate(10, 90, SEED_10_90, planted=True, h=45)
    rng = np.random.default_rng(SEED_10_90)
    cols = sorted(int(c) for c in rng.choice(90, 20, replace=False))
    vals = [int(x[c]) for c in cols]
    A2, d2, free = mi.restrict(A, d, cols, vals)
    sols = _fourlist_chunks(A2, d2.astype(np.int32), 8, state_path, f"10_70_sub_{SEED_10_90}")
    return {"m": 10, "n": 90, "seed": SEED_10_90, "planted": True, "h": 45,
            "fixed_cols": cols, "fixed_vals": vals, "solutions_restricted": sols}


def _fourlist_chunks(A, d, chunks, state_path, key):
    """The four-list oracle over ``chunks`` equal slice ranges of the default
    slicing; finished ranges are kept in ``state_path`` (resumable).  The
    ranges must have covered every left and right subset exactly once."""
    m, n = A.shape
    mods = oracle.default_slicing(m, n)
    S = 1
    for P in mods:
        S *= P
    key = f"{key}_{'x'.join(map(str, mods))}"
    state = {}
    if state_path and os.path.exists(state_path):
        state = json.load(open(state_path))
    done = state.setdefault(key, {})
    for c in range(chunks):
        a, b = S * c // chunks, S * (c + 1) // chunks
        if f"{a}-{b}" in done:
            continue
        tc = time.time()
        sols, rl, rr = oracle.fourlist(A, d, mods=mods, slice_range=(a, b), return_records=True)
        done[f"{a}-{b}"] = {"range": [a, b], "left": rl, "right": rr,
                            "solutions": [[f"{w:016x}" for w in s] for s in sols]}
        if state_path:
            tmp = state_path + ".tmp"
            json.dump(state, open(tmp, "w"))
            os.replace(tmp, state_path)
        print(f"  {key} chunk {c + 1}/{chunks}: {len(sols)} solutions, {time.time() - tc:.1f}s", flush=True)
    ranges = [S * c // chunks for c in range(chunks + 1)]
    use = [done[f"{a}-{b}"] for a, b in zip(ranges[:-1], ranges[1:])]
    rl = sum(v["left"] for v in use)
    rr = sum(v["right"] for v in use)
    assert rl == 1 << (n // 2) and rr == 1 << (n - n // 2), (rl, rr)
    sols = sorted({tuple(s) for v in use for s in v["solutions"]},
                  key=lambda t: tuple(int(w, 16) for w in reversed(t)))
    return [list(s) for s in sols]


def entries_7_60_with_solutions(count, first_seed):
    """The first ``count`` plain (7,60) instances from seed ``first_seed`` on
    whose solution set (by the four-list oracle) is not empty."""
    out, seed = [], first_seed
    while len(out) < count:
        A, d, _ = mi.generate(7, 60, seed)
        sols = oracle.fourlist(A, d)
        print(f"  (7,60) seed={seed}: {len(sols)} solutions", flush=True)
        if sols:
            out.append({"m": 7, "n": 60, "seed": seed, "planted": False, "h": None,
                        "solutions": [[f"{w:016x}" for w in s] for s in sols]})
        seed += 1
    return out


def write(name, entries, oracle_name="oracle.mitm"):
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        json.dump({"generator": "msp_instances.generate", "oracle": oracle_name,
                   "instances": entries}, f, indent=0)
    print("wrote", path)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--big", action="store_true")
    ap.add_argument("--only", default=None)
    ap.add_argument("--state", default=None, help="progress file of the four-list runs")
    args = ap.parse_args()
    if args.only in (None, "4_30"):
        write("sols_4_30.json", [entry(4, 30, SEED_4_30, False, None),
                                 entry(4, 30, SEED_4_30, True, 15)])
    if args.only in (None, "6_50"):
        write("sols_6_50_batch.json",
              [entry(6, 50, SEED_BATCH_6_50 + k, k >= 32, 25 if k >= 32 else None) for k in range(64)])
    if args.big or args.only == "7_60":
        write("sols_7_60.json", [entry(7, 60, SEED_7_60, False, None, slices=16)])
    if args.big or args.only == "7_60_planted":
        write("sols_7_60_planted.json", [entry(7, 60, SEED_7_60, True, 30, slices=16)])
    if args.only == "8_70":
        state = args.state or os.path.join(HERE, "sols_8_70.state.json")
        write("sols_8_70.json", [entry_fourlist(8, 70, SEED_8_70, False, None, 8, state),
                                 entry_fourlist(8, 70, SEED_8_70, True, 35, 8, state)],
              "oracle.fourlist")
    if args.only == "10_70_sub":
        state = args.state or os.path.join(HERE, "sols_10_70.state.json")
        write("sols_10_70_subcube.json", [entry_10_70_subcube(state)], "oracle.fourlist")
    if args.only == "7_60_more":
        write("sols_7_60_more.json", entries_7_60_with_solutions(3, 70), "oracle.fourlist")
    if args.only == "9_80_planted":
        state = args.state or os.path.join(HERE, "sols_9_80_planted.state.json")
        write("sols_9_80_planted.json", [entry_fourlist(9, 80, 9, True, 40, 16, state)], "oracle.fourlist")
    if args.only == "9_80":
        state = args.state or os.path.join(HERE, "sols_9_80.state.json")
        write("sols_9_80.json", [entry_fourlist(9, 80, SEED_9_80, False, None, 16, state)],
              "oracle.fourlist")


if __name__ == "__main__":
    main()
