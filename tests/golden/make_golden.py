"""Write the stored solution sets of the benchmark-shaped instances.

Calls only the CPU oracle (``oracle/``) and the instance generator
(``msp_instances``); nothing here touches the CUDA path.  Run from the
repository root:

    python tests/golden/make_golden.py [--big]

``--big`` also writes the (7,60) instance, which takes minutes of CPU.
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


def entry(m, n, seed, planted, h, slices=None):
    A, d, _ = mi.generate(m, n, seed, planted=planted, h=h)
    t0 = time.time()
    sols = oracle.mitm(A, d, slices=slices)
    dt = time.time() - t0
    print(f"  ({m},{n}) seed={seed} planted={planted}: {len(sols)} solutions, {dt:.1f}s", flush=True)
    return {"m": m, "n": n, "seed": seed, "planted": planted, "h": h,
            "solutions": [[f"{w:016x}" for w in s] for s in sols]}


def write(name, entries):
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        json.dump({"generator": "msp_instances.generate", "oracle": "oracle.mitm",
                   "instances": entries}, f, indent=0)
    print("wrote", path)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--big", action="store_true")
    ap.add_argument("--only", default=None)
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


if __name__ == "__main__":
    main()
