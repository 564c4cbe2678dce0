"""The MSP_CHECKED build of libmsp on the small parity cases.

libmsp_checked.so tests every data-dependent index of the direct pass's and
the streaming pass's kernels before the access (csrc/checked.cuh); a failed
check skips the access and fails the solve with MSP_ECUDA.  Here the checked
library solves small seeded instances on both passes and must return the
oracle's solution sets with no check failing.  It runs in a child process,
since a process loads one libmsp.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, ROOT)
import numpy as np
import msp_instances as mi
import oracle
from paper_2507_05045_gb300 import build, msp
lib = msp.load_library(build.build(checked=True))
assert b"MSP_CHECKED" in lib.msp_version()
cases = []
for seed in range(12):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 9)); n = int(rng.integers(8, 23))
    K = int(rng.choice([2, 3, 20, 100]))
    cases.append(mi.generate(m, n, 40000 + seed, K=K, planted=bool(seed % 2), h=n // 2)[:2])
cases += [mi.generate(4, 30, 1, planted=True, h=15)[:2], mi.generate(5, 40, 7001, planted=True, h=20)[:2],
          mi.generate(6, 50, 1001)[:2]]
done = 0
for A, d in cases:
    n = A.shape[1]
    want = oracle.brute(A, d) if n <= 22 else oracle.mitm(A, d)
    for plan in ({"direct": 1}, {"direct": 0}):
        got = msp.solve_all(A, d, plan=plan)
        assert got == want, (A.shape, plan)
        done += 1
print(json.dumps({"solves": done}))
""".replace("ROOT", repr(ROOT))


def test_checked_build_small_parity_cases():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "-c", CHILD], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, (r.stdout + r.stderr)[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["solves"] == 30
