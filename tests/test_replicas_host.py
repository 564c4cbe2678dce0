"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

Every run of this pool has one GPU, so bench.py --gpus N runs N independent
replicas: residue classes and instances need no exchange, and the ranks only
meet in a barrier and in max / sum reductions of their timings and counts.
These tests run that logic with the gloo backend on the CPU.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    w, r, local, pg = bench.dist_init(None)
    assert (w, r) == (world, rank) and pg is not None and pg.get_backend() == "gloo"
    bench.barrier(pg)
    mx = bench.allreduce_max(pg, 10.0 * (rank + 1))
    sm = bench.allreduce_sum(pg, float(rank + 1))
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"max": mx, "sum": sm}, f)
    pg.destroy_process_group()


def test_barrier_and_reductions_world2(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    for rank in range(2):
        got = json.load(open(tmp_path / f"rank{rank}.json"))
        # the slowest rank's time and the units of all ranks
        assert got == {"max": 20.0, "sum": 3.0}


def test_reference_arm_under_torchrun_prints_one_line():
    pytest.importorskip("torch")
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--rows", "4", "--cols", "48", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1  # rank 0 alone runs and prints
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2
    assert out["value"] > 0 and out["cpu_baseline"]["kind"] == "oracle"
    assert out["e2e"]["h2d_bytes_per_step"] == 0
