"""Class sharding of one solve across ranks, on the CPU (gloo, world size 2).

Every run of this pool has one GPU, so the multi-rank path is tested here:
each rank "solves" its class pieces with a stub that returns the matching
slices of the four-list oracle (its own partition of the solution set), and
the gather and merge must give the full oracle set on every rank.  The GPU
form of a piece (an msp.Instance solve of class part k of P) is tested
against the oracle in tests/test_gpu_parity.py.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def stub_solver(A, d, mods):
    import oracle
    S = int(np.prod(mods))

    def solve_part(k, parts):
        return oracle.fourlist(A, d, mods=mods, slice_range=(S * k // parts, S * (k + 1) // parts))
    return solve_part


def _rank_main(rank, world, port, out_dir, parts):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import msp_instances as mi
    from paper_2507_05045_gb300 import shard
    dist.init_process_group("gloo")
    A, d, _ = mi.generate(3, 22, 77, K=4, planted=True, h=11)
    res = shard.solve_sharded(A, d, rank, world, parts=parts, pg=dist,
                              solve_part=stub_solver(A, d, (4, 3, 2)))
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"solutions": res["solutions"], "mine": res["mine"], "parts": res["parts"]}, f)
    dist.destroy_process_group()


@pytest.mark.parametrize("parts", [2, 5])
def test_sharded_solve_gathers_the_full_set_world2(tmp_path, parts):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import msp_instances as mi
    import oracle
    mp.start_processes(_rank_main, args=(2, free_port(), str(tmp_path), parts), nprocs=2,
                       start_method="spawn")
    A, d, _ = mi.generate(3, 22, 77, K=4, planted=True, h=11)
    want = [list(s) for s in oracle.brute(A, d)]
    assert len(want) > 10
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for g in got:
        assert g["solutions"] == want  # every rank holds the full sorted set
    assert got[0]["parts"] == list(range(0, parts, 2))
    assert got[1]["parts"] == list(range(1, parts, 2))
    # the ranks' own sets are disjoint and together make the full set
    assert not {tuple(s) for s in got[0]["mine"]} & {tuple(s) for s in got[1]["mine"]}
    assert sorted(got[0]["mine"] + got[1]["mine"]) == want


def test_merge_rejects_a_solution_reported_twice():
    from paper_2507_05045_gb300 import shard
    assert shard.merge([[(3,), (1,)], [(2,)]]) == [(1,), (2,), (3,)]
    assert shard.merge([[(1, 2), (5, 1)], [(0, 2)]]) == [(5, 1), (0, 2), (1, 2)]
    with pytest.raises(RuntimeError):
        shard.merge([[(1,)], [(1,)]])


def test_parts_of_each_rank():
    from paper_2507_05045_gb300 import shard
    assert shard.my_parts(0, 2, 5) == [0, 2, 4]
    assert shard.my_parts(1, 2, 5) == [1, 3]
    assert shard.my_parts(3, 4, 2) == []
    with pytest.raises(ValueError):
        shard.my_parts(2, 2, 4)
