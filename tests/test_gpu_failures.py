"""Failure handling of the library on the GPU, through the C ABI.

Every failure here is made on the host or by a bounded wait that is made to
run out; nothing faults, traps or hangs the device.  After each failure the
library and the device must stay usable: the next solve returns the oracle's
solution set.
"""
import json
import os
import time

import numpy as np
import pytest

import msp_instances as mi
import oracle

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ETIMEDOUT, ECANCELED, ENOMEM = -5, -7, -3


@pytest.fixture(scope="module")
def msp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_05045_gb300 import build
    build.build()
    import paper_2507_05045_gb300 as m
    return m


def golden_8_70_plain():
    g = json.load(open(os.path.join(GOLDEN, "sols_8_70.json")))
    e = [e for e in g["instances"] if not e["planted"]][0]
    A, d, _ = mi.generate(e["m"], e["n"], e["seed"])
    return A, d, [tuple(int(w, 16) for w in s) for s in e["solutions"]]


def wait_result(srv, rid, limit_s=120.0):
    t0 = time.time()
    while time.time() - t0 < limit_s:
        r = srv.poll(rid)
        if r is not None:
            return r
        time.sleep(0.002)
    raise AssertionError("request did not finish in time")


def test_bounded_wait_runs_out_and_the_device_stays_usable(msp):
    # the streaming join's blocks wait on a phase that no copy completes:
    # every wait gives up after its 1 ms limit and the solve reports it
    A, d, _ = mi.generate(6, 50, 4321, planted=True, h=25)
    t0 = time.time()
    with msp.Instance(A, d, plan={"direct": 0}, wait_limit_us=1000, wait_check=True) as inst:
        with pytest.raises(msp.MspError) as e:
            inst.solve_all()
    assert e.value.code == ETIMEDOUT
    assert time.time() - t0 < 30
    # the same instance without the check, and with a short but sufficient
    # limit, is solved exactly
    want = oracle.mitm(A, d)
    with msp.Instance(A, d, plan={"direct": 0}, wait_limit_us=200_000) as inst:
        assert inst.solve_all() == want
    assert msp.solve_all(A, d) == want


def test_wait_options_are_validated(msp):
    A, d, _ = mi.generate(4, 30, 1)
    for kw in ({"wait_limit_us": 0}, {"wait_limit_us": 60_000_001}):
        with pytest.raises(msp.MspError) as e:
            msp.Instance(A, d, **kw)
        assert e.value.code == -2


def test_instance_budget_too_small(msp):
    A, d, _ = golden_8_70_plain()
    with msp.Instance(A, d, memory_budget=1 << 20) as inst:
        with pytest.raises(msp.MspError) as e:
            inst.solve_all()
    assert e.value.code == ENOMEM
    # a later solve with the default budget is exact
    A, d, want = golden_8_70_plain()
    assert msp.solve_all(A, d) == want


def test_server_rejects_a_request_beyond_its_budget(msp):
    # 170 MB: a (4,30) request needs about 160 MB (direct pass, with the
    # match list and margin), an (8,70) one at least the streaming pass's
    # 140 MB of reserves plus 38 MB of quarter lists
    A, d, _ = golden_8_70_plain()
    assert msp.plan_info(4, 30)["device_bytes"] <= 170 << 20
    with msp.Server(hbm_budget=170 << 20, max_inflight=1) as srv:
        with pytest.raises(msp.MspError) as e:
            srv.submit(A, d)
        assert e.value.code == ENOMEM
        # a small request still fits and is served exactly
        A2, d2, _ = mi.generate(4, 30, 1, planted=True, h=15)
        rid = srv.submit(A2, d2)
        assert wait_result(srv, rid) == oracle.mitm(A2, d2)


def test_server_cancels_a_queued_request(msp):
    # one worker: the (8,70) request runs, the small one waits behind it and
    # is canceled before it starts; the running one is unaffected
    A, d, want = golden_8_70_plain()
    A2, d2, _ = mi.generate(4, 30, 1, planted=True, h=15)
    with msp.Server(max_inflight=1) as srv:
        big = srv.submit(A, d)
        small = srv.submit(A2, d2)
        srv.cancel(small)
        with pytest.raises(msp.MspError) as e:
            wait_result(srv, small)
        assert e.value.code == ECANCELED
        assert wait_result(srv, big) == want
        # the server keeps serving after the cancellation
        again = srv.submit(A2, d2)
        assert wait_result(srv, again) == oracle.mitm(A2, d2)


def test_server_cancels_a_running_request_between_launches(msp):
    # a (9,80) request (512 join launches of about 15 ms) is canceled while it
    # runs: it stops at the next launch boundary, far before its 8 s
    A, d, _ = mi.generate(9, 80, 9080)
    with msp.Server(max_inflight=1) as srv:
        rid = srv.submit(A, d)
        time.sleep(1.0)
        t0 = time.time()
        srv.cancel(rid)
        with pytest.raises(msp.MspError) as e:
            wait_result(srv, rid, limit_s=60)
        assert e.value.code == ECANCELED
        assert time.time() - t0 < 3.0
        A2, d2, _ = mi.generate(5, 40, 7001, planted=True, h=20)
        rid2 = srv.submit(A2, d2)
        assert wait_result(srv, rid2) == oracle.mitm(A2, d2)


def test_cancel_and_poll_of_unknown_requests(msp):
    with msp.Server(max_inflight=1) as srv:
        with pytest.raises(msp.MspError) as e:
            srv.cancel(12345)
        assert e.value.code == -1
        with pytest.raises(msp.MspError) as e:
            srv.poll(12345)
        assert e.value.code == -1
