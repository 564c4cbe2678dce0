"""Benchmark: exhaustive solve of one (9,80) market split instance.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

One step = one exhaustive solve (every solution of A x = d) of a seeded
plain (9,80) instance: a_ij uniform in [0,99], d_i = floor(row sum / 2).
The headline value is row-1 candidate pairs per second, C1 / step time,
where C1 = #{(l, r) : row1(l) + row1(r) = d_1} is the number of row-1
candidate pairs of Algorithm 2 that the solve rules on (an exact count from
the library's counters, independent of the implementation); the step time
is also the time-to-all-solutions (ms_per_step).

With N > 1 (torchrun) every rank solves its own instance (seed + rank): the
units are independent, so there is no data-path collective ("weak"
scaling); value = candidate pairs of all ranks / the slowest rank's time.

The default run (rank 0, one GPU) then adds a ``secondary`` block with short
runs of the other configurations (``--no-secondary`` skips it): the (10,90)
1/64 part with its projected full time, the served mixed stream against
sequential solving (p50/p99, 256 requests at the sequential service rate),
the batch of 64 (6,50) instances, time to the first solution over four
planted (9,80) instances and the (11,100,50) 1/4096 part.

``--impl reference`` times the CPU oracle (the four-list meet in the middle
over residue slices) on a bounded sample of the same instance: its lists are
built in full and 1/2048 of its slices joined, and the time to all solutions
is projected by the records enumerated; the rate is C1 / that time, in the
same unit.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import msp_instances as mi  # noqa: E402

METRIC = "time-to-all-solutions & candidate pairs/s at (9,80); p50/p99 latency, mixed stream"
UNIT = "candidate pairs/s"
M_, N_ = 9, 80
SEED = 9080
SAMPLE_DIV = 2048  # the CPU oracle's timed sample: 1/2048 of the residue slices


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    # --rows / --cols (--m / --n also work when bench.py is run directly;
    # torch.distributed.run would read those two as abbreviations of its own)
    ap.add_argument("--rows", "--m", dest="m", type=int, default=M_)
    ap.add_argument("--cols", "--n", dest="n", type=int, default=N_)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="default workload: skip the short runs of the other configurations")
    ap.add_argument("--config", choices=["9_80", "batch_6_50", "serving", "10_90_part", "profile_part",
                                         "profile_small", "first_9_80", "k_sweep", "first_10_90",
                                         "11_100_part"],
                    default="9_80",
                    help="9_80 (default): the headline exhaustive solve; batch_6_50: 64 (6,50) "
                         "instances in one batched call vs one at a time; serving: the mixed Poisson "
                         "request stream through the server vs sequential solving; 10_90_part: one "
                         "seeded 1/64 of the residue classes of a (10,90) instance; profile_part: "
                         "the case the ncu traffic captures use (the (9,80) instance of the default "
                         "workload over 1/4096 of its residue classes, one solve); profile_small: one "
                         "direct-pass solve of a (7,60) instance (lists of 8 MB), the case of the "
                         "full-section captures; first_9_80: time to the first solution (the "
                         "quantity of the paper's tables) of the plain bench instance and of a "
                         "planted (9,80) instances; k_sweep: plain (8,70) and (9,80) instances with "
                         "a_ij in [0, K) for K = 50, 100, 200 (the paper's (m, n, K) classes); "
                         "first_10_90: time to the first solution of a planted (10,90) instance on the "
                         "streaming pass; 11_100_part: one seeded 1/4096 of the residue classes of a plain "
                         "(11,100) instance with a_ij in [0,49] (the paper's (11,100,50) class)")
    ap.add_argument("--path", type=int, default=1, choices=[0, 1],
                    help="profile_part: 1 = direct pass, 0 = streaming pass")
    ap.add_argument("--requests", type=int, default=512)
    ap.add_argument("--instances", type=int, default=4,
                    help="first_9_80 / first_10_90: planted instances to average")
    ap.add_argument("--rate-factor", type=float, default=0.8)
    return ap.parse_args()


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def allreduce_max(pg, x: float) -> float:
    if pg is None:
        return x
    import torch
    dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(pg, x: float) -> float:
    if pg is None:
        return x
    import torch
    dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def oracle_sample(A, d, div=SAMPLE_DIV, seed=SEED):
    """The four-list CPU oracle on the whole instance, timed over the first
    1/div of its residue slices (its inner lists are built in full), with
    the time of every slice projected from the records it enumerated:
    projected = build + join x (all records / records enumerated)."""
    import oracle
    oracle.build()
    m, n = np.asarray(A).shape
    mods = oracle.default_slicing(m, n)
    S = int(np.prod(mods))
    hi = max(1, S // div)
    tm = {}
    t0 = time.perf_counter()
    sols, rl, rr = oracle.fourlist(A, d, mods=mods, slice_range=(0, hi), return_records=True, timing=tm)
    wall = time.perf_counter() - t0
    total = (1 << (n // 2)) + (1 << (n - n // 2))
    done = max(1, rl + rr)
    projected = tm["build"] + tm["join"] * total / done
    cores = os.cpu_count() or 1
    sample = (f"the ({m},{n}) instance of seed {seed} itself: four-list CPU oracle (OpenMP, {cores} threads) "
              f"with its inner lists built in full ({tm['build']:.2f} s) and residue slices [0, {hi}) of "
              f"{S} joined ({tm['join']:.2f} s, {done} of {total} half-subset records, {len(sols)} "
              f"solutions there); time to all solutions projected by records: {projected:.0f} s")
    return {"projected_s": projected, "wall_s": wall, "build_s": tm["build"], "join_s": tm["join"],
            "records": done, "records_total": total, "slices": [0, hi, S], "cores": cores,
            "sample": sample, "solutions_in_sample": len(sols)}


def run_cpu_baseline(A, d, cand):
    """cpu_baseline of the bench line: the oracle's projected time to all
    solutions of the same instance, as candidate pairs per second."""
    o = oracle_sample(A, d)
    return {"value": cand / o["projected_s"], "unit": UNIT, "cores": o["cores"], "kind": "oracle",
            "sample": o["sample"], "projected_s": o["projected_s"], "seconds": o["wall_s"]}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, path, gpu_index):
        self.path = path
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            return summarize_clocks(f)


def summarize_clocks(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen in
    nvidia-smi CSV rows of ClockSampler.FIELDS (no header, no units); None
    without a parsable row."""
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            rows.append((float(parts[1]), float(parts[2]), parts[3], parts[5:9]))
        except ValueError:
            continue
    if not rows:
        return None
    sm = sorted(r[0] for r in rows)
    smax = max(r[1] for r in rows)
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
    return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": reasons, "samples": len(rows)}


def l2_note(st):
    """How a step's device-memory working set compares with the 129 MB L2."""
    if st.get("path") == "direct":
        q = st["quarter"]
        gb = 8.0 * ((1 << q[2]) + (1 << q[3])) / 1e9
        return (f"inputs larger than L2: the direct pass reads bucketed inner quarter lists of {gb:.1f} GB "
                f"(32-bit keys plus subset masks) every step; no per-record buffer")
    return ("inputs larger than L2: every step streams ~16 B per half-pair record through HBM pass "
            "buffers of tens of GB")


def _capture(kernel):
    """The committed ncu figures of a kernel, or None when its source changed
    since they were taken."""
    import hashlib
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        k = t["kernels"][kernel]
        src = open(os.path.join(ROOT, k["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest() != k["source_sha256"]:
            return None
        return k
    except Exception:
        return None


def traffic_per_launch(kernel, alg_bytes_per_launch):
    """DRAM bytes per launch from the committed ncu capture, scaled by the
    algorithmic bytes of a launch; None when the kernel source changed since."""
    k = _capture(kernel)
    if k is None:
        return None
    return alg_bytes_per_launch * k["dram_bytes"] / k["algorithmic_bytes"]


def native(args, world, rank, local, pg):
    import torch
    from paper_2507_05045_gb300 import build
    build.build()
    import paper_2507_05045_gb300 as msp

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    A, d, _ = mi.generate(args.m, args.n, SEED + rank)

    inst = msp.Instance(A, d, stream=stream.cuda_stream, profiling=True)
    for _ in range(args.warmup):
        inst.solve_all()
    st0 = inst.stats()
    cand = st0["row1_candidates"]

    # raw clock samples: $MSP_BENCH_OUT (default: the temporary directory)
    out_dir = os.environ.get("MSP_BENCH_OUT") or tempfile.gettempdir()
    os.makedirs(out_dir, exist_ok=True)
    clk = ClockSampler(os.path.join(out_dir, f"clocks_rank{rank}.csv"), local)
    clk.start()
    kern = {}
    launches = 0
    barrier(pg)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev0.record(stream)
    step_ev[0].record(stream)
    sols = None
    for i in range(args.steps):
        sols = inst.solve_all()
        step_ev[i + 1].record(stream)
        st = inst.stats()
        launches += st["kernel_launches"]
        for k, v in st["kernels"].items():
            a = kern.setdefault(k, {"ms": 0.0, "launches": 0, "bytes": 0})
            a["ms"] += v["ms"]
            a["launches"] += v["launches"]
            a["bytes"] += v["bytes"]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    step_ms = [step_ev[i].elapsed_time(step_ev[i + 1]) for i in range(args.steps)]
    ms_max = allreduce_max(pg, ms)
    cand_all = allreduce_sum(pg, float(cand))
    value = cand_all / (ms_max / 1000.0)

    # end to end through the public API: host buffers in, solutions out
    e2e_ms = []
    h2d = d2h = 0
    for _ in range(min(args.steps, 3)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with msp.Instance(A, d) as e_inst:
            e_sols = e_inst.solve_all()
            est = e_inst.stats()
        e2e_ms.append((time.perf_counter() - t0) * 1000.0)
        h2d = est["h2d_bytes"] + A.nbytes + d.nbytes
        d2h = est["d2h_bytes"]
        assert e_sols == sols
    e2e_ms_max = allreduce_max(pg, float(np.mean(e2e_ms)))
    inst.close()

    # dominant kernel and its roofline
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    dom = max(kern.items(), key=lambda kv: kv[1]["ms"]) if kern else (None, None)
    byte_kernels = {k: v for k, v in kern.items() if v["bytes"]}
    roof = None
    if dom[0] is not None:
        name, v = dom
        if v["bytes"]:
            achieved = v["bytes"] / (v["ms"] / 1000.0) / 1e9
            roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": None, "peak_source": peak_src,
                    "bytes_per_launch": v["bytes"] / max(1, v["launches"]),
                    "ms_per_launch": v["ms"] / max(1, v["launches"])}
        else:
            roof = {"bound": "alu", "kernel": name, "achieved": None, "peak": None, "unit": "GB/s",
                    "frac": None, "traffic": None, "peak_source": peak_src}
    if roof is not None and roof.get("bound") == "hbm":
        roof["traffic"] = traffic_per_launch(roof["kernel"], roof["bytes_per_launch"])
        # the HBM fraction is low by design (no record reaches device memory):
        # the on-chip limits of the same kernel source, from ncu
        # the join's own rate: every half-pair record of a step joined in its time
        if roof["kernel"] == "direct" and dom[1]["ms"] > 0:
            recs = (st0["records_left"] + st0["records_right"]) * args.steps
            roof["records_per_s"] = recs / (dom[1]["ms"] / 1000.0)
        cap = _capture(roof["kernel"])
        if cap is not None and "onchip" in cap:
            roof["onchip"] = dict(cap["onchip"], source="ncu, profiles/" + cap["onchip"]["case"])
            roof["onchip"].pop("case")
    for k, v in byte_kernels.items():
        v["achieved_gbs"] = v["bytes"] / (v["ms"] / 1000.0) / 1e9
        v["frac_of_measured_hbm"] = v["achieved_gbs"] / hbm_peak

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"({args.m},{args.n}) plain instance, exhaustive (all solutions)",
                   "m": args.m, "n": args.n, "seed": SEED, "a_range": "[0,99]",
                   "rhs": "d_i = floor(row sum / 2)", "parallelism": f"replicas x{world}",
                   "l2": l2_note(st0)},
        "time_to_all_solutions_s": ms_max / 1000.0,
        # every timed step of this rank, and time x median SM clock (comparable across boxes
        # that ran at different clocks)
        "step_ms": {"all": step_ms, "median": float(np.median(step_ms)), "min": min(step_ms),
                    "max": max(step_ms)},
        "ms_x_sm_mhz": (ms * clocks["sm_mhz"]) if clocks else None,
        "row1_candidates_per_rank": cand,
        "solutions": len(sols) if sols is not None else None,
        "records_per_side": [st0["records_left"], st0["records_right"]],
        "passes": st0["passes"],
        "kernels": kern,
        "roofline": roof,
        "e2e": {"value": cand_all / (e2e_ms_max / 1000.0), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms_max},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_secondary:
        out["secondary"] = secondary(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = run_cpu_baseline(A, d, cand)
        out["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "projected_s")}
    if rank == 0:
        print(json.dumps(out), flush=True)


def reference(args, world, rank, pg):
    """The reference arm: the CPU oracle on the same instance, each step a
    bounded sample of its residue slices projected to the whole solve."""
    if rank != 0:
        return
    import oracle
    A, d, _ = mi.generate(args.m, args.n, SEED)
    cand = oracle.row1_candidates(A, d)
    for _ in range(args.warmup):
        oracle_sample(A, d)
    proj, walls, o = [], [], None
    for _ in range(args.steps):
        o = oracle_sample(A, d)
        proj.append(o["projected_s"])
        walls.append(o["wall_s"])
    t = float(np.mean(proj))
    value = cand / t
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1000.0, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "i32", "data": "synthetic",
           "config": {"workload": f"({args.m},{args.n}) plain instance, exhaustive (all solutions)",
                      "m": args.m, "n": args.n, "seed": SEED, "oracle_slices_timed": o["slices"]},
           "time_to_all_solutions_s": t, "sample_wall_s_per_step": float(np.mean(walls)),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": o["cores"], "kind": "oracle",
                            "sample": o["sample"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# Secondary workloads (rank 0, one GPU): batched, served, (10,90) part.
# ---------------------------------------------------------------------------
def _emit(obj):
    print(json.dumps(obj), flush=True)


def _done(emit, obj):
    if emit:
        _emit(obj)
    return obj


def bench_batch(args, emit=True):
    import paper_2507_05045_gb300 as msp
    from paper_2507_05045_gb300 import build
    build.build()
    insts = mi.batch(6, 50, 64, 1000, h=25)
    pairs = [(A, d) for A, d, _ in insts]
    for _ in range(args.warmup):
        msp.solve_batch(pairs)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rb = msp.solve_batch(pairs)
    tb = (time.perf_counter() - t0) / args.steps
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rs = [msp.solve_all(A, d) for A, d in pairs]
    ts = (time.perf_counter() - t0) / args.steps
    assert rb == rs
    # the streaming pass's batch (one scatter and one join launch per pass)
    msp.solve_batch(pairs, path=0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rst = msp.solve_batch(pairs, path=0)
    tst = (time.perf_counter() - t0) / args.steps
    assert rst == rb
    h2d = sum(A.nbytes + d.nbytes for A, d in pairs)
    d2h = sum(len(r) * 8 for r in rb)
    return _done(emit, {"metric": "instances/s, 64 (6,50) instances per batched call", "value": 64 / tb,
           "unit": "instances/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": tb * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "u64", "data": "synthetic",
           "config": {"workload": "64 (6,50) instances, seeds 1000..1063, 32 plain + 32 planted (25 ones)",
                      "path": "direct pass: every instance's lists, one join launch over the 4096 classes "
                              "of all 64 instances, one verification launch"},
           "sequential": {"value": 64 / ts, "unit": "instances/s", "ms_per_step": ts * 1e3},
           "streaming_batch": {"value": 64 / tst, "unit": "instances/s", "ms_per_step": tst * 1e3},
           "speedup_vs_sequential": ts / tb,
           "e2e": {"value": 64 / tb, "unit": "instances/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h}})


SERVE_SHAPES = [(4, 30), (5, 40), (6, 50), (7, 60), (8, 70)]


def serving_trace(nreq, seed=4242):
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(nreq):
        m, n = SERVE_SHAPES[int(rng.integers(0, len(SERVE_SHAPES)))]
        planted = bool(rng.integers(0, 2))
        A, d, _ = mi.generate(m, n, 50000 + k, planted=planted, h=n // 2)
        reqs.append((A, d))
    gaps = rng.exponential(1.0, size=nreq)  # scaled by 1/lambda later
    return reqs, gaps


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(round(q / 100.0 * (len(xs) - 1))))]


def bench_serving(args, emit=True):
    import threading
    import paper_2507_05045_gb300 as msp
    from paper_2507_05045_gb300 import build
    build.build()
    reqs, gaps = serving_trace(args.requests)
    # sequential service rate of the mix, measured on one solve per shape
    svc = []
    for (m, n) in SERVE_SHAPES:
        A, d, _ = mi.generate(m, n, 7)
        msp.solve_all(A, d)
        t0 = time.perf_counter()
        msp.solve_all(A, d)
        svc.append(time.perf_counter() - t0)
    mean_svc = float(np.mean(svc))
    lam = args.rate_factor / mean_svc
    arrivals = np.cumsum(gaps / lam)

    def run_sequential():
        lat, t_start = [], time.perf_counter()
        clock = 0.0
        results = []
        for (A, d), at in zip(reqs, arrivals):
            now = time.perf_counter() - t_start
            if now < at:
                time.sleep(at - now)
            results.append(msp.solve_all(A, d))
            lat.append(time.perf_counter() - t_start - at)
        return lat, time.perf_counter() - t_start, results

    def run_served():
        srv = msp.Server(max_inflight=4)
        ids = [None] * len(reqs)
        done_at = [None] * len(reqs)
        results = [None] * len(reqs)
        t_start = time.perf_counter()
        sub_done = threading.Event()

        def submitter():
            for k, ((A, d), at) in enumerate(zip(reqs, arrivals)):
                now = time.perf_counter() - t_start
                if now < at:
                    time.sleep(at - now)
                ids[k] = srv.submit(A, d)
            sub_done.set()

        th = threading.Thread(target=submitter)
        th.start()
        pending = set()
        nxt = 0
        while True:
            while nxt < len(reqs) and ids[nxt] is not None:
                pending.add(nxt)
                nxt += 1
            for k in list(pending):
                r = srv.poll(ids[k])
                if r is not None:
                    results[k] = r
                    done_at[k] = time.perf_counter() - t_start
                    pending.discard(k)
            if sub_done.is_set() and nxt == len(reqs) and not pending:
                break
            time.sleep(0.0005)
        th.join()
        srv.close()
        lat = [done_at[k] - arrivals[k] for k in range(len(reqs))]
        return lat, time.perf_counter() - t_start, results

    lat_s, span_s, res_s = run_served()
    lat_q, span_q, res_q = run_sequential()
    same = res_s == res_q
    out = {"metric": "p50/p99 latency, mixed stream (time from arrival to all solutions)",
           "value": len(reqs) / span_s, "unit": "requests/s", "n_gpus": 1, "steps": 1, "warmup": 0,
           "ms_per_step": span_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "u64", "data": "synthetic",
           "config": {"workload": f"{len(reqs)} requests, Poisson arrivals at {args.rate_factor} x the "
                                  f"sequential service rate ({lam:.2f}/s), (m,n) uniform over "
                                  f"{SERVE_SHAPES}, 50% planted", "max_inflight": 4},
           "served": {"p50_ms": _pct(lat_s, 50) * 1e3, "p99_ms": _pct(lat_s, 99) * 1e3,
                      "throughput_rps": len(reqs) / span_s},
           "sequential": {"p50_ms": _pct(lat_q, 50) * 1e3, "p99_ms": _pct(lat_q, 99) * 1e3,
                          "throughput_rps": len(reqs) / span_q},
           "results_identical": same, "mean_service_s": mean_svc,
           "e2e": {"value": len(reqs) / span_s, "unit": "requests/s",
                   "h2d_bytes_per_step": int(sum(A.nbytes + d.nbytes for A, d in reqs)),
                   "d2h_bytes_per_step": int(sum(len(r) * 8 for r in res_s))}}
    return _done(emit, out)


def _bench_part(args, m, n, seed, part, K=100, emit=True):
    """One plain (m, n) instance over a fixed 1/part[1] of its residue
    classes; the full time is projected from the records joined: the list
    build once, the rest of the part's time scaled by all records / records
    joined."""
    import paper_2507_05045_gb300 as msp
    from paper_2507_05045_gb300 import build
    build.build()
    A, d, _ = mi.generate(m, n, seed, K=K)
    with msp.Instance(A, d, class_part=part, profiling=True) as inst:
        for _ in range(args.warmup):
            inst.solve_all()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            inst.solve_all()
        dt = (time.perf_counter() - t0) / args.steps
        st = inst.stats()
    total = st["records_left"] + st["records_right"]
    # the quarter lists, their class buckets and C1 are built once per solve;
    # the rest (class sizes, passes, verification) grows with the classes
    once_s = sum(st["kernels"].get(k, {}).get("ms", 0.0) for k in ("gray", "bucket", "c1")) / 1000.0
    proj = once_s + (dt - once_s) * total / st["records_done"]
    c1 = st["row1_candidates"]
    return _done(emit, {"metric": f"candidate pairs/s at ({m},{n}) over a seeded 1/{part[1]} of the residue classes "
                     "(projected full time)", "value": c1 / proj, "unit": "candidate pairs/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
           "data": "synthetic",
           "config": {"workload": f"({m},{n}) plain instance seed {seed}, a_ij in [0,{K - 1}], "
                                  f"classes part {part[0]} of {part[1]}",
                      "path": st["path"], "l2": "pass buffers of tens of GB, larger than L2"},
           "projected_full_time_s": proj, "list_build_s": once_s,
           "records_done": st["records_done"], "records_total": total,
           "classes_done": st["classes_done"], "classes_total": st["classes_total"],
           "kernels": st["kernels"]})


def bench_10_90(args, emit=True):
    # fixed, seeded choice of one 1/64 of the residue classes
    return _bench_part(args, 10, 90, 1090, (37, 64), emit=emit)


def bench_11_100(args, emit=True):
    # the paper's (11,100,50) class: coefficients in [0, 50); a fixed, seeded
    # 1/4096 of the 2^26 residue classes of the n >= 96 streaming plan
    return _bench_part(args, 11, 100, 11100, (2731, 4096), K=50, emit=emit)


def bench_profile_part(args):
    """One solve of the (9,80) bench instance over residue-class part 0 of
    4096: the case the ncu captures under profiles/ are taken on.  The
    direct pass (default) builds the full inner lists, then joins 1/4096 of
    the classes in one launch; ``--path 0`` takes the streaming pass with a
    1500 MB budget (a few passes of a few hundred MB)."""
    import paper_2507_05045_gb300 as msp
    from paper_2507_05045_gb300 import build
    build.build()
    A, d, _ = mi.generate(M_, N_, SEED)
    kw = {"plan": {"direct": 0}, "memory_budget": 1500 << 20} if args.path == 0 else {"plan": {"direct": 1}}
    with msp.Instance(A, d, class_part=(0, 4096), profiling=True, **kw) as inst:
        t0 = time.perf_counter()
        inst.solve_all()
        dt = time.perf_counter() - t0
        st = inst.stats()
    _emit({"config": {"workload": f"({M_},{N_}) plain instance seed {SEED}, classes part 0 of 4096, "
                                  f"{st['path']} pass"},
           "seconds": dt, "passes": st["passes"], "records_done": st["records_done"],
           "class_bits": st["class_bits"], "digit_bits": st["digit_bits"], "kernels": st["kernels"]})


def bench_profile_small(args):
    """One direct-pass solve of the plain (7,60) instance of seed 7: inner
    lists of 8 MB and 2^31 records, the small case the full-section ncu
    captures use."""
    import paper_2507_05045_gb300 as msp
    from paper_2507_05045_gb300 import build
    build.build()
    A, d, _ = mi.generate(7, 60, 7)
    with msp.Instance(A, d, plan={"direct": 1}, profiling=True) as inst:
        t0 = time.perf_counter()
        sols = inst.solve_all()
        dt = time.perf_counter() - t0
        st = inst.stats()
    _emit({"config": {"workload": "(7,60) plain instance seed 7, direct pass"}, "seconds": dt,
           "solutions": len(sols), "records_done": st["records_done"], "kernels": st["kernels"]})


def bench_first(args, emit=True):
    """Time to the first solution (the paper's Algorithm 2 returns the first
    x; its Table 1 times are most likely time to first), on the direct pass:
    the plain bench instance (7 solutions) and, averaged like the paper's,
    four planted ones (seeds 9..12)."""
    import paper_2507_05045_gb300 as msp
    from paper_2507_05045_gb300 import build
    build.build()
    rows = []
    insts = [("plain seed 9080", mi.generate(M_, N_, SEED))]
    insts += [(f"planted seed {s} (40 ones)", mi.generate(M_, N_, s, planted=True, h=40))
              for s in range(9, 9 + args.instances)]
    for name, (A, d, _) in insts:
        with msp.Instance(A, d, first=True) as inst:
            for _ in range(args.warmup):
                inst.solve_all()
            ts = []
            for _ in range(args.steps):
                t0 = time.perf_counter()
                sols = inst.solve_all()
                ts.append(time.perf_counter() - t0)
            st = inst.stats()
        rows.append({"instance": f"({M_},{N_}) {name}", "time_to_first_s": float(np.mean(ts)),
                     "solutions_found": len(sols), "classes_done": st["classes_done"],
                     "classes_total": st["classes_total"]})
    planted = [r["time_to_first_s"] for r in rows[1:]]
    return _done(emit, {"metric": "time to first solution at (9,80)", "value": rows[0]["time_to_first_s"], "unit": "s",
           "planted_average_s": float(np.mean(planted)) if planted else None,
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
           "dtype": "u32", "data": "synthetic",
           "config": {"workload": f"(9,80) plain seed 9080 and planted seeds 9..{8 + args.instances}, direct "
                                  "pass, stop after the first launch (about 2^32 records) that yields a "
                                  "solution"},
           "instances": rows,
           "paper": "236.07 s average over four QOBLIB (9,80,100) instances, hybrid CPU+H200 (Table 1)"})


def bench_first_10_90(args):
    """Time to the first solution at (10,90) on the streaming pass (the
    quantity of the paper's Table 1), averaged like the paper's over four
    feasible instances: the planted (10,90) instances of seeds 1090..1093
    (x* with 45 ones).  The residue passes run in class order, the matches
    are verified after every pass and the solve stops at the first pass
    that yields a solution."""
    import paper_2507_05045_gb300 as msp
    from paper_2507_05045_gb300 import build
    build.build()
    rows = []
    for seed in range(1090, 1090 + args.instances):
        A, d, _ = mi.generate(10, 90, seed, planted=True, h=45)
        with msp.Instance(A, d, first=True) as inst:
            t0 = time.perf_counter()
            sols = inst.solve_all()
            dt = time.perf_counter() - t0
            st = inst.stats()
        rows.append({"seed": seed, "time_to_first_s": dt, "solutions_found": len(sols),
                     "classes_done": st["classes_done"], "classes_total": st["classes_total"],
                     "passes": st["passes"], "path": st["path"]})
    _emit({"metric": "time to first solution at (10,90), average over planted instances", 
           "value": float(np.mean([r["time_to_first_s"] for r in rows])), "unit": "s", "n_gpus": 1,
           "steps": 1, "warmup": 0, "higher_is_better": False, "dtype": "u64", "data": "synthetic",
           "config": {"workload": f"(10,90) planted instances seeds 1090..{1089 + args.instances} (45 ones), "
                                  "a_ij in [0,99], streaming pass, stop after the first residue pass that "
                                  "yields a solution"},
           "instances": rows,
           "paper": "148 663 s average over four QOBLIB (10,90,100) instances, hybrid CPU+H200 (Table 1)"})


def bench_k_sweep(args):
    """The coefficient range K of the paper's (m, n, K) classes (Table 1):
    plain (8,70) and (9,80) instances with a_ij in [0, K) for K in
    {50, 100, 200}, each solved exhaustively on the direct pass; reports the
    time to all solutions, C1, the matched keys checked exactly and the
    solutions."""
    import paper_2507_05045_gb300 as msp
    from paper_2507_05045_gb300 import build
    build.build()
    rows = []
    for (m, n) in ((8, 70), (9, 80)):
        for K in (50, 100, 200):
            A, d, _ = mi.generate(m, n, SEED if (m, n) == (M_, N_) else 8, K=K)
            with msp.Instance(A, d, profiling=True) as inst:
                for _ in range(args.warmup):
                    inst.solve_all()
                ts = []
                for _ in range(args.steps):
                    t0 = time.perf_counter()
                    sols = inst.solve_all()
                    ts.append(time.perf_counter() - t0)
                st = inst.stats()
            rows.append({"class": f"({m},{n},{K})", "seed": SEED if (m, n) == (M_, N_) else 8,
                         "time_to_all_s": float(np.median(ts)), "row1_candidates": st["row1_candidates"],
                         "key_matches": st["key_matches"], "pairs_verified": st["pairs_verified"],
                         "solutions": len(sols), "path": st["path"], "class_bits": st["class_bits"]})
    _emit({"metric": "time to all solutions over the coefficient range K (Table 1 classes)",
           "value": rows[-2]["time_to_all_s"], "unit": "s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "higher_is_better": False, "dtype": "u32", "data": "synthetic",
           "config": {"workload": "plain (8,70) seed 8 and (9,80) seed 9080, a_ij in [0, K), K = 50, 100, 200"},
           "classes": rows})


def _with(args, **kw):
    a = argparse.Namespace(**vars(args))
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def secondary(args):
    """Short runs of the other configurations, after the headline's timed
    region (each in its own try, so that one failure leaves the line): the
    (10,90) 1/64 part and its projection, the served mixed stream against
    sequential solving (p50/p99), the batch of 64 (6,50) instances, time to
    the first solution over four planted (9,80) instances and the
    (11,100,50) 1/4096 part."""
    runs = {
        # one warm-up solve first: the first solve's setup (pass buffers,
        # kernel attributes) would otherwise be scaled up with the classes
        "10_90_part": lambda: bench_10_90(_with(args, steps=1, warmup=1), emit=False),
        "serving": lambda: bench_serving(_with(args, requests=256, rate_factor=1.0), emit=False),
        "batch_6_50": lambda: bench_batch(_with(args, steps=3, warmup=2), emit=False),
        "first_9_80": lambda: bench_first(_with(args, steps=1, warmup=0, instances=4), emit=False),
        "11_100_part": lambda: bench_11_100(_with(args, steps=1, warmup=1), emit=False),
    }
    keep = {
        "10_90_part": ("metric", "ms_per_step", "projected_full_time_s", "list_build_s", "records_done",
                       "records_total", "config"),
        "serving": ("value", "unit", "served", "sequential", "results_identical", "config"),
        "batch_6_50": ("value", "unit", "ms_per_step", "sequential", "streaming_batch", "speedup_vs_sequential"),
        "first_9_80": ("value", "planted_average_s", "instances", "paper"),
        "11_100_part": ("metric", "ms_per_step", "projected_full_time_s", "list_build_s", "config"),
    }
    out = {}
    for name, run in runs.items():
        t0 = time.perf_counter()
        try:
            r = run()
            out[name] = {k: r[k] for k in keep[name] if k in r}
        except Exception as e:  # reported in the line, the headline stands
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = time.perf_counter() - t0
    return out


def main():
    args = parse()
    world, rank, local, pg = dist_init(args)
    try:
        if args.impl == "reference":
            reference(args, world, rank, pg)
        elif args.config == "batch_6_50":
            if rank == 0:
                bench_batch(args)
        elif args.config == "serving":
            if rank == 0:
                bench_serving(args)
        elif args.config == "10_90_part":
            if rank == 0:
                bench_10_90(args)
        elif args.config == "profile_part":
            if rank == 0:
                bench_profile_part(args)
        elif args.config == "profile_small":
            if rank == 0:
                bench_profile_small(args)
        elif args.config == "first_9_80":
            if rank == 0:
                bench_first(args)
        elif args.config == "11_100_part":
            if rank == 0:
                bench_11_100(args)
        elif args.config == "first_10_90":
            if rank == 0:
                bench_first_10_90(args)
        elif args.config == "k_sweep":
            if rank == 0:
                bench_k_sweep(args)
        else:
            native(args, world, rank, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    main()
