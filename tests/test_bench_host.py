"""Host-side pieces of bench.py, on the CPU: the clock summary the JSON line
carries, and the ncu traffic lookup keyed by the kernel source's sha256."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

ROW = "0, {sm}, 2070, 600.0, 0x0000000000000000, {a}, {b}, {c}, {d}\n"


def rows(*specs):
    return [ROW.format(sm=sm, a=a, b=b, c=c, d=d) for sm, (a, b, c, d) in specs]


QUIET = ("Not Active",) * 4


def test_clock_summary_median_and_no_reason():
    got = bench.summarize_clocks(rows((2070, QUIET), (1900, QUIET), (2070, QUIET)))
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


def test_clock_summary_reasons():
    pc = ("Not Active", "Not Active", "Not Active", "Active")
    th = ("Not Active", "Active", "Not Active", "Not Active")
    got = bench.summarize_clocks(rows((2070, QUIET), (1800, pc), (1700, th)))
    assert got["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert got["sm_mhz"] == 1800.0 and got["samples"] == 3


def test_clock_summary_skips_bad_rows():
    lines = ["garbage\n", "0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active\n"]
    assert bench.summarize_clocks(lines) is None
    assert bench.summarize_clocks(lines + rows((2000, QUIET)))["samples"] == 1


def test_traffic_lookup_follows_the_source_hash(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    entry = {"source": "k.cu", "source_sha256": hashlib.sha256(src.read_bytes()).hexdigest(),
             "dram_bytes": 150, "algorithmic_bytes": 100,
             "onchip": {"l1tex_pct_of_peak": 70.0, "case": "k.md"}}
    (prof / "traffic.json").write_text(json.dumps({"kernels": {"k": entry}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_per_launch("k", 1000.0) == 1500.0
    assert bench._capture("k")["onchip"]["l1tex_pct_of_peak"] == 70.0
    assert bench.traffic_per_launch("other", 1000.0) is None
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.traffic_per_launch("k", 1000.0) is None
    assert bench._capture("k") is None


def test_committed_traffic_entries_name_existing_sources():
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for name, k in t["kernels"].items():
        assert os.path.exists(os.path.join(ROOT, k["source"])), name
        assert os.path.exists(os.path.join(ROOT, "profiles", k["case"])), name


def test_oracle_sample_projects_the_whole_instance():
    # the CPU baseline times the four-list oracle on a bounded slice range of
    # the same instance and projects the time to all solutions by records
    import bench
    import msp_instances as mi
    A, d, _ = mi.generate(4, 40, 3)
    o = bench.oracle_sample(A, d, div=8, seed=3)
    assert o["records_total"] == 2 * (1 << 20)
    assert 0 < o["records"] < o["records_total"]
    lo, hi, S = o["slices"]
    assert lo == 0 and hi == max(1, S // 8)
    assert o["projected_s"] >= o["build_s"]
    assert abs(o["projected_s"] - (o["build_s"] + o["join_s"] * o["records_total"] / o["records"])) < 1e-9
    assert "seed 3 " in o["sample"] and str(o["cores"]) in o["sample"]


def test_secondary_block_reports_each_run_and_survives_a_failure(monkeypatch):
    import bench
    args = bench.argparse.Namespace(steps=20, warmup=3, requests=512, rate_factor=0.8, instances=4)
    seen = {}

    def fake(name, fail=False):
        def run(a, emit=True):
            assert emit is False
            seen[name] = a
            if fail:
                raise RuntimeError("no device")
            return {"value": 1.0, "unit": "u", "ms_per_step": 2.0, "projected_full_time_s": 3.0,
                    "metric": "m", "config": {}, "served": {}, "sequential": {}, "results_identical": True,
                    "planted_average_s": 4.0, "instances": [], "paper": "p", "unused": 0}
        return run

    monkeypatch.setattr(bench, "bench_10_90", fake("10_90"))
    monkeypatch.setattr(bench, "bench_serving", fake("serving", fail=True))
    monkeypatch.setattr(bench, "bench_batch", fake("batch"))
    monkeypatch.setattr(bench, "bench_first", fake("first"))
    monkeypatch.setattr(bench, "bench_11_100", fake("11_100"))
    out = bench.secondary(args)
    assert set(out) == {"10_90_part", "serving", "batch_6_50", "first_9_80", "11_100_part"}
    assert out["serving"]["error"] == "RuntimeError: no device"
    assert out["10_90_part"]["projected_full_time_s"] == 3.0 and "unused" not in out["10_90_part"]
    assert all("wall_s" in v for v in out.values())
    # short forms: one step, a 256-request stream at the service rate; the
    # caller's own arguments are left as they were
    assert seen["10_90"].steps == 1 and seen["10_90"].warmup == 1
    assert seen["serving"].requests == 256 and seen["serving"].rate_factor == 1.0
    assert seen["first"].instances == 4
    assert args.steps == 20 and args.requests == 512
