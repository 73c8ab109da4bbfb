"""Host-side plumbing of bench.py: the committed ncu traffic is used only for
the kernel source it was taken on, and the CPU baselines return well-formed
records."""
import importlib.util
import json
import os

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_only_for_the_profiled_source(bench):
    entries = json.load(open(os.path.join(ROOT, "profiles", "construct_dram_traffic.json")))
    key, e = next(iter(entries.items()))
    kernel, workload, prec = key.split(":")
    assert bench.traffic_from_profile(kernel, e["kernel_hash"], workload, prec) == e["dram_bytes_per_launch"]
    assert e["dram_bytes_per_launch"] == e["dram_bytes_read"] + e["dram_bytes_write"]
    assert bench.traffic_from_profile(kernel, "0" * 16, workload, prec) is None       # another source
    assert bench.traffic_from_profile(kernel, e["kernel_hash"], workload, "bf16") is None


def test_kernel_source_hash_follows_the_files(bench):
    h = bench.kernel_source_hash("construct_lean_kernel")
    assert len(h) == 16 and h == bench.kernel_source_hash("construct_lean_kernel")
    assert all(os.path.exists(os.path.join(ROOT, "paper_2404_04895_gb300", "csrc", f))
               for f in bench.KERNEL_SOURCES["construct_lean_kernel"])


def test_batch_cpu_baseline_record(bench):
    """Whole oracle iterations of sampled batch instances (small sizes here)."""
    r = bench.oracle_batch_sample([60, 70, 80, 90], budget_s=0.0, stride=2)
    assert r["kind"] == "oracle" and r["unit"] == bench.METRIC and r["cores"] >= 1
    assert r["value"] > 0 and "instances [0]" in r["sample"] and "whole iteration" in r["sample"]


def test_cpu_baseline_times_whole_iterations(bench):
    """The oracle leg runs complete iterations (M_p, tours, lengths, deposit)
    and reports what it timed; the budget stops it after at least one."""
    from paper_2404_04895_gb300 import instances
    w = dict(instances.WORKLOADS["n50_ir"])
    r = bench.oracle_iterations(w, instances.coords_for(w), 0, max_iters=3, warmup=1)
    assert r["iterations"] == 3 and len(r["_times"]) == 3 and r["first_iteration"] == 1
    assert r["value"] == round(3 * w["m"] * (w["n"] - 1) / sum(r["_times"]), 1)
    r = bench.oracle_iterations(w, instances.coords_for(w), 0, max_iters=50, budget_s=0.0)
    assert r["iterations"] == 1


def test_issue_roofline(bench):
    """Warp instructions per launch over the launch time, against 4 schedulers
    per SM issuing one instruction per cycle; missing inputs give None, never
    an exception."""
    entries = json.load(open(os.path.join(ROOT, "profiles", "construct_dram_traffic.json")))
    key, e = next(iter(entries.items()))
    kernel, workload, prec = key.split(":")
    inst = bench.profile_counter(kernel, e["kernel_hash"], workload, prec, "inst_executed_per_launch")
    assert inst == e["inst_executed_per_launch"] > 0
    r = bench.issue_roofline(kernel, 1.2e9, 2.0, 152, 2000.0)
    assert r["achieved"] == 1.2e9 / 2.0e-3 and r["peak"] == 152 * 4 * 2000.0e6
    assert r["frac"] == round(r["achieved"] / r["peak"], 4) and r["bound"] == "issue"
    for args in [(None, 2.0, 152, 2000.0), (1e9, 2.0, 152, None), (1e9, 0.0, 152, 2000.0)]:
        r = bench.issue_roofline(kernel, *args)
        assert r["frac"] is None


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the CPU oracle on the host cores, no GPU)
    prints one JSON line with the contract's keys, its cpu_baseline and an
    e2e equal to its own value."""
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1", "--workload", "n50_ir"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ["metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"]:
        assert k in d, k
    assert d["impl"] == "reference" and d["config"]["workload"] == "n50_ir" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # whole iterations, as many as were timed: steps x ms_per_step is the timed work
    assert d["steps"] == 1 and d["warmup"] == 1
    w = dict(__import__("paper_2404_04895_gb300.instances", fromlist=["x"]).WORKLOADS["n50_ir"])
    assert abs(d["value"] - w["m"] * (w["n"] - 1) / (d["ms_per_step"] / 1e3)) / d["value"] < 1e-2


def test_both_arms_name_the_same_config(bench):
    """The native and reference lines carry the identical config dict."""
    from paper_2404_04895_gb300 import instances

    class Args:
        workload, no_lists = "n5000_clustered", False
    w = dict(instances.WORKLOADS["n5000_clustered"])
    c = bench.config_of(Args(), w, 1)
    for k in ("workload", "n", "m", "alpha", "beta", "rho", "Q", "roulette", "deposit", "P_dtype", "construction",
              "l2", "parallelism"):
        assert k in c, k
    assert c == bench.config_of(Args(), dict(w), 1)
