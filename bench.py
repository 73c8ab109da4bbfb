#!/usr/bin/env python3
"""TensorACO benchmark: one JSON line per run.

A step is one whole ACO iteration on the GPU -- build M_p, construct all m
tours, tour lengths + best, evaporate + deposit -- on a synthetic instance
shaped like the paper's workloads.  Default workload: 5000 clustered cities
(50 Gaussian clusters, sigma 0.02), m = 1024 ants, alpha 1, beta 2, rho 0.1,
fp32 M_p, independent roulette, deterministic deposit.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

N > 1 (under torchrun): every rank solves its own instance (replicas; weak
scaling), the time is the max over ranks, value sums the ranks' ant-steps.
--impl reference times the CPU oracle (the plain C++ restatement of the
method) on the host cores, on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2404_04895_gb300 import instances  # noqa: E402

METRIC = "ant-steps/s"
STEPS = ["build_P", "build_lists", "construct", "tour_length", "best", "deposit"]
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="n5000_clustered", choices=sorted(instances.WORKLOADS))
    ap.add_argument("--prec", default=None, choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--no-variants", action="store_true", help="skip the bf16/fp16 comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--gap-seeds", type=int, default=5)
    ap.add_argument("--no-autotune", action="store_true", help="default full-scan shape (profiling runs)")
    ap.add_argument("--no-lists", action="store_true",
                    help="time the full-scan construction instead of the candidate-list one")
    ap.add_argument("--no-full-scan", action="store_true",
                    help="skip the side measurement of the full-scan construction kernel")
    ap.add_argument("--no-roulette", action="store_true",
                    help="skip the RW / IR / AdaIR comparison on the bench workload")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched measurement (256 instances, n ~ U{100..2000}, m = n, bf16)")
    ap.add_argument("--no-ceilings", action="store_true",
                    help="skip the live ceiling measurements (L2 row reads, Philox, dependent loads)")
    return ap.parse_args()


def workload(args):
    w = dict(instances.WORKLOADS[args.workload])
    if args.prec:
        w["prec"] = args.prec
    return w


def config_of(args, w, world):
    """The workload as both arms name it (identical dicts)."""
    lists = not args.no_lists
    return {"workload": args.workload, "kind": w["kind"], "n": w["n"], "m": w["m"], "alpha": w["alpha"],
            "beta": w["beta"], "rho": w["rho"], "Q": w["Q"], "roulette": "adair" if w["adair"] else "ir",
            "deposit": "deterministic", "P_dtype": w["prec"], "iterations_budget": w["iters"],
            "construction": "candidate lists (exact pruning)" if lists else "full scan",
            "l2": "GPU arm: flushed between timed steps (512 MiB write)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def solver_kwargs(w, seed):
    kw = dict(m=w["m"], alpha=w["alpha"], beta=w["beta"], rho=w["rho"], Q=w["Q"], seed=seed,
              prec=w["prec"], roulette="adair" if w["adair"] else "ir")
    if w["adair"]:
        kw.update(gamma_max=1.5, gamma_min=0.5, gamma_T=w["iters"])
    return kw


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = {
    # the candidate-list construction kernel and what shapes its traffic (the lists)
    "construct_lean_kernel": ("construct_lean.cuh", "construct.cuh", "common.cuh", "lists.cuh"),
    # the full-scan construction kernel
    "construct_kernel": ("construct.cuh", "shapes.h", "common.cuh", "lists.cuh"),
}


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(ROOT, "paper_2404_04895_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profile_counter(kernel, kernel_hash, workload_name, prec, field):
    """One per-launch counter of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "construct_dram_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(f"{kernel}:{workload_name}:{prec}")
    if not e or e.get("kernel_hash") != kernel_hash:
        return None
    return e.get(field)


def traffic_from_profile(kernel, kernel_hash, workload_name, prec):
    """dram bytes per launch of `kernel` (ncu), for the current source only."""
    return profile_counter(kernel, kernel_hash, workload_name, prec, "dram_bytes_per_launch")


SCHEDULERS_PER_SM = 4   # warp schedulers of a Blackwell SM, one instruction issued per cycle each


def issue_roofline(kernel, inst_per_launch, launch_ms, sms, sm_mhz):
    """Instruction-issue roofline: warp instructions per launch (ncu) over the
    launch time, against every scheduler issuing one per cycle at the SM
    clock sampled during the timed region."""
    peak = sms * SCHEDULERS_PER_SM * sm_mhz * 1e6 if sms and sm_mhz else None
    achieved = inst_per_launch / (launch_ms / 1e3) if inst_per_launch and launch_ms > 0 else None
    return {"bound": "issue", "kernel": kernel, "unit": "warp-instructions/s",
            "achieved": achieved, "peak": peak,
            "frac": round(achieved / peak, 4) if achieved and peak else None,
            "inst_per_launch": inst_per_launch, "sms": sms, "schedulers_per_sm": SCHEDULERS_PER_SM,
            "sm_mhz": sm_mhz, "avg_launch_ms": round(launch_ms, 4)}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for name, val in zip(names, f[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------- distributed
class Dist:
    def __init__(self, args):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            backend = "nccl" if args.impl == "native" else "gloo"
            dist.init_process_group(backend)
            self.dist = dist
            self.pg = True

    def barrier(self):
        if self.pg:
            self.dist.barrier()

    def max(self, x):
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64,
                         device="cuda" if self.dist.get_backend() == "nccl" else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.dist.destroy_process_group()


def whole_job_value(units_per_rank_step, world, t_max_ms, steps):
    """Units per second of the whole job: every rank's units of `steps`
    steps over the slowest rank's timed region (ms)."""
    return units_per_rank_step * world * steps / (t_max_ms / 1e3)


# ---------------------------------------------------------------- CPU oracle leg
def oracle_state(w, coords, seed):
    import oracle
    prec = {"fp32": oracle.FP32, "bf16": oracle.BF16, "fp16": oracle.FP16}[w["prec"]]
    return oracle.State(coords, w["m"], alpha=w["alpha"], beta=w["beta"], rho=w["rho"], Q=w["Q"], seed=seed,
                        prec=prec, adair=bool(w["adair"]), gamma_max=1.5, gamma_min=0.5, gamma_T=w["iters"])


def oracle_iterations(w, coords, seed, max_iters=1, budget_s=None, warmup=0):
    """Whole iterations of the CPU oracle on the workload (M_p, all m tours,
    lengths, best, deposit), on all host cores: `warmup` untimed ones, then
    timed ones until max_iters are done or budget_s is spent (at least one)."""
    import oracle
    threads = oracle.default_threads()
    st = oracle_state(w, coords, seed)
    for _ in range(warmup):
        st.run(1, nthreads=threads)
    times = []
    while len(times) < max_iters:
        t0 = time.perf_counter()
        st.run(1, nthreads=threads)
        times.append(time.perf_counter() - t0)
        if budget_s is not None and sum(times) + times[-1] > budget_s:
            break
    secs = sum(times)
    n, m = w["n"], w["m"]
    return {"value": round(len(times) * m * (n - 1) / secs, 1), "unit": METRIC, "cores": threads,
            "kind": "oracle", "iterations": len(times), "first_iteration": warmup,
            "sample": f"{len(times)} whole iteration(s) {warmup}..{warmup + len(times) - 1} of the workload "
                      f"(M_p, all {m} tours, lengths, best, deposit; n={n}), {secs:.2f} s",
            "_times": times}


def oracle_batch_sample(sizes, budget_s=15.0, stride=32):
    """The CPU oracle on a sample of the batch workload: one whole iteration
    (bf16 M_p, all m = n tours, lengths, deposit) of every `stride`-th
    instance, on all host cores, until the budget is spent."""
    import oracle
    threads = oracle.default_threads()
    ant_steps, secs, ids = 0, 0.0, []
    for i in range(0, len(sizes), stride):
        n = int(sizes[i])
        st = oracle.State(instances.uniform(n, 1000 + i), n, rho=0.1, seed=i, prec=oracle.BF16)
        t0 = time.perf_counter()
        st.run(1, nthreads=threads)
        secs += time.perf_counter() - t0
        ant_steps += n * (n - 1)
        ids.append(i)
        if secs >= budget_s:
            break
    return {"value": round(ant_steps / secs, 1), "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": f"one whole iteration (bf16 M_p, m = n tours, lengths, deposit) of instances {ids} "
                      f"(one in {stride}; n = {[int(sizes[i]) for i in ids]}), {secs:.3f} s"}


# ---------------------------------------------------------------- native leg
def run_native(args, w, dist):
    import torch
    from paper_2404_04895_gb300 import binding as B

    torch.cuda.set_device(dist.local)
    B.lib()
    coords = instances.coords_for(w)
    n, m = w["n"], w["m"]
    seed = w["seed"] + dist.rank
    st = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def timed_run(prec, steps, warmup, lists, profile=True, tau_prec="fp32"):
        kw = solver_kwargs(dict(w, prec=prec), seed)
        s = B.Solver(coords, stream=st, cand_lists=lists, tau_prec=tau_prec, **kw)
        if profile:
            s.set_profiling(True)
        s.iterate(warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        total = 0.0
        kern = np.zeros(len(STEPS))
        for q in range(steps):
            with torch.cuda.stream(st):
                flush.fill_(q & 0xFF)          # L2 flush, outside the timed region
                e0.record(st)
                s.iterate(1)
                e1.record(st)
            e1.synchronize()
            total += e0.elapsed_time(e1)
            if profile:
                kern += s.kernel_ms()
        torch.cuda.synchronize()
        best = s.best()[1]
        s.close()
        return total, kern, best

    lists = not args.no_lists
    peak, peak_src = peaks()
    peak_note = "measured (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback 6.8 TB/s"
    bp = 4 if w["prec"] == "fp32" else 2
    alg_bytes = m * n * (n - 1) / 2 * bp      # every unvisited M_p entry of every ant-step
    tuned = None
    if not lists or not args.no_full_scan:    # full-scan launch shape for this workload (untimed)
        tuned = ((0, 0, 0), None) if args.no_autotune else autotune(B, torch, w, coords, w["prec"], seed)
    dist.barrier()
    clk = ClockSampler(dist.local)
    torch.cuda.synchronize()
    dist.barrier()
    clk.start()
    total_ms, kern, best_len = timed_run(w["prec"], args.steps, args.warmup, lists)
    torch.cuda.synchronize()
    dist.barrier()
    clocks = clk.stop()
    t_max = dist.max(total_ms)
    ms_per_step = t_max / args.steps
    ant_steps = m * (n - 1)
    value = whole_job_value(ant_steps, dist.world, t_max, args.steps)

    def full_scan_roofline(construct_ms, shape, ceil=None):
        achieved = alg_bytes / (construct_ms / 1e3) / 1e9
        kh = kernel_source_hash("construct_kernel")
        out = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
               "frac": round(achieved / peak, 4), "peak_source": peak_note,
               "traffic": traffic_from_profile("construct_kernel", kh, args.workload, w["prec"]),
               "kernel": "construct_kernel", "algorithmic_bytes_per_launch": alg_bytes,
               "avg_launch_ms": round(construct_ms, 4), "kernel_source_hash": kh,
               "construct_shape": {"warps_per_ant": shape[0], "chunks_per_lane": shape[1],
                                   "mode": ["staged", "direct"][shape[2]] if shape[0] else "default"}}
        # M_p (100 MB fp32, 50 MB in 16 bits at n = 5000) mostly stays in the L2:
        # the ceiling its random row reads can reach is measured, not HBM's
        fp = (n * n * bp) >> 20
        rr = [r for r in (ceil or {}).get("row_reads", []) if r["footprint_MB"] == (100 if bp == 4 else 50)]
        if rr and fp <= 128:
            out["l2_ceiling_GBps"] = rr[0]["GBps"]
            out["frac_of_l2_ceiling"] = round(achieved / rr[0]["GBps"], 4)
        return out

    construct_ms = kern[2] / args.steps
    kernel_ms = dict(zip(STEPS, [round(x / args.steps, 4) for x in kern]))
    sms = torch.cuda.get_device_properties(dist.local).multi_processor_count
    ceil = None
    if dist.rank == 0 and not args.no_ceilings:
        from paper_2404_04895_gb300 import ceilings
        try:
            ceil = ceilings.measure(reps=3)
        except Exception as e:  # an auxiliary figure never costs the bench line
            ceil = {"error": repr(e)}
    fs = None
    if lists and not args.no_full_scan and dist.rank == 0:
        steps_f = min(args.steps, 20)
        _, kf, _ = timed_run(w["prec"], steps_f, 3, False)
        fs = full_scan_roofline(kf[2] / steps_f, tuned[0], ceil)
    if lists:
        # The candidate-list kernel decides most steps from a row's top
        # entries and reads a row only when the list cannot: it moves a small
        # fraction of the full scan's bytes and is bound by each ant's
        # dependent step chain, i.e. by instruction issue.  Its roofline is
        # issue: warp instructions per launch (ncu, this kernel source) over
        # the launch time, against 4 schedulers x 1 instruction per cycle per
        # SM at the sampled SM clock.
        kh = kernel_source_hash("construct_lean_kernel")
        inst = profile_counter("construct_lean_kernel", kh, args.workload, w["prec"], "inst_executed_per_launch")
        roofline = issue_roofline("construct_lean_kernel", inst, construct_ms, sms, clocks.get("sm_mhz"))
        roofline.update({
            "bound": "alu",
            "traffic": traffic_from_profile("construct_lean_kernel", kh, args.workload, w["prec"]),
            "kernel_source_hash": kh,
            "peak_source": f"{sms} SMs x {SCHEDULERS_PER_SM} schedulers x 1 warp instruction per cycle "
                           "x the SM clock sampled during the timed region",
            "inst_source": "ncu inst_executed of one launch of this kernel source (profiles/); None if the "
                           "source changed since the capture"})
        clk_mhz = clocks.get("sm_mhz") or 0.0
        chain = {"cycles_per_ant_step": round(construct_ms * 1e-3 * clk_mhz * 1e6 / (n - 1), 1) if clk_mhz else None,
                 "note": "launch time x SM clock / (n - 1): every ant walks its n - 1 steps concurrently"}
        if ceil and "chase" in ceil:
            chain["dependent_l2_load_cycles"] = ceil["chase"]["cycles_per_load_median"]
        roofline["step_chain"] = chain
        if fs:
            roofline["pruning_speedup"] = round(fs["avg_launch_ms"] / construct_ms, 3)
            roofline["pruning_note"] = ("full-scan construction time / candidate-list construction time on the "
                                        "same workload, same tours (both checked against the oracle)")
    else:
        roofline = full_scan_roofline(construct_ms, tuned[0], ceil)

    out = {
        "metric": METRIC, "value": round(value, 1), "unit": METRIC, "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16", "fp16": "f16"}[w["prec"]],
        "data": "synthetic",
        "config": config_of(args, w, dist.world),
        "iters_per_s": round(1e3 / ms_per_step, 2),
        "roofline": roofline,
        "kernel_ms": kernel_ms,
        # per iteration: construction, tour lengths, best, and the deterministic
        # deposit, which with lists also computes the next iteration's M_p and
        # lists; without lists M_p is a launch of its own
        "gpu_launches": args.steps * (4 if lists else 5),
        "clocks": clocks,
        "best_len_after_steps": best_len,
    }
    if fs and lists:
        out["full_scan_roofline"] = fs
    if ceil is not None:
        out["ceilings"] = ceil

    if dist.rank == 0 and not args.no_variants:
        # BF16 / FP16 M_p against fp32 on the same GPU: throughput and best-length gap
        variants = {}
        gaps = {}
        # (M_p precision, tau precision) pairs beside the main line
        forms = [("fp32", "fp32"), ("bf16", "fp32"), ("fp16", "fp32"), ("bf16", "bf16")]
        for prec, tprec in forms:
            name = prec if tprec == "fp32" else f"{prec}_P_{tprec}_tau"
            if (prec, tprec) != (w["prec"], "fp32"):
                steps_v = min(args.steps, 30)
                t, kv, _ = timed_run(prec, steps_v, 3, lists, tau_prec=tprec)
                cms = kv[2] / steps_v
                bpv = 4 if prec == "fp32" else 2
                ach = m * n * (n - 1) / 2 * bpv / (cms / 1e3) / 1e9
                variants[name] = {"ms_per_step": round(t / steps_v, 4),
                                  "value": round(ant_steps / (t / steps_v / 1e3), 1),
                                  "construct_ms": round(cms, 4), "construct_alg_GBps": round(ach, 1),
                                  "frac_of_hbm": round(ach / peak, 4),
                                  "kernel_ms": dict(zip(STEPS, [round(x / steps_v, 4) for x in kv]))}
            # best length after the workload's full iteration budget, mean over seeds
            lens = []
            for sd in range(args.gap_seeds):
                s = B.Solver(coords, stream=st, cand_lists=lists, tau_prec=tprec,
                             **solver_kwargs(dict(w, prec=prec), sd))
                s.iterate(w["iters"])
                lens.append(s.best()[1])
                s.close()
            gaps[name] = float(np.mean(lens))
        for name in gaps:
            if name != "fp32":
                variants.setdefault(name, {})["best_len_gap_vs_fp32"] = round(gaps[name] / gaps["fp32"] - 1, 5)
        out["variants"] = variants
        out["best_len_mean"] = {k: round(v, 6) for k, v in gaps.items()}
        out["best_len_protocol"] = f"mean over seeds 0..{args.gap_seeds - 1} after {w['iters']} iterations"

    if dist.rank == 0 and not args.no_roulette:
        out["roulette"] = run_roulette(B, torch, w, coords, seed)
    if dist.rank == 0 and not args.no_batched:
        out["batched"] = run_batched(B, torch, peak, value / dist.world if w["prec"] == "fp32" else None,
                                     cpu=not args.no_cpu_baseline and dist.world == 1)
    if dist.rank == 0 and not args.no_e2e:
        out["e2e"] = run_e2e(args, w, coords, seed)
    if dist.rank == 0 and not args.no_cpu_baseline and dist.world == 1:
        cb = oracle_iterations(w, coords, seed, max_iters=1)
        cb.pop("_times")
        out["cpu_baseline"] = cb
    return out


def run_roulette(B, torch, w, coords, seed, steps=10):
    """The paper's selection ablation on the bench workload: time per
    iteration and best length after the workload's iteration budget for the
    roulette wheel, independent roulette and AdaIR (gamma 1.5 -> 0.5)."""
    st = torch.cuda.Stream()
    out = {}
    for r in ("ir", "adair", "rw"):
        kw = solver_kwargs(dict(w, adair=False), seed)
        kw["roulette"] = r
        if r == "adair":
            kw.update(gamma_max=1.5, gamma_min=0.5, gamma_T=w["iters"])
        s = B.Solver(coords, stream=st, **kw)
        s.iterate(2)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            e0.record(st)
            s.iterate(steps)
            e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        s.iterate(max(0, w["iters"] - 2 - steps))
        out[r] = {"ms_per_iter": round(ms, 3), "best_len_after_budget": s.best()[1]}
        s.close()
    out["protocol"] = (f"{steps} timed iterations after 2; best length after {w['iters']} iterations, "
                       f"Philox seed {seed}; rw = exact-integer roulette wheel, one 256-thread CTA per ant, the row staged by one TMA bulk copy per step")
    return out


def run_batched(B, torch, peak, single_value, steps=5, warmup=2, cpu=False):
    """Many instances in one batch: 256 uniform instances, n ~ U{100..2000},
    m = n, alpha 1, beta 2, rho 0.1, bf16 M_p; every iteration is one graph
    replay whose construction is one persistent launch over all ants.  The
    instances' M_p (about 0.7 GB in bf16) exceed the L2, so no flush is needed."""
    sizes = [int(x) for x in instances.batch_sizes(256, 100, 2000, seed=7)]
    arena = sum(B.instance_bytes(n, n) for n in sizes) + (64 << 20)
    st = torch.cuda.Stream()
    bt = B.Batch(len(sizes), arena, prec="bf16", stream=st)
    for i, n in enumerate(sizes):
        if bt.add(instances.uniform(n, 1000 + i), n, iters=0, rho=0.1, seed=i) is None:
            bt.close()
            return {"unavailable": "batch arena too small"}
    bt.step(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        e0.record(st)
        bt.step(steps)
        e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    bt.close()
    ant_steps = float(sum(n * (n - 1) for n in sizes))
    alg = float(sum(n * n * (n - 1) / 2 for n in sizes)) * 2
    value = ant_steps / (ms / 1e3)
    extra = {"cpu_baseline": oracle_batch_sample(sizes)} if cpu else {}
    return {**extra, "workload": "256 uniform instances, n ~ U{100..2000} (seed 7), coords seeds 1000+i, m = n, "
                        "alpha 1, beta 2, rho 0.1, bf16 M_p, candidate lists",
            "steps": steps, "warmup": warmup, "ms_per_iter": round(ms, 3),
            "value": round(value, 1), "unit": METRIC,
            "construct_alg_GBps": round(alg / (ms / 1e3) / 1e9, 1),
            "frac_of_hbm_alg": round(alg / (ms / 1e3) / 1e9 / peak, 4),
            "vs_single_instance_fp32": round(value / single_value, 3) if single_value else None,
            "note": "whole-iteration time; the algorithmic bytes are the full-scan M_p reads of all "
                    "instances, so frac > 1 reflects the exact pruning"}


def autotune(B, torch, w, coords, prec, seed):
    """Pick the construct launch shape on the iteration-0 M_p of the workload
    (untimed); the library keeps it as the default for (n, m, precision)."""
    n, m = w["n"], w["m"]
    ld = B.ld_of(n)
    H = torch.empty((n, ld), dtype=torch.float32, device="cuda")
    tau = torch.empty_like(H)
    P = torch.empty_like(H)
    xy = torch.from_numpy(np.ascontiguousarray(coords)).cuda()
    B.op_heuristic(xy, n, w["beta"], None, H, ld)
    B.op_fill(tau, n, ld, 1.0)
    inv = B.inv_gamma(B.gamma(0, w["iters"], 1.5, 0.5)) if w["adair"] else 1.0
    B.op_build_P(tau, H, n, ld, w["alpha"], inv, B.PREC[prec], P)
    tours = torch.empty((m, n), dtype=torch.int32, device="cuda")
    shape, ms = B.autotune_construct(P, B.PREC[prec], n, ld, m, seed, tours, reps=2)
    torch.cuda.synchronize()
    return shape, ms


def run_e2e(args, w, coords, seed):
    """Same metric through the public C ABI with host buffers: aco_init copies
    the coordinates in, each step is aco_iterate(1) followed by aco_best()
    reading the best tour and length back to host memory."""
    import torch
    from paper_2404_04895_gb300 import binding as B
    L = B.lib()
    n, m = w["n"], w["m"]
    xy = torch.from_numpy(np.ascontiguousarray(coords)).pin_memory()
    tour = torch.empty(n, dtype=torch.int32).pin_memory()
    blen = torch.empty(1, dtype=torch.float64).pin_memory()
    B.check(L.aco_bind(None, 0, None))
    B.check(L.aco_set_precision(B.PREC[w["prec"]]))
    B.check(L.aco_set_variant(B.ADAIR if w["adair"] else B.IR, 1.5, 0.5, w["iters"]))
    B.check(L.aco_set_deposit(B.DEPOSIT_DET))

    def job(steps):
        B.check(L.aco_init(xy.data_ptr(), n, m, float(w["alpha"]), float(w["beta"]), w["rho"], w["Q"], seed))
        for _ in range(steps):
            B.check(L.aco_iterate(1))
            B.check(L.aco_best(tour.data_ptr(), blen.data_ptr()))
        B.check(L.aco_free())

    job(2)  # warm-up: module load, graph instantiation
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    job(args.steps)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    return {"value": round(args.steps * m * (n - 1) / secs, 1), "unit": METRIC,
            "h2d_bytes_per_step": round(n * 8 / args.steps, 2), "d2h_bytes_per_step": n * 4 + 8,
            "note": "one job = aco_init (coords host->device, distances, eta^beta) + steps x "
                    "(aco_iterate(1) + aco_best to host); h2d is the job's coordinates spread over its steps"}


# ---------------------------------------------------------------- reference leg
REFERENCE_BUDGET_S = 120.0   # timed whole iterations of the oracle stop once this is spent


def run_reference(args, w, dist):
    """The CPU oracle as it stands, on the host cores: whole iterations of the
    workload.  The steps actually timed (at most --steps, fewer once the time
    budget is spent) and warm-up iterations (at most one) are what the line
    reports, so steps x ms_per_step is the timed wall time."""
    coords = instances.coords_for(w)
    if dist.rank != 0:
        return None
    warm = min(args.warmup, 1)
    r = oracle_iterations(w, coords, w["seed"], max_iters=args.steps, budget_s=REFERENCE_BUDGET_S, warmup=warm)
    times = r.pop("_times")
    ms_per_step = 1e3 * sum(times) / len(times)
    return {
        "impl": "reference", "metric": METRIC, "value": r["value"], "unit": METRIC,
        "n_gpus": dist.world, "steps": len(times), "warmup": warm,
        "steps_requested": args.steps, "warmup_requested": args.warmup,
        "ms_per_step": round(ms_per_step, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "fp16": "f16"}[w["prec"]],
        "data": "synthetic",
        "config": config_of(args, w, dist.world),
        "cpu_baseline": {"value": r["value"], "unit": METRIC, "cores": r["cores"], "kind": "oracle",
                         "sample": r["sample"] + f"; timing stops once {REFERENCE_BUDGET_S:.0f} s are spent"},
        "e2e": {"value": r["value"], "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    w = workload(args)
    dist = Dist(args)
    try:
        out = run_reference(args, w, dist) if args.impl == "reference" else run_native(args, w, dist)
        if dist.rank == 0 and out is not None:
            print(json.dumps(out), flush=True)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
