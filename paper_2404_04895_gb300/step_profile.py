"""Per-step cycle breakdown of the candidate-list construction kernel on the
n = 5000 clustered workload (m = 1024, fp32 M_p), from the probed kernel
(aco_op_construct_probe): a solver runs to iteration `it`, its M_p and
candidate lists are rebuilt from its pheromone, and the probed construction
walks all 1024 ants while a few of them record every step's clock stamps.
The probed tours are checked against the solver's own iteration `it`.

  python -m paper_2404_04895_gb300.step_profile [--iters 0 30 99] [--ants 0 511 1023]

prints one JSON object: per iteration, the median / mean cycles of a step
and of its phases, and how often each path ran.
"""
import argparse
import json

import numpy as np

from . import instances

PHASES = ["list_entry_ready", "philox_done", "spec_loads_issued", "first_round_decided", "decided", "step_end"]


def _summary(rec):
    """rec: (steps, 8) u32 records of one ant's walk (t = 1 .. n-1)."""
    start = rec[:, 0].astype(np.int64)
    step = ((start[1:] - start[:-1]) % (1 << 32)).astype(np.float64)   # start to next start
    flags = rec[:, 7]
    fast = (flags & 1) != 0
    out = {"step_cycles_median": float(np.median(step)), "step_cycles_mean": float(step.mean())}
    for i, name in enumerate(PHASES, start=1):
        v = rec[:, i].astype(np.float64)
        out[f"{name}_median"] = float(np.median(v[fast])) if fast.any() else None
    out["end_fast_mean"] = float(rec[fast, 6].mean()) if fast.any() else None
    slow = ~fast
    out["end_slow_mean"] = float(rec[slow, 6].mean()) if slow.any() else None
    hit0, hit1 = (flags & 8) != 0, (flags & 16) != 0
    n = len(flags)
    out.update({"first_round_decides": float(fast.mean()), "later_rounds": float(((flags & 2) != 0).mean()),
                "full_scans": float(((flags & 4) != 0).mean()), "spec_hit_slot0": float(hit0.mean()),
                "spec_hit_slot1": float(hit1.mean()), "spec_miss": float((~hit0 & ~hit1).sum() / n)})
    # the whole walk's cycles split by path: where the step time goes
    st = np.concatenate([step, [np.median(step)]])
    out["cycle_share_fast_steps"] = float(st[fast].sum() / st.sum())
    out["cycle_share_slow_steps"] = float(st[slow].sum() / st.sum())
    return out


def measure(iters=(0, 30, 99), ants=(0, 511, 1023), workload="n5000_clustered"):
    import torch

    from . import binding as B
    B.lib()
    w = instances.WORKLOADS[workload]
    coords = instances.coords_for(w)
    n, m = w["n"], w["m"]
    ld = B.ld_of(n)
    prec = B.PREC[w["prec"]]
    st = torch.cuda.Stream()
    kw = dict(m=m, alpha=w["alpha"], beta=w["beta"], rho=w["rho"], Q=w["Q"], seed=w["seed"], prec=w["prec"])
    s = B.Solver(coords, stream=st, **kw)
    xy = torch.from_numpy(np.ascontiguousarray(coords)).cuda()
    H = torch.empty((n, ld), dtype=torch.float32, device="cuda")
    B.op_heuristic(xy, n, w["beta"], None, H, ld)
    P = torch.empty((n, ld), dtype=torch.float32 if prec == B.FP32 else torch.int16, device="cuda")
    lists = torch.empty((n, B.LIST_MAX, 2), dtype=torch.int32, device="cuda")
    lcnt = torch.empty(n, dtype=torch.int32, device="cuda")
    lkey = torch.empty(n, dtype=torch.int32, device="cuda")
    tours = torch.empty((m, n), dtype=torch.int32, device="cuda")
    probe = torch.zeros((n, 8), dtype=torch.int32, device="cuda")
    out = {"workload": workload, "n": n, "m": m, "prec": w["prec"], "ants": list(ants), "iterations": {}}
    done = 0
    for it in sorted(iters):
        s.iterate(it - done)
        done = it
        torch.cuda.synchronize()
        tau = torch.from_numpy(np.ascontiguousarray(s.tau())).cuda()
        taup = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
        taup[:, :n] = tau
        B.op_build_P(taup, H, n, ld, w["alpha"], 1.0, prec, P)
        B.op_build_lists(P, prec, n, ld, lists, lcnt, lkey)
        recs = []
        for a in ants:
            B.op_construct_probe(P, prec, n, ld, m, w["seed"], it, tours, lists, lkey, a, probe)
            torch.cuda.synchronize()
            recs.append(probe.cpu().numpy().view(np.uint32)[1:n].copy())
        s.iterate(1)
        done += 1
        torch.cuda.synchronize()
        assert np.array_equal(tours.cpu().numpy(), s.tours()), f"probed tours differ at iteration {it}"
        per = [_summary(r) for r in recs]
        agg = {k: float(np.mean([p[k] for p in per if p[k] is not None])) if any(p[k] is not None for p in per)
               else None for k in per[0]}
        out["iterations"][str(it)] = {"mean_over_ants": agg, "per_ant": per}
    s.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, nargs="+", default=[0, 30, 99])
    ap.add_argument("--ants", type=int, nargs="+", default=[0, 511, 1023])
    a = ap.parse_args()
    print(json.dumps(measure(a.iters, a.ants)))


if __name__ == "__main__":
    main()
