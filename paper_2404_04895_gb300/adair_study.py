"""The AdaIR visualisation study (Sec. 3.3.1, Fig. 4 of the paper), on
synthetic instances and on the GPU.

Rows of the transition matrix M_p are sampled while a solver runs.  For the
city with the largest probability in a row, the study compares

  p_max        its roulette-wheel probability, p_max / sum of the row, and
  p_hat'_max   how often independent roulette (gamma = 1) and AdaIR
               (gamma > 1) pick it, over m x 10,000 Bernoulli trials
               (aco_op_selection_counts on the row raised to 1/gamma, as the
               path computes AdaIR),

next to the exact probability of that event under the IR law,
int_0^1 prod_{i != max} min(1, x q_max / q_i) dx with q = p^(1/gamma).  The
paper reports that the maximum's probability is first shifted to a higher
value and then approaches the roulette-wheel one as the colony converges.

  python -m paper_2404_04895_gb300.adair_study --n 100 422 --iters 0 5 20 100

prints one JSON line per (instance, iteration, gamma), averaged over the
sampled rows.
"""
import argparse
import json
import math

import numpy as np

from . import instances


def ir_law_max(q):
    """Exact probability that the largest entry of q wins argmax(r_j q_j)
    with r_j i.i.d. uniform on (0, 1).  With b_i = q_i / q_max sorted
    ascending, on [b_k, b_(k+1)] the first k factors are saturated (= 1) and
    the rest give x^(n-1-k) / prod_{i > k} b_i; integrated in log space."""
    q = np.asarray(q, dtype=np.float64)
    q = q[q > 0]
    if q.size <= 1:
        return 1.0
    jm = int(np.argmax(q))
    b = np.sort(np.delete(q, jm) / q[jm])          # in (0, 1]
    n1 = b.size
    logb = np.log(b)
    suffix = np.concatenate([np.cumsum(logb[::-1])[::-1], [0.0]])  # sum_{i >= k} log b_i
    total = 0.0
    lo = 0.0
    for k in range(n1 + 1):
        hi = b[k] if k < n1 else 1.0
        e = n1 - k                                   # unsaturated factors on [lo, hi]
        if hi > lo:
            if e == 0:
                total += hi - lo
            else:
                # (hi^(e+1) - lo^(e+1)) / ((e+1) prod_{i >= k} b_i)
                lhi = (e + 1) * math.log(hi) - suffix[k] - math.log(e + 1)
                term = math.exp(lhi)
                if lo > 0:
                    term -= math.exp((e + 1) * math.log(lo) - suffix[k] - math.log(e + 1))
                total += term
        lo = hi
    return total


def _rows_p(B, torch, xy, tau, beta, alpha=1):
    """M_p = tau^alpha * eta^beta on the device (fp32), via the library's kernels."""
    n = xy.shape[0]
    ld = B.ld_of(n)
    H = torch.empty((n, ld), dtype=torch.float32, device="cuda")
    B.op_heuristic(torch.from_numpy(np.ascontiguousarray(xy)).cuda(), n, beta, None, H, ld)
    T = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
    T[:, :n] = torch.from_numpy(tau).cuda()
    P = torch.empty_like(H)
    B.op_build_P(T, H, n, ld, alpha, 1.0, B.FP32, P)
    return P


def run(n_list=(100, 422), iters=(0, 1, 2, 5, 10, 20, 50, 100), gammas=(1.0, 1.5, 2.0), rows=8,
        trials_per_ant=10_000, rho=0.1, seed=0):
    import torch

    from . import binding as B
    B.lib()
    out = []
    for n in n_list:
        m = n
        xy = instances.uniform(n, 900 + n)
        s = B.Solver(xy, m=m, rho=rho, seed=seed, stream=torch.cuda.Stream())
        done = 0
        rng = np.random.default_rng(n)
        cities = rng.choice(n, size=rows, replace=False)
        for it in sorted(set(iters)):  # the solver only moves forward
            s.iterate(it - done)
            done = it
            P = _rows_p(B, torch, xy, s.tau(), beta=2)
            trials = m * trials_per_ant
            for g in gammas:
                recs = []
                for r, i in enumerate(cities):
                    p = P[int(i), :n].contiguous()
                    vis = torch.zeros(n, dtype=torch.uint8, device="cuda")
                    vis[int(i)] = 1
                    q = torch.empty_like(p)
                    B.op_pow_own(p, float(np.float32(1.0 / g)), q, n)
                    counts = torch.zeros(n, dtype=torch.int64, device="cuda")
                    B.op_selection_counts(q, n, trials, seed + 7919 * it + r, counts, salt=int(i), visited=vis)
                    ph = p.cpu().numpy().astype(np.float64)
                    ph[int(i)] = 0.0
                    qh = q.cpu().numpy().astype(np.float64)
                    qh[int(i)] = 0.0
                    jm = int(np.argmax(ph))
                    c = counts.cpu().numpy()
                    recs.append((ph[jm] / ph.sum(), c[jm] / trials, ir_law_max(qh)))
                a = np.array(recs)
                out.append({"n": n, "m": m, "iteration": it, "gamma": g, "rows": rows, "trials_per_row": trials,
                            "p_max_rw": round(float(a[:, 0].mean()), 5),
                            "p_hat_max": round(float(a[:, 1].mean()), 5),
                            "p_max_ir_law": round(float(a[:, 2].mean()), 5),
                            "max_abs_hat_minus_law": round(float(np.abs(a[:, 1] - a[:, 2]).max()), 5)})
        s.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, nargs="+", default=[100, 422])
    ap.add_argument("--iters", type=int, nargs="+", default=[0, 1, 2, 5, 10, 20, 50, 100])
    ap.add_argument("--gammas", type=float, nargs="+", default=[1.0, 1.5, 2.0])
    ap.add_argument("--rows", type=int, default=8)
    ap.add_argument("--trials-per-ant", type=int, default=10_000)
    a = ap.parse_args()
    for rec in run(a.n, a.iters, a.gammas, a.rows, a.trials_per_ant):
        print(json.dumps(rec), flush=True)


if __name__ == "__main__":
    main()
