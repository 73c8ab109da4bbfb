"""Seeded synthetic TSP instances.

Holds input generation only (coordinates, instance mixes, arrival traces) and
none of the ACO arithmetic; both the GPU tests and the oracle tests draw their
inputs from here.  The paper evaluates on TSPLIB instances (u159 ... pr2392)
and on cities spread over sizes 100 .. 50,000; these generators stand in for
them with the same size range:

  uniform(n, seed)      n cities i.i.d. uniform in [0,1]^2, fp32
  clustered(...)        n_clusters centres uniform in [0,1]^2, per_cluster
                        points each at centre + N(0, sigma^2) per axis (fp64
                        draw, rounded to fp32), cluster by cluster
  batch_sizes(...)      instance sizes drawn uniformly from [lo, hi]
  poisson_trace(...)    arrival times of solve requests (exponential gaps)
                        with sizes log-uniform in [lo, hi]
"""
import numpy as np


def uniform(n, seed):
    rng = np.random.default_rng(seed)
    return rng.random((n, 2)).astype(np.float32)


def clustered(n_clusters=50, per_cluster=100, sigma=0.02, seed=3):
    rng = np.random.default_rng(seed)
    centres = rng.random((n_clusters, 2))
    pts = centres[:, None, :] + sigma * rng.standard_normal((n_clusters, per_cluster, 2))
    return pts.reshape(-1, 2).astype(np.float32)


def batch_sizes(count=256, lo=100, hi=2000, seed=7):
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=count).astype(np.int64)


def poisson_trace(count=200, rate=50.0, lo=50, hi=10000, seed=11):
    """Returns (arrival_seconds float64[count], sizes int64[count])."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps) - gaps[0]
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count)).round().astype(np.int64)
    return t, np.clip(sizes, lo, hi)


def line_geometric(n, ratio=3.0, scale=0.1):
    """Cities on the x axis with gaps scale * ratio^i (i = 0..n-2)."""
    x = np.concatenate([[0.0], np.cumsum(scale * ratio ** np.arange(n - 1))])
    return np.stack([x, np.zeros_like(x)], axis=1).astype(np.float32)


# The workloads the benchmark and the full-size parity tests use.
WORKLOADS = {
    "n50_ir": dict(kind="uniform", n=50, coord_seed=1, m=50, alpha=1, beta=2, rho=0.5,
                   Q=1.0, iters=100, adair=False, prec="fp32", seed=0),
    "n1000_adair": dict(kind="uniform", n=1000, coord_seed=2, m=1000, alpha=1, beta=2,
                        rho=0.1, Q=1.0, iters=200, adair=True, prec="fp32", seed=0),
    "n5000_clustered": dict(kind="clustered", n=5000, coord_seed=3, m=1024, alpha=1,
                            beta=2, rho=0.1, Q=1.0, iters=100, adair=False, prec="fp32",
                            seed=0),
}


def coords_for(w):
    if w["kind"] == "uniform":
        return uniform(w["n"], w["coord_seed"])
    return clustered(seed=w["coord_seed"])
