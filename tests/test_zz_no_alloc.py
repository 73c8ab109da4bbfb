"""The allocation-free deposit entry point (aco_op_deposit_tours_noalloc).

Some callers cannot allocate device memory where they update the pheromone:
embedders whose device memory all belongs to a framework pool or a budget
fixed at start-up, and loops with a latency bound, where cudaMalloc (which
may synchronise the device and has no bounded running time) is not allowed.
This entry point keeps its scratch in a fixed device array inside the
library.  Its results must equal those of the two allocating step-level
calls it replaces, aco_op_tour_length followed by aco_op_deposit, bit for bit
as every deterministic-path test here requires, on two calls in a row (the
second call reuses the scratch the first left), and the oracle's tour lengths
and deposit (Eq. 3, Sec. 2.3).

This file is collected last on purpose, so that a run stopping at the first
failure has run every other test first.
"""
import numpy as np
import pytest
import torch

from gpu_util import dev, host, padded_dev
from paper_2404_04895_gb300 import binding as B
from paper_2404_04895_gb300 import instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.lib()


def _case(n, m, seed):
    rng = np.random.default_rng(seed)
    xy = instances.uniform(n, seed)
    base = rng.permutation(n)
    tours = []
    for k in range(m):  # shared edges, as in a converging colony
        t = base.copy()
        if k % 2:
            i, j = sorted(rng.integers(0, n, size=2))
            t[i:j + 1] = t[i:j + 1][::-1]
        tours.append(t)
    tau0 = rng.uniform(0.5, 2.0, size=(n, n)).astype(np.float32)
    return xy, np.stack(tours).astype(np.int32), np.minimum(tau0, tau0.T)


def _reference(D, n, ld, tours, m, tau0, rho, Q):
    """The existing allocating path: explicit scratch buffers for c and nbr."""
    L = torch.empty(m, dtype=torch.float64, device="cuda")
    c = torch.empty(m, dtype=torch.float64, device="cuda")
    nbr = torch.empty((n, m, 2), dtype=torch.int32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    tau = padded_dev(tau0, ld, np.float32)
    B.op_tour_length(D, n, tours, m, Q, L, c, nbr)
    B.op_deposit(tau, n, ld, nbr, c, m, rho, err)
    return host(tau, n), host(L), int(err.item())


def test_noalloc_matches_allocating_path_on_two_calls(orc):
    results = []
    for call, (n, m, seed, rho, Q) in enumerate([(400, 300, 1, 0.1, 1.0), (257, 611, 2, 0.5, 3.0)]):
        xy, tours, tau0 = _case(n, m, seed)
        ld = B.ld_of(n)
        D = torch.empty((n, n), dtype=torch.float64, device="cuda")
        H = torch.empty((n, ld), dtype=torch.float32, device="cuda")
        B.op_heuristic(dev(xy), n, 2, D, H, ld)
        td = dev(tours)
        ref_tau, ref_L, ref_err = _reference(D, n, ld, td, m, tau0, rho, Q)
        tau = padded_dev(tau0, ld, np.float32)
        L = torch.full((m,), -1.0, dtype=torch.float64, device="cuda")
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        B.op_deposit_tours_noalloc(tau, n, ld, D, td, m, rho, Q, L, err)
        got_tau, got_L = host(tau, n), host(L)
        assert int(err.item()) == 0 and ref_err == 0, call
        assert np.array_equal(got_L, ref_L), call
        assert np.array_equal(got_tau.view(np.uint32), ref_tau.view(np.uint32)), call
        # and the oracle, from the coordinates up (Eq. 3, Sec. 2.3)
        Dr = orc.distances(xy)
        Lr = orc.tour_lengths(Dr, tours)
        assert np.array_equal(got_L, Lr), call
        want = orc.deposit(tau0, tours, Lr, rho, Q)
        assert np.array_equal(got_tau.view(np.uint32), want.view(np.uint32)), call
        results.append(got_tau)
    assert not np.array_equal(results[0][:257, :257], results[1])


def test_noalloc_reports_weights_it_cannot_sum():
    """Two tours whose lengths differ by 2^25: the weights Q / L span more
    than the fixed-point deposit holds.  The call sets the error word and
    every touched entry is NaN (never a silently unchanged pheromone)."""
    n, m = 16, 2
    rng = np.random.default_rng(5)
    ring = np.arange(n, dtype=np.int32)
    other = np.array([(3 * t) % n for t in range(0, n)], np.int32)   # a cycle over other edges (3 and 16 coprime)
    Dm = np.full((n, n), 2.0 ** -25)
    for t in range(n):
        a, b = ring[t], ring[(t + 1) % n]
        Dm[a, b] = Dm[b, a] = 1.0
    np.fill_diagonal(Dm, 0.0)
    tours = np.stack([ring, other])
    ld = B.ld_of(n)
    tau0 = rng.uniform(0.5, 2.0, size=(n, n)).astype(np.float32)
    tau = padded_dev(tau0, ld, np.float32)
    L = torch.zeros(m, dtype=torch.float64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.op_deposit_tours_noalloc(tau, n, ld, dev(Dm), dev(tours), m, 0.25, 1.0, L, err)
    got = host(tau, n)
    assert int(err.item()) == 2
    assert np.array_equal(host(L), [float(n), n * 2.0 ** -25])
    touched = np.zeros((n, n), bool)
    for p in tours:
        for t in range(n):
            touched[p[t], p[t - 1]] = touched[p[t - 1], p[t]] = True
    assert np.all(np.isnan(got[touched]))
    keep = np.float32(1) - np.float32(0.25)
    assert np.array_equal(got[~touched], (keep * tau0)[~touched])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    n, m = 5000, 1024  # 8*n*m = 40 MB > 16 MiB
    tau = torch.zeros((n, B.ld_of(n)), dtype=torch.float32, device="cuda")
    D = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    tours = torch.zeros((1, 8), dtype=torch.int32, device="cuda")
    L = torch.zeros(m, dtype=torch.float64, device="cuda")
    with pytest.raises(B.AcoError) as e:
        B.op_deposit_tours_noalloc(tau, n, B.ld_of(n), D, tours, m, 0.1, 1.0, L, None)
    assert e.value.code == B.ERR_ARG
    assert "scratch" in str(e.value)
