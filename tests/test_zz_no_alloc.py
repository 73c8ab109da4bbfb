"""The allocation-free deposit entry point (aco_op_deposit_tours_noalloc).

Callers that cannot allocate device memory at pheromone-update time (inside
stream capture, in loops that must not wait on the allocator, under a
framework-owned pool) use this entry point; it keeps its scratch in a fixed
device array inside the library.  Its results must equal those of the two
allocating step-level calls it replaces, aco_op_tour_length followed by
aco_op_deposit, bit for bit as every deterministic-path test here requires,
on two calls in a row (the second call reuses the scratch the first left).

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
    tau = padded_dev(tau0, ld, np.float32)
    B.op_tour_length(D, n, tours, m, Q, L, c, nbr)
    B.op_deposit(tau, n, ld, nbr, c, m, rho)
    return host(tau, n), host(L)


def test_noalloc_matches_allocating_path_on_two_calls():
    results = []
    for call, (n, m, seed, rho, Q) in enumerate([(400, 300, 1, 0.1, 1.0), (257, 611, 2, 0.5, 3.0)]):
        xy, tours, tau0 = _case(n, m, seed)
        ld = B.ld_of(n)
        D = torch.empty((n, n), dtype=torch.float64, device="cuda")
        H = torch.empty((n, ld), dtype=torch.float32, device="cuda")
        B.op_heuristic(dev(xy), n, 2, D, H, ld)
        td = dev(tours)
        ref_tau, ref_L = _reference(D, n, ld, td, m, tau0, rho, Q)
        tau = padded_dev(tau0, ld, np.float32)
        L = torch.full((m,), -1.0, dtype=torch.float64, device="cuda")
        B.op_deposit_tours_noalloc(tau, n, ld, D, td, m, rho, Q, L)
        got_tau, got_L = host(tau, n), host(L)
        assert np.array_equal(got_L, ref_L), call
        assert np.array_equal(got_tau.view(np.uint32), ref_tau.view(np.uint32)), call
        results.append(got_tau)
    assert not np.array_equal(results[0][:257, :257], results[1])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    n, m = 5000, 1024  # 8*n*m = 40 MB > 16 MiB
    tau = torch.zeros((n, B.ld_of(n)), dtype=torch.float32, device="cuda")
    D = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    tours = torch.zeros((1, 8), dtype=torch.int32, device="cuda")
    L = torch.zeros(m, dtype=torch.float64, device="cuda")
    with pytest.raises(B.AcoError) as e:
        B.op_deposit_tours_noalloc(tau, n, B.ld_of(n), D, tours, m, 0.1, 1.0, L)
    assert e.value.code == B.ERR_ARG
    assert "scratch" in str(e.value)
