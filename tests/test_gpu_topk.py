"""GPU parity of the paper's deposit-path selection (Sec. 2.3: the solution
set sorted by fitness, the top k paths deposit) against the oracle: the
selection itself (ties broken by ant index), the selected deposit, whole
solver runs with k = n/10 (the paper's setting), and a batch instance."""
import numpy as np
import pytest
import torch

from gpu_util import dev, host, padded_dev
from paper_2404_04895_gb300 import binding as B
from paper_2404_04895_gb300 import instances

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m", [1, 7, 50, 1000, 5000, 70000])
def test_selection_matches_oracle(orc, m):
    rng = np.random.default_rng(m)
    L = rng.integers(1, 40, size=m).astype(np.float64) * 0.25  # many equal lengths
    if m > 3:
        L[: m // 3] = rng.uniform(0.5, 10, size=m // 3)
    for k in sorted({1, 2, max(1, m // 10), max(1, m - 1), m, m + 3, 0}):
        c = torch.ones(m, dtype=torch.float64, device="cuda")
        B.op_select_topk(dev(L), m, k, c)
        got = host(c) != 0
        assert np.array_equal(got, orc.select_topk(L, k)), (m, k)


@pytest.mark.parametrize("n,m,k", [(60, 40, 4), (300, 200, 30), (1000, 100, 1)])
def test_selected_deposit_matches_oracle(orc, n, m, k):
    xy = instances.uniform(n, 31)
    D = orc.distances(xy)
    rng = np.random.default_rng(n)
    tours = np.stack([rng.permutation(n) for _ in range(m)]).astype(np.int32)
    tau0 = rng.uniform(0.5, 2, size=(n, n)).astype(np.float32)
    ld = B.ld_of(n)
    L = torch.empty(m, dtype=torch.float64, device="cuda")
    c = torch.empty(m, dtype=torch.float64, device="cuda")
    nbr = torch.empty((n, m, 2), dtype=torch.int32, device="cuda")
    B.op_tour_length(dev(D), n, dev(tours), m, 1.0, L, c, nbr)
    B.op_select_topk(L, m, k, c)
    tau = padded_dev(tau0, ld, np.float32)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.op_deposit(tau, n, ld, nbr, c, m, 0.2, err)
    ref = orc.deposit_topk(tau0, tours, orc.tour_lengths(D, tours), 0.2, 1.0, k)
    assert int(err.item()) == 0
    assert np.array_equal(host(tau, n).view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("n,m", [(50, 50), (120, 120)])
def test_solver_top_n_over_10_bit_exact(orc, n, m):
    xy = instances.uniform(n, 41)
    kw = dict(m=m, alpha=1, beta=2, rho=0.1, Q=1.0, seed=3, topk=n // 10)
    g = B.Solver(xy, stream=torch.cuda.Stream(), **kw).iterate(30)
    ref = orc.State(xy, **kw).run(30)
    assert np.array_equal(g.tours(), ref.last_tours)
    assert np.array_equal(g.tau().view(np.uint32), ref.tau.view(np.uint32))
    tour, L = g.best()
    assert L == ref.best_len[0] and np.array_equal(tour, ref.best_tour)


def test_batch_instance_with_top_paths(orc):
    arena = 2 * B.instance_bytes(150, 80) + (1 << 20)
    bt = B.Batch(4, arena, stream=torch.cuda.Stream())
    xa, xb = instances.uniform(150, 5), instances.uniform(100, 6)
    a = bt.add(xa, 80, iters=9, rho=0.2, seed=7, topk=15)
    b = bt.add(xb, 60, iters=9, rho=0.2, seed=8)
    bt.step(9)
    for slot, xy, m, kw in [(a, xa, 80, dict(rho=0.2, seed=7, topk=15)), (b, xb, 60, dict(rho=0.2, seed=8))]:
        ref = orc.State(xy, m=m, **kw).run(9)
        tour, L = bt.best(slot)
        assert L == ref.best_len[0] and np.array_equal(tour, ref.best_tour)
        assert np.array_equal(bt.tau(slot).view(np.uint32), ref.tau.view(np.uint32))
    bt.close()


def test_global_api_topk(orc):
    xy = instances.uniform(40, 9)
    lib = B.lib()
    B.check(lib.aco_bind(None, 0, None))
    B.check(lib.aco_set_deposit_topk(4))
    try:
        B.check(lib.aco_init(np.ascontiguousarray(xy).ctypes.data, 40, 30, 1.0, 2.0, 0.3, 1.0, 2))
        B.check(lib.aco_iterate(12))
        tour = np.empty(40, np.int32)
        L = np.zeros(1, np.float64)
        B.check(lib.aco_best(tour.ctypes.data, L.ctypes.data))
        ref = orc.State(xy, m=30, rho=0.3, seed=2, topk=4).run(12)
        assert L[0] == ref.best_len[0] and np.array_equal(tour, ref.best_tour)
        assert lib.aco_set_deposit_topk(-1) != 0
    finally:
        B.check(lib.aco_set_deposit_topk(0))
        lib.aco_free()
