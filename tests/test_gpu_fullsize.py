"""GPU parity at the benchmark workloads' full sizes, in the solvers' launch
configuration (CUDA graph, candidate lists, the default shape).  The oracle
rebuilds a chosen iteration from the GPU's own pheromone state: every ant's
tour (Sec. 2.2, 2.4), every tour length (Eq. 3) and the deposit of that
iteration (Sec. 2.3), element by element, bit for bit.  Late iterations are
included: there the lists decide almost every step and the rare fallback
paths are the ones exercised."""
import numpy as np
import pytest
import torch

from paper_2404_04895_gb300 import binding as B
from paper_2404_04895_gb300 import instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.lib()


def _check_iteration(orc, coords, w, prec, run_iters, sample_ants=None, nthreads=None):
    """Run run_iters iterations on the GPU, then one more; check that iteration's
    tours (every ant, or sample_ants) and its deposit against the oracle
    started from the GPU's tau."""
    kw = dict(m=w["m"], alpha=w["alpha"], beta=w["beta"], rho=w["rho"], Q=w["Q"], seed=w["seed"],
              prec=prec, roulette="adair" if w["adair"] else "ir")
    if w["adair"]:
        kw.update(gamma_max=1.5, gamma_min=0.5, gamma_T=w["iters"])
    s = B.Solver(coords, stream=torch.cuda.Stream(), **kw)
    s.iterate(run_iters)
    tau_before = s.tau()
    s.iterate(1)
    tours = s.tours()
    lengths = s.lengths()
    tau_after = s.tau()
    it = run_iters
    n = coords.shape[0]
    # every tour is a permutation
    srt = np.sort(tours, axis=1)
    assert np.array_equal(srt, np.broadcast_to(np.arange(n, dtype=np.int32), srt.shape))
    # sampled ants against the oracle
    D = orc.distances(coords)
    H = orc.heuristic(D, w["beta"])
    inv = 1.0
    if w["adair"]:
        inv = orc.inv_gamma(orc.gamma(it, w["iters"], 1.5, 0.5))
    pid = {"fp32": orc.FP32, "bf16": orc.BF16, "fp16": orc.FP16}[prec]
    P, _, _ = orc.build_P(tau_before, H, w["alpha"], inv, pid)
    if sample_ants is None:
        ref = orc.construct(P, w["seed"], it, 0, w["m"], nthreads)
        bad = np.flatnonzero((ref != tours).any(axis=1))
        assert bad.size == 0, (prec, it, bad[:10].tolist())
    else:
        for k in sample_ants:
            ref = orc.construct(P, w["seed"], it, k, k + 1, nthreads)
            assert np.array_equal(tours[k], ref[0]), (prec, it, k)
    # lengths and the deposit of this iteration
    assert np.array_equal(lengths, orc.tour_lengths(D, tours))
    ref_tau = orc.deposit(tau_before, tours, lengths, w["rho"], w["Q"])
    assert np.array_equal(tau_after.view(np.uint32), ref_tau.view(np.uint32))
    s.close()


def test_n1000_adair_full_trajectory_start(orc):
    # 1000 uniform cities, 1000 ants, AdaIR: the first 2 iterations in full
    w = instances.WORKLOADS["n1000_adair"]
    coords = instances.coords_for(w)
    kw = dict(m=w["m"], alpha=1, beta=2, rho=w["rho"], Q=1.0, seed=w["seed"], gamma_max=1.5,
              gamma_min=0.5, gamma_T=w["iters"])
    g = B.Solver(coords, roulette="adair", stream=torch.cuda.Stream(), **kw).iterate(2)
    ref = orc.State(coords, adair=True, **kw).run(2)
    assert np.array_equal(g.tours(), ref.last_tours)
    assert np.array_equal(g.tau().view(np.uint32), ref.tau.view(np.uint32))
    assert g.best()[1] == ref.best_len[0]


def test_n1000_adair_last_iteration_every_ant(orc):
    # iteration 199, the last of the workload's budget (gamma at its minimum)
    w = instances.WORKLOADS["n1000_adair"]
    _check_iteration(orc, instances.coords_for(w), w, "fp32", 199)


@pytest.mark.parametrize("it", [3, 99])
@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_n5000_clustered_every_ant(orc, prec, it):
    # all 1024 ants of iteration 3 and of iteration 99 (the last of the budget)
    w = instances.WORKLOADS["n5000_clustered"]
    _check_iteration(orc, instances.coords_for(w), w, prec, it)


def test_n50_plain_all_iterations(orc):
    # the small workload end to end: every iteration's state
    w = instances.WORKLOADS["n50_ir"]
    coords = instances.coords_for(w)
    kw = dict(m=w["m"], rho=w["rho"], seed=w["seed"])
    g = B.Solver(coords, stream=torch.cuda.Stream(), **kw)
    ref = orc.State(coords, **kw)
    for _ in range(w["iters"] // 10):
        g.iterate(10)
        ref.run(10, nthreads=1)
        assert np.array_equal(g.tours(), ref.last_tours)
        assert np.array_equal(g.tau(), ref.tau)
        assert g.best()[1] == ref.best_len[0]
