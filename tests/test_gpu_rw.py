"""GPU parity of the roulette-wheel construction (Sec. 2.4, the selection
that independent roulette replaces; exact integer reading) against the
oracle: tours bit for bit at every storage precision, rows with zeros and
ties, whole solver runs, and the host-side limits."""
import numpy as np
import pytest
import torch

from gpu_util import P_device, dev, host
from paper_2404_04895_gb300 import binding as B
from paper_2404_04895_gb300 import instances

pytestmark = pytest.mark.gpu


def _P(orc, n, seed, prec, zeros=False, ties=False):
    xy = instances.clustered(-(-n // 40), 40, 0.02, seed=seed)[:n] if n >= 80 else instances.uniform(n, seed)
    H = orc.heuristic(orc.distances(xy), 2)
    tau = np.random.default_rng(seed).uniform(0.3, 2.0, size=(n, n)).astype(np.float32)
    if ties:
        tau[:] = 1.0
        H = np.where(H > np.median(H), np.float32(7.0), np.float32(3.0)).astype(np.float32)
        np.fill_diagonal(H, 0)
    if zeros:
        tau[:, ::3] = 0.0
    return orc.build_P(tau, H, 1, 1.0, prec)[:2]


@pytest.mark.parametrize("prec", [B.FP32, B.BF16, B.FP16])
@pytest.mark.parametrize("n,m,kind", [(5, 9, ""), (50, 40, ""), (333, 30, "zeros"), (1200, 24, ""),
                                      (700, 20, "ties"), (2001, 8, "")])
def test_rw_tours_bit_exact(orc, prec, n, m, kind):
    Pv, bits = _P(orc, n, 5 + n, prec, zeros=kind == "zeros", ties=kind == "ties")
    ld = B.ld_of(n)
    tours = torch.empty((m, n), dtype=torch.int32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.op_construct_rw(P_device(Pv, bits, prec, ld), prec, n, ld, m, 77, 3, tours, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert np.array_equal(host(tours), orc.construct_rw(Pv, 77, 3, 0, m))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_rw_solver_runs_bit_exact(orc, prec):
    xy = instances.uniform(80, 51)
    kw = dict(m=40, alpha=1, beta=2, rho=0.2, Q=1.0, seed=6)
    g = B.Solver(xy, prec=prec, roulette="rw", stream=torch.cuda.Stream(), **kw).iterate(15)
    ref = orc.State(xy, prec=orc.FP32 if prec == "fp32" else orc.BF16, rw=True, **kw).run(15)
    assert np.array_equal(g.tours(), ref.last_tours)
    assert np.array_equal(g.tau().view(np.uint32), ref.tau.view(np.uint32))
    tour, L = g.best()
    assert L == ref.best_len[0] and np.array_equal(tour, ref.best_tour)


def test_rw_limits():
    xy = instances.uniform(16385, 3)
    with pytest.raises(RuntimeError):
        B.Solver(xy, m=4, roulette="rw", workspace="library")
    bt = B.Batch(2, B.instance_bytes(60, 10) + (1 << 20))
    with pytest.raises(RuntimeError):                      # a size error, before the arena
        bt.add(xy, 4, roulette="rw")
    assert bt.add(instances.uniform(60, 4), 10, roulette="rw") is not None
    bt.close()
