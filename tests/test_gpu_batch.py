"""Batches of independent instances (multi-instance kernels, persistent
construction launch, graph replay) give every instance exactly the results
a standalone solver gives it, whatever else is in the batch."""
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


SIZES = [(13, 7), (50, 50), (130, 64), (257, 100), (600, 40), (1000, 33)]


def _alone(xy, m, iters, prec, **kw):
    s = B.Solver(xy, m=m, prec=prec, stream=torch.cuda.Stream(), **kw).iterate(iters)
    out = s.best(), s.tau()
    s.close()
    return out


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_batch_matches_standalone_solvers(prec):
    arena = sum(B.instance_bytes(n, m) for n, m in SIZES) + (1 << 20)
    bt = B.Batch(16, arena, prec=prec, stream=torch.cuda.Stream())
    slots = {}
    for q, (n, m) in enumerate(SIZES):
        xy = instances.uniform(n, 500 + q)
        kw = dict(rho=0.2, seed=q, roulette="adair" if q % 2 else "ir", gamma_T=12)
        slots[q] = (bt.add(xy, m, iters=12, **kw), xy, m, kw)
    bt.step(15)  # more than every budget: finished instances stop advancing
    for q, (slot, xy, m, kw) in slots.items():
        it, fin = bt.status(slot)
        assert it == 12 and fin
        (tour, L), tau = _alone(xy, m, 12, prec, **kw)
        bt_tour, bt_L = bt.best(slot)
        assert bt_L == L and np.array_equal(bt_tour, tour), q
        assert np.array_equal(bt.tau(slot).view(np.uint32), tau.view(np.uint32)), q
    bt.close()


def test_batch_membership_changes_and_oracle(orc):
    arena = 3 * B.instance_bytes(200, 60) + (1 << 20)
    bt = B.Batch(4, arena, stream=torch.cuda.Stream())
    xa, xb, xc = instances.uniform(200, 1), instances.uniform(150, 2), instances.uniform(90, 3)
    a = bt.add(xa, 60, iters=10, rho=0.3, seed=4)
    bt.step(3)
    b = bt.add(xb, 40, iters=0, rho=0.1, seed=5)   # joins mid-run, no budget
    bt.step(4)
    c = bt.add(xc, 25, iters=5, rho=0.5, seed=6)
    bt.step(8)
    assert bt.status(a) == (10, True)
    assert bt.status(b) == (12, False)
    assert bt.status(c) == (5, True)
    for slot, xy, m, it, kw in [(a, xa, 60, 10, dict(rho=0.3, seed=4)),
                                (b, xb, 40, 12, dict(rho=0.1, seed=5)),
                                (c, xc, 25, 5, dict(rho=0.5, seed=6))]:
        ref = orc.State(xy, m=m, **kw).run(it)
        tour, L = bt.best(slot)
        assert L == ref.best_len[0] and np.array_equal(tour, ref.best_tour)
        assert np.array_equal(bt.tau(slot), ref.tau)
    bt.close()


def test_batch_memory_gated_admission():
    one = B.instance_bytes(300, 50)
    bt = B.Batch(8, 2 * one + 512, stream=torch.cuda.Stream())
    s1 = bt.add(instances.uniform(300, 1), 50, iters=2)
    s2 = bt.add(instances.uniform(300, 2), 50, iters=2)
    assert s1 is not None and s2 is not None
    assert bt.add(instances.uniform(300, 3), 50, iters=2) is None      # arena full
    info = bt.info()
    assert info["active"] == 2 and info["free_bytes"] < one
    bt.remove(s1)
    s3 = bt.add(instances.uniform(300, 3), 50, iters=2)                # fits again
    assert s3 is not None
    bt.step(2)
    assert bt.status(s2) == (2, True) and bt.status(s3) == (2, True)
    bt.close()


# (n, m, roulette): roulette-wheel instances lead, sit inside and trail the
# batch's n-descending order
MIXED = [(300, 20, "rw"), (257, 30, "ir"), (130, 40, "rw"), (100, 25, "adair"), (64, 33, "ir"), (40, 16, "rw")]


@pytest.mark.parametrize("case", ["lists", "classes", "rw_only"])
def test_batch_mixes_roulette_wheel_instances(orc, case):
    """Roulette-wheel instances (Sec. 2.4; their own multi-instance kernel,
    one CTA per ant) beside IR and AdaIR ones: on the candidate-list path, on
    size classes (IR instances without lists) and alone, every instance ends
    with a standalone solver's results, and a roulette-wheel instance with the
    oracle's."""
    sizes = [x for x in MIXED if case != "rw_only" or x[2] == "rw"]
    arena = sum(B.instance_bytes(n, m) for n, m, _ in sizes) + (1 << 20)
    bt = B.Batch(8, arena, stream=torch.cuda.Stream())
    slots = []
    for q, (n, m, rou) in enumerate(sizes):
        xy = instances.uniform(n, 900 + q)
        kw = dict(rho=0.25, seed=20 + q, roulette=rou, gamma_T=9, cand_lists=case != "classes")
        slots.append((bt.add(xy, m, iters=9, **kw), xy, m, kw))
    bt.step(11)
    for slot, xy, m, kw in slots:
        assert bt.status(slot) == (9, True)
        (tour, L), tau = _alone(xy, m, 9, "fp32", **kw)
        bt_tour, bt_L = bt.best(slot)
        assert bt_L == L and np.array_equal(bt_tour, tour), kw
        assert np.array_equal(bt.tau(slot).view(np.uint32), tau.view(np.uint32)), kw
    slot, xy, m, kw = next(s for s in slots if s[3]["roulette"] == "rw" and s[2] == 40)
    ref = orc.State(xy, m=m, rho=kw["rho"], seed=kw["seed"], rw=True).run(9)
    tour, L = bt.best(slot)
    assert L == ref.best_len[0] and np.array_equal(tour, ref.best_tour)
    assert np.array_equal(bt.tau(slot), ref.tau)
    bt.close()


def test_batch_over_the_batched_workloads_size_range(orc):
    """24 instances drawn like the batched workload (uniform cities, n from
    100 to 2000, m = n, rho 0.1, bf16 M_p), the largest at n = 2000: after 3
    batched iterations the largest and a mid-size instance equal the oracle's
    whole runs (tours of the last iteration, tau, best) bit for bit."""
    sizes = [int(x) for x in instances.batch_sizes(24, 100, 2000, seed=8)]
    sizes[0] = 2000
    arena = sum(B.instance_bytes(n, n) for n in sizes) + (16 << 20)
    bt = B.Batch(len(sizes), arena, prec="bf16", stream=torch.cuda.Stream())
    slots = [bt.add(instances.uniform(n, 1000 + i), n, iters=0, rho=0.1, seed=i) for i, n in enumerate(sizes)]
    assert all(sl is not None for sl in slots)
    bt.step(3)
    mid = int(np.argsort(sizes)[len(sizes) // 2])
    for i in (0, mid):
        n = sizes[i]
        ref = orc.State(instances.uniform(n, 1000 + i), n, rho=0.1, seed=i, prec=orc.BF16).run(3)
        tour, L = bt.best(slots[i])
        assert L == ref.best_len[0] and np.array_equal(tour, ref.best_tour), (i, n)
        assert np.array_equal(bt.tau(slots[i]).view(np.uint32), ref.tau.view(np.uint32)), (i, n)
    bt.close()
