"""M_tau stored in bfloat16: whole runs bit-exact with the oracle's bf16
reading (the exact deposit sum rounded once to bf16), checkpoints, and the
combinations that are refused."""
import numpy as np
import pytest
import torch

from paper_2404_04895_gb300 import binding as B
from paper_2404_04895_gb300 import instances

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kw,oracle_kw", [
    (dict(m=50, rho=0.5, seed=0), {}),
    (dict(m=60, rho=0.1, seed=4, topk=6), {}),
    (dict(m=40, rho=0.2, seed=8, prec="bf16"), dict(prec=1)),
    (dict(m=45, rho=0.1, seed=2, roulette="adair", gamma_T=30), dict(adair=True)),
])
def test_tau_bf16_runs_bit_exact(orc, kw, oracle_kw):
    xy = instances.uniform(120, 71)
    g = B.Solver(xy, tau_prec="bf16", stream=torch.cuda.Stream(), **kw).iterate(30)
    okw = {k: v for k, v in kw.items() if k not in ("prec", "roulette")}
    ref = orc.State(xy, tau_bf16=True, **okw, **oracle_kw).run(30)
    tau = g.tau()
    assert np.all((tau.view(np.uint32) & 0xFFFF) == 0)          # bf16 values
    assert np.array_equal(tau.view(np.uint32), ref.tau.view(np.uint32))
    assert np.array_equal(g.tours(), ref.last_tours)
    tour, L = g.best()
    assert L == ref.best_len[0] and np.array_equal(tour, ref.best_tour)


def test_tau_bf16_checkpoint_resume():
    xy = instances.uniform(90, 72)
    kw = dict(m=30, rho=0.2, seed=5, tau_prec="bf16")
    st = torch.cuda.Stream()
    whole = B.Solver(xy, stream=st, **kw).iterate(16)
    part = B.Solver(xy, stream=st, **kw).iterate(8)
    again = B.Solver(xy, stream=st, **kw).restore(part.state()).iterate(8)
    assert np.array_equal(again.tau().view(np.uint32), whole.tau().view(np.uint32))
    assert again.best()[1] == whole.best()[1]


def test_tau_bf16_refusals():
    xy = instances.uniform(60, 73)
    with pytest.raises(B.AcoError):
        B.Solver(xy, m=10, tau_prec="bf16", deposit="atomic")
    with pytest.raises(B.AcoError):
        B.Solver(xy, m=10, tau_prec="fp16")
    bt = B.Batch(2, B.instance_bytes(60, 10) + (1 << 20))
    with pytest.raises(B.AcoError):
        bt.add(xy, 10, tau_prec="fp16")
    bt.close()


def test_tau_bf16_in_batches_matches_standalone():
    """Instances storing M_tau in bf16 and in fp32, side by side in one batch,
    end exactly where standalone solvers (themselves pinned to the oracle
    above) end."""
    st = torch.cuda.Stream()
    cases = [(90, 30, dict(rho=0.2, seed=1, tau_prec="bf16")),
             (70, 25, dict(rho=0.3, seed=2)),
             (110, 40, dict(rho=0.1, seed=3, tau_prec="bf16", roulette="adair", gamma_T=10))]
    arena = sum(B.instance_bytes(n, m) for n, m, _ in cases) + (1 << 20)
    bt = B.Batch(4, arena, stream=st)
    slots = []
    for q, (n, m, kw) in enumerate(cases):
        xy = instances.uniform(n, 80 + q)
        slots.append((bt.add(xy, m, iters=10, **kw), xy, m, kw))
    bt.step(10)
    for slot, xy, m, kw in slots:
        s = B.Solver(xy, m=m, stream=st, **kw).iterate(10)
        tau = bt.tau(slot)
        assert np.array_equal(tau.view(np.uint32), s.tau().view(np.uint32))
        if kw.get("tau_prec") == "bf16":
            assert np.all((tau.view(np.uint32) & 0xFFFF) == 0)
        tour, L = s.best()
        bt_tour, bt_L = bt.best(slot)
        assert bt_L == L and np.array_equal(bt_tour, tour)
        s.close()
    bt.close()
