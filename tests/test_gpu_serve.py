"""Continuous batching on the GPU: requests that arrive while others run are
admitted as memory frees up and share batched steps, and every request's
result equals the result of solving it alone, bit for bit."""
import numpy as np
import pytest
import torch

from paper_2404_04895_gb300 import binding as B
from paper_2404_04895_gb300 import serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.lib()


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_served_results_equal_solo_results(prec):
    reqs = serve.poisson_requests(14, 400.0, 20, 400, 15, mmax=48, seed=5, rho=0.2)
    arena = 3 * B.instance_bytes(400, 48) + (1 << 20)   # a few requests at a time
    gb = serve.GpuBatch(arena, 16, prec)
    done, wall, steps = serve.Server(gb).run(reqs, realtime=True)
    gb.close()
    assert sorted(r.rid for r in done) == list(range(14))
    assert steps < sum(r.iters for r in done)            # requests shared steps
    for r in done:
        s = B.Solver(r.coords, m=r.m, prec=prec, seed=r.seed, rho=0.2, stream=torch.cuda.Stream())
        tour, L = s.iterate(r.iters).best()
        s.close()
        assert r.best_len == L and np.array_equal(r.tour, tour), r.rid
    stats = serve.summarize(done, wall)
    assert stats["latency_p99_s"] >= stats["latency_p50_s"] > 0


def test_large_request_in_a_mix_equals_its_solo_run():
    """A request of 5000 cities (m = 1024) served beside smaller ones that
    arrive while it runs gives the result of solving it alone, bit for bit."""
    from paper_2404_04895_gb300 import instances
    sizes = [5000, 300, 1200, 64, 700]
    reqs = []
    for i, n in enumerate(sizes):
        reqs.append(serve.Request(rid=i, arrival=0.003 * i, coords=instances.uniform(n, 900 + i),
                                  m=min(n, 1024), seed=40 + i, iters=6 + (i % 3), params=dict(rho=0.1)))
    arena = sum(B.instance_bytes(n, min(n, 1024)) for n in sizes) + (16 << 20)
    gb = serve.GpuBatch(arena, 8, "bf16")
    done, wall, steps = serve.Server(gb).run(reqs, realtime=True)
    gb.close()
    assert sorted(r.rid for r in done) == list(range(len(sizes)))
    assert steps < sum(r.iters for r in done)
    for r in done:
        s = B.Solver(r.coords, m=r.m, prec="bf16", seed=r.seed, rho=0.1, stream=torch.cuda.Stream())
        tour, L = s.iterate(r.iters).best()
        s.close()
        assert r.best_len == L and np.array_equal(r.tour, tour), r.rid


def test_device_batches_on_one_gpu_equal_solo_runs():
    """The multi-device placement path (one batch per device, each instance
    on the device with the most free arena memory) with two batches on this
    one GPU: requests spread over both, and every result equals the request
    solved alone, bit for bit -- as it does with one batch."""
    reqs = serve.poisson_requests(10, 400.0, 30, 500, 8, mmax=40, seed=9, rho=0.2)
    arena = 3 * B.instance_bytes(500, 40) + (1 << 20)
    db = serve.DeviceBatches([serve.GpuBatch(arena, 8, "bf16", device=0), serve.GpuBatch(arena, 8, "bf16", device=0)])
    placed = []
    add = db.add

    def add_logged(*a, **kw):
        s = add(*a, **kw)
        if s is not None:
            placed.append(s[0])
        return s

    db.add = add_logged
    done, wall, steps = serve.Server(db).run(reqs, realtime=True)
    db.close()
    assert sorted(r.rid for r in done) == list(range(10))
    assert set(placed) == {0, 1}                          # both batches served requests
    for r in done:
        s = B.Solver(r.coords, m=r.m, prec="bf16", seed=r.seed, rho=0.2, stream=torch.cuda.Stream())
        tour, L = s.iterate(r.iters).best()
        s.close()
        assert r.best_len == L and np.array_equal(r.tour, tour), r.rid
