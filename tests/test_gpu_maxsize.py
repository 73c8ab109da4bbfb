"""The largest n each construction kernel serves.  The candidate-list (lean)
and roulette-wheel kernels: 16384 cities, where the staged row and the
visited flags take 80 KB of shared memory per CTA and every thread of the
roulette wheel weighs its widest column block; their tours equal the
oracle's.  The full-scan kernel: 49152 fp32 columns (a 192 KB staged row)
and 65536 bf16 columns, checked on sampled steps; and sizes beyond the
kernels are refused when a batch instance is added."""
import numpy as np
import pytest
import torch

from gpu_util import P_device, host
from paper_2404_04895_gb300 import binding as B

pytestmark = pytest.mark.gpu

N_MAX = 16384


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.lib()


@pytest.fixture(scope="module")
def rows():
    """M_p rows with the wide value spread of (1/d)^2 heuristics: log-uniform
    over 12 binades, zero diagonal; fp32 and its bf16 truncation."""
    rng = np.random.default_rng(16384)
    v = np.exp2(rng.uniform(-12.0, 0.0, size=(N_MAX, N_MAX)).astype(np.float32))
    np.fill_diagonal(v, 0.0)
    bits = (v.view(np.uint32) >> 16).astype(np.uint16)
    vb = (bits.astype(np.uint32) << 16).view(np.float32)
    return {B.FP32: (v, None), B.BF16: (vb, bits)}


@pytest.mark.parametrize("prec", [B.FP32, B.BF16])
def test_lean_construction_at_max_n(orc, rows, prec):
    Pv, bits = rows[prec]
    ld = B.ld_of(N_MAX)
    Pd = P_device(Pv, bits, prec, ld)
    lists = torch.zeros((N_MAX, B.LIST_MAX, 2), dtype=torch.int32, device="cuda")
    lcnt = torch.zeros(N_MAX, dtype=torch.int32, device="cuda")
    lkey = torch.zeros(N_MAX, dtype=torch.int32, device="cuda")
    B.op_build_lists(Pd, prec, N_MAX, ld, lists, lcnt, lkey)
    m = 2
    t = torch.zeros((m, N_MAX), dtype=torch.int32, device="cuda")
    B.op_construct_ex(Pd, prec, N_MAX, ld, m, 3, 1, t, lists, lcnt, lkey, shape=(1, 0, 2))
    assert np.array_equal(host(t), orc.construct(Pv, 3, 1, 0, m))


@pytest.mark.parametrize("prec", [B.FP32, B.BF16])
def test_roulette_wheel_at_max_n(orc, rows, prec):
    Pv, bits = rows[prec]
    ld = B.ld_of(N_MAX)
    Pd = P_device(Pv, bits, prec, ld)
    m = 2
    tours = torch.empty((m, N_MAX), dtype=torch.int32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.op_construct_rw(Pd, prec, N_MAX, ld, m, 4, 2, tours, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert np.array_equal(host(tours), orc.construct_rw(Pv, 4, 2, 0, m))


@pytest.mark.parametrize("prec,n", [(B.FP32, B.MAX_N_FP32), (B.BF16, B.MAX_N)])
def test_full_scan_construction_at_largest_n(orc, prec, n):
    """M_p drawn on the device (uniform, zero diagonal), default shape: both
    tours are permutations from the oracle's start city, and sampled steps
    (the first, the last, the middle and random ones) equal the oracle's
    selection on the same row and visited set."""
    g = torch.Generator(device="cuda")
    g.manual_seed(n)
    P = torch.rand((n, n), generator=g, device="cuda")
    P.fill_diagonal_(0.0)
    if prec == B.BF16:
        P = P.to(torch.bfloat16)
    m, seed, it = 2, 12, 3
    tours = torch.empty((m, n), dtype=torch.int32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.op_construct(P, prec, n, n, m, seed, it, tours, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    t = host(tours)
    rng = np.random.default_rng(n)
    for k in range(m):
        assert np.array_equal(np.sort(t[k]), np.arange(n, dtype=np.int32))
        assert t[k, 0] == orc.start_city(seed, it, k, n)
        steps = {1, 2, 3, n // 2, n - 3, n - 2, n - 1, *rng.integers(4, n - 3, size=8).tolist()}
        for st in sorted(steps):
            row = P[int(t[k, st - 1])].float().cpu().numpy()
            vis = np.zeros(n, np.uint8)
            vis[t[k, :st]] = 1
            assert orc.select(row, vis, seed, it, k, st) == t[k, st], (k, st)
    del P
    torch.cuda.empty_cache()


def test_batch_refuses_sizes_its_kernels_do_not_serve():
    bt = B.Batch(2, B.instance_bytes(60, 10) + (1 << 20), prec="fp32")
    with pytest.raises(B.AcoError) as e:
        bt.add(np.zeros((B.MAX_N_FP32_BATCH + 1, 2), np.float32), 2)
    assert e.value.code == B.ERR_UNSUPPORTED
    assert bt.info()["active"] == 0
    bt.close()
