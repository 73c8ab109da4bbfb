"""The largest n the candidate-list (lean) and roulette-wheel construction
kernels serve: 16384 cities, where the staged row and the visited flags
take 80 KB of shared memory per CTA and every thread of the roulette wheel
weighs its widest column block.  The tours equal the oracle's."""
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
