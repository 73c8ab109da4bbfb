"""GPU parity of whole iterations through the C ABI solvers (handle API and the
single-instance aco_init / aco_iterate / aco_best API) against the oracle."""
import ctypes as C

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


def _same(gpu, ref):
    assert np.array_equal(gpu.tours(), ref.last_tours)
    assert np.array_equal(gpu.lengths(), ref.last_L)
    assert np.array_equal(gpu.tau().view(np.uint32), ref.tau.view(np.uint32))
    tour, L = gpu.best()
    assert L == ref.best_len[0] and np.array_equal(tour, ref.best_tour)


@pytest.mark.parametrize("graph", [False, True])
def test_plain_ant_system_n50_bit_exact(orc, graph):
    # 50 uniform cities, 50 ants, alpha 1, beta 2, rho 0.5, Q 1, 100 iterations, fp32, seed 0
    xy = instances.uniform(50, 1)
    kw = dict(m=50, alpha=1, beta=2, rho=0.5, Q=1.0, seed=0)
    stream = torch.cuda.Stream() if graph else None
    g = B.Solver(xy, stream=stream, **kw).iterate(100)
    ref = orc.State(xy, **kw).run(100)
    _same(g, ref)
    assert g.iteration == 100


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_low_precision_runs_bit_exact(orc, prec):
    xy = instances.clustered(8, 10, 0.02, seed=6)
    kw = dict(m=30, alpha=1, beta=2, rho=0.2, Q=1.0, seed=11)
    g = B.Solver(xy, prec=prec, stream=torch.cuda.Stream(), **kw).iterate(25)
    ref = orc.State(xy, prec=orc.BF16 if prec == "bf16" else orc.FP16, **kw).run(25)
    _same(g, ref)


def test_adair_schedule_run_bit_exact(orc):
    xy = instances.uniform(90, 2)
    kw = dict(m=40, alpha=1, beta=2, rho=0.1, Q=1.0, seed=5, gamma_max=1.5, gamma_min=0.5, gamma_T=30)
    g = B.Solver(xy, roulette="adair", stream=torch.cuda.Stream(), **kw).iterate(36)
    ref = orc.State(xy, adair=True, **kw).run(36)
    _same(g, ref)


def test_resume_across_calls_and_graph_equivalence(orc):
    xy = instances.uniform(64, 9)
    kw = dict(m=20, rho=0.3, seed=2)
    a = B.Solver(xy, stream=torch.cuda.Stream(), **kw).iterate(7).iterate(5).iterate(8)
    b = B.Solver(xy, **kw).iterate(20)
    assert np.array_equal(a.tau(), b.tau()) and np.array_equal(a.tours(), b.tours())
    assert a.best()[1] == b.best()[1]


def test_library_allocated_workspace(orc):
    xy = instances.uniform(40, 4)
    a = B.Solver(xy, m=10, workspace="library").iterate(10)
    ref = orc.State(xy, m=10).run(10)
    _same(a, ref)


def test_atomic_deposit_first_iteration_close(orc):
    xy = instances.uniform(300, 3)
    kw = dict(m=200, rho=0.1, seed=1)
    g = B.Solver(xy, deposit="atomic", **kw).iterate(1)
    ref = orc.State(xy, **kw).run(1)
    assert np.array_equal(g.tours(), ref.last_tours)
    got = g.tau().astype(np.float64)
    assert np.max(np.abs(got - ref.tau) / ref.tau) < 1e-5


def test_global_api(orc):
    L = B.lib()
    xy = instances.uniform(45, 12)
    B.check(L.aco_bind(None, 0, None))
    B.check(L.aco_set_precision(B.FP32))
    B.check(L.aco_set_deposit(B.DEPOSIT_DET))
    B.check(L.aco_set_variant(B.IR, 1.5, 0.5, 100))
    B.check(L.aco_init(xy.ctypes.data, 45, 17, 1.0, 2.0, 0.25, 2.0, 77))
    tour = np.zeros(45, np.int32)
    ln = np.zeros(1, np.float64)
    assert L.aco_best(tour.ctypes.data, ln.ctypes.data) == B.ERR_STATE
    B.check(L.aco_iterate(6))
    B.check(L.aco_iterate(0))
    B.check(L.aco_best(tour.ctypes.data, ln.ctypes.data))
    ref = orc.State(xy, m=17, rho=0.25, Q=2.0, seed=77).run(6)
    assert ln[0] == ref.best_len[0] and np.array_equal(tour, ref.best_tour)
    tau = np.zeros((45, 45), np.float32)
    B.check(L.aco_get_tau(tau.ctypes.data))
    assert np.array_equal(tau, ref.tau)
    tours = np.zeros((17, 45), np.int32)
    B.check(L.aco_get_tours(tours.ctypes.data))
    assert np.array_equal(tours, ref.last_tours)
    lens = np.zeros(17, np.float64)
    B.check(L.aco_get_lengths(lens.ctypes.data))
    assert np.array_equal(lens, ref.last_L)
    # bound torch workspace and stream
    nbytes = B.workspace_bytes(45, 17)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = torch.cuda.Stream()
    B.check(L.aco_bind(ws.data_ptr(), nbytes, st.cuda_stream))
    B.check(L.aco_init(xy.ctypes.data, 45, 17, 1.0, 2.0, 0.25, 2.0, 77))
    B.check(L.aco_iterate(6))
    B.check(L.aco_best(tour.ctypes.data, ln.ctypes.data))
    assert ln[0] == ref.best_len[0]
    B.check(L.aco_free())
    B.check(L.aco_bind(None, 0, None))


def test_invalid_arguments_return_codes():
    L = B.lib()
    xy = instances.uniform(10, 1)
    assert L.aco_init(xy.ctypes.data, 2, 5, 1.0, 2.0, 0.5, 1.0, 0) == B.ERR_ARG
    assert L.aco_init(xy.ctypes.data, 10, 0, 1.0, 2.0, 0.5, 1.0, 0) == B.ERR_ARG
    assert L.aco_init(xy.ctypes.data, 10, 5, 1.5, 2.0, 0.5, 1.0, 0) == B.ERR_UNSUPPORTED
    assert L.aco_init(xy.ctypes.data, 10, 5, 1.0, 2.0, 1.5, 1.0, 0) == B.ERR_ARG
    assert L.aco_init(None, 10, 5, 1.0, 2.0, 0.5, 1.0, 0) == B.ERR_ARG
    bad = xy.copy()
    bad[3, 1] = np.nan
    assert L.aco_init(bad.ctypes.data, 10, 5, 1.0, 2.0, 0.5, 1.0, 0) == B.ERR_ARG
    assert b"not finite" in L.aco_last_error()
    assert L.aco_set_precision(7) == B.ERR_ARG
    assert L.aco_free() == B.OK
    assert L.aco_iterate(1) == B.ERR_STATE
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    p = B.Params()
    B.check(L.aco_params_default(C.byref(p)))
    p.n, p.m = 10, 5
    h = C.c_void_p()
    assert L.aco_create(C.byref(h), xy.ctypes.data, C.byref(p), small.data_ptr(), 1024, None) == B.ERR_OOM
