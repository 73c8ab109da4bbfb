"""The C-ABI library builds, loads without a GPU, and exports every function
declared in include/tensoraco.h (no compute calls here)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tensoraco.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(aco_[A-Za-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2404_04895_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_path():
    names = declared_functions()
    for required in ["aco_init", "aco_iterate", "aco_best", "aco_free", "aco_op_build_P",
                     "aco_op_construct", "aco_op_tour_length", "aco_op_deposit",
                     "aco_op_deposit_atomic", "aco_create", "aco_solver_iterate"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2404_04895_gb300 import binding
    assert set(declared_functions()) <= set(binding.exported_symbols())


def test_error_text_without_gpu(lib):
    lib.aco_last_error.restype = ctypes.c_char_p
    lib.aco_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_size_t)]
    out = ctypes.c_size_t(0)
    assert lib.aco_workspace_bytes(2, 10, 0, ctypes.byref(out)) == -1     # n < 3
    assert b"out of range" in lib.aco_last_error()
    assert lib.aco_workspace_bytes(5000, 1024, 0, ctypes.byref(out)) == 0
    assert out.value > 5000 * 5000 * 8


def test_gamma_schedule_matches_oracle(lib, orc):
    # the host-side schedule the solvers upload is the oracle's, bit for bit
    lib.aco_gamma.restype = ctypes.c_float
    lib.aco_gamma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_float]
    lib.aco_inv_gamma.restype = ctypes.c_float
    lib.aco_inv_gamma.argtypes = [ctypes.c_float]
    for T in (1, 7, 100, 200):
        for it in range(T + 3):
            g = lib.aco_gamma(it, T, 1.5, 0.5)
            assert g == orc.gamma(it, T, 1.5, 0.5)
            assert lib.aco_inv_gamma(g) == orc.inv_gamma(g)


def test_list_sizes_match_header_and_are_enforced():
    import re
    import numpy as np
    from paper_2404_04895_gb300 import binding as B
    text = open(os.path.join(ROOT, "include", "tensoraco.h")).read()
    assert int(re.search(r"#define ACO_LIST_MAX (\d+)", text).group(1)) == B.LIST_MAX
    assert int(re.search(r"#define ACO_LIST_TARGET (\d+)", text).group(1)) == B.LIST_TARGET
    n = 50
    ok = (np.zeros((n, B.LIST_MAX, 2), np.int32), np.zeros(n, np.int32), np.zeros(n, np.uint32))
    B._check_lists(n, *ok)
    with pytest.raises(ValueError):
        B._check_lists(n, np.zeros((n, B.LIST_MAX // 2, 2), np.int32), ok[1], ok[2])
    with pytest.raises(ValueError):
        B._check_lists(n, ok[0], np.zeros(n - 1, np.int32), ok[2])


def test_sizes_no_kernel_serves_are_refused_at_creation(lib):
    """Solvers beyond the construction kernels' limits (fp32 M_p above
    ACO_MAX_N_FP32, the roulette wheel above ACO_MAX_N_RW) are refused by
    aco_create before any device work; the binding's limits are the header's."""
    import numpy as np
    from paper_2404_04895_gb300 import binding as B
    text = open(os.path.join(ROOT, "include", "tensoraco.h")).read()
    for name, val in [("ACO_MAX_N", B.MAX_N), ("ACO_MAX_N_FP32", B.MAX_N_FP32),
                      ("ACO_MAX_N_FP32_BATCH", B.MAX_N_FP32_BATCH), ("ACO_MAX_N_RW", B.MAX_N_RW)]:
        assert int(re.search(rf"#define {name} (\d+)", text).group(1)) == val
    L = B.lib()
    for prec, n, rou, want in [(B.FP32, B.MAX_N_FP32 + 1, B.IR, B.ERR_UNSUPPORTED),
                               (B.FP32, B.MAX_N_FP32 + 1, B.ADAIR, B.ERR_UNSUPPORTED),
                               (B.BF16, B.MAX_N_RW + 1, B.RW, B.ERR_UNSUPPORTED),
                               (B.BF16, B.MAX_N + 1, B.IR, B.ERR_ARG)]:
        p = B.make_params(n, 1, prec=prec, roulette=rou)
        xy = np.zeros((n, 2), np.float32)
        h = ctypes.c_void_p()
        assert L.aco_create(ctypes.byref(h), xy.ctypes.data, ctypes.byref(p), None, 0, None) == want
        assert h.value is None


def test_create_refuses_each_invalid_parameter_before_device_work(lib):
    """aco_create checks every field of aco_params (and the coordinates)
    against the header's ranges before it touches the device: each invalid
    value returns its documented code with a message and no handle."""
    import numpy as np
    from paper_2404_04895_gb300 import binding as B
    L = B.lib()
    n = 10
    cases = [("n", 2, B.ERR_ARG), ("n", B.MAX_N + 1, B.ERR_ARG), ("m", 0, B.ERR_ARG),
             ("m", (1 << 20) + 1, B.ERR_ARG), ("alpha", 9, B.ERR_UNSUPPORTED), ("beta", -1, B.ERR_UNSUPPORTED),
             ("rho", -0.1, B.ERR_ARG), ("rho", 1.5, B.ERR_ARG), ("rho", float("nan"), B.ERR_ARG),
             ("Q", 0.0, B.ERR_ARG), ("Q", float("inf"), B.ERR_ARG), ("tau0", -1.0, B.ERR_ARG),
             ("topk", -1, B.ERR_ARG), ("tau_prec", B.FP16, B.ERR_UNSUPPORTED), ("prec", 3, B.ERR_ARG),
             ("roulette", 3, B.ERR_ARG), ("deposit", 2, B.ERR_ARG)]
    xy = np.random.default_rng(0).random((B.MAX_N + 1, 2)).astype(np.float32)

    def create(p):
        h = ctypes.c_void_p()
        rc = L.aco_create(ctypes.byref(h), xy.ctypes.data, ctypes.byref(p), None, 0, None)
        assert h.value is None
        return rc

    for field, value, want in cases:
        p = B.make_params(n, 5)
        setattr(p, field, value)
        assert create(p) == want, (field, value)
        assert L.aco_last_error(), field
    p = B.make_params(n, 5, tau_prec="bf16", deposit="atomic")   # bf16 tau needs the exact deposit
    assert create(p) == B.ERR_UNSUPPORTED
    for gmax, gmin, T in [(0.0, 0.5, 10), (1.5, 17.0, 10), (1.5, 0.5, 0)]:
        p = B.make_params(n, 5, roulette="adair", gamma_max=gmax, gamma_min=gmin, gamma_T=T)
        assert create(p) == B.ERR_ARG, (gmax, gmin, T)
    bad = xy.copy()
    bad[3, 1] = np.nan                                             # a coordinate that is not finite
    h = ctypes.c_void_p()
    assert L.aco_create(ctypes.byref(h), bad.ctypes.data, ctypes.byref(B.make_params(n, 5)), None, 0,
                        None) == B.ERR_ARG
    assert L.aco_create(ctypes.byref(h), None, ctypes.byref(B.make_params(n, 5)), None, 0, None) == B.ERR_ARG


def test_calls_refuse_null_buffers_and_handles_before_device_work(lib):
    """Every step-level call refuses a NULL device buffer, and the handle
    calls a NULL handle, with ACO_ERR_ARG; the single-instance calls before
    aco_init answer ACO_ERR_STATE.  Each case fails its checks before any
    launch, so this runs on the CPU."""
    from paper_2404_04895_gb300 import binding as B
    L = B.lib()
    N = None
    ops = [
        ("aco_op_heuristic", (N, 10, 2, N, N, 16, N)),
        ("aco_op_fill", (N, 10, 16, 1.0, N)),
        ("aco_op_build_P", (N, N, 10, 16, 1, 1.0, B.FP32, N, N)),
        ("aco_op_construct", (N, B.FP32, 10, 16, 4, 0, 0, N, N, N)),
        ("aco_op_construct_rw", (N, B.FP32, 10, 16, 4, 0, 0, N, N, N)),
        ("aco_op_construct_shape", (N, B.FP32, 10, 16, 4, 0, 0, N, N, 1, 1, 1, N)),
        ("aco_op_build_lists", (N, B.FP32, 10, 16, N, N, N, N)),
        ("aco_op_construct_ex", (N, B.FP32, 10, 16, 4, 0, 0, N, N, N, N, N, 0, 0, 0, N)),
        ("aco_op_tour_length", (N, 10, N, 4, 1.0, N, N, N, N)),
        ("aco_op_best", (N, N, 10, 4, N, N, N)),
        ("aco_op_deposit", (N, 10, 16, N, N, 4, 0.5, N, N)),
        ("aco_op_deposit_atomic", (N, 10, 16, N, N, 4, 0.5, N)),
        ("aco_op_deposit_tours_noalloc", (N, 10, 16, N, N, 4, 0.5, 1.0, N, N, N)),
        ("aco_op_select_topk", (N, 4, 2, N, N)),
        ("aco_op_selection_counts", (N, N, 10, 100, 0, 0, N, N)),
        ("aco_op_philox", (N, 0, N, 4, N)),
        ("aco_op_pow_own", (N, 0.5, N, 4, N)),
        ("aco_solver_iterate", (N, 1)),
        ("aco_solver_best", (N, N, N)),
        ("aco_solver_get_tau", (N, N)),
        ("aco_solver_set_shape", (N, 1, 1, 1)),
        ("aco_batch_add", (N, N, N, 1, N)),
        ("aco_batch_step", (N, 1)),
        ("aco_batch_best", (N, 0, N, N)),
        ("aco_batch_remove", (N, 0)),
    ]
    for name, args in ops:
        assert getattr(L, name)(*args) == B.ERR_ARG, name
        assert L.aco_last_error(), name
    assert L.aco_destroy(None) == B.OK            # destroying nothing is allowed
    assert L.aco_iterate(1) == B.ERR_STATE
    assert L.aco_best(N, N) == B.ERR_STATE
