"""ctypes/numpy wrappers over liboracle.so (test infrastructure only)."""
import ctypes as C
import math

import numpy as np

from .build import build as _build_lib

FP32, BF16, FP16 = 0, 1, 2

_lib = None


class OrcParams(C.Structure):
    _fields_ = [("n", C.c_int), ("m", C.c_int), ("alpha", C.c_int), ("beta", C.c_int),
                ("rho", C.c_float), ("Q", C.c_float), ("seed", C.c_uint64),
                ("prec", C.c_int), ("adair", C.c_int), ("gamma_max", C.c_float),
                ("gamma_min", C.c_float), ("gamma_T", C.c_int), ("topk", C.c_int), ("rw", C.c_int), ("tau_bf16", C.c_int)]


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build_lib())
        v, u32, u64, i32, f32, f64 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int32, C.c_float, C.c_double
        sig = {
            "orc_philox4x32_10": (None, [v, v, v]),
            "orc_draw": (u32, [u64, u32, u32, u32, u32]),
            "orc_uniform": (f32, [u32]),
            "orc_start_city": (i32, [u64, u32, u32, i32]),
            "orc_to_bf16": (C.c_uint16, [f32]),
            "orc_from_bf16": (f32, [C.c_uint16]),
            "orc_to_fp16": (C.c_uint16, [f32]),
            "orc_from_fp16": (f32, [C.c_uint16]),
            "orc_to_bf16_array": (None, [v, v, C.c_int64]),
            "orc_to_fp16_array": (None, [v, v, C.c_int64]),
            "orc_powi_f32": (f32, [f32, C.c_int]),
            "orc_powi_f64": (f64, [f64, C.c_int]),
            "orc_log2_own": (f32, [f32]),
            "orc_exp2_own": (f32, [f32]),
            "orc_pow_own": (f32, [f32, f32]),
            "orc_pow_own_array": (None, [v, f32, v, C.c_int64]),
            "orc_gamma": (f32, [C.c_int, C.c_int, f32, f32]),
            "orc_inv_gamma": (f32, [f32]),
            "orc_adair_deviate": (f64, [f64, f64]),
            "orc_distances": (None, [v, C.c_int, v]),
            "orc_heuristic": (None, [v, C.c_int, C.c_int, v]),
            "orc_build_P": (None, [v, v, C.c_int, C.c_int, f32, C.c_int, v, v, v]),
            "orc_construct": (None, [v, C.c_int, u64, u32, C.c_int, C.c_int, v, C.c_int]),
            "orc_select": (i32, [v, v, C.c_int, u64, u32, u32, u32]),
            "orc_select_literal_adair": (i32, [v, v, C.c_int, u64, u32, u32, u32, f64]),
            "orc_tour_lengths": (None, [v, C.c_int, v, C.c_int, v]),
            "orc_exact_sum": (f64, [v, C.c_int64]),
            "orc_exact_sum_f32": (C.c_float, [v, C.c_int64]),
            "orc_exact_sum_bf16": (C.c_float, [v, C.c_int64]),
            "orc_deposit_tau_bf16": (None, [v, C.c_int, v, v, C.c_int, C.c_float, C.c_float]),
            "orc_select_topk": (None, [v, C.c_int, C.c_int, v]),
            "orc_selection_counts": (None, [v, v, C.c_int, u64, u64, u32, v]),
            "orc_rw_quantum": (u64, [C.c_float, C.c_int]),
            "orc_select_rw": (i32, [v, v, C.c_int, u64, u32, u32, u32]),
            "orc_construct_rw": (None, [v, C.c_int, u64, u32, C.c_int, C.c_int, v, C.c_int]),
            "orc_deposit_topk": (None, [v, C.c_int, v, v, C.c_int, C.c_float, C.c_float, C.c_int]),
            "orc_index_matrix": (None, [v, C.c_int, v]),
            "orc_deposit": (None, [v, C.c_int, v, v, C.c_int, f32, f32]),
            "orc_deposit_fp32_order": (None, [v, C.c_int, v, v, C.c_int, f32, f32, v]),
            "orc_run": (None, [v, v, v, v, u32, C.c_int, v, v, v, v, C.c_int]),
            "orc_init_tau": (None, [v, C.c_int, f32]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def default_threads():
    import os
    return max(1, len(os.sched_getaffinity(0)))


# ---------------- random numbers ----------------
def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def draw(seed, it, k, t, j):
    return int(lib().orc_draw(seed, it, k, t, j))


def uniform(x):
    return float(lib().orc_uniform(x))


def start_city(seed, it, k, n):
    return int(lib().orc_start_city(seed, it, k, n))


# ---------------- rounding / elementary functions ----------------
def to_bf16(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.shape, dtype=np.uint16)
    lib().orc_to_bf16_array(_p(x), _p(out), x.size)
    return out


def to_fp16(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.shape, dtype=np.uint16)
    lib().orc_to_fp16_array(_p(x), _p(out), x.size)
    return out


def powi_f32(x, a):
    return float(lib().orc_powi_f32(x, a))


def powi_f64(x, a):
    return float(lib().orc_powi_f64(x, a))


def log2_own(x):
    return float(lib().orc_log2_own(x))


def exp2_own(y):
    return float(lib().orc_exp2_own(y))


def pow_own(x, e):
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty_like(x)
    lib().orc_pow_own_array(_p(x), e, _p(out), x.size)
    return out


def gamma(it, T, gmax, gmin):
    return float(lib().orc_gamma(it, T, gmax, gmin))


def inv_gamma(g):
    return float(lib().orc_inv_gamma(g))


def gamma_schedule(iters, T, gmax, gmin, it0=0):
    return np.array([gamma(it0 + i, T, gmax, gmin) for i in range(iters)], dtype=np.float32)


def adair_deviate(r, g):
    return float(lib().orc_adair_deviate(r, g))


# ---------------- the path ----------------
def distances(xy):
    xy = np.ascontiguousarray(xy, dtype=np.float32)
    n = xy.shape[0]
    D = np.empty((n, n), dtype=np.float64)
    lib().orc_distances(_p(xy), n, _p(D))
    return D


def heuristic(D, beta):
    D = np.ascontiguousarray(D, dtype=np.float64)
    n = D.shape[0]
    H = np.empty((n, n), dtype=np.float32)
    lib().orc_heuristic(_p(D), n, beta, _p(H))
    return H


def build_P(tau, H, alpha, inv_gamma=1.0, prec=FP32):
    """Returns (P_val fp32, P_bits uint16, row_exp int32)."""
    tau = np.ascontiguousarray(tau, dtype=np.float32)
    H = np.ascontiguousarray(H, dtype=np.float32)
    n = tau.shape[0]
    P = np.empty((n, n), dtype=np.float32)
    bits = np.zeros((n, n), dtype=np.uint16)
    rexp = np.zeros(n, dtype=np.int32)
    lib().orc_build_P(_p(tau), _p(H), n, alpha, inv_gamma, prec, _p(P), _p(bits), _p(rexp))
    return P, bits, rexp


def construct(P_val, seed, it, k_begin, k_end, nthreads=None):
    P_val = np.ascontiguousarray(P_val, dtype=np.float32)
    n = P_val.shape[0]
    tours = np.empty((k_end - k_begin, n), dtype=np.int32)
    lib().orc_construct(_p(P_val), n, seed, it, k_begin, k_end, _p(tours),
                        nthreads or default_threads())
    return tours


def select(row, visited, seed, it, k, t):
    row = np.ascontiguousarray(row, dtype=np.float32)
    vis = np.ascontiguousarray(visited, dtype=np.uint8)
    return int(lib().orc_select(_p(row), _p(vis), row.size, seed, it, k, t))


def select_literal_adair(row, visited, seed, it, k, t, g):
    row = np.ascontiguousarray(row, dtype=np.float32)
    vis = np.ascontiguousarray(visited, dtype=np.uint8)
    return int(lib().orc_select_literal_adair(_p(row), _p(vis), row.size, seed, it, k, t, g))


def tour_lengths(D, tours):
    D = np.ascontiguousarray(D, dtype=np.float64)
    tours = np.ascontiguousarray(tours, dtype=np.int32)
    m, n = tours.shape
    L = np.empty(m, dtype=np.float64)
    lib().orc_tour_lengths(_p(D), n, _p(tours), m, _p(L))
    return L


def exact_sum(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(lib().orc_exact_sum(_p(x), x.size))


def exact_sum_f32(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    return np.float32(lib().orc_exact_sum_f32(_p(x), x.size))


def exact_sum_bf16(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    return np.float32(lib().orc_exact_sum_bf16(_p(x), x.size))


def deposit_tau_bf16(tau, tours, L, rho, Q):
    tau = np.array(tau, dtype=np.float32, copy=True, order="C")
    tours = np.ascontiguousarray(tours, dtype=np.int32)
    L = np.ascontiguousarray(L, dtype=np.float64)
    m, n = tours.shape
    lib().orc_deposit_tau_bf16(_p(tau), n, _p(tours), _p(L), m, rho, Q)
    return tau


def index_matrix(tour):
    tour = np.ascontiguousarray(tour, dtype=np.int32)
    I = np.empty((tour.size, 2), dtype=np.int32)
    lib().orc_index_matrix(_p(tour), tour.size, _p(I))
    return I


def deposit(tau, tours, L, rho, Q):
    tau = np.array(tau, dtype=np.float32, copy=True, order="C")
    tours = np.ascontiguousarray(tours, dtype=np.int32)
    L = np.ascontiguousarray(L, dtype=np.float64)
    m, n = tours.shape
    lib().orc_deposit(_p(tau), n, _p(tours), _p(L), m, rho, Q)
    return tau


def rw_quantum(p, e):
    return int(lib().orc_rw_quantum(float(p), int(e)))


def select_rw(row, visited, seed, it, k, t):
    row = np.ascontiguousarray(row, dtype=np.float32)
    vis = np.ascontiguousarray(visited, dtype=np.uint8)
    return int(lib().orc_select_rw(_p(row), _p(vis), row.size, seed, it, k, t))


def construct_rw(P_val, seed, it, k_begin, k_end, nthreads=None):
    P_val = np.ascontiguousarray(P_val, dtype=np.float32)
    n = P_val.shape[0]
    tours = np.empty((k_end - k_begin, n), dtype=np.int32)
    lib().orc_construct_rw(_p(P_val), n, seed, it, k_begin, k_end, _p(tours), nthreads or default_threads())
    return tours


def selection_counts(q, trials, seed, salt=0, visited=None):
    q = np.ascontiguousarray(q, dtype=np.float32)
    vis = None if visited is None else np.ascontiguousarray(visited, dtype=np.uint8)
    counts = np.zeros(q.size, dtype=np.uint64)
    lib().orc_selection_counts(_p(q), None if vis is None else _p(vis), q.size, trials, seed, salt, _p(counts))
    return counts


def select_topk(L, k):
    L = np.ascontiguousarray(L, dtype=np.float64)
    sel = np.zeros(L.size, dtype=np.uint8)
    lib().orc_select_topk(_p(L), L.size, k, _p(sel))
    return sel.astype(bool)


def deposit_topk(tau, tours, L, rho, Q, k):
    tau = np.array(tau, dtype=np.float32, copy=True, order="C")
    tours = np.ascontiguousarray(tours, dtype=np.int32)
    L = np.ascontiguousarray(L, dtype=np.float64)
    m, n = tours.shape
    lib().orc_deposit_topk(_p(tau), n, _p(tours), _p(L), m, rho, Q, k)
    return tau


def deposit_fp32_order(tau, tours, L, rho, Q, perm=None):
    tau = np.array(tau, dtype=np.float32, copy=True, order="C")
    tours = np.ascontiguousarray(tours, dtype=np.int32)
    L = np.ascontiguousarray(L, dtype=np.float64)
    m, n = tours.shape
    pp = None
    if perm is not None:
        perm = np.ascontiguousarray(perm, dtype=np.int64)
        pp = _p(perm)
    lib().orc_deposit_fp32_order(_p(tau), n, _p(tours), _p(L), m, rho, Q, pp)
    return tau


def init_tau(n, tau0=1.0):
    tau = np.empty((n, n), dtype=np.float32)
    lib().orc_init_tau(_p(tau), n, tau0)
    return tau


class State:
    """Oracle solver state: tau, best tour / length, iteration counter."""

    def __init__(self, xy, m, alpha=1, beta=2, rho=0.5, Q=1.0, seed=0, prec=FP32,
                 adair=False, gamma_max=1.5, gamma_min=0.5, gamma_T=100, tau0=1.0, topk=0,
                 rw=False, tau_bf16=False):
        self.xy = np.ascontiguousarray(xy, dtype=np.float32)
        n = self.xy.shape[0]
        self.prm = OrcParams(n=n, m=m, alpha=alpha, beta=beta, rho=rho, Q=Q, seed=seed,
                             prec=prec, adair=int(adair), gamma_max=gamma_max,
                             gamma_min=gamma_min, gamma_T=gamma_T, topk=topk, rw=int(rw),
                             tau_bf16=int(tau_bf16))
        self.D = distances(self.xy)
        self.H = heuristic(self.D, beta)
        self.tau = init_tau(n, tau0)
        if tau_bf16:  # tau0 stored in bfloat16
            self.tau = (to_bf16(self.tau).astype(np.uint32) << 16).view(np.float32).reshape(n, n)
        self.it = 0
        self.best_tour = np.zeros(n, dtype=np.int32)
        self.best_len = np.array([math.inf], dtype=np.float64)
        self.last_tours = np.zeros((m, n), dtype=np.int32)
        self.last_L = np.zeros(m, dtype=np.float64)

    def inv_gamma_at(self, it):
        if not self.prm.adair:
            return 1.0
        return inv_gamma(gamma(it, self.prm.gamma_T, self.prm.gamma_max, self.prm.gamma_min))

    def run(self, iters, nthreads=None):
        lib().orc_run(C.byref(self.prm), _p(self.D), _p(self.H), _p(self.tau), self.it, iters,
                      _p(self.best_tour), _p(self.best_len), _p(self.last_tours),
                      _p(self.last_L), nthreads or default_threads())
        self.it += iters
        return self
