"""ctypes binding over libtensoraco.so (include/tensoraco.h): argument
marshalling only -- every step of the ACO path runs in the library's CUDA
kernels.  There is no fallback: if the library is missing or fails to load,
calls raise."""
import ctypes as C
import os

import numpy as np

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_STATE, ERR_UNSUPPORTED, ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
FP32, BF16, FP16 = 0, 1, 2
IR, ADAIR, RW = 0, 1, 2
DEPOSIT_DET, DEPOSIT_ATOMIC = 0, 1
MAX_N = 65536
MAX_N_FP32, MAX_N_FP32_BATCH, MAX_N_RW = 49152, 32768, 16384   # construction limits of tensoraco.h
WAIT_POLLS_DEFAULT = 1048576

PREC = {"fp32": FP32, "bf16": BF16, "fp16": FP16}
ROULETTE = {"ir": IR, "adair": ADAIR, "rw": RW}
DEPOSIT = {"det": DEPOSIT_DET, "atomic": DEPOSIT_ATOMIC}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtensoraco.so")


class AcoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tensoraco error {code}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("n", C.c_int), ("m", C.c_int), ("alpha", C.c_int), ("beta", C.c_int),
                ("rho", C.c_float), ("Q", C.c_float), ("tau0", C.c_float),
                ("seed", C.c_uint64), ("prec", C.c_int), ("roulette", C.c_int),
                ("deposit", C.c_int), ("gamma_max", C.c_float), ("gamma_min", C.c_float),
                ("gamma_T", C.c_int), ("cand_lists", C.c_int), ("topk", C.c_int),
                ("tau_prec", C.c_int)]


_lib = None
v, i32, u32, u64, f32, sz = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64, C.c_float, C.c_size_t
_SIGS = {
    "aco_last_error": (C.c_char_p, []),
    "aco_init": (i32, [v, i32, i32, f32, f32, f32, f32, u64]),
    "aco_set_variant": (i32, [i32, f32, f32, i32]),
    "aco_set_precision": (i32, [i32]),
    "aco_set_deposit": (i32, [i32]),
    "aco_set_deposit_topk": (i32, [i32]),
    "aco_set_tau_precision": (i32, [i32]),
    "aco_op_select_topk": (i32, [v, i32, i32, v, v]),
    "aco_op_selection_counts": (i32, [v, v, i32, C.c_ulonglong, u64, u32, v, v]),
    "aco_iterate": (i32, [i32]),
    "aco_best": (i32, [v, v]),
    "aco_get_tau": (i32, [v]),
    "aco_get_tours": (i32, [v]),
    "aco_get_lengths": (i32, [v]),
    "aco_free": (i32, []),
    "aco_workspace_bytes": (i32, [i32, i32, i32, C.POINTER(sz)]),
    "aco_bind": (i32, [v, sz, v]),
    "aco_params_default": (i32, [C.POINTER(Params)]),
    "aco_create": (i32, [C.POINTER(v), v, C.POINTER(Params), v, sz, v]),
    "aco_destroy": (i32, [v]),
    "aco_solver_iterate": (i32, [v, i32]),
    "aco_solver_best": (i32, [v, v, v]),
    "aco_solver_get_tau": (i32, [v, v]),
    "aco_solver_get_tours": (i32, [v, v]),
    "aco_solver_get_lengths": (i32, [v, v]),
    "aco_solver_device_state": (i32, [v, C.POINTER(v), C.POINTER(i32), C.POINTER(v), C.POINTER(v),
                                      C.POINTER(v), C.POINTER(v)]),
    "aco_solver_iteration": (i32, [v, C.POINTER(u32)]),
    "aco_solver_state_bytes": (i32, [v, v]),
    "aco_solver_save": (i32, [v, v, sz]),
    "aco_solver_load": (i32, [v, v, sz]),
    "aco_solver_set_profiling": (i32, [v, i32]),
    "aco_solver_kernel_ms": (i32, [v, v]),
    "aco_solver_set_shape": (i32, [v, i32, i32, i32]),
    "aco_solver_set_wait_polls": (i32, [v, u32]),
    "aco_op_construct_probe": (i32, [v, i32, i32, i32, i32, u64, u32, v, v, v, v, i32, v, v]),
    "aco_op_build_P_lists": (i32, [v, v, i32, i32, i32, f32, f32, i32, v, v, v, v, v]),
    "aco_ceiling_row_reads": (i32, [v, sz, i32, i32, i32, u32, v, v]),
    "aco_ceiling_philox": (i32, [u64, i32, i32, u32, v, v]),
    "aco_ceiling_chase": (i32, [v, sz, i32, i32, v, v, v]),
    "aco_autotune_construct": (i32, [v, i32, i32, i32, i32, u64, v, i32, C.POINTER(i32),
                                     C.POINTER(i32), C.POINTER(i32), C.POINTER(f32), v]),
    "aco_batch_create": (i32, [C.POINTER(v), i32, sz, i32, v, v]),
    "aco_batch_destroy": (i32, [v]),
    "aco_batch_add": (i32, [v, v, C.POINTER(Params), i32, C.POINTER(i32)]),
    "aco_batch_remove": (i32, [v, i32]),
    "aco_batch_step": (i32, [v, i32]),
    "aco_batch_best": (i32, [v, i32, v, v]),
    "aco_batch_get_tau": (i32, [v, i32, v]),
    "aco_batch_status": (i32, [v, i32, C.POINTER(u32), C.POINTER(i32)]),
    "aco_batch_info": (i32, [v, C.POINTER(i32), C.POINTER(sz), C.POINTER(sz)]),
    "aco_batch_set_shape": (i32, [v, i32, i32, i32]),
    "aco_batch_instance_bytes": (i32, [i32, i32, C.POINTER(sz)]),
    "aco_op_heuristic": (i32, [v, i32, i32, v, v, i32, v]),
    "aco_op_fill": (i32, [v, i32, i32, f32, v]),
    "aco_op_build_P": (i32, [v, v, i32, i32, i32, f32, i32, v, v]),
    "aco_op_construct": (i32, [v, i32, i32, i32, i32, u64, u32, v, v, v]),
    "aco_op_construct_rw": (i32, [v, i32, i32, i32, i32, u64, u32, v, v, v]),
    "aco_op_construct_shape": (i32, [v, i32, i32, i32, i32, u64, u32, v, v, i32, i32, i32, v]),
    "aco_op_build_lists": (i32, [v, i32, i32, i32, v, v, v, v]),
    "aco_op_construct_ex": (i32, [v, i32, i32, i32, i32, u64, u32, v, v, v, v, v, i32, i32, i32, v]),
    "aco_op_tour_length": (i32, [v, i32, v, i32, f32, v, v, v, v]),
    "aco_op_best": (i32, [v, v, i32, i32, v, v, v]),
    "aco_op_deposit": (i32, [v, i32, i32, v, v, i32, f32, v, v]),
    "aco_op_deposit_atomic": (i32, [v, i32, i32, v, v, i32, f32, v]),
    "aco_op_deposit_tours_noalloc": (i32, [v, i32, i32, v, v, i32, f32, f32, v, v, v]),
    "aco_op_philox": (i32, [v, u64, v, i32, v]),
    "aco_op_pow_own": (i32, [v, f32, v, i32, v]),
    "aco_gamma": (f32, [i32, i32, f32, f32]),
    "aco_inv_gamma": (f32, [f32]),
}


def lib():
    """Load libtensoraco.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def check(rc):
    if rc != OK:
        raise AcoError(rc, lib().aco_last_error().decode())
    return rc


def call(name, *args):
    return check(getattr(lib(), name)(*args))


def ptr(x):
    """Device or host address of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream or None


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


# ---------------------------------------------------------------- step-level calls
def op_heuristic(coords, n, beta, D, H, ld, stream=None):
    call("aco_op_heuristic", ptr(coords), n, beta, ptr(D), ptr(H), ld, stream_ptr(stream))


def op_fill(a, n, ld, value, stream=None):
    call("aco_op_fill", ptr(a), n, ld, value, stream_ptr(stream))


def op_build_P(tau, H, n, ld, alpha, inv_gamma, prec, P, stream=None):
    call("aco_op_build_P", ptr(tau), ptr(H), n, ld, alpha, inv_gamma, prec, ptr(P), stream_ptr(stream))


def op_construct(P, prec, n, ld, m, seed, it, tours, err=None, shape=None, stream=None):
    if shape is None:
        call("aco_op_construct", ptr(P), prec, n, ld, m, seed, it, ptr(tours), ptr(err), stream_ptr(stream))
    else:
        call("aco_op_construct_shape", ptr(P), prec, n, ld, m, seed, it, ptr(tours), ptr(err),
             shape[0], shape[1], shape[2], stream_ptr(stream))


LIST_TARGET, LIST_MAX = 256, 512   # ACO_LIST_TARGET, ACO_LIST_MAX of tensoraco.h


def _check_lists(n, lists, lcnt, lkey):
    """Refuse list buffers smaller than the library writes or reads."""
    for name, t, need in (("lists", lists, n * LIST_MAX * 8), ("lcnt", lcnt, n * 4), ("lkey", lkey, n * 4)):
        if t is None or isinstance(t, int):
            continue
        size = t.numel() * t.element_size() if hasattr(t, "element_size") else t.nbytes
        if size < need:
            raise ValueError(f"{name} holds {size} bytes; n={n} needs {need}")


def op_build_lists(P, prec, n, ld, lists, lcnt, lkey, stream=None):
    _check_lists(n, lists, lcnt, lkey)
    call("aco_op_build_lists", ptr(P), prec, n, ld, ptr(lists), ptr(lcnt), ptr(lkey), stream_ptr(stream))


def op_build_P_lists(tau, H, n, ld, alpha, inv_gamma, rho, prec, P, lists, lcnt, lkey, stream=None):
    _check_lists(n, lists, lcnt, lkey)
    call("aco_op_build_P_lists", ptr(tau), ptr(H), n, ld, alpha, inv_gamma, rho, prec, ptr(P), ptr(lists),
         ptr(lcnt), ptr(lkey), stream_ptr(stream))


def op_construct_rw(P, prec, n, ld, m, seed, it, tours, err=None, stream=None):
    call("aco_op_construct_rw", ptr(P), prec, n, ld, m, seed, it, ptr(tours), ptr(err), stream_ptr(stream))


def op_construct_ex(P, prec, n, ld, m, seed, it, tours, lists=None, lcnt=None, lkey=None, err=None,
                    shape=(0, 0, 0), stream=None):
    if lists is not None:
        _check_lists(n, lists, lcnt, lkey)
    call("aco_op_construct_ex", ptr(P), prec, n, ld, m, seed, it, ptr(tours), ptr(err), ptr(lists),
         ptr(lcnt), ptr(lkey), shape[0], shape[1], shape[2], stream_ptr(stream))


def op_tour_length(D, n, tours, m, Q, L, c=None, nbr=None, stream=None):
    call("aco_op_tour_length", ptr(D), n, ptr(tours), m, Q, ptr(L), ptr(c), ptr(nbr), stream_ptr(stream))


def op_best(L, tours, n, m, best_tour, best_len, stream=None):
    call("aco_op_best", ptr(L), ptr(tours), n, m, ptr(best_tour), ptr(best_len), stream_ptr(stream))


def op_deposit(tau, n, ld, nbr, c, m, rho, err=None, stream=None):
    call("aco_op_deposit", ptr(tau), n, ld, ptr(nbr), ptr(c), m, rho, ptr(err) if err is not None else None,
         stream_ptr(stream))


def op_selection_counts(q, n, trials, seed, counts, salt=0, visited=None, stream=None):
    call("aco_op_selection_counts", ptr(q), ptr(visited), n, trials, seed, salt, ptr(counts), stream_ptr(stream))


def op_select_topk(L, m, k, c, stream=None):
    call("aco_op_select_topk", ptr(L), m, k, ptr(c), stream_ptr(stream))


def op_deposit_atomic(tau, n, ld, tours, c, m, rho, stream=None):
    call("aco_op_deposit_atomic", ptr(tau), n, ld, ptr(tours), ptr(c), m, rho, stream_ptr(stream))


def op_deposit_tours_noalloc(tau, n, ld, D, tours, m, rho, Q, L, err=None, stream=None):
    call("aco_op_deposit_tours_noalloc", ptr(tau), n, ld, ptr(D), ptr(tours), m, rho, Q, ptr(L),
         ptr(err), stream_ptr(stream))


NOALLOC_SCRATCH_BYTES = 16 << 20


def op_construct_probe(P, prec, n, ld, m, seed, it, tours, lists, lkey, probe_ant, probe, err=None, stream=None):
    call("aco_op_construct_probe", ptr(P), prec, n, ld, m, seed, it, ptr(tours), ptr(err), ptr(lists), ptr(lkey),
         probe_ant, ptr(probe), stream_ptr(stream))


def ceiling_row_reads(buf, nbytes, row_bytes, warps, rows_per_warp, salt, sink, stream=None):
    call("aco_ceiling_row_reads", ptr(buf), nbytes, row_bytes, warps, rows_per_warp, salt, ptr(sink),
         stream_ptr(stream))


def ceiling_philox(seed, threads, blocks_per_thread, salt, sink, stream=None):
    call("aco_ceiling_philox", seed, threads, blocks_per_thread, salt, ptr(sink), stream_ptr(stream))


def ceiling_chase(nxt, slots, chains, hops, cycles, sink, stream=None):
    call("aco_ceiling_chase", ptr(nxt), slots, chains, hops, ptr(cycles), ptr(sink), stream_ptr(stream))


def op_philox(ctr, seed, out, count, stream=None):
    call("aco_op_philox", ptr(ctr), seed, ptr(out), count, stream_ptr(stream))


def op_pow_own(x, e, out, count, stream=None):
    call("aco_op_pow_own", ptr(x), e, ptr(out), count, stream_ptr(stream))


def autotune_construct(P, prec, n, ld, m, seed, tours_scratch, reps=3, stream=None):
    w, c, md, ms = i32(0), i32(0), i32(0), f32(0)
    call("aco_autotune_construct", ptr(P), prec, n, ld, m, seed, ptr(tours_scratch), reps,
         C.byref(w), C.byref(c), C.byref(md), C.byref(ms), stream_ptr(stream))
    return (w.value, c.value, md.value), ms.value


def gamma(it, T, gmax, gmin):
    return float(lib().aco_gamma(it, T, gmax, gmin))


def inv_gamma(g):
    return float(lib().aco_inv_gamma(g))


def workspace_bytes(n, m, prec=FP32):
    out = sz(0)
    call("aco_workspace_bytes", n, m, prec, C.byref(out))
    return out.value


def ld_of(n):
    return (n + 7) & ~7


# ---------------------------------------------------------------- handle API
class Solver:
    """One TSP instance solved on the GPU (the C handle API).

    workspace="torch" places the solver's device state in a torch uint8 tensor
    (the library then allocates nothing); "library" lets it cudaMalloc.
    """

    def __init__(self, coords, m, alpha=1, beta=2, rho=0.5, Q=1.0, seed=0, prec="fp32",
                 roulette="ir", deposit="det", gamma_max=1.5, gamma_min=0.5, gamma_T=100,
                 tau0=1.0, workspace="torch", stream=None, cand_lists=True, topk=0, tau_prec="fp32"):
        import torch
        xy = _host(coords, np.float32)
        n = xy.shape[0]
        p = Params()
        call("aco_params_default", C.byref(p))
        p.n, p.m, p.alpha, p.beta = n, m, alpha, beta
        p.rho, p.Q, p.tau0, p.seed = rho, Q, tau0, seed
        p.prec = PREC[prec] if isinstance(prec, str) else prec
        p.roulette = ROULETTE[roulette] if isinstance(roulette, str) else roulette
        p.deposit = DEPOSIT[deposit] if isinstance(deposit, str) else deposit
        p.gamma_max, p.gamma_min, p.gamma_T = gamma_max, gamma_min, gamma_T
        p.cand_lists = int(cand_lists)
        p.topk = int(topk)
        p.tau_prec = PREC[tau_prec] if isinstance(tau_prec, str) else tau_prec
        self.params = p
        self.n, self.m = n, m
        self.stream = stream
        self._ws = None
        ws_ptr, ws_bytes = None, 0
        if workspace == "torch":
            ws_bytes = workspace_bytes(n, m, p.prec)
            self._ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
            ws_ptr = self._ws.data_ptr()
        h = v()
        call("aco_create", C.byref(h), xy.ctypes.data, C.byref(p), ws_ptr, ws_bytes, stream_ptr(stream))
        self._h = h

    def iterate(self, k=1):
        call("aco_solver_iterate", self._h, k)
        return self

    def best(self):
        tour = np.empty(self.n, dtype=np.int32)
        L = np.zeros(1, dtype=np.float64)
        call("aco_solver_best", self._h, tour.ctypes.data, L.ctypes.data)
        return tour, float(L[0])

    def tau(self):
        out = np.empty((self.n, self.n), dtype=np.float32)
        call("aco_solver_get_tau", self._h, out.ctypes.data)
        return out

    def tours(self):
        out = np.empty((self.m, self.n), dtype=np.int32)
        call("aco_solver_get_tours", self._h, out.ctypes.data)
        return out

    def lengths(self):
        out = np.empty(self.m, dtype=np.float64)
        call("aco_solver_get_lengths", self._h, out.ctypes.data)
        return out

    @property
    def iteration(self):
        it = u32(0)
        call("aco_solver_iteration", self._h, C.byref(it))
        return it.value

    def device_state(self):
        tau, ld, tours, L, bt, bl = v(), i32(0), v(), v(), v(), v()
        call("aco_solver_device_state", self._h, C.byref(tau), C.byref(ld), C.byref(tours),
             C.byref(L), C.byref(bt), C.byref(bl))
        return dict(tau=tau.value, ld=ld.value, tours=tours.value, lengths=L.value,
                    best_tour=bt.value, best_len=bl.value)

    def set_profiling(self, on=True):
        call("aco_solver_set_profiling", self._h, int(on))
        return self

    def kernel_ms(self):
        """Durations (ms) of the last iteration's steps: build_P, build_lists,
        construct, tour_length, best, deposit."""
        out = np.zeros(6, dtype=np.float32)
        call("aco_solver_kernel_ms", self._h, out.ctypes.data)
        return out

    def state(self):
        """The solver's checkpoint as bytes (tau, best tour/length, iteration, parameters)."""
        nbytes = sz(0)
        call("aco_solver_state_bytes", self._h, C.byref(nbytes))
        buf = np.empty(nbytes.value, dtype=np.uint8)
        call("aco_solver_save", self._h, buf.ctypes.data, nbytes.value)
        return buf.tobytes()

    def restore(self, blob):
        """Restore a checkpoint taken from a solver with the same coordinates and parameters."""
        buf = np.frombuffer(blob, dtype=np.uint8).copy()
        call("aco_solver_load", self._h, buf.ctypes.data, buf.size)
        return self

    def set_shape(self, warps=0, chunks=0, mode=0):
        call("aco_solver_set_shape", self._h, warps, chunks, mode)

    def set_wait_polls(self, polls=None):
        """Bound on the roulette-wheel kernel's row-copy waits (None: default)."""
        call("aco_solver_set_wait_polls", self._h, WAIT_POLLS_DEFAULT if polls is None else polls)
        return self

    def close(self):
        if getattr(self, "_h", None):
            lib().aco_destroy(self._h)
            self._h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_params(n, m, alpha=1, beta=2, rho=0.5, Q=1.0, seed=0, prec="fp32", roulette="ir",
                deposit="det", gamma_max=1.5, gamma_min=0.5, gamma_T=100, tau0=1.0, cand_lists=True,
                topk=0, tau_prec="fp32"):
    p = Params()
    call("aco_params_default", C.byref(p))
    p.n, p.m, p.alpha, p.beta = n, m, alpha, beta
    p.rho, p.Q, p.tau0, p.seed = rho, Q, tau0, seed
    p.prec = PREC[prec] if isinstance(prec, str) else prec
    p.roulette = ROULETTE[roulette] if isinstance(roulette, str) else roulette
    p.deposit = DEPOSIT[deposit] if isinstance(deposit, str) else deposit
    p.gamma_max, p.gamma_min, p.gamma_T = gamma_max, gamma_min, gamma_T
    p.cand_lists = int(cand_lists)
    p.topk = int(topk)
    p.tau_prec = PREC[tau_prec] if isinstance(tau_prec, str) else tau_prec
    return p


def instance_bytes(n, m):
    out = sz(0)
    call("aco_batch_instance_bytes", n, m, C.byref(out))
    return out.value


class Batch:
    """Many independent instances advanced together (the C batch API)."""

    def __init__(self, max_instances, arena_bytes, prec="fp32", stream=None, arena="torch"):
        import torch
        self.prec = PREC[prec] if isinstance(prec, str) else prec
        self._arena = None
        arena_ptr = None
        if arena == "torch":
            self._arena = torch.empty(arena_bytes, dtype=torch.uint8, device="cuda")
            arena_ptr = self._arena.data_ptr()
        self.stream = stream
        h = v()
        call("aco_batch_create", C.byref(h), max_instances, arena_bytes, self.prec, arena_ptr,
             stream_ptr(stream))
        self._h = h
        self.n_of = {}

    def add(self, coords, m, iters=0, **kw):
        """Admit an instance; returns its slot, or None if it does not fit now."""
        xy = _host(coords, np.float32)
        n = xy.shape[0]
        p = make_params(n, m, prec=self.prec, **kw)
        slot = i32(-1)
        rc = lib().aco_batch_add(self._h, xy.ctypes.data, C.byref(p), iters, C.byref(slot))
        if rc == ERR_OOM:
            return None
        check(rc)
        self.n_of[slot.value] = n
        return slot.value

    def remove(self, slot):
        call("aco_batch_remove", self._h, slot)
        self.n_of.pop(slot, None)

    def step(self, k=1):
        call("aco_batch_step", self._h, k)
        return self

    def best(self, slot):
        n = self.n_of[slot]
        tour = np.empty(n, dtype=np.int32)
        L = np.zeros(1, dtype=np.float64)
        call("aco_batch_best", self._h, slot, tour.ctypes.data, L.ctypes.data)
        return tour, float(L[0])

    def tau(self, slot):
        n = self.n_of[slot]
        out = np.empty((n, n), dtype=np.float32)
        call("aco_batch_get_tau", self._h, slot, out.ctypes.data)
        return out

    def status(self, slot):
        it, fin = u32(0), i32(0)
        call("aco_batch_status", self._h, slot, C.byref(it), C.byref(fin))
        return it.value, bool(fin.value)

    def info(self):
        a, f, l = i32(0), sz(0), sz(0)
        call("aco_batch_info", self._h, C.byref(a), C.byref(f), C.byref(l))
        return dict(active=a.value, free_bytes=f.value, largest_block=l.value)

    def set_shape(self, warps=0, chunks=0, mode=0):
        call("aco_batch_set_shape", self._h, warps, chunks, mode)

    def close(self):
        if getattr(self, "_h", None):
            lib().aco_batch_destroy(self._h)
            self._h = None
        self._arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
