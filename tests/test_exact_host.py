"""The kernels' exact arithmetic compiled for the host, against the
oracle's independent exact summation (Eq. 3, Sec. 2.3):
  - the deposit (csrc/exact.cuh): tau' plus the weights of the paths through
    an entry, split into 24-bit fixed-point chunks, summed and rounded once,
    equals the fp32 (and bfloat16) rounding of the exact rational sum -- on
    random entries, ties, near-ties, subnormal and overflow boundaries;
  - the tour length (csrc/exact_len.cuh): edge lengths dealt to partial sums
    as lanes and warps take them, summed in fixed point and rounded once,
    equal the oracle's f bit for bit, however the edges are split.
CPU only: this pins the GPU path's rounding code in every CPU run."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from conftest import ROOT

CSRC = os.path.join(ROOT, "paper_2404_04895_gb300", "csrc")


@pytest.fixture(scope="module")
def hx():
    out_dir = os.path.join(ROOT, "tests", "_build")
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libexact_host.so")
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-I", CSRC, "-o", lib,
                    os.path.join(ROOT, "tests", "exact_host.cpp")], check=True)
    L = ctypes.CDLL(lib)
    L.hx_deposit_entry.restype = ctypes.c_int
    L.hx_deposit_entry.argtypes = [ctypes.c_float, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_uint32)]
    L.hx_tour_length.restype = ctypes.c_int
    L.hx_tour_length.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    return L


def _lib_entry(hx, tp, c, bf16):
    c = np.ascontiguousarray(c, dtype=np.float64)
    out = ctypes.c_uint32(0)
    assert hx.hx_deposit_entry(np.float32(tp), c.ctypes.data, c.size, int(bf16), ctypes.byref(out)) == 0
    return out.value


def _check(orc, hx, tp, c):
    x = np.concatenate([[np.float64(np.float32(tp))], np.asarray(c, np.float64)])
    ref32 = np.float32(orc.exact_sum_f32(x)).view(np.uint32)
    assert _lib_entry(hx, tp, c, False) == int(ref32), (float(tp), list(map(float.hex, map(float, c))))
    refb = np.float32(orc.exact_sum_bf16(x)).view(np.uint32)
    assert int(refb) & 0xFFFF == 0
    assert _lib_entry(hx, tp, c, True) == int(refb) >> 16, (float(tp), list(map(float.hex, map(float, c))))


def test_random_entries_match_the_exact_rounding(orc, hx):
    rng = np.random.default_rng(2404)
    for _ in range(4000):
        k = int(rng.integers(1, 65))
        span = float(rng.uniform(0, 19))
        base = float(rng.uniform(-40, 10))
        c = np.exp2(base + span * rng.random(k))          # weights Q / L_k within 2^19 of each other
        tp = np.float32(np.exp2(rng.uniform(-60, 20)))   # the evaporated pheromone
        _check(orc, hx, tp, c)


def test_converged_entries_repeat_one_weight(orc, hx):
    """Many ants on the same edge: one weight repeated up to 2048 times."""
    rng = np.random.default_rng(7)
    for _ in range(300):
        k = int(rng.integers(1, 2049))
        c = np.full(k, np.exp2(rng.uniform(-20, 0)))
        _check(orc, hx, np.float32(rng.uniform(0, 50)), c)


def test_ties_near_ties_and_range_boundaries(orc, hx):
    one = np.float32(1.0)
    _check(orc, hx, one, [2.0 ** -24])                        # tie at 1 + 2^-24: to even (1)
    _check(orc, hx, one, [2.0 ** -24, 2.0 ** -42])            # just above the tie
    _check(orc, hx, np.float32(1 + 2.0 ** -23), [2.0 ** -24])  # tie to even (up)
    _check(orc, hx, one, [2.0 ** -25] * 2)                    # the tie reached by two weights
    _check(orc, hx, np.float32(0.0), [2.0 ** -150])           # half the smallest subnormal: to 0
    _check(orc, hx, np.float32(0.0), [2.0 ** -150, 2.0 ** -165])  # above it: the smallest subnormal
    _check(orc, hx, np.float32(2.0 ** -149), [2.0 ** -149])   # subnormal sums
    _check(orc, hx, np.float32(np.finfo(np.float32).max), [2.0 ** 103])  # tie at the top: to inf
    _check(orc, hx, np.float32(np.finfo(np.float32).max), [2.0 ** 102])  # below the tie: stays
    _check(orc, hx, np.float32(2.0 ** 100), [2.0 ** -100])    # far below: sticky only
    _check(orc, hx, np.float32(2.0 ** -100), [2.0 ** 100, 2.0 ** 81])  # the weights dominate


def test_weights_beyond_the_span_are_refused(hx):
    c = np.array([1.0, 2.0 ** -(hx.hx_dep_span() + 1)])
    out = ctypes.c_uint32(0)
    assert hx.hx_deposit_entry(np.float32(1.0), c.ctypes.data, 2, 0, ctypes.byref(out)) == -1


def _length(hx, edges, groups):
    e = np.ascontiguousarray(edges, dtype=np.float64)
    out = ctypes.c_double(0.0)
    rc = hx.hx_tour_length(e.ctypes.data, e.size, groups, ctypes.byref(out))
    return None if rc else out.value


def test_tour_length_fixed_point_matches_oracle(orc, hx):
    """Planar tours (uniform and clustered, n ragged) and wide-range edge sets
    within [2^-149, 2^130), split over 1, 3, 32 and 128 partial sums."""
    rng = np.random.default_rng(2405)
    for trial in range(600):
        kind = trial % 3
        n = int(rng.integers(3, 3000 if kind == 0 else 200))
        if kind == 0:
            xy = rng.uniform(0, 1, size=(n, 2)).astype(np.float32)
            if trial % 2:
                c = rng.uniform(0, 1, size=(max(1, n // 50), 2))
                xy = (c[rng.integers(0, len(c), size=n)] + rng.normal(0, 0.02, size=(n, 2))).astype(np.float32)
            p = rng.permutation(n)
            q = np.roll(p, -1)
            dx = xy[p, 0].astype(np.float64) - xy[q, 0].astype(np.float64)
            dy = xy[p, 1].astype(np.float64) - xy[q, 1].astype(np.float64)
            edges = np.sqrt(dx * dx + dy * dy)
        elif kind == 1:
            edges = np.exp2(rng.uniform(-149, 129, size=n)) * rng.uniform(1, 2, size=n)
            edges = np.minimum(edges, float.fromhex("0x1.fffffffffffffp+129"))
        else:
            edges = np.exp2(rng.uniform(-2, 1, size=n))       # a narrow band, a few tiny outliers
            tiny = rng.random(n) < 0.1
            edges[tiny] = np.exp2(rng.uniform(-149, -40, size=int(tiny.sum())))
            edges[rng.random(n) < 0.05] = 2.0 ** -149
        edges[rng.random(n) < 0.02] = 0.0
        ref = orc.exact_sum(edges)
        for groups in (1, 3, 32, 128):
            assert _length(hx, edges, groups) == ref, (trial, groups)


def test_tour_length_golden_and_range(orc, hx):
    rows = [ln.split() for ln in open(os.path.join(ROOT, "tests", "golden", "tour_length_exact.txt"))
            if ln.strip() and not ln.startswith("#")]
    for row in rows:
        edges = [float.fromhex(v) for v in row[:-1]]
        for groups in (1, 2, 7):
            assert _length(hx, edges, groups) == float.fromhex(row[-1]), row
    assert _length(hx, [0.0, 0.0, 0.0], 1) == 0.0
    big = float.fromhex("0x1.fffffffffffffp+129")
    assert _length(hx, [big] * 65536, 32) == orc.exact_sum(np.full(65536, big))
    # outside the range the kernel holds: refused (the kernel writes NaN)
    for bad in (2.0 ** -150, 2.0 ** 130, -1.0, float("inf"), float("nan")):
        assert _length(hx, [1.0, bad, 1.0], 1) is None, bad
