"""GPU parity of the exact deposit (Sec. 2.3, Eq. 3) against the oracle, bit
for bit, on the cases the fixed-point design has to get right: half-way
ties, weights spanning the widest allowed range, infinite weights (a zero
tour length), fp32 subnormal and overflow results, rows with more touched
columns than one pass holds, and the out-of-range error.  The exact tour
length (Eq. 3) is checked at sizes that split a tour over many lanes and
warps."""
import warnings

import numpy as np
import pytest
import torch

from conftest import golden_path
from gpu_util import dev, host, padded_dev
from paper_2404_04895_gb300 import binding as B
from paper_2404_04895_gb300 import instances

pytestmark = pytest.mark.gpu


def _nbr(tours):
    m, n = tours.shape
    nbr = np.empty((n, m, 2), np.int32)
    for k in range(m):
        p = tours[k]
        nbr[p, k, 0] = np.roll(p, 1)
        nbr[p, k, 1] = np.roll(p, -1)
    return nbr


def _deposit(orc, tours, L, tau0, rho, Q=1.0):
    """GPU aco_op_deposit and the oracle on the same tours, lengths, tau."""
    m, n = tours.shape
    ld = B.ld_of(n)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        c = np.float64(np.float32(Q)) / np.asarray(L, np.float64)  # c_k = fl64(Q / L_k)
    tau = padded_dev(tau0, ld, np.float32)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.op_deposit(tau, n, ld, dev(_nbr(tours)), dev(c), m, rho, err)
    torch.cuda.synchronize()
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        ref = orc.deposit(tau0, tours, L, rho, Q)
    return host(tau, n), ref, int(err.item())


def _same(a, b):
    return np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_half_way_tie_rounds_once(orc):
    ref = np.loadtxt(golden_path("deposit_single_rounding.txt"), dtype=np.float64)
    tours = np.array([[0, 1, 2], [1, 2, 0]], np.int32)
    got, _, err = _deposit(orc, tours[:1], [float.fromhex("0x1.fffffffp-17")],
                           np.full((3, 3), 2.0 ** 40, np.float32), 0.0)
    assert err == 0 and np.array_equal(got.astype(np.float64), ref)
    one = np.ones((3, 3), np.float32)
    for L, want in [([2.0 ** 24, 2.0 ** 40], 1 + 2.0 ** -23),   # above the tie: up
                    ([2.0 ** 24], 1.0),                          # exact tie: to even
                    ([2.0 ** 23 / 3, 2.0 ** 30], None)]:
        got, ref, err = _deposit(orc, tours[:len(L)], L, one, 0.0)
        assert err == 0 and _same(got, ref)
        if want is not None:
            assert got[0, 1] == np.float32(want)


@pytest.mark.parametrize("span,ok", [(19, True), (20, False)])
def test_weight_span_limit(orc, span, ok):
    rng = np.random.default_rng(span)
    n, m = 40, 6
    tours = np.stack([rng.permutation(n) for _ in range(m)]).astype(np.int32)
    L = np.array([1.0, 2.0 ** span, 1.5, 3.0, 2.0 ** (span - 1), 7.0])
    tau0 = rng.uniform(0.5, 2, size=(n, n)).astype(np.float32)
    got, ref, err = _deposit(orc, tours, L, tau0, 0.3)
    if ok:
        assert err == 0 and _same(got, ref)
    else:  # the weights cannot be summed: the kernel reports it, touched entries are NaN
        assert err == 2
        _check_refused(got, tours, tau0, 0.3)


@pytest.mark.parametrize("top", [1.0, 1.999, 2.0, 3.99, 4.0, 16.0])
def test_two_and_three_chunk_weights(orc, top):
    """Weights whose exponents differ by at most one are summed as two 27-bit
    chunks, wider spans as three 24-bit ones: lengths from 1 up to `top`
    (exponent spans 0, 1, 1, 2, 2 and 4), many ants sharing edges, each form
    against the oracle bit for bit."""
    rng = np.random.default_rng(int(top * 1000))
    n, m = 300, 96
    base = rng.permutation(n)
    tours = []
    for k in range(m):
        t = base.copy()
        if k % 2:
            i, j = sorted(rng.integers(0, n, size=2))
            t[i:j + 1] = t[i:j + 1][::-1]
        tours.append(t)
    tours = np.asarray(tours, np.int32)
    L = rng.uniform(1.0, top, size=m)
    L[0], L[-1] = 1.0, top
    tau0 = rng.uniform(0.5, 2, size=(n, n)).astype(np.float32)
    got, ref, err = _deposit(orc, tours, L, tau0, 0.1)
    assert err == 0 and _same(got, ref)


def _check_refused(got, tours, tau0, rho):
    """Every entry some path uses is NaN, every other one evaporated."""
    n = tau0.shape[0]
    touched = np.zeros((n, n), bool)
    for p in tours:
        for t in range(n):
            touched[p[t], p[t - 1]] = touched[p[t - 1], p[t]] = True
    assert np.all(np.isnan(got[touched]))
    assert _same(got[~touched], ((np.float32(1) - np.float32(rho)) * tau0)[~touched])


def test_negative_weight_reports_error(orc):
    n, m = 12, 3
    rng = np.random.default_rng(3)
    tours = np.stack([rng.permutation(n) for _ in range(m)]).astype(np.int32)
    tau0 = rng.uniform(0.5, 2, size=(n, n)).astype(np.float32)
    got, _, err = _deposit(orc, tours, np.array([2.0, -3.0, 4.0]), tau0, 0.25)
    assert err == 2
    _check_refused(got, tours, tau0, 0.25)


def test_infinite_weights(orc):
    """A zero length gives c = +inf: the entries of that tour become +inf,
    entries only other ants use stay finite and exact."""
    rng = np.random.default_rng(4)
    n = 30
    tours = np.stack([rng.permutation(n) for _ in range(3)]).astype(np.int32)
    tau0 = rng.uniform(0.5, 2, size=(n, n)).astype(np.float32)
    got, ref, err = _deposit(orc, tours, np.array([0.0, 5.0, 9.0]), tau0, 0.1)
    assert err == 0 and _same(got, ref)
    assert np.isinf(got[tours[0, 0], tours[0, 1]])


def test_subnormal_and_overflow_results(orc):
    rng = np.random.default_rng(5)
    n, m = 16, 4
    tours = np.stack([rng.permutation(n) for _ in range(m)]).astype(np.int32)
    tiny = (rng.integers(0, 50, size=(n, n)) * np.float32(2.0 ** -149)).astype(np.float32)
    got, ref, err = _deposit(orc, tours, 2.0 ** (140 + rng.uniform(0, 2, m)), tiny, 0.5)
    assert err == 0 and _same(got, ref)
    assert np.any((got > 0) & (got < np.float32(2.0 ** -126)))
    big = np.full((n, n), np.float32(3.0e38))
    got, ref, err = _deposit(orc, tours, np.array([1e-38, 2e-38, 3e-38, 1e-37]), big, 0.0)
    assert err == 0 and _same(got, ref) and np.isinf(got).any()


@pytest.mark.parametrize("n,m,converged", [(997, 300, False), (2000, 1024, True), (4500, 2000, False)])
def test_random_colonies_bit_exact(orc, n, m, converged):
    """Random and converged colonies; (4500, 2000) has rows with more touched
    columns than one pass of the slot table holds."""
    rng = np.random.default_rng(n)
    if converged:
        base = rng.permutation(n)
        tours = np.repeat(base[None, :], m, axis=0).astype(np.int32)
        for k in range(1, m, 2):  # half the ants with one 2-opt move
            i, j = sorted(rng.integers(0, n, size=2))
            tours[k, i:j + 1] = tours[k, i:j + 1][::-1]
    else:
        tours = np.stack([rng.permutation(n) for _ in range(m)]).astype(np.int32)
    L = rng.uniform(0.7, 1.3, size=m) * n ** 0.5
    tau0 = rng.uniform(0.01, 2, size=(n, n)).astype(np.float32)
    got, ref, err = _deposit(orc, tours, L, tau0, 0.1)
    assert err == 0 and _same(got, ref)


@pytest.mark.parametrize("n,m", [(1025, 9), (5000, 5), (65, 3), (3, 4), (511, 7), (2048, 3), (8192, 2)])
def test_exact_tour_length_bit_exact(orc, n, m):
    xy = instances.uniform(n, 21)
    Dr = orc.distances(xy)
    rng = np.random.default_rng(n)
    tours = np.stack([rng.permutation(n) for _ in range(m)]).astype(np.int32)
    L = torch.empty(m, dtype=torch.float64, device="cuda")
    c = torch.empty(m, dtype=torch.float64, device="cuda")
    B.op_tour_length(dev(Dr), n, dev(tours), m, 1.0, L, c, None)
    Lr = orc.tour_lengths(Dr, tours)
    assert np.array_equal(host(L), Lr)
    assert np.array_equal(host(c), np.float64(1.0) / Lr)
