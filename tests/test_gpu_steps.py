"""GPU parity, one step at a time, through the C ABI's step-level calls:
every kernel against the CPU oracle on the same seeded inputs.  Integer and
index results (tours, neighbours, start cities) and every floating-point
result of the deterministic path are compared bit for bit; the float-atomic
deposit within 1e-5 relative."""
import numpy as np
import pytest
import torch

from gpu_util import P_device, covers, dev, host, padded_dev, shapes
from paper_2404_04895_gb300 import binding as B
from paper_2404_04895_gb300 import instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.lib()


def test_philox_bit_exact(orc):
    rng = np.random.default_rng(0)
    cnt = 20000
    ctr = rng.integers(0, 1 << 32, size=(cnt, 4), dtype=np.uint64).astype(np.uint32)
    for seed in (0, 1, 0xDEADBEEFCAFEF00D):
        out = torch.zeros((cnt, 4), dtype=torch.int32, device="cuda")
        B.op_philox(dev(ctr.view(np.int32)), seed, out, cnt)
        got = host(out).view(np.uint32)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for q in range(0, cnt, 97):
            assert np.array_equal(got[q], orc.philox(ctr[q], key))
    # the published known-answer vectors, on the device
    out = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
    B.op_philox(dev(np.zeros((1, 4), np.int32)), 0, out, 1)
    assert host(out).view(np.uint32)[0].tolist() == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]


def test_pow_own_bit_exact(orc):
    rng = np.random.default_rng(1)
    x = np.exp(rng.uniform(np.log(1e-30), np.log(1e30), size=400000)).astype(np.float32)
    x[:8] = [0.0, 1.0, 2.0, 0.5, 1e-40, 3e38, 1.4142135, 0.70710677]
    xd = dev(x)
    for e in [0.5, 2.0 / 3.0, 0.8, 1.0, 1.25, 1.5, 2.0]:
        e32 = float(np.float32(e))
        out = torch.empty_like(xd)
        B.op_pow_own(xd, e32, out, x.size)
        got = host(out)
        ref = orc.pow_own(x, e32)
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), e


@pytest.mark.parametrize("n", [3, 50, 257, 1000])
@pytest.mark.parametrize("beta", [0, 2, 5])
@pytest.mark.parametrize("extra_ld", [0, 72])
def test_heuristic_bit_exact(orc, n, beta, extra_ld):
    """Every entry (both triangles, the diagonal, and the padding columns up
    to a caller's ld beyond the last 32-column tile) against the oracle."""
    xy = instances.uniform(n, n)
    xy[n // 2] = xy[0]  # a coincident pair exercises the 1e-9 floor
    ld = B.ld_of(n) + extra_ld
    D = torch.full((n, n), np.nan, dtype=torch.float64, device="cuda")
    H = torch.full((n, ld), 7.0, dtype=torch.float32, device="cuda")
    B.op_heuristic(dev(xy), n, beta, D, H, ld)
    Dr = orc.distances(xy)
    Hr = orc.heuristic(Dr, beta)
    assert np.array_equal(host(D), Dr)
    Hg = host(H)
    assert np.array_equal(Hg[:, :n], Hr)
    assert np.all(Hg[:, n:] == 0)


@pytest.mark.parametrize("prec", [B.FP32, B.BF16, B.FP16])
@pytest.mark.parametrize("n,alpha,g", [(3, 1, 1.0), (61, 2, 1.0), (61, 1, 1.5), (1000, 1, 0.75),
                                       (1000, 3, 1.0)])
def test_build_P_bit_exact(orc, prec, n, alpha, g):
    xy = instances.clustered(10, (n + 9) // 10, 0.03, seed=n)[:n]
    ld = B.ld_of(n)
    Dr = orc.distances(xy)
    Hr = orc.heuristic(Dr, 2)
    tau = np.random.default_rng(n).uniform(0.01, 3.0, size=(n, n)).astype(np.float32)
    inv = orc.inv_gamma(np.float32(g))
    P = torch.zeros((n, ld), dtype=torch.float32, device="cuda")  # big enough for every precision
    B.op_build_P(padded_dev(tau, ld, np.float32), padded_dev(Hr, ld, np.float32), n, ld, alpha, inv,
                 prec, P)
    Pv, bits, _ = orc.build_P(tau, Hr, alpha, inv, prec)
    if prec == B.FP32:
        got = host(P)
        assert np.array_equal(got[:, :n].view(np.uint32), Pv.view(np.uint32))
        assert np.all(got[:, n:] == 0)
    else:
        got = P.view(torch.int16).reshape(-1)[: n * ld].reshape(n, ld).cpu().numpy().view(np.uint16)
        assert np.array_equal(got[:, :n], bits)
        assert np.all(got[:, n:] == 0)


def _P_for(orc, xy, prec, alpha=1, beta=2, g=1.0, seed=0):
    n = xy.shape[0]
    Hr = orc.heuristic(orc.distances(xy), beta)
    tau = np.random.default_rng(seed).uniform(0.2, 2.0, size=(n, n)).astype(np.float32)
    tau = np.minimum(tau, tau.T)
    Pv, bits, _ = orc.build_P(tau, Hr, alpha, orc.inv_gamma(np.float32(g)), prec)
    return Pv, bits


@pytest.mark.parametrize("prec", [B.FP32, B.BF16, B.FP16])
@pytest.mark.parametrize("n,m", [(3, 1), (4, 9), (5, 33), (33, 16), (129, 40), (1000, 24)])
def test_construct_bit_exact(orc, prec, n, m):
    xy = instances.uniform(n, 1000 + n)
    Pv, bits = _P_for(orc, xy, prec, seed=n)
    ld = B.ld_of(n)
    Pd = P_device(Pv, bits, prec, ld)
    tours = torch.full((m, n), -1, dtype=torch.int32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    seed, it = 12345 + n, 7
    B.op_construct(Pd, prec, n, ld, m, seed, it, tours, err)
    assert int(err.item()) == 0
    ref = orc.construct(Pv, seed, it, 0, m)
    assert np.array_equal(host(tours), ref)


@pytest.mark.parametrize("prec", [B.FP32, B.BF16])
def test_construct_every_shape_agrees(orc, prec):
    n, m = 1000, 12
    eb = 4 if prec == B.FP32 else 2
    xy = instances.clustered(20, 50, 0.02, seed=4)
    Pv, bits = _P_for(orc, xy, prec, seed=5)
    ld = B.ld_of(n)
    Pd = P_device(Pv, bits, prec, ld)
    ref = orc.construct(Pv, 99, 3, 0, m)
    tried = 0
    for shp in shapes(eb):
        if not covers(shp, n, eb):
            continue
        tours = torch.full((m, n), -1, dtype=torch.int32, device="cuda")
        B.op_construct(Pd, prec, n, ld, m, 99, 3, tours, None, shape=shp)
        assert np.array_equal(host(tours), ref), shp
        tried += 1
    assert tried >= 8


def test_construct_adair_matrix_and_ties(orc):
    # AdaIR's M_p^(1/gamma) and a row of exact ties (lowest index must win)
    n, m = 70, 30
    xy = instances.uniform(n, 5)
    Pv, bits = _P_for(orc, xy, B.FP32, g=1.5, seed=9)
    Pv[:, 10:20] = np.float32(0.0)
    ld = B.ld_of(n)
    tours = torch.zeros((m, n), dtype=torch.int32, device="cuda")
    B.op_construct(P_device(Pv, bits, B.FP32, ld), B.FP32, n, ld, m, 4, 0, tours)
    assert np.array_equal(host(tours), orc.construct(Pv, 4, 0, 0, m))
    # all-equal matrix: every score is r_j * c, ties broken by lowest index
    Pc = np.ones((n, n), np.float32)
    np.fill_diagonal(Pc, 0)
    B.op_construct(P_device(Pc, None, B.FP32, ld), B.FP32, n, ld, m, 4, 1, tours)
    assert np.array_equal(host(tours), orc.construct(Pc, 4, 1, 0, m))


@pytest.mark.parametrize("n,m", [(3, 2), (50, 50), (301, 77), (2100, 7), (2100, 6), (5000, 8), (7168, 4),
                                 (7200, 4)])
def test_tour_length_neighbours_best(orc, n, m):
    """Lengths, c, the index mapping and the best, for every kernel form: one
    warp, two and four warps per ant, two ants per CTA with the mapping staged
    in shared memory (2048 <= n <= 7168, m even), and four warps per ant
    otherwise (m odd, or n beyond that)."""
    xy = instances.uniform(n, 3)
    Dr = orc.distances(xy)
    rng = np.random.default_rng(n)
    tours = np.stack([rng.permutation(n) for _ in range(m)]).astype(np.int32)
    tours[m - 1] = tours[0]  # a tie in length: the lower ant index must win
    L = torch.empty(m, dtype=torch.float64, device="cuda")
    c = torch.empty(m, dtype=torch.float64, device="cuda")
    nbr = torch.full((n, m, 2), -1, dtype=torch.int32, device="cuda")
    td = dev(tours)
    B.op_tour_length(dev(Dr), n, td, m, 2.5, L, c, nbr)
    Lr = orc.tour_lengths(Dr, tours)
    assert np.array_equal(host(L), Lr)
    assert np.array_equal(host(c), 2.5 / Lr)
    nb = host(nbr)
    for k in range(m):
        for t in range(n):
            a = tours[k, t]
            assert nb[a, k, 0] == tours[k, t - 1] and nb[a, k, 1] == tours[k, (t + 1) % n]
    best_tour = torch.zeros(n, dtype=torch.int32, device="cuda")
    best_len = torch.full((1,), float("inf"), dtype=torch.float64, device="cuda")
    B.op_best(L, td, n, m, best_tour, best_len)
    kb = int(np.argmin(Lr))
    assert best_len.item() == Lr[kb] and np.array_equal(host(best_tour), tours[kb])
    # a later, equal length does not replace the best
    B.op_best(L, dev(np.roll(tours, 1, axis=0)), n, m, best_tour, best_len)
    assert np.array_equal(host(best_tour), tours[kb])


@pytest.mark.parametrize("n,m", [(3, 1), (20, 5), (200, 64), (1000, 100)])
def test_deposit_deterministic_bit_exact(orc, n, m):
    xy = instances.uniform(n, 8)
    Dr = orc.distances(xy)
    rng = np.random.default_rng(m)
    base = rng.permutation(n)
    tours = []
    for k in range(m):  # many ants share edges, as a converging colony does
        t = base.copy()
        if k % 3:
            i, j = sorted(rng.integers(0, n, size=2))
            t[i:j + 1] = t[i:j + 1][::-1]
        tours.append(t)
    tours = np.stack(tours).astype(np.int32)
    tau0 = rng.uniform(0.5, 2.0, size=(n, n)).astype(np.float32)
    tau0 = np.minimum(tau0, tau0.T)
    ld = B.ld_of(n)
    L = torch.empty(m, dtype=torch.float64, device="cuda")
    c = torch.empty(m, dtype=torch.float64, device="cuda")
    nbr = torch.empty((n, m, 2), dtype=torch.int32, device="cuda")
    B.op_tour_length(dev(Dr), n, dev(tours), m, 1.0, L, c, nbr)
    tau = padded_dev(tau0, ld, np.float32)
    B.op_deposit(tau, n, ld, nbr, c, m, 0.1)
    ref = orc.deposit(tau0, tours, orc.tour_lengths(Dr, tours), 0.1, 1.0)
    got = host(tau, n)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    # atomic variant: same step within 1e-5 relative
    tau = padded_dev(tau0, ld, np.float32)
    B.op_deposit_atomic(tau, n, ld, dev(tours), c, m, 0.1)
    got = host(tau, n)
    assert np.max(np.abs(got.astype(np.float64) - ref) / ref) < 1e-5
