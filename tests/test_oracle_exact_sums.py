"""Oracle pins for the order-free readings of two sums of the path:
the deposit (Sec. 2.3, Eq. 3: the real sum of the paths' weights added to the
evaporated pheromone, rounded once to fp32) and the fitness f (Eq. 3: the
exact sum of a tour's fp64 edge lengths rounded once).  Exact rational arithmetic (fractions.Fraction) and
math.fsum are the independent references."""
import math
from fractions import Fraction

import numpy as np

from conftest import golden_path

F32_INF_AT = Fraction(2) ** 128 - Fraction(2) ** 103  # fp32 overflow threshold (rounds to inf)


def _rn32(x: Fraction) -> np.float32:
    """Nearest fp32 to the rational x, ties to even, by exact comparison."""
    if x < 0:
        return -_rn32(-x)
    if x >= F32_INF_AT:
        return np.float32(np.inf)
    g = np.float32(float(x))
    cands = {g, np.nextafter(g, np.float32(np.inf)), np.nextafter(g, np.float32(0))}
    cands = [c for c in cands if np.isfinite(c)]

    def dist(c):
        return abs(Fraction(float(c)) - x)

    best = min(dist(c) for c in cands)
    tied = [c for c in cands if dist(c) == best]
    if len(tied) == 1:
        return tied[0]
    even = [c for c in tied if (np.array(c, np.float32).view(np.uint32) & 1) == 0]
    assert len(even) == 1
    return even[0]


def _cases(rng):
    out = []
    for _ in range(3000):
        k = int(rng.integers(1, 12))
        kind = int(rng.integers(0, 5))
        if kind == 0:
            x = rng.uniform(1e-4, 2.0, size=k)
        elif kind == 1:
            x = np.exp(rng.normal(0, 30, size=k))
        elif kind == 2:
            x = rng.normal(0, 1, size=k) * np.exp(rng.normal(0, 10, size=k))
        elif kind == 3:
            # an fp32 value, half of its ulp, and a tiny push either way or none
            a = np.float32(rng.uniform(0.5, 4.0))
            half = math.ulp(float(a)) * 2.0 ** 29 / 2.0  # half an fp32 ulp (fp32 has 29 fewer bits)
            tiny = [0.0, 2.0 ** -70, -(2.0 ** -70), 2.0 ** -30][int(rng.integers(0, 4))]
            x = np.array([float(a), half, tiny])
        else:
            # cancellation: large values that cancel and leave small ones
            big = rng.uniform(1e10, 1e12, size=k)
            x = np.concatenate([big, -big, rng.uniform(-1, 1, size=2)])
            rng.shuffle(x)
        out.append(np.asarray(x, dtype=np.float64))
    return out


def test_exact_sum_matches_fsum(orc):
    rng = np.random.default_rng(11)
    for x in _cases(rng):
        assert orc.exact_sum(x) == math.fsum(x)


def test_exact_sum_f32_matches_rational(orc):
    rng = np.random.default_rng(12)
    for x in _cases(rng):
        exact = sum((Fraction(float(v)) for v in x), Fraction(0))
        got = orc.exact_sum_f32(x)
        ref = _rn32(exact)
        assert (np.isinf(got) and np.isinf(ref) and got == ref) or got == ref, (x.tolist(), got, ref)


def test_exact_sum_f32_boundaries(orc):
    big = float(np.finfo(np.float32).max)
    half = 2.0 ** 103  # half an ulp at the top of the fp32 range
    assert orc.exact_sum_f32(np.array([big, half])) == np.float32(np.inf)          # tie -> even -> inf
    assert orc.exact_sum_f32(np.array([big, half, -(2.0 ** 40)])) == np.float32(big)
    sub = float(np.float32(2.0 ** -149))
    assert orc.exact_sum_f32(np.array([sub, sub / 2])) == np.float32(2.0 ** -148)   # tie -> even
    assert orc.exact_sum_f32(np.array([sub / 2, 2.0 ** -200])) == np.float32(sub)
    assert orc.exact_sum_f32(np.array([1.0, 2.0 ** -24])) == np.float32(1.0)
    assert orc.exact_sum_f32(np.array([1.0, 2.0 ** -24, 2.0 ** -80])) == np.float32(1 + 2.0 ** -23)
    assert np.isinf(orc.exact_sum_f32(np.array([1.0, np.inf])))


def test_deposit_single_rounding_golden(orc):
    ref = np.loadtxt(golden_path("deposit_single_rounding.txt"), dtype=np.float64)
    tours = np.array([[0, 1, 2]], dtype=np.int32)
    L = np.array([float.fromhex("0x1.fffffffp-17")])
    tau = orc.deposit(np.full((3, 3), 2.0 ** 40, np.float32), tours, L, rho=0.0, Q=1.0)
    assert np.array_equal(tau.astype(np.float64), ref)
    # weights far apart (36 binades): 1 + 2^-24 + 2^-60 is above the tie at 1 + 2^-24
    tau = orc.deposit(np.ones((3, 3), np.float32), np.array([[0, 1, 2], [1, 2, 0]], np.int32),
                      np.array([2.0 ** 24, 2.0 ** 60]), rho=0.0, Q=1.0)
    assert tau[0, 1] == np.float32(1 + 2.0 ** -23) and tau[0, 0] == np.float32(1)


def test_deposit_is_rounded_exact_sum(orc):
    """Brute force with rationals on small colonies: every entry equals the
    fp32 rounding of fl32(keep * tau) + the weights of the paths using it."""
    rng = np.random.default_rng(13)
    for trial in range(6):
        n, m = int(rng.integers(3, 9)), int(rng.integers(1, 7))
        tours = np.stack([rng.permutation(n) for _ in range(m)]).astype(np.int32)
        if trial % 2:
            tours[1:] = tours[0]  # a converged colony: every ant on one tour
        L = rng.uniform(0.5, 3.0, size=m) * (2.0 ** rng.integers(-3, 4, size=m))
        rho, Q = np.float32(rng.uniform(0, 1)), np.float32(rng.uniform(0.1, 5))
        tau0 = rng.uniform(0.01, 2, size=(n, n)).astype(np.float32)
        got = orc.deposit(tau0, tours, L, float(rho), float(Q))
        keep = np.float32(np.float32(1) - rho)
        w = [Fraction(float(np.float64(Q) / L[k])) for k in range(m)]
        acc = [[Fraction(float(np.float32(keep * tau0[i, j]))) for j in range(n)] for i in range(n)]
        touched = np.zeros((n, n), bool)
        for k in range(m):
            for t in range(n):
                a, b = int(tours[k, t]), int(tours[k, t - 1])
                acc[a][b] += w[k]
                acc[b][a] += w[k]
                touched[a, b] = touched[b, a] = True
        for i in range(n):
            for j in range(n):
                ref = _rn32(acc[i][j]) if touched[i, j] else np.float32(keep * tau0[i, j])
                assert got[i, j] == ref, (trial, i, j)


def test_tour_length_integer_grid_exact(orc):
    """On a line of integer points every edge and every partial sum is an
    integer below 2^53, so any summation order gives the exact length."""
    rng = np.random.default_rng(14)
    n = 1000
    x = rng.permutation(4 * n)[:n].astype(np.float32)
    xy = np.stack([x, np.zeros(n, np.float32)], axis=1)
    D = orc.distances(xy)
    tours = np.stack([rng.permutation(n) for _ in range(3)]).astype(np.int32)
    L = orc.tour_lengths(D, tours)
    for k in range(3):
        p = tours[k]
        exact = sum(abs(int(x[p[t]]) - int(x[p[(t + 1) % n]])) for t in range(n))
        assert L[k] == float(exact)


def _tour_edges(D, p):
    n = len(p)
    return [float(D[p[t], p[(t + 1) % n]]) for t in range(n)]


def test_tour_length_is_the_correctly_rounded_sum(orc):
    """Eq. 3 fixes no order: the oracle's f is the exact sum of the n fp64
    edge lengths rounded once, i.e. math.fsum (correctly rounded), bit for
    bit, on random planar tours of ragged lengths and on tours that revisit
    short and long edges (clustered cities)."""
    rng = np.random.default_rng(15)
    for n in (3, 4, 31, 32, 33, 63, 1000, 1025):
        for kind in ("uniform", "clustered"):
            if kind == "uniform":
                xy = rng.uniform(0, 1, size=(n, 2)).astype(np.float32)
            else:
                c = rng.uniform(0, 1, size=(max(1, n // 16), 2))
                xy = (c[rng.integers(0, len(c), size=n)] + rng.normal(0, 1e-3, size=(n, 2))).astype(np.float32)
            D = orc.distances(xy)
            tours = np.stack([rng.permutation(n) for _ in range(4)]).astype(np.int32)
            L = orc.tour_lengths(D, tours)
            for k in range(4):
                assert L[k] == math.fsum(_tour_edges(D, tours[k])), (n, kind, k)


def test_tour_length_wide_range_matches_rational(orc):
    """Edge lengths spanning the whole range distances of fp32 coordinates can
    take ([2^-149, 2^130)) and zeros: the oracle equals the nearest double to
    the exact rational sum (Python's float(Fraction) rounds correctly)."""
    rng = np.random.default_rng(16)
    for trial in range(300):
        n = int(rng.integers(3, 40))
        e = rng.uniform(-149, 129, size=(n, n))
        if trial % 3 == 1:                       # a narrow band plus a few outliers
            e = rng.uniform(-3, 1, size=(n, n))
            e[rng.random((n, n)) < 0.05] = rng.uniform(-149, -60)
        D = np.exp2(e) * rng.uniform(1, 2, size=(n, n))
        D[rng.random((n, n)) < 0.1] = 0.0        # coincident cities
        D = np.minimum(D, D.T)
        np.fill_diagonal(D, 0.0)
        tours = np.stack([rng.permutation(n) for _ in range(3)]).astype(np.int32)
        L = orc.tour_lengths(D, tours)
        for k in range(3):
            edges = _tour_edges(D, tours[k])
            exact = sum((Fraction(v) for v in edges), Fraction(0))
            assert L[k] == float(exact), (trial, k)
            assert L[k] == math.fsum(edges)


def test_tour_length_ties_and_lost_bits_golden(orc):
    """Hand-worked sums where any fixed-order fp64 summation is wrong: a tie
    settled by an edge far below it, and edges each below half an ulp of the
    running sum that together move it (tests/golden/tour_length_exact.txt)."""
    rows = [ln.split() for ln in open(golden_path("tour_length_exact.txt")) if ln.strip() and not ln.startswith("#")]
    assert len(rows) >= 7
    differ = 0
    for row in rows:
        edges = [float.fromhex(v) for v in row[:-1]]
        want = float.fromhex(row[-1])
        n = len(edges)
        # a cycle 0 -> 1 -> ... -> n-1 -> 0 whose t-th edge has length edges[t]
        D = np.zeros((n, n))
        for t in range(n):
            a, b = t, (t + 1) % n
            D[a, b] = D[b, a] = edges[t]
        L = orc.tour_lengths(D, np.arange(n, dtype=np.int32)[None, :])
        assert L[0] == want, row
        naive = 0.0
        for v in edges:
            naive += v
        differ += naive != want
    assert differ >= 4   # a left-to-right sum would fail this pin


def _rnbf16(x: Fraction) -> np.float32:
    """Nearest bfloat16 to the rational x >= 0 (ties to even), as fp32."""
    if x >= Fraction(2) ** 128 - Fraction(2) ** 119:
        return np.float32(np.inf)
    if x == 0:
        return np.float32(0)
    e = math.floor(math.log2(x)) if x >= Fraction(2) ** -126 else -126
    while Fraction(2) ** e > x:          # guard the float log2 against rounding
        e -= 1
    while Fraction(2) ** (e + 1) <= x and e >= -126:
        e += 1
    q = Fraction(2) ** (max(e, -126) - 7)
    lo = (x // q) * q
    hi = lo + q
    if x - lo < hi - x:
        r = lo
    elif hi - x < x - lo:
        r = hi
    else:
        r = lo if (lo / q) % 2 == 0 else hi
    return np.float32(float(r))


def test_exact_sum_bf16_matches_rational(orc):
    rng = np.random.default_rng(16)
    cases = []
    for _ in range(3000):
        k = int(rng.integers(1, 10))
        kind = int(rng.integers(0, 4))
        if kind == 0:
            x = rng.uniform(1e-4, 2.0, size=k)
        elif kind == 1:
            x = np.exp(rng.normal(0, 20, size=k).clip(-700, 80))
        elif kind == 2:  # a bf16 value plus half its quantum, and a push either way or none
            bits = np.array([rng.uniform(0.5, 4.0)], np.float32).view(np.uint32) & np.uint32(0xFFFF0000)
            a = float(bits.view(np.float32)[0])                  # a bf16 value
            half = 2.0 ** (math.floor(math.log2(a)) - 8)         # half its quantum
            x = np.array([a, half, [0.0, 2.0 ** -60, 2.0 ** -20][int(rng.integers(0, 3))]])
        else:  # the subnormal bf16 range
            x = rng.uniform(0, 2.0 ** -126, size=k)
        cases.append(np.asarray(x, np.float64))
    for x in cases:
        exact = sum((Fraction(float(v)) for v in x), Fraction(0))
        got = orc.exact_sum_bf16(x)
        ref = _rnbf16(exact)
        assert got == ref, (x.tolist(), got, ref)
        assert (np.array(got, np.float32).view(np.uint32) & 0xFFFF) == 0   # a bf16 value


def test_deposit_tau_bf16_is_rounded_exact_sum(orc):
    rng = np.random.default_rng(17)
    for trial in range(4):
        n, m = int(rng.integers(3, 8)), int(rng.integers(1, 6))
        tours = np.stack([rng.permutation(n) for _ in range(m)]).astype(np.int32)
        L = rng.uniform(0.5, 3.0, size=m)
        rho, Q = np.float32(rng.uniform(0, 1)), np.float32(rng.uniform(0.1, 5))
        tau0 = (orc.to_bf16(rng.uniform(0.01, 2, size=(n, n)).astype(np.float32)).astype(np.uint32) << 16).view(np.float32)
        got = orc.deposit_tau_bf16(tau0, tours, L, float(rho), float(Q))
        keep = np.float32(np.float32(1) - rho)
        acc = [[Fraction(float(np.float32(keep * tau0[i, j]))) for j in range(n)] for i in range(n)]
        for k in range(m):
            w = Fraction(float(np.float64(Q) / L[k]))
            for t in range(n):
                a, b = int(tours[k, t]), int(tours[k, t - 1])
                acc[a][b] += w
                acc[b][a] += w
        for i in range(n):
            for j in range(n):
                assert got[i, j] == _rnbf16(acc[i][j]), (trial, i, j)
