"""Oracle pins for the path itself: distances and eta (Sec. 2.1), M_p (Eq. 1),
IR / AdaIR selection laws (Sec. 2.4), fitness (Eq. 3), index matrix (Eq. 2),
evaporation + deposit (Sec. 2.3), and whole runs against brute-force optima."""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

from conftest import golden_path
from paper_2404_04895_gb300 import instances

SQUARE = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float32)


# ---------------------------------------------------------------- Sec. 2.1
def test_distances_closed_forms(orc):
    D = orc.distances(SQUARE)
    assert D[0, 1] == 1.0 and D[1, 2] == 1.0 and D[0, 3] == 1.0
    assert D[0, 2] == math.sqrt(2.0) and D[1, 3] == math.sqrt(2.0)
    assert np.all(np.diag(D) == 0)
    xy = instances.uniform(60, 5)
    D = orc.distances(xy)
    assert np.array_equal(D, D.T)                      # bitwise symmetric
    i, j, k = np.random.default_rng(0).integers(0, 60, size=(3, 2000))
    assert np.all(D[i, k] <= D[i, j] + D[j, k] + 1e-15)  # triangle inequality
    # 3-4-5 triangle
    D = orc.distances(np.array([[0, 0], [0.75, 0], [0.75, 1.0]], dtype=np.float32))
    assert D[0, 2] == 1.25


def test_heuristic_closed_forms(orc):
    xy = np.array([[0, 0], [0.5, 0], [0.5, 0.25], [0.5, 0.25]], dtype=np.float32)
    D = orc.distances(xy)
    H = orc.heuristic(D, 2)
    assert H[0, 1] == 4.0                              # (1/0.5)^2
    assert H[1, 2] == 16.0                             # (1/0.25)^2
    assert H[2, 3] == np.float32(1e18)                 # coincident: (1/1e-9)^2
    assert np.all(np.diag(H) == 0)
    assert orc.heuristic(D, 0)[0, 1] == 1.0
    assert orc.heuristic(D, 3)[0, 1] == 8.0


def test_build_P_eq1_unnormalised(orc):
    xy = instances.uniform(40, 7)
    H = orc.heuristic(orc.distances(xy), 2)
    tau = np.ones((40, 40), dtype=np.float32)
    P, _, _ = orc.build_P(tau, H, alpha=1)
    assert np.array_equal(P, H)                         # tau = 1: M_p = eta^beta
    P, _, _ = orc.build_P(2 * tau, H, alpha=3)
    assert np.array_equal(P, 8 * H)                     # 2^3 scales exactly
    P0, _, _ = orc.build_P(np.full_like(tau, 0.3), H, alpha=0)
    assert np.array_equal(P0, H)
    assert np.all(np.diag(P) == 0)
    # BF16: the stored value is the RNE rounding of the fp32 product
    rng = np.random.default_rng(1)
    tau = rng.uniform(0.1, 3, size=(40, 40)).astype(np.float32)
    P32, _, _ = orc.build_P(tau, H, alpha=2)
    Pb, bits, _ = orc.build_P(tau, H, alpha=2, prec=orc.BF16)
    import torch
    ref = torch.from_numpy(P32).to(torch.bfloat16).float().numpy()
    assert np.array_equal(Pb, ref)
    assert np.array_equal(bits, orc.to_bf16(P32))


def test_build_P_fp16_row_scale(orc):
    xy = instances.clustered(5, 20, 0.02, seed=3)
    H = orc.heuristic(orc.distances(xy), 2)
    tau = np.ones(H.shape, dtype=np.float32)
    P32, _, _ = orc.build_P(tau, H, alpha=1)
    Ph, bits, e = orc.build_P(tau, H, alpha=1, prec=orc.FP16)
    for i in range(H.shape[0]):
        rowmax = P32[i].max()
        scaled = rowmax * 2.0 ** (-int(e[i]))
        assert 2.0 ** 14 <= scaled < 2.0 ** 15
        # the stored value is the fp16 RNE rounding of X * 2^-e_i
        ref = (P32[i] * np.float32(2.0 ** (-int(e[i])))).astype(np.float16).astype(np.float32)
        assert np.array_equal(Ph[i], ref)
    assert np.all(np.isfinite(Ph))


def test_build_P_adair_exponent(orc):
    xy = instances.uniform(30, 9)
    H = orc.heuristic(orc.distances(xy), 2)
    tau = np.random.default_rng(2).uniform(0.5, 2, size=H.shape).astype(np.float32)
    X, _, _ = orc.build_P(tau, H, alpha=1)
    inv = orc.inv_gamma(1.5)
    Pg, _, _ = orc.build_P(tau, H, alpha=1, inv_gamma=inv)
    assert np.array_equal(Pg, orc.pow_own(X, inv))
    # gamma = 1 is the plain IR matrix, bit for bit
    P1, _, _ = orc.build_P(tau, H, alpha=1, inv_gamma=orc.inv_gamma(1.0))
    assert np.array_equal(P1, X)


# ---------------------------------------------------------------- Sec. 2.4
def ir_law(p):
    """Exact IR selection law: P(j) = int_0^1 prod_{i != j} min(1, x p_j / p_i) dx."""
    p = np.asarray(p, dtype=np.float64)
    out = np.zeros(p.size)
    for j in range(p.size):
        if p[j] <= 0:
            continue
        others = np.delete(p, j)
        bps = sorted({0.0, 1.0} | {float(q / p[j]) for q in others if q / p[j] < 1.0})
        tot = 0.0
        for a, b in zip(bps[:-1], bps[1:]):
            mid = 0.5 * (a + b)
            act = others[mid < others / p[j]]
            c = float(np.prod(p[j] / act))
            q = act.size
            tot += c * (b ** (q + 1) - a ** (q + 1)) / (q + 1)
        out[j] = tot
    return out


def test_ir_law_is_a_distribution():
    p = np.array([0.1, 0.5, 2.0, 2.0, 7.0])
    pi = ir_law(p)
    assert abs(pi.sum() - 1) < 1e-12
    assert abs(pi[2] - pi[3]) < 1e-15
    # two candidates: the larger wins with probability 1 - a/2, a = small/large
    pi2 = ir_law([1.0, 4.0])
    assert abs(pi2[1] - (1 - 0.25 / 2)) < 1e-15


def _first_step_counts(orc, P, m, seed):
    n = P.shape[0]
    tours = orc.construct(P, seed, 0, 0, m)
    counts = np.zeros((n, n))
    np.add.at(counts, (tours[:, 0], tours[:, 1]), 1)
    return counts


def test_first_step_follows_exact_ir_law(orc):
    P = np.array([[0, 1, 3, 9, 0.5],
                  [2, 0, 2, 5, 1],
                  [8, 0.3, 0, 1, 4],
                  [1, 1, 1, 0, 1],
                  [0.2, 6, 0.7, 2.5, 0]], dtype=np.float32)
    counts = _first_step_counts(orc, P, 60000, seed=123)
    chi, dof, chi_norm = 0.0, 0, 0.0
    for s in range(5):
        cand = [j for j in range(5) if j != s]
        obs = counts[s, cand]
        N = obs.sum()
        exp_ir = N * ir_law(P[s, cand])
        exp_norm = N * P[s, cand] / P[s, cand].sum()
        chi += ((obs - exp_ir) ** 2 / exp_ir).sum()
        chi_norm += ((obs - exp_norm) ** 2 / exp_norm).sum()
        dof += len(cand) - 1
    assert stats.chi2.sf(chi, dof) > 1e-4
    # negative control: IR is not the normalised-row roulette (Fig. 4's lateral shift)
    assert stats.chi2.sf(chi_norm, dof) < 1e-9


@pytest.mark.parametrize("g", [1.0, 0.5, 2.0])
def test_two_candidate_closed_form(orc, g):
    # three cities: from start s the two candidates have p_small, p_large;
    # IR picks the larger with prob 1 - a/2, a = (p_small/p_large)^(1/gamma) under AdaIR
    H = np.array([[0, 1, 4], [1, 0, 2], [4, 2, 0]], dtype=np.float32)
    tau = np.ones_like(H)
    P, _, _ = orc.build_P(tau, H, alpha=1, inv_gamma=orc.inv_gamma(g))
    counts = _first_step_counts(orc, P, 90000, seed=7)
    for s in range(3):
        a_, b_ = [j for j in range(3) if j != s]
        lo, hi = sorted([H[s, a_], H[s, b_]])
        big = a_ if H[s, a_] > H[s, b_] else b_
        a = (lo / hi) ** (1.0 / g)
        p_big = 1 - a / 2
        N = counts[s, a_] + counts[s, b_]
        z = (counts[s, big] - N * p_big) / math.sqrt(N * p_big * (1 - p_big))
        assert abs(z) < 4.5, (s, z)


def test_literal_adair_agrees_with_power_form(orc):
    # argmax(r^gamma p) == argmax(r p^(1/gamma)) except at near-ties
    rng = np.random.default_rng(4)
    agree = total = 0
    for trial in range(3000):
        n = 40
        row = np.exp(rng.normal(0, 2, size=n)).astype(np.float32)
        vis = (rng.random(n) < 0.3).astype(np.uint8)
        if vis.all():
            continue
        g = float(rng.choice([0.5, 0.75, 1.25, 1.5]))
        inv = orc.inv_gamma(np.float32(g))
        a = orc.select(orc.pow_own(row, inv), vis, 11, 2, trial, 3)
        b = orc.select_literal_adair(row, vis, 11, 2, trial, 3, float(np.float32(g)))
        agree += a == b
        total += 1
    assert agree / total >= 0.9999


def test_row_normalisation_invariance(orc):
    # Eq. 1 divides each row by its sum; IR's argmax ignores a positive row scale
    rng = np.random.default_rng(5)
    same_pow2 = same_norm = 0
    for trial in range(2000):
        row = np.exp(rng.normal(0, 2, size=30)).astype(np.float32)
        vis = (rng.random(30) < 0.2).astype(np.uint8)
        a = orc.select(row, vis, 3, 0, trial, 1)
        same_pow2 += a == orc.select(row * np.float32(2.0 ** -7), vis, 3, 0, trial, 1)
        same_norm += a == orc.select(row / row.sum(dtype=np.float32), vis, 3, 0, trial, 1)
    assert same_pow2 == 2000
    assert same_norm >= 1995


def test_construct_permutations_and_starts(orc):
    xy = instances.uniform(37, 2)
    H = orc.heuristic(orc.distances(xy), 2)
    P, _, _ = orc.build_P(np.ones_like(H), H, alpha=1)
    tours = orc.construct(P, 99, 4, 10, 30)
    for r, k in enumerate(range(10, 30)):
        assert sorted(tours[r]) == list(range(37))
        assert tours[r, 0] == orc.start_city(99, 4, k, 37)


def test_nearest_neighbour_limit(orc):
    # beta = 30 on cities whose nearest unvisited neighbour is always >= 2x closer
    # than the next: the P ratio 2^30 exceeds 1/min(r) = 2^24, so IR is greedy.
    xy = instances.line_geometric(6, ratio=3.0, scale=0.1)
    D = orc.distances(xy)
    H = orc.heuristic(D, 30)
    P, _, _ = orc.build_P(np.ones_like(H), H, alpha=0)
    tours = orc.construct(P, 5, 0, 0, 60)
    for tour in tours:
        cur, vis, nn = int(tour[0]), {int(tour[0])}, [int(tour[0])]
        for _ in range(5):
            cand = [j for j in range(6) if j not in vis]
            cur = min(cand, key=lambda j: D[cur, j])
            vis.add(cur)
            nn.append(cur)
        assert list(tour) == nn


# ---------------------------------------------------------------- Eq. 3 fitness
def test_tour_length_closed_forms(orc):
    D = orc.distances(SQUARE)
    L = orc.tour_lengths(D, np.array([[0, 1, 2, 3], [0, 2, 1, 3]], dtype=np.int32))
    assert L[0] == 4.0
    assert abs(L[1] - (2 + 2 * math.sqrt(2))) < 1e-15
    xy = np.array([[0, 0], [0.5, 0], [1.5, 0], [3, 0]], dtype=np.float32)
    L = orc.tour_lengths(orc.distances(xy), np.array([[0, 1, 2, 3], [2, 0, 3, 1]], dtype=np.int32))
    assert L[0] == 6.0                                  # out and back along the line
    assert L[1] == 1.5 + 3 + 2.5 + 1.0


# ---------------------------------------------------------------- Sec. 2.3
def test_index_matrix_eq2(orc):
    I = orc.index_matrix(np.array([3, 0, 2, 1], dtype=np.int32))
    assert I.tolist() == [[3, 1], [0, 3], [2, 0], [1, 2]]


def test_deposit_worked_example(orc):
    ref = np.loadtxt(golden_path("deposit_unit_square.txt"), dtype=np.float64)
    D = orc.distances(SQUARE)
    tours = np.array([[0, 1, 2, 3]], dtype=np.int32)
    L = orc.tour_lengths(D, tours)
    assert L[0] == 4.0
    tau = orc.deposit(np.ones((4, 4), np.float32), tours, L, rho=0.5, Q=1.0)
    assert np.array_equal(tau.astype(np.float64), ref)


def test_evaporation_closed_form(orc):
    rng = np.random.default_rng(6)
    tours = np.stack([rng.permutation(12) for _ in range(5)]).astype(np.int32)
    L = rng.uniform(1, 5, size=5)
    rho = np.float32(0.1)
    tau = np.ones((12, 12), np.float32)
    keep = np.float32(1) - rho              # evaporation in fp32, the precision of M_tau
    for t in range(1, 61):
        tau = orc.deposit(tau, tours, L, rho=float(rho), Q=0.0)
        exact = float(keep) ** t
        ulp = 2.0 ** (math.frexp(exact)[1] - 24)
        assert np.all(np.abs(tau.astype(np.float64) - exact) <= t * ulp)
        assert np.all(tau == tau[0, 0])


def test_deposit_symmetry_sum_and_support(orc):
    rng = np.random.default_rng(7)
    n, m = 25, 9
    tours = np.stack([rng.permutation(n) for _ in range(m)]).astype(np.int32)
    L = rng.uniform(2, 9, size=m)
    tau0 = rng.uniform(0.5, 2, size=(n, n)).astype(np.float32)
    tau0 = np.minimum(tau0, tau0.T)                      # symmetric start
    rho, Q = 0.25, 3.0
    tau = orc.deposit(tau0, tours, L, rho, Q)
    assert np.array_equal(tau, tau.T)
    evap = (np.float32(1) - np.float32(rho)) * tau0      # fp32 evaporation
    delta = tau.astype(np.float64) - evap.astype(np.float64)
    c = Q / L
    assert abs(delta.sum() - 2 * n * c.sum()) < 1e-5 * 2 * n * c.sum()
    # one ant changes exactly its 2n directed tour entries
    one = orc.deposit(tau0, tours[:1], L[:1], rho, Q)
    changed = one != evap
    assert changed.sum() == 2 * n
    I = orc.index_matrix(tours[0])
    for a, b in I:
        assert changed[a, b] and changed[b, a]


def test_fp32_atomic_reading_close_to_fp64(orc):
    rng = np.random.default_rng(8)
    n, m = 30, 200
    tours = np.stack([rng.permutation(n) for _ in range(m)]).astype(np.int32)
    L = rng.uniform(2, 9, size=m)
    tau0 = np.ones((n, n), np.float32)
    ref = orc.deposit(tau0, tours, L, 0.1, 1.0)
    perm = rng.permutation(2 * m * n)
    got = orc.deposit_fp32_order(tau0, tours, L, 0.1, 1.0, perm)
    assert np.max(np.abs(got - ref) / ref) < 1e-5


# ---------------------------------------------------------------- whole runs
def _brute_force_opt(D):
    n = D.shape[0]
    best = math.inf
    for perm in itertools.permutations(range(1, n)):
        p = (0,) + perm
        if p[1] > p[-1]:
            continue
        s = sum(D[p[t], p[(t + 1) % n]] for t in range(n))
        best = min(best, s)
    return best


def test_whole_oracle_reaches_brute_force_optimum(orc):
    hits = total = 0
    for n in (5, 6, 7, 8):
        for seed in range(6):
            xy = instances.uniform(n, 100 + seed)
            st = orc.State(xy, m=n, alpha=1, beta=2, rho=0.5, Q=1.0, seed=seed).run(100, nthreads=1)
            opt = _brute_force_opt(st.D)
            assert st.best_len[0] >= opt * (1 - 1e-12)      # never below the optimum
            assert st.best_len[0] <= opt * 1.05             # a heuristic, but a good one
            hits += abs(st.best_len[0] - opt) <= 1e-12 * opt
            total += 1
            for k, tour in enumerate(st.last_tours):
                assert sorted(tour) == list(range(n))
                assert tour[0] == orc.start_city(seed, 99, k, n)
    # Ant System with m = n ants, rho = 1/2 stagnates on a few seeds; most reach the optimum
    assert hits >= 0.75 * total, (hits, total)


def test_run_resume_is_bit_exact(orc):
    xy = instances.uniform(20, 3)
    a = orc.State(xy, m=10, rho=0.2, seed=5, adair=True, gamma_T=30).run(30, nthreads=2)
    b = orc.State(xy, m=10, rho=0.2, seed=5, adair=True, gamma_T=30).run(12, nthreads=2).run(18, nthreads=2)
    assert np.array_equal(a.tau, b.tau)
    assert np.array_equal(a.best_tour, b.best_tour) and a.best_len[0] == b.best_len[0]
    assert np.array_equal(a.last_tours, b.last_tours)
