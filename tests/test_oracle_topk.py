"""Oracle pins for the paper's selection of deposit paths (Sec. 2.3,
"tensorization of ant path": the solution set sorted by fitness, the top k
paths deposit; k = n/10 in the paper's experiments)."""
from fractions import Fraction

import numpy as np

from test_oracle_exact_sums import _rn32


def test_selection_matches_lexsort_with_ties(orc):
    rng = np.random.default_rng(21)
    for trial in range(40):
        m = int(rng.integers(1, 300))
        L = rng.integers(1, 12, size=m).astype(np.float64) * 0.5  # many equal lengths
        for k in (1, 3, max(1, m // 10), m - 1, m, m + 5, 0, -2):
            got = orc.select_topk(L, k)
            take = m if (k <= 0 or k >= m) else k
            order = np.lexsort((np.arange(m), L))            # length, then ant index
            want = np.zeros(m, bool)
            want[order[:take]] = True
            assert np.array_equal(got, want), (trial, m, k)


def test_all_paths_is_ant_system(orc):
    rng = np.random.default_rng(22)
    n, m = 30, 12
    tours = np.stack([rng.permutation(n) for _ in range(m)]).astype(np.int32)
    L = rng.uniform(2, 9, size=m)
    tau0 = rng.uniform(0.5, 2, size=(n, n)).astype(np.float32)
    ref = orc.deposit(tau0, tours, L, 0.2, 1.5)
    for k in (0, m, m + 1):
        got = orc.deposit_topk(tau0, tours, L, 0.2, 1.5, k)
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_single_best_path_closed_form(orc):
    rng = np.random.default_rng(23)
    n, m = 11, 7
    tours = np.stack([rng.permutation(n) for _ in range(m)]).astype(np.int32)
    L = rng.uniform(2, 9, size=m)
    L[4] = L.min() * 0.5
    L[5] = L[4]                                          # a tie: ant 4 (lower index) is first
    tau0 = rng.uniform(0.5, 2, size=(n, n)).astype(np.float32)
    rho, Q = np.float32(0.3), np.float32(2.0)
    got = orc.deposit_topk(tau0, tours, L, float(rho), float(Q), 1)
    keep = np.float32(1) - rho
    evap = keep * tau0
    c = Fraction(float(np.float64(Q) / L[4]))
    on = np.zeros((n, n), bool)
    p = tours[4]
    for t in range(n):
        on[p[t], p[t - 1]] = on[p[t - 1], p[t]] = True
    for i in range(n):
        for j in range(n):
            want = _rn32(Fraction(float(evap[i, j])) + c) if on[i, j] else evap[i, j]
            assert got[i, j] == want
    assert on.sum() == 2 * n


def test_whole_run_with_top_paths(orc):
    """k = 2 of m = n ants on small instances still finds near-optimal tours
    and never reports a length below the brute-force optimum."""
    import itertools
    from paper_2404_04895_gb300 import instances
    gaps = []
    for n in (6, 7, 8):
        xy = instances.uniform(n, 300 + n)
        D = orc.distances(xy)
        best = min(sum(D[p[t], p[(t + 1) % n]] for t in range(n))
                   for p in ((0,) + q for q in itertools.permutations(range(1, n))))
        s = orc.State(xy, m=n, rho=0.3, seed=n, topk=2).run(60)
        assert s.best_len[0] >= best - 1e-12
        gaps.append(s.best_len[0] / best - 1)
    assert max(gaps) < 0.05
