"""Oracle pins for the roulette-wheel selection (Sec. 2.4: the classical
selection that independent roulette replaces), in its exact integer reading:
q_j = floor(p_j 2^(40-e)) with e = floor(log2 max unvisited p), a 64-bit
Philox uniform u, target floor(u S / 2^64), first unvisited j whose running
sum exceeds it."""
import itertools
import math
from fractions import Fraction

import numpy as np
from scipy import stats

from paper_2404_04895_gb300 import instances


def _exponent(p):
    return math.floor(math.log2(Fraction(float(p))))  # exact for fp32 values


def test_quantum_is_exact_floor(orc):
    rng = np.random.default_rng(31)
    vals = np.concatenate([rng.uniform(0, 1, 3000), np.exp(rng.normal(0, 30, 3000).clip(-100, 88)),
                           (rng.integers(1, 1 << 23, 500) * 2.0 ** -149)]).astype(np.float32)
    vals = vals[np.isfinite(vals) & (vals > 0)]
    for p in vals:
        for shift in (0, 1, 5, 40, 70):
            e = _exponent(p) + shift            # any row maximum at or above p
            want = math.floor(Fraction(float(p)) * Fraction(2) ** (40 - e))
            assert orc.rw_quantum(p, e) == want
    assert orc.rw_quantum(0.0, 3) == 0


def _select_reference(orc, row, visited, seed, it, k, t):
    """The definition with Python integers (Philox words from the pinned block)."""
    unv = [j for j in range(len(row)) if not visited[j]]
    pmax = max(float(row[j]) for j in unv)
    if pmax == 0:
        return unv[0]
    e = _exponent(np.float32(pmax))
    q = {j: math.floor(Fraction(float(row[j])) * Fraction(2) ** (40 - e)) for j in unv}
    S = sum(q.values())
    w = orc.philox([1 << 30, t, k, it], [seed & 0xFFFFFFFF, seed >> 32])
    u = (int(w[0]) << 32) | int(w[1])
    v = (u * S) >> 64
    run = 0
    for j in unv:
        run += q[j]
        if run > v:
            return j
    raise AssertionError("no pick")


def test_selection_matches_integer_definition(orc):
    rng = np.random.default_rng(32)
    for trial in range(400):
        n = int(rng.integers(2, 40))
        row = (rng.uniform(0, 1, n) ** 3 * np.exp(rng.normal(0, 8, n))).astype(np.float32)
        if trial % 5 == 0:
            row[rng.integers(0, n, n // 2)] = 0
        visited = rng.random(n) < 0.4
        if visited.all():
            visited[rng.integers(0, n)] = False
        seed = int(rng.integers(0, 1 << 62))
        it, k, t = (int(x) for x in rng.integers(0, 1000, 3))
        assert orc.select_rw(row, visited, seed, it, k, t) == _select_reference(orc, row, visited, seed, it, k, t)


def test_all_zero_row_picks_lowest_unvisited(orc):
    row = np.zeros(9, np.float32)
    vis = np.array([1, 1, 0, 1, 0, 0, 1, 0, 0], bool)
    for k in range(20):
        assert orc.select_rw(row, vis, 5, 0, k, 1) == 2


def test_first_step_follows_normalised_row(orc):
    """Chi-square: RW's first-step choices follow the normalised P row (the
    law IR does not follow, see test_oracle_path), and IR's do not."""
    P = np.array([[0, 1, 3, 9, 0.5],
                  [2, 0, 2, 5, 1],
                  [8, 0.3, 0, 1, 4],
                  [1, 1, 1, 0, 1],
                  [0.2, 6, 0.7, 2.5, 0]], dtype=np.float32)
    m = 60000
    counts_rw = np.zeros((5, 5))
    tours = orc.construct_rw(P, 321, 0, 0, m)
    np.add.at(counts_rw, (tours[:, 0], tours[:, 1]), 1)
    counts_ir = np.zeros((5, 5))
    tours = orc.construct(P, 321, 0, 0, m)
    np.add.at(counts_ir, (tours[:, 0], tours[:, 1]), 1)
    chi_rw = chi_ir = 0.0
    dof = 0
    for s in range(5):
        cand = [j for j in range(5) if j != s]
        norm = P[s, cand] / P[s, cand].sum()
        for counts, acc in ((counts_rw, "rw"), (counts_ir, "ir")):
            obs = counts[s, cand]
            exp = obs.sum() * norm
            val = ((obs - exp) ** 2 / exp).sum()
            if acc == "rw":
                chi_rw += val
            else:
                chi_ir += val
        dof += len(cand) - 1
    assert stats.chi2.sf(chi_rw, dof) > 1e-4
    assert stats.chi2.sf(chi_ir, dof) < 1e-9


def test_whole_rw_runs_valid_and_never_below_optimum(orc):
    for n in (6, 7):
        xy = instances.uniform(n, 400 + n)
        D = orc.distances(xy)
        best = min(sum(D[p[t], p[(t + 1) % n]] for t in range(n))
                   for p in ((0,) + q for q in itertools.permutations(range(1, n))))
        s = orc.State(xy, m=n, rho=0.3, seed=n, rw=True).run(40)
        assert s.best_len[0] >= best - 1e-12
        assert s.best_len[0] <= best * 1.1
        for tour in s.last_tours:
            assert sorted(tour.tolist()) == list(range(n))
