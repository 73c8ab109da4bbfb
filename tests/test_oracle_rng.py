"""Oracle pins: Philox4x32-10, the uniform map, T_start (Sec. 2.2 / 2.4)."""
import numpy as np
import pytest
from scipy import stats

from conftest import golden_path


def _kat():
    rows = []
    with open(golden_path("philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert list(orc.philox(ctr, key)) == out


def test_draw_counter_layout(orc):
    # word j&3 of Philox(counter=(j>>2, t, k, it), key=(seed lo, seed hi))
    seed = 0x0123456789ABCDEF
    for (it, k, t, j) in [(0, 0, 1, 0), (3, 17, 5, 6), (199, 999, 998, 1023), (7, 2, 9, 4097)]:
        ref = orc.philox([j >> 2, t, k, it], [seed & 0xFFFFFFFF, seed >> 32])[j & 3]
        assert orc.draw(seed, it, k, t, j) == ref
    # distinct candidates of one block draw distinct words
    w = {orc.draw(1, 0, 0, 1, j) for j in range(4)}
    assert len(w) == 4


def test_uniform_map_exact_and_open(orc):
    assert orc.uniform(0) == 2.0 ** -24
    assert orc.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert orc.uniform(0x100) == 2.0 ** -24          # (1 | 1) * 2^-24
    assert orc.uniform(0x200) == 3 * 2.0 ** -24      # (2 | 1) * 2^-24
    assert orc.uniform(0x80000000) == 0.5 + 2.0 ** -24


def test_uniform_moments(orc):
    rng = np.random.default_rng(0)
    xs = [orc.uniform(orc.draw(5, 0, int(k), 1, int(j)))
          for k, j in rng.integers(0, 1 << 20, size=(20000, 2))]
    xs = np.array(xs)
    assert np.all((xs > 0) & (xs < 1))
    # mean 1/2, variance 1/12 within 5 sigma
    assert abs(xs.mean() - 0.5) < 5 * np.sqrt(1 / 12 / xs.size)
    assert stats.kstest(xs, "uniform").pvalue > 1e-3


def test_start_city_range_and_uniformity(orc):
    n = 7
    counts = np.zeros(n)
    for k in range(14000):
        s = orc.start_city(42, 3, k, n)
        assert 0 <= s < n
        counts[s] += 1
    assert stats.chisquare(counts).pvalue > 1e-3
    # Lemire: start = (x * n) >> 32 with x = word 0 of counter (0, 0, k, it)
    x = orc.philox([0, 0, 5, 3], [42, 0])[0]
    assert orc.start_city(42, 3, 5, 1000) == (int(x) * 1000) >> 32
