"""Oracle pins: IEEE rounding to BF16/FP16, integer powers, own pow for AdaIR,
the cosine-annealed gamma schedule and the law of r^gamma (Sec. 2.4, Eq. 4-5)."""
import math
from fractions import Fraction

import numpy as np
import pytest
import torch
from scipy import stats


def _bf16_bits_torch(x):
    return torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)


def _sample_fp32_patterns():
    hi = np.arange(1 << 16, dtype=np.uint32) << 16
    lows = np.array([0, 1, 0x7FFF, 0x8000, 0x8001, 0xFFFF, 0x4000, 0xC000], dtype=np.uint32)
    pats = (hi[:, None] | lows[None, :]).ravel()
    rng = np.random.default_rng(1)
    pats = np.concatenate([pats, rng.integers(0, 1 << 32, size=1 << 21, dtype=np.uint64).astype(np.uint32)])
    return pats


def test_bf16_rne_matches_torch(orc):
    pats = _sample_fp32_patterns()
    x = pats.view(np.float32)
    finite = ~np.isnan(x)
    got = orc.to_bf16(x)
    ref = _bf16_bits_torch(x)
    assert np.array_equal(got[finite], ref[finite])
    nan_bits = (got[~finite].astype(np.uint32) << 16).view(np.float32)
    assert np.all(np.isnan(nan_bits))


def test_fp16_rne_matches_numpy_and_torch(orc):
    pats = _sample_fp32_patterns()
    x = pats.view(np.float32)
    finite = ~np.isnan(x)
    got = orc.to_fp16(x)
    ref_np = x.astype(np.float16).view(np.uint16)
    ref_t = torch.from_numpy(x).to(torch.float16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(got[finite], ref_np[finite])
    assert np.array_equal(got[finite], ref_t[finite])
    # boundary cases: max normal, first overflow tie, smallest subnormal and its half
    cases = np.array([65504.0, 65519.996, 65520.0, 2.0 ** -24, 2.0 ** -25, 1.5 * 2.0 ** -25,
                      2.0 ** -14, 2.0 ** -14 - 2.0 ** -25], dtype=np.float32)
    assert np.array_equal(orc.to_fp16(cases), cases.astype(np.float16).view(np.uint16))


def test_powi_exact_within_rounding_bound(orc):
    rng = np.random.default_rng(2)
    xs = np.exp(rng.uniform(np.log(1e-3), np.log(1e3), size=400)).astype(np.float32)
    for x in xs:
        for a in range(0, 9):
            r = orc.powi_f32(float(x), a)
            exact = Fraction(float(x)) ** a
            if a == 0:
                assert r == 1.0
                continue
            # a-1 roundings, each within 2^-24 relative
            bound = ((1 + Fraction(1, 1 << 24)) ** (a - 1) - 1) * exact
            assert abs(Fraction(r) - exact) <= bound
            r64 = orc.powi_f64(float(x), a)
            bound64 = ((1 + Fraction(1, 1 << 53)) ** (a - 1) - 1) * exact
            assert abs(Fraction(r64) - exact) <= bound64
    # powers of two are exact
    for k in range(-10, 11):
        assert orc.powi_f32(2.0 ** k, 3) == 2.0 ** (3 * k)


def _ulp32(v):
    v = abs(float(v))
    if v == 0:
        return 2.0 ** -149
    e = math.frexp(v)[1] - 1
    return 2.0 ** max(e - 23, -149)


def test_log2_exp2_exact_points(orc):
    for k in range(-140, 128):
        assert orc.log2_own(2.0 ** k) == k
    for i in range(-126, 128):
        assert orc.exp2_own(float(i)) == 2.0 ** i
    assert orc.exp2_own(200.0) == math.inf
    assert orc.exp2_own(-200.0) == 0.0


def test_pow_own_accuracy_and_monotone(orc):
    rng = np.random.default_rng(3)
    x = np.exp(rng.uniform(np.log(1e-20), np.log(1e20), size=200000)).astype(np.float32)
    for e in [0.5, 2.0 / 3.0, 0.8, 1.25, 1.5, 2.0]:
        e32 = float(np.float32(e))
        got = orc.pow_own(x, e32).astype(np.float64)
        ref = np.power(x.astype(np.float64), e32)
        ok = (ref < 3.0e38) & (ref > 1.2e-38)   # results inside the fp32 normal range
        got, ref = got[ok], ref[ok]
        ulps = np.abs(got - ref) / np.array([_ulp32(v) for v in ref])
        y = np.abs(e32 * np.log2(x[ok].astype(np.float64)))
        # error budget: a few ulps from the polynomials plus the fp32 rounding of
        # y = e * log2(x), amplified by ln2 * |y| in 2^y
        assert np.all(ulps <= 8 + 3.0 * y), ulps.max()
        xs = np.sort(x)
        gs = orc.pow_own(xs, e32).astype(np.float64)
        gs = gs[np.isfinite(gs)]
        assert np.all(np.diff(gs) >= 0), "pow_own must be nondecreasing in x"
    assert orc.pow_own(np.float32([0.0, 1.0, 3.0]), 1.0).tolist() == [0.0, 1.0, 3.0]
    assert orc.pow_own(np.float32([0.0]), 0.5)[0] == 0.0
    assert orc.pow_own(np.float32([1.0]), 0.5)[0] == 1.0


def test_gamma_schedule_cosine(orc):
    T, gmax, gmin = 200, 1.5, 0.5
    g = orc.gamma_schedule(T + 5, T, gmax, gmin)
    assert g[0] == np.float32(gmax)
    assert g[T // 2] == np.float32((gmax + gmin) / 2)
    assert np.all(g[T:] == np.float32(gmin))
    assert np.all(np.diff(g[:T + 1]) <= 0)
    # symmetric about the midpoint: gamma_t + gamma_{T-t} = gmax + gmin
    t = np.arange(1, T)
    assert np.allclose(g[t] + g[T - t], gmax + gmin, atol=1e-6)
    assert orc.inv_gamma(1.0) == 1.0
    assert orc.inv_gamma(0.5) == 2.0


@pytest.mark.parametrize("g", [0.5, 1.0, 1.5, 2.0])
def test_eq5_law_of_r_power_gamma(orc, g):
    # Eq. 5: Y = X^gamma, X ~ U(0,1)  ->  F_Y(y) = y^(1/gamma), E[Y] = 1/(1+gamma)
    ys = np.array([orc.adair_deviate(orc.uniform(orc.draw(9, 1, k, 2, 0)), g) for k in range(20000)])
    assert stats.kstest(ys, lambda y: np.clip(y, 0, 1) ** (1.0 / g)).pvalue > 1e-3
    var = 1 / (1 + 2 * g) - 1 / (1 + g) ** 2
    assert abs(ys.mean() - 1 / (1 + g)) < 5 * math.sqrt(var / ys.size)
    if g != 1.0:
        # the law has power: the untransformed CDF is rejected
        assert stats.kstest(ys, "uniform").pvalue < 1e-6
