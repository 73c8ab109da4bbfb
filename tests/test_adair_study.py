"""The AdaIR visualisation study (Sec. 3.3.1, Fig. 4): the exact law of the
row maximum under independent roulette, the GPU Bernoulli-trial kernel
against the oracle and against that law, and an end-to-end run."""
import numpy as np
import pytest

from paper_2404_04895_gb300 import adair_study
from test_oracle_path import ir_law


def test_max_law_matches_piecewise_ir_law():
    rng = np.random.default_rng(41)
    for trial in range(60):
        n = int(rng.integers(2, 9))
        q = rng.uniform(0.01, 5, size=n) ** rng.uniform(0.5, 3)
        if trial % 4 == 0:
            q[1:3] = q[0] * rng.uniform(0.999, 1.0)    # near ties with the maximum
        assert abs(adair_study.ir_law_max(q) - ir_law(q)[int(np.argmax(q))]) < 1e-12


def test_max_law_limits():
    assert adair_study.ir_law_max(np.array([1.0])) == 1.0
    assert abs(adair_study.ir_law_max(np.array([1.0, 1.0])) - 0.5) < 1e-15
    assert abs(adair_study.ir_law_max(np.array([2.0, 1.0])) - 0.75) < 1e-15   # 1 - a/2
    # a large row (the study's sizes) is a probability and stays finite
    q = np.random.default_rng(1).uniform(0, 1, 422) ** 6
    v = adair_study.ir_law_max(q)
    assert 0 < v <= 1 and np.isfinite(v)


@pytest.mark.gpu
def test_selection_counts_match_oracle(orc):
    import torch
    from paper_2404_04895_gb300 import binding as B
    rng = np.random.default_rng(42)
    n = 37
    q = (rng.uniform(0, 1, n) ** 4).astype(np.float32)
    q[5] = 0.0
    vis = np.zeros(n, np.uint8)
    vis[[2, 9, 30]] = 1
    trials = 3000
    got = torch.zeros(n, dtype=torch.int64, device="cuda")
    B.op_selection_counts(torch.from_numpy(q).cuda(), n, trials, 77, got, salt=3,
                          visited=torch.from_numpy(vis).cuda())
    ref = orc.selection_counts(q, trials, 77, salt=3, visited=vis)
    assert np.array_equal(got.cpu().numpy().astype(np.uint64), ref)
    assert int(ref.sum()) == trials and ref[[2, 9, 30]].sum() == 0


@pytest.mark.gpu
def test_selection_frequency_follows_ir_law():
    import torch
    from paper_2404_04895_gb300 import binding as B
    rng = np.random.default_rng(43)
    n = 60
    q = (rng.uniform(0, 1, n) ** 3).astype(np.float32)
    trials = 4_000_000
    counts = torch.zeros(n, dtype=torch.int64, device="cuda")
    B.op_selection_counts(torch.from_numpy(q).cuda(), n, trials, 5, counts)
    c = counts.cpu().numpy()
    jm = int(np.argmax(q))
    pi = adair_study.ir_law_max(q.astype(np.float64))
    phat = c[jm] / trials
    assert abs(phat - pi) < 5 * np.sqrt(pi * (1 - pi) / trials)


@pytest.mark.gpu
def test_study_runs_end_to_end():
    out = adair_study.run(n_list=(40,), iters=(0, 3), gammas=(1.0, 1.5), rows=3, trials_per_ant=500)
    assert len(out) == 4
    for rec in out:
        assert 0 < rec["p_max_rw"] <= 1 and 0 < rec["p_hat_max"] <= 1
        assert rec["max_abs_hat_minus_law"] < 0.02
    # AdaIR (gamma 1.5) favours the maximum less than IR, the paper's exploration knob
    by = {(r["iteration"], r["gamma"]): r for r in out}
    assert by[(0, 1.5)]["p_max_ir_law"] < by[(0, 1.0)]["p_max_ir_law"]
