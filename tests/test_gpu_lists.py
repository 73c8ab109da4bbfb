"""Candidate lists (the exact fast path of the construction step): the list
of every row holds its top values with a correct bound for everything left
out, and construction with lists gives exactly the tours of the full scan
and of the oracle."""
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


def _keys(Pv, bits, prec):
    if prec == B.FP32:
        return Pv.view(np.uint32)
    return Pv.astype(np.float32).view(np.uint32)


LMAX, LTARGET = B.LIST_MAX, B.LIST_TARGET


def _build(Pd, prec, n, ld):
    lists = torch.zeros((n, LMAX, 2), dtype=torch.int32, device="cuda")
    lcnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    lkey = torch.zeros(n, dtype=torch.int32, device="cuda")
    B.op_build_lists(Pd, prec, n, ld, lists, lcnt, lkey)
    return lists, lcnt, lkey


def _P(orc, n, seed, prec, ties=False):
    xy = instances.clustered(-(-n // 40), 40, 0.02, seed=seed)[:n] if n >= 80 else instances.uniform(n, seed)
    assert xy.shape == (n, 2)
    H = orc.heuristic(orc.distances(xy), 2)
    tau = np.random.default_rng(seed).uniform(0.3, 2.0, size=(n, n)).astype(np.float32)
    if ties:
        tau[:] = 1.0
        H = np.where(H > np.median(H), np.float32(7.0), np.float32(3.0)).astype(np.float32)
        np.fill_diagonal(H, 0)
    Pv, bits, _ = orc.build_P(tau, H, 1, 1.0, prec)
    return Pv, bits


@pytest.mark.parametrize("prec", [B.FP32, B.BF16, B.FP16])
@pytest.mark.parametrize("n,ties", [(40, False), (B.LIST_MAX, False), (B.LIST_MAX + 1, False), (900, False),
                                    (900, True), (2001, False)])
def test_list_invariants(orc, prec, n, ties):
    Pv, bits = _P(orc, n, 7 + n, prec, ties)
    ld = B.ld_of(n)
    lists, lcnt, lkey = _build(P_device(Pv, bits, prec, ld), prec, n, ld)
    L, C, K = host(lists), host(lcnt), host(lkey).view(np.uint32)
    keys = _keys(Pv, bits, prec)
    for i in range(n):
        row = keys[i]
        c = int(C[i])
        ent = L[i, :c]
        cols = ent[:, 1].astype(np.int64)
        vals = ent[:, 0].view(np.uint32).astype(np.int64)
        assert len(set(cols.tolist())) == c
        assert np.array_equal(ent[:, 0].view(np.uint32), row[cols])      # stored values
        pad = L[i, c:].view(np.uint32)                                   # slots past the count
        assert np.all(pad[:, 0] == 0) and np.all(pad[:, 1] == 0xFFFFFFFF)
        # sorted by value descending, ties by column ascending
        assert all((vals[q] > vals[q + 1]) or (vals[q] == vals[q + 1] and cols[q] < cols[q + 1])
                   for q in range(c - 1))
        if n <= LMAX:
            assert c == n and K[i] == 0
            continue
        T = np.sort(row)[-LTARGET]
        assert LTARGET <= c <= LMAX
        assert np.all(row[cols] >= T)
        assert set(np.nonzero(row > T)[0]) <= set(cols.tolist())
        out = np.setdiff1d(np.arange(n), cols)
        # bound on the score key (bits + 1) of unlisted columns
        assert np.all(row[out].astype(np.uint64) + 1 <= K[i])
        assert K[i] == (T if (row >= T).sum() <= LMAX else T + 1)


@pytest.mark.parametrize("prec", [B.FP32, B.BF16, B.FP16])
@pytest.mark.parametrize("n,m", [(5, 9), (60, 40), (333, 30), (1200, 24)])
def test_construct_with_lists_equals_full_scan_and_oracle(orc, prec, n, m):
    Pv, bits = _P(orc, n, 3 + n, prec)
    ld = B.ld_of(n)
    Pd = P_device(Pv, bits, prec, ld)
    lists, lcnt, lkey = _build(Pd, prec, n, ld)
    ref = orc.construct(Pv, 21, 5, 0, m)
    t_full = torch.zeros((m, n), dtype=torch.int32, device="cuda")
    t_list = torch.zeros((m, n), dtype=torch.int32, device="cuda")
    B.op_construct_ex(Pd, prec, n, ld, m, 21, 5, t_full)
    B.op_construct_ex(Pd, prec, n, ld, m, 21, 5, t_list, lists, lcnt, lkey)
    assert np.array_equal(host(t_full), ref)
    assert np.array_equal(host(t_list), ref)
    # the lean kernel: list steps with compact fallback scans, and compact scans only
    B.op_construct_ex(Pd, prec, n, ld, m, 21, 5, t_list, lists, lcnt, lkey, shape=(1, 0, 2))
    assert np.array_equal(host(t_list), ref)
    B.op_construct_ex(Pd, prec, n, ld, m, 21, 5, t_list, shape=(1, 0, 2))
    assert np.array_equal(host(t_list), ref)
    eb = 4 if prec == B.FP32 else 2
    for shp in shapes(eb):   # every single-warp shape with lists
        if shp[0] != 1 or not covers(shp, n, eb):
            continue
        B.op_construct_ex(Pd, prec, n, ld, m, 21, 5, t_list, lists, lcnt, lkey, shape=shp)
        assert np.array_equal(host(t_list), ref), shp


@pytest.mark.parametrize("prec", [B.FP32, B.BF16, B.FP16])
@pytest.mark.parametrize("n", [31, 32, 33, 40])
def test_lean_kernel_around_full_first_round(orc, prec, n):
    """n >= 32 selects the lean instantiation whose first list round has no
    padded slot (every list then holds >= 32 entries); both sides of the
    switch give the oracle's tours."""
    m = 37
    Pv, bits = _P(orc, n, 11 + n, prec)
    ld = B.ld_of(n)
    Pd = P_device(Pv, bits, prec, ld)
    lists, lcnt, lkey = _build(Pd, prec, n, ld)
    assert int(host(lcnt).min()) >= min(n, 32)
    ref = orc.construct(Pv, 9, 4, 0, m)
    t = torch.zeros((m, n), dtype=torch.int32, device="cuda")
    B.op_construct_ex(Pd, prec, n, ld, m, 9, 4, t, lists, lcnt, lkey, shape=(1, 0, 2))
    assert np.array_equal(host(t), ref)


def test_tie_heavy_rows_with_lists(orc):
    n, m = 300, 50
    Pv, bits = _P(orc, n, 1, B.FP32, ties=True)
    ld = B.ld_of(n)
    Pd = P_device(Pv, bits, B.FP32, ld)
    lists, lcnt, lkey = _build(Pd, B.FP32, n, ld)
    t = torch.zeros((m, n), dtype=torch.int32, device="cuda")
    ref = orc.construct(Pv, 3, 0, 0, m)
    B.op_construct_ex(Pd, B.FP32, n, ld, m, 3, 0, t, lists, lcnt, lkey)
    assert np.array_equal(host(t), ref)
    B.op_construct_ex(Pd, B.FP32, n, ld, m, 3, 0, t, shape=(1, 0, 2))
    assert np.array_equal(host(t), ref)


@pytest.mark.parametrize("lists", [True, False])
def test_solver_with_and_without_lists(orc, lists):
    xy = instances.clustered(10, 30, 0.02, seed=2)
    kw = dict(m=40, rho=0.1, seed=3)
    g = B.Solver(xy, cand_lists=lists, stream=torch.cuda.Stream(), **kw).iterate(15)
    ref = orc.State(xy, **kw).run(15)
    assert np.array_equal(g.tours(), ref.last_tours)
    assert np.array_equal(g.tau(), ref.tau)


def _fused_case(orc, n, seed, ties):
    xy = instances.clustered(-(-n // 40), 40, 0.02, seed=seed)[:n] if n >= 80 else instances.uniform(n, seed)
    H = orc.heuristic(orc.distances(xy), 2)
    tau = np.random.default_rng(seed).uniform(0.3, 2.0, size=(n, n)).astype(np.float32)
    if ties:
        tau[:] = 1.0
        H = np.where(H > np.median(H), np.float32(7.0), np.float32(3.0)).astype(np.float32)
        np.fill_diagonal(H, 0)
    return tau, H


@pytest.mark.parametrize("prec", [B.FP32, B.BF16, B.FP16])
@pytest.mark.parametrize("n,ties", [(40, False), (B.LIST_MAX, False), (B.LIST_MAX + 1, False), (900, True),
                                    (2001, False), (5000, False)])
def test_fused_build_equals_two_passes(orc, prec, n, ties):
    """aco_op_build_P_lists (M_p and lists in one pass, the threshold guessed
    from lkey) gives the M_p, lists, counts and bounds of aco_op_build_P +
    aco_op_build_lists whatever lkey holds: the previous bounds (the fast
    path), none, garbage, far too high or far too low (the fallback)."""
    tau, H = _fused_case(orc, n, 11 + n, ties)
    ld = B.ld_of(n)
    taud, Hd = padded_dev(tau, ld, np.float32), padded_dev(H, ld, np.float32)
    esz = torch.float32 if prec == B.FP32 else torch.int16
    P2 = torch.zeros((n, ld), dtype=esz, device="cuda")
    B.op_build_P(taud, Hd, n, ld, 1, 1.0, prec, P2)
    l2, c2, k2 = _build(P2, prec, n, ld)
    ref = (host(P2).view(np.uint8), host(l2), host(c2), host(k2))
    kb = host(k2).view(np.uint32)
    rng = np.random.default_rng(n)
    guesses = {"previous": kb.copy(), "none": np.zeros(n, np.uint32),
               "garbage": rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32),
               "high": np.full(n, 0x7F000000, np.uint32), "low": np.full(n, 0x00800000, np.uint32)}
    for name, g in guesses.items():
        P1 = torch.zeros((n, ld), dtype=esz, device="cuda")
        l1 = torch.zeros((n, LMAX, 2), dtype=torch.int32, device="cuda")
        c1 = torch.zeros(n, dtype=torch.int32, device="cuda")
        k1 = dev(g.view(np.int32))
        B.op_build_P_lists(taud, Hd, n, ld, 1, 1.0, 0.0, prec, P1, l1, c1, k1)
        got = (host(P1).view(np.uint8), host(l1), host(c1), host(k1))
        for a, b, what in zip(got, ref, ("M_p", "lists", "counts", "bounds")):
            assert np.array_equal(a, b), (name, what)
    if n >= 2000 and not ties:
        # the previous bounds scaled by 0.95 put a few hundred columns above the
        # threshold in most rows: the one-pass path is the one exercised
        keys = host(P2).view(np.uint32) if prec == B.FP32 else None
        if keys is not None:
            g95 = (kb.view(np.float32) * np.float32(0.95)).view(np.uint32)
            cnt = (keys[:, :n] >= g95[:, None]).sum(axis=1)
            assert np.mean((cnt > 260) & (cnt < 500)) > 0.3
