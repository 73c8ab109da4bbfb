"""Checkpoint / resume of a solver: a run interrupted, saved, restored into a
fresh solver and continued is bit-identical to the uninterrupted run (the
random numbers are counter-based on seed, iteration, ant and step);
corrupted or mismatched checkpoints are refused and leave the solver as it
was."""
import numpy as np
import pytest
import torch

from paper_2404_04895_gb300 import binding as B
from paper_2404_04895_gb300 import instances

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kw", [dict(m=60, rho=0.2, seed=3),
                                dict(m=48, rho=0.1, seed=5, roulette="adair", gamma_T=40, topk=6),
                                dict(m=40, rho=0.3, seed=7, prec="bf16")])
def test_resume_is_bit_exact(kw):
    xy = instances.uniform(150, 61)
    st = torch.cuda.Stream()
    whole = B.Solver(xy, stream=st, **kw).iterate(40)
    first = B.Solver(xy, stream=st, **kw).iterate(20)
    blob = first.state()
    first.close()
    second = B.Solver(xy, stream=st, **kw).restore(blob)
    assert second.iteration == 20
    second.iterate(20)
    assert np.array_equal(second.tau().view(np.uint32), whole.tau().view(np.uint32))
    assert np.array_equal(second.tours(), whole.tours())
    t1, l1 = second.best()
    t2, l2 = whole.best()
    assert l1 == l2 and np.array_equal(t1, t2)


def test_bad_checkpoints_are_refused():
    xy = instances.uniform(80, 62)
    kw = dict(m=30, rho=0.2, seed=9)
    s = B.Solver(xy, stream=torch.cuda.Stream(), **kw).iterate(5)
    blob = bytearray(s.state())
    tau_before = s.tau()
    t = B.Solver(xy, stream=torch.cuda.Stream(), **kw).iterate(3)
    tau_t = t.tau()
    corrupt = bytearray(blob)
    corrupt[len(corrupt) // 2] ^= 0x40                       # one flipped bit in tau
    with pytest.raises(B.AcoError):
        t.restore(bytes(corrupt))
    with pytest.raises(B.AcoError):
        t.restore(bytes(blob[:-9]))                          # truncated
    other = B.Solver(xy, stream=torch.cuda.Stream(), m=30, rho=0.25, seed=9)
    with pytest.raises(B.AcoError):
        other.restore(bytes(blob))                           # different rho
    wrong = bytearray(blob)
    wrong[0:8] = b"XXXXXXXX"
    with pytest.raises(B.AcoError):
        t.restore(bytes(wrong))
    assert t.iteration == 3 and np.array_equal(t.tau(), tau_t)   # unchanged
    t.restore(bytes(blob))
    assert t.iteration == 5 and np.array_equal(t.tau(), tau_before)
