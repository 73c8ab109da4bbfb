"""Failure detection on the GPU without a fault.  The roulette-wheel kernel
(Sec. 2.4) waits for each step's row copy with a bounded number of polls; a
bound of 0 makes every wait run out while the copy still lands.  The host
then gets ACO_ERR_TIMEOUT once, the CUDA context and the solver stay usable,
and a checkpoint taken before the failure restores a run that continues bit
for bit like one that never failed."""
import numpy as np
import pytest
import torch

from paper_2404_04895_gb300 import binding as B
from paper_2404_04895_gb300 import instances

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("graph", [True, False])
def test_wait_that_runs_out_reports_timeout_and_the_solver_recovers(graph):
    xy = instances.uniform(120, 71)
    kw = dict(m=24, rho=0.2, seed=11, roulette="rw")
    st = torch.cuda.Stream() if graph else None   # None: the legacy stream, launches without a graph
    whole = B.Solver(xy, stream=st, **kw).iterate(10)
    t_ref, l_ref = whole.best()
    s = B.Solver(xy, stream=st, **kw).iterate(5)
    blob = s.state()
    s.set_wait_polls(0).iterate(1)
    with pytest.raises(B.AcoError) as e:
        s.best()
    assert e.value.code == B.ERR_TIMEOUT and "wait ran out" in str(e.value)
    # reported once: the error word was cleared when it was read
    s.set_wait_polls().restore(blob)
    assert s.iteration == 5
    s.iterate(5)
    t1, l1 = s.best()
    assert l1 == l_ref and np.array_equal(t1, t_ref)
    assert np.array_equal(s.tau().view(np.uint32), whole.tau().view(np.uint32))
    assert np.array_equal(s.tours(), whole.tours())
    assert torch.ones(4, device="cuda").sum().item() == 4   # the context still runs work
