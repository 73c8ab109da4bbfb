"""bench.py's multi-rank plumbing on CPU: two gloo ranks, started the way
torchrun starts `bench.py --gpus 2` (RANK, WORLD_SIZE, LOCAL_RANK and
MASTER_* in the environment), meet at the barriers and agree on the max over
ranks of their timed regions; the whole-job value counts every rank's units
over that slowest time."""
import importlib.util
import json
import os
import socket
import subprocess
import sys

from conftest import ROOT

RANK_CODE = r"""
import importlib.util, json, os, sys
spec = importlib.util.spec_from_file_location("bench", os.path.join(sys.argv[1], "bench.py"))
bench = importlib.util.module_from_spec(spec)
spec.loader.exec_module(bench)

class Args:
    impl = "reference"          # the gloo backend (the native arm takes NCCL)

d = bench.Dist(Args())
try:
    d.barrier()
    t_max = d.max(10.0 + 3.0 * d.rank)   # rank r timed 10 + 3r ms
    d.barrier()
    print(json.dumps({"rank": d.rank, "world": d.world, "t_max": t_max}))
finally:
    d.close()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_agree_on_the_slowest_time():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_CODE, ROOT], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=180) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    res = sorted((json.loads(o.strip().splitlines()[-1]) for o, _ in outs), key=lambda x: x["rank"])
    assert res == [{"rank": 0, "world": 2, "t_max": 13.0}, {"rank": 1, "world": 2, "t_max": 13.0}]


def test_whole_job_value_counts_every_rank_over_the_slowest():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    # 2 ranks, 4 steps of 1000 units each, the slowest rank took 13 ms in all
    assert bench.whole_job_value(1000, 2, 13.0, 4) == 2 * 4 * 1000 / 13.0e-3
    assert bench.whole_job_value(1000, 1, 13.0, 4) == 4 * 1000 / 13.0e-3


def test_reference_arm_under_two_ranks_prints_once():
    """`bench.py --impl reference --gpus 2` as torchrun starts it: rank 0
    alone runs the oracle and prints the line; rank 1 exits 0 without work."""
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                                       "--gpus", "2", "--steps", "1", "--warmup", "1", "--workload", "n50_ir"],
                                      env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    lines0 = [x for x in outs[0][0].splitlines() if x.strip()]
    assert len(lines0) == 1 and json.loads(lines0[0])["n_gpus"] == 2
    assert outs[1][0].strip() == ""
