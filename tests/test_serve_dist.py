"""Requests served by one process per GPU, the host side on CPU: two gloo
ranks started the way torchrun starts them place the same trace with the
same deterministic split, serve their shares with no communication, and
rank 0 gathers every result; the results equal a one-rank run's."""
import json
import os
import socket
import subprocess
import sys

from conftest import ROOT

CHILD = r"""
import json, os, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
from paper_2404_04895_gb300 import serve

class ResultBatch:
    # a batch whose result is a function of the instance alone, as on the GPU
    def __init__(self, capacity):
        self.capacity, self.used, self.slots, self.next = capacity, 0, {}, 0
    def add(self, coords, m, iters, **kw):
        need = coords.shape[0]
        if self.used + need > self.capacity:
            return None
        s = self.next; self.next += 1
        self.slots[s] = [coords, iters, 0]; self.used += need
        return s
    def step(self, k):
        for v in self.slots.values():
            v[2] = min(v[1], v[2] + k)
    def status(self, s):
        v = self.slots[s]
        return v[2], v[2] >= v[1]
    def best(self, s):
        c = self.slots[s][0]
        return np.argsort(c[:, 0], kind="stable").astype(np.int32), float(c.sum())
    def remove(self, s):
        self.used -= self.slots.pop(s)[0].shape[0]
    def sync(self):
        pass

def trace():
    rng = np.random.default_rng(4)
    return [serve.Request(rid=i, arrival=0.0, coords=rng.random((int(n), 2)).astype(np.float32), m=4, seed=i,
                          iters=int(1 + i % 4)) for i, n in enumerate(rng.integers(20, 90, size=14))]

dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
def gather(obj):
    out = [None] * world if rank == 0 else None
    dist.gather_object(obj, out, dst=0)
    return out
need = lambda r: r.n
res = serve.serve_ranks(trace(), ResultBatch(200), rank, world, need, gather=gather, realtime=False)
mine = [r.rid for r in serve.place_requests(trace(), world, need)[rank]]
if rank == 0:
    one = serve.serve_ranks(trace(), ResultBatch(200), 0, 1, need, realtime=False)
    same = [(a[0], a[1].tolist(), a[2]) for a in res["results"]] == [(a[0], a[1].tolist(), a[2]) for a in one["results"]]
    print(json.dumps({"rids": [r[0] for r in res["results"]], "same_as_one_rank": same, "mine": mine,
                      "steps": res["steps"]}))
else:
    assert res is None
    print(json.dumps({"mine": mine}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_split_serve_and_gather():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    r0 = json.loads(outs[0][0].strip().splitlines()[-1])
    r1 = json.loads(outs[1][0].strip().splitlines()[-1])
    assert r0["rids"] == list(range(14)) and r0["same_as_one_rank"]
    assert r0["mine"] and r1["mine"] and sorted(r0["mine"] + r1["mine"]) == list(range(14))
    assert len(r0["steps"]) == 2
