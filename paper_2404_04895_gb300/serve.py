"""Continuous-batching solve server over the batch C API.

Requests (TSP instances with an iteration budget) arrive over time.  The loop
admits arrived requests in arrival order as soon as a batch slot and arena
memory for their workspace are free (memory-gated admission; the head of the
queue waits rather than being overtaken), advances every admitted instance by
one iteration per batched step -- requests that arrived while others were on
the GPU join the next step, so their work overlaps on the device -- and
retires finished requests between steps, reading their best tour and freeing
their slot and memory.  Each instance's state (tau, M_p, tours, best) stays
resident on the device from admission to retirement.

  python -m paper_2404_04895_gb300.serve --requests 200 --rate 50

prints one JSON line: p50/p99 latency, throughput, offered and served load.
"""
import argparse
import dataclasses
import json
import sys
import time

import numpy as np

from . import instances
from .binding import ERR_ARG, ERR_UNSUPPORTED

# library status codes that describe the request itself: such a request is
# rejected, the others keep being served
REQUEST_ERRORS = (ERR_ARG, ERR_UNSUPPORTED)


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds from the start of the trace
    coords: np.ndarray      # n x 2 fp32
    m: int
    seed: int
    iters: int
    params: dict = dataclasses.field(default_factory=dict)
    cancel_at: float = None  # seconds from the start of the trace; None: never
    cancelled: bool = False
    rejected: str = None     # why the solver library refused the request (invalid or unsupported)
    admitted: float = None
    finished: float = None
    best_len: float = None
    tour: np.ndarray = None

    @property
    def n(self):
        return self.coords.shape[0]

    @property
    def ant_steps(self):
        return self.iters * self.m * (self.n - 1)

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival


def poisson_requests(count, rate, nmin, nmax, iters, mmax=1024, seed=11, **params):
    """Arrivals of a Poisson process at `rate` per second, sizes log-uniform."""
    t, sizes = instances.poisson_trace(count, rate, nmin, nmax, seed=seed)
    reqs = []
    for i, (ti, n) in enumerate(zip(t, sizes)):
        n = int(n)
        reqs.append(Request(rid=i, arrival=float(ti), coords=instances.uniform(n, 10_000 + i),
                            m=min(n, mmax), seed=i, iters=iters, params=dict(params)))
    return reqs


class Server:
    """Admission, batched stepping and retirement around one batch.

    batch: an object with add(coords, m, iters, **kw) -> slot or None,
    step(k), status(slot) -> (iterations, finished), best(slot), remove(slot),
    sync() -- paper_2404_04895_gb300.binding.Batch plus a stream sync.
    """

    def __init__(self, batch, clock=time.perf_counter, sleep=time.sleep):
        self.batch = batch
        self.clock = clock
        self.sleep = sleep

    def run(self, requests, realtime=True):
        """Serve `requests`; returns (finished requests, wall seconds, batched
        steps).  A request whose cancel_at has passed is dropped from the
        queue, or, once admitted, removed between steps (its slot and memory
        freed, no result); it is marked cancelled and not returned.  A
        request the library refuses (invalid or unsupported parameters or
        size) is marked rejected with the reason and not returned."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        active = {}
        done = []
        t0 = self.clock()
        steps = 0
        while pending or active:
            now = self.clock() - t0
            # cancellations: queued requests leave the queue, admitted ones their slot
            for r in [r for r in pending if r.cancel_at is not None and r.cancel_at <= now]:
                r.cancelled = True
                pending.remove(r)
            for s in [s for s, r in active.items() if r.cancel_at is not None and r.cancel_at <= now]:
                active.pop(s).cancelled = True
                self.batch.remove(s)
            # admit arrived requests in order while they fit
            while pending and (pending[0].arrival <= now or not realtime):
                r = pending[0]
                try:
                    slot = self.batch.add(r.coords, r.m, iters=r.iters, seed=r.seed, **r.params)
                except RuntimeError as e:
                    if getattr(e, "code", None) not in REQUEST_ERRORS:
                        raise
                    r.rejected = str(e)
                    pending.pop(0)
                    continue
                if slot is None:
                    break
                pending.pop(0)
                r.admitted = self.clock() - t0
                active[slot] = r
            if not active:
                if pending:
                    head = pending[0]
                    if not realtime or head.arrival <= now:  # it was offered to an empty batch
                        raise RuntimeError(f"request {head.rid} (n={head.n}) does not fit an empty batch")
                    self.sleep(max(0.0, head.arrival - (self.clock() - t0)))
                continue
            self.batch.step(1)
            steps += 1
            finished = [s for s in active if self.batch.status(s)[1]]
            if finished:
                self.batch.sync()
                t = self.clock() - t0
                for s in finished:
                    r = active.pop(s)
                    r.tour, r.best_len = self.batch.best(s)
                    r.finished = t
                    self.batch.remove(s)
                    done.append(r)
        wall = self.clock() - t0
        return done, wall, steps


def summarize(done, wall):
    if not done:  # every request was cancelled
        return {"requests": 0, "latency_p50_s": None, "latency_p99_s": None, "latency_mean_s": None,
                "throughput_req_per_s": 0.0, "ant_steps_per_s": 0.0, "offered_req_per_s": float("nan"),
                "offered_ant_steps_per_s": float("nan"), "offered_over_served": float("nan"), "wall_s": wall}
    lat = np.array([r.latency for r in done])
    ant_steps = float(sum(r.ant_steps for r in done))
    span = max(r.arrival for r in done) - min(r.arrival for r in done) if len(done) > 1 else 0.0
    offered_rate = (len(done) - 1) / span if span > 0 else float("nan")
    return {
        "requests": len(done),
        "latency_p50_s": float(np.percentile(lat, 50)),
        "latency_p99_s": float(np.percentile(lat, 99)),
        "latency_mean_s": float(lat.mean()),
        "throughput_req_per_s": len(done) / wall,
        "ant_steps_per_s": ant_steps / wall,
        "offered_req_per_s": offered_rate,
        "offered_ant_steps_per_s": ant_steps / span if span > 0 else float("nan"),
        "offered_over_served": (ant_steps / span) / (ant_steps / wall) if span > 0 else float("nan"),
        "wall_s": wall,
    }


class GpuBatch:
    """binding.Batch on its own stream of one device (default: the current
    one), with the sync the server needs; every call runs with that device
    current."""

    def __init__(self, arena_bytes, max_slots, prec, device=None):
        import torch

        from . import binding
        binding.lib()
        self.torch = torch
        self.device = torch.cuda.current_device() if device is None else device
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.Stream()
            self.b = binding.Batch(max_slots, arena_bytes, prec=prec, stream=self.stream)

    def _on(self):
        return self.torch.cuda.device(self.device)

    def add(self, coords, m, iters, **kw):
        with self._on():
            return self.b.add(coords, m, iters=iters, **kw)

    def step(self, k):
        with self._on():
            self.b.step(k)

    def status(self, slot):
        with self._on():
            return self.b.status(slot)

    def best(self, slot):
        with self._on():
            return self.b.best(slot)

    def remove(self, slot):
        with self._on():
            self.b.remove(slot)

    def free_bytes(self):
        with self._on():
            return self.b.info()["free_bytes"]

    def sync(self):
        self.stream.synchronize()

    def close(self):
        with self._on():
            self.b.close()


class DeviceBatches:
    """Independent instances spread over several GPUs of one process: one
    batch per device, and an arriving instance goes to the device whose arena
    has the most free memory (the next ones in that order when it does not
    fit).  Each device steps only its own instances, on its own stream, so
    the devices run concurrently and nothing crosses between them -- no
    collective on the data path.  A slot is (device index, the batch's slot).

    batches: objects as Server expects (add, step, status, best, remove,
    sync) that also report free_bytes()."""

    def __init__(self, batches):
        self.batches = list(batches)
        self.active = [0] * len(self.batches)

    def add(self, coords, m, iters, **kw):
        order = sorted(range(len(self.batches)), key=lambda d: (-self.batches[d].free_bytes(), d))
        for d in order:
            slot = self.batches[d].add(coords, m, iters, **kw)
            if slot is not None:
                self.active[d] += 1
                return (d, slot)
        return None

    def step(self, k):
        for d, b in enumerate(self.batches):  # asynchronous launches: the devices overlap
            if self.active[d]:
                b.step(k)

    def status(self, slot):
        return self.batches[slot[0]].status(slot[1])

    def best(self, slot):
        return self.batches[slot[0]].best(slot[1])

    def remove(self, slot):
        self.batches[slot[0]].remove(slot[1])
        self.active[slot[0]] -= 1

    def sync(self):
        for b in self.batches:
            b.sync()

    def close(self):
        for b in self.batches:
            if hasattr(b, "close"):
                b.close()


def place_requests(requests, world, need):
    """Requests for one process per GPU: in arrival order, each goes to the
    rank with the fewest workspace bytes placed so far (need(r): its bytes;
    ties to the lower rank).  Deterministic, so every rank computes the same
    split from the same trace without communicating."""
    load = [0] * world
    out = [[] for _ in range(world)]
    for r in sorted(requests, key=lambda r: (r.arrival, r.rid)):
        d = min(range(world), key=lambda q: (load[q], q))
        out[d].append(r)
        load[d] += need(r)
    return out


def serve_ranks(requests, batch, rank, world, need, gather=None, **run_kw):
    """Serve this rank's share of `requests` (place_requests) on `batch`;
    gather(obj) -> list of every rank's obj on rank 0 (None elsewhere), e.g.
    torch.distributed.gather_object.  Rank 0 returns every request's
    (rid, tour, best_len, latency) in rid order and the slowest rank's wall
    time; the other ranks return None."""
    mine = place_requests(requests, world, need)[rank]
    done, wall, steps = Server(batch).run(mine, **run_kw)
    part = {"rank": rank, "wall": wall, "steps": steps,
            "results": [(r.rid, r.tour, r.best_len, r.latency) for r in done]}
    parts = gather(part) if gather else [part]
    if parts is None:
        return None
    results = sorted((x for p in parts for x in p["results"]), key=lambda x: x[0])
    return {"results": results, "wall": max(p["wall"] for p in parts),
            "steps": [p["steps"] for p in sorted(parts, key=lambda p: p["rank"])]}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--nmin", type=int, default=50)
    ap.add_argument("--nmax", type=int, default=10000)
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--prec", default="bf16")
    ap.add_argument("--arena-gb", type=float, default=80.0)
    ap.add_argument("--slots", type=int, default=1024)
    ap.add_argument("--rho", type=float, default=0.1)
    ap.add_argument("--gpus", type=int, default=1, help="devices of this process, one batch each")
    args = ap.parse_args(argv)
    reqs = poisson_requests(args.requests, args.rate, args.nmin, args.nmax, args.iters, rho=args.rho)
    arena = int(args.arena_gb * (1 << 30))
    if args.gpus > 1:
        gb = DeviceBatches([GpuBatch(arena, args.slots, args.prec, device=d) for d in range(args.gpus)])
    else:
        gb = GpuBatch(arena, args.slots, args.prec)
    done, wall, steps = Server(gb).run(reqs, realtime=True)
    gb.close()
    out = summarize(done, wall)
    out.update({"config": {"requests": args.requests, "rate": args.rate, "n": [args.nmin, args.nmax],
                           "m": "min(n, 1024)", "iters": args.iters, "P_dtype": args.prec,
                           "arena_gb": args.arena_gb, "gpus": args.gpus}, "batched_steps": steps,
                "rejected": sum(1 for r in reqs if r.rejected)})
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
