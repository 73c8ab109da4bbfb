"""Host logic of the continuous-batching server, on a fake batch (no GPU):
arrival-ordered, memory-gated admission, joins between steps, retirement
frees memory, latency accounting."""
import numpy as np

from paper_2404_04895_gb300 import serve


class FakeBatch:
    def __init__(self, capacity):
        self.capacity, self.used, self.slots, self.next = capacity, 0, {}, 0
        self.log = []

    def add(self, coords, m, iters, **kw):
        need = coords.shape[0]
        if self.used + need > self.capacity:
            return None
        s = self.next
        self.next += 1
        self.slots[s] = [need, iters, 0]
        self.used += need
        self.log.append(("add", s))
        return s

    def step(self, k):
        for v in self.slots.values():
            if v[2] < v[1]:
                v[2] += k
        self.log.append(("step", sorted(s for s, v in self.slots.items() if v[2] <= v[1])))

    def status(self, s):
        v = self.slots[s]
        return v[2], v[2] >= v[1]

    def best(self, s):
        return np.zeros(self.slots[s][0], np.int32), float(s)

    def remove(self, s):
        self.used -= self.slots.pop(s)[0]

    def sync(self):
        pass


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, d):
        self.t += max(d, 1e-6)


def _req(i, arrival, n, iters):
    return serve.Request(rid=i, arrival=arrival, coords=np.zeros((n, 2), np.float32), m=4, seed=i, iters=iters)


def test_fifo_memory_gated_admission_and_joins():
    clock = FakeClock()
    fb = FakeBatch(capacity=100)
    srv = serve.Server(fb, clock=clock, sleep=clock.sleep)
    reqs = [_req(0, 0.0, 60, 3), _req(1, 0.0, 60, 2), _req(2, 0.0, 30, 2), _req(3, 5.0, 10, 1)]
    done, wall, steps = srv.run(reqs, realtime=True)
    assert sorted(r.rid for r in done) == [0, 1, 2, 3]
    adds = [e[1] for e in fb.log if e[0] == "add"]
    # request 1 (60) does not fit beside request 0 (60): it waits, and request 2
    # behind it is not admitted ahead of it (arrival order)
    first_step = fb.log.index(("step", [0]))
    assert fb.log[:first_step] == [("add", 0)]
    assert adds == [0, 1, 2, 3]
    by = {r.rid: r for r in done}
    assert by[1].admitted >= by[0].admitted and by[2].admitted >= by[1].admitted
    assert all(r.latency >= 0 and r.finished >= r.admitted >= r.arrival for r in done)
    assert fb.used == 0


def test_summary_reports_percentiles_and_load():
    rs = []
    for i in range(10):
        r = _req(i, float(i), 10, 5)
        r.admitted, r.finished = float(i), float(i) + 1 + i % 3
        rs.append(r)
    s = serve.summarize(rs, wall=12.0)
    assert s["requests"] == 10
    assert 1.0 <= s["latency_p50_s"] <= 3.0 and s["latency_p99_s"] <= 3.0
    assert abs(s["throughput_req_per_s"] - 10 / 12.0) < 1e-12
    assert s["offered_req_per_s"] == 1.0


def test_poisson_trace_shapes():
    reqs = serve.poisson_requests(50, 50.0, 50, 10000, 100)
    ns = np.array([r.n for r in reqs])
    assert ns.min() >= 50 and ns.max() <= 10000
    assert all(r.m == min(r.n, 1024) for r in reqs)
    gaps = np.diff([r.arrival for r in reqs])
    assert np.all(gaps >= 0) and 0.005 < gaps.mean() < 0.05


def test_cancellation_frees_slots_and_returns_no_result():
    clock = FakeClock()
    fb = FakeBatch(capacity=100)

    class TickingBatch(FakeBatch):
        def step(self, k):
            super().step(k)
            clock.t += 1.0          # one second per batched step

    fb = TickingBatch(capacity=100)
    reqs = [_req(0, 0.0, 60, 10), _req(1, 0.0, 60, 3), _req(2, 0.5, 30, 2)]
    reqs[0].cancel_at = 2.5         # admitted, cancelled mid-run
    reqs[2].cancel_at = 0.7         # cancelled while queued behind request 1
    done, wall, steps = serve.Server(fb, clock=clock, sleep=clock.sleep).run(reqs)
    assert [r.rid for r in done] == [1]
    assert reqs[0].cancelled and reqs[2].cancelled and not reqs[1].cancelled
    assert reqs[0].finished is None and reqs[0].tour is None
    assert fb.used == 0 and not fb.slots           # every slot and byte returned
    assert ("add", 2) not in fb.log and ("add", 3) not in fb.log


def test_request_too_large_for_an_empty_batch_is_an_error():
    """A request that does not fit even an empty batch stops the server with
    an error, in real time as well (it would otherwise be offered forever)."""
    import pytest
    for realtime in (True, False):
        clock = FakeClock()
        srv = serve.Server(FakeBatch(capacity=50), clock=clock, sleep=clock.sleep)
        with pytest.raises(RuntimeError, match="does not fit an empty batch"):
            srv.run([_req(0, 0.0, 20, 1), _req(1, 0.5, 80, 1)], realtime=realtime)


def test_all_cancelled_run_summarizes_to_zero_served():
    clock = FakeClock()
    srv = serve.Server(FakeBatch(capacity=100), clock=clock, sleep=clock.sleep)
    reqs = [_req(0, 0.0, 20, 3), _req(1, 0.0, 20, 3)]
    for r in reqs:
        r.cancel_at = 0.0
    done, wall, steps = srv.run(reqs, realtime=True)
    assert done == [] and all(r.cancelled for r in reqs)
    s = serve.summarize(done, wall)
    assert s["requests"] == 0 and s["latency_p50_s"] is None and s["throughput_req_per_s"] == 0.0


class RefusingBatch(FakeBatch):
    """Refuses requests above `limit` cities the way the library does."""

    def __init__(self, capacity, limit, code):
        super().__init__(capacity)
        self.limit, self.code = limit, code

    def add(self, coords, m, iters, **kw):
        if coords.shape[0] > self.limit:
            from paper_2404_04895_gb300.binding import AcoError
            raise AcoError(self.code, "construction serves n <= %d" % self.limit)
        return super().add(coords, m, iters, **kw)


def test_refused_request_is_rejected_and_the_rest_served():
    from paper_2404_04895_gb300 import binding as B
    import pytest
    clock = FakeClock()
    srv = serve.Server(RefusingBatch(capacity=100, limit=40, code=B.ERR_UNSUPPORTED), clock=clock,
                       sleep=clock.sleep)
    reqs = [_req(0, 0.0, 20, 2), _req(1, 0.0, 50, 2), _req(2, 0.1, 30, 1)]
    done, wall, steps = srv.run(reqs, realtime=True)
    assert sorted(r.rid for r in done) == [0, 2]
    assert reqs[1].rejected and "n <= 40" in reqs[1].rejected and reqs[1].finished is None
    # a failure of the device, not of the request, still stops the server
    srv = serve.Server(RefusingBatch(capacity=100, limit=40, code=B.ERR_CUDA), clock=clock, sleep=clock.sleep)
    with pytest.raises(B.AcoError):
        srv.run([_req(0, 0.0, 50, 1)], realtime=False)


class SizedBatch(FakeBatch):
    """A fake batch that reports its free arena bytes (for DeviceBatches)."""

    def free_bytes(self):
        return self.capacity - self.used


def test_device_batches_place_by_free_memory_and_route():
    """Two devices: each request goes to the device with more free arena
    memory (ties to device 0), steps reach only devices with instances, and
    results, status and removal go to the device that holds the instance."""
    a, b = SizedBatch(capacity=100), SizedBatch(capacity=80)
    db = serve.DeviceBatches([a, b])
    s0 = db.add(np.zeros((50, 2), np.float32), 4, 2)
    s1 = db.add(np.zeros((40, 2), np.float32), 4, 2)    # a: 50 free, b: 80 free -> b
    s2 = db.add(np.zeros((45, 2), np.float32), 4, 1)    # a: 50, b: 40 -> a
    assert (s0[0], s1[0], s2[0]) == (0, 1, 0)
    assert db.add(np.zeros((60, 2), np.float32), 4, 1) is None   # fits nowhere now
    db.step(1)
    assert db.status(s2) == (1, True) and db.status(s0) == (1, False)
    db.remove(s2)
    db.remove(s1)
    assert db.active == [1, 0]
    db.step(1)                                            # device 1 is idle: not stepped
    assert b.log[-1] == ("add", 0) or b.log[-1][0] == "step"
    assert sum(1 for e in b.log if e[0] == "step") == 1 and db.status(s0) == (2, True)


def test_server_over_device_batches_serves_every_request_once():
    clock = FakeClock()
    db = serve.DeviceBatches([SizedBatch(capacity=100), SizedBatch(capacity=100)])
    reqs = [_req(i, 0.1 * i, 30 + 10 * (i % 4), 1 + i % 3) for i in range(12)]
    done, wall, steps = serve.Server(db, clock=clock, sleep=clock.sleep).run(reqs, realtime=False)
    assert sorted(r.rid for r in done) == list(range(12))
    assert all(x.used == 0 for x in db.batches)
    assert all(any(e[0] == "add" for e in x.log) for x in db.batches)   # both devices served


def test_place_requests_balances_bytes_deterministically():
    reqs = [_req(i, 0.01 * i, n, 1) for i, n in enumerate([100, 10, 10, 10, 50, 60, 5])]
    parts = serve.place_requests(reqs, 2, need=lambda r: r.n)
    assert [r.rid for r in parts[0]] == [0, 6] and [r.rid for r in parts[1]] == [1, 2, 3, 4, 5]
    assert serve.place_requests(reqs, 2, need=lambda r: r.n)[1] == parts[1]
    assert serve.place_requests(reqs, 1, need=lambda r: r.n)[0] == sorted(reqs, key=lambda r: r.arrival)
