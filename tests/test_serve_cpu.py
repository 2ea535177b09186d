"""Host-side logic of the serving loop (no GPU): FIFO admission under the
slot count and the HBM byte budget, rejection of requests larger than the
budget, continuous batching (new requests start while others run)."""
import numpy as np

from paper_1706_01613_gb300 import serve


class FakeArray:
    def __init__(self, nbytes):
        self.nbytes = nbytes


class FakeExecutor:
    """Completes a request `dur` simulated seconds after it was submitted."""

    def __init__(self, clock, dur):
        self.clock, self.dur = clock, dur
        self.running = {}
        self.log = []

    def start(self):
        pass

    def submit(self, slot, req):
        self.running[slot] = (req, self.clock.t + self.dur(req))
        self.log.append(("start", req.id, slot, self.clock.t, dict(self.running)))

    def poll(self, slot):
        return self.running[slot][1] <= self.clock.t

    def finish(self, slot, req):
        _, end = self.running.pop(slot)
        self.log.append(("end", req.id, slot, end))
        return end


class Clock:
    def __init__(self):
        self.t = 0.0

    def now(self):
        return self.t

    def tick(self):
        self.t += 0.001


def _reqs(sizes, arrivals):
    return [serve.Request(i, "soa", (FakeArray(s),), 1, a) for i, (s, a) in enumerate(zip(sizes, arrivals))]


def test_budget_and_slots_limit_concurrency():
    clk = Clock()
    ex = FakeExecutor(clk, lambda r: 0.05)
    reqs = _reqs([400, 400, 400, 400], [0.0, 0.0, 0.0, 0.0])
    sched = serve.run_stream(reqs, ex, slots=3, budget_bytes=1000, now=clk.now, idle=clk.tick)
    starts = [e for e in ex.log if e[0] == "start"]
    # 417 bytes each (400 + 17 outputs): only two fit in 1000 bytes at once
    assert max(len(e[4]) for e in starts) == 2
    assert not sched.rejected and all(r.done is not None for r in reqs)
    assert sched.in_use == 0 and len(sched.free_slots) == 3


def test_too_large_is_rejected_and_fifo_order_kept():
    clk = Clock()
    ex = FakeExecutor(clk, lambda r: 0.01)
    reqs = _reqs([100, 5000, 100, 100], [0.0, 0.001, 0.002, 0.003])
    sched = serve.run_stream(reqs, ex, slots=1, budget_bytes=1000, now=clk.now, idle=clk.tick)
    assert [r.id for r in sched.rejected] == [1]
    order = [e[1] for e in ex.log if e[0] == "start"]
    assert order == [0, 2, 3]


def test_continuous_batching_admits_while_running():
    """A short request arriving while a long one runs starts at once on a
    free slot and finishes first."""
    clk = Clock()
    ex = FakeExecutor(clk, lambda r: 1.0 if r.id == 0 else 0.01)
    reqs = _reqs([100, 100], [0.0, 0.1])
    serve.run_stream(reqs, ex, slots=2, budget_bytes=10_000, now=clk.now, idle=clk.tick)
    assert reqs[1].admitted < reqs[0].done and reqs[1].done < reqs[0].done
    s = serve.latency_summary(reqs)
    assert s["requests"] == 2 and s["p50_ms"] > 0


def test_latency_summary_percentiles():
    reqs = _reqs([1] * 100, [0.0] * 100)
    for i, r in enumerate(reqs):
        r.done = (i + 1) * 1e-3
    s = serve.latency_summary(reqs)
    assert abs(s["p50_ms"] - np.percentile(np.arange(1, 101), 50)) < 1e-9
    assert abs(s["p99_ms"] - np.percentile(np.arange(1, 101), 99)) < 1e-9


def test_slot_scratch_is_charged_to_the_budget():
    """The slots' fixed scratch (here 600 of 1000 bytes) comes off the budget
    first: a 417-byte request that would fit in the bare budget is refused,
    a 317-byte one runs."""
    clk = Clock()
    ex = FakeExecutor(clk, lambda r: 0.01)
    ex.fixed_bytes = 600
    reqs = _reqs([400, 300], [0.0, 0.0])
    sched = serve.run_stream(reqs, ex, slots=2, budget_bytes=1000, now=clk.now, idle=clk.tick)
    assert [r.id for r in sched.rejected] == [0]
    assert reqs[1].done is not None and reqs[0].done is None
    assert sched.budget == 400


def test_latency_by_size_decade():
    reqs = [serve.Request(i, "soa", (FakeArray(1),), n, 0.0)
            for i, n in enumerate([150, 900, 5_000, 50_000, 2_000_000, 9_999_999])]
    for k, r in enumerate(reqs):
        r.done = 1e-3 * (k + 1)
    s = serve.latency_summary(reqs)
    assert list(s["by_size"]) == ["1e2-1e3", "1e3-1e4", "1e4-1e5", "1e6-1e7"]
    assert s["by_size"]["1e2-1e3"]["requests"] == 2
    assert abs(s["by_size"]["1e6-1e7"]["p50_ms"] - 5.5) < 1e-9


def test_pool_requests_are_cut_lazily():
    """SoA requests of a pool hold (planes, offset) and no host copy; their
    byte count is the device footprint of inputs and outputs."""
    import torch
    X = torch.arange(8 * 3 * 50, dtype=torch.float64).reshape(8, 3, 50)
    r = serve.Request(0, "soa", None, 7, 0.0, source=(X, 11))
    assert r.bytes == (192 + 17) * 7
    got = r.host_arrays()[0]
    assert got.is_contiguous() and torch.equal(got, X[:, :, 11:18])


def test_short_requests_pass_long_ones_on_their_slot():
    """With one of three slots kept for requests of at most 1000 elements, a
    short request arriving while two long ones run and a third waits starts
    at once on that slot; long requests never take it and keep FIFO order."""
    clk = Clock()
    ex = FakeExecutor(clk, lambda r: 1.0 if r.n > 1000 else 0.01)
    reqs = [serve.Request(i, "soa", (FakeArray(10),), n, a)
            for i, (n, a) in enumerate([(5000, 0.0), (5000, 0.0), (5000, 0.0), (50, 0.1),
                                        (5000, 0.2)])]
    serve.run_stream(reqs, ex, slots=3, budget_bytes=1 << 30, now=clk.now, idle=clk.tick,
                     small_slots=1, small_n=1000)
    starts = {e[1]: (e[2], e[3]) for e in ex.log if e[0] == "start"}
    assert starts[3][0] == 0 and starts[3][1] < 0.12  # the kept slot, at once
    assert all(starts[i][0] != 0 for i in (0, 1, 2, 4))
    order = [e[1] for e in ex.log if e[0] == "start"]
    assert order.index(2) < order.index(4)  # FIFO among the long ones
    assert reqs[3].done < reqs[0].done
