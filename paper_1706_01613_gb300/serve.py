"""Continuous-batching validation server on one GPU.

Requests (meshes of very different sizes) arrive over time.  The server keeps
a fixed set of slots; each slot owns one library handle (its refinement
queue and exact-tier scratch stay on the device) and one CUDA stream.  A
request is admitted as soon as a slot is free and its device footprint
(inputs + outputs) fits in the HBM budget next to the requests already in
flight; the slots' own scratch (refinement queues, exact-tier stacks, node
records: fixed when the handles are created) is charged to the budget
first.  Admitted requests overlap on the device (copy in, bulk pass, tail,
copy out, all on the slot's stream).  Admission is first come, first served;
a request larger than what the budget leaves next to the slots' scratch is
rejected.

Latency = GPU completion time (an event on the slot's stream, read against
an event recorded when the run started) minus the arrival time.

The scheduling logic (`Scheduler`) is plain host code and is tested on the
CPU with a fake executor; `GpuExecutor` runs the work through the C ABI.
"""
import collections
import gc
import heapq
import math
import time

import numpy as np


class Request:
    __slots__ = ("id", "kind", "arrays", "source", "n", "arrival", "bytes", "result", "done",
                 "admitted")

    def __init__(self, rid, kind, arrays, n, arrival, source=None):
        self.id = rid
        self.kind = kind          # "soa": (corners,), "indexed": (nodes, conn)
        self.arrays = arrays      # host arrays (pinned torch tensors for the GPU executor)
        # or, for SoA requests cut from a pool, (pool planes (8, 3, N), offset):
        # the executor copies the n columns of each plane straight to the
        # device, so no per-request host copy is made
        self.source = source
        self.n = int(n)           # elements
        self.arrival = float(arrival)
        if arrays is not None:
            in_bytes = sum(int(a.numel() * a.element_size()) if hasattr(a, "numel")
                           else int(a.nbytes) for a in arrays)
        else:
            in_bytes = 192 * self.n
        self.bytes = in_bytes + 17 * self.n  # + flags, bmin, bmax
        self.result = None
        self.done = None
        self.admitted = None

    def host_arrays(self):
        """The request's inputs as contiguous host arrays."""
        if self.arrays is not None:
            return self.arrays
        X, off = self.source
        return (X[:, :, off:off + self.n].contiguous(),)


class Scheduler:
    """FIFO admission under a slot count and a byte budget.  The first
    `small_slots` slots take only requests of at most `small_n` elements, so
    that a short request arriving while long ones hold the other slots
    starts at once instead of waiting behind them (it may pass requests that
    wait for a general slot; among those the order stays FIFO)."""

    def __init__(self, slots, budget_bytes, reserved_bytes=0, small_slots=0, small_n=0):
        self.small = set(range(min(small_slots, max(0, slots - 1))))  # a general slot is kept
        self.small_n = int(small_n)
        self.free_slots = list(range(slots))
        self.budget = int(budget_bytes) - int(reserved_bytes)  # left for requests
        self.in_use = 0
        self.pending = collections.deque()
        self.rejected = []

    def arrive(self, req):
        if req.bytes > self.budget:
            self.rejected.append(req)
        else:
            self.pending.append(req)

    def _take(self, small_ok):
        for i, s in enumerate(self.free_slots):
            if s not in self.small:
                return self.free_slots.pop(i)
        if small_ok:
            for i, s in enumerate(self.free_slots):
                if s in self.small:
                    return self.free_slots.pop(i)
        return None

    def admissible(self):
        """Pops and returns (slot, request) pairs that can start now."""
        out = []
        kept = collections.deque()
        general_blocked = False  # an earlier request waits for a general slot
        while self.pending:
            req = self.pending.popleft()
            small_ok = bool(self.small) and req.n <= self.small_n
            slot = None
            if self.in_use + req.bytes <= self.budget:
                if not general_blocked:
                    slot = self._take(small_ok)
                elif small_ok:
                    slot = self._take_small()
            if slot is None:
                kept.append(req)
                general_blocked = True
                if not self.small:
                    break  # plain FIFO: nothing behind the head may start
                continue
            self.in_use += req.bytes
            out.append((slot, req))
        kept.extend(self.pending)
        self.pending = kept
        return out

    def _take_small(self):
        for i, s in enumerate(self.free_slots):
            if s in self.small:
                return self.free_slots.pop(i)
        return None

    def release(self, slot, req):
        self.in_use -= req.bytes
        self.free_slots.append(slot)


def run_stream(requests, executor, slots, budget_bytes, now=time.perf_counter, idle=None,
               small_slots=0, small_n=0):
    """Serves `requests` (sorted by arrival, times in seconds from the start)
    on `executor`; returns the scheduler (for the rejected list).  The
    executor's fixed device memory (`fixed_bytes`, the slots' scratch) is
    charged to the budget before any request; `small_slots` slots are kept
    for requests of at most `small_n` elements."""
    sched = Scheduler(slots, budget_bytes, getattr(executor, "fixed_bytes", 0), small_slots,
                      small_n)
    order = sorted(requests, key=lambda r: r.arrival)
    # the loop's latency is the requests' latency: no pauses of the cyclic
    # garbage collector while it runs (reference counting still frees)
    gc_was_enabled = gc.isenabled()
    gc.disable()
    try:
        t0 = now()
        executor.start()
        nxt = 0
        inflight = {}
        while nxt < len(order) or sched.pending or inflight:
            t = now() - t0
            while nxt < len(order) and order[nxt].arrival <= t:
                sched.arrive(order[nxt])
                nxt += 1
            for slot, req in sched.admissible():
                req.admitted = t
                executor.submit(slot, req)
                inflight[slot] = req
            for slot in list(inflight):
                if executor.poll(slot):
                    req = inflight.pop(slot)
                    req.done = executor.finish(slot, req)
                    sched.release(slot, req)
            if idle is not None:
                idle()
    finally:
        if gc_was_enabled:
            gc.enable()
    return sched


def latency_summary(requests):
    """p50 / p99 / max latency over the completed requests, throughput over
    the span from the first arrival to the last completion, and p50 / p99
    per size decade ([10^k, 10^(k+1)) elements)."""
    done = [r for r in requests if r.done is not None]
    lat = np.array([r.done - r.arrival for r in done])
    hexes = sum(r.n for r in done)
    if not len(lat):
        return {}
    span = max(r.done for r in done) - min(r.arrival for r in requests)
    by_size = {}
    dec = np.array([int(math.floor(math.log10(max(1, r.n)))) for r in done])
    for k in sorted(set(dec.tolist())):
        sel = lat[dec == k]
        by_size["1e%d-1e%d" % (k, k + 1)] = {
            "requests": int(len(sel)), "p50_ms": float(np.percentile(sel, 50) * 1e3),
            "p99_ms": float(np.percentile(sel, 99) * 1e3)}
    return {"requests": int(len(lat)), "hexes": int(hexes),
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "max_ms": float(lat.max() * 1e3),
            "hex_per_s": float(hexes / span) if span > 0 else None,
            "by_size": by_size}


class GpuExecutor:
    """Runs requests through the library, one handle and stream per slot."""

    def __init__(self, slots, precision="fp32", max_depth=8, keep_results=True, **caps):
        import torch
        from . import hexval as hv
        self.torch = torch
        # False: a finished request drops its outputs once they are on the
        # host (a long stream's outputs would otherwise pile up in memory)
        self.keep_results = keep_results
        self.hv = hv
        self.v = [hv.Validator(precision=precision, max_depth=max_depth, **caps)
                  for _ in range(slots)]
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.fixed_bytes = sum(v.scratch_bytes() for v in self.v)
        self.events = [None] * slots
        self.buffers = [None] * slots
        # without kept results each slot copies its outputs into one pinned
        # host buffer of its own, grown to the largest request it has run,
        # instead of new pinned memory per request
        self.host_out = [None] * slots
        self.t0 = None

    def start(self):
        torch = self.torch
        torch.cuda.synchronize()
        self.t0 = torch.cuda.Event(enable_timing=True)
        self.t0.record()
        self.t0_host = time.perf_counter()
        torch.cuda.synchronize()

    def submit(self, slot, req):
        torch = self.torch
        s = self.streams[slot]
        with torch.cuda.stream(s):
            if req.kind == "soa" and req.source is not None:
                X, off = req.source
                d = torch.empty((8, 3, req.n), dtype=X.dtype, device="cuda")
                self.hv.copy_soa_range(d, X, off, stream=s)  # one strided copy
                dev = (d,)
            elif req.kind == "soa":
                X = req.arrays[0]
                dev = (X.to("cuda", non_blocking=True),)
            else:
                dev = tuple(a.to("cuda", non_blocking=True) for a in req.arrays)
            out = (torch.empty(req.n, dtype=torch.uint8, device="cuda"),
                   torch.empty(req.n, dtype=torch.float64, device="cuda"),
                   torch.empty(req.n, dtype=torch.float64, device="cuda"))
            if req.kind == "soa":
                self.v[slot].check_soa(dev[0], out=out, stream=s)
            else:
                self.v[slot].check_indexed(dev[0], dev[1], out=out, stream=s)
            host = self._host_outputs(slot, req.n)
            for h, d in zip(host, out):
                h.copy_(d, non_blocking=True)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(s)
        self.events[slot] = ev
        self.buffers[slot] = (dev, out, host)

    def _host_outputs(self, slot, n):
        torch = self.torch
        if self.keep_results:
            return (torch.empty(n, dtype=torch.uint8, pin_memory=True),
                    torch.empty(n, dtype=torch.float64, pin_memory=True),
                    torch.empty(n, dtype=torch.float64, pin_memory=True))
        buf = self.host_out[slot]
        if buf is None or buf[0].shape[0] < n:  # the slot's previous request is done
            buf = (torch.empty(n, dtype=torch.uint8, pin_memory=True),
                   torch.empty(n, dtype=torch.float64, pin_memory=True),
                   torch.empty(n, dtype=torch.float64, pin_memory=True))
            self.host_out[slot] = buf
        return tuple(t[:n] for t in buf)

    def poll(self, slot):
        return self.events[slot].query()

    def finish(self, slot, req):
        ev = self.events[slot]
        ev.synchronize()
        _, _, host = self.buffers[slot]
        req.result = tuple(h.numpy() for h in host) if self.keep_results else None
        self.buffers[slot] = None
        done = self.t0_host + self.t0.elapsed_time(ev) / 1e3
        return done - self.t0_host

    def status(self):
        return [v.status() for v in self.v]

    def close(self):
        for v in self.v:
            v.close()


# ------------------------------------------------------ request streams ----

class Pool:
    """Pinned host inputs that requests slice: SoA pools of independent
    elements (perturbed cubes, affine mixture) and one large structured grid
    whose first n hexes (and the nodes they use) form an indexed request."""

    def __init__(self, max_n, seed=20175000):
        import torch
        from . import synth
        self.torch = torch
        self.max_n = int(max_n)
        self.soa = {1: torch.from_numpy(synth.perturbed_cubes(self.max_n, seed=seed + 1)).pin_memory(),
                    3: torch.from_numpy(synth.affine_mixture(self.max_n, seed=seed + 3)[0]).pin_memory()}
        a = max(2, int(math.ceil(self.max_n ** (1.0 / 3.0))))
        nodes, conn = synth.structured_grid(a, a, a, seed=seed + 2)
        self.nodes = torch.from_numpy(nodes).pin_memory()
        self.conn = torch.from_numpy(conn).pin_memory()
        self.node_hi = np.maximum.accumulate(conn.max(axis=1))

    def request(self, rid, kind, n, arrival, offset=0):
        torch = self.torch
        n = int(min(n, self.max_n))
        if kind == 2:
            n = min(n, self.conn.shape[0])
            hi = int(self.node_hi[n - 1]) + 1
            return Request(rid, "indexed", (self.nodes[:hi], self.conn[:n]), n, arrival)
        off = int(offset) % max(1, self.max_n - n + 1)
        return Request(rid, "soa", None, n, arrival, source=(self.soa[kind], off))


def poisson_stream(pool, n_requests, rate, seed, size_min=100, size_max=10_000_000):
    """Requests with sizes log-uniform in [size_min, size_max] (capped by the
    pool), generator kinds 1-3 uniformly, Poisson arrivals at `rate`/s."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = np.exp(rng.uniform(math.log(size_min), math.log(size_max), n_requests))
    kinds = rng.integers(1, 4, n_requests)
    offs = rng.integers(0, 1 << 30, n_requests)
    return [pool.request(i, int(kinds[i]), int(sizes[i]), float(arrivals[i]), int(offs[i]))
            for i in range(n_requests)]
