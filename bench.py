"""Benchmark of the GB300 linear-hexahedron validity test.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config 2|1|3|4|4b]

A step is one pass of the whole hot path (bulk pass, refinement, exact tier)
over one synthetic workload already resident in HBM.  The default workload
is the indexed structured mesh of 128^3 hexahedra (129^3 FP64 nodes, interior
nodes displaced by N(0, 0.15^2), int32 connectivity).  `value` is the
FP32-filtered form; the plain FP64 form is measured on the same input and
reported under "fp64".  Flags are exact (certified) in both forms.

Timing: W warm-up steps, then K steps, each bracketed by CUDA events on the
launch stream; L2 is flushed (256 MB write) between steps because the
workload (119 MB) fits in the 129 MB L2.  Multi-GPU (torchrun): every rank
validates its own mesh (weak scaling, no collective on the data path);
barrier + synchronize around the timed region and the max over ranks.

One JSON line is printed by rank 0.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "validated hexes/s on 1 GB300, FP32-filtered vs plain FP64 (exact flags); p50/p99 latency"
UNIT = "hex/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
PROFILE_EVERY = 10
# Roofline denominators of the arithmetic-bound kernels, from the profiling
# recipe's nominal figures for one GB300 (152 SMs, 2070 MHz): dense FP64 at
# 1.25 TFLOP/s is 0.625 T FP64 instructions/s (an FMA counts as 2 flops);
# FP32 at 128 lanes per SM is 40.3 T FP32 instructions/s.
FP64_PEAK = 1.25 / 2
FP32_PEAK = 152 * 128 * 2.07e9 / 1e12
# FP64 instructions of one hexahedron in the FP64 bulk pass, as ncu counts
# them (DADD 132, DFMA 107, DMUL 103 per element on the 128^3 mesh:
# profiles/bulk64_mesh128.txt), and of one box expansion (three unscaled de
# Casteljau passes over 9, 15 and 25 rows, 3 additions a row; the same count
# in FP32 for an FP32 box)
OPS_PER_HEX = 366
OPS_PER_BOX = 147


# ------------------------------------------------------------- workloads ----

def workload(cfg, rank, world=1, n=None):
    """Host arrays of one configuration.  With several ranks the headline
    mesh is one 128 x 128 x 128N mesh of which each rank takes its element
    range (a slab of 128^3 hexes with its nodes: weak scaling, no exchange);
    the other configurations are drawn per rank (rank-dependent seed).  n:
    a smaller case of the same SoA workload (its first n elements), for
    profiler captures that must stay small."""
    from paper_1706_01613_gb300 import shard, synth
    if cfg == 2:
        name = "structured mesh 128^3 hexes (129^3 FP64 nodes, sigma 0.15, int32 conn)"
        if world > 1:
            nodes, conn = synth.structured_grid(128, 128, 128 * world, seed=20170002)
            nodes, conn, _, _ = shard.shard_indexed(nodes, conn, rank, world)
            name = ("element range %d of %d of a 128 x 128 x %d structured mesh: 128^3 hexes, "
                    "%d FP64 nodes (sigma 0.15, int32 conn)" % (rank, world, 128 * world,
                                                               nodes.shape[0]))
        else:
            nodes, conn = synth.structured_grid(128, seed=20170002)
        return dict(kind="indexed", nodes=nodes, conn=conn, n=conn.shape[0], depth=8,
                    name=name, bytes_per_hex=32 + 17, n_nodes=nodes.shape[0])
    if cfg == 1:
        X = synth.perturbed_cubes(n or 10_000, seed=20170001 + 1000 * rank)
        return dict(kind="soa", X=X, n=X.shape[2], depth=8,
                    name="{:,} perturbed unit cubes (U[-0.3,0.3], SoA FP64)".format(X.shape[2]),
                    bytes_per_hex=192 + 17, n_nodes=0)
    if cfg == 3:
        X, _, _ = synth.affine_mixture(n or 16_777_216, seed=20170003 + 1000 * rank)
        return dict(kind="soa", X=X, n=X.shape[2], depth=8,
                    name="{:,} affine / near-degenerate / inverted hexes (SoA FP64)".format(
                        X.shape[2]),
                    bytes_per_hex=192 + 17, n_nodes=0)
    if cfg == 4:
        X = synth.twisted_layers(n or 4_194_304, seed=20170004 + 1000 * rank)
        return dict(kind="soa", X=X, n=X.shape[2], depth=10,
                    name="{:,} twisted boundary-layer hexes (SoA FP64, depth cap 10)".format(
                        X.shape[2]),
                    bytes_per_hex=192 + 17, n_nodes=0)
    if cfg == "4b":  # stress variant: twists up to 180 degrees, deep refinement
        X = synth.twisted_layers(n or 4_194_304, seed=20170004 + 1000 * rank,
                                 theta_max_deg=180.0)
        return dict(kind="soa", X=X, n=X.shape[2], depth=10,
                    name="{:,} boundary-layer hexes twisted by up to 180 degrees (SoA FP64, "
                         "depth cap 10)".format(X.shape[2]),
                    bytes_per_hex=192 + 17, n_nodes=0,
                    caps=dict(queue_capacity=min(1 << 25, 8 * X.shape[2])))  # ~2.6 live boxes
                                                                          # per element
    raise ValueError(cfg)


def algorithmic_bytes(w, kernel):
    """Bytes the method must move per launch (the per-element figures of the
    scope table): an element's connectivity (32 B) or its 24 FP64
    coordinates (192 B), its outputs (17 B: flag, bmin, bmax) and, for an
    indexed mesh, each FP64 node once (24 B).  nodes32 alone: 24 B read and
    16 B written per node."""
    if kernel == "nodes32":
        return 40 * w["n_nodes"]
    return w["bytes_per_hex"] * w["n"] + 24 * w["n_nodes"]


# ------------------------------------------------------------ clock probe ---

class ClockSampler:
    """nvidia-smi samples (SM clock, max clock, throttle reasons) while the
    timed region runs."""
    FIELDS = ("pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id):
        self.bus_id = (bus_id or "").lower()
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()

    def summary(self, t0, t1):
        rows = [r for t, r in self.rows if len(r) >= 9 and
                (not self.bus_id or self.bus_id.endswith(r[0].lower()[-12:]))]
        inside = [r for t, r in self.rows if t0 <= t <= t1 and len(r) >= 9]
        use = inside if inside else rows
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = sorted(float(r[1]) for r in use if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in use if r[2].replace(".", "").isdigit())
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in use:
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(use),
                "window": "timed region" if inside else "whole run (timed region shorter "
                                                        "than the 50 ms sampling period)"}


# ----------------------------------------------------------------- timing ---

def timed_steps(v, w, dev_in, steps, warmup, flush, profile=False):
    """Runs warm-up + timed steps of one Validator; returns per-step ms."""
    import torch
    out = (torch.empty(w["n"], dtype=torch.uint8, device=v.device),
           torch.empty(w["n"], dtype=torch.float64, device=v.device),
           torch.empty(w["n"], dtype=torch.float64, device=v.device))

    def step():
        if w["kind"] == "indexed":
            v.check_indexed(dev_in[0], dev_in[1], out=out)
        else:
            v.check_soa(dev_in[0], out=out)

    for _ in range(warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    v.raise_on_status()
    if profile:
        v.profile_read(reset=True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    wall0 = time.time()
    for i in range(steps):
        # per-kernel event timing on every PROFILE_EVERY-th step of the timed
        # region (the events add a few microseconds to the steps they are in)
        sampled = profile and i % PROFILE_EVERY == 0
        if sampled:
            v.profile(True)
        flush.zero_()
        starts[i].record()
        step()
        ends[i].record()
        if sampled:
            v.profile(False)
    torch.cuda.synchronize()
    wall1 = time.time()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    prof = v.profile_read(reset=True) if profile else None
    if profile:
        v.profile(False)
    v.raise_on_status()
    return ms, prof, (wall0, wall1), out


def e2e_steps(v, w, steps, warmup, chunks=4):
    """Public API on host data: pinned host inputs copied in and all three
    outputs (flags, bmin, bmax) copied out every step, the copies of each
    chunk of elements overlapping the checks of the others, the sequence
    replayed from a CUDA graph (HostPipeline)."""
    import torch
    if w["kind"] == "indexed":
        host = (torch.from_numpy(w["nodes"]).pin_memory(), torch.from_numpy(w["conn"]).pin_memory())
    else:
        host = (torch.from_numpy(w["X"]).pin_memory(),)
    h2d = sum(t.numel() * t.element_size() for t in host)
    d2h = 17 * w["n"]
    pipe = v.host_pipeline(w["kind"], *host, chunks=chunks)
    for _ in range(warmup):
        pipe.run()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(steps):
        res = pipe.run()
    t1.record()
    torch.cuda.synchronize()
    v.raise_on_status()
    ms = t0.elapsed_time(t1) / steps
    return ms, h2d, d2h, res


def traffic_for(kernel):
    """DRAM bytes per launch from the committed ncu capture, if the kernel
    source has not changed since it was taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    if source_sha(rec["source"]) != rec.get("source_sha"):
        return None
    return rec["dram_bytes_per_launch"]


def source_sha(source):
    """Hash of a kernel's source file and every header of the CUDA sources
    (any of which it may include)."""
    csrc = os.path.join(ROOT, "paper_1706_01613_gb300", "csrc")
    h = hashlib.sha256()
    for part in [source] + sorted(f for f in os.listdir(csrc) if f.endswith(".cuh")):
        with open(os.path.join(csrc, part), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return FALLBACK_HBM_GBS, "fallback"


# --------------------------------------------------------- multi-GPU ------

def aggregate(total_ms, n_units, steps, world, dist=None, device="cpu"):
    """Whole-job throughput of a weak-scaling run: every rank processed
    n_units per step; the job time is the slowest rank's.  Returns
    (units/s over all ranks, max total ms)."""
    if world > 1:
        import torch
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * n_units * steps / (total_ms / 1e3), total_ms


# ------------------------------------------------------------ CPU oracle ----

def oracle_rate(w, seconds, threads):
    """The oracle (as it stands) on a bounded sample of the same workload: the
    first k hexes, k doubling from 4096 until about `seconds` have been spent
    or the whole workload was done; the rate of the last (largest) pass.
    Returns (hex/s, sample description)."""
    import oracle
    oracle.build()
    k, t_all = min(w["n"], 4096), time.time()
    while True:
        sub = _subset(w, k)
        t0 = time.time()
        _oracle_call(sub, threads)
        dt = time.time() - t0
        if k >= w["n"] or time.time() - t_all >= seconds / 2:
            break
        k = min(w["n"], 2 * k)
    return k / dt, "the first %d of the %d hexes, one pass in %.2f s (%.1f s in all)" % (
        k, w["n"], dt, time.time() - t_all)


def reference_arm(args, w):
    """--impl reference: the CPU oracle on the host cores, K steps of a bounded
    sample each (sized from a calibration run so the whole run takes a few
    minutes)."""
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    k = 20_000
    sub = _subset(w, k)
    t0 = time.time()
    _oracle_call(sub, threads)
    rate = k / max(time.time() - t0, 1e-6)
    budget = 120.0
    per_step = max(1000, min(w["n"], int(rate * budget / max(1, args.steps + args.warmup))))
    sub = _subset(w, per_step)
    for _ in range(args.warmup):
        _oracle_call(sub, threads)
    t0 = time.time()
    for _ in range(args.steps):
        _oracle_call(sub, threads)
    dt = time.time() - t0
    value = per_step * args.steps / dt
    sample = "first %d hexes of the workload per step, %d threads" % (per_step, threads)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": w["name"], "sample_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def quad_run(steps, warmup, flush):
    """Linear quadrangles (Sec. 2.1): a 4096^2 structured 2D mesh (indexed),
    FP32-filtered and FP64 forms, device-resident inputs, L2 flushed between
    calls; CUDA events per call on the launch stream."""
    import torch
    from paper_1706_01613_gb300 import hexval as hv
    from paper_1706_01613_gb300 import synth
    nodes, conn = synth.structured_grid_2d(4096)
    N, C = torch.from_numpy(nodes).cuda(), torch.from_numpy(conn).cuda()
    n = conn.shape[0]
    out = {}
    for prec in ("fp32", "fp64"):
        v = hv.Validator(precision=prec, queue_capacity=1 << 10, max_batch=1 << 10,
                         max_nodes=1 << 10, exact_capacity=1 << 10)
        res = (torch.empty(n, dtype=torch.uint8, device="cuda"),
               torch.empty(n, dtype=torch.float64, device="cuda"),
               torch.empty(n, dtype=torch.float64, device="cuda"))
        for _ in range(warmup):
            flush.zero_()
            v.check_quads_indexed(N, C, out=res)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record()
            v.check_quads_indexed(N, C, out=res)
            b.record()
        torch.cuda.synchronize()
        v.raise_on_status()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        out[prec] = (n / (ms / 1e3), ms)
        v.close()
    abytes = (16 + 17) * n + 16 * nodes.shape[0]
    hbm, kind = peaks()
    achieved = abytes / (out["fp32"][1] / 1e3) / 1e9
    return {"workload": "4096^2 structured 2D mesh (4097^2 FP64 nodes, sigma 0.15, int32 conn)",
            "n_quad": n, "value": out["fp32"][0], "unit": "quad/s", "ms_per_call": out["fp32"][1],
            "fp64": {"value": out["fp64"][0], "unit": "quad/s", "ms_per_call": out["fp64"][1]},
            "roofline": {"bound": "hbm", "kernel": "quad32", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "peak_kind": kind + " (hbm_gbs)",
                         "algorithmic_bytes_per_launch": abytes, "traffic": None}}


def filter_run(steps, warmup, flush):
    """Candidate filtering: 40 candidate hexahedra per node over a 65^3 node
    array (cells of a perturbed grid relabelled by random cube symmetries),
    FP32-filtered check + compaction of the valid ids, per call with CUDA
    events, L2 flushed between calls."""
    import torch
    from paper_1706_01613_gb300 import hexval as hv
    from paper_1706_01613_gb300 import synth
    nodes, conn, _, _ = synth.hex_candidates()
    N, C = torch.from_numpy(nodes).cuda(), torch.from_numpy(conn).cuda()
    n = conn.shape[0]
    v = hv.Validator(precision="fp32", max_depth=8)
    flags = torch.empty(n, dtype=torch.uint8, device="cuda")
    out = (torch.empty(n, dtype=torch.int32, device="cuda"),
           torch.empty(1, dtype=torch.int32, device="cuda"))

    def call():
        v.check_indexed(N, C, out=(flags, None, None))
        v.compact(flags, (hv.VALID,), out=out)

    for _ in range(warmup):
        flush.zero_()
        call()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for a, b in ev:
        flush.zero_()
        a.record()
        call()
        b.record()
    torch.cuda.synchronize()
    v.raise_on_status()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    kept = int(out[1].item())
    v.close()
    return {"workload": "%d candidate hexes over %d nodes (40 per node, cube-symmetry relabelled "
                        "cells of a perturbed 64^3 grid)" % (n, nodes.shape[0]),
            "value": n / (ms / 1e3), "unit": "candidate/s", "ms_per_call": ms, "kept": kept}


def quality_run(w, dev_in, steps, warmup, flush):
    """Corner scaled Jacobian (Sec. 7's quality measure) on the benchmark
    mesh, per call with CUDA events, L2 flushed; HBM roofline on the bytes
    it must move (connectivity 32 B and output 4 B per element, 24 B per
    FP64 node)."""
    import torch
    from paper_1706_01613_gb300 import hexval as hv
    v = hv.Validator(precision="fp64", queue_capacity=1 << 10, max_batch=1 << 10,
                     max_nodes=1 << 10, exact_capacity=1 << 10)
    out = torch.empty(w["n"], dtype=torch.float32, device="cuda")

    def call():
        if w["kind"] == "indexed":
            v.corner_quality_indexed(dev_in[0], dev_in[1], out=out)
        else:
            v.corner_quality(dev_in[0], out=out)

    for _ in range(warmup):
        flush.zero_()
        call()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for a, b in ev:
        flush.zero_()
        a.record()
        call()
        b.record()
    torch.cuda.synchronize()
    v.raise_on_status()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    v.close()
    abytes = (32 + 4) * w["n"] + 24 * w["n_nodes"] if w["kind"] == "indexed" else 196 * w["n"]
    hbm, kind = peaks()
    achieved = abytes / (ms / 1e3) / 1e9
    return {"workload": w["name"], "value": w["n"] / (ms / 1e3), "unit": "hex/s",
            "ms_per_call": ms,
            "roofline": {"bound": "hbm", "kernel": "quality", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm,
                         "peak_kind": kind + " (hbm_gbs)", "algorithmic_bytes_per_launch": abytes,
                         "traffic": None}}


def minj_run(w, dev_in, steps, warmup, flush, rel_tol=1e-6, max_depth=12):
    """Minimum of J to a tolerance on the benchmark mesh (FP64 branch and
    bound on the coefficients), per call with CUDA events, L2 flushed."""
    import torch
    from paper_1706_01613_gb300 import hexval as hv
    v = hv.Validator(precision="fp64", max_depth=max_depth)

    def call():
        if w["kind"] == "indexed":
            return v.min_jacobian_indexed(dev_in[0], dev_in[1], rel_tol, max_depth)
        return v.min_jacobian(dev_in[0], rel_tol, max_depth)

    for _ in range(warmup):
        flush.zero_()
        call()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for a, b in ev:
        flush.zero_()
        a.record()
        lo, hi, dep = call()
        b.record()
    torch.cuda.synchronize()
    v.raise_on_status()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    d = dep.cpu().numpy()
    v.close()
    return {"workload": w["name"], "rel_tol": rel_tol, "max_depth": max_depth,
            "value": w["n"] / (ms / 1e3), "unit": "hex/s", "ms_per_call": ms,
            "mean_levels": float((d & 0x7F).mean()), "not_converged": int((d & 0x80).astype(bool).sum())}


def serving_run(precision, rate, n_requests, pool, slots=5, budget=40 << 30, seed=20175000,
                small_slots=1, small_n=100_000):
    """One continuous-batching run: Poisson arrivals at `rate`/s, sizes
    log-uniform in [100, pool size], `small_slots` of the slots kept for
    requests of at most `small_n` elements; returns the latency summary."""
    from paper_1706_01613_gb300 import serve
    reqs = serve.poisson_stream(pool, n_requests, rate, seed=seed + int(rate),
                                size_max=pool.max_n)
    ex = serve.GpuExecutor(slots, precision=precision, max_depth=8, keep_results=False,
                           queue_capacity=1 << 21, max_batch=1 << 24, max_nodes=1 << 24,
                           exact_capacity=1 << 14)
    try:
        sched = serve.run_stream(reqs, ex, slots=slots, budget_bytes=budget,
                                 small_slots=small_slots, small_n=small_n)
        bad = [s for s in ex.status() if s != 0]
    finally:
        ex.close()
    out = serve.latency_summary(reqs)
    out.update({"rate_per_s": rate, "rejected": len(sched.rejected), "status_errors": len(bad),
                "precision": precision, "slots": slots, "hbm_budget_gb": budget / 2**30,
                "slots_for_short_requests": small_slots, "short_request_max_n": small_n,
                "slot_scratch_gb": ex.fixed_bytes / 2**30})
    return out


def _subset(w, k):
    k = min(k, w["n"])
    if w["kind"] == "indexed":
        return dict(w, conn=w["conn"][:k], n=k)
    return dict(w, X=np.ascontiguousarray(w["X"][:, :, :k]), n=k)


def _oracle_call(w, threads):
    import oracle
    if w["kind"] == "indexed":
        return oracle.check_indexed(w["nodes"], w["conn"], max_depth=w["depth"], threads=threads)
    return oracle.check_soa(w["X"], max_depth=w["depth"], threads=threads)


# ------------------------------------------------- rooflines, summaries ----

def coeff_err(out32, out64):
    """bmin/bmax of the FP32-filtered form against the FP64 form's on the
    same input, relative to the element's largest |bmin|, |bmax|: max and
    99th percentile over the finite elements."""
    import torch
    lo32, hi32, lo64, hi64 = out32[1], out32[2], out64[1], out64[2]
    fin = torch.isfinite(lo64)
    scale = torch.maximum(lo64.abs(), hi64.abs())[fin]
    err = torch.maximum((lo32 - lo64).abs(), (hi32 - hi64).abs())[fin]
    rel = (err / torch.where(scale > 0, scale, torch.ones_like(scale))).sort().values
    if rel.numel() == 0:
        return None
    return {"max": float(rel[-1]), "p99": float(rel[int(0.99 * (rel.numel() - 1))]),
            "against": "FP64 form, same input", "elements": int(rel.numel())}


def roofline_of(w, prof, stats, calls):
    """Roofline of the dominant kernel of a form's step, from the per-phase
    event times: bytes for the bulk passes and the node conversion (HBM),
    FP64 instructions for the FP64 bulk pass, box expansions for the tail
    (FP64 boxes on the FP64 pipe, FP32 boxes on the FP32 pipe: the larger
    fraction is the bound).  Also the phase shares."""
    phases = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(phases, key=lambda k: phases[k][0])
    dom_ms = phases[dom][0] / phases[dom][1]
    share = {k: round(v[0] / sum(x[0] for x in phases.values()), 4) for k, v in phases.items()}
    hbm, peak_kind = peaks()
    if dom in ("bulk32", "nodes32"):
        abytes = algorithmic_bytes(w, dom)
        achieved = abytes / (dom_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": achieved / hbm, "peak_kind": peak_kind + " (hbm_gbs)",
                "traffic": traffic_for("bulk32_indexed" if w["kind"] == "indexed"
                                       else "bulk32_soa") if dom == "bulk32" else None,
                "algorithmic_bytes_per_launch": abytes, "avg_launch_ms": dom_ms}
    elif dom == "bulk64":
        achieved = OPS_PER_HEX * w["n"] / (dom_ms / 1e3) / 1e12
        roof = {"bound": "alu", "pipe": "fp64", "kernel": dom, "achieved": achieved,
                "peak": FP64_PEAK,
                "unit": "T FP64-inst/s", "frac": achieved / FP64_PEAK,
                "peak_kind": "nominal (1.25 TFLOP/s FP64, FMA = 2 flops)",
                "ops_per_hex": OPS_PER_HEX, "avg_launch_ms": dom_ms}
    else:
        b32 = stats.get("boxes_fp32", 0) / calls
        b64 = stats.get("boxes", 0) / calls - b32
        redo = stats.get("redone_tail", 0) / calls
        if b32 + b64 + redo == 0:  # nothing to do: the tail is its launch and barriers
            return {"bound": "latency", "kernel": dom, "avg_launch_ms": dom_ms,
                    "note": "no box to split, no element to redo; launch latency"}, share
        r64 = (OPS_PER_BOX * b64 + OPS_PER_HEX * redo) / (dom_ms / 1e3) / 1e12
        r32 = OPS_PER_BOX * b32 / (dom_ms / 1e3) / 1e12
        f64, f32 = r64 / FP64_PEAK, r32 / FP32_PEAK
        roof = {"bound": "alu", "pipe": "fp64" if f64 >= f32 else "fp32", "kernel": dom,
                "achieved": r64 if f64 >= f32 else r32,
                "peak": FP64_PEAK if f64 >= f32 else FP32_PEAK,
                "unit": "T FP64-inst/s" if f64 >= f32 else "T FP32-inst/s",
                "frac": max(f64, f32), "fp64_frac": f64, "fp32_frac": f32,
                "peak_kind": "nominal (recipe's unit counts at 2070 MHz)",
                "box_expansions_per_call": {"fp64": b64, "fp32": b32},
                "fp64_redone_per_call": redo, "ops_per_box": OPS_PER_BOX,
                "ops_per_hex": OPS_PER_HEX, "avg_launch_ms": dom_ms}
    return roof, share


def config_summary(cfg, steps, warmup, flush, retune=False):
    """One configuration in both forms (tuned launch configurations, device-
    resident inputs, L2 flushed between steps): throughput, the dominant
    kernel's roofline, flags equality and the FP32 coefficient error."""
    import torch
    from paper_1706_01613_gb300 import hexval as hv
    from paper_1706_01613_gb300 import tune
    w = workload(cfg, 0)
    if w["kind"] == "indexed":
        dev_in = (torch.from_numpy(w["nodes"]).cuda(), torch.from_numpy(w["conn"]).cuda())
    else:
        dev_in = (torch.from_numpy(w["X"]).cuda(),)
    caps = w.get("caps", {})
    out = {"workload": w["name"], "n_hex": w["n"], "unit": UNIT}
    res = {}
    for prec in ("fp32", "fp64"):
        k = steps if prec == "fp32" else max(3, steps // 5)
        cfgp = tune.best_config(prec, w["kind"], w["n"], dev_in, retune=retune,
                                max_depth=w["depth"], **caps)
        v = hv.Validator(precision=prec, max_depth=w["depth"], **cfgp, **caps)
        v.stats(reset=True)
        ms, prof, _, o = timed_steps(v, w, dev_in, k, warmup, flush, profile=True)
        st = v.stats()
        roof, share = roofline_of(w, prof, st, k + warmup)
        res[prec] = o
        out[prec] = {"value": w["n"] / (sum(ms) / k / 1e3), "ms_per_step": sum(ms) / k,
                     "steps": k, "launch": cfgp, "roofline": roof, "phase_share": share,
                     "stats_per_call": {a: b / (k + warmup) for a, b in st.items()}}
        v.close()
    out["value"] = out["fp32"]["value"]
    out["flags_equal"] = bool(torch.equal(res["fp32"][0] & 0x7F, res["fp64"][0] & 0x7F))
    out["fp32_coeff_err"] = coeff_err(res["fp32"], res["fp64"])
    del dev_in, res
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------- main ---

def profile_case(args, hv, torch):
    """--case: three calls of one kernel sequence on the workload (--config,
    --n), nothing timed, for profiler captures of committed code."""
    w = workload(args.config, 0, n=args.n)
    if w["kind"] == "indexed":
        dev = (torch.from_numpy(w["nodes"]).cuda(), torch.from_numpy(w["conn"]).cuda())
    else:
        dev = (torch.from_numpy(w["X"]).cuda(),)
    prec = "fp64" if args.case == "fp64" else "fp32"
    v = hv.Validator(precision=prec, max_depth=w["depth"], options=args.options | hv.OPT_NO_REPLAY,
                     **w.get("caps", {}))
    for _ in range(3):
        if args.case == "quality":
            if w["kind"] == "indexed":
                v.corner_quality_indexed(*dev)
            else:
                v.corner_quality(*dev)
        elif w["kind"] == "indexed":
            v.check_indexed(*dev)
        else:
            v.check_soa(*dev)
    torch.cuda.synchronize()
    v.raise_on_status()
    print(json.dumps({"case": args.case, "workload": w["name"], "calls": 3}))
    v.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=lambda c: c if c == "4b" else int(c), default=2,
                    choices=[1, 2, 3, 4, "4b"])
    ap.add_argument("--fp64-steps", type=int, default=None)
    ap.add_argument("--n", type=int, default=None,
                    help="first n elements of an SoA configuration (small profiler cases)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--serve", action="store_true",
                    help="sweep Poisson arrival rates of the serving workload instead")
    ap.add_argument("--serve-max-n", type=int, default=10_000_000)
    ap.add_argument("--serve-requests", type=int, default=10_000,
                    help="requests of the serving stream measured in the default run")
    ap.add_argument("--serve-rate", type=float, default=300.0,
                    help="Poisson arrival rate (requests/s) of that stream")
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="skip the other configurations and the serving stream")
    ap.add_argument("--retune", action="store_true",
                    help="time every launch configuration again instead of using the cache")
    ap.add_argument("--bulk-threads", type=int, default=None,
                    help="fixed FP32 launch configuration instead of the autotuner's")
    ap.add_argument("--options", type=int, default=0, help="options with --bulk-threads")
    ap.add_argument("--case", choices=["quality", "fp32", "fp64"], default=None,
                    help="profiler captures: run one kernel sequence on the workload three "
                         "times and exit (corner quality, or a check in one form with "
                         "--options)")
    ap.add_argument("--no-quads", dest="quads", action="store_false",
                    help="skip the quadrangle and candidate-filtering measurements")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        w = workload(args.config, 0)
        print(json.dumps(reference_arm(args, w)))
        return 0

    import torch
    import torch.distributed as dist
    from paper_1706_01613_gb300 import hexval as hv
    from paper_1706_01613_gb300 import _build

    torch.cuda.set_device(local)
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    if args.case:
        return profile_case(args, hv, torch)
    if args.serve:
        from paper_1706_01613_gb300 import serve
        pool = serve.Pool(args.serve_max_n)
        sweep = []
        for precision in ("fp32", "fp64"):
            for rate in (10, 30, 100, 300, 1000, 2000):
                n_req = int(min(400, max(40, 5 * rate)))
                sweep.append(serving_run(precision, rate, n_req, pool))
        if rank == 0:
            print(json.dumps({"metric": METRIC, "mode": "serving sweep",
                              "sizes": [100, args.serve_max_n], "sweep": sweep}))
        return 0
    w = workload(args.config, rank, world, args.n)
    if w["kind"] == "indexed":
        dev_in = (torch.from_numpy(w["nodes"]).cuda(), torch.from_numpy(w["conn"]).cuda())
    else:
        dev_in = (torch.from_numpy(w["X"]).cuda(),)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    props = torch.cuda.get_device_properties(local)
    bus = getattr(props, "pci_bus_id", None)

    # launch configuration of the FP32 form from the autotuner (timed here on
    # this workload, cached per device and shape)
    from paper_1706_01613_gb300 import tune
    if args.bulk_threads is not None:  # fixed launch configuration (profiling runs)
        tuned = {"options": args.options, "bulk_threads": args.bulk_threads}
        tuned64 = {}
    else:
        tuned = tune.best_config("fp32", w["kind"], w["n"], dev_in, retune=args.retune,
                                 max_depth=w["depth"], **w.get("caps", {}))
        tuned64 = tune.best_config("fp64", w["kind"], w["n"], dev_in, retune=args.retune,
                                   max_depth=w["depth"], **w.get("caps", {}))
    v32 = hv.Validator(precision="fp32", max_depth=w["depth"], **tuned, **w.get("caps", {}))
    v64 = hv.Validator(precision="fp64", max_depth=w["depth"], **tuned64, **w.get("caps", {}))

    clocks = ClockSampler(bus)
    if rank == 0:
        clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    v32.stats(reset=True)
    ms32, prof32, window, out32 = timed_steps(v32, w, dev_in, args.steps, args.warmup, flush,
                                              profile=True)
    st32 = v32.stats()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.stop()
    value, total = aggregate(sum(ms32), w["n"], args.steps, world, dist, "cuda")
    ms_step = total / args.steps

    # plain FP64 form, same input, fewer steps (about 70x slower)
    k64 = args.fp64_steps or max(3, args.steps // 50)
    w64 = max(3, args.warmup // 5)
    v64.stats(reset=True)
    ms64, prof64, _, out64 = timed_steps(v64, w, dev_in, k64, w64, flush, profile=True)
    st64 = v64.stats()
    value64, tot64 = aggregate(sum(ms64), w["n"], k64, world, dist, "cuda")
    same = bool(torch.equal(out32[0] & 0x7F, out64[0] & 0x7F))
    err32 = coeff_err(out32, out64)

    # end to end through the public API with host buffers
    e2e_ms, h2d, d2h, _ = e2e_steps(v32, w, args.e2e_steps, 3)
    e2e_val, _ = aggregate(e2e_ms, w["n"], 1, world, dist, "cuda")

    if rank != 0:
        dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel of each form's step
    roof, share = roofline_of(w, prof32, st32, args.steps + args.warmup)
    if roof["kernel"] == "bulk32":
        # the same bytes over the whole step (node conversion and tail included)
        roof["whole_step_frac"] = roof["algorithmic_bytes_per_launch"] / (ms_step / 1e3) / 1e9 / \
            roof["peak"]
    roof64, share64 = roofline_of(w, prof64, st64, k64 + w64)

    cpu = None
    if world == 1:
        import oracle
        oracle.build()
        thr = oracle.max_threads()
        rate, sample = oracle_rate(w, args.cpu_seconds, thr)
        cpu = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample}

    # the single-GPU sections (the other rows of the scope table, the other
    # configurations, serving) only in a one-GPU run: with several ranks the
    # others have left and their GPUs would be held for nothing
    extras = args.quads and world == 1
    quads = quad_run(max(5, args.steps // 20), 3, flush) if extras else None
    filt = filter_run(max(5, args.steps // 50), 3, flush) if extras else None
    mj = minj_run(w, dev_in, 5, 2, flush) if extras else None
    qual = quality_run(w, dev_in, max(5, args.steps // 50), 3, flush) if extras else None

    # the other configurations (device-resident, both forms) and the serving
    # stream of the scope table: 10,000 requests, sizes log-uniform in
    # [100, 10^7], Poisson arrivals, both forms
    others, latency = {}, None
    if args.configs and args.config == 2 and world == 1:
        v32.close()
        v64.close()
        del dev_in
        torch.cuda.empty_cache()
        for c in (1, 3, 4):
            others["config%d" % c] = config_summary(c, max(20, args.steps // 100), 3, flush,
                                                    args.retune)
        from paper_1706_01613_gb300 import serve
        pool = serve.Pool(args.serve_max_n)
        latency = {prec: serving_run(prec, args.serve_rate, args.serve_requests, pool)
                   for prec in ("fp32", "fp64")}
        del pool

    sampled_steps = (args.steps + PROFILE_EVERY - 1) // PROFILE_EVERY
    launches_per_step = sum(v[1] for v in prof32.values() if v[1] > 0) / sampled_steps
    rec = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (certified, f64/exact escalation)",
        "data": "synthetic",
        "config": {"workload": w["name"], "n_hex": w["n"], "form": "fp32-filtered",
                   "max_depth": w["depth"], "launch": tuned, "launch_fp64": tuned64,
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": ("element-range shards of one mesh, one per GPU, no "
                                   "collective on the data path" if world > 1 and
                                   args.config == 2 else
                                   "replicas (one input per GPU, no collective)")},
        "fp64": {"value": value64, "unit": UNIT, "steps": k64, "ms_per_step": tot64 / k64,
                 "flags_equal_fp32_form": same, "roofline": roof64, "phase_share": share64},
        "fp32_coeff_err": err32,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "link_gbs": (h2d + d2h) / (e2e_ms / 1e3) / 1e9,
                "outputs": "flags, bmin, bmax", "chunks": 4},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "roofline": roof,
        "phase_share": share,
        "stats_fp32": st32,
        "cpu_baseline": cpu,
        "latency": latency,
        "configs": others,
        "quads": quads,
        "filter": filt,
        "min_jacobian": mj,
        "corner_quality": qual,
        "clocks": clocks.summary(*window),
    }
    print(json.dumps(rec))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
