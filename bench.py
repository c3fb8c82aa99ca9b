#!/usr/bin/env python
"""Benchmark of the CDUGKS phase-space step on GB300.

Metric: phase-space point-updates per second (one point-update = g and b
advanced one time step at one (cell, discrete velocity) point, the "phase space
cell update" of the paper's scaling study).

Default workload: the 3D shear-wave problem with FP32 storage, 64^3 periodic
cells x 24^3 velocities on [-6,6]^3, Kn = 1e-4, Pr = 2/3 (synthetic initial
fields; 3.6e9 phase-space points, 29 GB per state buffer).  One bench step =
one full time step of the scheme.  The same line carries, as sub-objects, the
plain FP64 path on the same workload, the batched form (256 uneven 1D
thermoacoustic instances in FP32) with its FP64 one-instance-at-a-time
comparison, and the served stream (the first 8 requests of the Poisson stream
of 2D solves to t = 1, capped at 60 s of wall time) with modelled one-at-a-time
FP32 and FP64 servers of the same requests.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c1|c2|c3|c3s|c3m|c3p|c4|c5|einfeldt] [--tune]

N > 1 runs independent replicas (the path does not shard across GPUs on this
build), one per rank under torch.distributed.run; value = all points / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2208_09132_gb300 import workloads as wl  # noqa: E402

METRIC = "phase-space point-updates/s"
UNIT = "point-updates/s"
ALGO_BYTES = {  # algorithmic bytes per phase-space point per launch (state read/write only)
    "sweep_a": {"fp32": 8, "fp64": 16},     # read g*, b*
    "sweep_b": {"fp32": 16, "fp64": 32},    # read g*, b*; write g*, b*
}
MODE_NAMES = {0: "fused", 1: "prepared phibar+", 2: "stored phibar+ and slopes", 4: "fused, face store",
              5: "prepared phibar+, face store", 6: "stored phibar+ and slopes, face store"}


def design_bytes(mode, D, elt):
    """Bytes per phase-space point each launch of a sweep mode moves by design
    (state, prepared arrays, stored face values; halo re-reads not counted)."""
    src, faces = mode & 3, bool(mode & 4)
    d = {}
    if src == 1:
        d["prep"] = 4 * elt                                   # read phi*, write phibar+
    elif src == 2:
        d["slopes"] = (4 + 2 * D) * elt                       # read phi*, write phibar+ and D slopes
    a_in = {0: 2, 1: 2, 2: 2 + 2 * D}[src] * elt
    d["sweep_a"] = a_in + (2 * D * elt if faces else 0)       # (+ write the face values)
    d["sweep_b"] = (2 * D + 4) * elt if faces else a_in + (2 if src else 0) * elt + 2 * elt
    if mode & 16:                                             # Shakhov: raw moments of the faces and of phi*
        d["face_moments"] = 2 * D * elt
        d["cell_moments"] = 2 * elt
    if mode & 32:                                             # acceleration: the force terms, written and read
        d["prep"] += 2 * elt
        d["sweep_b"] += 2 * elt
    return d


def pick_workload(name):
    if name == "c1":
        return wl.workload_c1()
    if name == "c2":
        return wl.workload_c2()
    if name == "c3":
        return wl.workload_c3(kn=1e-4)
    if name == "c3s":        # 3D shear at half resolution in space and velocity
        return wl.workload_c3(kn=1e-4, scale=2, nv=12)
    if name == "c3m":        # 3D shear on the full velocity grid at half resolution in space
        return wl.workload_c3(kn=1e-4, scale=2, nv=24)
    if name == "c3p":        # the same at quarter resolution in space (a few GB: the counter-capture size)
        return wl.workload_c3(kn=1e-4, scale=4, nv=24)
    if name == "einfeldt":   # the paper's high-resolution Einfeldt run (Sec. 3.2), FP64, to t = 0.125
        cfg, f = wl.einfeldt(nx=8192, nv=129)
        cfg["precision"] = "fp64"
        return cfg, f
    raise SystemExit(f"unknown workload {name}")


def points(cfg):
    return wl.ncells(cfg) * wl.nvel(cfg)


# --------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers

def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_sha():
    """Hash of the sweep kernels' source (the section of kernels.cuh that holds
    them, the lean sweeps, the persistent batched step and their launch
    helpers): profile counters taken on other source are not reported."""
    csrc = os.path.join(ROOT, "paper_2208_09132_gb300", "csrc")
    txt = open(os.path.join(csrc, "kernels.cuh")).read()
    a = txt.index("// --------------------------------------------------------------- the sweep")
    b = txt.index("// Face constants from the group-summed face W")
    h = hashlib.sha256(txt[a:b].encode())
    for f in ("lean.cuh", "persist.cuh", "sweeps_impl.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(workload, kernel, precision, tile_id=None, groups=None, field="dram_bytes_per_point"):
    """DRAM bytes (or, with field="thread_instructions_per_point", executed
    thread instructions) per point for a kernel from the committed ncu
    summary, if it was taken on the current kernel source in the same launch
    configuration; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("kernel_source_sha") != kernel_source_sha():
        return None
    e = d.get("entries", {}).get(f"{workload}:{precision}:{kernel}")
    if e is None:
        return None
    if (tile_id is not None and e.get("tile_id") != tile_id) or (groups is not None and e.get("velocity_groups") != groups):
        return None
    return float(e[field]) if field in e else None


def issue_roofline(ipp, points_per_launch, seconds, sms, sm_mhz):
    """A kernel against the instruction-issue ceiling: ipp thread instructions
    per point over a launch of points_per_launch points taking seconds, against
    sms x 128 thread instructions per clock (4 schedulers x 32 lanes) at sm_mhz."""
    rate = ipp * points_per_launch / seconds
    peak = sms * 128 * sm_mhz * 1e6
    return {"thread_instructions_per_point": ipp, "achieved": round(rate / 1e12, 3), "peak": round(peak / 1e12, 3),
            "unit": "T thread-instructions/s", "frac": round(rate / peak, 4)}


def cpu_baseline(cfg, budget_s=12.0):
    """The CPU oracle, as it stands, on a bounded sample of the workload: the same
    velocity grid and physics on a reduced spatial grid."""
    import oracle
    oracle.build()
    sample = dict(cfg)
    D = cfg["dim"]
    side = {1: 256, 2: 32, 3: 8}[D]
    sample["n"] = [min(cfg["n"][a], side) if a < D else 1 for a in range(3)]
    if D == 3 and wl.nvel(cfg) > 4096:
        sample["n"] = [4, 4, 4]
    sample["dt"] = 0.0
    _, X = wl.cell_centres(sample)
    nc = wl.ncells(sample)
    rng_fields = np.column_stack([np.ones(nc)] + [0.1 * np.sin(2 * math.pi * X[0])] * D + [np.full(nc, cfg["T_ref"])])
    o = oracle.Oracle(sample)
    o.init(rng_fields)
    k, el0 = 1, 0.0               # per-step time from a calibration run of at least 0.25 s
    while True:
        t0 = time.perf_counter()
        o.step(k)
        el0 = time.perf_counter() - t0
        if el0 >= 0.25 or k >= 4096:
            break
        k *= 4
    t1 = el0 / k
    n = max(1, min(200000, int(budget_s / max(t1, 1e-7))))
    t0 = time.perf_counter()
    o.step(n)
    el = time.perf_counter() - t0
    pts = wl.ncells(sample) * wl.nvel(sample)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": pts * n / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{'x'.join(str(v) for v in sample['n'][:D])} cells x {wl.nvel(sample)} velocities, "
                      f"{n} steps, {el:.1f} s (same velocity grid and physics as the workload)"}


# ------------------------------------------------------------------- ranks

def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- our arm

def run_batched(args, ws, rank, local, sub=False):
    """Many uneven 1D instances (the batched thermoacoustic workload) stepped
    together.  Headline: the persistent batched step (every phase of every
    member in one launch, replayed from a CUDA graph of 10 steps, one launch per
    graph); beside it the same batch with one launch per kernel and phase.  All
    members take the 1D face-store shape of 128 cells with one velocity group
    (one shape per persistent batch; measured the fastest uniform choice).
    With sub=True it is the "batched" part of the default line (200 timed
    steps) and returns the sub-object."""
    import torch

    from paper_2208_09132_gb300 import cdugks

    dev = f"cuda:{local}"
    torch.cuda.set_device(local)
    probs = wl.workload_c4()
    P = sum(points(c) for c, _ in probs)
    tile = cdugks.find_tile(cdugks.FP32, 1, (128,), 4)
    gsteps = 10
    K = 200 if sub else max(gsteps, args.steps // gsteps * gsteps)

    def make(persistent):
        members = []
        for cfg, f in probs:
            s = cdugks.Solver(cfg, precision=cdugks.FP32, device=dev, tile_id=tile, velocity_groups=1)
            s.init(f)
            members.append(s)
        return members, cdugks.Batch(members, device=dev, persistent=persistent)

    def timed(batch, steps):
        stream = batch.stream
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps // gsteps + 1)]
        barrier(ws)
        torch.cuda.synchronize()
        ev[0].record(stream)
        for k in range(steps // gsteps):
            batch.step(gsteps)
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        return max_over_ranks(ev[0].elapsed_time(ev[-1]), ws)

    # one launch per kernel and phase (context)
    members, batch = make(False)
    batch.capture(gsteps)
    batch.step(max(args.warmup, 3) * gsteps)
    if batch.sync() != 0:
        raise RuntimeError("a member's status flagged a broken state during warm-up")
    kern_ms = timed(batch, K)
    kern_ok = batch.sync() == 0
    del batch, members
    torch.cuda.empty_cache()

    # the persistent step (headline)
    members, batch = make(True)
    batch.capture(gsteps)
    batch.step(max(args.warmup, 3) * gsteps)
    if batch.sync() != 0:
        raise RuntimeError("a member's status flagged a broken state during warm-up")
    clocks = ClockSampler(local)
    clocks.start()
    total_ms = timed(batch, K)
    clk = clocks.stop()
    status = batch.sync()
    value = ws * P * K / (total_ms / 1e3)
    peak, peak_kind = measured_peak_hbm()
    achieved = 24 * P / (total_ms / K / 1e3) / 1e9
    # DRAM bytes of one launch (gsteps steps of every member) from the committed capture
    tpp = ncu_traffic("c4", "persistent", "fp32", tile, 1)
    traffic = None if tpp is None else tpp * P * gsteps
    # step latency: single-step graph replays (one launch each), each between two events
    stream = batch.stream
    batch.capture(1)
    nlat = 500
    lev = [torch.cuda.Event(enable_timing=True) for _ in range(nlat + 1)]
    torch.cuda.synchronize()
    lev[0].record(stream)
    for k in range(nlat):
        batch.step(1)
        lev[k + 1].record(stream)
    torch.cuda.synchronize()
    per_step = [lev[k].elapsed_time(lev[k + 1]) for k in range(nlat)]
    status = status or batch.sync()

    # the plain FP64 path, one instance at a time, on the same instances
    fp64 = None
    if not args.skip_fp64:
        plain = []
        for cfg, f in probs:
            s = cdugks.Solver(cfg, precision=cdugks.FP64, device=dev)
            s.init(f)
            plain.append(s)
        n64 = 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(n64):
            for s in plain:
                s.step(1)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        fp64 = {"value": P * n64 / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / n64, "steps": n64,
                "what": "each instance stepped alone in FP64, one after another"}
        del plain
    del batch, members
    torch.cuda.empty_cache()
    if rank != 0:
        return None
    lat = {"p50": float(np.percentile(per_step, 50)), "p99": float(np.percentile(per_step, 99)),
           "samples": nlat, "what": "per batched step, single-step graph replays between two CUDA events"}
    per_kernel = {"value": ws * P * K / (kern_ms / 1e3), "unit": UNIT, "ms_per_step": kern_ms / K,
                  "launch": f"4 launches per step (sweep A, face constants, sweep B, W update), CUDA graph of {gsteps} steps",
                  "status_ok": kern_ok}
    launch = f"persistent: every phase of every member, {gsteps} steps per launch (CUDA graph: memset + 1 kernel)"
    if sub:
        return {"workload": "batched_thermoacoustic_1d_256_instances", "value": value, "unit": UNIT,
                "ms_per_step": total_ms / K, "steps": K, "instances": len(probs), "points": P,
                "launch": launch, "tile": [128], "velocity_groups": 1, "latency_ms": lat,
                "per_kernel_launches": per_kernel, "fp64_plain": fp64,
                "vs_fp64_plain": (value / fp64["value"]) if fp64 else None,
                "step_hbm_frac": round(achieved / peak, 4),
                "roofline": {"bound": "hbm", "kernel": "persistent batched step", "achieved": round(achieved, 1),
                             "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                             "algorithmic_bytes_per_point": 24, "traffic": traffic,
                             "traffic_per": f"launch ({gsteps} steps of every member)"},
                "status_ok": status == 0}
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": args.warmup,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched_thermoacoustic_1d_256_instances", "instances": len(probs), "points": P,
                   "launch": launch, "tile": [128], "velocity_groups": 1,
                   "l2": "inputs larger than L2" if P * 8 > 129e6 else "state fits in L2"},
        "latency_ms": lat,
        "roofline": {"bound": "hbm", "kernel": "persistent batched step", "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                     "algorithmic_bytes_per_point": 24, "traffic": traffic},
        "cpu_baseline": None, "e2e": None, "fp64_plain": fp64, "per_kernel_launches": per_kernel,
        "gpu_launches": K // gsteps, "clocks": clk, "status_ok": status == 0,
    }


def solo_step_ms(req, prec, dev, steps=3):
    """Milliseconds per step of one served request stepped alone (its untuned
    default shape for the precision): a warm-up step, then `steps` timed."""
    import torch

    from paper_2208_09132_gb300 import cdugks, tune

    tile, groups = tune.choose(req.cfg, prec, context="alone", device=dev)
    s = cdugks.Solver(req.cfg, precision=prec, device=dev, tile_id=tile, velocity_groups=groups)
    s.init(req.fields)
    s.step(1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    s.step(steps)
    e1.record(s.stream)
    e1.synchronize()
    ok = s.sync_status() == 0
    ms = e0.elapsed_time(e1) / steps
    del s
    return ms, ok


def one_at_a_time(reqs, step_ms, cap_s, order="fifo"):
    """A server that solves the same requests one at a time, each taking
    nsteps x its measured step time, in arrival order ("fifo") or, whenever it
    is free, the shortest waiting solve first ("sjf", non-preemptive): the
    time-to-solution statistics of the requests it finishes within cap_s and
    the point-updates per second it delivers within the cap."""
    jobs = sorted(zip(reqs, step_ms), key=lambda j: j[0].arrival)
    t, tts, pu_done, busy = 0.0, [], 0.0, 0.0
    waiting = []
    while (jobs or waiting) and t < cap_s:
        while jobs and jobs[0][0].arrival <= t:
            waiting.append(jobs.pop(0))
        if not waiting:
            t = jobs[0][0].arrival
            continue
        k = 0 if order == "fifo" else min(range(len(waiting)), key=lambda i: waiting[i][0].nsteps * waiting[i][1])
        q, ms = waiting.pop(k)
        dur = q.nsteps * ms * 1e-3
        run = min(dur, cap_s - t)
        pu_done += q.points * q.nsteps * run / dur
        busy += run
        t += dur
        if t <= cap_s:
            tts.append(t - q.arrival)
    wall = min(cap_s, t)
    return {"finished": len(tts),
            "p50_time_to_solution_s": float(np.percentile(tts, 50)) if tts else None,
            "p99_time_to_solution_s": float(np.percentile(tts, 99)) if tts else None,
            "aggregate_point_updates_per_s": pu_done / wall if wall > 0 else None,
            "device_point_updates_per_s": pu_done / busy if busy > 0 else None}


def run_served(args, ws, rank, local, sub=False):
    """The served stream: Poisson arrivals (50/s) of 2D Gresho-vortex and
    Kelvin-Helmholtz solves, grids 64^2-512^2, velocity grids 16^2-48^2, Kn
    1e-4..1, each run to t = 1, admitted by device-memory footprint and stepped
    together (one launch per kernel and step), for at most
    args.serve_cap seconds of wall time.  Then each request is timed alone in
    FP32 and in FP64, and a one-at-a-time server of the same requests is modelled
    from those step times under the same cap.  sub=True: the "served" part of
    the default line (args.requests requests)."""
    import torch

    from paper_2208_09132_gb300 import cdugks, serving

    dev = f"cuda:{local}"
    torch.cuda.set_device(local)
    reqs = serving.stream_c5(count=args.requests, t_end=args.t_end)
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.6 * free)
    # warm-up: two short solves load and initialise everything
    serving.Server(budget_bytes=budget, device=dev).run(serving.stream_c5(count=2, t_end=0.002))
    torch.cuda.synchronize()
    srv = serving.Server(budget_bytes=budget, max_slots=64, max_round=64, device=dev, policy=args.policy,
                         fill_points=args.fill_points, persistent=args.serve_launch == "persistent",
                         velocity_groups=args.serve_groups)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    srv.run(reqs, time_limit=args.serve_cap)
    torch.cuda.synchronize()
    wall = max_over_ranks(time.perf_counter() - t0, ws)
    clk = clocks.stop()
    rep = srv.report(wall)
    del srv
    torch.cuda.empty_cache()
    # every request alone, FP32 and FP64 (same requests, full nsteps modelled)
    ms32, ms64, ok = [], [], True
    for q in sorted(reqs, key=lambda q: q.arrival) if not args.skip_alone else []:
        a, oa = solo_step_ms(q, cdugks.FP32, dev)
        b, ob = solo_step_ms(q, cdugks.FP64, dev)
        torch.cuda.empty_cache()
        ms32.append(a)
        ms64.append(b)
        ok = ok and oa and ob
    cap = args.serve_cap
    alone32 = {o: one_at_a_time(reqs, ms32, cap, o) for o in ("fifo", "sjf")} if ms32 else None
    alone64 = {o: one_at_a_time(reqs, ms64, cap, o) for o in ("fifo", "sjf")} if ms64 else None
    value = ws * rep["point_updates"] / wall
    total_pu = sum(q.points * q.nsteps for q in reqs)
    cfgd = {"workload": f"served_stream_{len(reqs)}_requests", "arrivals": "Poisson 50/s, seed 1",
            "requests": len(reqs), "t_end": args.t_end, "wall_cap_s": cap,
            "sizes": "cells 64^2-512^2, velocities 16^2-48^2 (log-uniform sides), Gresho or Kelvin-Helmholtz, "
                     "Kn 1e-4..1 (log-uniform), FP32",
            "total_point_updates_requested": total_pu,
            "admission": "device-memory footprint within 60% of free memory, <= 64 slots",
            "tile_id": serving.persistent_tile(cdugks.FP32, 2), "tile": [32, 8],
            "sweep_mode": "fused, face store", "launch": rep["launch"], "policy": rep["policy"]}
    served = {"value": value, "unit": UNIT, **rep,
              "fp32_one_at_a_time": alone32, "fp64_one_at_a_time": alone64,
              "vs_fp64_one_at_a_time": value / alone64["fifo"]["aggregate_point_updates_per_s"]
              if alone64 and alone64["fifo"]["aggregate_point_updates_per_s"] else None,
              "one_at_a_time_what": "each request timed alone (3 steps after a warm-up, its default shape), "
                                    "then a one-at-a-time server of the same arrivals modelled from those step "
                                    "times under the same cap: first come first served (fifo) and shortest "
                                    "solve first, non-preemptive (sjf)",
              "status_ok": ok}
    if rank != 0:
        return None
    if sub:
        return {"workload": cfgd["workload"], **{k: cfgd[k] for k in ("requests", "t_end", "wall_cap_s", "sizes",
                                                                      "total_point_updates_requested")},
                **served}
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": rep["rounds"], "warmup": 1, "ms_per_step": wall * 1e3 / max(rep["rounds"], 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": cfgd,
        "latency_ms": {"p50": (rep["p50_time_to_solution_s"] or math.nan) * 1e3,
                       "p99": (rep["p99_time_to_solution_s"] or math.nan) * 1e3,
                       "what": "time to solution from arrival, finished requests"},
        "served": served, "cpu_baseline": None, "e2e": None, "roofline": None,
        "gpu_launches": rep["kernel_launches"], "clocks": clk,
    }


def time_fp64_plain(cfg, fields, dev, budget_s=20.0):
    """The plain FP64 path on the same workload, one instance: a warm-up step,
    then as many timed steps (at least 2, at most 20) as fit the time budget."""
    import torch

    from paper_2208_09132_gb300 import cdugks

    from paper_2208_09132_gb300 import tune
    tile, groups = tune.choose(cfg, cdugks.FP64, context="alone", device=dev)
    try:
        s64 = cdugks.Solver(cfg, precision=cdugks.FP64, device=dev, tile_id=tile, velocity_groups=groups)
    except torch.OutOfMemoryError:        # the shape's extra buffers do not fit beside the FP64 state
        torch.cuda.empty_cache()
        s64 = cdugks.Solver(cfg, precision=cdugks.FP64, device=dev)
    s64.init(fields)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s64.stream)
    s64.step(1)
    e1.record(s64.stream)
    torch.cuda.synchronize()
    one = e0.elapsed_time(e1) / 1e3
    n64 = int(max(2, min(20, budget_s / max(one, 1e-6))))
    e0.record(s64.stream)
    s64.step(n64)
    e1.record(s64.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    P = points(cfg)
    info = s64.info()
    out = {"value": P * n64 / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / n64, "steps": n64,
           "tile": list(info.tile)[:cfg["dim"]], "tile_id": info.tile_id,
           "velocity_groups": info.velocity_groups, "status_ok": s64.sync_status() == 0}
    del s64
    torch.cuda.empty_cache()
    return out


def run_ours(args, ws, rank, local):
    import torch

    from paper_2208_09132_gb300 import cdugks

    dev = f"cuda:{local}"
    torch.cuda.set_device(local)
    cfg, fields = pick_workload(args.workload)
    if args.recon:
        cfg["recon"] = args.recon
    if args.collision:
        cfg["collision"] = args.collision
    if args.accel:
        cfg["accel"] = ([float(v) for v in args.accel.split(",")] + [0.0, 0.0])[:3]
    if args.precision:
        cfg["precision"] = args.precision
    prec = cdugks.FP64 if cfg["precision"] == "fp64" else cdugks.FP32
    pname = "fp64" if prec == cdugks.FP64 else "fp32"
    P = points(cfg)
    tile, groups = 0, 0
    if args.tile is not None:
        tile, groups = args.tile, args.groups or 0
    else:
        from paper_2208_09132_gb300 import tune
        tile, groups = tune.choose(cfg, prec, context="alone", device=dev, allow_tuning=args.tune)
    s = cdugks.Solver(cfg, precision=prec, device=dev, stream=torch.cuda.Stream(device=dev), tile_id=tile,
                      velocity_groups=groups)
    stream = s.stream
    s.init(fields)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(args.warmup):
        if k == args.warmup - 1:
            e0.record(stream)
        s.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    if s.sync_status() != 0:
        raise RuntimeError("device status flagged a broken state during warm-up")
    step_est = e0.elapsed_time(e1) / 1e3

    # steps replayed from CUDA graphs of gsteps steps when the count allows and
    # the step is short enough for launch overhead to matter (one launch per
    # gsteps steps; the same kernels and results)
    gsteps = args.graph if (args.graph > 1 and args.steps % args.graph == 0 and step_est < 5e-3) else 1
    if gsteps > 1:
        s.capture(gsteps)
        s.step(gsteps)              # first replay, untimed
        torch.cuda.synchronize()

    # ---- device-resident timed region
    clocks = ClockSampler(local)
    clocks.start()
    nwin = args.steps // gsteps
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(nwin + 1)]
    barrier(ws)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(nwin):
        s.step(gsteps)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    per_step = [ev[k].elapsed_time(ev[k + 1]) / gsteps for k in range(nwin)]
    total_ms = ev[0].elapsed_time(ev[nwin])
    total_ms = max_over_ranks(total_ms, ws)
    status = s.sync_status()
    value = ws * P * args.steps / (total_ms / 1e3)

    # ---- step latency: every step on its own between two events, as many steps
    # as about 10 s allow (at least the timed count, at most 500)
    nlat = int(max(nwin if gsteps == 1 else 0, min(500, 10.0 / max(step_est, 1e-6))))
    if gsteps == 1 and nlat <= nwin:
        lat = per_step
    else:
        if gsteps > 1:
            s.capture(1)
        lev = [torch.cuda.Event(enable_timing=True) for _ in range(nlat + 1)]
        torch.cuda.synchronize()
        lev[0].record(stream)
        for k in range(nlat):
            s.step(1)
            lev[k + 1].record(stream)
        torch.cuda.synchronize()
        lat = [lev[k].elapsed_time(lev[k + 1]) for k in range(nlat)]

    # ---- per-kernel durations of the same launches (CUDA events on the bound stream)
    nprof = int(max(3, min(args.steps, 50, 5.0 / max(step_est, 1e-6))))
    ph = s.profile_step(nprof)
    names = ["sweep_a", "face_constants", "sweep_b", "w_update"]
    dom = max(("sweep_a", "sweep_b"), key=lambda k: ph[names.index(k)])
    t_dom = ph[names.index(dom)] / 1e3
    abytes = ALGO_BYTES[dom][pname] * P
    mode = cdugks.tile_shape(prec, cfg["dim"], s.info().tile_id)[1]
    peak, peak_kind = measured_peak_hbm()
    achieved = abytes / t_dom / 1e9
    traffic_pp = ncu_traffic(args.workload, dom, pname, s.info().tile_id, s.info().velocity_groups)
    step_bytes = ALGO_BYTES["sweep_a"][pname] + ALGO_BYTES["sweep_b"][pname]
    step_ms = total_ms / args.steps
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                "algorithmic_bytes_per_point": ALGO_BYTES[dom][pname],
                "traffic": None if traffic_pp is None else traffic_pp * P,
                "phase_ms": {n: round(float(v), 4) for n, v in zip(names, ph)},
                "design_bytes_per_point": design_bytes(mode, cfg["dim"], 4 if pname == "fp32" else 8),
                "step_bytes_per_point": step_bytes,
                "step_achieved": round(step_bytes * P / (step_ms / 1e3) / 1e9, 1),
                "step_hbm_frac": round(step_bytes * P / (step_ms / 1e3) / 1e9 / peak, 4)}
    # The sweeps are bound by instruction issue rather than HBM: the same kernel
    # against the issue ceiling, SMs x 128 thread instructions per clock at the
    # maximum SM clock, from the executed instructions of the ncu capture.
    ipp = ncu_traffic(args.workload, dom, pname, s.info().tile_id, s.info().velocity_groups,
                      field="thread_instructions_per_point")
    if ipp is not None:
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        roofline["issue"] = issue_roofline(ipp, P, t_dom, sms, (clk or {}).get("sm_max_mhz") or 2070.0)

    # ---- end to end through the C ABI with pinned host buffers
    NM = 2 + cfg["dim"]
    host_in = torch.empty((wl.ncells(cfg), NM), dtype=torch.float64, pin_memory=True)
    host_in.numpy()[:] = fields
    host_out = torch.empty((wl.ncells(cfg), NM), dtype=torch.float64, pin_memory=True)
    e2e_steps = args.steps
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.init(host_in.numpy())
    s.step(e2e_steps)
    s.moments(host_out.numpy())
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, ws)
    e2e = {"value": ws * P * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": host_in.numel() * 8 / e2e_steps,
           "d2h_bytes_per_step": host_out.numel() * 8 / e2e_steps,
           "what": "cdugks_init from pinned host fields + cdugks_step(K) + cdugks_moments to pinned host"}
    info = s.info()
    dt_used = s.dt
    launches_per_step = 4 + (1 if mode & 3 else 0) + (2 if mode & 16 else 0)
    del s
    torch.cuda.empty_cache()

    # ---- the batched form (C4) with its own FP64 one-at-a-time comparison
    batched = None
    if args.workload == "c3" and not args.skip_batched:
        batched = run_batched(args, ws, rank, local, sub=True)

    # ---- the served stream (C5) under its wall-clock cap
    served = None
    if args.workload == "c3" and not args.skip_served:
        served = run_served(args, ws, rank, local, sub=True)

    # ---- the plain FP64 path on the same workload (the one-instance comparison)
    fp64 = None
    if prec == cdugks.FP32 and not args.skip_fp64:
        fp64 = time_fp64_plain(cfg, fields, dev)

    result = None
    if rank == 0:
        cpu = cpu_baseline(cfg) if (ws == 1 and not args.skip_cpu) else None
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "time_to_solution_s": (step_ms * cfg["steps"] / 1e3) if args.workload == "einfeldt" else None,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if pname == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": cfg["name"], "precision": pname, "cells": wl.ncells(cfg),
                       "velocities": wl.nvel(cfg), "points": P, "dt": dt_used,
                       "state_bytes": info.state_bytes,
                       "tile": list(info.tile)[:cfg["dim"]], "velocity_groups": info.velocity_groups,
                       "tile_id": info.tile_id, "sweep_mode": MODE_NAMES.get(mode & 7, str(mode)),
                       "reconstruction": "face gradient" if mode & 8 else "upwind cell",
                       "collision": "Shakhov" if mode & 16 else "two relaxation times (Sec. 2)",
                       "acceleration": list(cfg.get("accel", [0.0, 0.0, 0.0]))[:cfg["dim"]],
                       "launch": f"CUDA graphs of {gsteps} steps" if gsteps > 1 else "one launch per kernel",
                       "l2": "inputs larger than L2 (state > 129 MB)" if info.state_bytes > 129e6
                             else "state fits in L2",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "samples": len(lat), "what": "per step, each step between two CUDA events"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "fp64_plain": fp64,
            "batched": batched,
            "served": served,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
            "status_ok": status == 0,
        }
    return result


# ---------------------------------------------------------- reference arm

def run_reference(args, ws, rank):
    """The CPU oracle as it stands, each step a bounded sample of the workload."""
    if rank != 0:
        return None
    import oracle
    oracle.build()
    cfg, _ = pick_workload(args.workload)
    if args.recon:
        cfg["recon"] = args.recon
    if args.collision:
        cfg["collision"] = args.collision
    if args.accel:
        cfg["accel"] = ([float(v) for v in args.accel.split(",")] + [0.0, 0.0])[:3]
    D = cfg["dim"]
    sample = dict(cfg)
    side = {1: 256, 2: 32, 3: 4}[D]
    sample["n"] = [min(cfg["n"][a], side) if a < D else 1 for a in range(3)]
    sample["dt"] = 0.0
    nc = wl.ncells(sample)
    _, X = wl.cell_centres(sample)
    f = np.column_stack([np.ones(nc)] + [0.1 * np.sin(2 * math.pi * X[0])] * D + [np.full(nc, cfg["T_ref"])])
    o = oracle.Oracle(sample)
    o.init(f)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    pts = wl.ncells(sample) * wl.nvel(sample)
    v = pts * args.steps / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    samp = f"{'x'.join(str(v) for v in sample['n'][:D])} cells x {wl.nvel(sample)} velocities per step"
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "precision": "fp64 oracle"},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": samp, "value": v, "unit": UNIT},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 1000; einfeldt: to t_end)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c3")
    ap.add_argument("--skip-cpu", action="store_true", help="omit the CPU oracle baseline")
    ap.add_argument("--skip-fp64", action="store_true", help="omit the FP64 plain comparison")
    ap.add_argument("--skip-batched", action="store_true", help="omit the batched sub-object of the 3D workload")
    ap.add_argument("--tune", dest="tune", action="store_true",
                    help="tune sizes missing from the tuner cache (default: cached choice, else a default shape)")
    ap.add_argument("--tile", type=int, default=None, help="pin the tile shape id (skips tuning)")
    ap.add_argument("--graph", type=int, default=10, help="steps per captured CUDA graph (1: plain launches)")
    ap.add_argument("--recon", type=int, default=0, help="1: the face-gradient reconstruction (1D/2D workloads)")
    ap.add_argument("--collision", type=int, default=0, help="1: the Shakhov collision model")
    ap.add_argument("--accel", default="", help="uniform external acceleration, e.g. 0,-0.5")
    ap.add_argument("--groups", type=int, default=None, help="with --tile: velocity groups")
    ap.add_argument("--requests", type=int, default=None,
                    help="served stream: number of requests (default 64; 8 in the default line)")
    ap.add_argument("--t-end", type=float, default=1.0, help="served stream: end time of each solve")
    ap.add_argument("--serve-cap", type=float, default=None,
                    help="served stream: wall-clock cap in seconds (default 120; 60 in the default line)")
    ap.add_argument("--policy", choices=["srpt", "share"], default="srpt",
                    help="served stream: shortest remaining work first, or every request every round")
    ap.add_argument("--fill-points", type=float, default=3e7,
                    help="served stream, srpt: points per step the shortest requests of a round fill")
    ap.add_argument("--serve-launch", choices=["persistent", "per-kernel"], default="per-kernel",
                    help="served stream: the persistent batched step (per-member step counts) or one launch per kernel")
    ap.add_argument("--serve-groups", type=int, default=0,
                    help="served stream: velocity groups of every request (0: the library's choice per request)")
    ap.add_argument("--skip-alone", action="store_true",
                    help="served stream: omit timing each request alone (the one-at-a-time models)")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default=None,
                    help="override the workload's storage precision")
    ap.add_argument("--skip-served", action="store_true", help="omit the served sub-object of the 3D workload")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.steps is None:   # the einfeldt workload runs its whole solve; the 3D workload 20 steps, others 1000
        args.steps = (pick_workload("einfeldt")[0]["steps"] if args.workload == "einfeldt"
                      else (20 if args.workload in ("c3", "c3s", "c3m", "c3p") else 1000))
    if args.requests is None:
        args.requests = 64 if args.workload == "c5" else 8
    if args.serve_cap is None:
        args.serve_cap = 120.0 if args.workload == "c5" else 60.0
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        res = run_reference(args, ws, rank)
    elif args.workload == "c4":
        res = run_batched(args, ws, rank, local)
    elif args.workload == "c5":
        res = run_served(args, ws, rank, local)
    else:
        res = run_ours(args, ws, rank, local)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
