"""Continuous batching of CDUGKS solves on one GPU.

Requests (problem description, initial fields, end time) arrive over time.
The server

* admits a waiting request as soon as a slot and enough device memory are
  free (admission by HBM footprint: the request's workspace bytes from
  ``cdugks_workspace_bytes``, against a byte budget), allocating its
  workspace and initialising its state on the device;
* steps every active request together as one batch (one launch per kernel for
  all of them, ``cdugks_batch_*``), in rounds that never carry a request past
  its own step count, so a request computes exactly what it would alone;
* retires a request when it reaches its end time: reads its macroscopic
  fields back, frees its workspace, and records its time to solution;
* changes the batch's membership in place between rounds
  (``cdugks_batch_admit`` / ``cdugks_batch_retire``), so requests that arrive
  while others run join them at the next round; a batch is created only when
  none is running.

All arithmetic runs in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import dataclasses
import math
import time
from collections import deque

import numpy as np

from . import cdugks
from . import workloads as wl


@dataclasses.dataclass
class Request:
    rid: int
    cfg: dict
    fields: np.ndarray
    t_end: float
    arrival: float = 0.0          # seconds after the stream starts
    precision: int = cdugks.FP32
    tile_id: int = 0
    velocity_groups: int = 0
    # filled by the server
    nsteps: int = 0
    done_steps: int = 0
    admitted_at: float = math.nan
    finished_at: float = math.nan
    result: np.ndarray | None = None
    footprint: int = 0
    solver: cdugks.Solver | None = None

    @property
    def points(self) -> int:
        return wl.ncells(self.cfg) * wl.nvel(self.cfg)


def steps_to(cfg_dt: float, t_end: float) -> int:
    return max(1, int(math.ceil(t_end / cfg_dt - 1e-9)))


def footprint_bytes(req: Request) -> int:
    """Device bytes the request needs (its workspace), without touching the GPU."""
    import ctypes

    lib = cdugks.load()
    g, v, p = cdugks.describe(req.cfg, req.precision)
    h = ctypes.c_void_p()
    cdugks._check(lib.cdugks_create(ctypes.byref(g), ctypes.byref(v), ctypes.byref(p), ctypes.byref(h)))
    try:
        if req.cfg.get("collision", 0):
            cdugks._check(lib.cdugks_set_collision(h, int(req.cfg["collision"])))
        if any(req.cfg.get("accel", (0.0, 0.0, 0.0))):
            acc = np.zeros(3)
            acc[: len(req.cfg["accel"])] = req.cfg["accel"]
            cdugks._check(lib.cdugks_set_acceleration(h, cdugks._dptr(acc)))
        if req.cfg.get("recon", 0):
            cdugks._check(lib.cdugks_set_reconstruction(h, int(req.cfg["recon"])))
        if req.tile_id:
            cdugks._check(lib.cdugks_set_tile(h, int(req.tile_id)))
        if req.velocity_groups:
            cdugks._check(lib.cdugks_set_velocity_groups(h, int(req.velocity_groups)))
        n = ctypes.c_size_t()
        cdugks._check(lib.cdugks_workspace_bytes(h, ctypes.byref(n)))
        info = cdugks.Info()
        cdugks._check(lib.cdugks_info(h, ctypes.byref(info)))
        req.nsteps = steps_to(info.dt, req.t_end)
        return int(n.value) + 256
    finally:
        lib.cdugks_destroy(h)


class Server:
    def __init__(self, budget_bytes: int, max_slots: int = 64, max_round: int = 64, device: str = "cuda:0",
                 clock=time.perf_counter):
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.max_round = int(max_round)
        self.device = device
        self.clock = clock
        self.waiting: deque[Request] = deque()
        self.active: list[Request] = []
        self.finished: list[Request] = []
        self.used = 0
        self.batch = None
        self.point_updates = 0
        self.rounds = 0
        self.rebuilds = 0          # batches created
        self.membership_changes = 0
        self.launches = 0          # kernels of this library launched by the server

    # -- admission --------------------------------------------------------
    def submit(self, req: Request):
        req.footprint = footprint_bytes(req)
        if req.footprint > self.budget:
            raise ValueError(f"request {req.rid} needs {req.footprint} bytes, more than the budget {self.budget}")
        self.waiting.append(req)

    def _admit(self, now: float) -> list:
        admitted = []
        while self.waiting and len(self.active) < self.max_slots:
            req = self.waiting[0]
            if self.used + req.footprint > self.budget:
                break
            self.waiting.popleft()
            s = cdugks.Solver(req.cfg, precision=req.precision, device=self.device, tile_id=req.tile_id,
                              velocity_groups=req.velocity_groups)
            s.init(req.fields)
            self.launches += 1                    # the initial state
            req.solver = s
            req.admitted_at = now
            self.used += req.footprint
            self.active.append(req)
            admitted.append(req)
        return admitted

    # -- retirement -------------------------------------------------------
    def _retire(self, now: float):
        done = [q for q in self.active if q.done_steps >= q.nsteps]
        self.active = [q for q in self.active if q.done_steps < q.nsteps]
        if done and self.batch is not None:
            if self.active:
                for req in done:
                    self.batch.retire(req.solver)
                    self.membership_changes += 1
            else:
                self.batch = None                  # the last members leave: drop the batch first
        for req in done:
            req.result = req.solver.moments()
            self.launches += 1                    # the moments
            req.finished_at = now
            req.solver = None                      # frees its workspace
            self.used -= req.footprint
            self.finished.append(req)

    # -- one round ----------------------------------------------------------
    def _round(self):
        r = min([self.max_round] + [q.nsteps - q.done_steps for q in self.active])
        self.batch.step(r)
        rc = self.batch.sync()
        if rc != 0:
            raise RuntimeError(f"a member reported status {rc}")
        for q in self.active:
            q.done_steps += r
        self.point_updates += r * sum(q.points for q in self.active)
        self.rounds += 1
        # per batched step: sweep A and sweep B per tile shape, face constants, W update
        self.launches += r * (2 * len({q.tile_id for q in self.active}) + 2)

    def run(self, requests, time_limit: float | None = None):
        """Serve requests whose ``arrival`` times are seconds after the start.
        Returns when all are finished (or the time limit passes)."""
        pending = deque(sorted(requests, key=lambda q: q.arrival))
        t0 = self.clock()
        while pending or self.waiting or self.active:
            now = self.clock() - t0
            if time_limit is not None and now > time_limit:
                break
            while pending and pending[0].arrival <= now:
                self.submit(pending.popleft())
            admitted = self._admit(now)
            if not self.active:
                if pending:
                    time.sleep(min(0.001, max(0.0, pending[0].arrival - now)))
                continue
            if self.batch is None:
                self.batch = cdugks.Batch([q.solver for q in self.active], device=self.device)
                self.rebuilds += 1
            else:
                for req in admitted:
                    self.batch.admit(req.solver)
                    self.membership_changes += 1
            self._round()
            self._retire(self.clock() - t0)
        return self.finished

    # -- report ---------------------------------------------------------------
    def report(self, wall_s: float) -> dict:
        tts = [q.finished_at - q.arrival for q in self.finished]
        return {
            "finished": len(self.finished),
            "p50_time_to_solution_s": float(np.percentile(tts, 50)) if tts else None,
            "p99_time_to_solution_s": float(np.percentile(tts, 99)) if tts else None,
            "point_updates": self.point_updates,
            "aggregate_point_updates_per_s": self.point_updates / wall_s if wall_s > 0 else None,
            "rounds": self.rounds,
            "batch_rebuilds": self.rebuilds,
            "membership_changes": self.membership_changes,
            "kernel_launches": self.launches,
        }


def stream_c5(count=64, seed=1, rate=50.0, side_range=(32, 128), vside_range=(8, 24), t_end=0.05, tile_id=0):
    """The served workload: Poisson arrivals of 2D Gresho-vortex and
    Kelvin-Helmholtz solves of varied size, Kn and velocity grid (FP32), all
    with the sweep tile shape tile_id."""
    out = []
    for k, (t, cfg, f) in enumerate(wl.workload_c5(count=count, seed=seed, rate=rate, side_range=side_range,
                                                   vside_range=vside_range, t_end=t_end)):
        out.append(Request(rid=k, cfg=cfg, fields=f, t_end=t_end, arrival=t, precision=cdugks.FP32,
                           tile_id=tile_id))
    return out
