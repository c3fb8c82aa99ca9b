"""Continuous batching of CDUGKS solves on one GPU.

Requests (problem description, initial fields, end time) arrive over time.
The server

* admits a waiting request as soon as a slot and enough device memory are
  free (admission by HBM footprint: the request's workspace bytes from
  ``cdugks_workspace_bytes``, against a byte budget), allocating its
  workspace and initialising its state on the device while the batch runs;
* steps the selected requests together as one batch, in rounds of one
  launch per kernel and step (or, with the persistent batched step, one
  launch per round in which each member advances its own number of steps,
  ``cdugks_batch_step_members``), never past a request's own step count, so
  a request computes exactly what it would alone;
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


def persistent_tile(precision: int, dim: int) -> int:
    """The tile shape with the persistent batched step for (precision, dim)."""
    shapes = {(cdugks.FP32, 1): (128,), (cdugks.FP32, 2): (32, 8), (cdugks.FP64, 1): (64,)}
    if (precision, dim) not in shapes:
        raise ValueError(f"no persistent batched step for precision {precision}, dim {dim}")
    return cdugks.find_tile(precision, dim, shapes[(precision, dim)], 4)


class Server:
    """Continuous batching on one GPU.

    A request is *resident* once its state is on the device (prepared); the
    batch steps a subset of the resident requests each round.  Two policies:

    * ``"srpt"`` (the default): shortest remaining work first.  Each round the
      resident requests are ordered by remaining point-updates (cells x
      velocities x remaining steps, known exactly) and the shortest are taken
      until their points per step reach ``fill_points`` (enough parallel work
      to fill the GPU); the others stay resident and wait, out of the batch.
      Short requests overtake long ones, which then use the GPU alone.
    * ``"share"``: every resident request advances every round (processor
      sharing).

    By default a round steps the batch with one launch per kernel and step,
    for min over its members of their remaining steps (a member never runs
    past its own step count).  persistent=True uses the persistent batched
    step instead: a round is one launch in which every member advances
    min(round steps, its remaining steps), so a member near its end does not
    shorten the round for the others; with the few large members the
    shortest-first policy selects it is slower than the launch chain (its
    loads are coherent and its phases wait per member), so it is not the
    default.  The round length adapts so that a round takes about
    ``round_target_s`` of device time (from the measured point-update rate),
    which bounds how long a new request waits to be scheduled.

    While a round runs on the device, a worker thread does the host-side work:
    it creates and initialises requests that fit the memory budget (their own
    streams) and reads back the results of finished ones; the main thread polls
    the round's completion event and changes the membership (in place, for a
    persistent batch with room) and launches only at round boundaries.  The
    library releases the GIL in every call, so the two threads run at once.
    """

    def __init__(self, budget_bytes: int, max_slots: int = 64, max_round: int = 64, device: str = "cuda:0",
                 clock=time.perf_counter, persistent: bool = False, round_target_s: float = 0.025,
                 max_items: int = 1 << 18, policy: str = "srpt", fill_points: float = 3e7,
                 velocity_groups: int = 0):
        if policy not in ("srpt", "share"):
            raise ValueError(f"unknown policy {policy}")
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.max_round = int(max_round)
        self.device = device
        self.clock = clock
        self.persistent = bool(persistent)
        self.round_target_s = float(round_target_s)
        self.max_items = int(max_items)
        self.policy = policy
        self.fill_points = float(fill_points)
        self.velocity_groups = int(velocity_groups)     # for requests that name none (0: the library's choice)
        self.waiting: list[Request] = []           # submitted, not yet prepared
        self.resident: list[Request] = []          # prepared (state on the device), not finished
        self.active: list[Request] = []            # batch members, in the batch's member order
        self.done_in_batch: list[Request] = []     # finished, still batch members until the next boundary
        self.leaving: deque[Request] = deque()     # out of the batch, result not read back yet
        self.finished: list[Request] = []
        self.used = 0
        self.batch = None
        self.point_updates = 0
        self.rounds = 0
        self.rebuilds = 0          # batches created
        self.membership_changes = 0
        self.launches = 0          # kernels of this library launched by the server
        self.rate = 3e10           # point-updates/s, refined from the rounds
        self.device_s = 0.0        # device time of the rounds (CUDA events)
        self._pool = None
        self._job = None           # the worker thread's current job (future, kind, request)

    @staticmethod
    def remaining_work(q: Request) -> int:
        return q.points * (q.nsteps - q.done_steps)

    # -- admission --------------------------------------------------------
    def _default_tile(self, req: Request) -> int:
        """The face-store shape with the persistent step for requests of the
        default physics (the shape the persistent batch needs, and the tuned one
        for the 2D workloads); the library's default shape for the request's
        physics otherwise (collision model, force, reconstruction)."""
        plain = not (req.cfg.get("collision", 0) or req.cfg.get("recon", 0) or any(req.cfg.get("accel", (0.0,))))
        if self.persistent or plain:
            try:
                return persistent_tile(req.precision, int(req.cfg["dim"]))
            except ValueError:
                if self.persistent:
                    raise
        return 0

    def submit(self, req: Request):
        if not req.tile_id:
            req.tile_id = self._default_tile(req)
        if not req.velocity_groups:
            req.velocity_groups = self.velocity_groups
        req.footprint = footprint_bytes(req)
        if req.footprint > self.budget:
            raise ValueError(f"request {req.rid} needs {req.footprint} bytes, more than the budget {self.budget}")
        self.waiting.append(req)

    def _next_to_prepare(self):
        """The waiting request to prepare next (shortest work first under srpt,
        arrival order otherwise), if a slot and the memory budget allow it."""
        if not self.waiting or len(self.resident) >= self.max_slots:
            return None
        k = min(range(len(self.waiting)), key=lambda i: self.remaining_work(self.waiting[i])) \
            if self.policy == "srpt" else 0
        return k if self.used + self.waiting[k].footprint <= self.budget else None

    def _prepare(self, req: Request):
        """Workspace, velocity tables and initial state of a request (worker thread)."""
        import torch

        st = torch.cuda.Stream(torch.device(self.device))
        s = cdugks.Solver(req.cfg, precision=req.precision, device=self.device, tile_id=req.tile_id,
                          velocity_groups=req.velocity_groups, stream=st)
        s.init(req.fields)              # returns when the state is on the device
        req.solver = s

    def _collect(self, req: Request):
        """Read the result of a finished request back (worker thread)."""
        req.result = req.solver.moments()

    def _host_work(self, now: float) -> bool:
        """Start or finish one job of the worker thread; True if something happened."""
        if self._job is not None:
            fut, kind, req = self._job
            if not fut.done():
                return False
            fut.result()               # re-raises an error of the job
            self._job = None
            self.launches += 1         # the initial state, or the moments
            if kind == "prepare":
                self.resident.append(req)
            else:
                req.finished_at = self.clock() - self._t0
                req.solver = None      # frees its workspace
                self.used -= req.footprint
                self.finished.append(req)
            return True
        if self.leaving:
            req = self.leaving.popleft()
            self._job = (self._pool.submit(self._collect, req), "collect", req)
            return True
        k = self._next_to_prepare()
        if k is not None:
            req = self.waiting.pop(k)
            self.used += req.footprint
            req.admitted_at = now
            self._job = (self._pool.submit(self._prepare, req), "prepare", req)
            return True
        return False

    # -- rounds -------------------------------------------------------------
    def _select(self) -> list:
        """The resident requests the next round steps."""
        if self.policy == "share" or not self.resident:
            return list(self.resident)
        order = sorted(self.resident, key=self.remaining_work)
        out, pts = [], 0
        for q in order:
            out.append(q)
            pts += q.points
            if pts >= self.fill_points:
                break
        return out

    def _boundary(self):
        """Membership changes at a round boundary (nothing of the batch in
        flight): finished members leave, the selected requests join, the rest
        of the members step out (they stay resident)."""
        want = self._select()
        wanted = {id(q) for q in want}
        if not want:
            if self.batch is not None:
                self.batch = None          # nothing left to step: drop the batch
                self.leaving.extend(self.done_in_batch)
                self.done_in_batch = []
                self.active = []
            return
        if self.batch is None:
            self.batch = cdugks.Batch([q.solver for q in want], device=self.device, persistent=self.persistent,
                                      max_members=self.max_slots if self.persistent else 0,
                                      max_items=self.max_items if self.persistent else 0)
            self.rebuilds += 1
            self.active = list(want)
            return
        members = {id(q) for q in self.active} | {id(q) for q in self.done_in_batch}
        for q in want:                      # join first, so the batch never empties
            if id(q) not in members:
                self.batch.admit(q.solver)
                self.active.append(q)
                self.membership_changes += 1
        for q in self.done_in_batch:
            self.batch.retire(q.solver)
            self.membership_changes += 1
            self.leaving.append(q)
        self.done_in_batch = []
        for q in [q for q in self.active if id(q) not in wanted]:
            self.batch.retire(q.solver)
            self.active.remove(q)
            self.membership_changes += 1
        # the batch's member order: the Python side appends on admit and drops on retire
        self.active = [q for s in self.batch.members for q in self.active if q.solver is s]

    def _launch(self):
        import torch

        pts = sum(q.points for q in self.active)
        r = max(1, min(self.max_round, int(self.round_target_s * self.rate / max(pts, 1))))
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(self.batch.stream)
        if self.persistent:
            steps = [min(r, q.nsteps - q.done_steps) for q in self.active]
            self.batch.step_members(steps)
            self.launches += 1
        else:
            r = min([r] + [q.nsteps - q.done_steps for q in self.active])
            steps = [r] * len(self.active)
            self.batch.step(r)
            # per batched step: sweep A and sweep B per tile shape, face constants, W update
            self.launches += r * (2 * len({q.tile_id for q in self.active}) + 2)
        ev1.record(self.batch.stream)
        return ev0, ev1, steps

    def _finish_round(self, inflight):
        ev0, ev1, steps = inflight
        rc = self.batch.sync()          # the stream is idle: reads the status words
        if rc != 0:
            raise RuntimeError(f"a member reported status {rc}")
        ms = ev0.elapsed_time(ev1)
        pu = sum(n * q.points for n, q in zip(steps, self.active))
        for n, q in zip(steps, self.active):
            q.done_steps += n
        self.point_updates += pu
        self.device_s += ms * 1e-3
        if ms > 0 and pu > 0:
            self.rate = 0.5 * self.rate + 0.5 * pu / (ms * 1e-3)
        self.rounds += 1
        done = [q for q in self.active if q.done_steps >= q.nsteps]
        if done:
            ids = {id(q) for q in done}
            self.active = [q for q in self.active if id(q) not in ids]
            self.resident = [q for q in self.resident if id(q) not in ids]
            self.done_in_batch.extend(done)

    def run(self, requests, time_limit: float | None = None):
        """Serve requests whose ``arrival`` times are seconds after the start.
        Returns when all are finished, or once the time limit has passed (the
        round in flight is completed; unfinished requests keep their progress
        in ``done_steps``)."""
        from concurrent.futures import ThreadPoolExecutor

        pending = deque(sorted(requests, key=lambda q: q.arrival))
        self._t0 = self.clock()
        self._pool = ThreadPoolExecutor(max_workers=1)
        inflight = None
        try:
            while True:
                now = self.clock() - self._t0
                over = time_limit is not None and now > time_limit
                while pending and pending[0].arrival <= now and not over:
                    self.submit(pending.popleft())
                if inflight is not None and inflight[1].query():
                    self._finish_round(inflight)
                    inflight = None
                if inflight is None and (not over or self.done_in_batch):
                    if over:                    # finished members still leave
                        self.resident, kept = [], self.resident
                        self._boundary()
                        self.resident = kept
                    else:
                        self._boundary()
                        if self.active:
                            inflight = self._launch()
                busy = self._host_work(now)
                if over and inflight is None and self._job is None and not self.leaving \
                        and not self.done_in_batch:
                    break
                if not (pending or self.waiting or self.resident or self.leaving or self.done_in_batch
                        or self._job is not None or inflight is not None):
                    break
                if not busy:
                    wait = 2e-4
                    if inflight is None and self._job is None and pending:
                        wait = min(1e-3, max(0.0, pending[0].arrival - now))
                    time.sleep(wait)
        finally:
            self._pool.shutdown(wait=True)
            self._pool = None
        self.batch = None
        self.wall_s = self.clock() - self._t0
        return self.finished

    # -- report ---------------------------------------------------------------
    def report(self, wall_s: float | None = None) -> dict:
        wall_s = self.wall_s if wall_s is None else wall_s
        tts = [q.finished_at - q.arrival for q in self.finished]
        return {
            "finished": len(self.finished),
            "unfinished": len(self.waiting) + len(self.resident),
            "p50_time_to_solution_s": float(np.percentile(tts, 50)) if tts else None,
            "p99_time_to_solution_s": float(np.percentile(tts, 99)) if tts else None,
            "point_updates": self.point_updates,
            "aggregate_point_updates_per_s": self.point_updates / wall_s if wall_s > 0 else None,
            "wall_s": wall_s,
            "device_busy_frac": self.device_s / wall_s if wall_s > 0 else None,
            "rounds": self.rounds,
            "batch_rebuilds": self.rebuilds,
            "membership_changes": self.membership_changes,
            "kernel_launches": self.launches,
            "launch": "persistent batched step, one launch per round" if self.persistent
            else "one launch per kernel per batched step",
            "policy": {"srpt": f"shortest remaining work first, {self.fill_points:.0e} points per step filled",
                       "share": "every resident request every round"}[self.policy],
        }


def stream_c5(count=64, seed=1, rate=50.0, side_range=(64, 512), vside_range=(16, 48), t_end=1.0, tile_id=0):
    """The served workload: Poisson arrivals (rate per second) of 2D
    Gresho-vortex and Kelvin-Helmholtz solves of log-uniform grid side and
    velocity-grid side and Kn in [1e-4, 1] (FP32), each run to t_end, all with
    the sweep tile shape tile_id (0: the server's choice)."""
    out = []
    for k, (t, cfg, f) in enumerate(wl.workload_c5(count=count, seed=seed, rate=rate, side_range=side_range,
                                                   vside_range=vside_range, t_end=t_end)):
        out.append(Request(rid=k, cfg=cfg, fields=f, t_end=t_end, arrival=t, precision=cdugks.FP32,
                           tile_id=tile_id))
    return out
