"""Tuner for the sweep launch shape: spatial tile x velocity-group split.

For an instance size (dim, cells bucket, velocity count, precision) it times
every candidate (tile id, velocity groups) for a few steps with CUDA events in
the context the instance will run in:

* ``context="alone"`` -- the instance by itself (one solver fills the GPU);
* ``context="batch"`` -- copies of the instance stepped as one batch, as many
  as needed to give every SM work, scored by time per phase-space point.

Group counts are tried at powers of two, then refined around the best one
for its shape (how many CTAs a launch has against the SM count decides how
full its last wave is).  The fastest candidate is cached in a JSON file
(``CDUGKS_TUNE_CACHE`` or
``~/.cache/cdugks_tune.json``) keyed by the size bucket, so a later process
reuses it.  Choices never change results beyond rounding order: every tile and
group split computes the same scheme.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import cdugks
from . import workloads as wl

SMS = 152


def cache_path() -> str:
    return os.environ.get("CDUGKS_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "cdugks_tune.json"))


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(path, d):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def size_key(cfg, precision, context):
    D = cfg["dim"]
    cells = wl.ncells(cfg)
    bucket = 2 ** int(round(math.log2(max(cells, 1))))
    recon = ":faces-gradient" if cfg.get("recon", 0) else ""
    coll = (":shakhov" if cfg.get("collision", 0) else "") + (":accel" if any(cfg.get("accel", (0, 0, 0))) else "")
    return (f"{'fp32' if precision == cdugks.FP32 else 'fp64'}:{context}:D{D}:cells~{bucket}:nv{wl.nvel(cfg)}"
            f"{recon}{coll}")


def candidates(cfg, precision, context="alone"):
    nt = cdugks.load().cdugks_tile_count(precision, cfg["dim"])
    nvt = (wl.nvel(cfg) + 3) // 4
    groups = [g for g in (1, 2, 4, 8, 16, 32) if g <= nvt]
    dirichlet = any(wl.BC_DIRICHLET in cfg["bc"][a] for a in range(cfg["dim"]))
    r2 = bool(cfg.get("recon", 0))
    sk = bool(cfg.get("collision", 0))
    ac = any(cfg.get("accel", (0.0, 0.0, 0.0)))
    tiles = []
    for t in range(nt):
        mode = cdugks.tile_shape(precision, cfg["dim"], t)[1]
        if bool(mode & 8) != r2 or bool(mode & 16) != sk or bool(mode & 32) != ac:
            continue                      # shapes of another reconstruction, collision or force compute another scheme
        if context != "alone" and sk:
            continue                      # Shakhov instances are not batched
        if context != "alone" and mode & 3 != 0:
            continue                      # only shapes that form phibar+ themselves are batched
        if mode & 3 == 2 and dirichlet:
            continue                      # stored slopes: periodic / specular only
        tiles.append(t)
    return [(t, g) for t in tiles for g in groups]


def _uniform_fields(cfg):
    nc = wl.ncells(cfg)
    D = cfg["dim"]
    _, X = wl.cell_centres(cfg)
    f = np.zeros((nc, 2 + D))
    f[:, 0] = 1.0 + 0.01 * np.sin(2 * math.pi * X[0])
    f[:, 1 + D] = cfg["T_ref"]
    return f


def _time(cfg, precision, tile, groups, context, steps, device):
    import torch

    f = _uniform_fields(cfg)
    if context == "alone":
        s = cdugks.Solver(cfg, precision=precision, device=device, tile_id=tile, velocity_groups=groups)
        s.init(f)
        s.step(2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s.stream)
        s.step(steps)
        e1.record(s.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps / (wl.ncells(cfg) * wl.nvel(cfg))
    # batch: enough copies that the launch covers the GPU a few times over
    info_s = cdugks.Solver(cfg, precision=precision, device=device, tile_id=tile, velocity_groups=groups)
    inf = info_s.info()
    tiles = 1
    for a in range(cfg["dim"]):
        tiles *= (cfg["n"][a] + inf.tile[a] - 1) // inf.tile[a]
    per = tiles * inf.velocity_groups
    copies = max(1, min(64, math.ceil(4 * SMS / per)))
    members = [info_s] + [cdugks.Solver(cfg, precision=precision, device=device, tile_id=tile,
                                        velocity_groups=groups) for _ in range(copies - 1)]
    for m in members:
        m.init(f)
    b = cdugks.Batch(members, device=device)
    b.step(2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b.sync()
    e0.record(b.stream)
    b.step(steps)
    e1.record(b.stream)
    b.sync()
    return e0.elapsed_time(e1) / steps / (copies * wl.ncells(cfg) * wl.nvel(cfg))


def tune(cfg, precision, context="alone", steps=5, device="cuda:0", cache=None, refresh=False):
    """Best (tile_id, velocity_groups) for this instance size; cached."""
    path = cache or cache_path()
    d = _load_cache(path)
    key = size_key(cfg, precision, context)
    if key in d and not refresh:
        return tuple(d[key]["choice"])
    import torch

    results = []

    def trial(tile, groups):
        try:
            results.append((_time(cfg, precision, tile, groups, context, steps, device), tile, groups))
        except torch.OutOfMemoryError:     # this shape's extra buffers do not fit beside the state
            pass
        torch.cuda.empty_cache()

    for tile, groups in candidates(cfg, precision, context):
        trial(tile, groups)
    if not results:
        raise RuntimeError(f"no tile shape fits on {device} for {key}")
    # refine the group count of the best shape between the powers of two (the
    # number of CTAs against the SM count decides how full the last wave is)
    results.sort()
    _, t0, g0 = results[0]
    nvt = (wl.nvel(cfg) + 3) // 4
    tried = {(t, g) for _, t, g in results}
    for g in sorted({g0 - 1, g0 + 1, (3 * g0) // 4, (5 * g0) // 4, (3 * g0) // 2}):
        if 1 <= g <= nvt and (t0, g) not in tried:
            trial(t0, g)
    results.sort()
    best = results[0]
    d = _load_cache(path)
    d[key] = {"choice": [best[1], best[2]], "ms_per_point": best[0],
              "tried": [[t, g, ms] for ms, t, g in results]}
    _save_cache(path, d)
    return best[1], best[2]
