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
reuses it.  Choices this tuner made on a GB300 for the benchmark sizes ship
beside it (``tune_cache.json``, same format, each entry tagged with the shape
table it was tuned on); ``choose`` takes a cached choice, else tunes when
asked to, else a default shape.  ``python -m paper_2208_09132_gb300.tune``
tunes the benchmark sizes into the cache.  Choices never change results beyond rounding order: every tile and
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


PACKAGED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")


def source_tag() -> str:
    """Hash of the library's shape tables (every tile shape and sweep mode of
    both precisions, as the library reports them): a cached choice names a
    tile id, which means nothing in another table."""
    import hashlib
    h = hashlib.sha256()
    for prec in (cdugks.FP32, cdugks.FP64):
        for D in (1, 2, 3):
            for t in range(cdugks.load().cdugks_tile_count(prec, D)):
                h.update(repr((prec, D, t, cdugks.tile_shape(prec, D, t))).encode())
    return h.hexdigest()[:16]


def default_choice(cfg, precision):
    """Launch shape without tuning: a face-store shape of the default scheme
    with the most cells per tile that fits the problem, velocity groups chosen
    by the library (enough CTAs for a few waves).  Among them, as measured on
    the benchmark sizes: in FP64 the lean shapes (the FP64 exponentials of the
    equilibria become per-axis tables); in 3D FP32 the lean sweep A with the
    plain sweep B, then the full lean shape; in 1D / 2D FP32 the fused shapes."""
    D = cfg["dim"]
    best = None
    for t, _ in candidates(cfg, precision, "alone"):
        dims, mode = cdugks.tile_shape(precision, D, t)
        if not mode & 4:
            continue
        cells = int(np.prod(dims[:D]))
        if not mode & 128:
            lean = 0
        elif precision == cdugks.FP64:
            lean = 2
        elif D == 3:
            lean = 1 if mode & 256 else 2
        else:
            lean = -1
        pref = (lean, mode & 3 == 0, cells if cells <= wl.ncells(cfg) else -cells)
        if best is None or pref > best[0]:
            best = (pref, t)
    return (best[1] if best else 0), 0


def choose(cfg, precision, context="alone", device="cuda:0", allow_tuning=False):
    """The cached tuned shape (this machine's cache, then the one shipped
    beside the tuner) when it was tuned on the same shape table; else tune
    (allow_tuning) or take default_choice()."""
    key = size_key(cfg, precision, context)
    tag = source_tag()
    for path in (cache_path(), PACKAGED):
        d = _load_cache(path)
        if key in d and d[key].get("source") == tag:
            return tuple(d[key]["choice"])
    if allow_tuning:
        return tune(cfg, precision, context=context, device=device)
    return default_choice(cfg, precision)


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


def has_zero_node(cfg):
    """Some active axis of the velocity grid has a node at xi = 0."""
    for a in range(cfg["dim"]):
        n, lo, hi = cfg["nv"][a], cfg["vlo"][a], cfg["vhi"][a]
        if any(lo + (hi - lo) * k / (n - 1) == 0.0 for k in range(n)):
            return True
    return False


def candidates(cfg, precision, context="alone"):
    nt = cdugks.load().cdugks_tile_count(precision, cfg["dim"])
    nvt = (wl.nvel(cfg) + 3) // 4
    groups = [g for g in (1, 2, 4, 8, 16, 32) if g <= nvt]
    dirichlet = any(wl.BC_DIRICHLET in cfg["bc"][a] for a in range(cfg["dim"]))
    r2 = bool(cfg.get("recon", 0))
    sk = bool(cfg.get("collision", 0))
    ac = any(cfg.get("accel", (0.0, 0.0, 0.0)))
    tiles = []
    zero = has_zero_node(cfg)
    for t in range(nt):
        mode = cdugks.tile_shape(precision, cfg["dim"], t)[1]
        if mode & 128 and zero:
            continue                      # lean shapes need a velocity grid without a node at 0
        if bool(mode & 8) != r2 or bool(mode & 16) != sk or bool(mode & 32) != ac:
            continue                      # shapes of another reconstruction, collision or force compute another scheme
        if context != "alone" and mode & 3 != 0 and not mode & 32:
            continue                      # batched: the fused shapes and the acceleration shapes
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


def tune(cfg, precision, context="alone", steps=5, device="cuda:0", cache=None, refresh=False, tiles=None):
    """Best (tile_id, velocity_groups) for this instance size; cached.  tiles:
    consider only these tile ids (default: every candidate shape)."""
    path = cache or cache_path()
    d = _load_cache(path)
    key = size_key(cfg, precision, context)
    tag = source_tag()
    if key in d and not refresh and d[key].get("source") == tag:
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
        if tiles is None or tile in tiles:
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
    d[key] = {"choice": [best[1], best[2]], "ms_per_point": best[0], "source": tag,
              "tried": [[t, g, ms] for ms, t, g in results]}
    _save_cache(path, d)
    return best[1], best[2]


def bench_sizes():
    """(cfg, precision, context, tile ids or None) of every instance size the
    benchmark runs.  The full 3D workload is tuned over its face-store shapes
    only (each trial binds up to ~260 GB)."""
    c3 = wl.workload_c3(kn=1e-4)[0]
    nt3 = cdugks.load().cdugks_tile_count(cdugks.FP32, 3)
    c3_tiles = [t for t in range(nt3) if cdugks.tile_shape(cdugks.FP32, 3, t)[1] & 4
                and not cdugks.tile_shape(cdugks.FP32, 3, t)[1] & (16 | 32)]
    out = [(c3, cdugks.FP32, "alone", c3_tiles),
           (wl.workload_c3(kn=1e-4, scale=2, nv=12)[0], cdugks.FP32, "alone", None),
           (wl.workload_c2()[0], cdugks.FP32, "alone", None), (wl.workload_c2()[0], cdugks.FP64, "alone", None),
           (wl.workload_c1()[0], cdugks.FP64, "alone", None)]
    seen = set()
    for cfg, _ in wl.workload_c4():
        k = size_key(cfg, cdugks.FP32, "batch")
        if k not in seen:
            seen.add(k)
            out.append((cfg, cdugks.FP32, "batch", None))
    return out


if __name__ == "__main__":
    import sys
    dev = sys.argv[1] if len(sys.argv) > 1 else "cuda:0"
    for cfg, prec, ctx, tl in bench_sizes():
        print(size_key(cfg, prec, ctx), tune(cfg, prec, context=ctx, device=dev, refresh=True, tiles=tl), flush=True)
