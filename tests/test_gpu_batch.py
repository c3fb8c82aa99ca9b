"""Batched stepping: many uneven instances in one launch per kernel.

A member stepped inside a batch runs the same kernel body on the same work
items as when stepped alone, so the results must be identical bit for bit,
with or without CUDA-graph replay, whatever else is in the batch."""
import numpy as np
import pytest

from paper_2208_09132_gb300 import cdugks, workloads as wl

pytestmark = pytest.mark.gpu


def _members_1d(seed=0, count=6):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nx = int(rng.integers(40, 700))
        nv = int(rng.choice([8, 16, 24, 32]))
        kn = 10.0 ** rng.uniform(-4, 0)
        Pr = float(rng.choice([0.5, 2.0 / 3.0, 1.0, 2.0]))
        out.append(wl.thermoacoustic(nx=nx, nv=nv, kn=kn, Pr=Pr, delta=0.05))
    return out


def _batchable(prec, D):
    """Tile shapes with a batched step: the fused shapes (either collision
    model and reconstruction) and the acceleration shapes."""
    out = []
    for t in range(cdugks.load().cdugks_tile_count(prec, D)):
        mode = cdugks.tile_shape(prec, D, t)[1]
        if mode & 3 == 0 or mode & 32:
            out.append(t)
    return out


def _physics(cfg, prec, D, t):
    """The problem with the physics the tile shape implements."""
    mode = cdugks.tile_shape(prec, D, t)[1]
    acc = [0.4, -0.25, 0.15][:D] + [0.0] * (3 - D)
    return dict(cfg, recon=1 if mode & 8 else 0, collision=1 if mode & 16 else 0,
                accel=acc if mode & 32 else [0.0, 0.0, 0.0])


def _solo(cfg, f, prec, steps, tile=0, groups=0):
    s = cdugks.Solver(cfg, precision=prec, tile_id=tile, velocity_groups=groups)
    s.init(f)
    s.step(steps)
    return s.moments()


@pytest.mark.parametrize("prec", [cdugks.FP32, cdugks.FP64])
@pytest.mark.parametrize("graph", [0, 3])
def test_batch_equals_members_alone(prec, graph):
    steps = 7
    batched = _batchable(prec, 1)[:8]
    members = _members_1d(count=max(6, len(batched)))
    tiles = [batched[k % len(batched)] for k in range(len(members))]
    # every batchable shape, each member with the physics of its shape
    probs = [(_physics(cfg, prec, 1, t), f) for (cfg, f), t in zip(members, tiles)]
    solvers = []
    for (cfg, f), t in zip(probs, tiles):
        s = cdugks.Solver(cfg, precision=prec, tile_id=t)
        s.init(f)
        solvers.append(s)
    b = cdugks.Batch(solvers)
    if graph:
        b.capture(graph)
    b.step(steps)
    assert b.sync() == 0
    for (cfg, f), t, s in zip(probs, tiles, solvers):
        ref = _solo(cfg, f, prec, steps, tile=t)
        assert np.array_equal(s.moments(), ref)
        assert s.info().steps == steps


@pytest.mark.parametrize("prec", [cdugks.FP32, cdugks.FP64])
@pytest.mark.parametrize("D", [2, 3])
def test_batch_mixes_collision_models_and_acceleration(prec, D):
    """One member per batchable shape of the dimension (two-time and Shakhov
    collision models, the face-gradient reconstruction, the acceleration, the
    lean shapes), stepped together in one batch and replayed from a graph:
    each equals stepping it alone."""
    tiles = _batchable(prec, D)[:8]
    probs = []
    for k, t in enumerate(tiles):
        if D == 2:
            cfg, f = wl.random_smooth(dim=2, n=(21 + 3 * k, 13 + k), nv=(10, 8), seed=40 + k, amp=0.3, kn=4e-3,
                                      Pr=2.0 / 3.0)
        else:
            cfg, f = wl.random_smooth(dim=3, n=(9 + k, 7, 6), nv=(6, 6, 6), seed=60 + k, amp=0.3, kn=4e-3,
                                      Pr=2.0 / 3.0)
        probs.append((_physics(cfg, prec, D, t), f))
    solvers = []
    for (cfg, f), t in zip(probs, tiles):
        s = cdugks.Solver(cfg, precision=prec, tile_id=t)
        s.init(f)
        solvers.append(s)
    b = cdugks.Batch(solvers)
    b.capture(2)
    b.step(5)
    assert b.sync() == 0
    modes = set()
    for (cfg, f), t, s in zip(probs, tiles, solvers):
        modes.add(cdugks.tile_shape(prec, D, t)[1])
        assert np.array_equal(s.moments(), _solo(cfg, f, prec, 5, tile=t)), (t, cfg.get("collision"), cfg["accel"])
    assert any(m & 32 for m in modes)                  # an acceleration member took part
    if D == 2:
        assert any(m & 16 for m in modes)              # and a Shakhov member


def test_batch_2d_members_and_uneven_steps():
    a = wl.random_smooth(dim=2, n=(19, 13), nv=(8, 6), seed=5, amp=0.3, kn=5e-3)
    c = wl.kelvin_helmholtz(n=24, nv=8, kn=1e-3)
    sa = cdugks.Solver(a[0], precision=cdugks.FP32)
    sa.init(a[1])
    sa.step(3)                        # members may start at different step counts
    sc = cdugks.Solver(c[0], precision=cdugks.FP32, tile_id=1)
    sc.init(c[1])
    b = cdugks.Batch([sa, sc])
    b.capture(2)
    b.step(5)
    assert b.sync() == 0
    assert np.array_equal(sa.moments(), _solo(a[0], a[1], cdugks.FP32, 8))
    assert np.array_equal(sc.moments(), _solo(c[0], c[1], cdugks.FP32, 5, tile=1))


def test_tile_shapes_agree_with_the_oracle(oracle_mod):
    cfg, f = wl.random_smooth(dim=1, n=(300,), nv=(16,), seed=3, amp=0.3, kn=3e-3)
    for t in range(cdugks.load().cdugks_tile_count(cdugks.FP64, 1)):
        mode = cdugks.tile_shape(cdugks.FP64, 1, t)[1]
        c = dict(cfg, recon=1 if mode & 8 else 0, collision=1 if mode & 16 else 0,
                 accel=[0.4, 0.0, 0.0] if mode & 32 else [0.0, 0.0, 0.0])
        o = oracle_mod.Oracle(c)
        o.init(f)
        o.step(20)
        ref = o.moments()
        got = _solo(c, f, cdugks.FP64, 20, tile=t, groups=2)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("graph", [0, 2])
def test_admit_and_retire_between_steps(graph):
    """Continuous batching: membership changes between steps leave every
    member's trajectory identical to stepping it alone."""
    probs = _members_1d(seed=9, count=4)
    prec = cdugks.FP32
    solvers = []
    for cfg, f in probs:
        s = cdugks.Solver(cfg, precision=prec)
        s.init(f)
        solvers.append(s)
    s0, s1, s2, s3 = solvers
    b = cdugks.Batch([s0, s1])
    if graph:
        b.capture(graph)
    b.step(4)                          # s0, s1: 4
    b.admit(s2)
    if graph:
        b.capture(graph)
    b.step(3)                          # s0, s1: 7; s2: 3
    b.retire(s0)
    b.admit(s3)
    b.step(5)                          # s1: 12; s2: 8; s3: 5
    assert b.sync() == 0
    s0.step(2)                         # a retired member steps alone: 9
    with pytest.raises(cdugks.CdugksError):
        b.retire(s0)                   # not a member any more
    with pytest.raises(cdugks.CdugksError):
        b.admit(s1)                    # already a member
    for (cfg, f), s, n in zip(probs, solvers, (9, 12, 8, 5)):
        assert s.info().steps == n
        assert np.array_equal(s.moments(), _solo(cfg, f, prec, n))
    b.retire(s1)
    b.retire(s2)
    with pytest.raises(cdugks.CdugksError):
        b.retire(s3)                   # a batch keeps one member
