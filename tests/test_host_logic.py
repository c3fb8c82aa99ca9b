"""Host-side logic that needs no GPU: tile-shape tables, tuner candidates,
design-byte accounting of the bench, and the serving step count."""
import math

import pytest

import numpy as np

from paper_2208_09132_gb300 import cdugks, serving, tune
from paper_2208_09132_gb300 import workloads as wl

import bench


def _modes(prec, dim):
    return [cdugks.tile_shape(prec, dim, t)[1] for t in range(cdugks.load().cdugks_tile_count(prec, dim))]


def test_every_dimension_has_a_fused_default_and_a_face_store_shape():
    for prec in (cdugks.FP32, cdugks.FP64):
        for dim in (1, 2, 3):
            modes = _modes(prec, dim)
            assert modes[0] == 0                       # tile 0: fused, batchable, no extra buffers
            assert any(m & 4 for m in modes), (prec, dim, modes)
            # the face-gradient reconstruction: fused face-store shapes, in 1D and 2D
            assert all(m == 12 for m in modes if m & 8)
            assert any(m & 8 for m in modes) == (dim < 3)


def test_find_tile_returns_the_matching_shape():
    t = cdugks.find_tile(cdugks.FP32, 2, (32, 8), 4)
    assert cdugks.tile_shape(cdugks.FP32, 2, t) == ((32, 8, 1), 4)
    assert cdugks.find_tile(cdugks.FP32, 2, (7, 7), 4) == 0


def test_tuner_candidates_respect_batching_and_boundaries():
    cfg, _ = wl.workload_c2()
    alone = tune.candidates(cfg, cdugks.FP32, "alone")
    batch = tune.candidates(cfg, cdugks.FP32, "batch")
    modes = _modes(cdugks.FP32, 2)
    # periodic: every shape of the default reconstruction and collision; batched: the fused ones
    assert {t for t, _ in alone} == {t for t, m in enumerate(modes) if not m & 56}
    assert {t for t, _ in batch} == {t for t, m in enumerate(modes) if m & 3 == 0 and not m & 56}
    r2 = tune.candidates(dict(cfg, recon=1), cdugks.FP32, "alone")
    assert r2 and all(modes[t] & 8 for t, _ in r2)                      # the face-gradient shapes only
    sk = tune.candidates(dict(cfg, collision=wl.COLLISION_SHAKHOV), cdugks.FP32, "alone")
    assert sk and all(modes[t] & 16 for t, _ in sk)                     # the Shakhov shapes only
    skb = tune.candidates(dict(cfg, collision=wl.COLLISION_SHAKHOV), cdugks.FP32, "batch")
    assert skb and all(modes[t] & 16 and modes[t] & 3 == 0 for t, _ in skb)   # batched: the fused Shakhov shapes
    ac = tune.candidates(dict(cfg, accel=[0.5, 0.0, 0.0]), cdugks.FP32, "alone")
    assert ac and all(modes[t] & 32 for t, _ in ac)                     # the acceleration shapes only
    acb = tune.candidates(dict(cfg, accel=[0.5, 0.0, 0.0]), cdugks.FP32, "batch")
    assert {t for t, _ in acb} == {t for t, _ in ac}                     # which batch too (with their pre-pass)
    assert all(g <= (wl.nvel(cfg) + 3) // 4 for _, g in alone)
    dcfg, _ = wl.random_smooth(dim=2, n=(8, 8), nv=(4, 4), seed=1, amp=0.1, kn=1e-2)
    dcfg = dict(dcfg, bc=[[wl.BC_DIRICHLET] * 2, [wl.BC_PERIODIC] * 2, [wl.BC_PERIODIC] * 2])
    ts = {t for t, _ in tune.candidates(dcfg, cdugks.FP32, "alone")}
    assert any(m & 3 == 2 for m in modes)                               # there are stored shapes ...
    assert ts and all(modes[t] & 3 != 2 for t in ts)                    # ... but not with Dirichlet walls


def test_size_key_buckets_by_powers_of_two():
    cfg, _ = wl.workload_c2()
    k = tune.size_key(cfg, cdugks.FP32, "alone")
    assert k == "fp32:alone:D2:cells~65536:nv1024"


def test_design_bytes_of_each_mode():
    # FP32, 2D: fused sweeps read phi* (8 B) / read and write it (16 B)
    assert bench.design_bytes(0, 2, 4) == {"sweep_a": 8, "sweep_b": 16}
    # face store: sweep A also writes D face values (2 fields), k_flux reads them
    assert bench.design_bytes(4, 2, 4) == {"sweep_a": 24, "sweep_b": 32}
    # stored slopes + face store, 3D: the pre-pass writes phibar+ and 3 slopes
    assert bench.design_bytes(6, 3, 4) == {"slopes": 40, "sweep_a": 56, "sweep_b": 40}
    assert bench.design_bytes(1, 1, 8) == {"prep": 32, "sweep_a": 16, "sweep_b": 48}


def test_served_step_count_reaches_the_end_time():
    assert serving.steps_to(0.1, 1.0) == 10
    assert serving.steps_to(0.3, 1.0) == 4
    assert serving.steps_to(0.5, 1e-9) == 1
    assert math.isclose(serving.steps_to(1e-3, 0.05) * 1e-3, 0.05)


def test_sine_wave_reaches_its_end_time_within_the_cfl_bound():
    for nx in (64, 100, 1024):
        cfg, f = wl.sine_wave(nx=nx, nv=65, T0=1.0, t_end=0.1)
        dt_cfl = cfg["cfl"] * (1.0 / nx) / (2.0 * 6.0)
        assert cfg["dt"] <= dt_cfl * (1 + 1e-12)
        assert math.isclose(cfg["dt"] * cfg["steps"], 0.1, rel_tol=1e-12)
        assert cfg["rule"] == wl.RULE_BOOLE and (cfg["nv"][0] - 1) % 4 == 0
        # rho0 = 1, v = sin(2 pi x), T = T0 (c_v = (3 + K) R / 2 = 1 with K = 2, R = 1/2)
        _, (x,) = wl.cell_centres(cfg)
        assert (f[:, 0] == 1.0).all() and (f[:, 2] == 1.0).all()
        assert abs(f[:, 1] - np.sin(2 * np.pi * x)).max() < 1e-15


def _upwind_cell(l, T, D, rext):
    """Slope-box cell l (tile-local) is upwind of a face the tile forms; the
    rule sweep A uses to skip unread cells of shapes that load phibar+."""
    out, ok = 0, True
    for b in range(D):
        if l[b] < -1 or l[b] > T[b]:
            ok = False
        elif l[b] == -1:
            out += 1
        elif l[b] == T[b]:
            out += 1
            ok = ok and rext[b]
    return ok and out <= 1


def _needed_box_cell(l, T, D, rext):
    if _upwind_cell(l, T, D, rext):
        return True
    for b in range(D):
        for d in (-1, 1):
            m = list(l)
            m[b] += d
            if _upwind_cell(m, T, D, rext):
                return True
    return False


@pytest.mark.parametrize("D,T", [(1, (256,)), (2, (32, 8)), (2, (16, 8)), (3, (8, 4, 4)), (3, (8, 8, 4))])
def test_pruned_halo_covers_every_read_of_the_faces(D, T):
    """Every cell a face of the tile reads (both candidate upwind cells of each
    face formed, their phibar+ and the neighbours their slopes use) is in the
    set the sweeps keep, for interior, edge and ragged tiles, sweeps A and B."""
    import itertools
    import random
    rng = random.Random(1)
    T3 = list(T) + [1] * (3 - D)
    for _ in range(12):
        n = [rng.randint(1, 3 * T3[a] + 5) if a < D else 1 for a in range(3)]
        org = [rng.randint(0, (n[a] - 1) // T3[a]) * T3[a] if a < D else 0 for a in range(3)]
        for sweep_b in (False, True):
            rext = [sweep_b or org[a] + T3[a] >= n[a] for a in range(3)]
            ups = set()
            for la in itertools.product(*[range(T3[b]) for b in range(3)]):
                qa = [org[b] + la[b] for b in range(3)]
                if any(qa[b] >= n[b] for b in range(D)):
                    continue
                for a in range(D):
                    own_right = qa[a] == n[a] - 1
                    right = (la[a] == T3[a] - 1 or own_right) if sweep_b else own_right
                    for side in ([0, 1] if right else [0]):
                        left = list(la)
                        left[a] += side - 1
                        rgt = list(left)
                        rgt[a] += 1
                        ups.update([tuple(left), tuple(rgt)])
            assert all(_upwind_cell(u, T3, D, rext) for u in ups)
            for u in ups:
                for b in range(D):
                    for d in (-1, 1):
                        m = list(u)
                        m[b] += d
                        assert _needed_box_cell(m, T3, D, rext), (D, T, n, org, sweep_b, m)


def test_issue_roofline_of_a_sweep():
    """196 thread instructions per point over 67.1 M points in 0.617 ms on 152
    SMs at 2070 MHz: 21.3 T/s of a 40.3 T/s ceiling."""
    r = bench.issue_roofline(195.8, 67108864, 0.617e-3, 152, 2070.0)
    assert r["peak"] == pytest.approx(40.27, abs=0.01)
    assert r["achieved"] == pytest.approx(21.30, abs=0.01)
    assert r["frac"] == pytest.approx(0.529, abs=0.001)


def test_one_at_a_time_server_model():
    """The modelled one-at-a-time servers of the served-stream bench: a long
    solve at t = 0, then a medium and a short one; FIFO keeps arrival order,
    shortest-first takes the short one first when the server frees up, and the
    cap counts only what finishes by then."""
    import types

    import bench

    R = lambda a, n, p: types.SimpleNamespace(arrival=a, nsteps=n, points=p)
    reqs = [R(0.0, 100, 10), R(0.1, 10, 10), R(0.2, 1, 10)]
    fifo = bench.one_at_a_time(reqs, [10.0] * 3, 100.0, "fifo")
    sjf = bench.one_at_a_time(reqs, [10.0] * 3, 100.0, "sjf")
    # fifo: 0 -> 1.0, 1.0 -> 1.1, 1.1 -> 1.11 (times to solution 1.0, 1.0, 0.91);
    # sjf: 0 -> 1.0, 1.0 -> 1.01 (the short one), 1.01 -> 1.11 (1.0, 0.81, 1.01)
    assert fifo["finished"] == sjf["finished"] == 3
    assert fifo["p99_time_to_solution_s"] == pytest.approx(1.0, abs=1e-9)
    assert sjf["p99_time_to_solution_s"] == pytest.approx(float(np.percentile([1.0, 0.81, 1.01], 99)), abs=1e-9)
    assert fifo["aggregate_point_updates_per_s"] == pytest.approx(1110 / 1.11)
    capped = bench.one_at_a_time(reqs, [10.0] * 3, 0.5, "fifo")
    assert capped["finished"] == 0 and capped["aggregate_point_updates_per_s"] == pytest.approx(1000.0)


def test_default_choice_follows_the_measured_preferences():
    """Without a cached tuning the launch shape is a face-store shape: in 3D FP32
    the lean sweep A with the plain sweep B, in 1D / 2D FP32 a fused shape (no
    lean), in FP64 2D the lean pair; grids with a node at xi = 0 take no lean
    shape."""
    modes3 = _modes(cdugks.FP32, 3)
    modes2 = _modes(cdugks.FP32, 2)
    modes2d = _modes(cdugks.FP64, 2)
    cfg3, _ = wl.shear3d(n=16, nv=12, kn=1e-2)
    t, g = tune.default_choice(cfg3, cdugks.FP32)
    assert modes3[t] & 128 and not modes3[t] & 256 and g == 0
    cfg2, _ = wl.kelvin_helmholtz(n=128, nv=16, kn=1e-3)
    t2, _ = tune.default_choice(cfg2, cdugks.FP32)
    assert modes2[t2] & 4 and not modes2[t2] & 128 and modes2[t2] & 3 == 0
    t64, _ = tune.default_choice(cfg2, cdugks.FP64)
    assert modes2d[t64] & 128
    odd, _ = wl.kelvin_helmholtz(n=64, nv=15, kn=1e-3)       # 15 nodes on [-6, 6]: a node at 0
    assert tune.has_zero_node(odd)
    t0, _ = tune.default_choice(odd, cdugks.FP64)
    assert not modes2d[t0] & 128
