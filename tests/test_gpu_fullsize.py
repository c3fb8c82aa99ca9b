"""Parity at the benchmark sizes, in the launch configuration bench.py times.

The oracle cannot run the full 2D and 3D workloads, but one step of one cell
depends only on the cells within two of it (its faces need the slopes of their
upwind neighbours, which need one more neighbour).  For sampled cells the test
copies a periodic patch of 7 cells per axis around the cell from the GPU state
at step n into the oracle, advances the oracle one step, and compares the
centre cell's W and distributions with the GPU's step n+1.  At full size it
also checks conservation and the device status over the steps taken.
"""
import numpy as np
import pytest

from paper_2208_09132_gb300 import cdugks, tune, workloads as wl

pytestmark = pytest.mark.gpu
R = 3


def _patch(cfg, centre):
    D = cfg["dim"]
    n = cfg["n"]
    q = [centre % n[0], (centre // n[0]) % n[1], centre // (n[0] * n[1])]
    rng = [range(-R, R + 1) if a < D else range(1) for a in range(3)]
    cells = []
    for dz in rng[2]:
        for dy in rng[1]:
            for dx in rng[0]:
                x, y, z = (q[0] + dx) % n[0], (q[1] + dy) % n[1], (q[2] + dz) % n[2]
                cells.append(x + n[0] * (y + n[1] * z))
    return np.array(cells, dtype=np.int64)


def _check(oracle_mod, cfg, f, steps_before, nsamples, tile, groups, tol_W, tol_phi):
    D, NM = cfg["dim"], 2 + cfg["dim"]
    s = cdugks.Solver(cfg, precision=cdugks.FP32, tile_id=tile, velocity_groups=groups)
    s.init(f)
    S0 = s.conserved().sum(0)
    s.step(steps_before)
    rng = np.random.default_rng(7)
    centres = rng.integers(0, s.Nc, nsamples)
    patches = [_patch(cfg, int(c)) for c in centres]
    allc = np.unique(np.concatenate(patches))
    g_n, b_n = s.cell_distributions(allc)
    W_n = s.conserved()
    s.step(1)
    assert s.sync_status() == 0
    g1, b1 = s.cell_distributions(centres)
    W1 = s.conserved()
    # conservation over the steps taken (periodic)
    S1 = W1.sum(0)
    scale = np.array([S0[0]] * (1 + D) + [S0[-1]])
    assert np.all(np.abs(S1 - S0) <= 1e-6 * scale), (S1 - S0) / scale
    pos = {int(c): i for i, c in enumerate(allc)}
    centre_local = R + (2 * R + 1) * (R if D >= 2 else 0) + (2 * R + 1) ** 2 * (R if D >= 3 else 0)
    for k, c in enumerate(centres):
        sub = {key: (list(v) if isinstance(v, list) else v) for key, v in cfg.items()}
        sub["n"] = [2 * R + 1 if a < D else 1 for a in range(3)]
        sub["lo"] = [0.0, 0.0, 0.0]
        sub["hi"] = [(2 * R + 1) * (cfg["hi"][a] - cfg["lo"][a]) / cfg["n"][a] if a < D else 1.0 for a in range(3)]
        sub["bc"] = [[wl.BC_PERIODIC] * 2 for _ in range(3)]
        sub["dt"] = s.dt
        o = oracle_mod.Oracle(sub)
        idx = [pos[int(cc)] for cc in patches[k]]
        Wp = W_n[patches[k]]
        fields = np.zeros((len(idx), NM))
        fields[:, 0] = 1.0
        fields[:, -1] = 1.0
        o.init(fields)
        o.set_state(g_n[idx], b_n[idx], Wp)
        o.step(1)
        Wo = o.conserved()[centre_local]
        go, bo = o.distributions()
        Wscale = np.abs(W_n).max(axis=0)
        Wscale[1:1 + D] = Wscale[1:1 + D].max()
        assert np.all(np.abs(W1[c] - Wo) <= tol_W * Wscale), (k, W1[c], Wo)
        assert np.abs(g1[k] - go[centre_local]).max() <= tol_phi * np.abs(go).max()
        assert np.abs(b1[k] - bo[centre_local]).max() <= tol_phi * np.abs(bo).max()


def test_kelvin_helmholtz_full_size(oracle_mod):
    """256^2 cells x 32^2 velocities, FP32, the launch shape the bench times."""
    cfg, f = wl.workload_c2()
    tile, groups = tune.choose(cfg, cdugks.FP32, context="alone")      # the shape bench.py times
    _check(oracle_mod, cfg, f, steps_before=5, nsamples=4, tile=tile, groups=groups, tol_W=1e-5, tol_phi=1e-5)


def test_shear_3d_full_size(oracle_mod):
    """64^3 cells x 24^3 velocities, FP32 (about 29 GB per state buffer), the launch shape the bench
    times (the lean sweep A with the plain sweep B)."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    cfg, f = wl.workload_c3(kn=1e-2)
    if free < 120e9:
        pytest.skip("needs about 120 GB of free device memory")
    tile, groups = tune.choose(cfg, cdugks.FP32, context="alone")      # the shape bench.py times
    _check(oracle_mod, cfg, f, steps_before=2, nsamples=2, tile=tile, groups=groups, tol_W=1e-5, tol_phi=1e-5)


def test_batched_thermoacoustic_full_size(oracle_mod):
    """All 256 members of the batched workload in the launch configuration the
    bench times (the persistent batched step, 1D face-store tiles of 128 cells,
    one velocity group, a CUDA graph of 10 steps), 20 steps, every member
    against the oracle: relative L-infinity <= 1e-5 on rho and T, and on u
    relative to the thermal speed (the gas is at rest up to a conduction-driven
    flow ~1e-6 of it)."""
    import math

    probs = wl.workload_c4()
    tile = cdugks.find_tile(cdugks.FP32, 1, (128,), 4)
    members = []
    for cfg, f in probs:
        s = cdugks.Solver(cfg, precision=cdugks.FP32, tile_id=tile, velocity_groups=1)
        s.init(f)
        members.append(s)
    b = cdugks.Batch(members, persistent=True)
    b.capture(10)
    b.step(20)
    assert b.sync() == 0
    worst = np.zeros(3)
    for (cfg, f), s in zip(probs, members):
        o = oracle_mod.Oracle(cfg)
        o.init(f)
        o.step(20)
        got, ref = s.moments(), o.moments()
        err = np.abs(got - ref).max(axis=0) / np.abs(ref).max(axis=0)
        err[1] = np.abs(got[:, 1] - ref[:, 1]).max() / math.sqrt(cfg["R"] * cfg["T_ref"])
        worst = np.maximum(worst, err)
        assert np.all(err <= 1e-5), (cfg["name"], err)
    print(f"\n[fullsize] batched thermoacoustic, 256 members, 20 steps: worst rel Linf rho,u,T = "
          f"{', '.join(f'{e:.1e}' for e in worst)}")


def test_served_requests_full_size(oracle_mod):
    """The first three requests of the served stream at their stated sizes (86^2 x
    45^2, 150^2 x 29^2, 127^2 x 38^2, Gresho / Kelvin-Helmholtz, Kn from the
    stream), served together in the server's launch configuration, each to five
    of its steps, against the oracle (relative L-infinity <= 1e-5)."""
    from paper_2208_09132_gb300 import serving

    reqs = serving.stream_c5(count=3)
    for q in reqs:
        s = cdugks.Solver(q.cfg, precision=q.precision)     # its time step, through the library
        q.t_end = 5 * s.dt                                  # five steps
        q.arrival = 0.0
        del s
    srv = serving.Server(budget_bytes=32 << 30, max_round=2)
    done = srv.run(reqs)
    assert len(done) == 3
    for q in done:
        assert q.nsteps == 5 and q.done_steps == 5
        o = oracle_mod.Oracle(q.cfg)
        o.init(q.fields)
        o.step(5)
        ref = o.moments()
        den = np.abs(ref).max(axis=0)
        den[1:-1] = den[1:-1].max()
        err = np.abs(q.result - ref).max(axis=0) / den
        assert np.all(err <= 1e-5), (q.cfg["name"], err)
