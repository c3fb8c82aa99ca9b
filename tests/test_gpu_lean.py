"""The lean face-store shapes (separable Maxwellian factors formed in double,
stencil work on the cells the faces read, each face's value and flux formed
once) against the FP64 oracle.

They compute the scheme of the default shapes (two relaxation times,
upwind-cell reconstruction) on velocity grids without a node at 0, so they
must match the oracle to the FP32 target (relative L-infinity <= 1e-5 on rho,
u, T and on every distribution value, against the largest value) on every
boundary kind and corner, ragged tiles, several tiles per axis, velocity grids
whose first axis is (and is not) a whole number of four-velocity chunks, with
and without the b-source (Pr != 1, Pr = 1).  Their equilibria are products of
factors exp(-(xi_b - u_b)^2 / 2RT) formed in double: every value of the
initial Maxwellian must be within a few FP32 roundings of the oracle's, even
on wide grids at high Mach number where an FP32 exponent loses digits in
proportion to c^2 / 2RT.
"""
import numpy as np
import pytest

from paper_2208_09132_gb300 import cdugks, workloads as wl
from paper_2208_09132_gb300.tune import has_zero_node
from test_gpu_parity import case, rel_linf, _bc

pytestmark = pytest.mark.gpu

P, S, DI = wl.BC_PERIODIC, wl.BC_SPECULAR, wl.BC_DIRICHLET
TOL = 1e-5


def lean_tiles(precision, D):
    nt = cdugks.load().cdugks_tile_count(precision, D)
    return [t for t in range(nt) if cdugks.tile_shape(precision, D, t)[1] & 128]


def lean_cases():
    names = ["2d_periodic_ragged", "2d_specular_x_periodic_y", "2d_dirichlet_x_specular_y", "2d_kh_small",
             "3d_periodic_ragged", "3d_specular_corners", "3d_mixed_bc", "3d_shear_small"]
    for n in names:
        (cfg, f), steps = case(n)
        yield n, cfg, f, steps
    # several tiles per axis, interior and edge tiles, walls on one axis
    cfg, f = wl.random_smooth(dim=2, n=(100, 44), nv=(8, 6), seed=31, amp=0.3, kn=3e-3)
    yield "2d_interior_tiles", _bc(cfg, [(P, P), (S, S)]), f, 8
    cfg, f = wl.random_smooth(dim=3, n=(20, 18, 11), nv=(8, 6, 4), seed=32, amp=0.3, kn=3e-3)
    yield "3d_interior_tiles", _bc(cfg, [(P, P), (S, S), (DI, DI)]), f, 4
    cfg, f = wl.random_smooth(dim=3, n=(17, 9, 9), nv=(10, 4, 6), seed=33, amp=0.3, kn=3e-3)
    yield "3d_unaligned_grid", cfg, f, 4


@pytest.mark.parametrize("Pr", [2.0 / 3.0, 1.0])
@pytest.mark.parametrize("name,cfg,f,steps", list(lean_cases()), ids=[c[0] for c in lean_cases()])
def test_lean_shapes_match_oracle(oracle_mod, name, cfg, f, steps, Pr):
    cfg = dict(cfg, Pr=Pr)
    assert not has_zero_node(cfg)
    o = oracle_mod.Oracle(cfg)
    o.init(f)
    o.step(steps)
    ref = o.moments()
    go, bo = o.distributions()
    tiles = lean_tiles(cdugks.FP32, cfg["dim"])
    assert tiles
    for t in tiles:
        s = cdugks.Solver(cfg, precision=cdugks.FP32, tile_id=t, velocity_groups=3)
        s.init(f)
        s.step(steps)
        assert s.sync_status() == 0
        err = rel_linf(s.moments(), ref)
        assert np.all(err <= TOL), (name, t, err)
        g, b = s.distributions()
        assert np.abs(g - go).max() <= TOL * np.abs(go).max(), (name, t)
        assert np.abs(b - bo).max() <= TOL * np.abs(bo).max(), (name, t)


@pytest.mark.parametrize("name,cfg,f,steps", [c for c in lean_cases() if c[1]["dim"] == 2],
                         ids=[c[0] for c in lean_cases() if c[1]["dim"] == 2])
def test_lean_fp64_shapes_match_oracle(oracle_mod, name, cfg, f, steps):
    """The FP64 lean shapes (2D): the same scheme to 1e-12, every value."""
    o = oracle_mod.Oracle(cfg)
    o.init(f)
    o.step(steps)
    ref = o.moments()
    go, bo = o.distributions()
    tiles = lean_tiles(cdugks.FP64, 2)
    assert tiles
    for t in tiles:
        s = cdugks.Solver(cfg, precision=cdugks.FP64, tile_id=t, velocity_groups=3)
        s.init(f)
        s.step(steps)
        assert s.sync_status() == 0
        assert np.all(rel_linf(s.moments(), ref) <= 1e-12), (name, t)
        g, b = s.distributions()
        assert np.abs(g - go).max() <= 1e-12 * np.abs(go).max(), (name, t)
        assert np.abs(b - bo).max() <= 1e-12 * np.abs(bo).max(), (name, t)


@pytest.mark.parametrize("D", [2, 3])
def test_lean_uniform_maxwellian_is_a_fixed_point(D):
    """Every cell computes the same values from the same factors: a uniform
    drifting Maxwellian stays uniform bit for bit (every cell's distributions
    and conserved variables equal cell 0's) where both sweeps take the
    equilibria from the factor tables, its conserved variables do not change
    at all (within 1e-8 where sweep B is k_flux), and its
    distributions move only by the FP32 rounding of the relaxation factors
    (fa + fb = 1 only to rounding), within 1e-6 of the largest value."""
    cfg, f = wl.uniform(dim=D, n=(9, 7, 5), nv=(12, 8, 6), u=(0.3, -0.2, 0.1), T=1.1)
    for t in lean_tiles(cdugks.FP32, D):
        s = cdugks.Solver(cfg, precision=cdugks.FP32, tile_id=t)
        s.init(f)
        g0, b0 = s.distributions()
        W0 = s.conserved()
        s.step(20)
        g1, b1 = s.distributions()
        W1 = s.conserved()
        print(f"\n[lean fixed point] D={D} tile {t}: max |W1 - W0| / |W0| = "
              f"{(np.abs(W1 - W0).max(0) / np.abs(W0).max(0)).max():.2e}")
        if cdugks.tile_shape(cdugks.FP32, D, t)[1] & 256:      # sweep B from the face factor tables too
            assert np.all(W1 == W1[0])
            assert np.array_equal(W1, W0)
            assert np.all(g1 == g1[0]) and np.all(b1 == b1[0])
        else:
            # sweep B is k_flux: like the fused face-store shapes, it leaves the
            # uniform state uniform only to FP32 rounding of the fluxes (1e-9)
            assert np.all(np.abs(W1 - W0).max(0) <= 1e-8 * np.abs(W0).max(0))
        assert np.abs(g1 - g0).max() <= 1e-6 * g0.max()
        assert np.abs(b1 - b0).max() <= 1e-6 * b0.max()


def test_lean_batch_equals_members_alone():
    """2D members of different sizes, velocity grids and Pr (1 and not) in one
    batch, replayed from a graph, give the results of stepping each alone."""
    probs = [wl.random_smooth(dim=2, n=(40, 24), nv=(8, 6), seed=41, amp=0.3, kn=3e-3, Pr=1.0),
             wl.kelvin_helmholtz(n=48, nv=12, kn=1e-3),
             wl.random_smooth(dim=2, n=(19, 13), nv=(10, 4), seed=42, amp=0.3, kn=5e-3)]
    t = lean_tiles(cdugks.FP32, 2)[0]
    solvers = []
    for cfg, f in probs:
        s = cdugks.Solver(cfg, precision=cdugks.FP32, tile_id=t)
        s.init(f)
        solvers.append(s)
    b = cdugks.Batch(solvers)
    b.capture(3)
    b.step(7)
    assert b.sync() == 0
    for (cfg, f), s in zip(probs, solvers):
        a = cdugks.Solver(cfg, precision=cdugks.FP32, tile_id=t)
        a.init(f)
        a.step(7)
        assert np.array_equal(s.moments(), a.moments())


def test_lean_initial_maxwellian_at_high_mach(oracle_mod):
    """A Mach-3 flow on a wide velocity grid: the lean shapes' initial
    distributions (products of factors formed in double, each rounded once to
    FP32) match the oracle's Maxwellian value by value to a few FP32 roundings,
    relative to each value, down to 1e-30 of the largest."""
    cfg, f = wl.kelvin_helmholtz(n=16, nv=40, kn=1e-3, vmax=14.0)
    f = f.copy()
    f[:, 1] += 3.5
    f[:, 2] += 1.0
    o = oracle_mod.Oracle(cfg)
    o.init(f)
    go, bo = o.distributions()
    mask = np.abs(go) > 1e-30 * np.abs(go).max()
    for t in lean_tiles(cdugks.FP32, 2):
        s = cdugks.Solver(cfg, precision=cdugks.FP32, tile_id=t)
        s.init(f)
        g, _ = s.distributions()
        rel = np.abs(g[mask] - go[mask]) / np.abs(go[mask])
        assert rel.max() <= 5e-7, rel.max()
