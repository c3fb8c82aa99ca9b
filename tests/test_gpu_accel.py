"""GPU parity of the external-acceleration source terms against the oracle.

The same bars as the force-free path: FP64 relative L-infinity <= 1e-12 on
rho, u, T and on the distributions, FP32 storage <= 1e-5; D = 1, 2, 3,
ragged tiles, padded velocity tiles, periodic, specular (the force normal to
a wall) and Dirichlet boundaries, the collisionless limit."""
import numpy as np
import pytest

from paper_2208_09132_gb300 import cdugks, workloads as wl
from test_gpu_parity import case, rel_linf

pytestmark = pytest.mark.gpu

CASES = ["1d_periodic_ragged_padded", "1d_sod_dirichlet", "1d_sod_specular", "1d_boole_odd_grid",
         "1d_free_streaming", "2d_periodic_ragged", "2d_specular_x_periodic_y", "2d_dirichlet_x_specular_y",
         "3d_periodic_ragged", "3d_specular_corners", "3d_mixed_bc"]


def _acc(cfg):
    a = [0.6, -0.35, 0.25][:cfg["dim"]] + [0.0] * (3 - cfg["dim"])
    return dict(cfg, accel=a)


@pytest.mark.parametrize("precision,tol", [(cdugks.FP64, 1e-12), (cdugks.FP32, 1e-5)])
@pytest.mark.parametrize("name", CASES)
def test_acceleration_matches_oracle(oracle_mod, name, precision, tol):
    (cfg, f), steps = case(name)
    cfg = _acc(cfg)
    o = oracle_mod.Oracle(cfg)
    o.init(f)
    o.step(steps)
    s = cdugks.Solver(cfg, precision=precision)
    assert cdugks.tile_shape(precision, cfg["dim"], s.info().tile_id)[1] & 32
    assert s.dt == o.dt
    s.init(f)
    s.step(steps)
    assert s.sync_status() == 0
    err = rel_linf(s.moments(), o.moments())
    assert np.all(err <= tol), err
    g, b = s.distributions()
    go, bo = o.distributions()
    assert np.abs(g - go).max() <= tol * np.abs(go).max()
    assert np.abs(b - bo).max() <= tol * np.abs(bo).max()


@pytest.mark.parametrize("precision,tol", [(cdugks.FP64, 1e-12), (cdugks.FP32, 1e-5)])
def test_hydrostatic_atmosphere_matches_oracle(oracle_mod, precision, tol):
    """Gravity into a specular wall: the walls pass no mass on the GPU either."""
    a, RT = -1.0, 0.5
    cfg = wl._base(1, [96], [0], [1], [[wl.BC_SPECULAR] * 2], [48], [-8.0], [8.0], K=2.0, mu_ref=1e-3,
                   T_ref=1.0, omega=0.5, Pr=2.0 / 3.0, cfl=0.5)
    cfg["accel"] = [a, 0.0, 0.0]
    _, (x,) = wl.cell_centres(cfg)
    f = wl._fields(np.exp(a * x / RT), [np.zeros_like(x)], np.full_like(x, RT / 0.5))
    o = oracle_mod.Oracle(cfg)
    o.init(f)
    o.step(300)
    s = cdugks.Solver(cfg, precision=precision)
    s.init(f)
    m0 = s.conserved()[:, 0].sum()
    s.step(300)
    mg, mo = s.moments(), o.moments()
    assert np.all(rel_linf(mg[:, [0, 2]], mo[:, [0, 2]]) <= tol)
    # a gas at rest: its velocity's scale is the thermal speed, not the spurious flow
    assert np.abs(mg[:, 1] - mo[:, 1]).max() <= tol * np.sqrt(RT)
    assert abs(s.conserved()[:, 0].sum() - m0) <= (1e-13 if precision == cdugks.FP64 else 1e-6) * m0


@pytest.mark.parametrize("precision", [cdugks.FP64, cdugks.FP32])
def test_acceleration_checkpoint_and_graph_replay_are_bitwise(precision):
    import torch
    (cfg, f), _ = case("2d_periodic_ragged")
    cfg = _acc(cfg)
    a = cdugks.Solver(cfg, precision=precision)
    a.init(f)
    a.step(4)
    blob = a.get_state()
    a.step(6)
    b = cdugks.Solver(cfg, precision=precision, stream=torch.cuda.Stream())
    b.set_state(blob)
    b.capture(3)
    b.step(6)
    assert b.sync_status() == 0
    assert np.array_equal(a.moments(), b.moments())
    assert a.get_state() == b.get_state()
