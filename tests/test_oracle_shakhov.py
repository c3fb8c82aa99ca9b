"""Pins of the oracle's Shakhov S-model collision (collision = 1).

The paper reaches Pr != 1 with two relaxation times and a b-source; it names
the Shakhov model as the other route without giving its form.  The oracle
takes the S-model from the kinetic-theory literature (Shakhov 1968) for the
reduced distributions g, b.  These tests fix it by what the model is built
to satisfy, not by re-typing its formulas:

  reduced equilibrium      g_S, b_S equal the integrals over the unresolved
                           components of the full S-model distribution
                           (brute-force radial quadrature)
  moments                  g_S, b_S keep rho, rho u, rho E and P = p I of the
                           Maxwellian and carry the heat flux (1 - Pr) q
  Pr = 1                   the Shakhov scheme is the BGK scheme, bit for bit
  heat-flux bookkeeping    the heat flux each equilibrium uses equals the heat
                           flux of the distributions it belongs to
  walls                    specular walls equal the mirror image on a doubled
                           periodic domain (the heat flux mirrors too)
The Navier-Stokes limits (sound damping, isobaric conduction at chi = mu/(rho
Pr), Galilean invariance) are shared with the default model in
test_oracle_pins.py.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from paper_2208_09132_gb300 import workloads as wl

R = 0.5
SHAKHOV = wl.COLLISION_SHAKHOV


def _full_shakhov_reduced(xi, rho, u, T, q, Pr, D, K):
    """g and b at velocity xi from the S-model distribution of all N = 3 + K
    degrees of freedom, f_S = f_M [1 + (1 - Pr) c.q/((N+2) p RT) ((c^2 + eta^2)/RT - (N+2))],
    integrated over the L = 3 - D + K unresolved ones by radial quadrature."""
    RT = R * T
    N = 3 + K
    L = int(round(3 - D + K))
    c = np.asarray(xi[:D]) - np.asarray(u[:D])
    c2 = float(c @ c)
    cq = float(c @ np.asarray(q[:D]))
    xi2 = float(np.asarray(xi[:D]) @ np.asarray(xi[:D]))
    p = rho * RT

    def f(e2):   # full distribution at |eta|^2 = e2
        fm = rho / (2 * math.pi * RT) ** ((D + L) / 2) * math.exp(-(c2 + e2) / (2 * RT))
        return fm * (1 + (1 - Pr) * cq / ((N + 2) * p * RT) * ((c2 + e2) / RT - (N + 2)))

    if L == 0:
        return f(0.0), 0.5 * xi2 * f(0.0)
    area = 2 * math.pi ** (L / 2) / special.gamma(L / 2)      # surface of the unit sphere in R^L
    top = 12 * math.sqrt(RT)
    g = area * integrate.quad(lambda r: r ** (L - 1) * f(r * r), 0, top, epsabs=0, epsrel=1e-13, limit=200)[0]
    b = area * integrate.quad(lambda r: r ** (L - 1) * 0.5 * (xi2 + r * r) * f(r * r), 0, top,
                              epsabs=0, epsrel=1e-13, limit=200)[0]
    return g, b


@pytest.mark.parametrize("D", [1, 2, 3])
@pytest.mark.parametrize("K", [0.0, 2.0])
def test_reduced_equilibrium_is_the_integral_of_the_full_model(oracle_mod, D, K):
    cfg, _ = wl.uniform(dim=D, n=(2, 2, 2), nv=(9, 7, 5), vmax=4.0, K=K, Pr=2.0 / 3.0)
    cfg["collision"] = SHAKHOV
    o = oracle_mod.Oracle(cfg)
    xi, _ = o.velocities()
    rho, T = 1.3, 1.7
    u = np.array([0.4, -0.3, 0.2])
    q = np.array([0.35, -0.2, 0.15])
    ge, be = o.shakhov_equilibrium(rho, u[:D], T, q[:D])
    sel = np.linspace(0, o.Nv - 1, min(o.Nv, 25)).astype(int)
    for i in sel:
        g, b = _full_shakhov_reduced(xi[i], rho, u, T, q, 2.0 / 3.0, D, K)
        assert abs(ge[i] - g) <= 1e-11 * max(abs(g), 1e-3 * ge.max()), (i, ge[i], g)
        assert abs(be[i] - b) <= 1e-11 * max(abs(b), 1e-3 * np.abs(be).max()), (i, be[i], b)
    # the correction is really there (the Maxwellian differs)
    gm, _ = o.equilibrium(rho, u[:D], T)
    assert np.abs(ge - gm).max() > 1e-3 * gm.max()


@pytest.mark.parametrize("D", [1, 2, 3])
@pytest.mark.parametrize("K,Pr", [(0.0, 2.0 / 3.0), (2.0, 1.5)])
def test_shakhov_equilibrium_moments(oracle_mod, D, K, Pr):
    """rho, rho u, rho E and P = p I as the Maxwellian's; heat flux (1 - Pr) q."""
    nv = {1: 160, 2: 64, 3: 36}[D]
    cfg, _ = wl.uniform(dim=D, n=(2, 2, 2), nv=(nv, nv, nv), vmax=11.0, K=K, Pr=Pr)
    cfg["collision"] = SHAKHOV
    o = oracle_mod.Oracle(cfg)
    xi, w = o.velocities()
    xi = xi[:, :D]
    rho, T = 1.3, 1.7
    u = np.array([0.4, -0.3, 0.2])[:D]
    q = np.array([0.35, -0.2, 0.15])[:D]
    RT = R * T
    ge, be = o.shakhov_equilibrium(rho, u, T, q)
    gm, bm = o.equilibrium(rho, u, T)
    tol = 1e-10
    assert abs(w @ ge - rho) < tol * rho
    assert np.abs((w * ge) @ xi - rho * u).max() < tol * rho
    assert abs(w @ be - w @ bm) < tol * (w @ bm)
    P = (xi - u).T @ ((w * ge)[:, None] * (xi - u))
    assert np.abs(P - rho * RT * np.eye(D)).max() < tol * rho * RT
    rhoE = w @ be
    qS = (w * be) @ xi - u * rhoE - P @ u
    assert np.abs(qS - (1 - Pr) * q).max() < 1e-9 * np.abs(q).max(), (qS, (1 - Pr) * q)


def test_unit_prandtl_is_the_bgk_scheme_bit_for_bit(oracle_mod):
    cfg, f = wl.random_smooth(dim=2, n=(12, 9), nv=(10, 10), seed=4, amp=0.3, Pr=1.0, kn=3e-3)
    runs = []
    for coll in (0, SHAKHOV):
        o = oracle_mod.Oracle(dict(cfg, collision=coll))
        o.init(f)
        o.step(12)
        runs.append(np.concatenate([x.ravel() for x in o.distributions()] + [o.conserved().ravel()]))
    assert np.array_equal(runs[0], runs[1])


@pytest.mark.parametrize("Pr", [2.0 / 3.0, 1.5])
def test_tracked_heat_flux_in_a_sheared_2d_flow(oracle_mod, Pr):
    """The same identity in 2D, where the flow carries shear stress: the heat
    flux relative to W takes the pressure work of the off-diagonal stress
    components (sum over b of u_b P_ab, b other than a)."""
    n = 12       # 48 nodes per axis on [-11, 11]: the quadrature error is below the tolerance
    cfg = wl._base(2, [n, n], [0, 0], [1, 1], [[0, 0], [0, 0]], [48, 48], [-11.0, -11.0], [11.0, 11.0], K=2.0,
                   mu_ref=2e-2, T_ref=1.0, omega=0.5, Pr=Pr, cfl=0.5)
    cfg["collision"] = SHAKHOV
    _, (x, y) = wl.cell_centres(cfg)
    T = 1.0 + 0.3 * np.sin(2 * math.pi * x)
    f = wl._fields(1.0 / T, [0.3 + 0.2 * np.cos(2 * math.pi * y), 0.25 * np.sin(2 * math.pi * x)], T)
    o = oracle_mod.Oracle(cfg)
    o.init(f)
    o.step(20)
    P, qd = o.stress_heat_flux()
    qt = o.cell_heat_flux()
    assert np.abs(P[:, 0, 1]).max() > 1e-3            # shear stress is present
    assert np.abs(qd).max() > 1e-3
    assert np.abs(qt - qd).max() < 1e-9 * np.abs(qd).max(), np.abs(qt - qd).max()


@pytest.mark.parametrize("Pr", [2.0 / 3.0, 1.5])
def test_tracked_heat_flux_is_that_of_the_distributions(oracle_mod, Pr):
    """The heat flux the next equilibrium uses (from the update's explicit part,
    divided by 1 + dt Pr/(2 tau)) is the heat flux of the updated distributions."""
    nx = 32
    cfg = wl._base(1, [nx], [0], [1], [[0, 0]], [96], [-11.0], [11.0], K=2.0, mu_ref=2e-2, T_ref=1.0,
                   omega=0.5, Pr=Pr, cfl=0.5)
    cfg["collision"] = SHAKHOV
    _, (x,) = wl.cell_centres(cfg)
    T = 1.0 + 0.3 * np.sin(2 * math.pi * x)
    f = wl._fields(1.0 / T, [0.2 + 0.1 * np.cos(2 * math.pi * x)], T)
    o = oracle_mod.Oracle(cfg)
    o.init(f)
    assert np.abs(o.cell_heat_flux()).max() == 0.0
    o.step(30)
    qt = o.cell_heat_flux()[:, 0]
    _, qd = o.stress_heat_flux()
    qd = qd[:, 0]
    assert np.abs(qd).max() > 1e-3                      # conduction is under way
    assert np.abs(qt - qd).max() < 1e-9 * np.abs(qd).max(), np.abs(qt - qd).max()


def test_specular_equals_mirror_image_on_doubled_periodic_domain(oracle_mod):
    nx, nv = 24, 16
    cfg, f = wl.random_smooth(dim=1, n=(nx,), nv=(nv,), seed=11, amp=0.3, bc=wl.BC_SPECULAR, kn=5e-3,
                              Pr=2.0 / 3.0)
    cfg["collision"] = SHAKHOV
    o = oracle_mod.Oracle(cfg)
    o.init(f)
    cfg2 = dict(cfg)
    cfg2["n"] = [2 * nx, 1, 1]
    cfg2["hi"] = [2.0, 1.0, 1.0]
    cfg2["bc"] = [[wl.BC_PERIODIC] * 2] * 3
    f2 = np.concatenate([f, f[::-1] * np.array([1.0, -1.0, 1.0])], axis=0)
    o2 = oracle_mod.Oracle(cfg2)
    o2.init(f2)
    o.step(150)
    o2.step(150)
    m1, m2 = o.moments(), o2.moments()
    assert np.abs(m1 - m2[:nx]).max() <= 1e-12
    assert np.abs(m1 * np.array([1, -1, 1]) - m2[nx:][::-1]).max() <= 1e-12
    assert np.abs(o.cell_heat_flux()).max() > 1e-4


@pytest.mark.parametrize("D,nsteps,nv", [(1, 300, 32), (2, 30, 12), (3, 5, 8)])
def test_conservation_and_fixed_point(oracle_mod, D, nsteps, nv):
    cfg, f = wl.random_smooth(dim=D, n=(16, 10, 6), nv=(nv, nv, nv), seed=D, amp=0.3, Pr=2.0 / 3.0, kn=3e-3)
    cfg["collision"] = SHAKHOV
    o = oracle_mod.Oracle(cfg)
    o.init(f)
    S0 = o.conserved().sum(0)
    o.step(nsteps)
    S1 = o.conserved().sum(0)
    scale = np.array([S0[0]] + [S0[0]] * D + [S0[-1]])
    assert np.all(np.abs(S1 - S0) <= 1e-13 * scale)
    # a Maxwellian at rest on the symmetric grid has no discrete heat flux: an
    # exact fixed point; a drifting one carries the quadrature error of its
    # heat flux into the next equilibrium, so it stays put to that error
    # (a grid that resolves the drifting Maxwellian's moments to ~1e-12)
    fine = {1: 64, 2: 32, 3: 36}[D]
    for u, tol, m, vmax in (((0.0, 0.0, 0.0), 1e-14, nv, 6.0), ((0.3, -0.2, 0.1), 1e-10, fine, 7.0)):
        cfg, f = wl.uniform(dim=D, n=(5, 4, 3), nv=(m, m, m), u=u, T=1.2, Pr=2.0 / 3.0, kn=1e-2, vmax=vmax)
        cfg["collision"] = SHAKHOV
        o = oracle_mod.Oracle(cfg)
        o.init(f)
        g0, b0 = o.distributions()
        o.step(20)
        g1, b1 = o.distributions()
        assert np.abs(g1 - g0).max() <= tol * np.abs(g0).max()
        assert np.abs(b1 - b0).max() <= tol * np.abs(b0).max()
        assert np.abs(o.cell_heat_flux()).max() <= tol


@pytest.mark.slow
@pytest.mark.parametrize("Pr", [2.0 / 3.0, 1.5])
def test_conduction_matches_the_two_time_model_when_tau_is_below_the_step(oracle_mod, Pr):
    """Both collision models have the Navier-Stokes conductivity c_p mu/Pr, and
    on one grid they share every discretisation error but the collision's.  At
    h/tau ~ 2.4 the factors 1/(1 + h Pr/(2 tau)) and 1/(1 + dt Pr/(2 tau)) that
    take the heat flux from phibar and from the update's explicit part are far
    from 1; the isobaric conduction rates of the two models still agree."""
    mu, nx = 1e-4, 64
    k = 2 * math.pi
    rates = []
    for coll in (wl.COLLISION_TEDDF, SHAKHOV):
        cfg = wl._base(1, [nx], [0], [1], [[0, 0]], [64], [-8.0], [8.0], K=0.0, mu_ref=mu, T_ref=2.0,
                       omega=0.0, Pr=Pr, cfl=0.5)
        cfg["collision"] = coll
        _, (x,) = wl.cell_centres(cfg)
        rho = 1 + 1e-4 * np.sin(k * x)
        o = oracle_mod.Oracle(cfg)
        o.init(wl._fields(rho, [np.zeros_like(x)], 1.0 / (rho * R)))
        assert 0.5 * o.dt / mu > 2.0                     # h / tau

        def amp():
            m = o.moments()
            pp = m[:, 0] * R * m[:, 2]
            z = 2.0 * np.exp(-1j * k * x) / nx
            return abs(((m[:, 0] - m[:, 0].mean()) * z).sum() - ((pp - pp.mean()) * z).sum() / (5.0 / 3.0))

        n1, n2 = int(round(0.2 / o.dt)), int(round(1.0 / o.dt))
        o.step(n1)
        a1 = amp()
        o.step(n2 - n1)
        rates.append(math.log(a1 / amp()) / ((n2 - n1) * o.dt))
    pred = mu / Pr * k * k
    assert abs(rates[0] / pred - 1.0) < 0.2, rates        # the NS rate plus the grid's diffusion
    assert abs(rates[1] / rates[0] - 1.0) < 0.005, rates
