"""Seeded synthetic problem descriptions and initial fields.

This module only generates inputs: problem parameters and cell-centre initial
fields (rho, u[D], T) for the test problems of arXiv:2208.09132 Sec. 3 and for
the five benchmark workloads built on them.  It holds none of the scheme's
arithmetic; both the CUDA library and the CPU oracle consume what it returns.

A problem description is a plain dict:

    dim, n[3], lo[3], hi[3], bc[3][2], nv[3], vlo[3], vhi[3], rule,
    K, R, mu_ref, T_ref, omega, Pr, cfl, dt (0 -> CFL rule), steps

Fields are a float64 array [Nc][2 + dim] in cell order x fastest, then y, z.
"""
from __future__ import annotations

import math

import numpy as np

BC_PERIODIC, BC_SPECULAR, BC_DIRICHLET = 0, 1, 2
RULE_TRAPEZOID, RULE_BOOLE = 0, 1
# collision models: the paper's two relaxation times with the b-source (TEDDF),
# or the Shakhov S-model (one relaxation time, heat-flux-corrected equilibria)
COLLISION_TEDDF, COLLISION_SHAKHOV = 0, 1
R_GAS = 0.5          # the paper's gas constant (Sec. 2, "equal to 0.5 throughout")


def mu_from_kn(kn: float, rho_ref: float, rt_ref: float, length: float = 1.0) -> float:
    """Reference viscosity for a Knudsen number, hard-sphere convention.

    The paper specifies mu_r directly; the workloads are specified by Kn.  The
    conversion uses the hard-sphere mean free path lambda = 16 mu /
    (5 rho sqrt(2 pi R T)), i.e. mu_r = (5/16) Kn L rho_ref sqrt(2 pi R T_ref).
    This is an input convention shared by both implementations, not part of
    the scheme.
    """
    return 5.0 / 16.0 * kn * length * rho_ref * math.sqrt(2.0 * math.pi * rt_ref)


def _base(dim, n, lo, hi, bc, nv, vlo, vhi, K=2.0, mu_ref=1e-3, T_ref=1.0, omega=0.5,
          Pr=2.0 / 3.0, cfl=0.5, steps=1, rule=RULE_TRAPEZOID, dt=0.0, name=""):
    pad3 = lambda v, fill: [v[a] if a < dim else fill for a in range(3)]
    return {
        "name": name,
        "dim": dim,
        "n": pad3(list(n), 1),
        "lo": pad3(list(lo), 0.0),
        "hi": pad3(list(hi), 1.0),
        "bc": [list(bc[a]) if a < dim else [BC_PERIODIC, BC_PERIODIC] for a in range(3)],
        "nv": pad3(list(nv), 1),
        "vlo": pad3(list(vlo), 0.0),
        "vhi": pad3(list(vhi), 0.0),
        "rule": rule,
        "K": float(K),
        "R": R_GAS,
        "mu_ref": float(mu_ref),
        "T_ref": float(T_ref),
        "omega": float(omega),
        "Pr": float(Pr),
        "cfl": float(cfl),
        "dt": float(dt),
        "steps": int(steps),
    }


def ncells(cfg) -> int:
    return int(np.prod(cfg["n"][: cfg["dim"]]))


def nvel(cfg) -> int:
    return int(np.prod(cfg["nv"][: cfg["dim"]]))


def cell_centres(cfg):
    """Per-axis cell-centre coordinates and the meshgrid in cell order."""
    D = cfg["dim"]
    axes = []
    for a in range(D):
        n, lo, hi = cfg["n"][a], cfg["lo"][a], cfg["hi"][a]
        axes.append(lo + (np.arange(n) + 0.5) * (hi - lo) / n)
    grids = np.meshgrid(*axes[::-1], indexing="ij")     # z, y, x -> x fastest
    flat = [g.reshape(-1) for g in grids[::-1]]
    return axes, flat


def _fields(rho, u_list, T):
    cols = [np.asarray(rho, dtype=np.float64)] + [np.asarray(u, dtype=np.float64) for u in u_list] + \
           [np.asarray(T, dtype=np.float64)]
    return np.ascontiguousarray(np.stack(cols, axis=1))


# --------------------------------------------------------------------- problems

def sod(nx=256, nv=64, kn=1e-4, Pr=2.0 / 3.0, K=2.0, cfl=0.5, steps=200, bc=BC_SPECULAR,
        vmax=8.0, mu_ref=None, omega=0.5):
    """Sod shock tube (Sec. 3.1): (rho,u,p) = (1,0,1) | (1/8,0,1/10) at x = 0.5."""
    rt_ref = 1.0                       # p_L / rho_L
    mu = mu_from_kn(kn, 1.0, rt_ref) if mu_ref is None else mu_ref
    cfg = _base(1, [nx], [0.0], [1.0], [[bc, bc]], [nv], [-vmax], [vmax], K=K, mu_ref=mu,
                T_ref=rt_ref / R_GAS, omega=omega, Pr=Pr, cfl=cfl, steps=steps, name="sod")
    _, (x,) = cell_centres(cfg)
    left = x <= 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    return cfg, _fields(rho, [np.zeros_like(x)], p / (rho * R_GAS))


def kelvin_helmholtz(n=256, nv=32, kn=1e-3, Pr=1.0, K=2.0, cfl=0.8, steps=1000, vmax=6.0, seed=0):
    """Kelvin-Helmholtz shear layer (cf. Sec. 3.3): rho = 2 in |y-0.5| < 0.25 else 1,
    u_x = +-0.5, p = 2.5, v_y = 0.01 sin(4 pi x) times two Gaussian bands of
    width s = 0.05/sqrt(2) at y = 0.25, 0.75.  The perturbation is
    deterministic; ``seed`` is recorded for the workload name only."""
    rho_ref, rt_ref = 1.5, 2.5 / 1.5
    cfg = _base(2, [n, n], [0, 0], [1, 1], [[BC_PERIODIC] * 2] * 2, [nv, nv], [-vmax] * 2, [vmax] * 2,
                K=K, mu_ref=mu_from_kn(kn, rho_ref, rt_ref), T_ref=rt_ref / R_GAS, Pr=Pr, cfl=cfl,
                steps=steps, name=f"kh_seed{seed}")
    _, (x, y) = cell_centres(cfg)
    inside = np.abs(y - 0.5) < 0.25
    rho = np.where(inside, 2.0, 1.0)
    ux = np.where(inside, 0.5, -0.5)
    s = 0.05 / math.sqrt(2.0)
    uy = 0.01 * np.sin(4 * math.pi * x) * (np.exp(-(y - 0.25) ** 2 / (2 * s * s)) +
                                           np.exp(-(y - 0.75) ** 2 / (2 * s * s)))
    return cfg, _fields(rho, [ux, uy], 2.5 / (rho * R_GAS))


def shear3d(n=64, nv=24, kn=1e-4, Pr=2.0 / 3.0, K=2.0, cfl=0.7, steps=100, vmax=6.0):
    """3D shear wave (the Sec. 3.4 shear problem in three dimensions):
    rho = 1, T = 1, u_x = 0.1 sin(2 pi y)."""
    rho_ref, rt_ref = 1.0, R_GAS * 1.0
    cfg = _base(3, [n] * 3, [0] * 3, [1] * 3, [[BC_PERIODIC] * 2] * 3, [nv] * 3, [-vmax] * 3, [vmax] * 3,
                K=K, mu_ref=mu_from_kn(kn, rho_ref, rt_ref), T_ref=1.0, Pr=Pr, cfl=cfl, steps=steps,
                name="shear3d")
    _, (x, y, z) = cell_centres(cfg)
    ux = 0.1 * np.sin(2 * math.pi * y)
    return cfg, _fields(np.ones_like(x), [ux, np.zeros_like(x), np.zeros_like(x)], np.ones_like(x))


def thermoacoustic(nx=512, nv=64, kn=1e-3, Pr=2.0 / 3.0, K=2.0, cfl=0.5, steps=2000, delta=1e-3,
                   vmax=8.0, mu_ref=None):
    """Thermoacoustic wave (Sec. 3.5): rho = 1 - delta sin(4 pi x), RT = P0/rho, P0 = 1, u = 0, periodic."""
    rho_ref, rt_ref = 1.0, 1.0
    mu = mu_from_kn(kn, rho_ref, rt_ref) if mu_ref is None else mu_ref
    cfg = _base(1, [nx], [0.0], [1.0], [[BC_PERIODIC] * 2], [nv], [-vmax], [vmax], K=K, mu_ref=mu,
                T_ref=rt_ref / R_GAS, Pr=Pr, cfl=cfl, steps=steps, name="thermoacoustic")
    _, (x,) = cell_centres(cfg)
    rho = 1.0 - delta * np.sin(4 * math.pi * x)
    return cfg, _fields(rho, [np.zeros_like(x)], (1.0 / rho) / R_GAS)


def gresho(n=100, nv=101, kn=1e-4, Pr=2.0 / 3.0, K=2.0, cfl=0.8, steps=1, vmax=10.0, p0=5.0, bulk_vx=0.0):
    """Triangular Gresho vortex (Sec. 3.6) centred at (0.5, 0.5) in the periodic unit box."""
    rho_ref, rt_ref = 1.0, p0
    cfg = _base(2, [n, n], [0, 0], [1, 1], [[BC_PERIODIC] * 2] * 2, [nv, nv], [-vmax] * 2, [vmax] * 2,
                K=K, mu_ref=mu_from_kn(kn, rho_ref, rt_ref), T_ref=rt_ref / R_GAS, Pr=Pr, cfl=cfl,
                steps=steps, name="gresho")
    _, (x, y) = cell_centres(cfg)
    dx, dy = x - 0.5, y - 0.5
    r = np.sqrt(dx * dx + dy * dy)
    uphi = np.where(r <= 0.2, 5 * r, np.where(r <= 0.4, 2 - 5 * r, 0.0))
    rs = np.maximum(r, 1e-300)
    p = np.where(r <= 0.2, p0 + 12.5 * r * r,
                 np.where(r <= 0.4, p0 + 12.5 * r * r + 4 * (1 - 5 * r - math.log(0.2) + np.log(rs)),
                          p0 - 2 + 4 * math.log(2.0)))
    ux = -uphi * dy / rs + bulk_vx
    uy = uphi * dx / rs
    rho = np.ones_like(x)
    return cfg, _fields(rho, [ux, uy], p / (rho * R_GAS))


def einfeldt(nx=256, nv=129, mu_ref=1e-6, T_ref=1.0, K=2.0, Pr=2.0 / 3.0, cfl=0.4, vmax=10.0, t_end=0.125,
             rule=RULE_TRAPEZOID, bc=BC_DIRICHLET):
    """Einfeldt 1-2-0-3 rarefaction (Sec. 3.2): rho = 1, rho E = 3,
    u = 2 sgn(x - 1/2) on [0, 1] (so c_v T = 1, T = 0.8 with K = 2), hard-sphere
    viscosity, Pr = 2/3, velocities on [-10, 10], CFL 0.4, to t = 0.125.  The
    ends hold the initial equilibrium (Dirichlet; no signal reaches them by
    t_end).  The paper's high-resolution run has nx = 8192, nv = 129."""
    cfg = _base(1, [nx], [0.0], [1.0], [[bc, bc]], [nv], [-vmax], [vmax], K=K, mu_ref=mu_ref, T_ref=T_ref,
                Pr=Pr, cfl=cfl, rule=rule, name=f"einfeldt_1203_{nx}x{nv}")
    steps = int(np.ceil(t_end / (cfl * (1.0 / nx) / (2.0 * vmax)) - 1e-9))
    cfg["steps"] = steps
    cfg["dt"] = t_end / steps
    _, (x,) = cell_centres(cfg)
    cv = (3.0 + K) * R_GAS / 2.0
    u = 2.0 * np.sign(x - 0.5)
    T = (3.0 - 0.5 * u ** 2) / cv
    return cfg, _fields(np.ones(nx), [u], T)


def sine_wave(nx=128, nv=129, T0=0.1, mu_ref=1e-5, rho0=1.0, v0=1.0, K=2.0, Pr=2.0 / 3.0, cfl=0.5, vmax=6.0,
              rule=RULE_BOOLE, t_end=0.1):
    """Sine-wave perturbation (Sec. 3.7): rho = rho0, v = v0 sin(2 pi x),
    E = c_v T0 + v^2/2 on the periodic unit interval, velocities on
    [-vmax, vmax] (Newton-Cotes / Boole weights by default: nv = 4m + 1).
    With T = 1 it is the smooth case of the paper's convergence study
    (Sec. 4).  The time step is the largest one within the CFL bound that
    reaches t_end in a whole number of steps (cfg["steps"])."""
    cfg = _base(1, [nx], [0.0], [1.0], [[BC_PERIODIC, BC_PERIODIC]], [nv], [-vmax], [vmax], K=K,
                mu_ref=mu_ref, T_ref=T0, Pr=Pr, cfl=cfl, rule=rule, name=f"sine_wave_T{T0:g}_mu{mu_ref:g}")
    steps = int(np.ceil(t_end / (cfl * (1.0 / nx) / (2.0 * vmax)) - 1e-9))
    cfg["steps"] = steps
    cfg["dt"] = t_end / steps           # within the CFL bound, ending exactly at t_end
    _, (x,) = cell_centres(cfg)
    return cfg, _fields(np.full(nx, rho0), [v0 * np.sin(2 * np.pi * x)], np.full(nx, T0))


def uniform(dim=1, n=(8, 8, 8), nv=(8, 8, 8), rho=1.0, u=(0.0, 0.0, 0.0), T=1.0, vmax=6.0,
            kn=1e-2, Pr=2.0 / 3.0, K=2.0, cfl=0.5, bc=BC_PERIODIC):
    """A uniform Maxwellian state (the scheme's fixed point)."""
    cfg = _base(dim, list(n)[:dim], [0] * dim, [1] * dim, [[bc, bc]] * dim, list(nv)[:dim],
                [-vmax] * dim, [vmax] * dim, K=K, mu_ref=mu_from_kn(kn, rho, R_GAS * T),
                T_ref=T, Pr=Pr, cfl=cfl, name="uniform")
    Nc = ncells(cfg)
    return cfg, _fields(np.full(Nc, rho), [np.full(Nc, u[a]) for a in range(dim)], np.full(Nc, T))


def random_smooth(dim=2, n=(12, 10, 8), nv=(8, 8, 8), seed=0, amp=0.2, vmax=6.0, kn=1e-2,
                  Pr=2.0 / 3.0, K=2.0, cfl=0.5, bc=BC_PERIODIC, mu_ref=None, omega=0.5):
    """Seeded smooth random fields: a few random Fourier modes on rho, u, T."""
    rng = np.random.default_rng(seed)
    cfg = _base(dim, list(n)[:dim], [0] * dim, [1] * dim, [[bc, bc]] * dim, list(nv)[:dim],
                [-vmax] * dim, [vmax] * dim, K=K,
                mu_ref=mu_from_kn(kn, 1.0, R_GAS) if mu_ref is None else mu_ref,
                T_ref=1.0, omega=omega, Pr=Pr, cfl=cfl, name=f"random_smooth_seed{seed}")
    _, X = cell_centres(cfg)

    def field(base, a):
        f = np.full_like(X[0], base)
        for _ in range(3):
            k = rng.integers(1, 3, size=dim)
            ph = rng.uniform(0, 2 * math.pi)
            f = f + a * rng.uniform(-1, 1) * np.sin(2 * math.pi * sum(k[d] * X[d] for d in range(dim)) + ph)
        return f

    rho = field(1.0, amp / 3)
    T = field(1.0, amp / 3)
    us = [field(0.0, amp) for _ in range(dim)]
    return cfg, _fields(rho, us, T)


# ----------------------------------------------------------- benchmark workloads

def workload_c1():
    """1D Sod, FP64 plain method: Nx=256, Nv=64 on [-8,8], K=2, Kn=1e-4, Pr=2/3, CFL 0.5, 200 steps."""
    cfg, f = sod()
    cfg["precision"] = "fp64"
    cfg["name"] = "sod_1d_nx256_nv64"
    return cfg, f


def workload_c2(scale=1):
    """2D Kelvin-Helmholtz, FP32 storage: 256^2 periodic, 32^2 velocities on [-6,6]^2, Kn=1e-3, Pr=1, 1000 steps."""
    n = 256 // scale
    cfg, f = kelvin_helmholtz(n=n)
    cfg["precision"] = "fp32"
    cfg["name"] = f"kh_2d_{n}x{n}_nv32x32"
    return cfg, f


def workload_c3(kn=1e-4, scale=1, nv=24):
    """3D shear wave, FP32 storage: 64^3 periodic, 24^3 velocities on [-6,6]^3, Pr=2/3, 100 steps."""
    n = 64 // scale
    cfg, f = shear3d(n=n, nv=nv, kn=kn)
    cfg["precision"] = "fp32"
    cfg["name"] = f"shear_3d_{n}^3_nv{nv}^3_kn{kn:g}"
    return cfg, f


def workload_c4(count=256, seed=0, nx_range=(128, 4096), steps=2000):
    """Batched uneven 1D thermoacoustic waves (seeded per instance)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nx = int(round(math.exp(rng.uniform(math.log(nx_range[0]), math.log(nx_range[1])))))
        nv = int(rng.choice([32, 64, 128]))
        kn = 10.0 ** rng.uniform(-4.0, 1.0)
        Pr = float(rng.choice([0.5, 2.0 / 3.0, 1.0, 2.0]))
        cfg, f = thermoacoustic(nx=nx, nv=nv, kn=kn, Pr=Pr, steps=steps)
        cfg["precision"] = "fp32"
        cfg["name"] = f"ta_{k}_nx{nx}_nv{nv}"
        out.append((cfg, f))
    return out


def workload_c5(count=256, seed=1, rate=50.0, side_range=(64, 512), vside_range=(16, 48),
                t_end=1.0):
    """Served stream: Poisson arrivals of Gresho / Kelvin-Helmholtz solves.

    Returns a list of (arrival_time_s, cfg, fields)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += rng.exponential(1.0 / rate)
        kind = "gresho" if rng.uniform() < 0.5 else "kh"
        n = int(round(math.exp(rng.uniform(math.log(side_range[0]), math.log(side_range[1])))))
        nv = int(round(math.exp(rng.uniform(math.log(vside_range[0]), math.log(vside_range[1])))))
        kn = 10.0 ** rng.uniform(-4.0, 0.0)
        if kind == "gresho":
            cfg, f = gresho(n=n, nv=nv, kn=kn, cfl=0.8)
        else:
            cfg, f = kelvin_helmholtz(n=n, nv=nv, kn=kn, cfl=0.8)
        cfg["t_end"] = t_end
        cfg["precision"] = "fp32"
        cfg["name"] = f"{kind}_{k}_n{n}_nv{nv}"
        out.append((t, cfg, f))
    return out
