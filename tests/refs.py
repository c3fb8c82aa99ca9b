"""Independent textbook references used to pin the oracle.

Nothing here is the CDUGKS scheme: these are closed forms and classical
routines that the scheme must reduce to in a limit.

* ``exact_riemann`` -- exact solution of the Euler Riemann problem for an
  ideal gas (the standard two-rarefaction/shock pressure function solved by
  Newton iteration, then sampled along x/t), the Euler limit of Sec. 3.1.
* ``muscl_hancock_advection`` -- second-order upwind MUSCL-Hancock scheme for
  linear advection u_t + c u_x = 0 with the harmonic (van Leer) slope, the
  collisionless limit of the scheme for each discrete velocity.
* ``harmonic_slope`` -- the van Leer slope in its harmonic-mean form.
"""
from __future__ import annotations

import math

import numpy as np


def harmonic_slope(a, b):
    """van Leer slope 2ab/(a+b) when a and b have the same strict sign, else 0."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    same = a * b > 0
    out = np.zeros(np.broadcast(a, b).shape)
    den = np.where(same, a + b, 1.0)
    out = np.where(same, 2.0 * a * b / den, 0.0)
    return out


def muscl_hancock_advection(u0, c, dx, dt, nsteps, bc="periodic"):
    """Linear advection of the periodic array u0 with speed c (scalar).

    Face value at j+1/2 for c > 0: u_j + (1 - nu)/2 * dx * s_j, nu = c dt/dx,
    s_j the van Leer slope; mirrored for c < 0.  Conservative update."""
    u = np.array(u0, dtype=np.float64)
    nu = c * dt / dx
    for _ in range(nsteps):
        um = np.roll(u, 1)
        up = np.roll(u, -1)
        s = harmonic_slope((u - um) / dx, (up - u) / dx)
        if c > 0:
            face = u + 0.5 * (1.0 - nu) * dx * s            # value at j+1/2 from cell j
        elif c < 0:
            face = np.roll(u - 0.5 * (1.0 + nu) * dx * s, -1)  # value at j+1/2 from cell j+1
        else:
            face = np.zeros_like(u)
        flux = c * face
        u = u - dt / dx * (flux - np.roll(flux, 1))
    return u


def exact_riemann(rhoL, uL, pL, rhoR, uR, pR, gamma, x, t, x0=0.5):
    """Exact Euler Riemann solution sampled at positions x (array) and time t."""
    g = gamma
    cL = math.sqrt(g * pL / rhoL)
    cR = math.sqrt(g * pR / rhoR)

    def fk(p, rk, pk, ck):
        if p > pk:   # shock
            A = 2.0 / ((g + 1) * rk)
            B = (g - 1) / (g + 1) * pk
            f = (p - pk) * math.sqrt(A / (p + B))
            df = math.sqrt(A / (B + p)) * (1 - (p - pk) / (2 * (B + p)))
        else:        # rarefaction
            f = 2 * ck / (g - 1) * ((p / pk) ** ((g - 1) / (2 * g)) - 1)
            df = 1.0 / (rk * ck) * (p / pk) ** (-(g + 1) / (2 * g))
        return f, df

    p = 0.5 * (pL + pR)
    for _ in range(100):
        fL, dL = fk(p, rhoL, pL, cL)
        fR, dR = fk(p, rhoR, pR, cR)
        dp = (fL + fR + (uR - uL)) / (dL + dR)
        pn = max(p - dp, 1e-12)
        if abs(pn - p) < 1e-14 * p:
            p = pn
            break
        p = pn
    fL, _ = fk(p, rhoL, pL, cL)
    fR, _ = fk(p, rhoR, pR, cR)
    us = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    ps = p

    rho = np.empty_like(x, dtype=np.float64)
    u = np.empty_like(rho)
    pp = np.empty_like(rho)
    for k, xx in enumerate(np.asarray(x, dtype=np.float64)):
        s = (xx - x0) / t
        if s <= us:   # left of contact
            if ps > pL:   # left shock
                rs = rhoL * ((ps / pL + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pL + 1))
                SL = uL - cL * math.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
                st = (rhoL, uL, pL) if s < SL else (rs, us, ps)
            else:         # left rarefaction
                rs = rhoL * (ps / pL) ** (1 / g)
                csL = cL * (ps / pL) ** ((g - 1) / (2 * g))
                SHL, STL = uL - cL, us - csL
                if s < SHL:
                    st = (rhoL, uL, pL)
                elif s > STL:
                    st = (rs, us, ps)
                else:
                    uu = 2 / (g + 1) * (cL + (g - 1) / 2 * uL + s)
                    cc = 2 / (g + 1) * (cL + (g - 1) / 2 * (uL - s))
                    rr = rhoL * (cc / cL) ** (2 / (g - 1))
                    st = (rr, uu, pL * (cc / cL) ** (2 * g / (g - 1)))
        else:         # right of contact
            if ps > pR:   # right shock
                rs = rhoR * ((ps / pR + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pR + 1))
                SR = uR + cR * math.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
                st = (rhoR, uR, pR) if s > SR else (rs, us, ps)
            else:         # right rarefaction
                rs = rhoR * (ps / pR) ** (1 / g)
                csR = cR * (ps / pR) ** ((g - 1) / (2 * g))
                SHR, STR = uR + cR, us + csR
                if s > SHR:
                    st = (rhoR, uR, pR)
                elif s < STR:
                    st = (rs, us, ps)
                else:
                    uu = 2 / (g + 1) * (-cR + (g - 1) / 2 * uR + s)
                    cc = 2 / (g + 1) * (cR - (g - 1) / 2 * (uR - s))
                    rr = rhoR * (cc / cR) ** (2 / (g - 1))
                    st = (rr, uu, pR * (cc / cR) ** (2 * g / (g - 1)))
        rho[k], u[k], pp[k] = st
    return rho, u, pp


def fourier_amplitude(f, x, k):
    """|(2/N) sum f e^{-ikx}|: the amplitude of mode k of a periodic sample."""
    f = np.asarray(f, dtype=np.float64)
    z = np.sum((f - f.mean()) * np.exp(-1j * k * np.asarray(x)))
    return 2.0 * abs(z) / f.size
