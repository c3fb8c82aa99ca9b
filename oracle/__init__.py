"""Plain FP64 CPU oracle of the CDUGKS step (arXiv:2208.09132, Sec. 2, Sec. 2.1).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` leg of ``bench.py`` may import this
package.  The GPU product path never does, and the two share no code.

The arithmetic lives in ``cdugks_oracle.c`` (plain C, compiled here with gcc,
no FMA contraction so results agree across host architectures).  This module
only builds that library and marshals arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cdugks_oracle.c")
_HDR = os.path.join(_HERE, "cdugks_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

BC_PERIODIC, BC_SPECULAR, BC_DIRICHLET = 0, 1, 2
RULE_TRAPEZOID, RULE_BOOLE = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, C11, OpenMP)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
               "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("D", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("bc", (ctypes.c_int * 2) * 3),
        ("nv", ctypes.c_int * 3),
        ("vlo", ctypes.c_double * 3),
        ("vhi", ctypes.c_double * 3),
        ("rule", ctypes.c_int),
        ("K", ctypes.c_double),
        ("R", ctypes.c_double),
        ("mu_ref", ctypes.c_double),
        ("T_ref", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("Pr", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("recon", ctypes.c_int),
        ("collision", ctypes.c_int),
        ("accel", ctypes.c_double * 3),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d = ctypes.c_double
        dp = P(d)
        lib.oracle_create.restype = ctypes.c_void_p
        lib.oracle_create.argtypes = [P(_Params)]
        lib.oracle_destroy.argtypes = [ctypes.c_void_p]
        lib.oracle_init.argtypes = [ctypes.c_void_p, dp]
        lib.oracle_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        for name in ("oracle_moments", "oracle_conserved", "oracle_discrete_moments"):
            getattr(lib, name).argtypes = [ctypes.c_void_p, dp]
        lib.oracle_distributions.argtypes = [ctypes.c_void_p, dp, dp]
        lib.oracle_stress_heat_flux.argtypes = [ctypes.c_void_p, dp]
        lib.oracle_equilibrium.argtypes = [ctypes.c_void_p, d, dp, d, dp, dp]
        lib.oracle_shakhov_equilibrium.argtypes = [ctypes.c_void_p, d, dp, d, dp, dp, dp]
        lib.oracle_cell_heat_flux.argtypes = [ctypes.c_void_p, dp]
        lib.oracle_set_state.argtypes = [ctypes.c_void_p, dp, dp, dp]
        lib.oracle_face_W.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
        lib.oracle_face_moments.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
        lib.oracle_velocities.argtypes = [ctypes.c_void_p, dp, dp]
        lib.oracle_dt.restype = d
        lib.oracle_dt.argtypes = [ctypes.c_void_p]
        lib.oracle_nv.argtypes = [ctypes.c_void_p]
        lib.oracle_ncells.restype = ctypes.c_long
        lib.oracle_ncells.argtypes = [ctypes.c_void_p]
        lib.oracle_vanleer.restype = d
        lib.oracle_vanleer.argtypes = [d, d]
        lib.oracle_vgrid_1d.argtypes = [ctypes.c_int, d, d, ctypes.c_int, dp, dp]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def vanleer(s1: float, s2: float) -> float:
    return _load().oracle_vanleer(float(s1), float(s2))


def vgrid_1d(n: int, lo: float, hi: float, rule: int = RULE_TRAPEZOID):
    nodes = np.zeros(n)
    w = np.zeros(n)
    rc = _load().oracle_vgrid_1d(int(n), float(lo), float(hi), int(rule), _ptr(nodes), _ptr(w))
    if rc != 0:
        raise ValueError("invalid velocity grid")
    return nodes, w


class Oracle:
    """One CDUGKS problem instance on the CPU.

    ``cfg`` is a problem description dict (see ``paper_2208_09132_gb300.workloads``):
    keys dim, n, lo, hi, bc, nv, vlo, vhi, rule, K, R, mu_ref, T_ref, omega,
    Pr, dt, cfl; optional recon (0 upwind cell, 1 face gradient) and
    collision (0 the paper's two relaxation times, 1 Shakhov S-model) and
    accel (a uniform external acceleration, 3 components).
    """

    def __init__(self, cfg: dict):
        lib = _load()
        p = _Params()
        D = int(cfg["dim"])
        p.D = D
        for a in range(3):
            p.n[a] = int(cfg["n"][a]) if a < D else 1
            p.lo[a] = float(cfg["lo"][a]) if a < D else 0.0
            p.hi[a] = float(cfg["hi"][a]) if a < D else 1.0
            p.nv[a] = int(cfg["nv"][a]) if a < D else 1
            p.vlo[a] = float(cfg["vlo"][a]) if a < D else 0.0
            p.vhi[a] = float(cfg["vhi"][a]) if a < D else 0.0
            for s in range(2):
                p.bc[a][s] = int(cfg["bc"][a][s]) if a < D else 0
        p.rule = int(cfg.get("rule", 0))
        p.K = float(cfg["K"])
        p.R = float(cfg.get("R", 0.5))
        p.mu_ref = float(cfg["mu_ref"])
        p.T_ref = float(cfg["T_ref"])
        p.omega = float(cfg.get("omega", 0.5))
        p.Pr = float(cfg["Pr"])
        p.dt = float(cfg.get("dt", 0.0) or 0.0)
        p.cfl = float(cfg.get("cfl", 0.5))
        p.recon = int(cfg.get("recon", 0))
        p.collision = int(cfg.get("collision", 0))
        acc = list(cfg.get("accel", [0.0, 0.0, 0.0])) + [0.0, 0.0, 0.0]
        for a in range(3):
            p.accel[a] = float(acc[a])
        h = lib.oracle_create(ctypes.byref(p))
        if not h:
            raise ValueError("oracle_create rejected the problem description")
        self._h = h
        self._lib = lib
        self.D = D
        self.Nc = int(lib.oracle_ncells(h))
        self.Nv = int(lib.oracle_nv(h))
        self.dt = float(lib.oracle_dt(h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_destroy(h)
            self._h = None

    def init(self, rho_u_T: np.ndarray):
        a = np.ascontiguousarray(rho_u_T, dtype=np.float64).reshape(self.Nc, 2 + self.D)
        if self._lib.oracle_init(self._h, _ptr(a)) != 0:
            raise ValueError("oracle_init: non-positive density or temperature")

    def step(self, nsteps: int = 1):
        if self._lib.oracle_step(self._h, int(nsteps)) != 0:
            raise ValueError("oracle_step failed")

    def moments(self) -> np.ndarray:
        out = np.zeros((self.Nc, 2 + self.D))
        self._lib.oracle_moments(self._h, _ptr(out))
        return out

    def conserved(self) -> np.ndarray:
        out = np.zeros((self.Nc, 2 + self.D))
        self._lib.oracle_conserved(self._h, _ptr(out))
        return out

    def discrete_moments(self) -> np.ndarray:
        out = np.zeros((self.Nc, 2 + self.D))
        self._lib.oracle_discrete_moments(self._h, _ptr(out))
        return out

    def stress_heat_flux(self):
        """Per cell: pressure tensor P [Nc, D, D] and heat flux q [Nc, D] of the distributions."""
        D = self.D
        out = np.zeros((self.Nc, D * D + D))
        self._lib.oracle_stress_heat_flux(self._h, _ptr(out))
        return out[:, : D * D].reshape(self.Nc, D, D), out[:, D * D:]

    def cell_heat_flux(self) -> np.ndarray:
        """The heat flux each cell's equilibrium uses at the current time level,
        [Nc, D] (Shakhov model; zero otherwise)."""
        out = np.zeros((self.Nc, self.D))
        self._lib.oracle_cell_heat_flux(self._h, _ptr(out))
        return out

    def shakhov_equilibrium(self, rho: float, u, T: float, q):
        uu = np.zeros(3)
        uu[: self.D] = np.asarray(u, dtype=np.float64).reshape(-1)[: self.D]
        qq = np.zeros(3)
        qq[: self.D] = np.asarray(q, dtype=np.float64).reshape(-1)[: self.D]
        ge = np.zeros(self.Nv)
        be = np.zeros(self.Nv)
        self._lib.oracle_shakhov_equilibrium(self._h, float(rho), _ptr(uu), float(T), _ptr(qq), _ptr(ge), _ptr(be))
        return ge, be

    def distributions(self):
        g = np.zeros((self.Nc, self.Nv))
        b = np.zeros((self.Nc, self.Nv))
        self._lib.oracle_distributions(self._h, _ptr(g), _ptr(b))
        return g, b

    def set_state(self, g: np.ndarray, b: np.ndarray, W: np.ndarray):
        g = np.ascontiguousarray(g, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        W = np.ascontiguousarray(W, dtype=np.float64)
        self._lib.oracle_set_state(self._h, _ptr(g), _ptr(b), _ptr(W))

    def equilibrium(self, rho: float, u, T: float):
        uu = np.zeros(3)
        uu[: self.D] = np.asarray(u, dtype=np.float64).reshape(-1)[: self.D]
        ge = np.zeros(self.Nv)
        be = np.zeros(self.Nv)
        self._lib.oracle_equilibrium(self._h, float(rho), _ptr(uu), float(T), _ptr(ge), _ptr(be))
        return ge, be

    def velocities(self):
        xi = np.zeros((self.Nv, 3))
        w = np.zeros(self.Nv)
        self._lib.oracle_velocities(self._h, _ptr(xi), _ptr(w))
        return xi, w

    def face_W(self, axis: int, n: tuple) -> np.ndarray:
        cnt = 1
        for a in range(self.D):
            cnt *= (n[a] + 1) if a == axis else n[a]
        out = np.zeros((cnt, 2 + self.D))
        self._lib.oracle_face_W(self._h, int(axis), _ptr(out))
        return out

    def face_moments(self, axis: int, n: tuple) -> np.ndarray:
        """Moments of the face distributions of the last step, ordered as face_W."""
        cnt = 1
        for a in range(self.D):
            cnt *= (n[a] + 1) if a == axis else n[a]
        out = np.zeros((cnt, 2 + self.D))
        self._lib.oracle_face_moments(self._h, int(axis), _ptr(out))
        return out
