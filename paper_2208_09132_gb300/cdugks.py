"""Thin Python binding of the C ABI in ``include/cdugks.h`` (ctypes).

Argument marshalling only: every step of the scheme runs in the CUDA library.
PyTorch provides the device workspace and the stream.  There is no CPU
fallback; loading fails loudly when the library is missing or cannot be built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK = 0
ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_UNBOUND, ERR_NEGATIVE = -1, -2, -3, -4, -5, -6, -7
BC_PERIODIC, BC_SPECULAR, BC_DIRICHLET = 0, 1, 2
RULE_TRAPEZOID, RULE_BOOLE = 0, 1
FP64, FP32 = 0, 1

EXPORTS = [
    "cdugks_create", "cdugks_workspace_bytes", "cdugks_bind", "cdugks_init", "cdugks_step", "cdugks_capture",
    "cdugks_profile_step",
    "cdugks_sync_status", "cdugks_moments", "cdugks_stress_heat_flux", "cdugks_conserved", "cdugks_distributions",
    "cdugks_state_bytes", "cdugks_get_state", "cdugks_set_state", "cdugks_info",
    "cdugks_set_velocity_groups", "cdugks_set_reconstruction", "cdugks_set_collision", "cdugks_set_acceleration", "cdugks_test_wait_timeout",
    "cdugks_destroy", "cdugks_strerror", "cdugks_last_error",
    "cdugks_mu_from_kn", "cdugks_step_noalloc", "cdugks_tile_count", "cdugks_set_tile", "cdugks_tile_shape", "cdugks_cell_distributions",
    "cdugks_batch_create", "cdugks_batch_workspace_bytes", "cdugks_batch_bind", "cdugks_batch_capture",
    "cdugks_batch_step", "cdugks_batch_sync", "cdugks_batch_destroy", "cdugks_batch_admit", "cdugks_batch_retire",
    "cdugks_batch_set_persistent", "cdugks_batch_bound", "cdugks_batch_test_wait_timeout",
    "cdugks_batch_step_members",
]


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("bc", (ctypes.c_int * 2) * 3)]


class VGrid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("rule", ctypes.c_int)]


class Phys(ctypes.Structure):
    _fields_ = [("K", ctypes.c_double), ("R", ctypes.c_double), ("mu_ref", ctypes.c_double),
                ("T_ref", ctypes.c_double), ("omega", ctypes.c_double), ("Pr", ctypes.c_double),
                ("cfl", ctypes.c_double), ("dt", ctypes.c_double), ("precision", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("ncells", ctypes.c_longlong), ("nvel", ctypes.c_int),
                ("nvel_padded", ctypes.c_int), ("dt", ctypes.c_double), ("steps", ctypes.c_longlong),
                ("precision", ctypes.c_int), ("velocity_groups", ctypes.c_int),
                ("state_bytes", ctypes.c_double), ("tile_id", ctypes.c_int), ("tile", ctypes.c_int * 3)]


class CdugksError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load (building first if needed) the CUDA library and declare its ABI."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_needed else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run paper_2208_09132_gb300.build")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    dp = P(ctypes.c_double)
    sig = {
        "cdugks_create": (i, [P(Grid), P(VGrid), P(Phys), P(vp)]),
        "cdugks_workspace_bytes": (i, [vp, P(sz)]),
        "cdugks_bind": (i, [vp, vp, sz, vp]),
        "cdugks_init": (i, [vp, dp]),
        "cdugks_step": (i, [vp, i]),
        "cdugks_capture": (i, [vp, i]),
        "cdugks_profile_step": (i, [vp, i, dp]),
        "cdugks_sync_status": (i, [vp]),
        "cdugks_moments": (i, [vp, dp]),
        "cdugks_stress_heat_flux": (i, [vp, dp]),
        "cdugks_conserved": (i, [vp, dp]),
        "cdugks_distributions": (i, [vp, dp, dp]),
        "cdugks_state_bytes": (i, [vp, P(sz)]),
        "cdugks_get_state": (i, [vp, vp, sz]),
        "cdugks_set_state": (i, [vp, vp, sz]),
        "cdugks_info": (i, [vp, P(Info)]),
        "cdugks_set_velocity_groups": (i, [vp, i]),
        "cdugks_set_reconstruction": (i, [vp, i]),
        "cdugks_set_collision": (i, [vp, i]),
        "cdugks_set_acceleration": (i, [vp, dp]),
        "cdugks_test_wait_timeout": (i, [vp, i]),
        "cdugks_destroy": (None, [vp]),
        "cdugks_strerror": (ctypes.c_char_p, [i]),
        "cdugks_last_error": (ctypes.c_char_p, []),
        "cdugks_mu_from_kn": (d, [d, d, d, d, d]),
        "cdugks_step_noalloc": (i, [vp, vp, vp, vp, vp]),
        "cdugks_tile_count": (i, [i, i]),
        "cdugks_set_tile": (i, [vp, i]),
        "cdugks_tile_shape": (i, [i, i, i, P(i)]),
        "cdugks_cell_distributions": (i, [vp, P(ctypes.c_longlong), i, dp, dp]),
        "cdugks_batch_create": (i, [P(vp), i, P(vp)]),
        "cdugks_batch_workspace_bytes": (i, [vp, P(sz)]),
        "cdugks_batch_bind": (i, [vp, vp, sz, vp]),
        "cdugks_batch_capture": (i, [vp, i]),
        "cdugks_batch_step": (i, [vp, i]),
        "cdugks_batch_sync": (i, [vp]),
        "cdugks_batch_admit": (i, [vp, vp]),
        "cdugks_batch_retire": (i, [vp, vp]),
        "cdugks_batch_destroy": (None, [vp]),
        "cdugks_batch_set_persistent": (i, [vp, i, i, ctypes.c_longlong]),
        "cdugks_batch_bound": (i, [vp]),
        "cdugks_batch_test_wait_timeout": (i, [vp, i]),
        "cdugks_batch_step_members": (i, [vp, P(i), i]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != OK:
        lib = load()
        raise CdugksError(rc, lib.cdugks_last_error().decode() or lib.cdugks_strerror(rc).decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def describe(cfg: dict, precision: int | None = None):
    """C structs for a problem description dict (see ``workloads``)."""
    D = int(cfg["dim"])
    g, v, p = Grid(), VGrid(), Phys()
    g.dim = D
    for a in range(3):
        g.n[a] = int(cfg["n"][a]) if a < D else 1
        g.lo[a] = float(cfg["lo"][a]) if a < D else 0.0
        g.hi[a] = float(cfg["hi"][a]) if a < D else 1.0
        for s in range(2):
            g.bc[a][s] = int(cfg["bc"][a][s]) if a < D else 0
        v.n[a] = int(cfg["nv"][a]) if a < D else 1
        v.lo[a] = float(cfg["vlo"][a]) if a < D else 0.0
        v.hi[a] = float(cfg["vhi"][a]) if a < D else 0.0
    v.rule = int(cfg.get("rule", 0))
    p.K = float(cfg["K"])
    p.R = float(cfg.get("R", 0.5))
    p.mu_ref = float(cfg["mu_ref"])
    p.T_ref = float(cfg["T_ref"])
    p.omega = float(cfg.get("omega", 0.5))
    p.Pr = float(cfg["Pr"])
    p.cfl = float(cfg.get("cfl", 0.5))
    p.dt = float(cfg.get("dt", 0.0) or 0.0)
    if precision is None:
        precision = FP64 if cfg.get("precision", "fp64") == "fp64" else FP32
    p.precision = int(precision)
    return g, v, p


class Solver:
    """One CDUGKS problem instance on the GPU.

    The device workspace is a torch uint8 tensor on ``device``; all work runs
    on ``stream`` (default: torch's current stream for the device).
    """

    def __init__(self, cfg: dict, precision: int | None = None, device: str = "cuda:0", stream=None,
                 velocity_groups: int = 0, workspace=None, tile_id: int = 0):
        import torch

        self._lib = load()
        g, v, p = describe(cfg, precision)
        h = ctypes.c_void_p()
        _check(self._lib.cdugks_create(ctypes.byref(g), ctypes.byref(v), ctypes.byref(p), ctypes.byref(h)))
        self._h = h
        if cfg.get("collision", 0):          # the Shakhov model (and its default shape)
            _check(self._lib.cdugks_set_collision(h, int(cfg["collision"])))
        if any(cfg.get("accel", (0.0, 0.0, 0.0))):   # the external acceleration (and its default shape)
            acc = np.zeros(3)
            acc[: len(cfg["accel"])] = cfg["accel"]
            _check(self._lib.cdugks_set_acceleration(h, _dptr(acc)))
        if cfg.get("recon", 0):              # the face-gradient reconstruction (and its default shape)
            _check(self._lib.cdugks_set_reconstruction(h, int(cfg["recon"])))
        if tile_id:
            _check(self._lib.cdugks_set_tile(h, int(tile_id)))
        if velocity_groups:
            _check(self._lib.cdugks_set_velocity_groups(h, int(velocity_groups)))
        nbytes = ctypes.c_size_t()
        _check(self._lib.cdugks_workspace_bytes(h, ctypes.byref(nbytes)))
        self.workspace_bytes = int(nbytes.value)
        dev = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        if workspace is None:
            workspace = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=dev)
        self._ws = workspace
        base = workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        avail = workspace.numel() - (aligned - base)
        _check(self._lib.cdugks_bind(h, ctypes.c_void_p(aligned), ctypes.c_size_t(avail),
                                     ctypes.c_void_p(self.stream.cuda_stream)))
        self.D = int(cfg["dim"])
        inf = self.info()
        self.Nc = int(inf.ncells)
        self.Nv = int(inf.nvel)
        self.dt = float(inf.dt)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.cdugks_destroy(h)
            self._h = None

    def info(self) -> Info:
        inf = Info()
        _check(self._lib.cdugks_info(self._h, ctypes.byref(inf)))
        return inf

    def set_velocity_groups(self, groups: int):
        _check(self._lib.cdugks_set_velocity_groups(self._h, int(groups)))

    def init(self, rho_u_T: np.ndarray):
        a = np.ascontiguousarray(rho_u_T, dtype=np.float64).reshape(self.Nc, 2 + self.D)
        _check(self._lib.cdugks_init(self._h, _dptr(a)))

    def step(self, nsteps: int = 1):
        _check(self._lib.cdugks_step(self._h, int(nsteps)))

    def capture(self, steps_per_graph: int):
        """Replay whole multiples of steps_per_graph steps from CUDA graphs (0 drops them)."""
        _check(self._lib.cdugks_capture(self._h, int(steps_per_graph)))

    def profile_step(self, nsteps: int):
        """Advance nsteps steps; mean ms per step of (sweep A, face constants, sweep B, W update)."""
        out = np.zeros(4)
        _check(self._lib.cdugks_profile_step(self._h, int(nsteps), _dptr(out)))
        return out

    def sync_status(self) -> int:
        return int(self._lib.cdugks_sync_status(self._h))

    def moments(self, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty((self.Nc, 2 + self.D))
        _check(self._lib.cdugks_moments(self._h, _dptr(out)))
        return out

    def stress_heat_flux(self):
        """Per cell: pressure tensor P [Nc, D, D] and heat flux q [Nc, D] of the distributions."""
        D = self.D
        out = np.empty((self.Nc, D * D + D))
        _check(self._lib.cdugks_stress_heat_flux(self._h, _dptr(out)))
        return out[:, : D * D].reshape(self.Nc, D, D), out[:, D * D:]

    def conserved(self) -> np.ndarray:
        out = np.empty((self.Nc, 2 + self.D))
        _check(self._lib.cdugks_conserved(self._h, _dptr(out)))
        return out

    def distributions(self):
        g = np.empty((self.Nc, self.Nv))
        b = np.empty((self.Nc, self.Nv))
        _check(self._lib.cdugks_distributions(self._h, _dptr(g), _dptr(b)))
        return g, b

    def cell_distributions(self, cells):
        """g, b of the selected cells, [n][Nv] each."""
        idx = np.ascontiguousarray(cells, dtype=np.int64)
        g = np.empty((idx.size, self.Nv))
        b = np.empty((idx.size, self.Nv))
        _check(self._lib.cdugks_cell_distributions(self._h, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                                   int(idx.size), _dptr(g), _dptr(b)))
        return g, b

    def get_state(self) -> bytes:
        n = ctypes.c_size_t()
        _check(self._lib.cdugks_state_bytes(self._h, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(self._lib.cdugks_get_state(self._h, buf, n))
        return buf.raw

    def set_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(self._lib.cdugks_set_state(self._h, buf, ctypes.c_size_t(len(blob))))


class Batch:
    """Many Solvers stepped together in one launch per kernel (see include/cdugks.h)."""

    def __init__(self, solvers, stream=None, device: str = "cuda:0", persistent: bool = False, max_members: int = 0,
                 max_items: int = 0):
        import torch

        self._lib = load()
        self.members = list(solvers)
        arr = (ctypes.c_void_p * len(self.members))(*[s._h.value for s in self.members])
        h = ctypes.c_void_p()
        _check(self._lib.cdugks_batch_create(arr, len(self.members), ctypes.byref(h)))
        self._h = h
        if persistent:        # one launch per step call or graph (cdugks_batch_set_persistent)
            _check(self._lib.cdugks_batch_set_persistent(h, 1, int(max_members), int(max_items)))
        self._dev = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self._dev)
        self._ws = None
        self._bind()

    def _bind(self):
        """(Re)allocate the table workspace for the current members and bind it."""
        import torch

        n = ctypes.c_size_t()
        _check(self._lib.cdugks_batch_workspace_bytes(self._h, ctypes.byref(n)))
        if self._ws is None or self._ws.numel() < int(n.value) + 256:
            self._ws = torch.empty(int(n.value) + 256, dtype=torch.uint8, device=self._dev)
        base = self._ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        _check(self._lib.cdugks_batch_bind(self._h, ctypes.c_void_p(aligned),
                                           ctypes.c_size_t(self._ws.numel() - (aligned - base)),
                                           ctypes.c_void_p(self.stream.cuda_stream)))

    def admit(self, solver):
        """Add a member between steps (a persistent batch with room keeps its
        binding and graph; otherwise the tables are bound again)."""
        _check(self._lib.cdugks_batch_admit(self._h, solver._h))
        self.members.append(solver)
        if not self._lib.cdugks_batch_bound(self._h):
            self._bind()

    def retire(self, solver):
        """Remove a member between steps; it keeps its state (as for admit)."""
        _check(self._lib.cdugks_batch_retire(self._h, solver._h))
        self.members.remove(solver)
        if not self._lib.cdugks_batch_bound(self._h):
            self._bind()

    def test_wait_timeout(self, on: bool):
        _check(self._lib.cdugks_batch_test_wait_timeout(self._h, 1 if on else 0))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.cdugks_batch_destroy(h)
            self._h = None

    def capture(self, steps_per_graph: int):
        _check(self._lib.cdugks_batch_capture(self._h, int(steps_per_graph)))

    def step(self, nsteps: int = 1):
        _check(self._lib.cdugks_batch_step(self._h, int(nsteps)))

    def step_members(self, steps):
        """Persistent batches: member i (in self.members order) advances steps[i] steps, in one launch."""
        arr = (ctypes.c_int * len(steps))(*[int(v) for v in steps])
        _check(self._lib.cdugks_batch_step_members(self._h, arr, len(steps)))

    def sync(self) -> int:
        return int(self._lib.cdugks_batch_sync(self._h))


def tile_shape(precision: int, dim: int, tile_id: int):
    """(cells per axis, sweep mode) of an instantiated tile shape.  Mode bits
    0-1: 0 fused, 1 prepared phibar+, 2 stored phibar+ and slopes; bit 2 (4):
    face store (sweep A keeps the face values, sweep B only forms fluxes);
    bit 3 (8): the face-gradient reconstruction (cfg["recon"] = 1);
    bit 4 (16): the Shakhov collision model (cfg["collision"] = 1);
    bit 5 (32): the external acceleration (cfg["accel"] nonzero)."""
    out = (ctypes.c_int * 4)()
    _check(load().cdugks_tile_shape(int(precision), int(dim), int(tile_id), out))
    return tuple(out[:3]), int(out[3])


def find_tile(precision: int, dim: int, shape, mode: int) -> int:
    """Id of the instantiated tile shape with these cells per axis and sweep mode (0 if none)."""
    want = tuple(list(shape) + [1] * (3 - len(shape)))
    for t in range(load().cdugks_tile_count(int(precision), int(dim))):
        cells, m = tile_shape(precision, dim, t)
        if tuple(c if a < dim else 1 for a, c in enumerate(cells)) == want and m == mode:
            return t
    return 0


def mu_from_kn(kn, rho_ref, T_ref, R=0.5, length=1.0) -> float:
    return float(load().cdugks_mu_from_kn(kn, rho_ref, T_ref, R, length))
