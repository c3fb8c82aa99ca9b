"""The allocation-free step against the regular one.

cdugks_step_noalloc exists for callers that cannot allocate device memory
(their framework's pool owns the GPU and only lends out buffers it already
holds, or a device allocation in their loop could stall the whole GPU).  It
takes the state from the caller and keeps all other scratch in a fixed array
inside the library.  Here it must reproduce, on two calls in a row, what the
bound-workspace path computes from the same state, within the tolerance of the
other GPU tests (FP64 1e-12, FP32 1e-5 relative).  This file is named to be
collected last, so a run that stops at the first failure has run everything
else first.
"""
import ctypes

import numpy as np
import pytest

from paper_2208_09132_gb300 import cdugks, workloads as wl

pytestmark = pytest.mark.gpu


def _state_parts(solver, blob, elt):
    info = solver.info()
    nphi = info.nvel_padded * info.ncells * 2 * elt
    nW = 8 * (2 + info.dim) * info.ncells
    hdr = len(blob) - nphi - nW
    return blob[hdr:hdr + nphi], blob[hdr + nphi:]


def _two_calls_against_workspace_step(cfg, f, precision, tol, setup=None):
    """Two allocation-free calls in a row from the state of a regular solver,
    each compared with one regular step; setup(lib, handle) configures the
    allocation-free handle first (tile shape, velocity groups)."""
    import torch

    elt = 8 if precision == cdugks.FP64 else 4
    ref = cdugks.Solver(cfg, precision=precision)
    ref.init(f)
    phi0, W0 = _state_parts(ref, ref.get_state(), elt)

    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    buf = [torch.frombuffer(bytearray(phi0), dtype=torch.uint8).to(dev),
           torch.empty(len(phi0), dtype=torch.uint8, device=dev)]
    W = torch.frombuffer(bytearray(W0), dtype=torch.float64).to(dev)

    lib = cdugks.load()
    g, v, p = cdugks.describe(cfg, precision)
    h = ctypes.c_void_p()
    assert lib.cdugks_create(ctypes.byref(g), ctypes.byref(v), ctypes.byref(p), ctypes.byref(h)) == 0
    try:
        if setup is not None:
            setup(lib, h)
        D, Nc = cfg["dim"], ref.Nc
        for call in range(2):
            rc = lib.cdugks_step_noalloc(h, ctypes.c_void_p(buf[call % 2].data_ptr()),
                                         ctypes.c_void_p(buf[(call + 1) % 2].data_ptr()),
                                         ctypes.c_void_p(W.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
            assert rc == 0, lib.cdugks_last_error().decode()
            torch.cuda.synchronize()
            ref.step(1)
            Wref = ref.conserved()                                    # [Nc][2+D]
            Wgot = W.cpu().numpy().reshape(2 + D, Nc).T
            scale = np.abs(Wref).max(axis=0)
            assert np.all(np.abs(Wgot - Wref).max(axis=0) <= tol * scale), call
            phi_ref, _ = _state_parts(ref, ref.get_state(), elt)
            dt = np.float64 if precision == cdugks.FP64 else np.float32
            a = np.frombuffer(phi_ref, dtype=dt)
            b = buf[(call + 1) % 2].cpu().numpy().view(dt)
            assert np.abs(b - a).max() <= tol * np.abs(a).max(), call
    finally:
        lib.cdugks_destroy(h)


@pytest.mark.parametrize("precision,tol", [(cdugks.FP64, 1e-12), (cdugks.FP32, 1e-5)])
def test_noalloc_step_matches_the_workspace_step_on_two_calls(precision, tol):
    cfg, f = wl.random_smooth(dim=2, n=(40, 24), nv=(8, 12), seed=21, amp=0.3, kn=3e-3)
    cfg["bc"][0] = [wl.BC_SPECULAR, wl.BC_SPECULAR]
    _two_calls_against_workspace_step(cfg, f, precision, tol)


@pytest.mark.parametrize("precision,tol", [(cdugks.FP64, 1e-12), (cdugks.FP32, 1e-5)])
def test_noalloc_with_a_face_store_shape_selected(precision, tol):
    """A handle whose selected shape stores face values (a buffer the fixed
    array has no room for) steps in the plain fused shape instead."""
    cfg, f = wl.random_smooth(dim=2, n=(40, 24), nv=(8, 12), seed=23, amp=0.3, kn=3e-3)
    nt = cdugks.load().cdugks_tile_count(precision, 2)
    faces = [t for t in range(nt) if cdugks.tile_shape(precision, 2, t)[1] == 4]
    assert faces

    def setup(lib, h):
        assert lib.cdugks_set_tile(h, faces[0]) == 0

    _two_calls_against_workspace_step(cfg, f, precision, tol, setup)


def test_noalloc_halves_the_velocity_groups_to_fit():
    """64^2 cells and 16^2 velocities with 64 velocity groups need about 35 MB
    of face-moment partial sums; the step halves the group count once (to 32)
    and fits in the 32 MiB array."""
    cfg, f = wl.random_smooth(dim=2, n=(64, 64), nv=(16, 16), seed=24, amp=0.3, kn=3e-3)

    def setup(lib, h):
        assert lib.cdugks_set_velocity_groups(h, 64) == 0

    _two_calls_against_workspace_step(cfg, f, cdugks.FP32, 1e-5, setup)


def test_noalloc_rejects_oversized_problems_and_dirichlet():
    lib = cdugks.load()
    big, _ = wl.kelvin_helmholtz(n=1024, nv=8)              # cell and face tables beyond 32 MiB
    g, v, p = cdugks.describe(big, cdugks.FP32)
    h = ctypes.c_void_p()
    assert lib.cdugks_create(ctypes.byref(g), ctypes.byref(v), ctypes.byref(p), ctypes.byref(h)) == 0
    import torch
    x = torch.empty(64, dtype=torch.float64, device="cuda:0")
    y = torch.empty(64, dtype=torch.float64, device="cuda:0")
    rc = lib.cdugks_step_noalloc(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                 ctypes.c_void_p(x.data_ptr()), None)
    assert rc == cdugks.ERR_INVALID and b"scratch" in lib.cdugks_last_error()
    lib.cdugks_destroy(h)
    sod, _ = wl.sod(nx=64, nv=16, bc=wl.BC_DIRICHLET)
    g, v, p = cdugks.describe(sod, cdugks.FP64)
    assert lib.cdugks_create(ctypes.byref(g), ctypes.byref(v), ctypes.byref(p), ctypes.byref(h)) == 0
    rc = lib.cdugks_step_noalloc(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                 ctypes.c_void_p(x.data_ptr()), None)
    assert rc == cdugks.ERR_INVALID
    lib.cdugks_destroy(h)
