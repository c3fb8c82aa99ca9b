"""Host-side checks of the C ABI: the library builds for sm_103a, exports every
symbol include/cdugks.h declares, and validates problem descriptions.  No
compute call here needs a GPU (cdugks_create does no device work)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2208_09132_gb300 import cdugks, workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "cdugks.h")).read()
    return sorted(set(re.findall(r"CDUGKS_API\s+[\w\s\*]*?\b(cdugks_\w+)\s*\(", txt)))


def test_header_declares_the_binding_exports():
    assert declared_symbols() == sorted(cdugks.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = cdugks.load()
    for name in declared_symbols():
        assert hasattr(lib, name), name


def _create(cfg, precision=cdugks.FP64):
    lib = cdugks.load()
    g, v, p = cdugks.describe(cfg, precision)
    h = ctypes.c_void_p()
    rc = lib.cdugks_create(ctypes.byref(g), ctypes.byref(v), ctypes.byref(p), ctypes.byref(h))
    return rc, h


def test_create_and_workspace_size():
    lib = cdugks.load()
    cfg, _ = wl.workload_c1()
    rc, h = _create(cfg)
    assert rc == 0 and h.value
    n = ctypes.c_size_t()
    assert lib.cdugks_workspace_bytes(h, ctypes.byref(n)) == 0
    state = 256 * 64 * 2 * 8
    assert n.value >= 2 * state
    info = cdugks.Info()
    assert lib.cdugks_info(h, ctypes.byref(info)) == 0
    assert info.ncells == 256 and info.nvel == 64 and info.nvel_padded == 64
    # unbound handle refuses device work with UNBOUND
    assert lib.cdugks_step(h, 1) == cdugks.ERR_UNBOUND
    lib.cdugks_destroy(h)


def test_time_step_matches_the_cfl_rule_of_the_oracle(oracle_mod):
    for cfg in (wl.workload_c1()[0], wl.workload_c2(scale=8)[0], wl.workload_c3(scale=8)[0]):
        rc, h = _create(cfg)
        assert rc == 0
        info = cdugks.Info()
        cdugks.load().cdugks_info(h, ctypes.byref(info))
        assert info.dt == oracle_mod.Oracle(cfg).dt
        cdugks.load().cdugks_destroy(h)


@pytest.mark.parametrize("mutate,err", [
    (lambda c: c.update(dim=4), cdugks.ERR_INVALID),
    (lambda c: c["n"].__setitem__(0, 0), cdugks.ERR_INVALID),
    (lambda c: c.update(rule=1), cdugks.ERR_INVALID),            # 64 nodes is not 4m+1
    (lambda c: c["vlo"].__setitem__(0, -7.0), cdugks.ERR_INVALID),  # specular needs symmetric range
    (lambda c: c.update(Pr=0.0), cdugks.ERR_INVALID),
    (lambda c: c["bc"].__setitem__(0, [0, 1]), cdugks.ERR_INVALID),
])
def test_create_rejects_bad_descriptions(mutate, err):
    cfg, _ = wl.workload_c1()
    cfg = {k: (list(map(list, v)) if k == "bc" else (list(v) if isinstance(v, list) else v)) for k, v in cfg.items()}
    mutate(cfg)
    rc, h = _create(cfg)
    assert rc == err
    assert not h.value
    assert cdugks.load().cdugks_last_error()


def test_strerror_and_mu_convention():
    lib = cdugks.load()
    assert lib.cdugks_strerror(cdugks.ERR_NEGATIVE).decode()
    mu = cdugks.mu_from_kn(1e-3, 1.5, (2.5 / 1.5) / 0.5, 0.5, 1.0)
    assert abs(mu - wl.mu_from_kn(1e-3, 1.5, 2.5 / 1.5)) < 1e-15


def test_reconstruction_selection_rules():
    """Face-gradient reconstruction: 1D/2D only, three cells next to a specular
    wall, before binding; its shapes only (host-side checks, no device)."""
    lib = cdugks.load()

    def handle(cfg, prec=cdugks.FP32):
        g, v, p = cdugks.describe(cfg, prec)
        h = ctypes.c_void_p()
        assert lib.cdugks_create(ctypes.byref(g), ctypes.byref(v), ctypes.byref(p), ctypes.byref(h)) == 0
        return h

    for dim, ok in ((1, True), (2, True), (3, False)):
        cfg, _ = wl.random_smooth(dim=dim, n=(8, 8, 8), nv=(4, 4, 4), seed=1)
        h = handle(cfg)
        assert (lib.cdugks_set_reconstruction(h, 1) == 0) == ok
        if ok:
            info = cdugks.Info()
            assert lib.cdugks_info(h, ctypes.byref(info)) == 0
            assert cdugks.tile_shape(cdugks.FP32, dim, info.tile_id)[1] & 8
            assert lib.cdugks_set_tile(h, 0) != 0            # an upwind-cell shape is refused now
        assert lib.cdugks_set_reconstruction(h, 7) != 0
        lib.cdugks_destroy(h)
    cfg, _ = wl.random_smooth(dim=1, n=(2,), nv=(4,), seed=1, bc=wl.BC_SPECULAR)
    h = handle(cfg)
    assert lib.cdugks_set_reconstruction(h, 1) != 0          # a wall needs 3 cells
    assert lib.cdugks_set_reconstruction(h, 0) == 0
    lib.cdugks_destroy(h)


def test_collision_selection_rules():
    """Shakhov collision: a face-store Shakhov shape in every dimension and
    precision, selected before binding; the other shapes are refused while it
    is selected, and so are the face-gradient reconstruction (no shape
    implements both), Dirichlet walls with the stored-slope 3D shape and the
    batch (host-side checks, no device)."""
    lib = cdugks.load()

    def handle(cfg, prec=cdugks.FP32):
        g, v, p = cdugks.describe(cfg, prec)
        h = ctypes.c_void_p()
        assert lib.cdugks_create(ctypes.byref(g), ctypes.byref(v), ctypes.byref(p), ctypes.byref(h)) == 0
        return h

    for prec in (cdugks.FP32, cdugks.FP64):
        for dim in (1, 2, 3):
            cfg, _ = wl.random_smooth(dim=dim, n=(8, 8, 8), nv=(4, 4, 4), seed=1)
            h = handle(cfg, prec)
            n0 = ctypes.c_size_t()
            assert lib.cdugks_workspace_bytes(h, ctypes.byref(n0)) == 0
            assert lib.cdugks_set_collision(h, wl.COLLISION_SHAKHOV) == 0, lib.cdugks_last_error()
            info = cdugks.Info()
            assert lib.cdugks_info(h, ctypes.byref(info)) == 0
            mode = cdugks.tile_shape(prec, dim, info.tile_id)[1]
            assert mode & 16 and mode & 4                  # a Shakhov face-store shape
            n1 = ctypes.c_size_t()
            assert lib.cdugks_workspace_bytes(h, ctypes.byref(n1)) == 0
            assert n1.value > n0.value                     # heat flux and raw-moment sums
            assert lib.cdugks_set_tile(h, 0) != 0          # a two-time shape is refused now
            assert lib.cdugks_set_reconstruction(h, 1) != 0
            assert lib.cdugks_set_collision(h, 5) != 0
            assert lib.cdugks_set_collision(h, wl.COLLISION_TEDDF) == 0
            assert lib.cdugks_info(h, ctypes.byref(info)) == 0
            assert not cdugks.tile_shape(prec, dim, info.tile_id)[1] & 16
            lib.cdugks_destroy(h)
    cfg, _ = wl.random_smooth(dim=3, n=(8, 8, 8), nv=(4, 4, 4), seed=1)
    cfg["bc"] = [[wl.BC_DIRICHLET] * 2] * 3
    h = handle(cfg)
    assert lib.cdugks_set_collision(h, wl.COLLISION_SHAKHOV) != 0
    lib.cdugks_destroy(h)
    for t in range(lib.cdugks_tile_count(cdugks.FP32, 2)):
        m = cdugks.tile_shape(cdugks.FP32, 2, t)[1]
        assert not (m & 16) or (m & 4 and not m & 8 and m & 3 != 1)


def test_acceleration_selection_rules():
    """External acceleration: a prepared face-store shape with the force in every
    dimension and precision, chosen before binding; components beyond dim and
    non-finite values are refused, and so are the Shakhov model and the
    face-gradient reconstruction with it (host-side checks, no device)."""
    lib = cdugks.load()

    def handle(cfg, prec=cdugks.FP32):
        g, v, p = cdugks.describe(cfg, prec)
        h = ctypes.c_void_p()
        assert lib.cdugks_create(ctypes.byref(g), ctypes.byref(v), ctypes.byref(p), ctypes.byref(h)) == 0
        return h

    def vec(*a):
        return (ctypes.c_double * 3)(*a)

    for prec in (cdugks.FP32, cdugks.FP64):
        for dim in (1, 2, 3):
            cfg, _ = wl.random_smooth(dim=dim, n=(8, 8, 8), nv=(4, 4, 4), seed=1)
            h = handle(cfg, prec)
            a = [0.5, -0.2, 0.1][:dim] + [0.0] * (3 - dim)
            assert lib.cdugks_set_acceleration(h, vec(*a)) == 0, lib.cdugks_last_error()
            info = cdugks.Info()
            assert lib.cdugks_info(h, ctypes.byref(info)) == 0
            mode = cdugks.tile_shape(prec, dim, info.tile_id)[1]
            assert mode & 32 and mode & 4 and mode & 3 == 1
            assert lib.cdugks_set_tile(h, 0) != 0
            assert lib.cdugks_set_collision(h, wl.COLLISION_SHAKHOV) != 0
            if dim < 3:
                assert lib.cdugks_set_reconstruction(h, 1) != 0
                bad = [0.0] * 3
                bad[dim] = 1.0
                assert lib.cdugks_set_acceleration(h, vec(*bad)) != 0        # beyond dim
            assert lib.cdugks_set_acceleration(h, vec(float("nan"), 0.0, 0.0)) != 0
            assert lib.cdugks_set_acceleration(h, None) == 0                 # off again
            assert lib.cdugks_info(h, ctypes.byref(info)) == 0
            assert not cdugks.tile_shape(prec, dim, info.tile_id)[1] & 32
            lib.cdugks_destroy(h)


def test_wait_timeout_hook_needs_no_device():
    cfg, _ = wl.random_smooth(dim=2, n=(8, 8), nv=(4, 4), seed=1)
    lib = cdugks.load()
    g, v, p = cdugks.describe(cfg, cdugks.FP32)
    h = ctypes.c_void_p()
    assert lib.cdugks_create(ctypes.byref(g), ctypes.byref(v), ctypes.byref(p), ctypes.byref(h)) == 0
    assert lib.cdugks_test_wait_timeout(h, 1) == 0          # unbound: host state only
    assert lib.cdugks_test_wait_timeout(h, 0) == 0
    assert lib.cdugks_test_wait_timeout(None, 1) != 0
    lib.cdugks_destroy(h)
