"""Edge cases of the step and of batches: zero steps, one-cell-wide and
two-cell axes, the smallest velocity grids, empty and duplicate batches, the
persistent step's member limit, and negative counts.

Results that the method fixes are compared with the oracle (tolerances of the
parity tests); calls that must change nothing are compared bit for bit."""
import ctypes

import numpy as np
import pytest

from paper_2208_09132_gb300 import cdugks, workloads as wl
from test_gpu_parity import rel_linf

pytestmark = pytest.mark.gpu


def _solver(cfg, f, prec=cdugks.FP64, **kw):
    s = cdugks.Solver(cfg, precision=prec, **kw)
    s.init(f)
    return s


def test_zero_steps_change_nothing():
    cfg, f = wl.random_smooth(dim=2, n=(19, 13), nv=(8, 6), seed=5, amp=0.3, kn=5e-3)
    s = _solver(cfg, f, cdugks.FP32)
    s.step(3)
    before = s.get_state()
    s.step(0)
    assert s.sync_status() == 0
    assert s.get_state() == before and s.info().steps == 3
    with pytest.raises(cdugks.CdugksError):
        s.step(-1)
    # batches: zero steps, and zero steps for every member of a persistent batch
    t = cdugks.find_tile(cdugks.FP32, 2, (32, 8), 4)
    a = _solver(cfg, f, cdugks.FP32, tile_id=t)
    b = cdugks.Batch([a], persistent=True)
    b.step(0)
    b.step_members([0])
    assert b.sync() == 0
    assert a.info().steps == 0
    with pytest.raises(cdugks.CdugksError):
        b.step(-2)


@pytest.mark.parametrize("prec,tol", [(cdugks.FP64, 1e-12), (cdugks.FP32, 1e-5)])
def test_one_cell_wide_and_two_cell_axes_match_oracle(oracle_mod, prec, tol):
    """A periodic axis of one cell (its halo is the cell itself) and of two
    cells (each cell is both neighbours of the other), in 2D and 3D."""
    cases = [wl.random_smooth(dim=2, n=(1, 9), nv=(8, 8), seed=11, amp=0.3, kn=5e-3),
             wl.random_smooth(dim=2, n=(7, 2), nv=(6, 8), seed=12, amp=0.3, kn=5e-3),
             wl.random_smooth(dim=3, n=(2, 1, 5), nv=(4, 4, 6), seed=13, amp=0.3, kn=5e-3)]
    for cfg, f in cases:
        o = oracle_mod.Oracle(cfg)
        o.init(f)
        o.step(6)
        s = _solver(cfg, f, prec)
        s.step(6)
        assert s.sync_status() == 0
        err = rel_linf(s.moments(), o.moments())
        assert np.all(err <= tol), (cfg["n"], err)


@pytest.mark.parametrize("prec,tol", [(cdugks.FP64, 1e-12), (cdugks.FP32, 1e-5)])
def test_smallest_grids_match_oracle(oracle_mod, prec, tol):
    """Two cells and four velocities (one chunk) in 1D; a 3D grid of one
    chunk per velocity row."""
    for cfg, f in (wl.random_smooth(dim=1, n=(2,), nv=(4,), seed=14, amp=0.2, kn=1e-2),
                   wl.random_smooth(dim=1, n=(3,), nv=(5,), seed=15, amp=0.2, kn=1e-2),
                   wl.random_smooth(dim=3, n=(3, 3, 3), nv=(4, 4, 4), seed=16, amp=0.2, kn=1e-2)):
        o = oracle_mod.Oracle(cfg)
        o.init(f)
        o.step(8)
        s = _solver(cfg, f, prec)
        s.step(8)
        assert s.sync_status() == 0
        err = rel_linf(s.moments(), o.moments())
        assert np.all(err <= tol), (cfg["n"], cfg["nv"], err)


def test_batch_creation_rejects_empty_and_duplicate_members():
    lib = cdugks.load()
    h = ctypes.c_void_p()
    assert lib.cdugks_batch_create(None, 0, ctypes.byref(h)) == cdugks.ERR_INVALID
    cfg, f = wl.random_smooth(dim=1, n=(40,), nv=(8,), seed=17, amp=0.2, kn=1e-2)
    s = _solver(cfg, f, cdugks.FP32)
    arr = (ctypes.c_void_p * 2)(s._h.value, s._h.value)
    assert lib.cdugks_batch_create(arr, 2, ctypes.byref(h)) == cdugks.ERR_INVALID
    assert not h.value


def test_persistent_member_limit_and_room():
    """More than 1024 reserved members is refused; admitting past the reserved
    room falls back to an unbound batch that binds again."""
    lib = cdugks.load()
    t = cdugks.find_tile(cdugks.FP32, 1, (128,), 4)
    probs = [wl.thermoacoustic(nx=60 + 10 * k, nv=8, kn=1e-3, delta=0.05) for k in range(3)]
    solvers = [_solver(c, ff, cdugks.FP32, tile_id=t) for c, ff in probs]
    b = cdugks.Batch(solvers[:1])
    assert lib.cdugks_batch_set_persistent(b._h, 1, 1025, 0) == cdugks.ERR_INVALID
    b = cdugks.Batch(solvers[:1], persistent=True, max_members=1, max_items=0)
    b.step(2)
    b.admit(solvers[1])                      # no room reserved: unbind, plan, bind again
    b.step(2)
    assert b.sync() == 0
    assert lib.cdugks_batch_bound(b._h) == 1
    ref = _solver(probs[1][0], probs[1][1], cdugks.FP32, tile_id=t)
    ref.step(2)
    assert np.array_equal(solvers[1].moments(), ref.moments())
