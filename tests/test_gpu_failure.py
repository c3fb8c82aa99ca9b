"""The failure path of the bounded device waits, exercised without a fault.

Sweep A's tensor copies complete on an mbarrier whose wait gives up after a
bounded number of tries; the sweep then records ST_TIMEOUT and stops.  The
test hook makes the wait run out (no copy is issued, a short limit), and the
test checks that the host reads CDUGKS_ERR_TIMEOUT and that the same handle
and context compute correctly afterwards."""
import numpy as np
import pytest

from paper_2208_09132_gb300 import cdugks, workloads as wl

pytestmark = pytest.mark.gpu


def test_bounded_wait_timeout_is_reported_and_the_handle_recovers(oracle_mod):
    cfg, f = wl.random_smooth(dim=2, n=(72, 28), nv=(8, 8), seed=1, amp=0.3, kn=3e-3)
    tile = cdugks.find_tile(cdugks.FP32, 2, (32, 8), 4)       # stages interior tiles with tensor copies
    s = cdugks.Solver(cfg, precision=cdugks.FP32, tile_id=tile, velocity_groups=3)
    lib = cdugks.load()
    s.init(f)
    assert lib.cdugks_test_wait_timeout(s._h, 1) == 0
    s.step(1)
    assert s.sync_status() == cdugks.ERR_TIMEOUT
    assert lib.cdugks_test_wait_timeout(s._h, 0) == 0
    s.init(f)
    s.step(10)
    assert s.sync_status() == 0
    o = oracle_mod.Oracle(cfg)
    o.init(f)
    o.step(10)
    ref = o.moments()
    assert (np.abs(s.moments() - ref).max(axis=0) / np.abs(ref).max(axis=0)).max() <= 1e-5
