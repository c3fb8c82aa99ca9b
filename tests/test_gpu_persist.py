"""The persistent batched step: every phase of every member, for all the steps
of a call or of a captured graph, in one launch.

Its CTAs take work items in dependency order and wait per member for what an
item needs, so a member must compute exactly what the per-kernel launches (and
stepping it alone) compute: the results are compared bit for bit.  Membership
changes of a persistent batch with room rewrite its device tables in place and
keep the captured graph.  The bounded waits are tested without a fault: a test
hook makes one wait impossible, the step stops early, the status reads
TIMEOUT, and the batch steps correctly once the hook is off and the members'
state is restored."""
import numpy as np
import pytest

from paper_2208_09132_gb300 import cdugks, workloads as wl

pytestmark = pytest.mark.gpu


def _members_1d(seed, count, nv_choices=(8, 16, 24, 32)):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nx = int(rng.integers(40, 700))
        nv = int(rng.choice(nv_choices))
        kn = 10.0 ** rng.uniform(-4, 0)
        Pr = float(rng.choice([0.5, 2.0 / 3.0, 1.0, 2.0]))
        out.append(wl.thermoacoustic(nx=nx, nv=nv, kn=kn, Pr=Pr, delta=0.05))
    return out


def _solo(cfg, f, prec, steps, tile, groups=0):
    s = cdugks.Solver(cfg, precision=prec, tile_id=tile, velocity_groups=groups)
    s.init(f)
    s.step(steps)
    return s


@pytest.mark.parametrize("prec,shape", [(cdugks.FP32, (128,)), (cdugks.FP32, (64,)), (cdugks.FP64, (64,))])
@pytest.mark.parametrize("graph", [0, 3])
def test_persistent_batch_equals_members_alone(prec, shape, graph):
    tile = cdugks.find_tile(prec, 1, shape, 4)
    probs = _members_1d(seed=5, count=7)
    groups = [1, 2, 3, 1, 4, 2, 1]
    solvers = []
    for (cfg, f), g in zip(probs, groups):
        s = cdugks.Solver(cfg, precision=prec, tile_id=tile, velocity_groups=g)
        s.init(f)
        solvers.append(s)
    b = cdugks.Batch(solvers, persistent=True)
    if graph:
        b.capture(graph)
    b.step(7)                     # with a graph of 3: two replays and one launch of one step
    b.step(2)
    assert b.sync() == 0
    for (cfg, f), g, s in zip(probs, groups, solvers):
        ref = _solo(cfg, f, prec, 9, tile, g)
        assert s.info().steps == 9
        assert np.array_equal(s.moments(), ref.moments())
        assert s.get_state() == ref.get_state()


def test_persistent_batch_2d():
    tile = cdugks.find_tile(cdugks.FP32, 2, (32, 8), 4)
    probs = [wl.random_smooth(dim=2, n=(40, 24), nv=(8, 6), seed=51, amp=0.3, kn=3e-3, Pr=1.0),
             wl.kelvin_helmholtz(n=48, nv=12, kn=1e-3),
             wl.random_smooth(dim=2, n=(19, 13), nv=(10, 4), seed=52, amp=0.3, kn=5e-3)]
    solvers = []
    for cfg, f in probs:
        s = cdugks.Solver(cfg, precision=cdugks.FP32, tile_id=tile, velocity_groups=3)
        s.init(f)
        solvers.append(s)
    b = cdugks.Batch(solvers, persistent=True)
    b.capture(4)
    b.step(8)
    assert b.sync() == 0
    for (cfg, f), s in zip(probs, solvers):
        assert np.array_equal(s.moments(), _solo(cfg, f, cdugks.FP32, 8, tile, 3).moments())


def test_persistent_membership_changes_keep_the_graph():
    """Admit and retire between steps with room reserved: the batch stays bound
    (its captured graph is replayed after the change), and every member's
    trajectory equals stepping it alone."""
    prec = cdugks.FP32
    tile = cdugks.find_tile(prec, 1, (128,), 4)
    probs = _members_1d(seed=9, count=4)
    solvers = []
    for cfg, f in probs:
        s = cdugks.Solver(cfg, precision=prec, tile_id=tile)
        s.init(f)
        solvers.append(s)
    s0, s1, s2, s3 = solvers
    b = cdugks.Batch([s0, s1], persistent=True, max_members=8, max_items=4096)
    b.capture(2)
    b.step(4)                                   # s0, s1: 4
    lib = cdugks.load()
    b.admit(s2)
    assert lib.cdugks_batch_bound(b._h) == 1    # rewritten in place
    b.step(3)                                   # s0, s1: 7; s2: 3 (one graph replay, one launch)
    b.retire(s0)
    b.admit(s3)
    assert lib.cdugks_batch_bound(b._h) == 1
    b.step(5)                                   # s1: 12; s2: 8; s3: 5
    assert b.sync() == 0
    for (cfg, f), s, n in zip(probs, solvers, (7, 12, 8, 5)):
        assert s.info().steps == n
        assert np.array_equal(s.moments(), _solo(cfg, f, prec, n, tile).moments())


def test_persistent_wait_timeout_is_reported_and_recovers():
    prec = cdugks.FP32
    tile = cdugks.find_tile(prec, 1, (128,), 4)
    probs = _members_1d(seed=13, count=3)
    solvers = []
    for cfg, f in probs:
        s = cdugks.Solver(cfg, precision=prec, tile_id=tile)
        s.init(f)
        solvers.append(s)
    b = cdugks.Batch(solvers, persistent=True)
    b.test_wait_timeout(True)
    b.step(2)
    assert b.sync() == cdugks.ERR_TIMEOUT       # the launch stopped early; nothing faulted
    b.test_wait_timeout(False)
    for s, (cfg, f) in zip(solvers, probs):     # a valid state again (init clears the status word)
        s.init(f)
    b._bind()                                   # the members' buffer parities, uploaded again
    b.step(3)
    assert b.sync() == 0
    for (cfg, f), s in zip(probs, solvers):
        assert np.array_equal(s.moments(), _solo(cfg, f, prec, 3, tile).moments())


def test_persistent_step_members_own_counts():
    """One launch in which each member advances its own number of steps
    (zero included), then a captured graph of the whole batch: every member
    equals stepping it alone by its total."""
    prec = cdugks.FP32
    tile = cdugks.find_tile(prec, 1, (128,), 4)
    probs = _members_1d(seed=21, count=5)
    solvers = []
    for cfg, f in probs:
        s = cdugks.Solver(cfg, precision=prec, tile_id=tile, velocity_groups=2)
        s.init(f)
        solvers.append(s)
    b = cdugks.Batch(solvers, persistent=True)
    b.capture(2)
    own = [3, 0, 5, 1, 4]
    b.step_members(own)
    b.step(2)                                   # one graph replay after the per-member launch
    b.step_members([1, 2, 0, 2, 1])
    assert b.sync() == 0
    for (cfg, f), s, n in zip(probs, solvers, [3 + 2 + 1, 0 + 2 + 2, 5 + 2, 1 + 2 + 2, 4 + 2 + 1]):
        assert s.info().steps == n
        assert np.array_equal(s.moments(), _solo(cfg, f, prec, n, tile, 2).moments())


def test_step_members_rejects_bad_calls():
    prec = cdugks.FP32
    tile = cdugks.find_tile(prec, 1, (128,), 4)
    probs = _members_1d(seed=23, count=2)
    solvers = []
    for cfg, f in probs:
        s = cdugks.Solver(cfg, precision=prec, tile_id=tile)
        s.init(f)
        solvers.append(s)
    plain = cdugks.Batch(solvers)
    with pytest.raises(cdugks.CdugksError):
        plain.step_members([1, 1])             # needs the persistent step
    del plain
    b = cdugks.Batch(solvers, persistent=True)
    with pytest.raises(cdugks.CdugksError):
        b.step_members([1])                    # one count per member
    with pytest.raises(cdugks.CdugksError):
        b.step_members([1, -1])
    assert b.sync() == 0
