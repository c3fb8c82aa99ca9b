"""The serving loop: continuous batching with admission by device-memory footprint.

Host-side parts run on CPU (the scheduler against fake solvers and batches);
the GPU tests check that every request's result is the same alone and in the
mix, with the persistent batched step (each member its own steps per round)
and with one launch per kernel, and that admission never exceeds the budget."""
import threading

import numpy as np
import pytest

from paper_2208_09132_gb300 import cdugks, serving, workloads as wl


def _req(rid, n, nv, kind, arrival, t_end=0.004, kn=1e-3):
    if kind == "kh":
        cfg, f = wl.kelvin_helmholtz(n=n, nv=nv, kn=kn)
    else:
        cfg, f = wl.gresho(n=n, nv=nv, kn=kn)
    return serving.Request(rid=rid, cfg=cfg, fields=f, t_end=t_end, arrival=arrival)


def test_footprint_and_step_count_on_host():
    r = _req(0, 24, 8, "kh", 0.0)
    b = serving.footprint_bytes(r)
    assert b > 2 * 24 * 24 * 64 * 2 * 4          # at least the two state buffers
    assert r.nsteps >= 1
    # a larger grid needs more memory
    r2 = _req(1, 48, 8, "kh", 0.0)
    assert serving.footprint_bytes(r2) > b


def test_stream_is_seeded_and_poisson_ordered():
    a = serving.stream_c5(count=20)
    b = serving.stream_c5(count=20)
    assert [q.arrival for q in a] == [q.arrival for q in b]
    assert all(x.arrival <= y.arrival for x, y in zip(a, a[1:]))
    assert {q.cfg["name"].split("_")[0] for q in a} <= {"gresho", "kh"}
    # the stated ranges: grid sides 64..512, velocity sides 16..48, to t = 1
    assert all(64 <= q.cfg["n"][0] <= 512 and 16 <= q.cfg["nv"][0] <= 48 and q.t_end == 1.0 for q in a)


# ------------------------------------------------- the scheduler on the host

class _FakeEvent:
    def __init__(self, enable_timing=False):
        self.ms = 0.0

    def record(self, stream=None):
        pass

    def query(self):
        return True

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return 1.0


class _FakeSolver:
    log = []

    def __init__(self, cfg, precision=None, device=None, tile_id=0, velocity_groups=0, stream=None):
        self.cfg = cfg
        self.tile_id = tile_id
        self.steps = 0
        self.thread = None

    def init(self, f):
        self.thread = threading.current_thread().name
        self.f = np.asarray(f)

    def moments(self):
        return np.full((1, 4), float(self.steps))


class _FakeBatch:
    instances = []

    def __init__(self, solvers, device=None, persistent=False, max_members=0, max_items=0):
        self.members = list(solvers)
        self.persistent = persistent
        self.stream = None
        self.calls = []
        _FakeBatch.instances.append(self)

    def admit(self, s):
        self.members.append(s)

    def retire(self, s):
        assert len(self.members) > 1
        self.members.remove(s)

    def step_members(self, steps):
        assert len(steps) == len(self.members) and all(n >= 0 for n in steps)
        self.calls.append(("members", list(steps)))
        for s, n in zip(self.members, steps):
            s.steps += n

    def step(self, n):
        self.calls.append(("all", n))
        for s in self.members:
            s.steps += n

    def sync(self):
        return 0


@pytest.fixture
def fake_gpu(monkeypatch):
    import torch

    steps = {}

    def footprint(req):
        req.nsteps = steps[req.rid]
        return 1000

    monkeypatch.setattr(serving, "footprint_bytes", footprint)
    monkeypatch.setattr(serving, "persistent_tile", lambda p, d: 6)
    monkeypatch.setattr(cdugks, "Solver", _FakeSolver)
    monkeypatch.setattr(cdugks, "Batch", _FakeBatch)
    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: None)
    _FakeBatch.instances.clear()
    return steps


@pytest.mark.parametrize("persistent", [True, False])
def test_scheduler_never_runs_a_member_past_its_steps(fake_gpu, persistent):
    """Uneven step counts and staggered arrivals: every request ends with
    exactly its own step count, results are read back, the batch keeps at least
    one member, preparation runs on the worker thread, and with the persistent
    step a round gives each member min(round, remaining) steps."""
    nst = [7, 3, 12, 1, 5, 9]
    reqs = []
    for k, n in enumerate(nst):
        fake_gpu[k] = n
        q = _req(k, 16, 8, "kh", arrival=0.002 * k)
        reqs.append(q)
    srv = serving.Server(budget_bytes=3500, max_slots=3, max_round=4, persistent=persistent,
                         round_target_s=1e9)
    done = srv.run(reqs, time_limit=30.0)
    assert sorted(q.rid for q in done) == list(range(len(nst)))
    for q in done:
        assert q.done_steps == q.nsteps
        assert q.result[0, 0] == q.nsteps          # the solver advanced exactly nsteps
        assert q.solver is None                    # workspace released
    assert srv.used == 0
    b_calls = [c for b in _FakeBatch.instances for c in b.calls]
    if persistent:
        assert all(kind == "members" and max(v) <= 4 for kind, v in b_calls)
    else:
        assert all(kind == "all" and v <= 4 for kind, v in b_calls)
    assert srv.report()["finished"] == len(nst)


def test_srpt_lets_short_requests_overtake(fake_gpu):
    """Shortest remaining work first with room for one request per round: a
    short request that arrives while a long one runs finishes first; the long
    one steps out of the batch meanwhile (stays resident) and completes later
    with exactly its own steps."""
    fake_gpu[0] = 400
    fake_gpu[1] = 6
    fake_gpu[2] = 3
    reqs = [_req(0, 16, 8, "kh", 0.0), _req(1, 16, 8, "kh", 0.01), _req(2, 16, 8, "kh", 0.02)]
    srv = serving.Server(budget_bytes=10 ** 6, max_round=2, round_target_s=1e9, fill_points=1)
    real_launch = srv._launch
    sizes = []

    def slow_launch():
        sizes.append(len(srv.active))
        import time
        time.sleep(0.001)                      # rounds take time, so the later arrivals meet the long one
        return real_launch()

    srv._launch = slow_launch
    done = srv.run(reqs, time_limit=30.0)
    order = [q.rid for q in done]
    assert order.index(1) < order.index(0) and order.index(2) < order.index(0)
    assert all(q.done_steps == q.nsteps and q.result[0, 0] == q.nsteps for q in done)
    assert max(sizes) == 1                     # one member per round: the shortest
    assert srv.membership_changes >= 2


def test_share_policy_steps_every_resident_request(fake_gpu):
    for k in range(4):
        fake_gpu[k] = 5 + k
    reqs = [_req(k, 16, 8, "kh", 0.0) for k in range(4)]
    srv = serving.Server(budget_bytes=10 ** 6, max_round=2, round_target_s=1e9, policy="share")
    done = srv.run(reqs, time_limit=30.0)
    assert sorted(q.rid for q in done) == [0, 1, 2, 3]
    assert all(q.done_steps == q.nsteps for q in done)
    with pytest.raises(ValueError):
        serving.Server(budget_bytes=1, policy="lifo")


def test_scheduler_respects_budget_and_slots(fake_gpu):
    for k in range(7):
        fake_gpu[k] = 2 + k % 3
    reqs = [_req(k, 16, 8, "gresho", arrival=0.0) for k in range(7)]
    srv = serving.Server(budget_bytes=2500, max_slots=4, max_round=2, round_target_s=1e9)
    peak = {"used": 0, "members": 0}
    orig = srv._launch

    def watched():
        peak["used"] = max(peak["used"], srv.used)
        peak["members"] = max(peak["members"], len(srv.active))
        return orig()

    srv._launch = watched
    done = srv.run(reqs)
    assert len(done) == 7
    assert peak["used"] <= 2500 and peak["members"] <= 2     # two footprints of 1000 fit the budget


def test_scheduler_time_limit_stops_cleanly(fake_gpu):
    fake_gpu[0] = 10 ** 9
    fake_gpu[1] = 2
    reqs = [_req(0, 16, 8, "kh", 0.0), _req(1, 16, 8, "kh", 0.0)]
    srv = serving.Server(budget_bytes=10 ** 6, max_round=3, round_target_s=1e9)
    done = srv.run(reqs, time_limit=0.2)
    assert [q.rid for q in done] == [1]
    rep = srv.report()
    assert rep["finished"] == 1 and rep["unfinished"] == 1
    assert 0 < reqs[0].done_steps < reqs[0].nsteps


# -------------------------------------------------------------------- GPU

@pytest.mark.gpu
@pytest.mark.parametrize("persistent,policy,fill", [(True, "srpt", 3e7), (True, "srpt", 1.0), (True, "share", 3e7),
                                                    (False, "srpt", 1.0), (False, "share", 3e7)])
def test_each_result_is_the_same_alone_and_in_the_mix(persistent, policy, fill):
    """fill = 1 point: one request per round, so members step out of the batch
    and back in (membership rewritten in place) between their rounds."""
    reqs = [_req(0, 24, 8, "kh", 0.0, t_end=0.006), _req(1, 20, 12, "gresho", 0.0, t_end=0.004),
            _req(2, 28, 8, "gresho", 0.01, t_end=0.005), _req(3, 16, 16, "kh", 0.02, t_end=0.003)]
    srv = serving.Server(budget_bytes=8 << 30, max_round=3, persistent=persistent, policy=policy, fill_points=fill)
    done = srv.run(reqs)
    assert len(done) == 4
    for q in done:
        s = cdugks.Solver(q.cfg, precision=q.precision, tile_id=q.tile_id, velocity_groups=q.velocity_groups)
        s.init(q.fields)
        s.step(q.nsteps)
        assert q.done_steps == q.nsteps
        assert np.array_equal(s.moments(), q.result), q.rid


@pytest.mark.gpu
def test_admission_respects_the_memory_budget():
    """Five requests and room for two: the device memory held by prepared,
    running and retiring requests never exceeds the budget, and reaches two
    footprints (the worker prepares the next request as soon as it fits)."""
    reqs = [_req(k, 24, 8, "kh", 0.0, t_end=0.003) for k in range(5)]
    srv = serving.Server(budget_bytes=1, max_round=2)
    with pytest.raises(ValueError):
        srv.submit(reqs[0])
    one = reqs[0].footprint
    srv = serving.Server(budget_bytes=2 * one + one // 2, max_round=2)
    peak = {"used": 0}
    orig = srv._host_work

    def watched(now):
        r = orig(now)
        peak["used"] = max(peak["used"], srv.used)
        assert srv.used <= srv.budget
        return r

    srv._host_work = watched
    done = srv.run(reqs)
    assert len(done) == 5
    assert peak["used"] == 2 * one
    assert srv.used == 0


@pytest.mark.gpu
def test_server_mixes_collision_models_and_forces():
    """Two-time, Shakhov and accelerated requests served together (one
    launch per kernel: the batch holds several tile shapes), each equal to its
    solve alone."""
    base = [_req(0, 24, 12, "kh", 0.0, t_end=0.005), _req(1, 20, 12, "gresho", 0.0, t_end=0.004),
            _req(2, 28, 10, "kh", 0.005, t_end=0.004), _req(3, 18, 12, "gresho", 0.01, t_end=0.003)]
    base[1].cfg["collision"] = wl.COLLISION_SHAKHOV
    base[2].cfg["accel"] = [0.0, -0.5, 0.0]
    base[3].cfg["collision"] = wl.COLLISION_SHAKHOV
    srv = serving.Server(budget_bytes=8 << 30, max_round=2, persistent=False)
    done = srv.run(base)
    assert len(done) == 4
    for q in done:
        s = cdugks.Solver(q.cfg, precision=q.precision, tile_id=q.tile_id, velocity_groups=q.velocity_groups)
        s.init(q.fields)
        s.step(q.nsteps)
        assert np.array_equal(s.moments(), q.result), q.rid
