"""The serving loop: continuous batching with admission by device-memory footprint.

Host-side parts run on CPU; the GPU tests check that every request's result is
the same alone and in the mix, and that admission never exceeds the budget."""
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


@pytest.mark.gpu
def test_each_result_is_the_same_alone_and_in_the_mix():
    reqs = [_req(0, 24, 8, "kh", 0.0, t_end=0.006), _req(1, 20, 12, "gresho", 0.0, t_end=0.004),
            _req(2, 28, 8, "gresho", 0.01, t_end=0.005), _req(3, 16, 16, "kh", 0.02, t_end=0.003)]
    srv = serving.Server(budget_bytes=8 << 30, max_round=3)
    done = srv.run(reqs)
    assert len(done) == 4
    for q in done:
        s = cdugks.Solver(q.cfg, precision=q.precision)
        s.init(q.fields)
        s.step(q.nsteps)
        assert q.done_steps == q.nsteps
        assert np.array_equal(s.moments(), q.result), q.rid


@pytest.mark.gpu
def test_admission_respects_the_memory_budget():
    reqs = [_req(k, 24, 8, "kh", 0.0, t_end=0.003) for k in range(5)]
    one = serving.footprint_bytes(reqs[0])
    srv = serving.Server(budget_bytes=2 * one + one // 2, max_round=2)
    peak = {"active": 0}
    orig = srv._round

    def watched():
        peak["active"] = max(peak["active"], len(srv.active))
        assert srv.used <= srv.budget
        orig()

    srv._round = watched
    done = srv.run(reqs)
    assert len(done) == 5
    assert peak["active"] == 2
