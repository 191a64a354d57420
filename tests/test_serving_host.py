"""Host logic of the serving loop's deadline admission (no GPU): the
simulation of the remaining ticks that decides whether a request may join."""
import types

import pytest

from paper_2607_04127_gb300 import serve


def _server(kappa=1e-8, base=1e-3, slo_ms=50.0, margin=1.0):
    srv = serve.Server(slo_ms=slo_ms, slo_margin=margin)
    srv.kappa, srv.tick_base = kappa, base
    return srv


def _req(srv, sid, n, arrival, iters, done=0):
    srv.sessions[sid] = types.SimpleNamespace(n=n)
    srv.density[sid] = 1.0      # one binning pair per surfel: the model's cost is kappa * n
    r = serve.Request(sid, None, None, arrival, iters)
    r.done_iters = done
    return r


def test_single_request_deadline_by_tick_model():
    # a tick costs base + kappa * n = 1 ms + 1e-8 * 4e5 = 5 ms: ten ticks take 50 ms
    srv = _server()
    assert srv._feasible([_req(srv, 0, 400_000, 0.0, 10)], 0.0)          # exactly 50 ms
    assert not srv._feasible([_req(srv, 0, 400_000, 0.0, 10)], 0.001)    # 1 ms later: 51 ms
    assert not srv._feasible([_req(srv, 0, 500_000, 0.0, 10)], 0.0)      # 6 ms ticks: 60 ms


def test_batch_ticks_slow_every_member_until_it_leaves():
    srv = _server()
    a = _req(srv, 0, 200_000, 0.0, 10, done=8)    # 2 iterations left, deadline 50 ms
    b = _req(srv, 1, 200_000, 0.0, 10)            # 10 left
    # together: ticks of 1 + 4 = 5 ms while both run (2 ticks), then 3 ms ticks
    # for b alone: a ends at 10 ms, b at 10 + 8 * 3 = 34 ms
    assert srv._feasible([a, b], 0.0)
    c = _req(srv, 2, 600_000, 0.0, 10)            # adds 6 ms to every shared tick
    assert not srv._feasible([a, b, c], 0.0)
    # the margin scales the deadline: 34 ms does not fit 0.6 x 50 ms
    srv.slo_margin = 0.6
    assert not srv._feasible([a, b], 0.0)


def _tick(sids, host_period=None, paced_by_host=False, enqueue_seconds=None):
    return types.SimpleNamespace(sids=list(sids), host_period=host_period, enqueue_seconds=enqueue_seconds,
                                 prev_end=None if paced_by_host else object())


def test_map_costs_are_learned_per_session():
    # two maps of the same size whose iterations cost 2 ms and 6 ms on the
    # device: ticks that run them alone separate their costs, and a tick of
    # both is modelled as the sum
    srv = _server(kappa=None, base=1e-3)
    _req(srv, 0, 100_000, 0.0, 10)
    _req(srv, 1, 100_000, 0.0, 10)
    for _ in range(12):
        srv._learn(_tick([0]), 1e-3 + 2e-3)
        srv._learn(_tick([1]), 1e-3 + 6e-3)
    assert srv._tick_model([0]) == pytest.approx(3e-3, rel=0.1)
    assert srv._tick_model([1]) == pytest.approx(7e-3, rel=0.1)
    assert srv._tick_model([0, 1]) == pytest.approx(9e-3, rel=0.1)


def test_host_paced_ticks_set_a_floor_per_request():
    # the host needed 10 ms to enqueue a tick of two requests: a tick of four
    # is modelled at no less than 20 ms; time the host spent idle between
    # ticks (a long interval before a host-paced tick) does not count
    srv = _server(kappa=1e-9, base=1e-3)
    for k in range(4):
        _req(srv, k, 1000, 0.0, 10)
    srv._learn(_tick([0, 1], host_period=0.5, paced_by_host=True, enqueue_seconds=10e-3), 10e-3)
    assert 20e-3 * 0.999 <= srv._tick_model([0, 1, 2, 3]) <= 21e-3


def test_latency_stats_count_deadline_rejections():
    done = [types.SimpleNamespace(finish=0.02 * (i + 1), arrival=0.0) for i in range(4)]
    st = serve.latency_stats(done, 1.0, offered=10, rejected_sessions=0, n_sessions=2, dropped=2, late=3)
    assert st["deadline_rejected"] == 3 and st["request_rejection_rate"] == pytest.approx(0.5)
    assert st["p50_ms"] == pytest.approx(50.0) and st["completed"] == 4


# --- session admission by memory, with a fake tick (no GPU) -----------------------
import numpy as np
import torch

from paper_2607_04127_gb300 import lib, scenes


class FakeServer(serve.Server):
    """The serving loop with the device work replaced by a log: a tick
    records which sessions it ran and completes when waited for."""

    def __init__(self, ready=True, **kw):
        super().__init__(device=torch.device("cpu"), **kw)
        self.log, self.ready, self.outstanding, self.max_outstanding = [], ready, 0, 0
        self.used_peak = 0

    def _admit(self, sid, surf, need):
        super()._admit(sid, surf, need)
        self.used_peak = max(self.used_peak, self.used)

    def _enqueue_tick(self, active):
        t = serve._Tick(active, items=sum(self.sessions[r.session].n for r in active), surfels=0)
        t.first = self._ticks == 0
        self._ticks += 1
        t.done = self.ready
        self.log.append(sorted(r.session for r in active))
        self.outstanding += 1
        self.max_outstanding = max(self.max_outstanding, self.outstanding)
        return t

    def _tick_ready(self, t):
        return t.done

    def _wait_tick(self, t):
        t.done = True

    def _read_tick(self, t):
        self.outstanding -= 1
        return lib.LGS_OK, 6 * t.items, 1e-3, [float(r.session) for r in t.reqs]


def _surf(n, seed=0):
    rng = np.random.default_rng(seed)
    return scenes.Surfels(rng.normal(size=(n, 3)).astype(np.float32), rng.normal(size=(n, 4)).astype(np.float32),
                          np.full((n, 2), -3.0, np.float32), np.zeros(n, np.float32))


def test_a_session_waits_for_memory_and_is_admitted_when_another_closes():
    s = _surf(100)
    one = serve.session_bytes(100, 64)
    srv = FakeServer(hbm_budget_bytes=int(2.5 * one), slots=8)
    assert [srv.open_session(k, s, 64) for k in range(3)] == ["admitted", "admitted", "waiting"]
    reqs = [serve.Request(0, None, None, 0.0, 2, close=True), serve.Request(1, None, None, 0.0, 4),
            serve.Request(2, None, None, 0.0, 2)]
    done = srv.run(reqs)
    assert {r.session for r in done} == {0, 1, 2} and not srv.unserved
    assert srv.closed_sessions == [0] and srv.admitted_late == [2]
    # session 2 joins only after session 0's last tick has retired
    assert srv.log[:2] == [[0, 1], [0, 1]] and 2 not in srv.log[1] and [1, 2] in srv.log
    assert reqs[2].start >= reqs[0].finish
    assert srv.used_peak <= srv.budget and srv.used == 2 * one


def test_requests_of_a_session_never_admitted_are_unserved_and_counted():
    s = _surf(100)
    one = serve.session_bytes(100, 64)
    srv = FakeServer(hbm_budget_bytes=int(2.5 * one), slots=8)
    for k in range(3):
        srv.open_session(k, s, 64)
    reqs = [serve.Request(k, None, None, 0.0, 2) for k in range(3)]
    done = srv.run(reqs)
    assert {r.session for r in done} == {0, 1} and srv.unserved == [reqs[2]]
    st = serve.latency_stats(done, 1.0, offered=3, rejected_sessions=0, n_sessions=3, unserved=len(srv.unserved))
    assert st["request_rejection_rate"] == pytest.approx(1 / 3) and st["unserved_requests"] == 1


def test_a_session_larger_than_the_budget_is_rejected():
    srv = FakeServer(hbm_budget_bytes=serve.session_bytes(100, 64))
    assert srv.open_session(0, _surf(101), 64) == "rejected"
    assert srv.open_session(1, _surf(100), 64) == "admitted"
    assert srv.rejected_sessions == [0]
    done = srv.run([serve.Request(0, None, None, 0.0, 1), serve.Request(1, None, None, 0.0, 1)])
    assert [r.session for r in done] == [1] and [r.session for r in srv.unserved] == [0]


def test_requests_after_a_closing_request_are_unserved():
    s = _surf(50)
    srv = FakeServer(slots=4)
    srv.open_session(0, s, 64)
    reqs = [serve.Request(0, None, None, 0.0, 2, close=True), serve.Request(0, None, None, 0.0, 2)]
    done = srv.run(reqs)
    assert done == [reqs[0]] and srv.unserved == [reqs[1]] and 0 not in srv.sessions


def test_ticks_in_flight_never_exceed_the_pipeline_depth():
    """Ticks the device has not finished are waited for only when the
    pipeline is full: at most `pipeline` are outstanding, and with depth 2 a
    second tick is enqueued before the first is waited for."""
    s = _surf(50)
    for depth in (1, 2, 3):
        srv = FakeServer(ready=False, slots=4, pipeline=depth)
        srv.open_session(0, s, 64)
        srv.open_session(1, s, 64)
        done = srv.run([serve.Request(0, None, None, 0.0, 5), serve.Request(1, None, None, 0.0, 3)])
        assert len(done) == 2 and srv.max_outstanding == depth
        assert done[0].losses == [0.0] * 5 or done[0].losses == [1.0] * 3
