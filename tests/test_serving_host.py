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


def test_latency_stats_count_deadline_rejections():
    done = [types.SimpleNamespace(finish=0.02 * (i + 1), arrival=0.0) for i in range(4)]
    st = serve.latency_stats(done, 1.0, offered=10, rejected_sessions=0, n_sessions=2, dropped=2, late=3)
    assert st["deadline_rejected"] == 3 and st["request_rejection_rate"] == pytest.approx(0.5)
    assert st["p50_ms"] == pytest.approx(50.0) and st["completed"] == 4
