"""Serving loop: admission by the HBM budget, continuous batching across
sessions, and every request's result the same alone and in the mix."""
import numpy as np
import pytest

from paper_2607_04127_gb300 import scenes

pytestmark = pytest.mark.gpu

SIZES = [3000, 6000, 12000, 5000]
SHAPES = [(32, 256), (32, 512)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_04127_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def workload():
    return scenes.street_maps(5, SIZES, SHAPES, tile=(8, 8))


def _requests(workload, sids, iters=4):
    from paper_2607_04127_gb300 import serve
    reqs = []
    for sid in sids:
        surf, fr, tgt = workload[sid]
        for k in range(2):         # two keyframes per session, both queued at t = 0
            reqs.append(serve.Request(sid, fr, tgt, 0.0, iters))
    return reqs


def _serve(workload, sids, **kw):
    from paper_2607_04127_gb300 import serve
    srv = serve.Server(**kw)
    for sid in sids:
        surf, fr, _ = workload[sid]
        assert srv.open_session(sid, surf, fr.H * fr.W) == "admitted"
    done = srv.run(_requests(workload, sids))
    params = {sid: [p.cpu().numpy() for p in srv.sessions[sid].params] for sid in sids}
    losses = {}
    for r in sorted(done, key=lambda r: (r.session, r.start)):
        losses.setdefault(r.session, []).extend(r.losses)
    srv.close()
    return done, params, losses


def test_results_same_alone_and_in_the_mix(workload):
    sids = list(range(len(SIZES)))
    done, params, losses = _serve(workload, sids, slots=8)
    assert len(done) == 2 * len(sids)
    for sid in sids:
        _, p1, l1 = _serve(workload, [sid], slots=8)
        # the first iteration renders identical inputs: identical loss; later
        # ones differ only through the order of float atomics in the
        # gradients.  Many of these small maps' surfels sit at the scale clip
        # s_max, so after an Adam step each is in or out of the summed scale
        # regulariser's hinge (10 x 0.005 per surfel on a loss near 100): a
        # few hinge decisions taken the other way move the loss by ~1e-3
        assert l1[sid][0] == losses[sid][0]
        assert np.allclose(l1[sid], losses[sid], rtol=1e-2)
        for a, b in zip(params[sid], p1[sid]):
            d = np.abs(a - b)
            assert np.mean(d <= 1e-6 + 1e-6 * np.abs(b)) > 0.99
            assert d.max() <= 2 * 8 * 5e-3       # at most a few Adam steps apart


def test_plain_server_matches_batched(workload):
    sids = list(range(len(SIZES)))
    _, pb, lb = _serve(workload, sids, slots=8)
    _, pp, lp = _serve(workload, sids, plain=True)
    for sid in sids:
        # the first iteration renders identical inputs: identical loss; the
        # later ones differ through the order of float atomics in the
        # gradients, amplified by the scale regulariser's hinge (see above)
        assert lp[sid][0] == lb[sid][0]
        assert np.allclose(lp[sid], lb[sid], rtol=1e-2), (sid, lp[sid], lb[sid])


def test_admission_by_budget(workload):
    """A budget for two sessions: a third waits in the queue, a session
    larger than the whole budget is rejected."""
    from paper_2607_04127_gb300 import serve
    surf, fr, _ = workload[2]
    one = serve.session_bytes(surf.n, fr.H * fr.W)
    srv = serve.Server(hbm_budget_bytes=int(2.5 * one))
    assert srv.open_session(0, surf, fr.H * fr.W) == "admitted"
    assert srv.open_session(1, surf, fr.H * fr.W) == "admitted"
    assert srv.open_session(2, surf, fr.H * fr.W) == "waiting"
    big = scenes.street_maps(6, [4 * surf.n], [SHAPES[0]], tile=(8, 8))[0][0]
    assert srv.open_session(3, big, fr.H * fr.W) == "rejected"
    assert srv.rejected_sessions == [3] and [q[0] for q in srv.session_queue] == [2]
    srv.close()


def test_waiting_session_is_admitted_when_one_closes(workload):
    """Session 2 waits for memory; session 0's client closes it after its
    request; session 2 is then admitted, its request (queued since t = 0)
    runs after session 0's, and its losses equal those of a solo run."""
    from paper_2607_04127_gb300 import serve
    surf, fr, tgt = workload[2]
    one = serve.session_bytes(surf.n, fr.H * fr.W)
    srv = serve.Server(hbm_budget_bytes=int(2.5 * one), slots=8)
    for sid in (0, 1):
        assert srv.open_session(sid, surf, fr.H * fr.W) == "admitted"
    assert srv.open_session(2, surf, fr.H * fr.W) == "waiting"
    reqs = [serve.Request(0, fr, tgt, 0.0, 3, close=True), serve.Request(1, fr, tgt, 0.0, 3),
            serve.Request(2, fr, tgt, 0.0, 3)]
    done = srv.run(reqs)
    assert len(done) == 3 and not srv.unserved
    assert srv.closed_sessions == [0] and srv.admitted_late == [2]
    assert reqs[2].start >= reqs[0].finish
    assert srv.used <= srv.budget
    srv.close()
    solo = serve.Server(slots=8)
    assert solo.open_session(2, surf, fr.H * fr.W) == "admitted"
    alone = serve.Request(2, fr, tgt, 0.0, 3)
    solo.run([alone])
    solo.close()
    # the first loss is a pure function of the admitted map and frame;
    # later ones follow Adam steps on gradients summed with float atomics in
    # a run-dependent order, and Adam (eps 1e-15: nearly a sign step) turns
    # a near-zero gradient's sign into a full step, so a trajectory as
    # unstable as this one (1.6 -> 124 -> 100) agrees to about 1e-3
    assert alone.losses[0] == reqs[2].losses[0]
    assert np.allclose(alone.losses, reqs[2].losses, rtol=1e-2)


def test_poisson_stream_latency_stats(workload):
    from paper_2607_04127_gb300 import serve
    rng = np.random.default_rng(0)
    sids = list(range(len(SIZES)))
    srv = serve.Server(slots=8)
    for sid in sids:
        surf, fr, _ = workload[sid]
        srv.open_session(sid, surf, fr.H * fr.W)
    reqs = serve.poisson_requests(rng, sids, lambda s, k: workload[s][1], lambda s, k: workload[s][2], 0.5,
                                  iters=3)
    done = srv.run(reqs)
    st = serve.latency_stats(done, 0.5, len(reqs), 0, len(sids))
    assert st["completed"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()


def test_keep_latest_supersedes_waiting_keyframes(workload):
    from paper_2607_04127_gb300 import serve
    surf, fr, tgt = workload[0]
    srv = serve.Server(slots=4, keep_latest=True)
    srv.open_session(0, surf, fr.H * fr.W)
    reqs = [serve.Request(0, fr, tgt, 0.0, 2) for _ in range(3)]
    done = srv.run(reqs)
    assert len(done) == 1 and done[0] is reqs[2] and len(srv.dropped) == 2
    srv.close()


def test_deadline_admission(workload):
    """With a deadline, requests the tick model says would finish late are
    refused at once; the others complete, and every offered request is
    accounted for.  A generous deadline refuses nothing."""
    from paper_2607_04127_gb300 import serve
    sids = list(range(len(SIZES)))

    def run(slo_ms, waves=3):
        # admission against the whole deadline (margin 1): the default margin
        # keeps back a share of it for the tail, which this test does not study
        srv = serve.Server(slots=8, slo_ms=slo_ms, slo_margin=1.0)
        for sid in sids:
            surf, fr, _ = workload[sid]
            srv.open_session(sid, surf, fr.H * fr.W)
        # calibrate the tick model (first runs: warm-up), and time one request alone
        for _ in range(3):
            srv.run([serve.Request(2, workload[2][1], workload[2][2], 0.0, 4)])
        cal = serve.Request(2, workload[2][1], workload[2][2], 0.0, 4)
        srv.run([cal])
        srv.late.clear()
        # `waves` keyframes per session, all queued at t = 0 (one active per session)
        reqs = [serve.Request(sid, workload[sid][1], workload[sid][2], 0.0, 4) for _ in range(waves) for sid in sids]
        done = srv.run(reqs)
        late = list(srv.late)
        srv.close()
        return reqs, done, late, (cal.finish - cal.arrival) * 1e3

    reqs, done, late, alone_ms = run(10_000.0)
    assert not late and len(done) == len(reqs)
    # 1.5 x the time of the largest map alone: a first wave can fit, a third
    # wave (after two earlier requests of its session) cannot
    reqs, done, late, _ = run(1.5 * alone_ms)
    assert done and late
    assert len(done) + len(late) == len(reqs)
    assert not set(map(id, done)) & set(map(id, late))
    third = {id(r) for r in reqs[2 * len(sids):]}
    assert third <= set(map(id, late))
