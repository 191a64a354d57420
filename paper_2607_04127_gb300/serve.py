"""Serving loop for many concurrent mapping sessions (continuous batching).

Every session owns one surfel map whose parameters, gradients and Adam
moments stay resident on the device.  Clients submit render-and-optimise
requests (one keyframe: pose + measured range image + tracking normals,
``iters`` mapping iterations); a client's last request may close its session.

Admission by HBM budget.  A session is charged its resident bytes (the map and
its optimiser state, its share of the workspace, its frame buffers).  One that
fits is admitted; one that does not waits in a first-come queue and is
admitted as soon as closed sessions free enough memory; its requests wait
meanwhile (with ``keep_latest`` only the newest).  Only a session larger than
the whole budget is rejected, and requests of sessions never admitted by the
end of a run count as unserved.

The scheduler runs ticks.  A tick takes every active request one mapping
iteration further with ONE call per stage over all of their frames (each
frame renders its own session's map: ``lgs_*_batch`` with a frame->map
table), then one fused Adam launch over their maps.  Requests that arrived
meanwhile join at the next tick as slots free up (at most ``slots`` active
requests, at most one per session: a session's keyframes update the same map
and are served in arrival order).  A request completes after ``iters`` ticks;
its latency is the time its last tick is seen complete minus its arrival.

Ticks are pipelined: the host enqueues a tick without waiting for the device
(at most ``pipeline`` ticks in flight) and retires finished ticks by polling
their CUDA events.  Each tick copies its loss values and the status word of
its binning into pinned host memory on the stream (lgs_session_status_enqueue),
so no tick needs a host round trip.  The pair capacity of a tick is the sum
of its maps' pair densities (pairs per surfel, each measured once by a
checked binning of the session's first request, the only synchronisation)
times a head-room.  A tick whose binning still overflowed is counted (its
iteration ran on an empty render) and the densities grow.

With ``keep_latest`` a session keeps at most one waiting request: a newer
keyframe supersedes a waiting older one, which is dropped and counted
(mapping always works on the newest keyframe), so queues stay bounded.

With ``slo_ms`` the scheduler admits by deadline: a tick's duration is
modelled as the longer of the device's, ``a`` plus each active map's own cost
per iteration, and the host's enqueueing, a cost per request; both are
learned online from retired ticks (the device time between the ends of
back-to-back ticks, else a tick's own device span, and the host loop's
time per tick while it never idled).  A map's cost starts at a learned rate per binning pair times its
pairs and follows the ticks it runs in.  A waiting request joins only
if the simulated remaining ticks, after those in flight, let every active
request, itself included, finish within ``slo_ms`` of its arrival (with a
safety factor);
otherwise it is rejected at once and counted.

``plain=True`` serves the same requests one at a time with per-request
launches (the baseline the batched form is measured against).
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np
import torch

from . import lib, render

BYTES_PER_SURFEL = 160          # parameters, gradients, Adam m and v: 4 x 10 floats
WORKSPACE_PER_SURFEL = 220      # record, box, keys, counters, moments, about 6 pairs (upper estimate)
FRAME_BYTES_PER_PIXEL = 40      # forward planes, upstream planes, targets


@dataclasses.dataclass
class Request:
    session: int
    frame: object               # scenes.Frame (pose of the keyframe)
    target: object              # scenes.Target
    arrival: float              # seconds since the start of the run
    iters: int = 10
    close: bool = False         # the client's last request: close the session after it
    done_iters: int = 0
    start: float | None = None
    finish: float | None = None
    losses: list = dataclasses.field(default_factory=list)
    degraded: bool = False      # one of its ticks overflowed the pair capacity
    buffers: object = None      # device buffers while active: (target tensors, FwdBuffers, upstream planes)


class MapSession:
    def __init__(self, sid: int, surf, device, need: int):
        self.sid = sid
        self.params = render.map_tensors(surf, device)
        self.grads = [torch.zeros_like(p) for p in self.params]
        n = int(self.params[0].shape[0])
        self.m = torch.zeros(10 * n, device=device)
        self.v = torch.zeros(10 * n, device=device)
        self.t = 0
        self.n = n
        self.need = need            # bytes charged against the budget
        self.closing = False

    @property
    def resident_bytes(self) -> int:
        return BYTES_PER_SURFEL * self.n


def session_bytes(n_surfels: int, frame_pixels: int) -> int:
    """Bytes a session is charged: map and optimiser state, workspace share,
    one frame's buffers."""
    return (BYTES_PER_SURFEL + WORKSPACE_PER_SURFEL) * n_surfels + FRAME_BYTES_PER_PIXEL * frame_pixels


class _Tick:
    """One tick in flight: its requests (in frame order), those whose last
    iteration it runs, CUDA events around it, pinned copies of its losses and
    of its binning's status word."""

    def __init__(self, reqs, items: int, surfels: int):
        self.reqs = list(reqs)
        self.sids = [r.session for r in self.reqs]
        self.last: list[Request] = []
        self.items = items
        self.surfels = surfels
        self.predicted = None           # modelled seconds, when it was enqueued
        self.start = self.end = self.prev_end = None
        self.t_enqueue = 0.0            # host time the tick's enqueueing began
        self.enqueue_seconds = None     # host time its enqueueing took
        self.busy_period = None         # host time since the previous enqueueing, when the loop never idled
        self.host_period = None         # host time since the previous tick's enqueueing began
        self.loss = None
        self.status = None
        self.first = False


class Server:
    def __init__(self, device=0, hbm_budget_bytes: int = 150 << 30, slots: int = 16,
                 tuning: dict | None = None, lr=(1e-3, 1e-3, 5e-3, 5e-3), plain: bool = False,
                 keep_latest: bool = False, slo_ms: float | None = None, slo_margin: float = 0.6,
                 pipeline: int = 2, headroom: float = 1.3):
        self.device = device if isinstance(device, torch.device) else torch.device("cuda", device)
        self.budget = hbm_budget_bytes
        self.slots = 1 if plain else slots
        self.tuning = tuning
        self.lr = lr
        self.plain = plain
        self.pipeline = max(1, int(pipeline))
        self.headroom = headroom
        self.sessions: dict[int, MapSession] = {}
        self.session_queue: collections.deque = collections.deque()   # (sid, surf, need) waiting for memory
        self.rejected_sessions: list[int] = []    # larger than the whole budget
        self.admitted_late: list[int] = []        # waited in the queue, then admitted
        self.closed_sessions: list[int] = []
        self.used = 0
        self.rast = None
        self.keep_latest = keep_latest
        self.dropped: list[Request] = []          # superseded by a newer keyframe of their session
        self.unserved: list[Request] = []         # their session was never admitted (or was closed)
        self.slo = slo_ms / 1e3 if slo_ms else None
        self.slo_margin = slo_margin
        self.late: list[Request] = []             # rejected by the deadline admission
        self.tick_base = 4e-4                     # seconds of a tick independent of the maps
        self.kappa = None                         # seconds per pair-iteration, learned from retired ticks
        self.cost: dict[int, float] = {}          # device seconds per iteration of each session's map
        self.host_per_req = None                  # host seconds to enqueue one request's iteration
        self.overflow_ticks = 0
        self.density: dict[int, float] = {}       # pairs per surfel of each session's binning (probed)
        self._ticks = 0
        self._last_end = None                     # end event of the last enqueued tick
        self._last_enqueue = None                 # host time the last tick's enqueueing began
        self._idled = True                        # the loop slept or waited since the last enqueueing

    # -- admission ------------------------------------------------------------
    def open_session(self, sid: int, surf, frame_pixels: int) -> str:
        """'admitted' (resident now), 'waiting' (queued until memory frees up)
        or 'rejected' (larger than the whole budget)."""
        need = session_bytes(surf.n, frame_pixels)
        if need > self.budget:
            self.rejected_sessions.append(sid)
            return "rejected"
        if not self.session_queue and self.used + need <= self.budget:
            self._admit(sid, surf, need)
            return "admitted"
        self.session_queue.append((sid, surf, need))
        return "waiting"

    def _admit(self, sid, surf, need):
        self.sessions[sid] = MapSession(sid, surf, self.device, need)
        self.used += need

    def _admit_waiting(self):
        """First come, first served: admit queued sessions while the head fits."""
        while self.session_queue and self.used + self.session_queue[0][2] <= self.budget:
            sid, surf, need = self.session_queue.popleft()
            self._admit(sid, surf, need)
            self.admitted_late.append(sid)

    def close_session(self, sid: int):
        """Release a session's map and memory and admit waiting sessions.  The
        caller makes sure no tick of it is in flight (the serving loop closes
        a session when the tick of its last request has retired)."""
        s = self.sessions.pop(sid, None)
        if s is None:
            return
        self.used -= s.need
        self.closed_sessions.append(sid)
        self._admit_waiting()

    def close(self):
        if self.rast is not None:
            self.rast.close()
            self.rast = None
        self.sessions.clear()

    # -- one tick: enqueue, poll, wait, read --------------------------------------
    def _enqueue_tick(self, active) -> _Tick:
        """Enqueue one iteration of every active request: one call per stage
        over their frames, one fused Adam launch over their maps, the status
        word and the losses copied to pinned memory; no host synchronisation
        (but the one-off density probe of a session's first request)."""
        for r in active:
            if r.buffers is None:      # device buffers for the request's lifetime
                r.buffers = (render.target_tensors(r.target, self.device), lib.alloc_fwd(r.frame, self.device),
                             render.upstream_planes(r.frame, self.device))
        maps = [self.sessions[r.session] for r in active]
        tick = _Tick(active, items=sum(s.n for s in maps), surfels=sum(s.n for s in maps))
        tick.t_enqueue = time.perf_counter()
        if self._last_enqueue is not None:
            tick.host_period = tick.t_enqueue - self._last_enqueue
            if not self._idled:
                tick.busy_period = tick.host_period
        self._last_enqueue = tick.t_enqueue
        self._idled = False
        frames = [r.frame for r in active]
        fmap = list(range(len(active)))
        if self.rast is None:
            self.rast = render.Rasterizer(frames, frame_map=fmap, device=self.device.index, tuning=self.tuning)
            self.rast.session.headroom = self.headroom
        probed = [r for r in active if r.session not in self.density]
        for r in probed:
            self._probe(r)
        # pair capacity of this tick: every map at its own density, with head-room
        want = sum(self.sessions[r.session].n * self.density[r.session] for r in active)
        self.rast.session.pairs_per_item = self.headroom * want / max(tick.items, 1)
        self.rast.set_frames(frames, fmap, outs=[r.buffers[1] for r in active], ups=[r.buffers[2] for r in active])
        stream = torch.cuda.current_stream(self.device)
        tick.start = torch.cuda.Event(enable_timing=True)
        tick.end = torch.cuda.Event(enable_timing=True)
        tick.loss = torch.empty(len(active), dtype=torch.float32, pin_memory=True)
        tick.status = torch.zeros(lib.STATUS_WORD_BYTES, dtype=torch.uint8, pin_memory=True)
        tick.first = bool(probed)
        # back to back with the previous tick: the device time between their
        # ends is this tick's period (launch gaps included)
        tick.prev_end = self._last_end if self._last_end is not None and not self._last_end.query() else None
        tick.start.record(stream)
        params = [s.params for s in maps]
        grads = [s.grads for s in maps]      # zero: the previous Adam step cleared them
        out = self.rast.step(params, [r.buffers[0] for r in active], grads, check=False)
        lib.lgs_session_status_enqueue(self.rast.session.handle, tick.status.data_ptr(), stream.cuda_stream)
        k = 1 + lib.LOSS_TERMS * len(active)
        tick.loss.copy_(out[k: k + len(active)], non_blocking=True)
        for s in maps:
            s.t += 1
        render.adam_step_batch([(s.params, s.grads, s.m, s.v, s.t, self.lr) for s in maps], zero_grad=True)
        tick.end.record(stream)
        tick.enqueue_seconds = time.perf_counter() - tick.t_enqueue
        if self.kappa is not None:
            tick.predicted = self._tick_model(tick.sids)
        self._last_end = tick.end
        self._ticks += 1
        return tick

    def _probe(self, r):
        """A session's pair density (pairs per surfel of its binning), measured
        once, the first time one of its requests runs: a checked binning of
        its map alone (it synchronises, and grows the workspace if needed)."""
        s = self.sessions[r.session]
        self.rast.set_frames([r.frame], [0], outs=[r.buffers[1]], ups=[r.buffers[2]])
        self.rast.bin_sort([s.params], check=True)
        _, req = lib.lgs_session_status(self.rast.session.handle)
        self.density[r.session] = req / max(s.n, 1)

    def _tick_ready(self, tick) -> bool:
        return tick.end.query()

    def _wait_tick(self, tick):
        tick.end.synchronize()

    def _read_tick(self, tick):
        """(status, required pairs, device seconds, per-request losses) of a
        completed tick."""
        st, req = lib.lgs_status_of_word(tick.status.data_ptr())
        # device time: from the previous tick's end when the two ran back to
        # back (launch gaps included), else the tick's own span (the host's
        # pace is modelled apart, from its enqueueing time)
        t0 = tick.prev_end if tick.prev_end is not None else tick.start
        seconds = t0.elapsed_time(tick.end) / 1e3
        return st, req, seconds, tick.loss.numpy().tolist()

    def _retire(self, tick, now: float):
        """Book a completed tick: its losses, the completions of its requests'
        last iterations, the capacity and tick models.  Returns the completed
        requests."""
        st, req, seconds, losses = self._read_tick(tick)
        if st == lib.LGS_ERR_CAPACITY:
            # a denser binning than probed: its iteration ran on an empty
            # render (counted); the sessions' densities follow what it needed
            self.overflow_ticks += 1
            est = sum(self.sessions[r.session].n * self.density.get(r.session, 0.0) for r in tick.reqs
                      if r.session in self.sessions)
            grow = max(1.0, req / max(est, 1.0))
            for r in tick.reqs:
                r.degraded = True
                if r.session in self.density:
                    self.density[r.session] *= grow
        elif st != lib.LGS_OK:
            raise lib.LgsError(st, "device status of a serving tick")
        if not tick.first and st == lib.LGS_OK:
            self._learn(tick, seconds)
        for r, l in zip(tick.reqs, losses):
            r.losses.append(float(l))
        done = []
        for r in tick.last:
            r.finish = now
            r.buffers = None
            done.append(r)
            if r.close:
                self.close_session(r.session)
        return done

    # -- deadline admission --------------------------------------------------------
    def _pairs(self, sid) -> float:
        """Pairs of a session's binning: its surfels at its probed density
        (the mean of the probed ones before its first run)."""
        d = self.density.get(sid)
        if d is None:
            d = float(np.mean(list(self.density.values()))) if self.density else 8.0
        return self.sessions[sid].n * d

    def _session_cost(self, sid) -> float:
        c = self.cost.get(sid)
        return c if c is not None else self.kappa * self._pairs(sid)

    def _tick_model(self, sids) -> float:
        """Modelled seconds of a tick over these sessions' maps: the device's
        (a base plus every map's own cost) or the host's enqueueing, which
        paces the device when it is the longer."""
        dev = self.tick_base + sum(self._session_cost(s) for s in sids)
        host = self.host_per_req * len(sids) if self.host_per_req is not None else 0.0
        return max(dev, host)

    def _learn(self, tick, seconds: float):
        """Fit the tick model to a retired tick: the host's cost per request
        from the loop's time since the previous enqueueing when the loop never
        idled in between (else the enqueueing's own time), and from the device
        time the pair rate and every map's own cost, scaled by the damped
        ratio of measured to modelled."""
        host = getattr(tick, "busy_period", None)
        if host is None:
            host = getattr(tick, "enqueue_seconds", None)
        if host is not None:
            h = host / max(len(tick.sids), 1)
            self.host_per_req = h if self.host_per_req is None else 0.5 * self.host_per_req + 0.5 * h
        y = max(seconds - self.tick_base, 0.0)
        pairs = sum(self._pairs(s) for s in tick.sids if s in self.sessions)
        k = y / max(pairs, 1.0)
        self.kappa = k if self.kappa is None else 0.5 * self.kappa + 0.5 * k
        sids = [s for s in tick.sids if s in self.sessions]
        pred = sum(self._session_cost(s) for s in sids)
        if pred > 0:
            f = (y / pred) ** 0.5
            for s in sids:
                self.cost[s] = self._session_cost(s) * f

    def _feasible(self, active, now: float, backlog: float = 0.0) -> bool:
        """Simulate the remaining ticks of ``active`` (no further arrivals),
        after ``backlog`` seconds of ticks already in flight: does every
        request finish within the margin of its deadline?"""
        rem = [(r.iters - r.done_iters, r.session, r.arrival + self.slo_margin * self.slo) for r in active]
        t = now + backlog
        while rem:
            t += self._tick_model([sid for _, sid, _ in rem])
            nxt = []
            for k, sid, dl in rem:
                if k == 1:
                    if t > dl:
                        return False
                else:
                    nxt.append((k - 1, sid, dl))
            rem = nxt
        return True

    # -- the loop -------------------------------------------------------------------
    def run(self, requests):
        """Serve ``requests`` (sorted by arrival; times relative to now).
        Returns the completed requests."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        active, done = [], []
        inflight = collections.deque()
        busy = set()          # sessions with an active request
        t0 = time.perf_counter()
        while pending or waiting or active or inflight:
            # retire the ticks the device has finished (no blocking)
            while inflight and self._tick_ready(inflight[0]):
                done += self._retire(inflight.popleft(), time.perf_counter() - t0)
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                s = self.sessions.get(r.session)
                if r.session in self.rejected_sessions or r.session in self.closed_sessions or (s and s.closing):
                    self.unserved.append(r)
                    continue
                if self.keep_latest:
                    for old in [w for w in waiting if w.session == r.session]:
                        waiting.remove(old)
                        self.dropped.append(old)
                waiting.append(r)
            # fill free slots, at most one request per session, in arrival order;
            # requests of sessions still queued for memory keep waiting
            keep = collections.deque()
            while waiting:
                r = waiting.popleft()
                s = self.sessions.get(r.session)
                if s is not None and s.closing:
                    self.unserved.append(r)
                    continue
                if s is not None and len(active) < self.slots and r.session not in busy:
                    backlog = (sum(t.predicted if t.predicted is not None else self._tick_model(t.sids)
                                   for t in inflight) if self.kappa is not None else 0.0)
                    if self.slo is not None and self.kappa is not None and \
                            not self._feasible(active + [r], now, backlog):
                        self.late.append(r)      # would miss its deadline or make another one miss
                        continue
                    r.start = now
                    active.append(r)
                    busy.add(r.session)
                else:
                    keep.append(r)
            waiting = keep
            if active and len(inflight) < self.pipeline:
                tick = self._enqueue_tick(active)
                still = []
                for r in active:
                    r.done_iters += 1
                    if r.done_iters >= r.iters:
                        # the slot and the session are free for the next tick (the
                        # stream orders that tick after this one)
                        tick.last.append(r)
                        busy.discard(r.session)
                        if r.close:
                            self.sessions[r.session].closing = True
                    else:
                        still.append(r)
                active = still
                inflight.append(tick)
                continue
            if inflight:
                self._idled = True
                self._wait_tick(inflight[0])
                continue
            if pending:
                self._idled = True
                time.sleep(max(0.0, min(pending[0].arrival - now, 0.002)))
            elif waiting:
                # nothing runs and nothing arrives: these sessions' memory never frees up
                self.unserved.extend(waiting)
                waiting.clear()
        return done


def poisson_requests(rng: np.random.Generator, sessions, frames_of, targets_of, duration: float, rate_range=(10, 20),
                     iters: int = 10):
    """Requests of every session as a Poisson stream at a per-session rate
    U(rate_range) Hz over ``duration`` seconds.  ``frames_of(sid, k)`` and
    ``targets_of(sid, k)`` give the k-th keyframe of a session."""
    reqs = []
    for sid in sessions:
        rate = rng.uniform(*rate_range)
        t, k = rng.exponential(1.0 / rate), 0
        while t < duration:
            reqs.append(Request(sid, frames_of(sid, k), targets_of(sid, k), t, iters))
            t += rng.exponential(1.0 / rate)
            k += 1
    return sorted(reqs, key=lambda r: r.arrival)


def latency_stats(done, duration: float, offered: int, rejected_sessions: int, n_sessions: int, dropped: int = 0,
                  late: int = 0, unserved: int = 0, waited_sessions: int = 0, overflow_ticks: int = 0):
    """p50 / p99 latency (ms) of the completed requests, completed frames per
    second of wall time, and the rejections: sessions refused at admission
    (larger than the budget), requests superseded by a newer keyframe of their
    session, requests refused by the deadline admission, requests of sessions
    that were never admitted; sessions that waited for memory."""
    lat = np.array([r.finish - r.arrival for r in done]) * 1e3
    wall = max([r.finish for r in done] + [duration])
    return dict(completed=len(done), offered=offered, p50_ms=float(np.percentile(lat, 50)) if len(lat) else None,
                p99_ms=float(np.percentile(lat, 99)) if len(lat) else None,
                frames_per_s=len(done) / wall, rejected_sessions=rejected_sessions,
                session_rejection_rate=rejected_sessions / max(n_sessions, 1), waited_sessions=waited_sessions,
                dropped_requests=dropped, deadline_rejected=late, unserved_requests=unserved,
                request_rejection_rate=(dropped + late + unserved) / max(offered, 1),
                overflow_ticks=overflow_ticks)
