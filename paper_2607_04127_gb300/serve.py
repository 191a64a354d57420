"""Serving loop for many concurrent mapping sessions (continuous batching).

Every session owns one surfel map whose parameters, gradients and Adam
moments stay resident on the device.  Clients submit render-and-optimise
requests (one keyframe: pose + measured range image + tracking normals,
``iters`` mapping iterations).  Sessions are admitted against an HBM budget
(resident bytes of the map and its optimiser state plus the per-frame
buffers); a session that does not fit is rejected.

The scheduler runs ticks.  A tick takes every active request one mapping
iteration further with ONE call per stage over all of their frames (each
frame renders its own session's map: ``lgs_*_batch`` with a frame->map
table), then one Adam step per map.  Requests that arrived meanwhile join at
the next tick as slots free up (at most ``slots`` active requests, at most
one per session: a session's keyframes update the same map and are served in
arrival order).  A request completes after ``iters`` ticks; its latency is
completion time minus arrival time.  With ``keep_latest`` a session keeps at
most one waiting request: a newer keyframe supersedes a waiting older one,
which is dropped and counted (mapping always works on the newest keyframe),
so queues stay bounded under overload.

With ``slo_ms`` the scheduler admits by deadline: a tick's duration is
modelled as ``a + kappa * (surfels of its active maps)`` with ``kappa``
learned online from measured ticks, and a waiting request joins only if the
simulated remaining ticks let every active request, itself included, finish
within ``slo_ms`` of its arrival (with a safety factor); otherwise it is
rejected at once and counted.  Completed requests then meet the latency
target by construction of the admission, at the price of the reported
rejection rate.

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


@dataclasses.dataclass
class Request:
    session: int
    frame: object               # scenes.Frame (pose of the keyframe)
    target: object              # scenes.Target
    arrival: float              # seconds since the start of the run
    iters: int = 10
    done_iters: int = 0
    start: float | None = None
    finish: float | None = None
    losses: list = dataclasses.field(default_factory=list)
    buffers: object = None      # device buffers while active: (target tensors, FwdBuffers, upstream planes)


class MapSession:
    def __init__(self, sid: int, surf, device):
        self.sid = sid
        self.params = render.map_tensors(surf, device)
        self.grads = [torch.zeros_like(p) for p in self.params]
        n = int(self.params[0].shape[0])
        self.m = torch.zeros(10 * n, device=device)
        self.v = torch.zeros(10 * n, device=device)
        self.t = 0
        self.n = n

    @property
    def resident_bytes(self) -> int:
        return BYTES_PER_SURFEL * self.n


class Server:
    def __init__(self, device: int = 0, hbm_budget_bytes: int = 150 << 30, slots: int = 16,
                 tuning: dict | None = None, lr=(1e-3, 1e-3, 5e-3, 5e-3), plain: bool = False,
                 keep_latest: bool = False, slo_ms: float | None = None, slo_margin: float = 0.8):
        self.device = torch.device("cuda", device)
        self.budget = hbm_budget_bytes
        self.slots = 1 if plain else slots
        self.tuning = tuning
        self.lr = lr
        self.plain = plain
        self.sessions: dict[int, MapSession] = {}
        self.rejected_sessions: list[int] = []
        self.used = 0
        self.rast = None
        self.keep_latest = keep_latest
        self.dropped: list[Request] = []
        self.slo = slo_ms / 1e3 if slo_ms else None
        self.slo_margin = slo_margin
        self.late: list[Request] = []      # rejected by the deadline admission
        self.tick_base = 4e-4              # seconds of a tick independent of the maps (host work, launches)
        self.kappa = None                  # seconds per surfel-iteration, learned from measured ticks
        self._ticks = 0
        self._grew = False                 # the last tick grew the workspace (and ran twice)

    # -- admission ----------------------------------------------------------
    def open_session(self, sid: int, surf, frame_pixels: int) -> bool:
        need = BYTES_PER_SURFEL * surf.n + WORKSPACE_PER_SURFEL * surf.n + 40 * frame_pixels
        if self.used + need > self.budget:
            self.rejected_sessions.append(sid)
            return False
        self.sessions[sid] = MapSession(sid, surf, self.device)
        self.used += need
        return True

    def close(self):
        if self.rast is not None:
            self.rast.close()
        self.sessions.clear()

    # -- one tick -------------------------------------------------------------
    def _tick(self, active):
        """One iteration of every active request: one call per stage over their
        frames, a capacity check at the tick's single synchronisation, one
        fused Adam launch over their maps.  Returns the per-map losses."""
        for r in active:
            if r.buffers is None:      # device buffers for the request's lifetime
                r.buffers = (render.target_tensors(r.target, self.device), lib.alloc_fwd(r.frame, self.device),
                             render.upstream_planes(r.frame, self.device))
        frames = [r.frame for r in active]
        fmap = list(range(len(active)))
        outs = [r.buffers[1] for r in active]
        ups = [r.buffers[2] for r in active]
        if self.rast is None:
            self.rast = render.Rasterizer(frames, frame_map=fmap, device=self.device.index, tuning=self.tuning)
        self.rast.set_frames(frames, fmap, outs=outs, ups=ups)
        maps = [self.sessions[r.session] for r in active]
        params = [s.params for s in maps]
        grads = [s.grads for s in maps]      # zero: the previous Adam step cleared them
        targets = [r.buffers[0] for r in active]
        out = self.rast.step(params, targets, grads, check=False)
        torch.cuda.synchronize(self.device)
        st, _ = lib.lgs_session_status(self.rast.session.handle)
        self._grew = st == lib.LGS_ERR_CAPACITY
        if st == lib.LGS_ERR_CAPACITY:       # grow the workspace and redo the tick
            for g in grads:
                for x in g:
                    x.zero_()
            out = self.rast.step(params, targets, grads, check=True)
        F = len(active)
        k = 1 + lib.LOSS_TERMS * F
        losses = out[k: k + F].cpu().numpy()
        for s in maps:
            s.t += 1
        render.adam_step_batch([(s.params, s.grads, s.m, s.v, s.t, self.lr) for s in maps], zero_grad=True)
        return losses

    # -- deadline admission --------------------------------------------------
    def _learn(self, active, seconds: float):
        n = sum(self.sessions[r.session].n for r in active)
        k = max(seconds - self.tick_base, 0.0) / max(n, 1)
        self.kappa = k if self.kappa is None else 0.5 * self.kappa + 0.5 * k

    def _feasible(self, active, now: float) -> bool:
        """Simulate the remaining ticks of ``active`` (no further arrivals):
        does every request finish within the margin of its deadline?"""
        rem = [(r.iters - r.done_iters, self.sessions[r.session].n, r.arrival + self.slo_margin * self.slo)
               for r in active]
        t = now
        while rem:
            t += self.tick_base + self.kappa * sum(n for _, n, _ in rem)
            nxt = []
            for k, n, dl in rem:
                if k == 1:
                    if t > dl:
                        return False
                else:
                    nxt.append((k - 1, n, dl))
            rem = nxt
        return True

    # -- the loop ---------------------------------------------------------------
    def run(self, requests):
        """Serve ``requests`` (sorted by arrival; times relative to now).
        Returns the completed requests."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        active, done = [], []
        busy = set()
        t0 = time.perf_counter()
        while pending or waiting or active:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                if r.session not in self.sessions:
                    continue
                if self.keep_latest:
                    for old in [w for w in waiting if w.session == r.session]:
                        waiting.remove(old)
                        self.dropped.append(old)
                waiting.append(r)
            # fill free slots, at most one request per session, in arrival order
            keep = collections.deque()
            while waiting:
                r = waiting.popleft()
                if len(active) < self.slots and r.session not in busy:
                    if self.slo is not None and self.kappa is not None and not self._feasible(active + [r], now):
                        self.late.append(r)      # would miss its deadline or make another one miss
                        continue
                    r.start = now
                    active.append(r)
                    busy.add(r.session)
                else:
                    keep.append(r)
            waiting = keep
            if not active:
                if pending:
                    time.sleep(max(0.0, min(pending[0].arrival - now, 0.002)))
                continue
            t_tick = time.perf_counter()
            L = self._tick(active)     # per-map loss (one frame per map); the tick ends synchronised
            # the tick model learns from ordinary ticks only: not the server's
            # first (buffers and workspace are created) nor one that grew the
            # workspace and ran twice
            if self._ticks > 0 and not self._grew:
                self._learn(active, time.perf_counter() - t_tick)
            self._ticks += 1
            now = time.perf_counter() - t0
            still = []
            for r, l in zip(active, L):
                r.done_iters += 1
                r.losses.append(float(l))
                if r.done_iters >= r.iters:
                    r.finish = now
                    done.append(r)
                    busy.discard(r.session)
                    r.buffers = None
                else:
                    still.append(r)
            active = still
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
                  late: int = 0):
    """p50 / p99 latency (ms) of the completed requests, completed frames per
    second of wall time, and the rejections: sessions refused at admission,
    requests superseded by a newer keyframe of their session, requests
    refused by the deadline admission."""
    lat = np.array([r.finish - r.arrival for r in done]) * 1e3
    wall = max([r.finish for r in done] + [duration])
    return dict(completed=len(done), offered=offered, p50_ms=float(np.percentile(lat, 50)) if len(lat) else None,
                p99_ms=float(np.percentile(lat, 99)) if len(lat) else None,
                frames_per_s=len(done) / wall, rejected_sessions=rejected_sessions,
                session_rejection_rate=rejected_sessions / max(n_sessions, 1), dropped_requests=dropped,
                deadline_rejected=late, request_rejection_rate=(dropped + late) / max(offered, 1))
