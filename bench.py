#!/usr/bin/env python
"""Benchmark: fwd+bwd rays/s of the differentiable spherical surfel rasterizer
on the 200k-surfel 128 x 1024 street frame (one mapping step = bin + sort,
forward, mapping loss, backward to every surfel parameter).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload street|mapping|batched|serving]

One process per GPU (torchrun for N > 1); every rank renders its own replica
of the workload (the path has no exchange step), so scaling is weak and the
reported value is the sum over ranks.  Prints one JSON line on rank 0.

The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd rays/s at 200k surfels, 128x1024"
UNIT = "rays/s"
WORKLOAD = dict(workload="street 200k surfels, 128x1024 range image, +-45 deg", surfels=200_000,
                H=128, W=1024, frames=1, loss="depth L1 + 0.1 opacity BCE + 0.05 normal cosine + 10 scale")
# FP32 operations (FMA = 2) counted from the definition: an evaluation forms
# three dot products with the ray (n.d, a_u.d, a_v.d: 15), t = h/den (1),
# u, v (4), q (3), exp(-q/2) (2) and alpha G (1) plus the clamp (1) = 27; a
# composited pair adds T(1-a), w, A, S_t and the flipped normal sum (12); the
# reverse step of a contributing pair (dL/da through T and the suffix, and the
# chain to h, n, a_u, b_u, a_v, b_v, alpha as the reverse mode of the
# evaluation) costs 70.
FLOP_EVAL = 27
FLOP_COMPOSITE = 12
FLOP_BWD_VALID = 70
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12     # SMs x lanes x FMA x max clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile", default=None, help="tile shape HxW (default: the renderer's)")
    ap.add_argument("--fwd-batch", type=int, default=None)
    ap.add_argument("--bwd-batch", type=int, default=None)
    ap.add_argument("--group", type=int, default=None)
    ap.add_argument("--persistent", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--manage-n", type=int, default=2_000_000, help="map size of the manage workload")
    ap.add_argument("--workload", default="street",
                    choices=["street", "mapping", "batched", "serving", "tracking", "manage", "keyframe"],
                    help="street: the headline line; the others print their own line")
    ap.add_argument("--no-serving", action="store_true", help="skip the reduced serving run of the street line")
    ap.add_argument("--serve-seconds", type=float, default=None)
    return ap.parse_args()


def measured_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None
    when the kernel's sources changed since that capture."""
    import hashlib
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
    except (OSError, KeyError, ValueError):
        return None
    m = hashlib.sha256()
    for p in d["sources"]:
        try:
            m.update(open(os.path.join(ROOT, p), "rb").read())
        except OSError:
            return None
    return d["dram_bytes_per_launch"] if m.hexdigest()[:16] == d["sources_sha256_16"] else None


def kname(tuning, which):
    """Name of the compositing kernel a tuning runs for the forward or the
    backward (the chunked backward follows the shared-memory forward)."""
    b = tuning["fwd_batch" if which == "fwd" else "bwd_batch"]
    if b:
        return f"k_fwd<{b}>" if which == "fwd" else f"k_bwd<{b}>"
    if tuning["group"] == 16:
        if which == "fwd":
            return "k_fwd_s"
        return "k_bwd_c" if tuning["fwd_batch"] == 0 else "k_bwd_s"
    return f"k_fwd_w<{tuning['group']}>" if which == "fwd" else f"k_bwd_w<{tuning['group']}>"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replicas_value(local_seconds: float, units_per_rank: float, world: int, device=None):
    """Whole-job throughput of ``world`` independent replicas: every rank
    processed ``units_per_rank`` in ``local_seconds``; the job lasts as long
    as its slowest rank (max over ranks, the only collective).  Returns
    (job seconds, units per second of the whole job)."""
    t = float(local_seconds)
    if world > 1:
        import torch
        import torch.distributed as dist
        x = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return t, world * units_per_rank / t


# ---------------------------------------------------------------------------
def cpu_baseline(seconds: float):
    """The oracle, as it stands, on the full street frame, repeated for about
    ``seconds`` of wall time on all host cores."""
    from oracle import oracle as O
    from paper_2607_04127_gb300 import scenes
    O.build()
    surf, frame, tgt = scenes.street()
    reps = 0
    t0 = time.perf_counter()
    while True:
        O.forward_backward(surf, [frame], [(tgt.D, tgt.N)], nthreads=0)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds or reps >= 50:
            break
    cores = os.cpu_count() or 1
    return dict(value=reps * frame.H * frame.W / el, unit=UNIT, cores=cores, kind="oracle",
                sample=f"{reps} full fwd+loss+bwd passes of the street frame (FP64 oracle, OpenMP over tiles, "
                       f"{cores} threads) in {el:.1f} s")


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cb = cpu_baseline(args.cpu_seconds)
    line = dict(metric=METRIC, value=cb["value"], unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * WORKLOAD["H"] * WORKLOAD["W"] / cb["value"],
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(WORKLOAD, parallelism="host cores"), impl="reference", cpu_baseline=cb,
                e2e=dict(value=cb["value"], unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for ln in open(self.path):
                p = [x.strip() for x in ln.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["no samples"], samples=0)
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        load = [s for s in sm if mx and s >= 0.5 * max(mx)] or sm
        return dict(sm_mhz=statistics.median(load) if load else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=reasons, samples=len(rows))


# ---------------------------------------------------------------------------
def serving_work(n_sessions, sizes_range, seed=0, shapes=((128, 1024),)):
    """Maps with log-uniform sizes in ``sizes_range``, one keyframe each."""
    import numpy as np
    from paper_2607_04127_gb300 import render, scenes
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(sizes_range[0]), np.log(sizes_range[1]), n_sessions)).astype(int)
    return scenes.street_maps(seed, [int(x) for x in sizes], list(shapes), tile=render.DEFAULT_TILE)


def serving_run(work, seconds, seed=0, plain=False, slots=16, iters=10, budget=150 << 30, keep_latest=True,
                rates=(10, 20), slo_ms=None):
    """Every session a Poisson request stream at U(10, 20) Hz of
    ``iters``-iteration render-and-optimise requests for its keyframe;
    returns the latency statistics.  ``slo_ms``: deadline admission."""
    import numpy as np
    from paper_2607_04127_gb300 import serve
    rng = np.random.default_rng(seed)
    srv = serve.Server(hbm_budget_bytes=budget, slots=slots, plain=plain, keep_latest=keep_latest, slo_ms=slo_ms)
    sids = []
    for sid, (surf, fr, _) in enumerate(work):
        if srv.open_session(sid, surf, fr.H * fr.W):
            sids.append(sid)
    reqs = serve.poisson_requests(rng, sids, lambda sid, k: work[sid][1], lambda sid, k: work[sid][2], seconds,
                                  rate_range=rates, iters=iters)
    # warm-up request (kernels, workspace), not timed
    srv.run([serve.Request(sids[0], work[sids[0]][1], work[sids[0]][2], 0.0, 2)])
    srv.dropped.clear()
    srv.late.clear()
    done = srv.run(reqs)
    st = serve.latency_stats(done, seconds, len(reqs), len(srv.rejected_sessions), len(work), len(srv.dropped),
                             len(srv.late))
    sizes = [s.n for s, _, _ in work]
    mode = "plain per-request" if plain else f"continuous batching, {slots} slots"
    if slo_ms:
        mode += f", deadline admission {slo_ms:g} ms"
    st.update(sessions=len(work), map_sizes=[int(min(sizes)), int(max(sizes))], seconds=seconds, iters=iters,
              rate_hz=list(rates), keep_latest=keep_latest, mode=mode)
    srv.close()
    return st


def run_mapping(args):
    """Differentiable mapping window: 1M-surfel street track, 8 keyframes
    (128 x 1024) rendered together, 10 Adam iterations; fused and autograd
    drivers."""
    import torch
    from paper_2607_04127_gb300 import build, mapping, render, scenes
    build.build()
    surf, frames, targets = scenes.street_track()
    frames = [f.with_tiles(*render.DEFAULT_TILE) for f in frames]
    res = {}
    for ag in (False, True):
        w = mapping.MappingWindow(surf, frames, targets, autograd=ag)
        w.run(2)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        L = w.run(10)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        rays = 10 * sum(f.H * f.W for f in frames)
        res["autograd" if ag else "fused"] = dict(ms_per_iteration=ms / 10, rays_per_s=rays / (ms / 1e3),
                                                  loss_first=float(L[0]), loss_last=float(L[-1]))
        w.close()
    line = dict(metric="mapping window rays/s (1M surfels, 8 keyframes 128x1024, 10 Adam iterations)",
                value=res["fused"]["rays_per_s"], unit="rays/s", higher_is_better=True, dtype="f32",
                data="synthetic (seeded 200 m street track, scenes.street_track)", n_gpus=1,
                config=dict(workload="mapping window", surfels=surf.n, keyframes=len(frames), iterations=10,
                            tile="%dx%d" % render.DEFAULT_TILE), drivers=res)
    print(json.dumps(line), flush=True)


def run_batched(args):
    """Sixteen independent maps of 50k..2M surfels with 64x1024 / 128x1024 /
    128x2048 frames: one call per stage (autotuned, persistent, CUDA graph)
    against sixteen sequential plain launches."""
    import torch
    from paper_2607_04127_gb300 import autotune, batched, build, render, scenes
    build.build()
    sizes = [50_000, 100_000, 250_000, 500_000, 1_000_000, 2_000_000] * 3
    sizes = sizes[:16]
    work = scenes.street_maps(1, sizes, [(64, 1024), (128, 1024), (128, 2048)], tile=render.DEFAULT_TILE)
    maps, frames, targets = zip(*work)
    rays = sum(f.H * f.W for f in frames)
    steps = 10
    seq = batched.SequentialMaps(maps, frames, targets)
    t_seq = autotune.time_steps(seq, steps)
    seq.close()

    def make(tile, tun):
        return batched.BatchedMaps(maps, [f.with_tiles(*tile) for f in frames], targets, tuning=tun)

    tile, tun, log = autotune.autotune(make, steps=3)
    B = make(tile, tun)
    B.capture()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        B.replay()
    b.record()
    torch.cuda.synchronize()
    B.rast.session.check_status()
    t_b = a.elapsed_time(b) / steps
    B.close()
    line = dict(metric="batched fwd+bwd rays/s, 16 uneven maps (8.7M surfels) in one launch per stage",
                value=rays / (t_b / 1e3), unit="rays/s", higher_is_better=True, dtype="f32", n_gpus=1,
                data="synthetic (seeded street maps, scenes.street_maps)",
                config=dict(workload="16 maps 50k-2M surfels, 64x1024/128x1024/128x2048", surfels=int(sum(sizes)),
                            rays=rays, tile="%dx%d" % tile, **tun, graph=True),
                ms_per_step=t_b, sequential=dict(ms_per_step=t_seq, rays_per_s=rays / (t_seq / 1e3),
                                                 tile="%dx%d" % render.DEFAULT_TILE),
                speedup_vs_sequential=t_seq / t_b, autotune_ms=log)
    print(json.dumps(line), flush=True)


def run_serving(args):
    """Thirty-two sessions (100k..2M surfels), Poisson 10-20 Hz each, 10
    iterations per request, 150 GB budget: continuous batching against
    per-request plain launches."""
    from paper_2607_04127_gb300 import build
    build.build()
    secs = args.serve_seconds or 10.0
    work = serving_work(32, (100_000, 2_000_000), seed=2)
    b = serving_run(work, secs, seed=2)
    d = serving_run(work, secs, seed=2, slo_ms=50.0)
    p = serving_run(work, secs, seed=2, plain=True)
    line = dict(metric="serving p50/p99 frame latency and frames/s, 32 mapping sessions", value=d["p99_ms"],
                unit="ms (p99, deadline admission 50 ms)", higher_is_better=False, dtype="f32", n_gpus=1,
                data="synthetic (seeded street maps, Poisson request streams)", serving_slo=d, serving=b, plain=p)
    print(json.dumps(line), flush=True)


def run_tracking(args):
    """Tracking-side targets (Sec. 3.2) of the 1M-surfel street-track map:
    trackable selection, target covariances and weights per call, timed with
    CUDA events over a map larger than L2; HBM roofline of the three kernels."""
    import numpy as np
    import torch
    from paper_2607_04127_gb300 import build, lib, render, scenes
    build.build()
    surf, _, _ = scenes.street_track(n_keyframes=1)
    dev = torch.device("cuda", 0)
    params = render.map_tensors(surf, dev)
    rng = np.random.default_rng(0)
    n = surf.n
    mask = torch.from_numpy((rng.uniform(size=n) < 0.8).astype(np.uint8)).to(dev)
    kf = torch.from_numpy(rng.integers(0, 10, n).astype(np.int32)).to(dev)
    scratch = torch.empty(lib.lgs_trackable_scratch_bytes(n), dtype=torch.uint8, device=dev)
    idx = torch.empty(n, dtype=torch.int32, device=dev)
    mean = torch.empty(n, 3, device=dev)
    cov = torch.empty(n, 6, device=dev)
    w = torch.empty(n, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    p = lib.lgs_track_params(3, 0.5, 0.01, 1e-6, 10.0)
    S = lib.surfels_struct(*params)
    stream = torch.cuda.current_stream(dev).cuda_stream
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def call():
        lib.lgs_trackable_targets(S, mask.data_ptr(), kf.data_ptr(), p, scratch.data_ptr(), scratch.numel(),
                                  idx.data_ptr(), mean.data_ptr(), cov.data_ptr(), w.data_ptr(), cnt.data_ptr(),
                                  stream)
    for _ in range(max(args.warmup, 3)):
        call()
    torch.cuda.synchronize()
    k = selected = None
    ms = []
    for _ in range(max(args.steps // 10, 20)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        call()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    selected = int(cnt.item())
    t = statistics.median(ms) / 1e3
    # algorithmic bytes: select reads logit, mask, last_kf, log-scales of all
    # surfels; write re-reads them and reads mean and quaternion of the
    # selected, writing index, mean, covariance and weight (44 B) for them
    byts = n * (4 + 1 + 4 + 8) * 2 + selected * (12 + 16 + 44)
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    line = dict(metric="tracking targets: surfels/s (selection, target covariance, weight)", value=n / t,
                unit="surfels/s", higher_is_better=True, dtype="f32", n_gpus=1,
                data="synthetic (seeded 200 m street track, scenes.street_track)",
                config=dict(workload="1M-surfel map, 80 % trackable mask, 10 keyframe indices, k_min 3, alpha_min 0.5",
                            surfels=n, selected=selected, l2="flushed between calls (256 MB write)"),
                ms_per_call=t * 1e3,
                roofline=dict(bound="hbm", achieved=byts / t / 1e9, peak=peak, unit="GB/s",
                              frac=byts / t / 1e9 / peak, traffic=None))
    print(json.dumps(line), flush=True)


def run_manage(args):
    """Map management (Sec. 3.3 control score; Sec. 3.5 opacity prune, planar
    cover-and-prune over three planes, adaptive split) of a street-track map
    of --manage-n surfels with tracking signals from its own k-NN
    covariances.  A step is one lgs_map_manage call: device-timed with CUDA
    events (inputs resident, L2 flushed between steps); end to end from
    pinned host buffers with the new map read back; the oracle on a bounded
    sample of the same map."""
    import numpy as np
    import torch
    from paper_2607_04127_gb300 import build, lib, manage, scenes
    build.build()
    surf, _, _ = scenes.street_track(n=args.manage_n, n_keyframes=1)
    lam, res = scenes.manage_signals(surf.mean)
    host = [np.ascontiguousarray(x) for x in (surf.mean, surf.quat, surf.log_scale, surf.logit, lam, res)]
    n = surf.n
    dev = torch.device("cuda", 0)
    t = [torch.from_numpy(x).to(dev) for x in host]
    m = manage.MapManager(dev)
    p = manage.params()
    out = m.launch(t[:4], t[4], t[5], p)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 3)):
        m.launch(t[:4], t[4], t[5], p, out=out)
    torch.cuda.synchronize()
    steps = max(min(args.steps, 50), 10)
    ms = []
    with Clocks(0) as clk:
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            m.launch(t[:4], t[4], t[5], p, out=out)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
    counts = out["counts"].cpu().tolist()
    step_s = statistics.median(ms) / 1e3
    # end to end: pinned host inputs copied in, the new map's rows read back
    pinned = [torch.from_numpy(x).pin_memory() for x in host]
    dst = [torch.empty(out["capacity"] * w, dtype=torch.float32).pin_memory() for w in (3, 4, 2, 1)]
    h2d = sum(x.numel() * 4 for x in pinned)
    e2e_ms, d2h = [], 0
    for _ in range(5):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d, s_ in zip(t, pinned):
            d.copy_(s_, non_blocking=True)
        m.launch(t[:4], t[4], t[5], p, out=out)
        k = int(out["counts"][0].item())
        d2h = 48
        for d, key, w in zip(dst, ("mean", "quat", "log_scale", "logit"), (3, 4, 2, 1)):
            d[: k * w].copy_(out[key].reshape(-1)[: k * w], non_blocking=True)
            d2h += k * w * 4
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_s = statistics.median(e2e_ms) / 1e3
    # oracle on a bounded sample: the first surfels of the map, repeated for ~10 s
    from oracle import manage as omg
    sample = min(n, 100_000)
    P = omg.Params()
    sub = [x[:sample] for x in host]
    t0 = time.perf_counter()
    runs = 0
    while runs == 0 or time.perf_counter() - t0 < min(args.cpu_seconds, 10.0):
        omg.manage(*sub, P)
        runs += 1
    cpu_s = time.perf_counter() - t0
    # algorithmic bytes of a step: the inputs read once (mean 12, quat 16,
    # log-scale 8, logit 4, eigenvalues 12, residual 4) and the score (4) per
    # surfel, the new map (40) with its parent index and role (5) per row
    alg = n * (56 + 4) + counts[0] * 45
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    line = dict(metric="map management: surfels/s (control score, opacity prune, 3-pass cover-and-prune, split)",
                value=n / step_s, unit="surfels/s", higher_is_better=True, n_gpus=1, steps=steps,
                warmup=max(args.warmup, 3), ms_per_step=step_s * 1e3, scaling="weak", vs_baseline=None, dtype="f32",
                data="synthetic (seeded 200 m street track, scenes.street_track; k-NN signals, scenes.manage_signals)",
                config=dict(workload=f"{n}-surfel street-track map, library default parameters", surfels=n,
                            counts=dict(n_out=counts[0], opacity_pruned=counts[1], plane_pruned=counts[2:5],
                                        split=counts[5]),
                            l2="flushed between steps (256 MB write)"),
                roofline=dict(bound="hbm", kernel="whole step", achieved=alg / step_s / 1e9, peak=peak, unit="GB/s",
                              frac=alg / step_s / 1e9 / peak, traffic=None,
                              note="algorithmic bytes of the step over its CUDA-event time"),
                e2e=dict(value=n / e2e_s, unit="surfels/s", h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h),
                cpu_baseline=dict(value=sample * runs / cpu_s, unit="surfels/s", cores=1, kind="oracle",
                                  sample=f"{runs} oracle runs over the first {sample} surfels of the map "
                                         f"in {cpu_s:.1f} s (NumPy, one thread)"),
                gpu_launches=lib.lgs_manage_launches(p) * steps,
                clocks=clk.summary())
    print(json.dumps(line), flush=True)


def run_keyframe(args):
    """Keyframe initialisation (Sec. 3.2 k-NN covariance; Sec. 3.3 scale,
    confidence, opacity) of one 128 x 1024 street scan: a step is one
    lgs_keyframe_init call over every valid point (k = 20), device-timed with
    CUDA events (points resident, L2 flushed between steps); end to end from
    pinned host points with the new surfels read back; the oracle on sampled
    rows of the same scan."""
    import numpy as np
    import torch
    from paper_2607_04127_gb300 import build, keyframe, lib, scenes
    build.build()
    pts, pose = scenes.keyframe_points(11, 128, 1024)
    n = len(pts)
    dev = torch.device("cuda", 0)
    t = torch.from_numpy(pts).to(dev)
    p = keyframe.params()
    out = keyframe.initialise(t, pose, p)
    pairs = torch.zeros(1, dtype=torch.int64, device=dev)
    keyframe.initialise(t, pose, p, out=out, pairs=pairs)
    torch.cuda.synchronize()
    n_pairs = int(pairs.item())
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 3)):
        keyframe.initialise(t, pose, p, out=out)
    torch.cuda.synchronize()
    steps = max(min(args.steps, 50), 10)
    ms = []
    with Clocks(0) as clk:
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            keyframe.initialise(t, pose, p, out=out)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
    step_s = statistics.median(ms) / 1e3
    host = torch.from_numpy(pts).pin_memory()
    dst = {k: torch.empty(out[k].shape, dtype=out[k].dtype).pin_memory()
           for k in ("mean", "quat", "log_scale", "logit", "lam", "u")}
    e2e_ms = []
    for _ in range(5):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t.copy_(host, non_blocking=True)
        keyframe.initialise(t, pose, p, out=out)
        for k, d in dst.items():
            d.copy_(out[k], non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_s = statistics.median(e2e_ms) / 1e3
    d2h = sum(d.numel() * d.element_size() for d in dst.values())
    from oracle import init as oinit
    P = oinit.Params()
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    done = 0
    while done == 0 or time.perf_counter() - t0 < min(args.cpu_seconds, 10.0):
        rows = np.sort(rng.choice(n, 500, replace=False))
        oinit.initialise(pts, pose, P, rows=rows)
        done += rows.size
    cpu_s = time.perf_counter() - t0
    # ALU roofline: 8 FP32 operations per evaluated distance (3 sub, 3 mul,
    # 2 add) against one operation per FP32 lane per clock
    lanes_peak = 152 * 128 * 2.07e9 / 1e12
    achieved = n_pairs * 8 / step_s / 1e12
    line = dict(metric="keyframe initialisation: points/s (exact 20-NN covariance, eigendecomposition, scale, "
                       "confidence, opacity)",
                value=n / step_s, unit="points/s", higher_is_better=True, n_gpus=1, steps=steps,
                warmup=max(args.warmup, 3), ms_per_step=step_s * 1e3, scaling="weak", vs_baseline=None, dtype="f32",
                data="synthetic (seeded street scan, scenes.keyframe_points)",
                config=dict(workload=f"one 128x1024 street scan, {n} points, k = 20", points=n, k=p.k,
                            pairs_evaluated=n_pairs, brute_force_pairs=n * n,
                            l2="flushed between steps (256 MB write)"),
                roofline=dict(bound="alu", kernel="whole call (k-NN dominant)", achieved=achieved,
                              peak=lanes_peak, unit="Tops/s", frac=achieved / lanes_peak, traffic=None,
                              note="8 FP32 operations per evaluated distance over the call's CUDA-event time; "
                                   "peak = 152 SMs x 128 FP32 lanes x 2.07 GHz"),
                e2e=dict(value=n / e2e_s, unit="points/s", h2d_bytes_per_step=n * 12, d2h_bytes_per_step=d2h),
                cpu_baseline=dict(value=done / cpu_s, unit="points/s", cores=1, kind="oracle",
                                  sample=f"{done} sampled rows of the same scan in {cpu_s:.1f} s (NumPy brute-force "
                                         f"k-NN over all {n} points, FP64 frames)"),
                gpu_launches=int(lib.load().lgs_init_launches()) * steps, clocks=clk.summary())
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2607_04127_gb300 import build
    build.build()
    from paper_2607_04127_gb300 import render, scenes
    surf, frame, tgt = scenes.street()
    tile = tuple(int(x) for x in args.tile.split("x")) if args.tile else render.DEFAULT_TILE
    frame = frame.with_tiles(*tile)
    tuning = {k: v for k, v in (("fwd_batch", args.fwd_batch), ("bwd_batch", args.bwd_batch), ("group", args.group),
                                ("persistent", args.persistent)) if v is not None}
    params = render.map_tensors(surf, dev)
    targets = [render.target_tensors(tgt, dev)]
    grads = [[torch.zeros_like(p) for p in params]]
    rast = render.Rasterizer([frame], device=dev.index, tuning=tuning)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (126 MB)
    stream = torch.cuda.current_stream(dev)

    # warm-up (also sizes the workspace: the first bin_sort checks capacity)
    rast.step([params], targets, grads, check=True)
    for _ in range(max(args.warmup, 3)):
        rast.step([params], targets, grads)
    torch.cuda.synchronize()
    rast.session.check_status()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    c0 = rast.counters()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(dev.index)).split(",")[0])
                if os.environ.get("CUDA_VISIBLE_DEVICES", "").isdigit() else dev.index) as clk:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            e = ev[k]
            e[0].record(stream)
            S = rast.bin_sort([params], check=False)
            e[1].record(stream)
            rast.forward_loss([params], targets, grads[0:1], S)   # loss in the forward's epilogue
            e[2].record(stream)
            rast.backward([params], grads, S=S)
            e[4].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    rast.session.check_status()
    c1 = rast.counters()
    step_ms = [e[0].elapsed_time(e[4]) for e in ev]
    fwd_ms = [e[1].elapsed_time(e[2]) for e in ev]
    bwd_ms = [e[2].elapsed_time(e[4]) for e in ev]
    bin_ms = [e[0].elapsed_time(e[1]) for e in ev]
    rays = frame.H * frame.W
    total_s, value = replicas_value(sum(step_ms) / 1e3, args.steps * rays, world, dev)

    # algorithmic work of one step (counters are cumulative since the last
    # bin_sort): forward = list entries up to each pixel's stop point, backward
    # = entries up to each pixel's last contributor (the sum of n_contrib)
    c_last = rast.counters()
    evf, evb = c_last["evals_fwd"], c_last["evals_bwd"]
    cf, cb_ = c_last["contrib_fwd"], c_last["contrib_bwd"]
    alg_f = c_last["alg_fwd"]
    alg_b = int(rast.out[0].n_contrib.sum().item())
    fl_fwd = FLOP_EVAL * alg_f + FLOP_COMPOSITE * cf
    # the backward's contributing pairs are exactly the forward's composited
    # pairs (the chunked backward does not count them again)
    fl_bwd = FLOP_EVAL * alg_b + FLOP_BWD_VALID * cf

    # device time of every kernel group, from events the library records
    # around its own launches on this stream (a separate pass of the same steps)
    k_steps = min(args.steps, 20)
    rast.set_timing(True)
    for _ in range(k_steps):
        flush.zero_()
        S = rast.bin_sort([params], check=False)
        rast.forward_loss([params], targets, grads[0:1], S)
        rast.backward([params], grads, S=S)
    kt = rast.kernel_times()
    rast.set_timing(False)
    kernels_ms = {g: (ms / n if n else 0.0) for g, (ms, n) in kt.items()}
    fwd_s, bwd_s = kernels_ms["fwd"] / 1e3, kernels_ms["bwd"] / 1e3
    dominant = "bwd" if bwd_s >= fwd_s else "fwd"
    achieved = (fl_bwd / bwd_s if dominant == "bwd" else fl_fwd / fwd_s) / 1e12
    launches_per_step = (c1["launches"] - c0["launches"]) / args.steps

    # end to end through the public API with host buffers
    host = [p.cpu().pin_memory() for p in params]
    host_t = [t.cpu().pin_memory() for t in targets[0]]
    dev_p = [torch.empty_like(p) for p in params]
    dev_t = [torch.empty_like(t) for t in targets[0]]
    out_g = [torch.empty(p.shape, dtype=p.dtype, pin_memory=True) for p in params]
    out_l = torch.empty(1, pin_memory=True)
    h2d = sum(h.numel() * 4 for h in host) + sum(h.numel() * 4 for h in host_t)
    d2h = sum(g.numel() * 4 for g in out_g) + 4
    e2e_steps = max(10, args.steps // 2)
    ee = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(e2e_steps)]
    g2 = [[torch.zeros_like(p) for p in params]]
    for k in range(e2e_steps):
        flush.zero_()
        ee[k][0].record(stream)
        for d_, h_ in zip(dev_p, host):
            d_.copy_(h_, non_blocking=True)
        for d_, h_ in zip(dev_t, host_t):
            d_.copy_(h_, non_blocking=True)
        for g in g2[0]:
            g.zero_()
        L = rast.step([dev_p], [tuple(dev_t)], g2)
        for o, g in zip(out_g, g2[0]):
            o.copy_(g, non_blocking=True)
        out_l.copy_(L[:1], non_blocking=True)
        ee[k][1].record(stream)
    torch.cuda.synchronize()
    e2e_s, e2e_value = replicas_value(sum(e[0].elapsed_time(e[1]) for e in ee) / 1e3, e2e_steps * rays, world, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds)
    serving = None
    if rank == 0 and not args.no_serving:
        rast.close()
        work = serving_work(8, (100_000, 400_000), seed=4)
        serving = serving_run(work, args.serve_seconds or 2.0, seed=4, iters=10)
        serving_slo = serving_run(work, args.serve_seconds or 2.0, seed=4, iters=10, slo_ms=50.0)
    clocks = clk.summary()
    if rank != 0:
        return
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=total_s * 1e3 / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="f32", data="synthetic (seeded street scene, see scenes.street)",
        config=dict(WORKLOAD, parallelism=f"replicas x{world}", tile=f"{tile[0]}x{tile[1]}", **rast.tuning,
                    l2="flushed between steps (256 MB write); per-step CUDA events, flush not timed"),
        evals_per_s=world * args.steps * (alg_f + alg_b) / total_s,
        stages_ms=dict(bin_sort=statistics.mean(bin_ms), fwd_loss=statistics.mean(fwd_ms),
                       bwd=statistics.mean(bwd_ms)),
        kernels_ms=kernels_ms,
        work=dict(pairs=c_last["n_pairs"], visible_items=c_last["n_visible"], alg_evals_fwd=alg_f,
                  alg_evals_bwd=alg_b, culled_evals_fwd=evf, culled_evals_bwd=evb or None, composited_fwd=cf,
                  valid_bwd=cb_ or cf),
        roofline=dict(bound="alu", kernel=kname(rast.tuning, dominant), achieved=achieved,
                      peak=PEAK_FP32_TFLOPS, unit="TFLOP/s", frac=achieved / PEAK_FP32_TFLOPS,
                      traffic=measured_traffic(kname(rast.tuning, dominant)),
                      peak_source="derived: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2.07 GHz"),
        e2e=dict(value=e2e_value, unit=UNIT, h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h),
        gpu_launches=int(round(launches_per_step * args.steps)),
        clocks=clocks, wall_s=t_wall,
    )
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if serving is not None:
        line["serving"] = serving
        line["serving_slo"] = serving_slo
    print(json.dumps(line), flush=True)
    if serving is None:
        rast.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "mapping":
        run_mapping(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "tracking":
        run_tracking(args)
    elif args.workload == "manage":
        run_manage(args)
    elif args.workload == "keyframe":
        run_keyframe(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
