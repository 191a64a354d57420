#!/usr/bin/env python
"""Benchmark: fwd+bwd rays/s of the differentiable spherical surfel rasterizer
on the 200k-surfel 128 x 1024 street frame (one mapping step = bin + sort,
forward, mapping loss, backward to every surfel parameter), with the
mapping window, the batched uneven maps and the 32-session serving loop as
sub-objects of the same line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload street|mapping|batched|serving|tracking|manage|keyframe]

One process per GPU (torchrun for N > 1); every rank renders its own replica
of the workload (the path has no exchange step), so scaling is weak and the
reported value is the sum over ranks.  Prints one JSON line on rank 0.

The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores: K steps (after W warm-up steps), each a bounded band of tile rows of
the same street frame.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing
import os
import statistics
import subprocess
import sys
import tempfile
import time
import concurrent.futures as cf

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd rays/s at 200k surfels, 128x1024"
UNIT = "rays/s"
WORKLOAD = dict(workload="street 200k surfels, 128x1024 range image, +-45 deg", surfels=200_000,
                H=128, W=1024, frames=1, loss="depth L1 + 0.1 opacity BCE + 0.05 normal cosine + 10 scale")

# Algorithmic work per stage of a step (the hot path's measurement budget):
#   A1 preprocess       112 B per item (40 B parameters in, 64 B record + key
#                       + box + count out)
#   A2-A4 bin and sort  12 B per pair emitted, 24 B per pair for one sort pass
#                       (the per-tile sort reads and writes each key once)
#   A5 forward          35 FP32 instructions and 2 MUFU (reciprocal, exp2) per
#                       evaluation up to the stop point; 28 B per pixel out,
#                       64 B per pair of records read
#   A6 loss             60 B per pixel
#   A7 backward         80 FP32 instructions per contributing pair (and 1
#                       MUFU); 64 B per pair of records read.  The backward
#                       recomputes the forward per tile, so a second figure
#                       adds the 35 instructions and 2 MUFU of every
#                       evaluation up to each pixel's last contributor
#   A8 chain            130 B per surfel
# FLOPs (FMA = 2), a secondary figure: 27 per evaluation, 12 more per
# composited pair, 70 more per contributing pair in the backward.
B_PREPROCESS, B_EMIT, B_SORT_PASS, B_FWD_PIXEL, B_RECORD = 112, 12, 24, 28, 64
B_LOSS_PIXEL, B_CHAIN = 60, 130
I_EVAL, M_EVAL, I_BWD_CONTRIB, M_BWD_CONTRIB = 35, 2, 80, 1
FLOP_EVAL, FLOP_COMPOSITE, FLOP_BWD_VALID = 27, 12, 70
FP32_LANES_PER_SM, MUFU_PER_SM = 128, 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile", default=None, help="tile shape HxW (default: the renderer's)")
    ap.add_argument("--fwd-batch", type=int, default=None)
    ap.add_argument("--bwd-batch", type=int, default=None)
    ap.add_argument("--group", type=int, default=None)
    ap.add_argument("--persistent", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0, help="wall-time budget of the reference arm")
    ap.add_argument("--manage-n", type=int, default=2_000_000, help="map size of the manage workload")
    ap.add_argument("--workload", default="street",
                    choices=["street", "mapping", "batched", "serving", "tracking", "manage", "keyframe"],
                    help="street: the headline line (with the mapping, batched and serving sub-objects)")
    ap.add_argument("--no-extras", action="store_true",
                    help="street line only: skip the mapping, batched and serving sub-objects")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving sub-object")
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


def gpu_local_cpus(gpu_id: int):
    """The CPUs of the GPU's own NUMA node (its PCI device's local_cpulist
    in sysfs, bus id from nvidia-smi) that this thread may run on; None when
    unknown.  Pinned host pages are placed on the node of the thread that
    allocates them, so the end-to-end section allocates and copies from
    there."""
    try:
        r = subprocess.run(["nvidia-smi", "--query-gpu=pci.bus_id", "--format=csv,noheader", "-i", str(gpu_id)],
                           capture_output=True, text=True, timeout=30)
        dom, rest = r.stdout.strip().split(":", 1)
        with open(f"/sys/bus/pci/devices/{int(dom, 16):04x}:{rest.lower()}/local_cpulist") as f:
            cpus = parse_cpulist(f.read()) & os.sched_getaffinity(0)
        return cpus or None
    except (OSError, ValueError, subprocess.SubprocessError):
        return None


def parse_cpulist(text: str) -> set:
    """The CPUs of a kernel CPU list ("0-3,8,10-11")."""
    cpus = set()
    for part in text.strip().split(","):
        if part:
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
    return cpus


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


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def device_peaks(dev_index: int):
    """Peaks of the GPU the step runs on: SM count queried from the device,
    maximum SM clock from nvidia-smi (else the measured-peaks record, else
    the part's 2070 MHz), HBM the measured copy bandwidth (else the 6.8 TB/s
    fallback)."""
    import torch
    sms = torch.cuda.get_device_properties(dev_index).multi_processor_count
    mhz, clk_src = None, None
    try:
        q = subprocess.run(["nvidia-smi", f"--id={dev_index}", "--query-gpu=clocks.max.sm",
                            "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
        mhz = float(q.stdout.strip().splitlines()[0])
        clk_src = "nvidia-smi clocks.max.sm"
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        pass
    mp = measured_peaks()
    if mhz is None:
        mhz, clk_src = float(mp.get("sm_max_mhz", 2070.0)), "MEASURED_PEAKS.json sm_max_mhz"
    hbm = mp.get("hbm_gbs")
    return dict(sms=sms, sm_max_mhz=mhz, fp32_instr_per_s=sms * FP32_LANES_PER_SM * mhz * 1e6,
                mufu_per_s=sms * MUFU_PER_SM * mhz * 1e6, hbm_gbs=hbm if hbm else 6800.0,
                source=f"{sms} SMs (device properties), {mhz:.0f} MHz ({clk_src}); FP32 issue = SMs x "
                       f"{FP32_LANES_PER_SM} lanes x clock, MUFU = SMs x {MUFU_PER_SM} x clock; HBM "
                       + ("measured copy bandwidth" if hbm else "fallback 6.8 TB/s"))


def street_config(tuning: dict, tile, world: int = 1) -> dict:
    """The config both arms report for the street line."""
    return dict(WORKLOAD, parallelism=f"replicas x{world}", tile=f"{tile[0]}x{tile[1]}", **tuning,
                l2="flushed between steps (256 MB write); per-step CUDA events, flush not timed")


def gen_pool():
    """A process pool for the seeded input generators, started with spawn
    before the first CUDA call (the workers import only NumPy code)."""
    return cf.ProcessPoolExecutor(max_workers=min(32, os.cpu_count() or 1),
                                  mp_context=multiprocessing.get_context("spawn"))


# ---------------------------------------------------------------------------
# The oracle on the host cores (the CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_band(surf, frame, tgt, t0: int, rows: int):
    """Tile rows [t0, t0 + rows) of the frame as a frame of their own (the same
    pixel rays, the elevation bounds of the band) with their targets."""
    from paper_2607_04127_gb300 import scenes
    th = frame.tile_h
    r0, r1 = t0 * th, min((t0 + rows) * th, frame.H)
    dth = (frame.elev_max - frame.elev_min) / frame.H
    band = scenes.Frame(r1 - r0, frame.W, frame.tile_h, frame.tile_w, frame.elev_max - r1 * dth,
                        frame.elev_max - r0 * dth, frame.pose)
    return band, tgt.D[r0:r1].copy(), tgt.N[:, r0:r1].copy()


def oracle_step(O, surf, band):
    """One fwd + loss + bwd pass of the FP64 oracle over a band: the method
    alone, on all host cores (OpenMP over tiles)."""
    frame, D, N = band
    O.forward_backward(surf, [frame], [(D, N)], nthreads=0, allowance=False)


def street_for_oracle():
    from oracle import oracle as O
    from paper_2607_04127_gb300 import render, scenes
    O.build()
    surf, frame, tgt = scenes.street()
    return O, surf, frame.with_tiles(*render.DEFAULT_TILE), tgt


def cpu_baseline(seconds: float):
    """The oracle, as it stands, on bands of 4 tile rows of the street frame
    (cycling through the frame) for about ``seconds`` of wall time."""
    O, surf, frame, tgt = street_for_oracle()
    ntr = -(-frame.H // frame.tile_h)
    rows, k, pix, el = 4, 0, 0, 0.0
    while el < seconds or k == 0:
        band = oracle_band(surf, frame, tgt, (k * rows) % ntr, rows)
        t0 = time.perf_counter()
        oracle_step(O, surf, band)
        el += time.perf_counter() - t0
        pix += band[0].H * band[0].W
        k += 1
    cores = os.cpu_count() or 1
    return dict(value=pix / el, unit=UNIT, cores=cores, kind="oracle",
                sample=f"{k} bands of {rows} tile rows ({rows * frame.tile_h} x {frame.W} rays each) of the street "
                       f"frame: FP64 oracle fwd + loss + bwd, the method without its test allowance, OpenMP over "
                       f"tiles on {cores} threads, {el:.1f} s")


def run_reference(args):
    """The reference arm: the oracle on the host cores, --warmup untimed and
    --steps timed steps, each one band of tile rows of the street frame sized
    so that the whole run takes about --ref-seconds."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2607_04127_gb300 import render
    O, surf, frame, tgt = street_for_oracle()
    ntr = -(-frame.H // frame.tile_h)
    # calibrate on one band of 2 tile rows (the first warm-up step)
    t0 = time.perf_counter()
    oracle_step(O, surf, oracle_band(surf, frame, tgt, 0, 2))
    per_row = (time.perf_counter() - t0) / 2
    W, K = max(args.warmup, 1), max(args.steps, 1)
    rows = int(min(ntr, max(1, math.floor(args.ref_seconds / (K + W) / max(per_row, 1e-6)))))
    for w in range(W - 1):
        oracle_step(O, surf, oracle_band(surf, frame, tgt, (w * rows) % ntr, rows))
    ms, pix = [], 0
    for k in range(K):
        band = oracle_band(surf, frame, tgt, (k * rows) % ntr, rows)
        t0 = time.perf_counter()
        oracle_step(O, surf, band)
        ms.append((time.perf_counter() - t0) * 1e3)
        pix += band[0].H * band[0].W
    el = sum(ms) / 1e3
    value = pix / el
    cores = os.cpu_count() or 1
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=K, warmup=W,
                ms_per_step=statistics.mean(ms), higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic (seeded street scene, see scenes.street)",
                config=street_config(dict(render.DEFAULT_TUNING), render.DEFAULT_TILE, world), impl="reference",
                cpu_baseline=dict(value=value, unit=UNIT, cores=cores, kind="oracle",
                                  sample=f"each step one band of {rows} of {ntr} tile rows ({rows * frame.tile_h} x "
                                         f"{frame.W} rays) of the street frame, bands cycling; FP64 oracle fwd + "
                                         f"loss + bwd, the method without its test allowance, {cores} threads"),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
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
# Mapping window, batched maps, serving: sub-objects of the street line (and
# lines of their own with --workload)
# ---------------------------------------------------------------------------
def serving_work(n_sessions, sizes_range, seed=0, shapes=((128, 1024),), pool=None):
    """Maps with log-uniform sizes in ``sizes_range``, one keyframe each."""
    import numpy as np
    from paper_2607_04127_gb300 import render, scenes
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(sizes_range[0]), np.log(sizes_range[1]), n_sessions)).astype(int)
    return scenes.street_maps(seed, [int(x) for x in sizes], list(shapes), tile=render.DEFAULT_TILE, pool=pool)


def serving_run(work, seconds, seed=0, plain=False, slots=16, iters=10, budget=150 << 30, keep_latest=True,
                rates=(10, 20), slo_ms=None):
    """Every session a Poisson request stream at U(10, 20) Hz of
    ``iters``-iteration render-and-optimise requests for its keyframe;
    returns the latency statistics.  ``slo_ms``: deadline admission."""
    import numpy as np
    import torch
    from paper_2607_04127_gb300 import serve
    rng = np.random.default_rng(seed)
    srv = serve.Server(hbm_budget_bytes=budget, slots=slots, plain=plain, keep_latest=keep_latest, slo_ms=slo_ms)
    sids = [sid for sid, (surf, fr, _) in enumerate(work) if srv.open_session(sid, surf, fr.H * fr.W) != "rejected"]
    reqs = serve.poisson_requests(rng, sids, lambda sid, k: work[sid][1], lambda sid, k: work[sid][2], seconds,
                                  rate_range=rates, iters=iters)
    # warm-up requests (kernels, workspace, tick model), not timed
    srv.run([serve.Request(sid, work[sid][1], work[sid][2], 0.0, 2) for sid in sids[:slots]])
    srv.dropped.clear()
    srv.late.clear()
    srv.unserved.clear()
    torch.cuda.synchronize()
    with Clocks(0) as clk:
        done = srv.run(reqs)
    st = serve.latency_stats(done, seconds, len(reqs), len(srv.rejected_sessions), len(work), len(srv.dropped),
                             len(srv.late), len(srv.unserved), len(srv.admitted_late) + len(srv.session_queue),
                             srv.overflow_ticks)
    sizes = [s.n for s, _, _ in work]
    mode = "plain per-request" if plain else f"continuous batching, {slots} slots"
    if slo_ms:
        mode += f", deadline admission {slo_ms:g} ms"
    st.update(sessions=len(work), map_sizes=[int(min(sizes)), int(max(sizes))], seconds=seconds, iters=iters,
              rate_hz=list(rates), keep_latest=keep_latest, mode=mode, budget_gb=budget / 2 ** 30,
              loss_first_mean=float(np.mean([r.losses[0] for r in done])) if done else None,
              loss_last_mean=float(np.mean([r.losses[-1] for r in done])) if done else None,
              clocks=clk.summary())
    srv.close()
    return st


def mapping_sub(pool=None, inputs=None):
    """Differentiable mapping window: the 1M-surfel street track, 8 keyframes
    (128 x 1024) rendered together, 10 Adam iterations; the fused driver and
    the autograd.Function driver."""
    import torch
    from paper_2607_04127_gb300 import mapping, render, scenes
    surf, frames, targets = inputs if inputs is not None else scenes.street_track(pool=pool)
    frames = [f.with_tiles(*render.DEFAULT_TILE) for f in frames]
    res = {}
    with Clocks(0) as clk:
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
    return dict(metric="mapping window rays/s (1M surfels, 8 keyframes 128x1024, 10 Adam iterations)",
                value=res["fused"]["rays_per_s"], unit="rays/s", surfels=surf.n, keyframes=len(frames),
                iterations=10, tile="%dx%d" % render.DEFAULT_TILE, drivers=res, clocks=clk.summary(),
                data="synthetic (seeded 200 m street track, scenes.street_track)")


def batched_inputs(pool=None):
    from paper_2607_04127_gb300 import render, scenes
    sizes = ([50_000, 100_000, 250_000, 500_000, 1_000_000, 2_000_000] * 3)[:16]
    return scenes.street_maps(1, sizes, [(64, 1024), (128, 1024), (128, 2048)], tile=render.DEFAULT_TILE, pool=pool)


def batched_sub(pool=None, inputs=None):
    """Sixteen independent maps of 50k..2M surfels with 64x1024 / 128x1024 /
    128x2048 frames: one call per stage (autotuned, persistent, CUDA graph)
    against sixteen sequential plain launches."""
    import torch
    from paper_2607_04127_gb300 import autotune, batched, render, scenes
    work = inputs if inputs is not None else batched_inputs(pool)
    maps, frames, targets = zip(*work)
    sizes = [m.n for m in maps]
    rays = sum(f.H * f.W for f in frames)
    steps = 10
    with Clocks(0) as clk:
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
    return dict(metric="batched fwd+bwd rays/s, 16 uneven maps (8.7M surfels) in one launch per stage",
                value=rays / (t_b / 1e3), unit="rays/s", surfels=int(sum(sizes)), rays=rays,
                config=dict(tile="%dx%d" % tile, **tun, graph=True), ms_per_step=t_b,
                sequential=dict(ms_per_step=t_seq, rays_per_s=rays / (t_seq / 1e3),
                                tile="%dx%d" % render.DEFAULT_TILE),
                speedup_vs_sequential=t_seq / t_b, autotune_ms=log, clocks=clk.summary(),
                data="synthetic (seeded street maps, scenes.street_maps)")


def serving32_sub(seconds: float, pool=None, inputs=None):
    """Thirty-two sessions (100k..2M surfels), Poisson 10-20 Hz each, 10
    iterations per request, 150 GB budget: continuous batching, deadline
    admission (50 ms) and per-request plain launches."""
    work = inputs if inputs is not None else serving_work(32, (100_000, 2_000_000), seed=2, pool=pool)
    b = serving_run(work, seconds, seed=2)
    d = serving_run(work, seconds, seed=2, slo_ms=50.0)
    p = serving_run(work, seconds, seed=2, plain=True)
    return dict(metric="serving p50/p99 frame latency and frames/s, 32 mapping sessions", value=d["p99_ms"],
                unit="ms (p99, deadline admission 50 ms)", higher_is_better=False,
                data="synthetic (seeded street maps, Poisson request streams)", serving_slo=d, serving=b, plain=p)


def _standalone(args, fn, **kw):
    from paper_2607_04127_gb300 import build
    pool = gen_pool()
    try:
        build.build()
        import torch
        torch.cuda.set_device(0)
        sub = fn(pool=pool, **kw)
    finally:
        pool.shutdown()
    sub.setdefault("higher_is_better", True)
    sub.update(n_gpus=1, dtype="f32")
    print(json.dumps(sub), flush=True)


def run_mapping(args):
    _standalone(args, mapping_sub)


def run_batched(args):
    _standalone(args, batched_sub)


def run_serving(args):
    _standalone(args, serving32_sub, seconds=args.serve_seconds or 10.0)



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
    pk = device_peaks(0)
    lanes_peak = pk["fp32_instr_per_s"] / 1e12
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
                              note="8 FP32 operations per evaluated distance over the call's CUDA-event time",
                              peak_source=pk["source"]),
                e2e=dict(value=n / e2e_s, unit="points/s", h2d_bytes_per_step=n * 12, d2h_bytes_per_step=d2h),
                cpu_baseline=dict(value=done / cpu_s, unit="points/s", cores=1, kind="oracle",
                                  sample=f"{done} sampled rows of the same scan in {cpu_s:.1f} s (NumPy brute-force "
                                         f"k-NN over all {n} points, FP64 frames)"),
                gpu_launches=int(lib.load().lgs_init_launches()) * steps, clocks=clk.summary())
    print(json.dumps(line), flush=True)




# ---------------------------------------------------------------------------
# The street line
# ---------------------------------------------------------------------------
def street_roofline(pk, kernels_ms, ms_step, c, n_items, hw, n_surf, tuning):
    """Per-stage roofline of a street step from the measurement budget above
    (max of bytes / HBM, FP32 instructions / FP32 issue, MUFU / MUFU issue per
    stage), the step fraction (sum of the stage rooflines over the measured
    step), and the dominant compositing kernel in instruction units."""
    P, E_f, E_b, C = c["pairs"], c["alg_f"], c["alg_b"], c["contrib"]
    hbm = pk["hbm_gbs"] * 1e9

    def stage(name, ms, byts=0.0, instr=0.0, mufu=0.0):
        t = {"hbm": byts / hbm, "alu": instr / pk["fp32_instr_per_s"], "mufu": mufu / pk["mufu_per_s"]}
        bound = max(t, key=t.get)
        return dict(stage=name, ms=ms, roofline_ms=t[bound] * 1e3, bound=bound,
                    frac=t[bound] * 1e3 / ms if ms else None, bytes=byts, fp32_instr=instr, mufu=mufu)

    stages = [
        stage("bin and sort (A1-A4)", kernels_ms["bin"],
              B_PREPROCESS * n_items + B_EMIT * P + B_SORT_PASS * P),
        stage("forward with the loss epilogue (A5, A6)", kernels_ms["fwd"],
              B_FWD_PIXEL * hw + B_RECORD * P + B_LOSS_PIXEL * hw, I_EVAL * E_f, M_EVAL * E_f),
        stage("mask counts and scale regulariser (A6; the loss vector is written by the forward)", kernels_ms["loss"], 16 * hw + 16 * n_surf),
        stage("backward (A7)", kernels_ms["bwd"], B_RECORD * P, I_BWD_CONTRIB * C, M_BWD_CONTRIB * C),
        stage("chain to the parameters (A8)", kernels_ms["bwd_chain"], B_CHAIN * n_surf),
    ]
    bwd_re = stage("backward (A7) with its re-evaluation", kernels_ms["bwd"], B_RECORD * P,
                   I_BWD_CONTRIB * C + I_EVAL * E_b, M_BWD_CONTRIB * C + M_EVAL * E_b)
    roof = sum(s["roofline_ms"] for s in stages)
    roof_re = roof - stages[3]["roofline_ms"] + bwd_re["roofline_ms"]
    dom = "bwd" if kernels_ms["bwd"] >= kernels_ms["fwd"] else "fwd"
    t_dom = kernels_ms[dom] / 1e3
    instr = I_BWD_CONTRIB * C if dom == "bwd" else I_EVAL * E_f
    instr_re = I_BWD_CONTRIB * C + I_EVAL * E_b if dom == "bwd" else instr
    flops = (FLOP_EVAL * E_b + FLOP_BWD_VALID * C) if dom == "bwd" else (FLOP_EVAL * E_f + FLOP_COMPOSITE * C)
    peak = pk["fp32_instr_per_s"] / 1e12
    return dict(bound="alu", kernel=kname(tuning, dom), achieved=instr / t_dom / 1e12, peak=peak, unit="Tinstr/s",
                frac=instr / t_dom / 1e12 / peak, traffic=measured_traffic(kname(tuning, dom)),
                achieved_with_reevaluation=instr_re / t_dom / 1e12,
                frac_with_reevaluation=instr_re / t_dom / 1e12 / peak,
                frac_step=roof / ms_step, frac_step_with_reevaluation=roof_re / ms_step, roofline_step_ms=roof,
                stages=stages, peak_source=pk["source"],
                flops=dict(achieved=flops / t_dom / 1e12, peak=2 * peak, unit="TFLOP/s",
                           frac=flops / t_dom / 1e12 / (2 * peak),
                           note="FMA = 2; 27 FLOP per evaluation, 12 per composited, 70 per contributing pair"))


def run_ours(args):
    import threading
    rank, world, local = dist_env()
    extras = world == 1 and not args.no_extras
    pool, box, gen = None, {}, None
    if extras:
        # the sub-objects' inputs are generated on the host cores while the
        # street frame is set up, and are complete before its timed region
        pool = gen_pool()
        from paper_2607_04127_gb300 import scenes

        def produce():
            box["mapping"] = scenes.street_track(pool=pool)
            box["batched"] = batched_inputs(pool)
            if not args.no_serving:
                box["serving"] = serving_work(32, (100_000, 2_000_000), seed=2, pool=pool)
        gen = threading.Thread(target=produce, daemon=True)
        gen.start()
    import torch
    import torch.distributed as dist
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
    if gen is not None:
        gen.join()
        pool.shutdown()
    pk = device_peaks(dev.index)

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    c0 = rast.counters()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    gpu_id = int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[0]) if os.environ.get(
        "CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else dev.index
    with Clocks(gpu_id) as clk:
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
            e[3].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    rast.session.check_status()
    c1 = rast.counters()
    clocks = clk.summary()
    step_ms = [e[0].elapsed_time(e[3]) for e in ev]
    rays = frame.H * frame.W
    total_s, value = replicas_value(sum(step_ms) / 1e3, args.steps * rays, world, dev)
    ms_step = total_s * 1e3 / args.steps
    launches_per_step = (c1["launches"] - c0["launches"]) / args.steps

    # algorithmic work of one step (counters are cumulative since the last
    # bin_sort): forward = list entries up to each pixel's stop point, backward
    # = entries up to each pixel's last contributor (the sum of n_contrib);
    # the backward's contributing pairs are the forward's composited pairs
    c_last = rast.counters()
    work = dict(pairs=c_last["n_pairs"], alg_f=c_last["alg_fwd"], alg_b=int(rast.out[0].n_contrib.sum().item()),
                contrib=c_last["contrib_fwd"])

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
    roof = street_roofline(pk, kernels_ms, ms_step, work, surf.n, rays, surf.n, rast.tuning)

    # end to end through the public API with host buffers, the host side on
    # the GPU's own NUMA node (restored afterwards)
    saved_cpus = os.sched_getaffinity(0)
    local_cpus = gpu_local_cpus(gpu_id)
    if local_cpus:
        os.sched_setaffinity(0, local_cpus)
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
    os.sched_setaffinity(0, saved_cpus)
    e2e_s, e2e_value = replicas_value(sum(e[0].elapsed_time(e[1]) for e in ee) / 1e3, e2e_steps * rays, world, dev)
    rast.close()

    sub = {}
    if extras and rank == 0:
        sub["mapping"] = mapping_sub(inputs=box["mapping"])
        sub["batched"] = batched_sub(inputs=box["batched"])
        if not args.no_serving:
            sub["serving"] = serving32_sub(args.serve_seconds or 5.0, inputs=box["serving"])
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=ms_step, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="f32", data="synthetic (seeded street scene, see scenes.street)",
        config=street_config(rast.tuning, tile, world),
        evals_per_s=world * args.steps * (work["alg_f"] + work["alg_b"]) / total_s,
        stages_ms={k: statistics.mean([e[i].elapsed_time(e[i + 1]) for e in ev])
                   for i, k in enumerate(("bin_sort", "fwd_loss", "bwd"))},
        kernels_ms=kernels_ms,
        work=dict(pairs=work["pairs"], visible_items=c_last["n_visible"], alg_evals_fwd=work["alg_f"],
                  alg_evals_bwd=work["alg_b"], culled_evals_fwd=c_last["evals_fwd"],
                  composited_fwd=work["contrib"]),
        roofline=roof,
        e2e=dict(value=e2e_value, unit=UNIT, h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h,
                 host_cpus=f"GPU-local NUMA node, {len(local_cpus)} CPUs" if local_cpus else "not bound"),
        gpu_launches=int(round(launches_per_step * args.steps)),
        clocks=clocks, wall_s=t_wall,
    )
    if cpu is not None:
        line["cpu_baseline"] = cpu
    line.update(sub)
    print(json.dumps(line), flush=True)
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
