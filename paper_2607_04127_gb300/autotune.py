"""Autotuner of the compositing knobs: tile shape (8 x 8, 16 x 16, 32 columns
x 8 rows), forward and backward variants (a shared-memory batch of 64, 128,
256 or 512 records per CTA, the backward's up to 256; or the per-warp walk:
records of each chunk's hits staged in the warp's shared memory, or read
through L1 with 1, 2 or 4 hits per step) and persistent scheduling, chosen
by timing whole steps of the actual workload on the device.  The search is
coordinate-wise (tile shape first, then the forward, the backward and the
scheduling), each candidate timed over a few steps with CUDA events after a
checked warm-up step.

Every candidate computes the same results (bit-identical forward outputs,
gradients equal up to the order of float atomics), so the choice affects
time only.
"""
from __future__ import annotations

import torch

# tile shapes (rows, columns): 8 x 8, 16 x 16 and 32 columns x 8 rows; the
# "surfel batch" of a compositing CTA: 64 to 512 records staged in shared
# memory per batch (the backward's batch stops at 256: its gradient
# accumulators would take the CTA's static shared memory past 48 KB at 512),
# or 0 for the per-warp walks
TILES = ((8, 8), (16, 16), (8, 32))
FWD = ((0, 16), (64, 16), (128, 16), (256, 16), (512, 16), (0, 2))   # (fwd_batch, group when 0)
BWD = ((0, 16), (0, 2), (64, 16), (128, 16), (256, 16))              # (bwd_batch, group)


def time_steps(stepper, steps: int = 3) -> float:
    """Mean device milliseconds of ``stepper.step()`` after one checked step."""
    stepper.step(check=True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        stepper.step()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def autotune(make, base: dict | None = None, steps: int = 3, tiles=TILES, fwd=FWD, bwd=BWD):
    """``make(tile, tuning)`` builds a stepper (an object with ``step(check)``
    and ``close()``).  Returns (tile, tuning, {description: ms})."""
    tun = dict(fwd_batch=0, bwd_batch=0, group=16, persistent=0, **(base or {}))
    log = {}

    def run(tile, t):
        s = make(tile, t)
        try:
            ms = time_steps(s, steps)
        finally:
            s.close()
        log[f"tile {tile[0]}x{tile[1]} {t}"] = ms
        return ms

    best_tile, best = None, float("inf")
    for tile in tiles:
        ms = run(tile, tun)
        if ms < best:
            best_tile, best = tile, ms
    for key, cands in (("fwd", fwd), ("bwd", bwd), ("persistent", (0, 1))):
        choice = None
        for c in cands:
            t = dict(tun)
            if key == "fwd":
                t["fwd_batch"] = c[0]
                if c[0] == 0:
                    t["group"] = c[1]
            elif key == "bwd":
                t["bwd_batch"], t["group"] = c
            else:
                t["persistent"] = c
            if t == tun:
                continue
            ms = run(best_tile, t)
            if ms < best:
                best, choice = ms, t
        if choice is not None:
            tun = choice
    return best_tile, tun, log
