"""Many maps of uneven size rendered and differentiated together: one call
per stage (bin + sort, forward, loss, backward) covers every map's frames,
the compositing kernels can run persistent (CTAs claim tiles longest list
first from an atomic counter), and the whole step can be captured into a
CUDA graph and replayed.  ``SequentialMaps`` is the plain per-map launch the
batched form is measured against.
"""
from __future__ import annotations

import torch

from . import render


class BatchedMaps:
    """``maps``: list of scenes.Surfels; ``frames``: one scenes.Frame per map
    (any H x W, one tile shape); ``targets``: one scenes.Target per frame."""

    def __init__(self, maps, frames, targets, device: int = 0, tuning: dict | None = None,
                 lr=(1e-3, 1e-3, 5e-3, 5e-3)):
        self.device = torch.device("cuda", device)
        self.params = [render.map_tensors(m, self.device) for m in maps]
        self.grads = [[torch.zeros_like(p) for p in ps] for ps in self.params]
        self.targets = [render.target_tensors(t, self.device) for t in targets]
        self.rast = render.Rasterizer(frames, frame_map=list(range(len(maps))), device=device, tuning=tuning)
        self.m = [torch.zeros(10 * int(ps[0].shape[0]), device=self.device) for ps in self.params]
        self.v = [torch.zeros_like(m) for m in self.m]
        self.lr = lr
        self.t = 0
        self.graph = None
        self.rays = sum(f.H * f.W for f in frames)

    def step(self, check: bool = False):
        """bin + forward + loss + backward of every map (gradients zeroed
        first); asynchronous unless ``check`` (capacity check)."""
        for gs in self.grads:
            for g in gs:
                g.zero_()
        return self.rast.step(self.params, self.targets, self.grads, check=check)

    def adam(self):
        """One fused Adam launch over every map."""
        self.t += 1
        render.adam_step_batch([(ps, gs, m, v, self.t, self.lr)
                                for ps, gs, m, v in zip(self.params, self.grads, self.m, self.v)], zero_grad=False)

    def capture(self):
        """Size the workspace with one checked step, then capture one step
        (gradient zeroing and the four library calls) into a CUDA graph."""
        self.step(check=True)
        torch.cuda.synchronize(self.device)
        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            self.step()                 # warm-up on the capture stream
        torch.cuda.current_stream(self.device).wait_stream(s)
        torch.cuda.synchronize(self.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step()
        torch.cuda.synchronize(self.device)

    def replay(self):
        self.graph.replay()

    def outputs(self):
        return self.rast.out

    def close(self):
        self.graph = None
        self.rast.close()


class SequentialMaps:
    """The same maps, one rasterizer and one launch sequence per map."""

    def __init__(self, maps, frames, targets, device: int = 0, tuning: dict | None = None):
        self.device = torch.device("cuda", device)
        self.params = [render.map_tensors(m, self.device) for m in maps]
        self.grads = [[torch.zeros_like(p) for p in ps] for ps in self.params]
        self.targets = [render.target_tensors(t, self.device) for t in targets]
        self.rasts = [render.Rasterizer([f], device=device, tuning=tuning) for f in frames]
        self.rays = sum(f.H * f.W for f in frames)

    def step(self, check: bool = False):
        for r, ps, gs, t in zip(self.rasts, self.params, self.grads, self.targets):
            for g in gs:
                g.zero_()
            r.step([ps], [t], [gs], check=check)

    def outputs(self):
        return [r.out[0] for r in self.rasts]

    def close(self):
        for r in self.rasts:
            r.close()
