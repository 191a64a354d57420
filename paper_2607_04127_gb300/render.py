"""User-facing rasterizer: device buffers around one library session, the
fused mapping step, and torch.autograd.Functions over the C ABI.

Every numerical step runs in liblgs.so (binning, sorting, compositing, loss,
backward, Adam); this module only owns torch tensors and passes pointers.
Paper: Sec. 3.4 "Map Optimization" (rasterise the map into (D, A, N), the
losses of Eqs. depthloss / normalloss / scaleloss / totalloss, optimise
Theta = {mu, q, s~, alpha}).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import lib


@dataclass
class LossParams:
    """Weights of the paper's implementation details (Sec. 4.1)."""
    lambda_alpha: float = 0.1
    lambda_n: float = 1.0
    lambda_ng: float = 0.05
    lambda_s: float = 10.0
    s_max: float = 1.0
    lambda_ns: float = 0.0      # N_surf term: 0.01 once densification has begun (Sec. 3.4)

    def struct(self):
        return lib.lgs_loss_params(self.lambda_alpha, self.lambda_n, self.lambda_ng, self.lambda_s, self.s_max,
                                   self.lambda_ns)


def map_tensors(surf, device="cuda"):
    """scenes.Surfels (NumPy) -> [mean, quat, log_scale, logit] float32 device tensors."""
    return [torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)
            for a in (surf.mean, surf.quat, surf.log_scale, surf.logit)]


def target_tensors(tgt, device="cuda"):
    return (torch.from_numpy(np.ascontiguousarray(tgt.D, np.float32)).to(device),
            torch.from_numpy(np.ascontiguousarray(tgt.N, np.float32)).to(device))


# Compositing knobs (lgs_tuning) and tile shape the benchmark runs with: the
# 200k-surfel 128 x 1024 street frame renders fastest with 8 x 8 tiles and
# both passes as an independent walk per warp that stages the records of each
# 32-entry chunk's hits in its own shared memory.
DEFAULT_TUNING = dict(lib.DEFAULT_TUNING)
DEFAULT_TILE = (8, 8)


class Rasterizer:
    """Renders ``frames`` (scenes.Frame) of one or more maps; frame f shows
    map ``frame_map[f]``.  Holds the forward outputs and upstream-gradient
    planes of the last call."""

    def __init__(self, frames, frame_map=None, device: int = 0, loss: LossParams | None = None,
                 hbm_budget_bytes: int = 0, pairs_per_item: float = 4.0, tuning: dict | None = None):
        self.device = torch.device("cuda", device)
        self.session = lib.Session(device, hbm_budget_bytes, pairs_per_item=pairs_per_item)
        self.tuning = dict(DEFAULT_TUNING, **(tuning or {}))
        lib.lgs_session_set_tuning(self.session.handle, **self.tuning)
        self.loss_params = loss or LossParams()
        self.set_frames(frames, frame_map)

    def set_frames(self, frames, frame_map=None, outs=None, ups=None):
        """Frames of the next calls; ``outs`` / ``ups`` (per frame: FwdBuffers
        and the (dA, dS_t, dS_n) planes) may be supplied to avoid allocation."""
        self.frames = list(frames)
        self.frame_map = list(frame_map) if frame_map is not None else [0] * len(self.frames)
        self.fr = [lib.frame_struct(f) for f in self.frames]
        self.out = list(outs) if outs is not None else [lib.alloc_fwd(f, self.device) for f in self.frames]
        self.up = list(ups) if ups is not None else [upstream_planes(f, self.device) for f in self.frames]
        z = dict(dtype=torch.float32, device=self.device)
        self.n_maps = max(self.frame_map) + 1
        self.loss_out = torch.zeros(1 + lib.LOSS_TERMS * len(self.frames) + self.n_maps, **z)

    def set_timing(self, enable: bool):
        """Bracket every kernel group of this rasterizer with CUDA events."""
        lib.lgs_session_set_timing(self.session.handle, enable)

    def kernel_times(self):
        """{group: (device ms summed, calls)} of the timed calls since the last read."""
        return lib.lgs_session_kernel_times(self.session.handle)

    def close(self):
        self.session.close()

    @property
    def stream(self):
        return torch.cuda.current_stream(self.device).cuda_stream

    # -- the four calls of the hot path ------------------------------------
    def bin_sort(self, maps, check: bool = True):
        S = [lib.surfels_struct(*m) for m in maps]
        self.session.bin_sort(S, self.fr, self.frame_map, self.stream, check=check)
        return S

    def forward(self, maps, S=None):
        S = S or [lib.surfels_struct(*m) for m in maps]
        lib.lgs_render_fwd_batch(self.session.handle, S, self.fr, self.frame_map, [o.struct() for o in self.out],
                                 self.stream)
        return self.out

    def loss(self, maps, targets, grads=None, S=None):
        """Writes the upstream planes; adds the scale-regulariser gradient into
        ``grads`` (list per map of 4 tensors) when given.  Returns the device
        loss vector [L, per-frame terms..., per-map L]."""
        S = S or [lib.surfels_struct(*m) for m in maps]
        tg = [lib.lgs_target(d.data_ptr(), n.data_ptr()) for d, n in targets]
        go = [lib.lgs_fwd_grad_out(a.data_ptr(), b.data_ptr(), c.data_ptr()) for a, b, c in self.up]
        gs = [lib.grad_struct(*g) for g in grads] if grads is not None else None
        lib.lgs_loss_batch(self.session.handle, S, self.fr, self.frame_map, [o.struct() for o in self.out], tg,
                           self.loss_params.struct(), go, gs, self.loss_out.data_ptr(), self.stream)
        return self.loss_out

    def backward(self, maps, grads, upstream=None, S=None):
        S = S or [lib.surfels_struct(*m) for m in maps]
        up = upstream if upstream is not None else self.up
        lib.lgs_render_bwd_batch(self.session.handle, S, self.fr, self.frame_map, [o.struct() for o in self.out],
                                 [lib.lgs_fwd_grad(a.data_ptr(), b.data_ptr(), c.data_ptr()) for a, b, c in up],
                                 [lib.grad_struct(*g) for g in grads], self.stream)

    def forward_loss(self, maps, targets, grads=None, S=None):
        """Forward and loss in one library call (the image terms in the
        compositing kernel's epilogue when the tuning and the loss weights
        allow it; the same outputs either way)."""
        S = S or [lib.surfels_struct(*m) for m in maps]
        tg = [lib.lgs_target(d.data_ptr(), n.data_ptr()) for d, n in targets]
        go = [lib.lgs_fwd_grad_out(a.data_ptr(), b.data_ptr(), c.data_ptr()) for a, b, c in self.up]
        gs = [lib.grad_struct(*g) for g in grads] if grads is not None else None
        lib.lgs_render_fwd_loss_batch(self.session.handle, S, self.fr, self.frame_map, [o.struct() for o in self.out],
                                      tg, self.loss_params.struct(), go, gs, self.loss_out.data_ptr(), self.stream)
        return self.loss_out

    def step(self, maps, targets, grads, check: bool = False):
        """One mapping step: bin + sort, forward with the loss, backward.
        Gradients are accumulated into ``grads``; returns the device loss
        vector."""
        S = self.bin_sort(maps, check=check)
        self.forward_loss(maps, targets, grads, S)
        self.backward(maps, grads, S=S)
        return self.loss_out

    def counters(self):
        return lib.lgs_session_counters(self.session.handle)


def upstream_planes(frame, device):
    z = dict(dtype=torch.float32, device=device)
    return (torch.zeros(frame.H, frame.W, **z), torch.zeros(frame.H, frame.W, **z),
            torch.zeros(3, frame.H, frame.W, **z))


def adam_step_batch(items, betas=(0.9, 0.999), eps: float = 1e-15, zero_grad: bool = True, stream=None):
    """One fused Adam launch over several maps: items = [(params, grads,
    m_state, v_state, step, lr)] with each map's own step count."""
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    maps = []
    for params, grads, m, v, step, lr in items:
        maps.append(lib.lgs_adam_map(params[0].data_ptr(), params[1].data_ptr(), params[2].data_ptr(),
                                     params[3].data_ptr(), lib.grad_struct(*grads), m.data_ptr(), v.data_ptr(),
                                     int(params[0].shape[0]), int(step), (ctypes.c_float * 4)(*lr)))
    for k in range(0, len(maps), 64):
        lib.lgs_adam_step_batch(maps[k:k + 64], betas[0], betas[1], eps, zero_grad, s)


def adam_step(params, grads, m_state, v_state, step: int, lr=(1e-3, 1e-3, 5e-3, 5e-3), betas=(0.9, 0.999),
              eps: float = 1e-15, zero_grad: bool = True, stream=None):
    """Fused Adam over one map's 10 parameters per surfel (liblgs kernel).
    lr: (mean, quat, log_scale, logit)."""
    n = int(params[0].shape[0])
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    lib.lgs_adam_step(params[0].data_ptr(), params[1].data_ptr(), params[2].data_ptr(), params[3].data_ptr(),
                      lib.grad_struct(*grads), m_state.data_ptr(), v_state.data_ptr(), n, step, lr, betas[0],
                      betas[1], eps, zero_grad, s)


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------
class LgsRender(torch.autograd.Function):
    """(mean, quat, log_scale, logit) -> (A, S_t, S_n) stacked over the
    rasterizer's frames (all frames of one map, equal H x W).  The backward
    recomputes the forward per tile in reverse order (no stored lists)."""

    @staticmethod
    def forward(ctx, rast: Rasterizer, mean, quat, log_scale, logit):
        maps = [[mean.detach().contiguous(), quat.detach().contiguous(), log_scale.detach().contiguous(),
                 logit.detach().contiguous()]]
        S = rast.bin_sort(maps)
        rast.forward(maps, S)
        ctx.rast = rast
        ctx.maps = maps
        A = torch.stack([o.A for o in rast.out])
        St = torch.stack([o.S_t for o in rast.out])
        Sn = torch.stack([o.S_n for o in rast.out])
        return A, St, Sn

    @staticmethod
    def backward(ctx, gA, gSt, gSn):
        rast = ctx.rast
        maps = ctx.maps
        F = len(rast.frames)
        z = lambda t, ref: torch.zeros_like(ref) if t is None else t.contiguous()
        up = [(z(gA, rast.out[0].A.expand(F, -1, -1))[f].contiguous(),
               z(gSt, rast.out[0].S_t.expand(F, -1, -1))[f].contiguous(),
               z(gSn, rast.out[0].S_n.expand(F, -1, -1, -1))[f].contiguous()) for f in range(F)]
        grads = [[torch.zeros_like(t) for t in maps[0]]]
        rast.backward(maps, grads, upstream=up)
        return (None, *grads[0])


class LgsLoss(torch.autograd.Function):
    """Mapping loss of the paper (Eqs. depthloss, normalloss, scaleloss,
    totalloss) of the rasterizer's last forward: inputs (A, S_t, S_n) from
    LgsRender and log_scale; returns the scalar L (image terms averaged over
    frames + lambda_s L_scale)."""

    @staticmethod
    def forward(ctx, rast: Rasterizer, targets, A, St, Sn, mean, quat, log_scale, logit):
        for f, o in enumerate(rast.out):
            o.A.copy_(A[f]); o.S_t.copy_(St[f]); o.S_n.copy_(Sn[f])
        maps = [[mean.detach().contiguous(), quat.detach().contiguous(), log_scale.detach().contiguous(),
                 logit.detach().contiguous()]]
        g_ls = torch.zeros_like(maps[0][2])
        grads = [[torch.zeros_like(maps[0][0]), torch.zeros_like(maps[0][1]), g_ls, torch.zeros_like(maps[0][3])]]
        out = rast.loss(maps, targets, grads)
        ctx.save_for_backward(torch.stack([u[0] for u in rast.up]), torch.stack([u[1] for u in rast.up]),
                              torch.stack([u[2] for u in rast.up]), g_ls)
        return out[0].clone()

    @staticmethod
    def backward(ctx, go):
        gA, gSt, gSn, g_ls = ctx.saved_tensors
        return None, None, gA * go, gSt * go, gSn * go, None, None, g_ls * go, None
