"""Differentiable mapping over a window of keyframes (Sec. 3.4, map
optimisation): the surfel map is optimised against every keyframe's range
image and G-ICP normals by Adam steps on the mapping loss
(Eqs. depthloss, normalloss, scaleloss, totalloss).

Two drivers of the same kernels:

* ``autograd=True``: each iteration renders the window through
  ``render.LgsRender`` (forward; the backward recomputes the compositing per
  tile in reverse order, no per-pixel lists are stored), evaluates
  ``render.LgsLoss``, back-propagates with ``torch.autograd`` and takes one
  fused Adam step;
* ``autograd=False``: ``Rasterizer.step`` (bin + forward + loss + backward in
  four library calls) and the fused Adam step, without autograd bookkeeping.

The map's parameters and the Adam moments stay on the device.
"""
from __future__ import annotations

import torch

from . import render

# learning rates per parameter group (mean, quat, log_scale, logit): 1e-3 on
# positions, 5e-3 on scales and opacities; the rotation's rate is not given
# and takes the positions'
DEFAULT_LR = (1e-3, 1e-3, 5e-3, 5e-3)


class MappingWindow:
    """Optimises one surfel map (``scenes.Surfels``) against ``frames``
    (keyframes of equal H x W) with ``targets`` (``scenes.Target`` each)."""

    def __init__(self, surfels, frames, targets, device: int = 0, lr=DEFAULT_LR, betas=(0.9, 0.999),
                 eps: float = 1e-15, tuning: dict | None = None, loss: render.LossParams | None = None,
                 autograd: bool = True):
        self.device = torch.device("cuda", device)
        self.params = [p.requires_grad_(autograd) for p in render.map_tensors(surfels, self.device)]
        self.rast = render.Rasterizer(frames, device=device, tuning=tuning, loss=loss)
        self.targets = [render.target_tensors(t, self.device) for t in targets]
        n = self.params[0].shape[0]
        self.m = torch.zeros(10 * n, device=self.device)
        self.v = torch.zeros(10 * n, device=self.device)
        self.lr, self.betas, self.eps = tuple(lr), tuple(betas), eps
        self.autograd = autograd
        self.t = 0
        self.grads = None if autograd else [torch.zeros_like(p) for p in self.params]

    def set_loss_params(self, loss: render.LossParams):
        """Loss weights from the next iteration on (the paper switches the
        N_surf term, lambda_{n,s}, on once densification has begun)."""
        self.rast.loss_params = loss

    @property
    def n(self) -> int:
        return int(self.params[0].shape[0])

    def loss_and_grads(self):
        """One forward + backward; returns (loss tensor, [4 gradient tensors])."""
        if self.autograd:
            mean, quat, ls, logit = self.params
            for p in self.params:
                p.grad = None
            A, St, Sn = render.LgsRender.apply(self.rast, mean, quat, ls, logit)
            L = render.LgsLoss.apply(self.rast, self.targets, A, St, Sn, mean, quat, ls, logit)
            L.backward()
            return L.detach(), [p.grad for p in self.params]
        for g in self.grads:
            g.zero_()
        # the first bin sizes the workspace (a synchronising capacity check);
        # later ones reuse it and run() checks the status once at the end
        out = self.rast.step([[p.detach() for p in self.params]], self.targets, [self.grads], check=self.t == 0)
        return out[0].clone(), self.grads

    def iterate(self):
        """One mapping iteration (render all keyframes, loss, backward, Adam);
        returns the loss before the update (device scalar)."""
        L, grads = self.loss_and_grads()
        self.t += 1
        with torch.no_grad():
            render.adam_step([p.detach() for p in self.params], grads, self.m, self.v, self.t, lr=self.lr,
                             betas=self.betas, eps=self.eps, zero_grad=True)
        return L

    def run(self, iterations: int):
        """``iterations`` mapping iterations; returns their losses (device)."""
        losses = [self.iterate() for _ in range(iterations)]
        self.rast.session.check_status()
        return torch.stack([l.reshape(()) for l in losses])

    def close(self):
        self.rast.close()
