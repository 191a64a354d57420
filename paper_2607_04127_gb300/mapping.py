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

# floats per surfel of each parameter group, in the order of the Adam state's
# group-major layout [mean 3n | quat 4n | log-scale 2n | logit n]
GROUP_WIDTHS = (3, 4, 2, 1)


def state_blocks(state: torch.Tensor, n: int):
    """The four group blocks of an Adam state of n surfels as [n, width]
    views."""
    blocks, off = [], 0
    for w in GROUP_WIDTHS:
        blocks.append(state[off:off + w * n].view(n, w))
        off += w * n
    return blocks


def state_from_blocks(blocks) -> torch.Tensor:
    """The inverse of ``state_blocks``: the blocks' rows, group-major."""
    return torch.cat([b.reshape(-1) for b in blocks])


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
        self._check_next = False   # the map changed size: the next bin checks capacity
        self._manager = None

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
        out = self.rast.step([[p.detach() for p in self.params]], self.targets, [self.grads],
                             check=self.t == 0 or self._check_next)
        self._check_next = False
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

    # -- growing and budgeting the map ----------------------------------------
    def _adopt(self, params, m, v):
        self.params = [p.detach().contiguous().requires_grad_(self.autograd) for p in params]
        self.m, self.v = m.contiguous(), v.contiguous()
        if not self.autograd:
            self.grads = [torch.zeros_like(p) for p in self.params]
        self._check_next = True

    def insert_keyframe(self, points, pose, init=None):
        """New surfels at the points of a keyframe scan (Sec. 3.2 covariance,
        Sec. 3.3 range-adaptive scale, confidence and opacity), appended to the
        map with zero Adam moments.  points: [k, 3] float32 device tensor in
        the sensor frame; pose: 12 numbers (sensor -> world); init: the
        initialisation parameters (``keyframe.params``).  Returns the new
        surfels' covariance eigenvalues [k, 3] and confidence u [k]."""
        from . import keyframe
        k = int(points.shape[0])
        out = keyframe.initialise(points, pose, init)
        new = [out["mean"][:k], out["quat"][:k], out["log_scale"][:k], out["logit"][:k]]
        params = [torch.cat([p.detach(), q]) for p, q in zip(self.params, new)]
        n = self.n
        grown = []
        for state in (self.m, self.v):
            blocks = state_blocks(state, n)
            grown.append(state_from_blocks(
                [torch.cat([b, torch.zeros(k, b.shape[1], dtype=b.dtype, device=b.device)]) for b in blocks]))
        self._adopt(params, grown[0], grown[1])
        return out["lam"][:k], out["u"][:k]

    def manage(self, lam, res, params=None):
        """One map-management step (Sec. 3.3 control score; Sec. 3.5 opacity
        prune, planar cover-and-prune, structure-aware split) on the map.  lam
        [n, 3] and res [n]: the surfels' tracking covariance eigenvalues and
        G-ICP residuals (device, float32).  The Adam moments follow their
        surfels; children start from zero moments.  Returns the counts
        (n_out, opacity-pruned, pruned by the three passes, split) and each new
        surfel's parent index (device int32 [n_out])."""
        from . import manage
        n = self.n
        if self._manager is None:
            self._manager = manage.MapManager(self.device)
        out = self._manager.launch([p.detach() for p in self.params], lam, res, params)
        counts = [int(c) for c in out["counts"].cpu().tolist()]
        k = counts[0]
        carried = self._manager.gather(out, state_blocks(self.m, n) + state_blocks(self.v, n), zero_children=True)
        m = state_from_blocks([c[:k] for c in carried[:4]])
        v = state_from_blocks([c[:k] for c in carried[4:]])
        params = [out["mean"][:k], out["quat"][:k], out["log_scale"][:k], out["logit"][:k]]
        self._adopt([p.clone() for p in params], m, v)
        return counts, out["src"][:k].clone()

    def close(self):
        self.rast.close()
