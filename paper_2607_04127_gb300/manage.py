"""Map management on the device (paper Sec. 3.3 control score, Sec. 3.5
"Real-time Map Budget Control"): opacity prune, multi-pass planar
cover-and-prune and structure-aware split, computed by liblgs.so
(lgs_map_manage, lgs_map_gather).  This module only owns the torch buffers."""
from __future__ import annotations

import torch

from . import lib

FIELDS = ("alpha_prune", "alpha_min", "w_l", "w_c", "w_r", "q_res", "eps", "q_plane", "voxel", "n_passes",
          "q_cover", "slab", "prune_cap", "q_split", "split_cap", "split_shift", "split_dlog")


def params(**overrides) -> "lib.lgs_manage_params":
    """The library's default parameters with the given fields replaced."""
    p = lib.lgs_manage_default_params()
    for k, v in overrides.items():
        if k not in FIELDS:
            raise KeyError(f"unknown map-management parameter {k!r}")
        setattr(p, k, v)
    return p


class MapManager:
    """Runs map-management steps on one device; keeps the scratch buffer
    between calls (it grows with the map)."""

    def __init__(self, device=0):
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        self._scratch = None

    def _scratch_for(self, n: int) -> torch.Tensor:
        need = max(lib.lgs_manage_scratch_bytes(n), 256)
        if self._scratch is None or self._scratch.numel() < need:
            self._scratch = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
        return self._scratch

    def launch(self, surf, lam, res, p=None, out=None, stream=None):
        """Enqueue one step without a host sync.  surf: [mean, quat,
        log_scale, logit] float32 device tensors; lam [n, 3], res [n].
        Returns a dict of device tensors of full capacity: mean, quat,
        log_scale, logit (rows [0, counts[0]) valid), score [n], src, role,
        counts [6] (n_out, opacity-pruned, pruned by passes 0..2, split)."""
        p = p if p is not None else params()
        n = int(surf[0].shape[0])
        cap = lib.lgs_manage_capacity(n, p)
        if cap < 0:
            raise ValueError("invalid split_cap")
        dev = self.device
        if out is None:
            out = dict(mean=torch.empty(max(cap, 1), 3, device=dev), quat=torch.empty(max(cap, 1), 4, device=dev),
                       log_scale=torch.empty(max(cap, 1), 2, device=dev), logit=torch.empty(max(cap, 1), device=dev),
                       score=torch.empty(max(n, 1), device=dev),
                       src=torch.empty(max(cap, 1), dtype=torch.int32, device=dev),
                       role=torch.empty(max(cap, 1), dtype=torch.uint8, device=dev),
                       counts=torch.zeros(6, dtype=torch.int64, device=dev))
        for t in (lam, res):
            if not (t.is_cuda and t.is_contiguous() and t.dtype == torch.float32):
                raise ValueError("lam and res must be contiguous float32 CUDA tensors")
        scratch = self._scratch_for(n)
        base = scratch.data_ptr()
        aligned = (base + 255) // 256 * 256
        s = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
        o = lib.lgs_surfel_params_out(out["mean"].data_ptr(), out["quat"].data_ptr(), out["log_scale"].data_ptr(),
                                      out["logit"].data_ptr())
        lib.lgs_map_manage(lib.surfels_struct(*surf), lam.data_ptr(), res.data_ptr(), p, aligned,
                           scratch.numel() - (aligned - base), out["score"].data_ptr(), o, cap,
                           out["src"].data_ptr(), out["role"].data_ptr(), out["counts"].data_ptr(), s)
        out["capacity"] = cap
        return out

    def gather(self, out, arrays, zero_children: bool = True, stream=None):
        """Carry per-surfel arrays (e.g. Adam moments, [n, k] float32) over to
        the new map of a launched step: rows [0, capacity), children zeroed
        when asked."""
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        res = []
        for a in arrays:
            if not (a.is_cuda and a.is_contiguous() and a.element_size() == 4):
                raise ValueError("gathered arrays must be contiguous 32-bit CUDA tensors")
            words = 1
            for d in a.shape[1:]:
                words *= int(d)
            o = torch.empty((max(out["capacity"], 1),) + tuple(a.shape[1:]), dtype=a.dtype, device=a.device)
            lib.lgs_map_gather(out["src"].data_ptr(), out["role"].data_ptr(), out["counts"].data_ptr(),
                               out["capacity"], a.data_ptr(), o.data_ptr(), words, int(zero_children), s)
            res.append(o)
        return res

    def step(self, surf, lam, res, p=None, carry=(), zero_children: bool = True):
        """One step with one host read of the new map's size: returns
        (new surf list, carried arrays, info dict with score, src, role,
        counts as host ints)."""
        out = self.launch(surf, lam, res, p)
        carried = self.gather(out, carry, zero_children) if carry else []
        counts = out["counts"].cpu().tolist()
        k = counts[0]
        new = [out["mean"][:k], out["quat"][:k], out["log_scale"][:k], out["logit"][:k]]
        info = dict(score=out["score"][: int(surf[0].shape[0])], src=out["src"][:k], role=out["role"][:k],
                    counts=counts)
        return new, [c[:k] for c in carried], info
