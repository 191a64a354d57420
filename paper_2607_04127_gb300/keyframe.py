"""Keyframe initialisation of new surfels on the device (paper Sec. 3.2 k-NN
covariance; Sec. 3.3 range-adaptive scale, confidence u, opacity): liblgs.so's
lgs_keyframe_init.  This module only owns the torch buffers."""
from __future__ import annotations

import torch

from . import lib

FIELDS = ("k", "kappa", "s_min", "s_max", "r0", "c0", "eps", "alpha_min", "alpha_max")


def params(**overrides) -> "lib.lgs_init_params":
    """The library's default parameters with the given fields replaced."""
    p = lib.lgs_init_default_params()
    for key, v in overrides.items():
        if key not in FIELDS:
            raise KeyError(f"unknown initialisation parameter {key!r}")
        setattr(p, key, v)
    return p


def initialise(points: torch.Tensor, pose, p=None, stream=None, out=None, pairs=None):
    """points: [n, 3] float32 CUDA tensor of one scan in the sensor frame;
    pose: 12 numbers (sensor -> world, R row-major | t).  Returns a dict of
    device tensors: mean, quat, log_scale, logit (the new surfels), lam [n, 3]
    (covariance eigenvalues, descending), u [n] (confidence), knn [n, k].
    pairs: an optional int64 device tensor the k-NN adds its distance
    evaluations to."""
    if not (points.is_cuda and points.is_contiguous() and points.dtype == torch.float32):
        raise ValueError("points must be a contiguous float32 CUDA tensor")
    p = p if p is not None else params()
    n = int(points.shape[0])
    dev = points.device
    if out is None:
        m = max(n, 1)
        out = dict(mean=torch.empty(m, 3, device=dev), quat=torch.empty(m, 4, device=dev),
                   log_scale=torch.empty(m, 2, device=dev), logit=torch.empty(m, device=dev),
                   lam=torch.empty(m, 3, device=dev), u=torch.empty(m, device=dev),
                   knn=torch.empty(m, p.k, dtype=torch.int32, device=dev),
                   scratch=torch.empty(max(lib.lgs_init_scratch_bytes(n), 16), dtype=torch.uint8, device=dev))
    s = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
    o = lib.lgs_surfel_params_out(out["mean"].data_ptr(), out["quat"].data_ptr(), out["log_scale"].data_ptr(),
                                  out["logit"].data_ptr())
    lib.lgs_keyframe_init(points.data_ptr(), n, pose, p, out["scratch"].data_ptr(), out["scratch"].numel(),
                          out["knn"].data_ptr(), o, out["lam"].data_ptr(), out["u"].data_ptr(), s,
                          pairs.data_ptr() if pairs is not None else 0)
    return out
