"""Tracking-side view of the map (paper Sec. 3.2): the trackable subset of
Eq. trackable_select with each member's surfel-like target covariance and
geometry weight, computed on the device by liblgs.so (lgs_trackable_targets);
this module only owns the torch buffers."""
from __future__ import annotations

import torch

from . import lib


def trackable_targets(params, mask, last_kf, k_min: int, alpha_min: float, thickness: float = 0.01,
                      eps: float = 1e-6, w_max: float = 10.0, stream=None):
    """params: [mean, quat, log_scale, logit] device tensors of one map; mask
    (uint8) and last_kf (int32) device tensors of its surfels.  Returns
    (index int32, mean [k,3], cov [k,6], weight [k]) device tensors of the
    selected surfels in ascending index (one host read of the count)."""
    dev = params[0].device
    n = int(params[0].shape[0])
    s = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
    scratch = torch.empty(max(lib.lgs_trackable_scratch_bytes(n), 4), dtype=torch.uint8, device=dev)
    index = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    mean = torch.empty(max(n, 1), 3, dtype=torch.float32, device=dev)
    cov = torch.empty(max(n, 1), 6, dtype=torch.float32, device=dev)
    weight = torch.empty(max(n, 1), dtype=torch.float32, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    p = lib.lgs_track_params(int(k_min), float(alpha_min), float(thickness), float(eps), float(w_max))
    lib.lgs_trackable_targets(lib.surfels_struct(*params), mask.data_ptr(), last_kf.data_ptr(), p,
                              scratch.data_ptr(), scratch.numel(), index.data_ptr(), mean.data_ptr(),
                              cov.data_ptr(), weight.data_ptr(), count.data_ptr(), s)
    k = int(count.item())
    return index[:k], mean[:k], cov[:k], weight[:k]
