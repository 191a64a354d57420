"""Thin ctypes binding of ``liblgs.so`` (C ABI in ``include/lgs.h``).

Every function named ``lgs_*`` here marshals its arguments and calls the C
entry point of the same name; nothing of the rasterizer is computed in
Python.  ``Session`` adds workspace management on top (a torch-allocated
device buffer that grows when the pair capacity is exceeded) and accepts
torch CUDA tensors.  Loading fails loudly when the library is missing: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblgs.so")
_lib = None

LGS_MAX_FRAMES = 64
LGS_MAX_MAPS = 64
STATUS = {0: "LGS_OK", 1: "LGS_ERR_INVALID_ARG", 2: "LGS_ERR_CAPACITY", 3: "LGS_ERR_BUDGET", 4: "LGS_ERR_CUDA",
          5: "LGS_ERR_TIMEOUT", 6: "LGS_ERR_DEVICE_CHECK", 7: "LGS_ERR_NO_WORKSPACE", 8: "LGS_ERR_STATE"}
LGS_OK, LGS_ERR_CAPACITY = 0, 2
LOSS_TERMS = 4           # per-frame image terms in a loss vector: L_depth, L_alpha, L_ng, L_ns

P = ctypes.c_void_p
F32P = ctypes.POINTER(ctypes.c_float)


class lgs_frame(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("tile_w", ctypes.c_int32), ("elev_min", ctypes.c_float), ("elev_max", ctypes.c_float),
                ("pose", ctypes.c_float * 12)]


class lgs_surfels(ctypes.Structure):
    _fields_ = [("mean", P), ("quat", P), ("log_scale", P), ("opacity_logit", P), ("n", ctypes.c_int64)]


class lgs_fwd_out(ctypes.Structure):
    _fields_ = [("A", P), ("S_t", P), ("S_n", P), ("T_final", P), ("n_contrib", P)]


class lgs_fwd_grad(ctypes.Structure):
    _fields_ = [("dA", P), ("dS_t", P), ("dS_n", P)]


class lgs_fwd_grad_out(ctypes.Structure):
    _fields_ = [("dA", P), ("dS_t", P), ("dS_n", P)]


class lgs_surfel_grad(ctypes.Structure):
    _fields_ = [("d_mean", P), ("d_quat", P), ("d_log_scale", P), ("d_opacity_logit", P)]


class lgs_target(ctypes.Structure):
    _fields_ = [("D", P), ("N_gicp", P)]


class lgs_loss_params(ctypes.Structure):
    _fields_ = [("lambda_alpha", ctypes.c_float), ("lambda_n", ctypes.c_float), ("lambda_ng", ctypes.c_float),
                ("lambda_s", ctypes.c_float), ("s_max", ctypes.c_float), ("lambda_ns", ctypes.c_float)]


class lgs_adam_map(ctypes.Structure):
    _fields_ = [("mean", P), ("quat", P), ("log_scale", P), ("logit", P), ("grad", lgs_surfel_grad),
                ("m_state", P), ("v_state", P), ("n", ctypes.c_int64), ("step", ctypes.c_int64),
                ("lr", ctypes.c_float * 4)]


class lgs_tuning(ctypes.Structure):
    _fields_ = [("fwd_batch", ctypes.c_int32), ("bwd_batch", ctypes.c_int32), ("group", ctypes.c_int32),
                ("persistent", ctypes.c_int32)]


EXPORTS = [
    "lgs_session_create", "lgs_session_destroy", "lgs_session_workspace_size", "lgs_batch_workspace_size",
    "lgs_session_set_workspace", "lgs_session_status", "lgs_session_pair_count", "lgs_session_counters",
    "lgs_session_bins", "lgs_session_read_bins", "lgs_bin_sort", "lgs_render_fwd", "lgs_render_bwd", "lgs_loss", "lgs_bin_sort_batch",
    "lgs_render_fwd_batch", "lgs_render_bwd_batch", "lgs_loss_batch", "lgs_render_fwd_loss_batch",
    "lgs_session_set_tuning", "lgs_adam_step",
    "lgs_session_set_timing", "lgs_session_kernel_times", "lgs_image_loss_noalloc", "lgs_adam_step_batch",
    "lgs_status_string", "lgs_last_error", "lgs_constants", "lgs_version", "lgs_trackable_scratch_bytes",
    "lgs_trackable_targets", "lgs_manage_default_params", "lgs_manage_scratch_bytes", "lgs_manage_capacity", "lgs_manage_launches",
    "lgs_map_manage", "lgs_map_gather", "lgs_init_default_params", "lgs_init_scratch_bytes", "lgs_init_max_points", "lgs_init_launches",
    "lgs_keyframe_init", "lgs_session_status_enqueue", "lgs_status_of_word",
]


def load():
    """Load liblgs.so (built by ``build.py``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_2607_04127_gb300/build.py "
                           "(there is no CPU fallback for the rasterizer)")
    lib = ctypes.CDLL(LIB_PATH)
    i32, i64, sz = ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    S = ctypes.c_int
    sig = {
        "lgs_session_create": ([i32, sz, ctypes.POINTER(P)], S),
        "lgs_session_destroy": ([P], S),
        "lgs_session_workspace_size": ([P, i64, P, i32, i64, ctypes.POINTER(sz)], S),
        "lgs_batch_workspace_size": ([P, P, i32, P, P, i32, i64, ctypes.POINTER(sz)], S),
        "lgs_session_set_workspace": ([P, P, sz], S),
        "lgs_session_status": ([P, ctypes.POINTER(i64)], S),
        "lgs_session_pair_count": ([P, ctypes.POINTER(i64)], S),
        "lgs_session_status_enqueue": ([P, P, P], S),
        "lgs_status_of_word": ([P], S),
        "lgs_session_counters": ([P, P], S),
        "lgs_session_bins": ([P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P)], S),
        "lgs_session_read_bins": ([P, P, P, P, P, i64], S),
        "lgs_bin_sort": ([P, P, P, i32, P], S),
        "lgs_render_fwd": ([P, P, P, i32, P, P], S),
        "lgs_render_bwd": ([P, P, P, i32, P, P, P, P], S),
        "lgs_loss": ([P, P, P, i32, P, P, P, P, P, P, P], S),
        "lgs_bin_sort_batch": ([P, P, i32, P, P, i32, P], S),
        "lgs_render_fwd_batch": ([P, P, i32, P, P, i32, P, P], S),
        "lgs_render_bwd_batch": ([P, P, i32, P, P, i32, P, P, P, P], S),
        "lgs_loss_batch": ([P, P, i32, P, P, i32, P, P, P, P, P, P, P], S),
        "lgs_render_fwd_loss_batch": ([P, P, i32, P, P, i32, P, P, P, P, P, P, P], S),
        "lgs_trackable_scratch_bytes": ([i64], ctypes.c_size_t),
        "lgs_trackable_targets": ([P, P, P, P, P, ctypes.c_size_t, P, P, P, P, P, P], S),
        "lgs_manage_default_params": ([P], None),
        "lgs_manage_scratch_bytes": ([i64], ctypes.c_size_t),
        "lgs_manage_capacity": ([i64, P], i64),
        "lgs_manage_launches": ([P], i32),
        "lgs_map_manage": ([P, P, P, P, P, ctypes.c_size_t, P, P, i64, P, P, P, P], S),
        "lgs_map_gather": ([P, P, P, i64, P, P, i32, i32, P], S),
        "lgs_init_default_params": ([P], None),
        "lgs_init_scratch_bytes": ([i64], ctypes.c_size_t),
        "lgs_init_max_points": ([], i64),
        "lgs_init_launches": ([], i32),
        "lgs_keyframe_init": ([P, i64, P, P, P, ctypes.c_size_t, P, P, P, P, P, P], S),
        "lgs_session_set_tuning": ([P, P], S),
        "lgs_session_set_timing": ([P, i32], S),
        "lgs_session_kernel_times": ([P, P, P], S),
        "lgs_image_loss_noalloc": ([P, P, i32, P, P, P, P, P, P], S),
        "lgs_adam_step_batch": ([P, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float, i32, P], S),
        "lgs_adam_step": ([P, P, P, P, P, P, P, i64, i64, P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                           i32, P], S),
        "lgs_status_string": ([i32], ctypes.c_char_p),
        "lgs_last_error": ([], ctypes.c_char_p),
        "lgs_constants": ([P], None),
        "lgs_version": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


class LgsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(st: int):
    if st != LGS_OK:
        msg = load().lgs_last_error().decode()
        raise LgsError(st, msg)
    return st


def _ref(x):
    return ctypes.byref(x)


def _arr(ctype, items):
    a = (ctype * len(items))()
    for i, it in enumerate(items):
        a[i] = it
    return a


# ---------------------------------------------------------------------------
# Same-name wrappers of the C entry points (argument marshalling only)
# ---------------------------------------------------------------------------
def lgs_session_create(device: int = 0, hbm_budget_bytes: int = 0):
    h = P()
    _check(load().lgs_session_create(device, hbm_budget_bytes, ctypes.byref(h)))
    return h


def lgs_session_destroy(h):
    return load().lgs_session_destroy(h)


def lgs_session_workspace_size(h, n_surfels, frames, max_pairs) -> int:
    fr = _arr(lgs_frame, frames)
    out = ctypes.c_size_t()
    _check(load().lgs_session_workspace_size(h, n_surfels, fr, len(frames), max_pairs, ctypes.byref(out)))
    return out.value


def lgs_batch_workspace_size(h, map_sizes, frames, frame_map, max_pairs) -> int:
    ms = _arr(ctypes.c_int64, map_sizes)
    fr = _arr(lgs_frame, frames)
    fm = _arr(ctypes.c_int32, frame_map)
    out = ctypes.c_size_t()
    _check(load().lgs_batch_workspace_size(h, ms, len(map_sizes), fr, fm, len(frames), max_pairs,
                                           ctypes.byref(out)))
    return out.value


def lgs_session_set_workspace(h, ptr: int, nbytes: int):
    _check(load().lgs_session_set_workspace(h, P(ptr), nbytes))


def lgs_session_status(h):
    req = ctypes.c_int64()
    st = load().lgs_session_status(h, ctypes.byref(req))
    return st, req.value


def lgs_session_pair_count(h) -> int:
    n = ctypes.c_int64()
    _check(load().lgs_session_pair_count(h, ctypes.byref(n)))
    return n.value


def lgs_session_counters(h):
    out = (ctypes.c_int64 * 8)()
    _check(load().lgs_session_counters(h, out))
    return dict(n_pairs=out[0], n_visible=out[1], evals_fwd=out[2], evals_bwd=out[3], contrib_fwd=out[4],
                contrib_bwd=out[5], launches=out[6], alg_fwd=out[7])


TIME_GROUPS = ("desc", "bin", "fwd", "loss", "bwd", "bwd_chain")


def lgs_session_set_timing(h, enable: bool):
    _check(load().lgs_session_set_timing(h, 1 if enable else 0))


def lgs_session_kernel_times(h):
    """{group: (summed device ms, timed calls)} since the last read."""
    ms = (ctypes.c_double * 8)()
    n = (ctypes.c_int64 * 8)()
    _check(load().lgs_session_kernel_times(h, ms, n))
    return {g: (ms[i], n[i]) for i, g in enumerate(TIME_GROUPS)}


def lgs_session_bins(h):
    a, b, c, d = P(), P(), P(), P()
    _check(load().lgs_session_bins(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
    return a.value, b.value, c.value, d.value


def lgs_session_read_bins(h, n_items: int, n_tiles: int):
    """Host copies of the last bin_sort: (tile_of_pair, item_of_pair, ranges [T,2], depth_key)."""
    n_pairs = lgs_session_pair_count(h)
    tp = np.zeros(max(n_pairs, 1), np.uint32); ip = np.zeros(max(n_pairs, 1), np.uint32)
    rg = np.zeros((max(n_tiles, 1), 2), np.uint32); dk = np.zeros(max(n_items, 1), np.uint32)
    _check(load().lgs_session_read_bins(h, tp.ctypes.data, ip.ctypes.data, rg.ctypes.data, dk.ctypes.data,
                                        n_pairs))
    return tp[:n_pairs], ip[:n_pairs], rg[:n_tiles], dk[:n_items]


def lgs_bin_sort_batch(h, maps, frames, frame_map, stream):
    _check(load().lgs_bin_sort_batch(h, _arr(lgs_surfels, maps), len(maps), _arr(lgs_frame, frames),
                                     _arr(ctypes.c_int32, frame_map), len(frames), P(stream)))


def lgs_render_fwd_batch(h, maps, frames, frame_map, outs, stream):
    _check(load().lgs_render_fwd_batch(h, _arr(lgs_surfels, maps), len(maps), _arr(lgs_frame, frames),
                                       _arr(ctypes.c_int32, frame_map), len(frames), _arr(lgs_fwd_out, outs),
                                       P(stream)))


def lgs_render_bwd_batch(h, maps, frames, frame_map, fwd, upstream, grads, stream):
    _check(load().lgs_render_bwd_batch(h, _arr(lgs_surfels, maps), len(maps), _arr(lgs_frame, frames),
                                       _arr(ctypes.c_int32, frame_map), len(frames), _arr(lgs_fwd_out, fwd),
                                       _arr(lgs_fwd_grad, upstream), _arr(lgs_surfel_grad, grads), P(stream)))


def lgs_loss_batch(h, maps, frames, frame_map, fwd, targets, params, grads_out, grads, loss_out_ptr, stream):
    _check(load().lgs_loss_batch(h, _arr(lgs_surfels, maps), len(maps), _arr(lgs_frame, frames),
                                 _arr(ctypes.c_int32, frame_map), len(frames), _arr(lgs_fwd_out, fwd),
                                 _arr(lgs_target, targets), _ref(params), _arr(lgs_fwd_grad_out, grads_out),
                                 _arr(lgs_surfel_grad, grads) if grads is not None else None,
                                 P(loss_out_ptr), P(stream)))


def lgs_render_fwd_loss_batch(h, maps, frames, frame_map, fwd, targets, params, grads_out, grads, loss_out_ptr,
                              stream):
    _check(load().lgs_render_fwd_loss_batch(h, _arr(lgs_surfels, maps), len(maps), _arr(lgs_frame, frames),
                                            _arr(ctypes.c_int32, frame_map), len(frames), _arr(lgs_fwd_out, fwd),
                                            _arr(lgs_target, targets), _ref(params), _arr(lgs_fwd_grad_out, grads_out),
                                            _arr(lgs_surfel_grad, grads) if grads is not None else None,
                                            P(loss_out_ptr), P(stream)))


class lgs_track_params(ctypes.Structure):
    _fields_ = [("k_min", ctypes.c_int32), ("alpha_min", ctypes.c_float), ("thickness", ctypes.c_float),
                ("eps", ctypes.c_float), ("w_max", ctypes.c_float)]


def lgs_trackable_scratch_bytes(n):
    return int(load().lgs_trackable_scratch_bytes(int(n)))


def lgs_trackable_targets(surfels, mask_ptr, last_kf_ptr, params, scratch_ptr, scratch_bytes, index_ptr, mean_ptr,
                          cov_ptr, weight_ptr, count_ptr, stream):
    _check(load().lgs_trackable_targets(_ref(surfels), P(mask_ptr), P(last_kf_ptr), _ref(params), P(scratch_ptr),
                                        scratch_bytes, P(index_ptr), P(mean_ptr), P(cov_ptr), P(weight_ptr),
                                        P(count_ptr), P(stream)))


def lgs_bin_sort(h, surfels, frames, stream):
    _check(load().lgs_bin_sort(h, _ref(surfels), _arr(lgs_frame, frames), len(frames), P(stream)))


def lgs_render_fwd(h, surfels, frames, outs, stream):
    _check(load().lgs_render_fwd(h, _ref(surfels), _arr(lgs_frame, frames), len(frames), _arr(lgs_fwd_out, outs),
                                 P(stream)))


def lgs_render_bwd(h, surfels, frames, fwd, upstream, grad, stream):
    _check(load().lgs_render_bwd(h, _ref(surfels), _arr(lgs_frame, frames), len(frames), _arr(lgs_fwd_out, fwd),
                                 _arr(lgs_fwd_grad, upstream), _ref(grad), P(stream)))


def lgs_loss(h, surfels, frames, fwd, targets, params, grads_out, grad, loss_out_ptr, stream):
    _check(load().lgs_loss(h, _ref(surfels), _arr(lgs_frame, frames), len(frames), _arr(lgs_fwd_out, fwd),
                           _arr(lgs_target, targets), _ref(params), _arr(lgs_fwd_grad_out, grads_out),
                           _ref(grad) if grad is not None else None, P(loss_out_ptr), P(stream)))


class lgs_status_word(ctypes.Structure):
    _fields_ = [("required_pairs", ctypes.c_uint64), ("n_pairs", ctypes.c_uint64), ("n_visible", ctypes.c_uint32),
                ("overflow", ctypes.c_uint32), ("timeout", ctypes.c_uint32), ("check", ctypes.c_uint32)]


STATUS_WORD_BYTES = ctypes.sizeof(lgs_status_word)


def lgs_session_status_enqueue(h, out_ptr: int, stream):
    """Enqueue a copy of the status word into pinned host memory at out_ptr
    (STATUS_WORD_BYTES bytes); no synchronisation."""
    _check(load().lgs_session_status_enqueue(h, P(out_ptr), P(stream)))


def lgs_status_of_word(out_ptr: int):
    """(status code, required pairs) of a copied status word (read it only
    after the copy has completed)."""
    w = lgs_status_word.from_address(out_ptr)
    return int(load().lgs_status_of_word(P(out_ptr))), int(w.required_pairs)


# The session's own defaults (lgs_session_create): every knob left out of a
# set_tuning call takes these.
DEFAULT_TUNING = dict(fwd_batch=0, bwd_batch=0, group=16, persistent=0)


def lgs_session_set_tuning(h, fwd_batch: int = DEFAULT_TUNING["fwd_batch"], bwd_batch: int = DEFAULT_TUNING["bwd_batch"],
                           group: int = DEFAULT_TUNING["group"], persistent: int = DEFAULT_TUNING["persistent"]):
    _check(load().lgs_session_set_tuning(h, _ref(lgs_tuning(fwd_batch, bwd_batch, group, persistent))))


def lgs_adam_step(mean, quat, log_scale, logit, grad, m_state, v_state, n, step, lr, beta1, beta2, eps,
                  zero_grad, stream):
    lra = _arr(ctypes.c_float, [float(x) for x in lr])
    _check(load().lgs_adam_step(P(mean), P(quat), P(log_scale), P(logit), _ref(grad), P(m_state), P(v_state),
                                n, step, lra, beta1, beta2, eps, int(zero_grad), P(stream)))


def lgs_status_string(st: int) -> str:
    return load().lgs_status_string(st).decode()


def lgs_constants() -> np.ndarray:
    out = (ctypes.c_float * 16)()
    load().lgs_constants(out)
    return np.array(out[:], np.float32)


def lgs_version() -> str:
    return load().lgs_version().decode()


# ---------------------------------------------------------------------------
# Conversions from scenes.Frame / torch tensors
# ---------------------------------------------------------------------------
def frame_struct(fr) -> lgs_frame:
    f = lgs_frame()
    f.H, f.W, f.tile_h, f.tile_w = int(fr.H), int(fr.W), int(fr.tile_h), int(fr.tile_w)
    f.elev_min, f.elev_max = float(fr.elev_min), float(fr.elev_max)
    pose = np.asarray(fr.pose, np.float32).reshape(12)
    for k in range(12):
        f.pose[k] = float(pose[k])
    return f


class lgs_manage_params(ctypes.Structure):
    _fields_ = [("alpha_prune", ctypes.c_float), ("alpha_min", ctypes.c_float), ("w_l", ctypes.c_float),
                ("w_c", ctypes.c_float), ("w_r", ctypes.c_float), ("q_res", ctypes.c_float),
                ("eps", ctypes.c_float), ("q_plane", ctypes.c_float), ("voxel", ctypes.c_float),
                ("n_passes", ctypes.c_int32), ("q_cover", ctypes.c_float), ("slab", ctypes.c_float),
                ("prune_cap", ctypes.c_float), ("q_split", ctypes.c_float), ("split_cap", ctypes.c_float),
                ("split_shift", ctypes.c_float), ("split_dlog", ctypes.c_float)]


class lgs_surfel_params_out(ctypes.Structure):
    _fields_ = [("mean", P), ("quat", P), ("log_scale", P), ("opacity_logit", P)]


def lgs_manage_default_params() -> lgs_manage_params:
    p = lgs_manage_params()
    load().lgs_manage_default_params(_ref(p))
    return p


def lgs_manage_scratch_bytes(n) -> int:
    return int(load().lgs_manage_scratch_bytes(int(n)))


def lgs_manage_launches(params) -> int:
    return int(load().lgs_manage_launches(_ref(params)))


def lgs_manage_capacity(n, params) -> int:
    return int(load().lgs_manage_capacity(int(n), _ref(params)))


def lgs_map_manage(surfels, lam_ptr, res_ptr, params, scratch_ptr, scratch_bytes, score_ptr, out, capacity, src_ptr,
                   role_ptr, counts_ptr, stream):
    _check(load().lgs_map_manage(_ref(surfels), P(lam_ptr), P(res_ptr), _ref(params), P(scratch_ptr), scratch_bytes,
                                 P(score_ptr), _ref(out), int(capacity), P(src_ptr), P(role_ptr), P(counts_ptr),
                                 P(stream)))


def lgs_map_gather(src_ptr, role_ptr, counts_ptr, capacity, in_ptr, out_ptr, words_per_row, zero_children, stream):
    _check(load().lgs_map_gather(P(src_ptr), P(role_ptr), P(counts_ptr), int(capacity), P(in_ptr), P(out_ptr),
                                 int(words_per_row), int(zero_children), P(stream)))


class lgs_init_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("kappa", ctypes.c_float), ("s_min", ctypes.c_float),
                ("s_max", ctypes.c_float), ("r0", ctypes.c_float), ("c0", ctypes.c_float), ("eps", ctypes.c_float),
                ("alpha_min", ctypes.c_float), ("alpha_max", ctypes.c_float)]


def lgs_init_default_params() -> lgs_init_params:
    p = lgs_init_params()
    load().lgs_init_default_params(_ref(p))
    return p


def lgs_init_scratch_bytes(n) -> int:
    return int(load().lgs_init_scratch_bytes(int(n)))


def lgs_keyframe_init(points_ptr, n, pose, params, scratch_ptr, scratch_bytes, knn_ptr, out, lam_ptr, u_ptr, stream,
                      pairs_ptr=0):
    pose_arr = (ctypes.c_float * 12)(*[float(x) for x in pose])
    _check(load().lgs_keyframe_init(P(points_ptr), int(n), pose_arr, _ref(params), P(scratch_ptr), scratch_bytes,
                                    P(knn_ptr), _ref(out), P(lam_ptr), P(u_ptr), P(pairs_ptr) if pairs_ptr else None,
                                    P(stream)))


def surfels_struct(mean, quat, log_scale, logit) -> lgs_surfels:
    for t in (mean, quat, log_scale, logit):
        if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float32"):
            raise ValueError("surfel tensors must be contiguous float32 CUDA tensors")
    return lgs_surfels(mean.data_ptr(), quat.data_ptr(), log_scale.data_ptr(), logit.data_ptr(),
                       int(mean.shape[0]))


def grad_struct(g_mean, g_quat, g_ls, g_logit) -> lgs_surfel_grad:
    return lgs_surfel_grad(g_mean.data_ptr(), g_quat.data_ptr(), g_ls.data_ptr(), g_logit.data_ptr())


@dataclass
class FwdBuffers:
    """Per-frame forward outputs (torch CUDA tensors)."""
    A: "object"
    S_t: "object"
    S_n: "object"
    T_final: "object"
    n_contrib: "object"

    def struct(self) -> lgs_fwd_out:
        return lgs_fwd_out(self.A.data_ptr(), self.S_t.data_ptr(), self.S_n.data_ptr(), self.T_final.data_ptr(),
                           self.n_contrib.data_ptr())


def alloc_fwd(frame, device) -> FwdBuffers:
    import torch
    H, W = int(frame.H), int(frame.W)
    f32 = dict(dtype=torch.float32, device=device)
    return FwdBuffers(torch.empty(H, W, **f32), torch.empty(H, W, **f32), torch.empty(3, H, W, **f32),
                      torch.empty(H, W, **f32), torch.empty(H, W, dtype=torch.int32, device=device))


class Session:
    """A library session plus its torch-allocated workspace.

    ``bin_sort`` sizes the workspace from a pair estimate and, when the
    device reports that more pairs were needed, grows it and bins again
    (that check synchronises; pass ``check=False`` in steady-state loops whose
    workspace already has head-room, and call ``check_status`` later)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, pairs_per_item: float = 4.0,
                 headroom: float = 1.25):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.handle = lgs_session_create(device, hbm_budget_bytes)
        self.ws = None
        self.pairs_per_item = pairs_per_item
        self.headroom = headroom
        self.max_pairs = 0
        self._key = None

    def close(self):
        if self.handle:
            lgs_session_destroy(self.handle)
            self.handle = None
            self.ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, map_sizes, frames, frame_map, max_pairs: int):
        nbytes = lgs_batch_workspace_size(self.handle, map_sizes, frames, frame_map, max_pairs)
        if self.ws is None or self.ws.numel() < nbytes:
            self.ws = None
            self.ws = self.torch.empty(nbytes + 256, dtype=self.torch.uint8, device=self.device)
            base = (self.ws.data_ptr() + 255) // 256 * 256
            lgs_session_set_workspace(self.handle, base, nbytes)
        self.max_pairs = max_pairs
        self._key = (tuple(map_sizes), len(frames))

    def bin_sort(self, maps, frames, frame_map=None, stream=None, check: bool = True):
        """maps: list of lgs_surfels; frames: list of lgs_frame."""
        frame_map = list(frame_map) if frame_map is not None else [0] * len(frames)
        sizes = [int(m.n) for m in maps]
        items = sum(sizes[frame_map[f]] for f in range(len(frames)))
        want = int(max(1024, items * self.pairs_per_item))
        if self.ws is None or self._key != (tuple(sizes), len(frames)) or self.max_pairs < want:
            self.reserve(sizes, frames, frame_map, max(want, self.max_pairs))
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device).cuda_stream
        lgs_bin_sort_batch(self.handle, maps, frames, frame_map, s)
        if check:
            st, req = lgs_session_status(self.handle)
            if st == LGS_ERR_CAPACITY:
                self.pairs_per_item = max(self.pairs_per_item, self.headroom * req / max(items, 1))
                self.reserve(sizes, frames, frame_map, int(req * self.headroom) + 1024)
                lgs_bin_sort_batch(self.handle, maps, frames, frame_map, s)
                st, req = lgs_session_status(self.handle)
            _check(st)

    def check_status(self):
        st, req = lgs_session_status(self.handle)
        _check(st)
        return req


def lgs_image_loss_noalloc(shapes, fwd, targets, params, grads_out, loss_out_ptr: int, stream):
    """shapes: [(H, W)] per frame; fwd: [lgs_fwd_out]; targets: [lgs_target];
    params: lgs_loss_params; grads_out: [lgs_fwd_grad_out]; loss_out_ptr:
    device pointer to 1 + 3 n floats."""
    n = len(shapes)
    Hs = (ctypes.c_int32 * n)(*[h for h, _ in shapes])
    Ws = (ctypes.c_int32 * n)(*[w for _, w in shapes])
    _check(load().lgs_image_loss_noalloc(Hs, Ws, n, _arr(lgs_fwd_out, fwd), _arr(lgs_target, targets), _ref(params),
                                         _arr(lgs_fwd_grad_out, grads_out), loss_out_ptr, stream))


def lgs_adam_step_batch(items, beta1: float, beta2: float, eps: float, zero_grad: bool, stream):
    """items: list of lgs_adam_map."""
    _check(load().lgs_adam_step_batch(_arr(lgs_adam_map, items), len(items), beta1, beta2, eps,
                                      1 if zero_grad else 0, stream))
