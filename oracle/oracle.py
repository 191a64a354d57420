"""Python driver for the FP64 CPU oracle (``lgs_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the product path
never does.  It shares no code with the CUDA library: it builds its own shared
object with gcc and passes plain NumPy arrays through ctypes.

What the oracle computes follows the paper's map representation (Sec. 3.1)
and map optimisation (Sec. 3.4, Eqs. depthloss, normalloss, scaleloss,
totalloss); binning and the depth key are specified in binary32, everything
else is FP64 (see ``lgs_oracle.c``).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lgs_oracle.c")
# the method and, in its own translation unit, the binary32 allowance the
# parity tests add to their bars; both include the shared internal header
_SOURCES = [_SRC, os.path.join(_HERE, "lgs_fp32_allowance.c")]
_DEPS = _SOURCES + [os.path.join(_HERE, "lgs_oracle_impl.h")]
_LIB_PATH = os.path.join(_HERE, "liblgs_oracle.so")
_lib = None
_lock = threading.Lock()

# Loss weights of the paper's implementation details (Sec. 4.1): lambda_alpha,
# lambda_n, lambda_s, lambda_{n,g}, lambda_{n,s}.  The N_surf term (weight
# lambda_{n,s}) is switched on only once densification has begun (Sec. 3.4),
# so loss_image takes it as an argument that defaults to off.
LAMBDA_ALPHA = 0.1
LAMBDA_N = 1.0
LAMBDA_S = 10.0
LAMBDA_NG = 0.05
LAMBDA_NS = 0.01
S_MAX = 1.0


def build(force: bool = False, out: str | None = None, defines=()) -> str:
    """Compile the oracle with gcc (binary32 binning needs -ffp-contract=off).
    ``out`` and ``defines`` (``NAME=value`` strings) build a variant elsewhere:
    the allowance tests plant a mistake in a bound that way."""
    path = out or _LIB_PATH
    if (not force and out is None and os.path.exists(path)
            and all(os.path.getmtime(path) >= os.path.getmtime(f) for f in _DEPS)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", *[f"-D{d}" for d in defines], *_SOURCES, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64, i32, f32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_double
        lib.lgso_constants.argtypes = [P]
        lib.lgso_f32_exp_spec.argtypes = [f32]; lib.lgso_f32_exp_spec.restype = f32
        lib.lgso_f32_exp_spec_n.argtypes = [P, P, i64]
        lib.lgso_f32_sin_spec.argtypes = [f32]; lib.lgso_f32_sin_spec.restype = f32
        lib.lgso_f32_cos_spec.argtypes = [f32]; lib.lgso_f32_cos_spec.restype = f32
        lib.lgso_f32_col_dir.argtypes = [i32, i32, P, P]
        lib.lgso_bin_tables.argtypes = [i32, i32, i32, i32, f32, f32, P, P, P]
        lib.lgso_bin_frame.argtypes = [P, P, i64, i32, i32, i32, i32, f32, f32, P, P, P, P, P, i64, P]
        lib.lgso_bin_frame.restype = i64
        lib.lgso_render_fwd.argtypes = [P, P, P, P, i64, i32, i32, i32, i32, f64, f64, P, P, P,
                                        P, P, P, P, P, P, P, P, P, P, i32]
        lib.lgso_coverage_misses.argtypes = [P, P, P, P, i64, i32, i32, i32, i32, f64, f64, P, P, P]
        lib.lgso_coverage_misses.restype = i64
        lib.lgso_render_bwd.argtypes = [P, P, P, P, i64, i32, i32, i32, i32, f64, f64, P, P, P,
                                        P, P, P, P, P, P, P, P, P, i32]
        lib.lgso_loss_image.argtypes = [P, P, P, P, P, i64, f64, f64, f64, f64, P, P, P, P]
        lib.lgso_loss_image.restype = f64
        lib.lgso_surf_normal_loss.argtypes = [P, P, P, P, ctypes.c_int, ctypes.c_int, f64, f64, f64, f64, P, P, P,
                                              P]
        lib.lgso_surf_normal_loss.restype = f64
        lib.lgso_scale_reg.argtypes = [P, i64, f64, f64, P]
        lib.lgso_scale_reg.restype = f64
        lib.lgso_pixel_detail.argtypes = [P, P, P, P, i64, i32, i32, i32, i32, f64, f64, P, P, P, i32, i32,
                                          f64, f64, P, i64] + [P] * 17
        lib.lgso_pixel_detail.restype = i64
        lib.lgso_contrib_with.argtypes = [P, P, P, P, i64, i32, i32, f64, f64, P, i32, i32, P, f64, f64, f64, f64,
                                          P, P]
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def constants() -> np.ndarray:
    out = np.zeros(16, np.float64)
    _load().lgso_constants(_p(out))
    return out


# --- specified binary32 helpers (exported for their own tests) --------------
def f32_exp_spec(x: float) -> np.float32:
    return np.float32(_load().lgso_f32_exp_spec(float(np.float32(x))))


def f32_exp_spec_n(x) -> np.ndarray:
    """f32_exp_spec over an array (binary32 in, binary32 out)."""
    x = np.ascontiguousarray(x, np.float32)
    y = np.empty_like(x)
    _load().lgso_f32_exp_spec_n(_p(x), _p(y), x.size)
    return y


def f32_sin_spec(x: float) -> np.float32:
    return np.float32(_load().lgso_f32_sin_spec(float(np.float32(x))))


def f32_cos_spec(x: float) -> np.float32:
    return np.float32(_load().lgso_f32_cos_spec(float(np.float32(x))))


def f32_col_dir(c: int, W: int):
    cs = np.zeros(1, np.float32); sn = np.zeros(1, np.float32)
    _load().lgso_f32_col_dir(int(c), int(W), _p(cs), _p(sn))
    return cs[0], sn[0]


def bin_tables(frame):
    ntr = -(-frame.H // frame.tile_h); ntc = -(-frame.W // frame.tile_w)
    st = np.zeros(ntr, np.float32); sb = np.zeros(ntr, np.float32); c4 = np.zeros((ntc, 4), np.float32)
    _load().lgso_bin_tables(frame.H, frame.W, frame.tile_h, frame.tile_w, float(np.float32(frame.elev_min)),
                            float(np.float32(frame.elev_max)), _p(st), _p(sb), _p(c4))
    return st, sb, c4


# --- binning / sort ---------------------------------------------------------
def bin_frame(surfels, frame, want_pairs: bool = True):
    """Binary32 binning of one frame: depth key bits, tile counts, and the
    (tile<<32 | depth_bits, surfel) pairs in sorted order with tile ranges."""
    lib = _load()
    mean = _c(surfels.mean, np.float32); ls = _c(surfels.log_scale, np.float32)
    pose = _c(frame.pose, np.float32)
    n = mean.shape[0]
    ntiles = (-(-frame.H // frame.tile_h)) * (-(-frame.W // frame.tile_w))
    depth = np.zeros(n, np.uint32); cnt = np.zeros(n, np.int32)
    args = (frame.H, frame.W, frame.tile_h, frame.tile_w, float(np.float32(frame.elev_min)),
            float(np.float32(frame.elev_max)), _p(pose))
    total = lib.lgso_bin_frame(_p(mean), _p(ls), n, *args, _p(depth), _p(cnt), None, None, 0, None)
    out = dict(depth_bits=depth, count=cnt, n_pairs=int(total))
    if want_pairs:
        keys = np.zeros(max(total, 1), np.uint64); vals = np.zeros(max(total, 1), np.uint32)
        ranges = np.zeros((ntiles, 2), np.int64)
        lib.lgso_bin_frame(_p(mean), _p(ls), n, *args, None, None, _p(keys), _p(vals), total, _p(ranges))
        out.update(keys=keys[:total], vals=vals[:total], ranges=ranges)
    return out


def brute_lists(surfels, frame):
    """All-pairs lists: every tile lists every surfel, ordered by (binary32
    depth key, index) -- the order the tiled lists use."""
    b = bin_frame(surfels, frame, want_pairs=False)
    order = np.lexsort((np.arange(len(b["depth_bits"])), b["depth_bits"])).astype(np.uint32)
    ntiles = (-(-frame.H // frame.tile_h)) * (-(-frame.W // frame.tile_w))
    ranges = np.zeros((ntiles, 2), np.int64); ranges[:, 1] = len(order)
    return ranges, order


# --- FP64 forward / backward -------------------------------------------------
def _params64(surfels):
    return (_c(surfels.mean, np.float64), _c(surfels.quat, np.float64),
            _c(surfels.log_scale, np.float64), _c(surfels.logit, np.float64))


def _frame_args(frame):
    return (frame.H, frame.W, frame.tile_h, frame.tile_w, float(np.float32(frame.elev_min)),
            float(np.float32(frame.elev_max)), _c(np.asarray(frame.pose, np.float32), np.float64))


def render_fwd(surfels, frame, ranges, vals, params64=None, nthreads: int = 0, allowance: bool = True):
    """FP64 forward of one frame over the given tile lists.  allowance=False
    skips the binary32 allowance (flags, fp32_err_A / fp32_err_D are zero):
    the method alone, as the CPU baseline times it."""
    lib = _load()
    m, q, ls, lg = params64 if params64 is not None else _params64(surfels)
    H, W = frame.H, frame.W
    A = np.zeros(H * W); St = np.zeros(H * W); Sn = np.zeros(3 * H * W); Tf = np.zeros(H * W)
    nc = np.zeros(H * W, np.int32); ne = np.zeros(H * W, np.int64); fl = np.zeros(H * W, np.uint8)
    nv = np.zeros(H * W, np.int32); eA = np.zeros(H * W); eD = np.zeros(H * W)
    fa = _frame_args(frame)
    lib.lgso_render_fwd(_p(m), _p(q), _p(ls), _p(lg), m.shape[0], *fa[:6], _p(fa[6]),
                        _p(_c(ranges, np.int64)), _p(_c(vals, np.uint32)),
                        _p(A), _p(St), _p(Sn), _p(Tf), _p(nc), _p(ne), _p(fl) if allowance else None, _p(nv),
                        _p(eA) if allowance else None, _p(eD) if allowance else None, int(nthreads))
    return dict(A=A.reshape(H, W), S_t=St.reshape(H, W), S_n=Sn.reshape(3, H, W),
                T_final=Tf.reshape(H, W), n_contrib=nc.reshape(H, W), n_eval=ne.reshape(H, W),
                flags=fl.reshape(H, W), n_valid=nv.reshape(H, W), fp32_err_A=eA.reshape(H, W),
                fp32_err_D=eD.reshape(H, W))


def coverage_misses(surfels, frame, ranges, vals, params64=None) -> int:
    """Valid (pixel, surfel) evaluations whose surfel is missing from the
    pixel's tile list (brute force; 0 means binning is conservative)."""
    m, q, ls, lg = params64 if params64 is not None else _params64(surfels)
    fa = _frame_args(frame)
    return int(_load().lgso_coverage_misses(_p(m), _p(q), _p(ls), _p(lg), m.shape[0], *fa[:6], _p(fa[6]),
                                            _p(_c(ranges, np.int64)), _p(_c(vals, np.uint32))))


def render_bwd(surfels, frame, ranges, vals, gA, gSt, gSn, params64=None, grads=None,
               nthreads: int = 0, allowance: bool = True):
    """FP64 backward of one frame; accumulates into ``grads`` (dict of arrays).
    allowance=False skips the binary32 allowance (abs / flip untouched)."""
    lib = _load()
    m, q, ls, lg = params64 if params64 is not None else _params64(surfels)
    n = m.shape[0]
    if grads is None:
        grads = dict(mean=np.zeros((n, 3)), quat=np.zeros((n, 4)), log_scale=np.zeros((n, 2)),
                     logit=np.zeros(n), abs=np.zeros((n, 10)), flip=np.zeros((n, 10)))
    fa = _frame_args(frame)
    lib.lgso_render_bwd(_p(m), _p(q), _p(ls), _p(lg), n, *fa[:6], _p(fa[6]),
                        _p(_c(ranges, np.int64)), _p(_c(vals, np.uint32)),
                        _p(_c(gA, np.float64)), _p(_c(gSt, np.float64)), _p(_c(gSn, np.float64)),
                        _p(grads["mean"]), _p(grads["quat"]), _p(grads["log_scale"]), _p(grads["logit"]),
                        _p(grads["abs"]) if allowance else None, _p(grads["flip"]) if allowance else None,
                        int(nthreads))
    return grads


# --- the binary32 allowance, one pixel at a time (its pins) -------------------
def pixel_detail(surfels, frame, ranges, vals, r: int, c: int, gA=1.0, gSt=0.0, gSn=(0.0, 0.0, 0.0),
                 params64=None, lib=None):
    """Every list entry the method evaluated at pixel (r, c), with the
    allowance's per-entry and per-contributor values (see lgso_pixel_detail).
    ``lib``: a variant build of the oracle (a planted mistake)."""
    lib = lib or _load()
    m, q, ls, lg = params64 if params64 is not None else _params64(surfels)
    fa = _frame_args(frame)
    t = (r // frame.tile_h) * (-(-frame.W // frame.tile_w)) + c // frame.tile_w
    ranges = _c(ranges, np.int64)
    cap = max(int(ranges[t, 1] - ranges[t, 0]), 1)
    item = np.zeros(cap, np.uint32); valid = np.zeros(cap, np.int32); flags = np.zeros(cap, np.int32)
    contrib = np.zeros(cap, np.int32); ev = np.zeros((cap, 8)); unc = np.zeros((cap, 4)); would = np.zeros(cap)
    grad = np.zeros((cap, 10)); gunc = np.zeros((cap, 10)); gmaj = np.zeros((cap, 10))
    T = np.zeros(cap); S = np.zeros(cap); eT = np.zeros(cap); dS = np.zeros(cap); pix = np.zeros(8)
    pfl = np.zeros(1, np.int32); nco = np.zeros(1, np.int32)
    gsn = _c(np.asarray(gSn, np.float64), np.float64)
    k = lib.lgso_pixel_detail(_p(m), _p(q), _p(ls), _p(lg), m.shape[0], *fa[:6], _p(fa[6]), _p(ranges),
                              _p(_c(vals, np.uint32)), int(r), int(c), float(gA), float(gSt), _p(gsn), cap,
                              _p(item), _p(valid), _p(flags), _p(contrib), _p(ev), _p(unc), _p(would), _p(grad),
                              _p(gunc), _p(gmaj), _p(T), _p(S), _p(eT), _p(dS), _p(pix), _p(pfl), _p(nco))
    if k < 0:
        raise ValueError("more evaluated entries than the tile list holds")
    nc = int(nco[0])
    return dict(item=item[:k], valid=valid[:k].astype(bool), flags=flags[:k], contrib=contrib[:k], den=ev[:k, 0],
                t=ev[:k, 1], u=ev[:k, 2], v=ev[:k, 3], q=ev[:k, 4], G=ev[:k, 5], a=ev[:k, 6], araw=ev[:k, 7],
                eu=unc[:k, 0], ev=unc[:k, 1], dt=unc[:k, 2], da=unc[:k, 3], would=would[:k], grad=grad[:nc], gunc=gunc[:nc],
                gmaj=gmaj[:nc], T=T[:nc], S=S[:nc], eT=eT[:nc], dS=dS[:nc], A=pix[0], S_t=pix[1],
                S_n=pix[2:5].copy(), T_final=pix[5], eA=pix[6], eD=pix[7], pflags=int(pfl[0]), nc=nc)


def contrib_with(surfels, frame, i: int, r: int, c: int, den, t, u, v, G, a, araw, T, S, gA=1.0, gSt=0.0,
                 gSn=(0.0, 0.0, 0.0), params64=None, lib=None):
    """The method's raw-parameter contribution of surfel i at pixel (r, c)
    from the given evaluation quantities, transmittance and suffix (see
    lgso_contrib_with)."""
    lib = lib or _load()
    m, q, ls, lg = params64 if params64 is not None else _params64(surfels)
    fa = _frame_args(frame)
    q7 = np.array([den, t, u, v, G, a, araw], np.float64)
    out = np.zeros(10)
    lib.lgso_contrib_with(_p(m), _p(q), _p(ls), _p(lg), int(i), frame.H, frame.W, fa[4], fa[5], _p(fa[6]), int(r),
                          int(c), _p(q7), float(T), float(S), float(gA), float(gSt),
                          _p(_c(np.asarray(gSn, np.float64), np.float64)), _p(out))
    return out


def variant(defines, path):
    """A separately built oracle with the given -D defines (a planted
    mistake), loaded with the argument types of the oracle's own library."""
    build(force=True, out=path, defines=defines)
    lib = ctypes.CDLL(path)
    base = _load()
    for name in ("lgso_pixel_detail", "lgso_contrib_with", "lgso_render_fwd", "lgso_render_bwd"):
        getattr(lib, name).argtypes = getattr(base, name).argtypes
        getattr(lib, name).restype = getattr(base, name).restype
    return lib


def loss_image(fwd, D, Ng, lam_alpha=LAMBDA_ALPHA, lam_n=LAMBDA_N, lam_ng=LAMBDA_NG, scale=1.0, lam_ns=0.0,
               frame=None, ns_err=None):
    """Image terms of the mapping loss and their gradients w.r.t. (A, S_t, S_n).
    terms = (L_depth, L_alpha, L_ng, L_ns); the N_surf term (needs ``frame``
    for the pixel rays) is included when lam_ns != 0.  ``ns_err`` (a dict)
    receives the binary32 bounds of the N_surf term: dD (on dL/dDh per
    pixel), dS_n (per pixel) and L_ns (on terms[3])."""
    lib = _load()
    H, W = D.shape
    npix = H * W
    gA = np.zeros(npix); gSt = np.zeros(npix); gSn = np.zeros(3 * npix); terms = np.zeros(4)
    A = _c(fwd["A"], np.float64); St = _c(fwd["S_t"], np.float64); Sn = _c(fwd["S_n"], np.float64)
    Dm = _c(D, np.float32)
    L = lib.lgso_loss_image(_p(A), _p(St), _p(Sn), _p(Dm), _p(_c(Ng, np.float32)),
                            npix, lam_alpha, lam_n, lam_ng, scale, _p(gA), _p(gSt), _p(gSn), _p(terms))
    if lam_ns != 0.0:
        if frame is None:
            raise ValueError("the N_surf term needs the frame (pixel rays)")
        err = np.zeros(2 * npix + 1) if ns_err is not None else None
        lns = lib.lgso_surf_normal_loss(_p(A), _p(St), _p(Sn), _p(Dm), H, W, float(np.float32(frame.elev_min)),
                                        float(np.float32(frame.elev_max)), lam_n * lam_ns, scale, _p(gA), _p(gSt),
                                        _p(gSn), _p(err))
        if err is not None:
            ns_err.update(dD=err[:npix].reshape(H, W), dS_n=err[npix:2 * npix].reshape(H, W),
                          L_ns=err[2 * npix])
        terms[3] = lns
        L += scale * lam_n * lam_ns * lns
    return L, dict(dA=gA.reshape(H, W), dS_t=gSt.reshape(H, W), dS_n=gSn.reshape(3, H, W)), terms


def scale_reg(log_scale, s_max=S_MAX, lam_s=LAMBDA_S, dls=None):
    lib = _load()
    ls = _c(log_scale, np.float64)
    return lib.lgso_scale_reg(_p(ls), ls.shape[0], s_max, lam_s, _p(dls) if dls is not None else None)


def forward_backward(surfels, frames, targets, lam_alpha=LAMBDA_ALPHA, lam_n=LAMBDA_N,
                     lam_ng=LAMBDA_NG, lam_s=LAMBDA_S, s_max=S_MAX, params64=None, nthreads: int = 0,
                     brute: bool = False, lam_ns: float = 0.0, allowance: bool = True):
    """The whole step for a window of frames: per frame bin, render, image
    loss (averaged over frames), backward; plus lam_s L_scale once.
    ``targets`` is a list of (D, Ng).  Returns (L, per-frame forwards, grads, bins).
    allowance=False: the method alone (no binary32 allowance)."""
    n = surfels.mean.shape[0]
    grads = dict(mean=np.zeros((n, 3)), quat=np.zeros((n, 4)), log_scale=np.zeros((n, 2)),
                 logit=np.zeros(n), abs=np.zeros((n, 10)), flip=np.zeros((n, 10)))
    F = len(frames)
    L = 0.0
    fwds, bins = [], []
    for f, (frame, (D, Ng)) in enumerate(zip(frames, targets)):
        if brute:
            ranges, vals = brute_lists(surfels, frame)
            b = dict(ranges=ranges, vals=vals)
        else:
            b = bin_frame(surfels, frame)
        fw = render_fwd(surfels, frame, b["ranges"], b["vals"], params64, nthreads, allowance)
        Lf, g, _ = loss_image(fw, D, Ng, lam_alpha, lam_n, lam_ng, scale=1.0 / F, lam_ns=lam_ns, frame=frame)
        render_bwd(surfels, frame, b["ranges"], b["vals"], g["dA"], g["dS_t"], g["dS_n"], params64,
                   grads, nthreads, allowance)
        L += Lf
        fwds.append(fw); bins.append(b)
    ls = params64[2] if params64 is not None else surfels.log_scale
    L += scale_reg(ls, s_max, lam_s, grads["log_scale"])
    return L, fwds, grads, bins


def adam(p, g, m, v, step: int, lr, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15):
    """One Adam step in FP64 (Kingma and Ba, ICLR 2015, Algorithm 1).  The
    paper optimises the map (Sec. 3.4) without naming its optimiser; the
    mapping loop here uses Adam with per-parameter-group learning rates.
      m <- beta1 m + (1 - beta1) g,   v <- beta2 v + (1 - beta2) g^2,
      p <- p - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps)
    with t = ``step`` >= 1.  Returns the new (p, m, v) as float64 arrays."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


# --- tracking-side targets (Sec. 3.2) ------------------------------------------
def logit_threshold(alpha_min: float) -> np.float32:
    """The opacity threshold as a binary32 logit: alpha >= alpha_min is
    decided as logit >= this value in binary32 on both sides (the sigmoid is
    monotone), so the selection is exact and shared."""
    return np.float32(math.log(alpha_min / (1.0 - alpha_min)))


def trackable_targets(surfels, mask, last_kf, k_min: int, alpha_min: float, thickness: float = 0.01,
                      eps: float = 1e-6, w_max: float = 10.0):
    """Targets the tracker registers against (Sec. 3.2, Eqs. trackable_select,
    anisotropy, anisotropy_norm, weight_func), in FP64 from the FP32 inputs.

    Selection: m_i = 1, k_i >= k_min and alpha_i >= alpha_min (the last in
    binary32 on the logit).  For each selected surfel, in ascending index:
    its mean; the surfel-like covariance R(q) diag(s_x^2, s_y^2, thickness^2)
    R(q)^T (q normalised, columns of R the tangent axes and the normal); the
    anisotropy kappa = s_0 / (s_1 + eps) with s_0 >= s_1 the sorted in-plane
    scales, normalised over the selected set by its minimum and maximum
    (kappa_bar = 0 when they coincide), and the weight
    w = min(1 / (kappa_bar + eps), w_max).
    Returns (index int64 [k], mean [k,3], cov [k,6] as xx, xy, xz, yy, yz, zz,
    weight [k])."""
    lg = np.asarray(surfels.logit, np.float32)
    sel = (np.asarray(mask) != 0) & (np.asarray(last_kf) >= k_min) & (lg >= logit_threshold(alpha_min))
    idx = np.nonzero(sel)[0].astype(np.int64)
    mean = np.asarray(surfels.mean, np.float64)[idx]
    q = np.asarray(surfels.quat, np.float64)[idx]
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w_, x, y, z = q.T
    R = np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w_ * z), 2 * (x * z + w_ * y)], -1),
                  np.stack([2 * (x * y + w_ * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w_ * x)], -1),
                  np.stack([2 * (x * z - w_ * y), 2 * (y * z + w_ * x), 1 - 2 * (x * x + y * y)], -1)], 1)
    s = np.exp(np.asarray(surfels.log_scale, np.float64)[idx])
    lam = np.stack([s[:, 0] ** 2, s[:, 1] ** 2, np.full(len(idx), thickness ** 2)], 1)
    C = np.einsum("nij,nj,nkj->nik", R, lam, R)
    cov = np.stack([C[:, 0, 0], C[:, 0, 1], C[:, 0, 2], C[:, 1, 1], C[:, 1, 2], C[:, 2, 2]], 1)
    s0, s1 = s.max(1), s.min(1)
    kappa = s0 / (s1 + eps)
    if len(idx):
        kmin, kmax = kappa.min(), kappa.max()
        kb = (kappa - kmin) / (kmax - kmin) if kmax > kmin else np.zeros_like(kappa)
    else:
        kb = kappa
    weight = np.minimum(1.0 / (kb + eps), w_max)
    return idx, mean, cov, weight
