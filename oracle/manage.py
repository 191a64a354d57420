"""Map management on the surfel map: the control score (Sec. 3.3, Eq.
controlscore), opacity-based pruning (the baseline of Table 4), the multi-pass
planar cover-and-prune and the structure-aware adaptive split (Sec. 3.5).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the product path
never does.  It shares no code with the CUDA library.

Every outcome here is an integer decision (which surfels survive, which are
split) or a parameter copied or shifted from the inputs, so it is specified in
IEEE binary32: each operation below is one correctly rounded NumPy float32
operation (NumPy never contracts a*b+c into a fused multiply-add), in the
order written, so that a GPU implementation of the same definition agrees bit
for bit.  The surfels' scales s = exp(s~) use the oracle's fixed polynomial
exponential (``oracle.f32_exp_spec_n``).  Quantiles are the lower order
statistic: Q_q(x) = sorted(x)[floor(q (n - 1))].

Readings of what the paper leaves open (numbers it does not give, the
normalisation of the score terms, the cover region, the cap order, the
children) are the defaults of ``Params`` and are each stated where they are
used.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import oracle

F = np.float32


@dataclasses.dataclass
class Params:
    alpha_prune: float = 0.005   # opacity prune: alpha < alpha_prune is removed
    alpha_min: float = 0.1       # alpha_min of Sec. 3.5: cover-and-prune / split eligibility
    w_l: float = 0.55            # control-score weights (Sec. 3.3)
    w_c: float = 0.30
    w_r: float = 0.15
    q_res: float = 0.95          # the residual is normalised by this quantile of itself
    eps: float = 1e-6            # the epsilon of linear_i and curv_i
    q_plane: float = 0.3         # planar candidates: c_i <= Q_{q_plane}(c)
    voxel: float = 1.0           # edge of the projected 2D voxel (m)
    n_passes: int = 3            # planes xy, yz, zx in this order (0..3 of them)
    q_cover: float = 0.5         # fraction of a group's members the cover region includes
    slab: float = 0.05           # half-thickness about the representative's plane (m)
    prune_cap: float = 0.1       # at most this fraction of the surviving map per pass
    q_split: float = 0.9         # split candidates: c_i >= Q_{q_split}(c)
    split_cap: float = 0.05      # at most this fraction of the surviving map is split
    split_shift: float = 0.5     # children at mu +- split_shift * s_0 * a_i
    split_dlog: float = float(np.float32(math.log(0.5)))   # children's s~_0 increment


PLANES = ((0, 1), (1, 2), (2, 0))


def order_key(x) -> np.ndarray:
    """Total-order key of binary32 values (uint32, ascending with the value;
    -0 sorts just below +0)."""
    b = np.ascontiguousarray(x, F).view(np.uint32)
    return np.where(b >> 31 != 0, ~b, b | np.uint32(0x80000000)).astype(np.uint32)


def logit_threshold(alpha: float) -> np.float32:
    """alpha >= a is decided as logit >= this binary32 value (the sigmoid is
    monotone), on both sides of the parity check."""
    return F(math.log(alpha / (1.0 - alpha)))


def quantile_lower(x, q: float):
    """Q_q(x): the lower order statistic sorted(x)[floor(q (n - 1))], q taken
    as binary32 and the index formed in binary64."""
    x = np.asarray(x, F)
    if x.size == 0:
        return None
    k = int(math.floor(float(F(q)) * (x.size - 1)))
    return x[np.argsort(order_key(x), kind="stable")][k]


def quat_axes(quat):
    """Columns of R(q) for the normalised quaternion (w, x, y, z) in binary32:
    t_u = R e_0 (the in-plane major axis a_i of Sec. 3.5), t_v = R e_1 and the
    normal n = R e_2, as [n, 3] arrays."""
    q = np.asarray(quat, F)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    r = np.sqrt(((w * w + x * x) + y * y) + z * z)
    w, x, y, z = w / r, x / r, y / r, z / r
    one, two = F(1), F(2)
    tu = np.stack([one - two * (y * y + z * z), two * (x * y + w * z), two * (x * z - w * y)], 1)
    tv = np.stack([two * (x * y - w * z), one - two * (x * x + z * z), two * (y * z + w * x)], 1)
    nn = np.stack([two * (x * z + w * y), two * (y * z - w * x), one - two * (x * x + y * y)], 1)
    return tu, tv, nn


def _dot(a, b):
    return (a[..., 0] * b[..., 0] + a[..., 1] * b[..., 1]) + a[..., 2] * b[..., 2]


def control_score(lam, res, p: Params = Params()):
    """Control score c_i (Sec. 3.3, Eq. controlscore) in binary32.

    lambda_{i,0} >= lambda_{i,1} >= lambda_{i,2} are the tracking covariance's
    eigenvalues (sorted here; any input order), linear_i = (l0 - l1)/(l0 + eps),
    curv_i = l2 / (l0 + l1 + l2 + eps).  The paper combines normalised terms
    and does not spell the normalisation out; reading: linear_i already spans
    [0, 1] and is taken as is, curv_i spans [0, 1/3] and is scaled by 3, and
    the residual is normalised robustly by its own q_res quantile over the map,
    min(res_i / (Q_{q_res}(res) + eps), 1).  c_i = clip(w_l lin + w_c curv~ +
    w_r res~, 0, 1)."""
    lam = np.sort(np.asarray(lam, F), axis=1)[:, ::-1]
    res = np.asarray(res, F)
    eps = F(p.eps)
    l0, l1, l2 = lam[:, 0], lam[:, 1], lam[:, 2]
    lin = (l0 - l1) / (l0 + eps)
    cur = l2 / (((l0 + l1) + l2) + eps)
    cv = F(3) * cur
    cv = np.where(cv < F(1), cv, F(1))
    rq = quantile_lower(res, p.q_res)
    if rq is None:
        return np.zeros(0, F)
    rn = res / (F(rq) + eps)
    rn = np.where(rn < F(1), rn, F(1))
    c = (F(p.w_l) * lin + F(p.w_c) * cv) + F(p.w_r) * rn
    c = np.where(c < F(1), c, F(1))
    return np.where(c > F(0), c, F(0)).astype(F)


def _voxel(m, v):
    g = np.floor(np.asarray(m, F) / F(v))
    return np.clip(g, -(2.0 ** 30), 2.0 ** 30).astype(np.int64)


def cover_prune_pass(mean, quat, log_scale, logit, c, alive, plane, p: Params = Params()):
    """One pass of the multi-pass planar cover-and-prune (Sec. 3.5) over the
    surviving map ``alive``; returns the surfels it removes (bool [n]).

    Candidates: alive, c_i <= Q_{q_plane}(c over the survivors) and
    alpha_i >= alpha_min.  Each candidate's mean is projected onto the pass's
    plane and grouped by the 2D voxel (floor(mu_a / voxel), floor(mu_b /
    voxel)).  The group's representative is its candidate of largest alpha
    (ties: lowest index).  The other candidates are expressed in the
    representative's tangent frame, d = mu_j - mu_r, u = t_u.d / s_u,
    v = t_v.d / s_v, h = n.d; those within the slab |h| <= slab are the
    group's members.  Reading of the cover region: the representative's
    ellipse u^2 + v^2 <= beta^2 with beta^2 the ceil(q_cover m)-th smallest
    u^2 + v^2 of the m members, so the region includes a q_cover fraction of
    them; the members inside it are redundant.  The cap: at most
    floor(prune_cap * survivors) removals per pass, the most planar first
    (ascending c_i, then index)."""
    n = alive.size
    removed = np.zeros(n, bool)
    n_a = int(alive.sum())
    if n_a == 0:
        return removed
    qp = quantile_lower(c[alive], p.q_plane)
    cand = alive & (c <= qp) & (np.asarray(logit, F) >= logit_threshold(p.alpha_min))
    idx = np.nonzero(cand)[0]
    a, b = plane
    ga = _voxel(np.asarray(mean, F)[idx, a], p.voxel)
    gb = _voxel(np.asarray(mean, F)[idx, b], p.voxel)
    lkey = order_key(np.asarray(logit, F)[idx])
    tu, tv, nn = quat_axes(np.asarray(quat, F)[idx])
    s = oracle.f32_exp_spec_n(np.asarray(log_scale, F)[idx])
    mu = np.asarray(mean, F)[idx]
    groups = {}
    for j, key in enumerate(zip(ga.tolist(), gb.tolist())):
        groups.setdefault(key, []).append(j)
    flagged = []
    k_frac = float(F(p.q_cover))
    for mem in groups.values():
        mem = np.asarray(mem)
        r = mem[np.argmax(lkey[mem])]            # first maximum: lowest index
        others = mem[mem != r]
        if others.size == 0:
            continue
        d = mu[others] - mu[r]
        u = _dot(tu[r], d) / s[r, 0]
        v = _dot(tv[r], d) / s[r, 1]
        h = _dot(nn[r], d)
        inside = np.abs(h) <= F(p.slab)
        memb = others[inside]
        m = memb.size
        if m == 0:
            continue
        rk = (u * u + v * v)[inside].view(np.uint32)   # non-negative: bits order like values
        k = math.ceil(k_frac * m)
        if k == 0:
            continue
        beta2 = np.sort(rk)[k - 1]                     # the k-th smallest u^2 + v^2
        flagged.extend(idx[memb[rk <= beta2]].tolist())
    flagged = np.asarray(sorted(flagged), np.int64)
    cap = math.floor(float(F(p.prune_cap)) * n_a)
    if flagged.size > cap:
        ck = order_key(c[flagged]).astype(np.uint64)
        keys = (ck << np.uint64(32)) | flagged.astype(np.uint64)
        flagged = flagged[np.argsort(keys, kind="stable")[:cap]]
    removed[flagged] = True
    return removed


def split_select(c, logit, alive, p: Params = Params()):
    """Split candidates of the structure-aware adaptive split (Sec. 3.5):
    alive, c_i >= Q_{q_split}(c over the survivors) and alpha_i >= alpha_min,
    capped at floor(split_cap * survivors), the most complex first (descending
    c_i, then ascending index).  Returns bool [n]."""
    n = alive.size
    split = np.zeros(n, bool)
    n_a = int(alive.sum())
    if n_a == 0:
        return split
    qs = quantile_lower(c[alive], p.q_split)
    cand = alive & (c >= qs) & (np.asarray(logit, F) >= logit_threshold(p.alpha_min))
    idx = np.nonzero(cand)[0]
    cap = math.floor(float(F(p.split_cap)) * n_a)
    if idx.size > cap:
        ck = (~order_key(c[idx])).astype(np.uint64)
        keys = (ck << np.uint64(32)) | idx.astype(np.uint64)
        idx = idx[np.argsort(keys, kind="stable")[:cap]]
    split[idx] = True
    return split


def children(mean, quat, log_scale, p: Params = Params()):
    """The two children of each given surfel (Sec. 3.5): means shifted in
    opposite directions along the in-plane major axis a_i = R(q_i) e_0.
    Reading (the paper gives no magnitudes): mu +- split_shift * s_0 * a_i,
    with the children's s~_0 = s~_0 + split_dlog; orientation, s~_1 and
    opacity are the parent's.  Returns (mean_plus, mean_minus, log_scale)."""
    mean = np.asarray(mean, F)
    ls = np.asarray(log_scale, F)
    tu, _, _ = quat_axes(quat)
    s0 = oracle.f32_exp_spec_n(ls[:, 0])
    off = (F(p.split_shift) * s0)[:, None] * tu
    cls = ls.copy()
    cls[:, 0] = ls[:, 0] + F(p.split_dlog)
    return mean + off, mean - off, cls


def manage(mean, quat, log_scale, logit, lam, res, p: Params = Params()):
    """One map-management step: control score, opacity prune, the cover-and-
    prune passes over the planes xy, yz, zx (the first n_passes of them), then
    the split.  The new map lists the survivors in ascending index, a split
    surfel giving way to its two children (role 1: +shift, role 2: -shift) at
    its place; role 0 is a copy.

    Returns a dict: score c [n], src [n_out] int32 (the parent index of each
    new surfel), role [n_out] uint8, mean/quat/log_scale/logit of the new map,
    counts int64 [6] = (n_out, opacity-pruned, pruned by passes 0, 1, 2,
    split)."""
    mean = np.asarray(mean, F).reshape(-1, 3)
    quat = np.asarray(quat, F).reshape(-1, 4)
    log_scale = np.asarray(log_scale, F).reshape(-1, 2)
    logit = np.asarray(logit, F).reshape(-1)
    n = logit.size
    c = control_score(lam, res, p) if n else np.zeros(0, F)
    alive = logit >= logit_threshold(p.alpha_prune)
    counts = np.zeros(6, np.int64)
    counts[1] = n - int(alive.sum())
    for k in range(p.n_passes):
        rm = cover_prune_pass(mean, quat, log_scale, logit, c, alive, PLANES[k], p)
        counts[2 + k] = int(rm.sum())
        alive &= ~rm
    split = split_select(c, logit, alive, p)
    counts[5] = int(split.sum())
    src, role = [], []
    for i in np.nonzero(alive)[0].tolist():
        if split[i]:
            src += [i, i]; role += [1, 2]
        else:
            src.append(i); role.append(0)
    src = np.asarray(src, np.int32)
    role = np.asarray(role, np.uint8)
    counts[0] = src.size
    om, oq, ol, og = mean[src].copy(), quat[src].copy(), log_scale[src].copy(), logit[src].copy()
    ch = np.nonzero(role != 0)[0]
    if ch.size:
        mp, mm, cls = children(mean[src[ch]], quat[src[ch]], log_scale[src[ch]], p)
        om[ch] = np.where((role[ch] == 1)[:, None], mp, mm)
        ol[ch] = cls
    return dict(score=c, src=src, role=role, mean=om, quat=oq, log_scale=ol, logit=og, counts=counts)
