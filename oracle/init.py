"""Keyframe initialisation of new surfels from a LiDAR scan: the k-NN
covariance and its eigendecomposition (Sec. 3.2, "Covariance construction and
reuse"), the range-adaptive scale (Sec. 3.3, Eq. of the range-adaptive scale
initialisation), the physics-based confidence u (Eq. physconf) and the
opacity initialisation (Eq. alpha_init) -- CPU oracle.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the product path
never does.  It shares no code with the CUDA library.

Precisions: the neighbour sets are integer outcomes, so the squared
distances that decide them are specified in binary32, ((dx dx + dy dy) +
dz dz) with dx = q_x - p_x, each operation correctly rounded (NumPy float32),
ties to the lower index; everything after (covariance, eigendecomposition,
scales, confidence, opacity, orientation) is FP64 from the binary32 points.

Readings of what the paper leaves open are the defaults of ``Params``:
the neighbourhood includes the point itself (a k-NN query of the point's own
scan), the covariance is the biased mean of outer products about the
neighbourhood mean, sigma = sqrt(lambda) normalised by the largest (the
covariance normalisation of G-ICP: sigma_tan carries anisotropy, the range
carries spacing), the scale clip's lower end is s_min > 0 (so the log-scale
exists), the normal is the smallest eigenvector turned toward the sensor, the
in-plane axes are the other two eigenvectors (t_u the largest; its sign is not
fixed by the definition), and r in u is the point's range.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

F = np.float32


@dataclasses.dataclass
class Params:
    k: int = 20                 # neighbours (the point included)
    kappa: float = 0.0184       # 1.5 x the 128-beam, +-45 deg elevation pitch (rad)
    s_min: float = 1e-3         # lower clip of the initial scale (m)
    s_max: float = 1.0          # s_max of the scale clip (m)
    r0: float = 100.0           # range scale of the confidence (m)
    c0: float = 0.1             # incidence-cosine threshold of the confidence
    eps: float = 1e-6           # epsilon of Eq. physconf
    alpha_min: float = 0.3      # opacity at u = 0
    alpha_max: float = 0.9      # opacity at u = 1


def knn(points, k: int, rows=None, chunk: int = 512):
    """The k nearest neighbours of every point (or of the points ``rows``)
    among all the points (itself included), by binary32 squared distance,
    ties to the lower index, in ascending (distance, index) order.  Returns
    (index int32 [m, k], squared distance float32 [m, k])."""
    p = np.asarray(points, F)
    n = p.shape[0]
    if k > n:
        raise ValueError("k exceeds the number of points")
    rows = np.arange(n) if rows is None else np.asarray(rows)
    m = rows.size
    chunk = max(1, min(chunk, 20_000_000 // max(n, 1)))     # bounded temporaries
    idx = np.empty((m, k), np.int32)
    d2 = np.empty((m, k), F)
    cols = np.arange(n, dtype=np.int64)
    for a in range(0, m, chunk):
        q = p[rows[a:a + chunk]]
        dx = p[None, :, 0] - q[:, None, 0]
        dy = p[None, :, 1] - q[:, None, 1]
        dz = p[None, :, 2] - q[:, None, 2]
        dd = (dx * dx + dy * dy) + dz * dz
        # order by (distance bits, index): non-negative binary32 values order
        # like their bit patterns
        key = (dd.view(np.uint32).astype(np.uint64) << np.uint64(32)) | cols[None, :].astype(np.uint64)
        part = np.argpartition(key, k - 1, axis=1)[:, :k]
        pk = np.take_along_axis(key, part, 1)
        o = np.argsort(pk, axis=1)
        sel = np.take_along_axis(part, o, 1)
        idx[a:a + chunk] = sel
        d2[a:a + chunk] = np.take_along_axis(dd, sel, 1)
    return idx, d2


def covariance(points, idx):
    """Per point, the biased covariance of its neighbourhood about the
    neighbourhood mean, FP64 [n, 3, 3]."""
    p = np.asarray(points, np.float64)
    nb = p[idx]                                   # [n, k, 3]
    c = nb - nb.mean(1, keepdims=True)
    return np.einsum("nki,nkj->nij", c, c) / idx.shape[1]


def initialise(points, pose, p: Params = Params(), rows=None):
    """New surfels at the scan's points (sensor frame, binary32 [n, 3]) for a
    keyframe at ``pose`` (sensor -> world, R row-major | t, 12 values); with
    ``rows``, only for those points (their neighbours still among all).

    Returns a dict: knn [n, k] int32; lam [n, 3] eigenvalues descending (>= 0);
    normal_s, tu_s [n, 3] the sensor-frame normal (toward the sensor) and
    major in-plane axis; mean [n, 3] world; rot [n, 3, 3] world frame
    [t_u, t_v, n] as columns; quat [n, 4] (w, x, y, z), w >= 0; log_scale
    [n, 2]; u [n]; alpha [n]; logit [n]; all FP64 but knn."""
    pts = np.asarray(points, F)
    rows = np.arange(pts.shape[0]) if rows is None else np.asarray(rows)
    idx, _ = knn(pts, p.k, rows)
    C = covariance(pts, idx)
    w, v = np.linalg.eigh(C)                      # ascending
    lam = np.maximum(w[:, ::-1], 0.0)
    e0, e2 = v[:, :, 2], v[:, :, 0]
    ps = pts[rows].astype(np.float64)
    rng = np.linalg.norm(ps, axis=1)
    # normal toward the sensor (at the origin of the sensor frame)
    nrm = np.where(((e2 * ps).sum(1) > 0)[:, None], -e2, e2)
    tu = e0 - (e0 * nrm).sum(1, keepdims=True) * nrm
    tu /= np.linalg.norm(tu, axis=1, keepdims=True)
    tv = np.cross(nrm, tu)
    # range-adaptive scale: s = clip(kappa r sigma_tan, s_min, s_max),
    # r = max(|p|, 1), sigma_tan the two largest sigmas over the largest
    sig = np.sqrt(lam)
    s0 = sig[:, 0]
    sig_tan = np.where(s0[:, None] > 0, sig[:, :2] / np.where(s0 > 0, s0, 1.0)[:, None], 1.0)
    r = np.maximum(rng, 1.0)
    s = np.clip(p.kappa * r[:, None] * sig_tan, p.s_min, p.s_max)
    # physics-based confidence (Eq. physconf) and opacity (Eq. alpha_init)
    cosv = np.abs((nrm * ps).sum(1)) / rng
    u = np.exp(-(rng / p.r0) ** 2) * np.clip((cosv - p.c0) / (1.0 - p.c0 + p.eps), 0.0, 1.0)
    alpha = p.alpha_min + (p.alpha_max - p.alpha_min) * u
    P = np.asarray(pose, np.float64).reshape(3, 4)
    Rs = np.stack([tu, tv, nrm], axis=2)           # columns, sensor frame
    Rw = np.einsum("ij,njk->nik", P[:, :3], Rs)
    mean = ps @ P[:, :3].T + P[:, 3]
    return dict(knn=idx, lam=lam, normal_s=nrm, tu_s=tu, mean=mean, rot=Rw, quat=rot_to_quat(Rw),
                log_scale=np.log(s), u=u, alpha=alpha, logit=np.log(alpha / (1.0 - alpha)))


def rot_to_quat(R):
    """Rotation matrices [n, 3, 3] -> unit quaternions (w, x, y, z) with
    w >= 0, from the largest of 1 + tr, 1 + 2 R_ii - tr (Shepperd's rule)."""
    R = np.asarray(R, np.float64)
    n = R.shape[0]
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    cand = np.stack([1 + tr, 1 + 2 * R[:, 0, 0] - tr, 1 + 2 * R[:, 1, 1] - tr, 1 + 2 * R[:, 2, 2] - tr], 1)
    which = np.argmax(cand, 1)
    q = np.zeros((n, 4))
    for c in range(4):
        m = which == c
        if not m.any():
            continue
        Rm = R[m]
        t = np.sqrt(cand[m, c]) * 2                  # 4 |q_c|
        if c == 0:
            q[m] = np.stack([t / 4, (Rm[:, 2, 1] - Rm[:, 1, 2]) / t, (Rm[:, 0, 2] - Rm[:, 2, 0]) / t,
                             (Rm[:, 1, 0] - Rm[:, 0, 1]) / t], 1)
        elif c == 1:
            q[m] = np.stack([(Rm[:, 2, 1] - Rm[:, 1, 2]) / t, t / 4, (Rm[:, 0, 1] + Rm[:, 1, 0]) / t,
                             (Rm[:, 0, 2] + Rm[:, 2, 0]) / t], 1)
        elif c == 2:
            q[m] = np.stack([(Rm[:, 0, 2] - Rm[:, 2, 0]) / t, (Rm[:, 0, 1] + Rm[:, 1, 0]) / t, t / 4,
                             (Rm[:, 1, 2] + Rm[:, 2, 1]) / t], 1)
        else:
            q[m] = np.stack([(Rm[:, 1, 0] - Rm[:, 0, 1]) / t, (Rm[:, 0, 2] + Rm[:, 2, 0]) / t,
                             (Rm[:, 1, 2] + Rm[:, 2, 1]) / t, t / 4], 1)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return np.where(q[:, :1] < 0, -q, q)
