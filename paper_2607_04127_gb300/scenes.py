"""Seeded synthetic inputs: surfel maps, frames (sensor poses and range-image
grids) and LiDAR targets shaped like the paper's spinning-LiDAR scans.

This module is the one piece shared by the CUDA path, the oracle, the tests
and the benchmark.  It holds none of the rasterizer's arithmetic: it builds
scenes out of analytic primitives (planes, vertical cylinders, axis-aligned
boxes), simulates a LiDAR by casting rays against them, and initialises
surfels from the simulated points.

Workloads (all seeded):
  * ``box_room``   -- 2,000 surfels on the walls, floor and ceiling of a
    20 x 20 x 5 m room, sensor at the centre, 32 x 512 image over +-15 deg,
    16 x 16 tiles.
  * ``street``     -- ground plane, facades at y = +-8 m (12 m tall), 40
    cylinders, 2,000 boxes; two 128 x 1024 scans over +-45 deg (2 cm range
    noise, 10 % drops) merged and sub-sampled to the requested surfel count,
    with normals and tangent axes from k = 20 nearest-neighbour covariances
    and the range-adaptive scale of the paper's initialisation (Sec. 3.3).
  * ``street_track`` -- the same street extended to a 200 m track, scans every
    3 m; used for the 1M-surfel mapping window and the batched / served maps.
The paper's datasets (KITTI, Newer College, Oxford Spires) are not
available; these scenes stand in for them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------
# Plain data containers
# ----------------------------------------------------------------------------
@dataclass
class Frame:
    """One range image: H x W pixels split into tile_h x tile_w tiles,
    elevation range [elev_min, elev_max] (radians, azimuth always full 360
    degrees) and the sensor-to-world pose [R | t] (3 x 4, row-major)."""
    H: int
    W: int
    tile_h: int
    tile_w: int
    elev_min: float
    elev_max: float
    pose: np.ndarray = field(default_factory=lambda: np.array(
        [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32))

    def with_tiles(self, tile_h: int, tile_w: int) -> "Frame":
        return Frame(self.H, self.W, tile_h, tile_w, self.elev_min, self.elev_max, self.pose.copy())


@dataclass
class Surfels:
    """Structure-of-arrays surfel parameters, FP32: mean [n,3], quaternion
    (w,x,y,z) [n,4] (need not be unit), log-scales [n,2], opacity logit [n]."""
    mean: np.ndarray
    quat: np.ndarray
    log_scale: np.ndarray
    logit: np.ndarray

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def subset(self, idx) -> "Surfels":
        return Surfels(self.mean[idx].copy(), self.quat[idx].copy(), self.log_scale[idx].copy(),
                       self.logit[idx].copy())

    def copy(self) -> "Surfels":
        return self.subset(slice(None))


@dataclass
class Target:
    """Measured range image D [H,W] (0 = no return) and tracking normals
    N_gicp [3,H,W] (zero where undefined)."""
    D: np.ndarray
    N: np.ndarray


def pose_matrix(yaw: float = 0.0, t=(0.0, 0.0, 0.0), pitch: float = 0.0, roll: float = 0.0) -> np.ndarray:
    cy, sy = math.cos(yaw), math.sin(yaw)
    cp, sp = math.cos(pitch), math.sin(pitch)
    cr, sr = math.cos(roll), math.sin(roll)
    Rz = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1]])
    Ry = np.array([[cp, 0, sp], [0, 1, 0], [-sp, 0, cp]])
    Rx = np.array([[1, 0, 0], [0, cr, -sr], [0, sr, cr]])
    R = Rz @ Ry @ Rx
    P = np.zeros((3, 4)); P[:, :3] = R; P[:, 3] = t
    return P.astype(np.float32).reshape(12)


def rot_to_quat(R: np.ndarray) -> np.ndarray:
    """Rotation matrices [n,3,3] -> unit quaternions (w,x,y,z) [n,4]."""
    n = R.shape[0]
    q = np.zeros((n, 4))
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    m0 = tr > 0
    s = np.sqrt(np.maximum(tr[m0] + 1.0, 1e-12)) * 2
    q[m0, 0] = 0.25 * s
    q[m0, 1] = (R[m0, 2, 1] - R[m0, 1, 2]) / s
    q[m0, 2] = (R[m0, 0, 2] - R[m0, 2, 0]) / s
    q[m0, 3] = (R[m0, 1, 0] - R[m0, 0, 1]) / s
    rest = ~m0
    i1 = rest & (R[:, 0, 0] > R[:, 1, 1]) & (R[:, 0, 0] > R[:, 2, 2])
    s = np.sqrt(np.maximum(1.0 + R[i1, 0, 0] - R[i1, 1, 1] - R[i1, 2, 2], 1e-12)) * 2
    q[i1, 0] = (R[i1, 2, 1] - R[i1, 1, 2]) / s
    q[i1, 1] = 0.25 * s
    q[i1, 2] = (R[i1, 0, 1] + R[i1, 1, 0]) / s
    q[i1, 3] = (R[i1, 0, 2] + R[i1, 2, 0]) / s
    i2 = rest & ~i1 & (R[:, 1, 1] > R[:, 2, 2])
    s = np.sqrt(np.maximum(1.0 + R[i2, 1, 1] - R[i2, 0, 0] - R[i2, 2, 2], 1e-12)) * 2
    q[i2, 0] = (R[i2, 0, 2] - R[i2, 2, 0]) / s
    q[i2, 1] = (R[i2, 0, 1] + R[i2, 1, 0]) / s
    q[i2, 2] = 0.25 * s
    q[i2, 3] = (R[i2, 1, 2] + R[i2, 2, 1]) / s
    i3 = rest & ~i1 & ~i2
    s = np.sqrt(np.maximum(1.0 + R[i3, 2, 2] - R[i3, 0, 0] - R[i3, 1, 1], 1e-12)) * 2
    q[i3, 0] = (R[i3, 1, 0] - R[i3, 0, 1]) / s
    q[i3, 1] = (R[i3, 0, 2] + R[i3, 2, 0]) / s
    q[i3, 2] = (R[i3, 1, 2] + R[i3, 2, 1]) / s
    q[i3, 3] = 0.25 * s
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def frames_from_axes(tu: np.ndarray, n: np.ndarray) -> np.ndarray:
    """Right-handed frames [t_u, t_v, n] as columns from a tangent and a normal."""
    n = n / np.linalg.norm(n, axis=1, keepdims=True)
    tu = tu - (tu * n).sum(1, keepdims=True) * n
    tu = tu / np.linalg.norm(tu, axis=1, keepdims=True)
    tv = np.cross(n, tu)
    return np.stack([tu, tv, n], axis=2)


def _logit(a):
    return np.log(a / (1.0 - a))


# ----------------------------------------------------------------------------
# Simulated spinning LiDAR
# ----------------------------------------------------------------------------
def sensor_rays(H: int, W: int, elev_min: float, elev_max: float) -> np.ndarray:
    """Unit beam directions [H,W,3] of the simulated sensor: rows from the top
    elevation down, columns counter-clockwise from +x, beam centres at half
    steps."""
    th = elev_max - (np.arange(H) + 0.5) * (elev_max - elev_min) / H
    ph = (np.arange(W) + 0.5) * 2 * np.pi / W
    ct, st = np.cos(th)[:, None], np.sin(th)[:, None]
    return np.stack([ct * np.cos(ph)[None], ct * np.sin(ph)[None], np.broadcast_to(st, (H, W))], -1)


@dataclass
class Scene:
    ground_z: float | None = None
    facade_y: float | None = None      # facades at +-facade_y
    facade_top: float = 0.0
    x_extent: tuple = (-1e9, 1e9)
    room: tuple | None = None          # (xmin,xmax,ymin,ymax,zmin,zmax) seen from inside
    cylinders: np.ndarray = field(default_factory=lambda: np.zeros((0, 5)))   # cx, cy, r, z0, z1
    boxes: np.ndarray = field(default_factory=lambda: np.zeros((0, 6)))       # lo xyz, hi xyz


def cast(scene: Scene, origin: np.ndarray, dirs: np.ndarray, max_range: float = 150.0):
    """First hit along each ray: returns (t [M], normal [M,3]); t = inf on miss."""
    M = dirs.shape[0]
    o = origin.astype(np.float64)
    d = dirs.astype(np.float64)
    tbest = np.full(M, np.inf)
    nbest = np.zeros((M, 3))

    def take(t, nrm, mask):
        upd = mask & (t > 1e-6) & (t < tbest)
        tbest[upd] = t[upd]
        nbest[upd] = nrm[upd] if nrm.ndim == 2 else nrm
    with np.errstate(divide="ignore", invalid="ignore"):
        if scene.room is not None:
            x0, x1, y0, y1, z0, z1 = scene.room
            for axis, lo, hi in ((0, x0, x1), (1, y0, y1), (2, z0, z1)):
                for plane, sgn in ((lo, 1.0), (hi, -1.0)):
                    t = (plane - o[axis]) / d[:, axis]
                    nrm = np.zeros(3); nrm[axis] = sgn
                    take(t, np.broadcast_to(nrm, (M, 3)), np.isfinite(t))
        if scene.ground_z is not None:
            t = (scene.ground_z - o[2]) / d[:, 2]
            take(t, np.broadcast_to(np.array([0, 0, 1.0]), (M, 3)), d[:, 2] < 0)
        if scene.facade_y is not None:
            for yf, sgn in ((scene.facade_y, -1.0), (-scene.facade_y, 1.0)):
                t = (yf - o[1]) / d[:, 1]
                z = o[2] + t * d[:, 2]
                x = o[0] + t * d[:, 0]
                ok = (z <= scene.facade_top) & (x >= scene.x_extent[0]) & (x <= scene.x_extent[1])
                take(t, np.broadcast_to(np.array([0, sgn, 0.0]), (M, 3)), ok)
        for cx, cy, r, z0, z1 in scene.cylinders:
            ox, oy = o[0] - cx, o[1] - cy
            a = d[:, 0] ** 2 + d[:, 1] ** 2
            b = 2 * (ox * d[:, 0] + oy * d[:, 1])
            c = ox * ox + oy * oy - r * r
            disc = b * b - 4 * a * c
            ok = disc >= 0
            t = (-b - np.sqrt(np.where(ok, disc, 0))) / (2 * a)
            z = o[2] + t * d[:, 2]
            ok &= (z >= z0) & (z <= z1)
            p = o[None, :2] + t[:, None] * d[:, :2] - np.array([cx, cy])
            nrm = np.concatenate([p / r, np.zeros((M, 1))], 1)
            take(t, nrm, ok)
    if len(scene.boxes):
        # a box entirely beyond max_range cannot give a kept hit (hits beyond
        # it are discarded below): only the nearer boxes are tested
        B = np.asarray(scene.boxes, np.float64).reshape(-1, 6)
        gap = np.maximum(np.maximum(B[:, :3] - o, o - B[:, 3:]), 0.0)
        near = (gap * gap).sum(1) <= max_range * max_range
        _cast_boxes(B[near], o, d, tbest, nbest)
    tbest[tbest > max_range] = np.inf
    return tbest, nbest


def _cast_boxes(boxes, o, d, tbest, nbest):
    """Slab test of the rays against each axis-aligned box, restricted to the
    rays whose azimuth falls inside the box's azimuth span."""
    inv = np.where(np.abs(d) > 1e-12, 1.0 / np.where(np.abs(d) > 1e-12, d, 1.0), 1e12)
    az = np.arctan2(d[:, 1], d[:, 0])
    order = np.argsort(az)
    az_sorted = az[order]
    for b in boxes:
        lo, hi = b[:3] - o, b[3:] - o
        # azimuth span of the box (boxes never contain the sensor)
        cx = np.array([lo[0], hi[0], lo[0], hi[0]]); cy = np.array([lo[1], lo[1], hi[1], hi[1]])
        a = np.arctan2(cy, cx)
        ac = math.atan2(cy.mean(), cx.mean())
        rel = np.angle(np.exp(1j * (a - ac)))
        amin, amax = ac + rel.min() - 1e-3, ac + rel.max() + 1e-3
        segs = []
        for lo_a, hi_a in ((amin, amax), (amin - 2 * np.pi, amax - 2 * np.pi), (amin + 2 * np.pi, amax + 2 * np.pi)):
            i0, i1 = np.searchsorted(az_sorted, [lo_a, hi_a])
            if i1 > i0:
                segs.append(order[i0:i1])
        if not segs:
            continue
        idx = np.concatenate(segs)
        t0 = lo[None, :] * inv[idx]
        t1 = hi[None, :] * inv[idx]
        tn = np.minimum(t0, t1); tf = np.maximum(t0, t1)
        tenter = tn.max(1); texit = tf.min(1)
        hit = (tenter <= texit) & (tenter > 1e-6) & (tenter < tbest[idx])
        if not hit.any():
            continue
        ids = idx[hit]
        ax = tn[hit].argmax(1)
        nrm = np.zeros((len(ids), 3))
        nrm[np.arange(len(ids)), ax] = -np.sign(d[ids, ax])
        tbest[ids] = tenter[hit]
        nbest[ids] = nrm


def simulate_scan(scene: Scene, frame: Frame, rng: np.random.Generator, noise: float = 0.02,
                  drop: float = 0.1, max_range: float = 150.0):
    """Range image of the simulated sensor at the frame's pose.
    Returns (D [H,W] float32 with 0 = no return, points_world [H,W,3],
    true normals [H,W,3] oriented toward the sensor, valid [H,W])."""
    P = np.asarray(frame.pose, np.float64).reshape(3, 4)
    R, o = P[:, :3], P[:, 3]
    ds = sensor_rays(frame.H, frame.W, frame.elev_min, frame.elev_max).reshape(-1, 3)
    dw = ds @ R.T
    t, nrm = cast(scene, o, dw, max_range)
    valid = np.isfinite(t)
    r = np.where(valid, t + rng.normal(0.0, noise, t.shape) if noise > 0 else t, 0.0)
    if drop > 0:
        valid &= rng.random(t.shape) >= drop
    r = np.where(valid, r, 0.0)
    pts = o[None] + r[:, None] * dw
    flip = (nrm * dw).sum(1) > 0
    nrm = np.where(flip[:, None], -nrm, nrm)
    H, W = frame.H, frame.W
    return (r.reshape(H, W).astype(np.float32), pts.reshape(H, W, 3), nrm.reshape(H, W, 3),
            valid.reshape(H, W))


def knn_covariances(points: np.ndarray, k: int = 20):
    """Eigen-decomposition of the k-nearest-neighbour covariance of each point:
    eigenvalues descending [n,3] and eigenvectors as columns [n,3,3]."""
    from scipy.spatial import cKDTree
    tree = cKDTree(points)
    _, idx = tree.query(points, k=k, workers=-1)
    nb = points[idx]                                  # [n,k,3]
    c = nb - nb.mean(1, keepdims=True)
    cov = np.einsum("nki,nkj->nij", c, c) / k
    w, v = np.linalg.eigh(cov)                        # ascending
    return w[:, ::-1].copy(), v[:, :, ::-1].copy()


def surfels_from_points(points: np.ndarray, origins: np.ndarray, rng: np.random.Generator,
                        kappa: float, s_max: float = 1.0, k: int = 20, normals=None) -> Surfels:
    """Surfels at the given points.  Tangent axes and normal from the k-NN
    covariance eigenvectors (normal toward the observing sensor); scale from
    the paper's range-adaptive initialisation s = clip(kappa r sigma_tan, ., s_max)
    with sigma_tan the two largest standard deviations normalised by the
    largest and r = max(|p - origin|, 1); opacity U(0.3, 0.9)."""
    n = points.shape[0]
    if normals is None:
        lam, vec = knn_covariances(points, k)
        t0, nrm = vec[:, :, 0], vec[:, :, 2]
        sig = np.sqrt(np.maximum(lam[:, :2], 1e-18))
        sig_tan = sig / sig[:, :1]
    else:
        nrm = normals
        rnd = rng.normal(size=(n, 3))
        t0 = np.cross(nrm, rnd)
        sig_tan = np.stack([np.ones(n), rng.uniform(0.4, 1.0, n)], 1)
    view = origins - points
    flip = (nrm * view).sum(1) < 0
    nrm = np.where(flip[:, None], -nrm, nrm)
    Rm = frames_from_axes(t0, nrm)
    rng_r = np.maximum(np.linalg.norm(points - origins, axis=1), 1.0)
    s = np.clip(kappa * rng_r[:, None] * sig_tan, 1e-3, s_max)
    alpha = rng.uniform(0.3, 0.9, n)
    return Surfels(points.astype(np.float32), rot_to_quat(Rm).astype(np.float32),
                   np.log(s).astype(np.float32), _logit(alpha).astype(np.float32))


def target_from_scan(D, pts, valid, k: int = 20, true_normals=None, origin=None):
    """Tracking-normal target N_gicp [3,H,W]: smallest-eigenvector normal of
    the k-NN covariance of the scan's own points, oriented toward the sensor;
    zero where the pixel has no return."""
    H, W = D.shape
    N = np.zeros((H, W, 3), np.float32)
    if valid.any():
        p = pts[valid]
        if true_normals is not None:
            nv = true_normals[valid]
        else:
            _, vec = knn_covariances(p, k)
            nv = vec[:, :, 2]
            view = origin[None] - p
            nv = np.where(((nv * view).sum(1) < 0)[:, None], -nv, nv)
        N[valid] = nv
    return Target(D.astype(np.float32), np.ascontiguousarray(N.transpose(2, 0, 1)))


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------
def box_room(seed: int = 0, n: int = 2000, H: int = 32, W: int = 512, tile=(16, 16),
             yaw: float = 0.0):
    """2,000 surfels on the 6 faces of a 20 x 20 x 5 m room (uniform by area),
    centres jittered N(0, 2 cm) along the face normal, in-plane rotation
    U(0, 2 pi), scales U(5, 30) cm, opacity U(0.3, 0.9); sensor at the room
    centre; 32 x 512 image over +-15 deg.  Target: analytic range + N(0, 2 cm)."""
    rng = np.random.default_rng(seed)
    x0, x1, y0, y1, z0, z1 = -10.0, 10.0, -10.0, 10.0, 0.0, 5.0
    faces = [  # (axis, value, inward normal sign, area)
        (2, z0, 1.0, 400.0), (2, z1, -1.0, 400.0),
        (0, x0, 1.0, 100.0), (0, x1, -1.0, 100.0), (1, y0, 1.0, 100.0), (1, y1, -1.0, 100.0)]
    areas = np.array([f[3] for f in faces])
    fid = rng.choice(len(faces), size=n, p=areas / areas.sum())
    pts = np.zeros((n, 3)); nrm = np.zeros((n, 3))
    lo = np.array([x0, y0, z0]); hi = np.array([x1, y1, z1])
    for i, (ax, val, sgn, _) in enumerate(faces):
        m = fid == i
        k = int(m.sum())
        p = lo + rng.random((k, 3)) * (hi - lo)
        p[:, ax] = val
        nn = np.zeros((k, 3)); nn[:, ax] = sgn
        pts[m] = p + nn * rng.normal(0, 0.02, (k, 1))
        nrm[m] = nn
    t0 = np.cross(nrm, rng.normal(size=(n, 3)))
    Rm = frames_from_axes(t0, nrm)
    scale = rng.uniform(0.05, 0.30, (n, 2))
    alpha = rng.uniform(0.3, 0.9, n)
    surf = Surfels(pts.astype(np.float32), rot_to_quat(Rm).astype(np.float32),
                   np.log(scale).astype(np.float32), _logit(alpha).astype(np.float32))
    frame = Frame(H, W, tile[0], tile[1], -math.radians(15), math.radians(15),
                  pose_matrix(yaw, (0.0, 0.0, 2.5)))
    scene = Scene(room=(x0, x1, y0, y1, z0, z1))
    D, p, tn, valid = simulate_scan(scene, frame, rng, noise=0.02, drop=0.0)
    tgt = target_from_scan(D, p, valid, true_normals=tn)
    return surf, frame, tgt


def street_scene(rng: np.random.Generator, x_extent=(-60.0, 60.0), n_boxes: int = 2000,
                 n_cyl: int = 40, keep_clear=((0.0, 0.0),), clear_r: float = 2.5) -> Scene:
    """Ground z = -1.8 m, facades at y = +-8 m (12 m tall), vertical cylinders
    r in U(0.1, 0.4) m and 3 m tall, boxes with edges U(0.2, 1.5) m resting on
    the ground, kept clear of the sensor positions."""
    gz = -1.8
    xs, xe = x_extent
    cyl = np.zeros((n_cyl, 5))
    cyl[:, 0] = rng.uniform(xs, xe, n_cyl)
    cyl[:, 1] = rng.choice([-1.0, 1.0], n_cyl) * rng.uniform(4.0, 7.5, n_cyl)
    cyl[:, 2] = rng.uniform(0.1, 0.4, n_cyl)
    cyl[:, 3] = gz; cyl[:, 4] = gz + 3.0
    boxes = []
    clear = np.array(keep_clear, np.float64).reshape(-1, 2)
    while len(boxes) < n_boxes:
        m = 4 * (n_boxes - len(boxes))
        c = np.stack([rng.uniform(xs, xe, m), rng.uniform(-7.2, 7.2, m)], 1)
        e = rng.uniform(0.2, 1.5, (m, 3))
        dist = np.min(np.abs(c[:, None, 0] - clear[None, :, 0]) - e[:, None, 0] / 2, 1)
        dy = np.min(np.abs(c[:, None, 1] - clear[None, :, 1]) - e[:, None, 1] / 2, 1)
        ok = (dist > clear_r) | (dy > clear_r)
        for ci, ei in zip(c[ok], e[ok]):
            lo = [ci[0] - ei[0] / 2, ci[1] - ei[1] / 2, gz]
            hi = [ci[0] + ei[0] / 2, ci[1] + ei[1] / 2, gz + ei[2]]
            boxes.append(lo + hi)
            if len(boxes) >= n_boxes:
                break
    return Scene(ground_z=gz, facade_y=8.0, facade_top=gz + 12.0, x_extent=(xs - 40, xe + 40),
                 cylinders=cyl, boxes=np.array(boxes))


def lidar_frame(H=128, W=1024, tile=(16, 16), elev_deg=45.0, pose=None) -> Frame:
    return Frame(H, W, tile[0], tile[1], -math.radians(elev_deg), math.radians(elev_deg),
                 pose if pose is not None else pose_matrix())


def _kappa(frame: Frame) -> float:
    """kappa = 1.5 x the larger angular pixel pitch (radians)."""
    return 1.5 * max((frame.elev_max - frame.elev_min) / frame.H, 2 * math.pi / frame.W)


def street(seed: int = 0, n: int = 200_000, H: int = 128, W: int = 1024, tile=(16, 16),
           yaw: float = 0.3, second_scan_dx: float = 1.5):
    """Street map of ``n`` surfels from two merged 128 x 1024 scans at x = 0
    and x = +1.5 m (k = 20 NN covariance init), and the frame + target of the
    scan at x = 0."""
    rng = np.random.default_rng(seed)
    scene = street_scene(rng, keep_clear=((0.0, 0.0), (second_scan_dx, 0.0)))
    f0 = lidar_frame(H, W, tile, pose=pose_matrix(yaw, (0.0, 0.0, 0.0)))
    f1 = lidar_frame(H, W, tile, pose=pose_matrix(yaw + 0.1, (second_scan_dx, 0.0, 0.0)))
    D0, p0, n0, v0 = simulate_scan(scene, f0, rng)
    D1, p1, n1, v1 = simulate_scan(scene, f1, rng)
    pts = np.concatenate([p0[v0], p1[v1]])
    org = np.concatenate([np.broadcast_to(f0.pose.reshape(3, 4)[:, 3], (int(v0.sum()), 3)),
                          np.broadcast_to(f1.pose.reshape(3, 4)[:, 3], (int(v1.sum()), 3))])
    sel = rng.choice(pts.shape[0], size=min(n, pts.shape[0]), replace=False)
    sel.sort()
    surf = surfels_from_points(pts[sel], org[sel], rng, _kappa(f0))
    tgt = target_from_scan(D0, p0, v0, origin=f0.pose.reshape(3, 4)[:, 3].astype(np.float64))
    return surf, f0, tgt


def _track_scan(scene, seed: int, i: int, x: float, map_H: int, map_W: int, tile):
    """Map scan i of street_track (points, normals of the valid returns), from
    its own generator (seed, i)."""
    rng = np.random.default_rng([seed, i])
    fr = lidar_frame(map_H, map_W, tile, pose=pose_matrix(0.05 * i, (x, 0.0, 0.0)))
    _, p, nr, v = simulate_scan(scene, fr, rng)
    return p[v], nr[v]


def _track_keyframe(scene, seed: int, j: int, x: float, H: int, W: int, tile):
    rng = np.random.default_rng([seed, 10_000 + j])
    fr = lidar_frame(H, W, tile, pose=pose_matrix(0.02 * j, (x, 0.0, 0.0)))
    D, p, nr, v = simulate_scan(scene, fr, rng)
    return fr, target_from_scan(D, p, v, true_normals=nr)


def street_track(seed: int = 0, n: int = 1_000_000, n_keyframes: int = 8, spacing: float = 3.0,
                 length: float = 200.0, H: int = 128, W: int = 1024, tile=(16, 16),
                 map_H: int = 64, map_W: int = 1024, pool=None):
    """Street extended to a ``length`` m track.  The map: surfels at returns of
    scans every ``spacing`` m along the track (``map_H`` x ``map_W`` beams,
    true surface normals, range-adaptive scales), sub-sampled to ``n``.  The
    keyframes: ``n_keyframes`` consecutive poses ``spacing`` m apart in the
    middle of the track, each with its own target scan (H x W).  Every scan
    has its own generator, so ``pool`` (an executor) may simulate them in
    parallel."""
    rng = np.random.default_rng(seed)
    xs = np.arange(-length / 2, length / 2 + 1e-6, spacing)
    scene = street_scene(rng, x_extent=(-length / 2 - 10, length / 2 + 10),
                         n_boxes=int(2000 * (length + 20) / 120), keep_clear=[(x, 0.0) for x in xs])
    K = len(xs)
    scans = _map(pool, _track_scan, [scene] * K, [seed] * K, range(K), list(xs), [map_H] * K, [map_W] * K,
                 [tile] * K)
    pts = np.concatenate([p for p, _ in scans])
    nrm = np.concatenate([q for _, q in scans])
    org = np.concatenate([np.broadcast_to(np.array([x, 0.0, 0.0]), (len(p), 3)) for x, (p, _) in zip(xs, scans)])
    sel = rng.choice(pts.shape[0], size=min(n, pts.shape[0]), replace=False)
    sel.sort()
    kappa = _kappa(lidar_frame(map_H, map_W, tile))
    surf = surfels_from_points(pts[sel], org[sel], rng, kappa, normals=nrm[sel])
    k0 = len(xs) // 2 - n_keyframes // 2
    kf = _map(pool, _track_keyframe, [scene] * n_keyframes, [seed] * n_keyframes, range(n_keyframes),
              [xs[k0 + j] for j in range(n_keyframes)], [H] * n_keyframes, [W] * n_keyframes, [tile] * n_keyframes)
    return surf, [f for f, _ in kf], [t for _, t in kf]


def random_shell(seed: int, n: int, r_range=(2.0, 20.0), scale_range=(0.05, 0.6),
                 frame: Frame | None = None, face_sensor: bool = False):
    """Small test scene: surfels at random directions and ranges around the
    sensor with random orientations (or facing the sensor)."""
    rng = np.random.default_rng(seed)
    frame = frame or Frame(32, 64, 16, 16, -math.radians(30), math.radians(30))
    P = np.asarray(frame.pose, np.float64).reshape(3, 4)
    el = rng.uniform(frame.elev_min, frame.elev_max, n)
    az = rng.uniform(0, 2 * np.pi, n)
    r = rng.uniform(*r_range, n)
    ds = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], 1)
    pts = P[:, 3] + (r[:, None] * ds) @ P[:, :3].T
    if face_sensor:
        nrm = -(ds @ P[:, :3].T)
    else:
        nrm = rng.normal(size=(n, 3))
    Rm = frames_from_axes(rng.normal(size=(n, 3)), nrm)
    scale = rng.uniform(*scale_range, (n, 2))
    alpha = rng.uniform(0.3, 0.95, n)
    return Surfels(pts.astype(np.float32), rot_to_quat(Rm).astype(np.float32),
                   np.log(scale).astype(np.float32), _logit(alpha).astype(np.float32)), frame


def targets_for(frame: Frame, surf: Surfels, seed: int = 0, drop: float = 0.1):
    """A synthetic target for a test scene: ranges U(2, 20) m with ``drop``
    of the pixels empty, random unit normals with 5 % zeroed; it only
    exercises the loss and its masks."""
    rng = np.random.default_rng(seed)
    H, W = frame.H, frame.W
    D = rng.uniform(2.0, 20.0, (H, W)).astype(np.float32)
    D[rng.random((H, W)) < drop] = 0.0
    N = rng.normal(size=(3, H, W))
    N /= np.linalg.norm(N, axis=0, keepdims=True)
    N[:, rng.random((H, W)) < 0.05] = 0.0
    return Target(D, N.astype(np.float32))


def sample_street_surfaces(scene: Scene, rng: np.random.Generator, n: int, x_range):
    """``n`` points uniform by area on the street's surfaces with x in
    ``x_range`` (ground, both facades, cylinder sides, box tops and sides),
    with their true normals: a map that many viewpoints would have built."""
    x0, x1 = x_range
    gz, fy, ft = scene.ground_z, scene.facade_y, scene.facade_top
    cyl = scene.cylinders[(scene.cylinders[:, 0] >= x0) & (scene.cylinders[:, 0] <= x1)]
    box = scene.boxes[(scene.boxes[:, 0] >= x0) & (scene.boxes[:, 3] <= x1)]
    ex = box[:, 3:] - box[:, :3]
    parts = [("ground", 2 * fy * (x1 - x0)), ("facades", 2 * (x1 - x0) * (ft - gz)),
             ("cyl", float((2 * np.pi * cyl[:, 2] * (cyl[:, 4] - cyl[:, 3])).sum())),
             ("box", float((ex[:, 0] * ex[:, 1] + 2 * ex[:, 2] * (ex[:, 0] + ex[:, 1])).sum()))]
    areas = np.array([a for _, a in parts])
    counts = rng.multinomial(n, areas / areas.sum())
    P, N = [], []
    m = counts[0]
    P.append(np.stack([rng.uniform(x0, x1, m), rng.uniform(-fy, fy, m), np.full(m, gz)], 1))
    N.append(np.broadcast_to([0.0, 0.0, 1.0], (m, 3)))
    m = counts[1]
    side = rng.choice([-1.0, 1.0], m)
    P.append(np.stack([rng.uniform(x0, x1, m), side * fy, rng.uniform(gz, ft, m)], 1))
    N.append(np.stack([np.zeros(m), -side, np.zeros(m)], 1))
    m = counts[2]
    if m and len(cyl):
        w = 2 * np.pi * cyl[:, 2] * (cyl[:, 4] - cyl[:, 3])
        c = cyl[rng.choice(len(cyl), m, p=w / w.sum())]
        a = rng.uniform(0, 2 * np.pi, m)
        P.append(np.stack([c[:, 0] + c[:, 2] * np.cos(a), c[:, 1] + c[:, 2] * np.sin(a),
                           rng.uniform(c[:, 3], c[:, 4])], 1))
        N.append(np.stack([np.cos(a), np.sin(a), np.zeros(m)], 1))
    m = counts[3]
    if m and len(box):
        fa = np.stack([ex[:, 0] * ex[:, 1], ex[:, 1] * ex[:, 2], ex[:, 1] * ex[:, 2], ex[:, 0] * ex[:, 2],
                       ex[:, 0] * ex[:, 2]], 1)            # top, -x, +x, -y, +y
        flat = fa.ravel() / fa.sum()
        k = rng.choice(flat.size, m, p=flat)
        b, f = k // 5, k % 5
        lo, hi = box[b, :3], box[b, 3:]
        u = rng.uniform(lo, hi)
        nrm = np.zeros((m, 3))
        top = f == 0
        u[top, 2] = hi[top, 2]; nrm[top, 2] = 1.0
        for face, axis, sgn in ((1, 0, -1.0), (2, 0, 1.0), (3, 1, -1.0), (4, 1, 1.0)):
            sel = f == face
            u[sel, axis] = np.where(sgn > 0, hi[sel, axis], lo[sel, axis])
            nrm[sel, axis] = sgn
        P.append(u)
        N.append(nrm)
    return np.concatenate(P), np.concatenate(N)


def _street_map(scene, seed: int, i: int, n: int, x: float, shape, tile):
    """Map i of street_maps, from its own generator (seed, i)."""
    rng = np.random.default_rng([seed, i])
    H, W = shape
    half = 20.0 + n / 25000.0
    pts, nrm = sample_street_surfaces(scene, rng, int(n), (x - half, x + half))
    o = np.array([x, 0.0, 0.0])
    fr = lidar_frame(H, W, tile, pose=pose_matrix(0.1 * i, (x, 0.0, 0.0)))
    surf = surfels_from_points(pts, np.broadcast_to(o, pts.shape), rng, _kappa(fr), normals=nrm)
    D, p, nr, v = simulate_scan(scene, fr, rng)
    return surf, fr, target_from_scan(D, p, v, true_normals=nr)


def _map(pool, fn, *iterables):
    """map over a concurrent.futures executor, or serially without one (the
    results do not depend on it: every item has its own generator)."""
    return list(pool.map(fn, *iterables)) if pool is not None else list(map(fn, *iterables))


def street_maps(seed: int, sizes, shapes, tile=(8, 8), spacing: float = 25.0, noise_targets: bool = True,
                pool=None):
    """Independent maps of uneven size along one long street (one per entry of
    ``sizes``), each with one frame of shape ``shapes[i % len(shapes)]`` (H, W)
    at the map's centre and its simulated target scan.  Map ``i`` holds
    ``sizes[i]`` surfels on the street's surfaces within +-(20 + n / 25k) m
    of its sensor, with range-adaptive scales, drawn from its own generator
    (seed, i), so ``pool`` (an executor) may build the maps in parallel.
    Returns [(surfels, frame, target)]."""
    rng = np.random.default_rng(seed)
    M = len(sizes)
    xs = (np.arange(M) - (M - 1) / 2) * spacing
    span = max(20.0 + max(sizes) / 25000.0, spacing)
    scene = street_scene(rng, x_extent=(xs[0] - span - 10, xs[-1] + span + 10),
                         n_boxes=int(2000 * (xs[-1] - xs[0] + 2 * span) / 120),
                         keep_clear=[(x, 0.0) for x in xs])
    return _map(pool, _street_map, [scene] * M, [seed] * M, range(M), [int(n) for n in sizes], list(xs),
                [shapes[i % len(shapes)] for i in range(M)], [tile] * M)


# --- inputs of map management --------------------------------------------------
def manage_cluster(seed: int, n: int):
    """A small clustered map: surfels on two planes (z = -0.5 and x = 0.2,
    1 cm jitter) and scattered clutter in a 4 m box about the origin, with the
    tracking signals map management reads: covariance eigenvalues near
    (1, 0.8, 0) on the planes and random on the clutter, and exponential
    residuals.  Returns (mean, quat, log_scale, logit, lam, res), float32."""
    rng = np.random.default_rng(seed)
    kind = rng.integers(0, 3, n)
    pos = rng.uniform(-2, 2, (n, 3))
    pos[kind == 0, 2] = rng.normal(-0.5, 0.01, (kind == 0).sum())
    pos[kind == 1, 0] = rng.normal(0.2, 0.01, (kind == 1).sum())
    nrm = np.where((kind == 0)[:, None], [0, 0, 1.0],
                   np.where((kind == 1)[:, None], [1.0, 0, 0], rng.normal(size=(n, 3))))
    R = frames_from_axes(rng.normal(size=(n, 3)), nrm)
    quat = rot_to_quat(R).astype(np.float32)
    ls = np.log(rng.uniform(0.05, 0.4, (n, 2))).astype(np.float32)
    logit = rng.normal(0.5, 2.0, n).astype(np.float32)
    lam = np.where((kind == 2)[:, None], rng.uniform(0, 1, (n, 3)), [1.0, 0.8, 0.0])
    lam = (lam + rng.uniform(0, 0.05, (n, 3))).astype(np.float32)
    res = rng.exponential(0.02, n).astype(np.float32)
    return pos.astype(np.float32), quat, ls, logit, lam, res


def manage_signals(points: np.ndarray, k: int = 20, seed: int = 0, noise: float = 0.01):
    """Stand-ins for the per-surfel signals tracking hands to map management
    (Sec. 3.3): the eigenvalues (descending) of the k-NN covariance of the
    map's own means, and a registration residual: the distance from the
    point to its neighbours' plane plus |N(0, noise)|.  Returns float32
    (lam [n, 3], res [n])."""
    from scipy.spatial import cKDTree
    pts = np.asarray(points, np.float64)
    tree = cKDTree(pts)
    _, idx = tree.query(pts, k=k, workers=-1)
    lam = np.empty((pts.shape[0], 3))
    res = np.empty(pts.shape[0])
    step = 1 << 18
    for a in range(0, pts.shape[0], step):
        nb = pts[idx[a:a + step]]
        mu = nb.mean(1)
        c = nb - mu[:, None]
        cov = np.einsum("nki,nkj->nij", c, c) / k
        w, v = np.linalg.eigh(cov)
        lam[a:a + step] = np.maximum(w[:, ::-1], 0.0)
        res[a:a + step] = np.abs(((pts[a:a + step] - mu) * v[:, :, 0]).sum(1))
    res += np.abs(np.random.default_rng(seed).normal(0.0, noise, pts.shape[0]))
    return lam.astype(np.float32), res.astype(np.float32)


def keyframe_points(seed: int = 0, H: int = 128, W: int = 1024, elev_deg: float = 45.0, yaw: float = 0.3,
                    t=(0.0, 0.0, 0.0), drop: float = 0.1):
    """One simulated scan of the street (range noise 2 cm, ray drops) as the
    points of a keyframe in the sensor frame, in scan order (row-major over
    the range image), with its pose.  Returns (points float32 [n, 3], pose
    float64 [12])."""
    rng = np.random.default_rng(seed)
    scene = street_scene(rng, keep_clear=((t[0], t[1]),))
    fr = lidar_frame(H, W, (16, 16), elev_deg=elev_deg, pose=pose_matrix(yaw, t))
    _, pw, _, valid = simulate_scan(scene, fr, rng, drop=drop)
    P = np.asarray(fr.pose, np.float64).reshape(3, 4)
    ps = (pw.reshape(-1, 3)[valid.reshape(-1)] - P[:, 3]) @ P[:, :3]
    return ps.astype(np.float32), P.reshape(-1)
