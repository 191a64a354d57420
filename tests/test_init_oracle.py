"""Pins of the keyframe-initialisation oracle (k-NN covariance, Sec. 3.2;
range-adaptive scale, confidence u and opacity, Sec. 3.3 Eqs. physconf and
alpha_init) against a library k-NN, brute force with ties, closed-form
covariances and special cases.  CPU only.

  I1 k-NN == scipy cKDTree (distances; sets away from near-ties)
  I2 k-NN == brute force over sorted (distance, index) on a grid full of ties
  I3 a regular 5 x 4 grid facing the sensor: eigenvalues (2 a^2, 1.25 b^2, 0),
     normal toward the sensor, in-plane axes, scales kappa r (1, sqrt(l1/l0))
  I4 a line: l1 = l2 = 0, scale floor; coincident points: l = 0, sigma_tan (1, 1)
  I5 confidence: straight-on exp(-(r/r0)^2), at or below c0 zero, alpha ends
  I6 frames orthonormal and right-handed, the quaternion reproduces them,
     world mean and frame follow the pose
"""
import math

import numpy as np
import pytest

F = np.float32


@pytest.fixture(scope="module")
def oi():
    from oracle import init
    return init


def _quat_to_rot(q):
    """Textbook unit quaternion (w, x, y, z) -> rotation matrix."""
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_knn_matches_kdtree(oi):
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(0)
    pts = (rng.normal(size=(3000, 3)) * [10, 10, 2]).astype(F)
    idx, d2 = oi.knn(pts, 20)
    dist, kidx = cKDTree(pts.astype(np.float64)).query(pts.astype(np.float64), k=21)
    assert np.allclose(np.sqrt(d2.astype(np.float64)), dist[:, :20], rtol=1e-6, atol=1e-6)
    clear = dist[:, 20] - dist[:, 19] > 1e-4 * dist[:, 20]
    assert clear.mean() > 0.9
    same = [set(a) == set(b) for a, b in zip(idx[clear], kidx[clear, :20])]
    assert all(same)
    assert np.all(idx[:, 0] == np.arange(3000))          # each point is its own nearest


def test_knn_ties_brute_force(oi):
    """Integer grid: many exact distance ties, broken by index."""
    g = np.stack(np.meshgrid(np.arange(4), np.arange(5), np.arange(3), indexing="ij"), -1).reshape(-1, 3)
    pts = g[np.random.default_rng(1).permutation(len(g))].astype(F)
    k = 9
    idx, d2 = oi.knn(pts, k)
    for i in range(len(pts)):
        cand = sorted((float(((pts[j] - pts[i]) ** 2).sum()), j) for j in range(len(pts)))[:k]
        assert idx[i].tolist() == [j for _, j in cand]
        assert d2[i].tolist() == [d for d, _ in cand]


def _grid(a=0.2, b=0.1, x=50.0, y0=0.0, z0=0.0):
    """5 x 4 grid in the plane x = const: 5 points along y (spacing a), 4 along
    z (spacing b)."""
    yy, zz = np.meshgrid(np.arange(5) * a + y0, np.arange(4) * b + z0, indexing="ij")
    return np.stack([np.full(yy.size, x), yy.ravel(), zz.ravel()], 1).astype(F)


def test_grid_covariance_and_scales(oi):
    """Variance of 0..4 spacing a is 2 a^2, of 0..3 spacing b 1.25 b^2; the
    grid's normal is -x (toward the sensor at the origin); t_u is +-y."""
    a, b = 0.2, 0.1
    pts = _grid(a, b)
    P = oi.Params(k=20, kappa=0.01, s_min=1e-4, s_max=10.0)
    out = oi.initialise(pts, np.eye(3, 4).ravel(), P)
    assert np.allclose(out["lam"], [[2 * a * a, 1.25 * b * b, 0.0]], atol=1e-9)
    assert np.allclose(out["normal_s"], [[-1, 0, 0]], atol=1e-7)
    assert np.allclose(np.abs(out["tu_s"]), [[0, 1, 0]], atol=1e-7)
    r = np.linalg.norm(pts.astype(np.float64), axis=1)
    ratio = math.sqrt(1.25 * b * b / (2 * a * a))
    assert np.allclose(np.exp(out["log_scale"]), 0.01 * r[:, None] * [1.0, ratio], rtol=1e-9)
    # clip: at s_max and at r = max(|p|, 1) near the sensor
    out = oi.initialise(pts, np.eye(3, 4).ravel(), oi.Params(k=20, kappa=0.01, s_max=0.3))
    assert np.allclose(np.exp(out["log_scale"][:, 0]), 0.3)
    near = _grid(a, b, x=0.05, y0=-0.4, z0=-0.15) * F(0.5)
    out = oi.initialise(near, np.eye(3, 4).ravel(), oi.Params(k=20, kappa=0.01))
    rr = np.linalg.norm(near.astype(np.float64), axis=1)
    assert np.all(rr < 1.0)
    assert np.allclose(np.exp(out["log_scale"][:, 0]), 0.01)


def test_line_and_coincident(oi):
    line = np.stack([np.full(20, 10.0), np.arange(20) * 0.05, np.full(20, 1.0)], 1).astype(F)
    out = oi.initialise(line, np.eye(3, 4).ravel(), oi.Params(k=20, kappa=0.01, s_min=1e-3))
    assert np.all(out["lam"][:, 1:] < 1e-12)
    assert np.allclose(np.abs(out["tu_s"]), [[0, 1, 0]], atol=1e-6)
    assert np.allclose(np.exp(out["log_scale"][:, 1]), 1e-3)
    same = np.tile(np.array([[3.0, 4.0, 0.0]], F), (20, 1))
    out = oi.initialise(same, np.eye(3, 4).ravel(), oi.Params(k=20, kappa=0.01, s_min=1e-3))
    assert np.all(out["lam"] == 0)
    assert np.allclose(np.exp(out["log_scale"]), 0.05)          # kappa * 5 m * (1, 1)


def test_confidence_and_opacity(oi):
    """A tiny patch straight ahead along x at 50 m: c = 1 to 1e-8, so
    u = exp(-(50/100)^2) (1 - c0) / (1 - c0 + eps).  Tilted so that c < c0: u = 0, alpha = alpha_min."""
    P = oi.Params(k=20, r0=100.0, c0=0.1)
    pts = _grid(0.002, 0.001, x=50.0, y0=-0.004, z0=-0.0015)   # a tiny patch: c ~ 1
    out = oi.initialise(pts, np.eye(3, 4).ravel(), P)
    # at c = 1 the ramp is (1 - c0) / (1 - c0 + eps), not quite 1
    u1 = math.exp(-0.25) * 0.9 / (0.9 + 1e-6)
    assert np.allclose(out["u"], u1, rtol=1e-7)
    assert np.allclose(out["alpha"], 0.3 + 0.6 * u1, rtol=1e-7)
    # a plane containing the ray (normal perpendicular to the view): c = 0
    graze = np.stack([np.linspace(40, 41, 20), np.linspace(0, 0.5, 20) * 0 + 0.0,
                      np.tile([0.0, 0.1, 0.2, 0.3], 5)], 1).astype(F)
    out = oi.initialise(graze, np.eye(3, 4).ravel(), P)
    assert np.allclose(out["u"], 0.0) and np.allclose(out["alpha"], 0.3)
    assert np.allclose(out["logit"], math.log(0.3 / 0.7))


def test_frames_quaternions_and_pose(oi):
    rng = np.random.default_rng(5)
    pts = (rng.normal(size=(400, 3)) * [5, 5, 0.3] + [20, 0, -1.5]).astype(F)
    yaw = 0.7
    Rz = np.array([[math.cos(yaw), -math.sin(yaw), 0], [math.sin(yaw), math.cos(yaw), 0], [0, 0, 1]])
    t = np.array([3.0, -2.0, 1.0])
    pose = np.concatenate([Rz, t[:, None]], 1).ravel()
    out = oi.initialise(pts, pose, oi.Params())
    R = out["rot"]
    assert np.allclose(np.einsum("nij,nik->njk", R, R), np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(R), 1.0)
    for q, Rm in zip(out["quat"][:50], R[:50]):
        assert q[0] >= 0 and np.allclose(_quat_to_rot(q), Rm, atol=1e-12)
    assert np.allclose(out["mean"], pts.astype(np.float64) @ Rz.T + t)
    assert np.allclose(R[:, :, 2], out["normal_s"] @ Rz.T)
    assert np.all((out["normal_s"] * pts).sum(1) <= 0)            # toward the sensor
    base = oi.initialise(pts, np.eye(3, 4).ravel(), oi.Params())
    for key in ("lam", "u", "log_scale", "logit"):
        assert np.allclose(out[key], base[key])
    assert np.array_equal(out["knn"], base["knn"])


def test_knn_binary32_distance_order(oi):
    """The squared distance is ((dx dx + dy dy) + dz dz) in binary32: a
    scalar restatement over all pairs of random points, sorted by (distance
    bits, index), picks the same neighbours and distances."""
    rng = np.random.default_rng(7)
    pts = (rng.normal(size=(80, 3)) * [3.0, 0.01, 1e3] + [1e3, 0, 0]).astype(F)
    idx, d2 = oi.knn(pts, 6)
    f = np.float32
    for i in range(len(pts)):
        cand = []
        for j in range(len(pts)):
            dx, dy, dz = (f(pts[j][t] - pts[i][t]) for t in range(3))
            d = f(f(f(dx * dx) + f(dy * dy)) + f(dz * dz))
            cand.append((int(np.array([d], f).view(np.uint32)[0]), j, d))
        cand.sort()
        assert idx[i].tolist() == [j for _, j, _ in cand[:6]]
        assert d2[i].tolist() == [d for _, _, d in cand[:6]]


def test_confidence_uses_the_range_itself(oi):
    """u takes r = |p| (the scale takes max(|p|, 1)): a patch facing the
    sensor at 0.5 m with r0 = 1 gives exp(-|p|^2) times the ramp."""
    pts = _grid(0.002, 0.001, x=0.5, y0=-0.004, z0=-0.0015)
    out = oi.initialise(pts, np.eye(3, 4).ravel(), oi.Params(k=20, r0=1.0, c0=0.1))
    r = np.linalg.norm(pts.astype(np.float64), axis=1)
    # the patch lies in the plane x = 0.5 (normal -x), so c = 0.5 / |p|
    assert np.allclose(out["u"], np.exp(-r * r) * (0.5 / r - 0.1) / (0.9 + 1e-6), rtol=1e-7)


def test_exact_scaling_invariance(oi):
    """Doubling every point is exact in binary32: squared distances scale by
    exactly 4 (same neighbour lists, same order), the covariance by exactly
    4, so the eigenvalues scale by 4 and the frames do not change."""
    rng = np.random.default_rng(13)
    pts = (rng.normal(size=(600, 3)) * [4.0, 2.0, 0.3] + [15.0, -3.0, 1.0]).astype(F)
    a = oi.initialise(pts, np.eye(3, 4).ravel(), oi.Params(k=12))
    b = oi.initialise(pts * F(2), np.eye(3, 4).ravel(), oi.Params(k=12))
    assert np.array_equal(a["knn"], b["knn"])
    ia, da = oi.knn(pts, 12)
    ib, db = oi.knn(pts * F(2), 12)
    assert np.array_equal(ia, ib) and np.array_equal(db, da * F(4))
    assert np.allclose(b["lam"], 4 * a["lam"], rtol=1e-12, atol=1e-15)
    gap = (a["lam"][:, 1] - a["lam"][:, 2]) > 1e-6 * a["lam"][:, 0]
    assert np.allclose(b["normal_s"][gap], a["normal_s"][gap], atol=1e-9)
