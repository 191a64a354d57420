"""Keyframe initialisation on the device (Sec. 3.2 k-NN covariance; Sec. 3.3
range-adaptive scale, Eq. physconf, Eq. alpha_init) against the oracle
through the C-ABI.  Neighbour sets bit-exact (specified binary32 distances,
ties by index); the rest within tolerances derived from binary32 arithmetic:

  eigenvalues: the covariance is formed from exact neighbour offsets, each
    product and sum rounded (k <= 32 terms) and Jacobi adds a few ulps of the
    largest eigenvalue: |d lambda| <= 2e-6 lambda_0 + 1e-12;
  normal / major axis: an eigenvector moves by |d A| / gap, so they are
    compared where the gap exceeds 1e-3 lambda_0 (|n . n'| >= 1 - 1e-5 and
    |t_u . t_u'| >= 1 - 1e-5, the sign of t_u being free);
  log-scales: d log s_1 = (d lambda_1 / lambda_1 - d lambda_0 / lambda_0) / 2,
    i.e. <= 2e-6 lambda_0 / lambda_1 + 1e-5 off the clip bounds;
  confidence: u depends on the normal through c, |d u| <= |d c| / (1 - c0) +
    1e-6 with |d c| <= the normal's error.
"""
import math

import numpy as np
import pytest

from paper_2607_04127_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_04127_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def oi():
    from oracle import init
    return init


def _gpu(points, pose, **kw):
    import torch
    from paper_2607_04127_gb300 import keyframe
    t = torch.from_numpy(np.ascontiguousarray(points, np.float32)).cuda()
    out = keyframe.initialise(t, pose, keyframe.params(**kw))
    torch.cuda.synchronize()
    n = len(points)
    return {k: v[:n].cpu().numpy() for k, v in out.items() if k != "scratch"}


def _rot(q):
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                     np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                     np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)


def _compare(oi, points, pose, rows=None, **kw):
    got = _gpu(points, pose, **kw)
    P = oi.Params(**kw)
    want = oi.initialise(points, pose, P, rows=rows)
    rows = np.arange(len(points)) if rows is None else np.asarray(rows)
    g = {k: v[rows] for k, v in got.items()}
    assert np.array_equal(g["knn"], want["knn"])
    lam, wl = g["lam"].astype(np.float64), want["lam"]
    l0 = wl[:, :1]
    assert np.all(np.abs(lam - wl) <= 2e-6 * l0 + 1e-12)
    gap_n = (wl[:, 1] - wl[:, 2]) > 1e-3 * wl[:, 0]
    gap_t = (wl[:, 0] - wl[:, 1]) > 1e-3 * wl[:, 0]
    R = _rot(g["quat"].astype(np.float64))
    Rw = want["rot"]
    assert np.all((R[gap_n, :, 2] * Rw[gap_n, :, 2]).sum(1) >= 1 - 1e-5)
    assert np.all(np.abs((R[gap_n & gap_t, :, 0] * Rw[gap_n & gap_t, :, 0]).sum(1)) >= 1 - 1e-5)
    assert np.allclose(np.linalg.norm(g["quat"], axis=1), 1.0, atol=1e-6)
    assert np.all(g["quat"][:, 0] >= 0)
    pts = np.asarray(points, np.float64)[rows]
    assert np.all(np.abs(g["mean"] - want["mean"]) <= 1e-6 * (np.abs(want["mean"]) + 1.0))
    ls, wls = g["log_scale"].astype(np.float64), want["log_scale"]
    assert np.all(np.abs(ls[:, 0] - wls[:, 0]) <= 2e-6)
    ok1 = wl[:, 1] > 1e-6 * wl[:, 0]
    tol1 = 2e-6 * wl[ok1, 0] / wl[ok1, 1] + 1e-5
    assert np.all(np.abs(ls[ok1, 1] - wls[ok1, 1]) <= tol1)
    err_n = np.where(gap_n, 1e-5, 2.0)
    assert np.all(np.abs(g["u"] - want["u"]) <= err_n / (1 - P.c0) + 2e-6)
    alpha = 1 / (1 + np.exp(-g["logit"].astype(np.float64)))
    assert np.allclose(alpha, P.alpha_min + (P.alpha_max - P.alpha_min) * g["u"], atol=2e-6)
    return got, want, pts


@pytest.mark.parametrize("n,k", [(20, 20), (21, 20), (300, 20), (1000, 3), (2049, 32), (5000, 16)])
def test_random_clouds(oi, n, k):
    """Ragged sizes around the 256-point tile, k at its bounds; anisotropic
    clouds of several scales at several ranges."""
    rng = np.random.default_rng(n + k)
    c = rng.uniform(-40, 40, (8, 3)) + [0, 0, 0]
    pts = (c[rng.integers(0, 8, n)] + rng.normal(size=(n, 3)) * rng.uniform(0.05, 2.0, (n, 3))).astype(np.float32)
    _compare(oi, pts, np.eye(3, 4).ravel(), k=k)


def test_street_keyframe(oi):
    """A 64 x 1024 keyframe of the street (52k points, scan order) at a
    rotated and shifted pose: every neighbour set of 3,000 sampled points
    bit-exact, their frames within the tolerances."""
    pts, pose = scenes.keyframe_points(3, 64, 1024, t=(4.0, -1.0, 0.5))
    rows = np.random.default_rng(0).choice(len(pts), 3000, replace=False)
    rows.sort()
    _compare(oi, pts, pose, rows=rows)


def test_full_scan_sampled(oi):
    """A full 128 x 1024 scan (about 105k points): sampled rows against the
    oracle, and every row's neighbour list sorted, self-first and in range."""
    pts, pose = scenes.keyframe_points(5, 128, 1024)
    rows = np.random.default_rng(1).choice(len(pts), 1500, replace=False)
    got, _, _ = _compare(oi, pts, pose, rows=rows)
    knn = got["knn"]
    assert np.all((knn >= 0) & (knn < len(pts)))
    assert np.all(np.any(knn == np.arange(len(pts))[:, None], axis=1))   # each point among its own


def test_duplicates_and_degenerate(oi):
    """Coincident points (ties broken by index), a line, an exact plane
    facing the sensor, points inside 1 m."""
    rng = np.random.default_rng(9)
    dup = np.repeat(rng.normal(size=(30, 3)).astype(np.float32) * 5 + [10, 0, 0], 4, axis=0)
    line = np.stack([np.linspace(5, 6, 40), np.zeros(40), np.full(40, -1.0)], 1)
    yy, zz = np.meshgrid(np.arange(10) * 0.1, np.arange(8) * 0.1)
    plane = np.stack([np.full(yy.size, 20.0), yy.ravel(), zz.ravel()], 1)
    near = rng.normal(size=(50, 3)) * 0.2 + [0.5, 0.1, 0.0]
    pts = np.concatenate([dup, line, plane, near]).astype(np.float32)
    _compare(oi, pts, np.eye(3, 4).ravel(), k=12)


def test_surfels_render(oi):
    """The initialised surfels are a valid map: finite parameters, scales in
    [s_min, s_max], unit quaternions, opacity in [alpha_min, alpha_max]."""
    pts, pose = scenes.keyframe_points(7, 64, 512)
    g = _gpu(pts, pose)
    for key in ("mean", "quat", "log_scale", "logit", "lam", "u"):
        assert np.all(np.isfinite(g[key])), key
    s = np.exp(g["log_scale"].astype(np.float64))
    assert np.all(s >= 1e-3 * (1 - 1e-6)) and np.all(s <= 1.0 + 1e-6)
    a = 1 / (1 + np.exp(-g["logit"].astype(np.float64)))
    assert np.all(a >= 0.3 - 1e-6) and np.all(a <= 0.9 + 1e-6)
    assert np.all(g["lam"][:, 0] >= g["lam"][:, 1]) and np.all(g["lam"][:, 1] >= g["lam"][:, 2])
