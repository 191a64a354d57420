"""Pins of the map-management oracle (control score, Sec. 3.3 Eq. controlscore;
opacity prune, Table 4 baseline; planar cover-and-prune and adaptive split,
Sec. 3.5) against closed forms, library routines, hand-worked cases and an
independent brute-force restatement.  CPU only.

  M1 control score closed forms: line, plane, isotropic, residual saturation,
     eigenvalue order independence, range [0, 1]
  M2 lower quantile == numpy.quantile(method="lower") == sorted[floor(q(n-1))]
  M3 total-order key sorts like the values
  M4 quaternion axes == the rotation matrix the quaternion came from
  M5 one cover-and-prune group worked by hand (slab, non-candidates, lone
     voxels, opacity prune, cap order)
  M6 split worked by hand (axis, shift, log-scale, cap order, layout)
  M7 brute-force O(n^2) restatement == the oracle, bitwise, on tiny maps
  M8 invariants on a clustered map
"""
import math

import numpy as np
import pytest

from paper_2607_04127_gb300 import scenes

F = np.float32


@pytest.fixture(scope="module")
def mg(oracle):
    from oracle import manage
    return manage


def _lam(rows):
    return np.asarray(rows, F)


# --- M1 ------------------------------------------------------------------------
def test_control_score_closed_forms(mg):
    """line (4,1,0): lin = 3/4, curv = 0; isotropic (1,1,1): lin = 0,
    curv = 1/3 -> 1 after the x3 normalisation; plane (1,1,0): lin = curv = 0.
    Residuals (1, 0, 1, 1) normalised by their 0.95 quantile 1."""
    lam = _lam([[4, 1, 0], [1, 1, 1], [1, 1, 0], [2, 0, 0]])
    res = np.array([1, 0, 1, 1], F)
    c = mg.control_score(lam, res).astype(np.float64)
    assert c[0] == pytest.approx(0.55 * 0.75 + 0.15 * 1.0, abs=2e-6)
    assert c[1] == pytest.approx(0.30 * 1.0 + 0.15 * 0.0, abs=2e-6)
    assert c[2] == pytest.approx(0.15, abs=2e-6)
    assert c[3] == pytest.approx(0.55 + 0.15, abs=2e-6)


def test_control_score_residual_saturates_and_orders(mg):
    """res~ = min(res / Q_0.95(res), 1): residuals 0..99 have Q_0.95 = 94
    (index floor(0.95 * 99) = 94), so a plane's score is 0.15 min(r/94, 1)."""
    n = 100
    lam = np.tile(_lam([[1, 1, 0]]), (n, 1))
    res = np.arange(n, dtype=F)
    c = mg.control_score(lam, res).astype(np.float64)
    want = 0.15 * np.minimum(np.arange(n) / 94.0, 1.0)
    assert np.allclose(c, want, atol=2e-6)
    assert np.all(c[94:] == c[94])


def test_control_score_eigenvalue_order_and_range(mg):
    rng = np.random.default_rng(3)
    lam = rng.uniform(0, 2, (500, 3)).astype(F)
    res = rng.exponential(1.0, 500).astype(F)
    c = mg.control_score(lam, res)
    for perm in ([2, 1, 0], [1, 0, 2], [0, 2, 1]):
        assert np.array_equal(mg.control_score(lam[:, perm], res), c)
    assert c.dtype == np.float32 and np.all(c >= 0) and np.all(c <= 1)


# --- M2, M3 --------------------------------------------------------------------
@pytest.mark.parametrize("q", [0.0, 0.3, 0.5, 0.9, 0.95, 1.0])
def test_quantile_lower_matches_numpy(mg, q):
    rng = np.random.default_rng(int(q * 100))
    for n in (1, 2, 7, 50, 257):
        x = rng.normal(size=n).astype(F)
        got = mg.quantile_lower(x, q)
        assert got == np.quantile(x, float(F(q)), method="lower")
        assert got == np.sort(x)[math.floor(float(F(q)) * (n - 1))]
    assert mg.quantile_lower(np.zeros(0, F), q) is None


def test_order_key_sorts_like_values(mg):
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.normal(size=300) * 10 ** rng.uniform(-30, 30, 300),
                        [0.0, np.inf, -np.inf, 1e-45, -1e-45]]).astype(F)
    k = mg.order_key(x)
    assert np.array_equal(x[np.argsort(k)], np.sort(x))
    assert mg.order_key(np.array([-0.0], F))[0] < mg.order_key(np.array([0.0], F))[0]


# --- M4 ------------------------------------------------------------------------
def test_quat_axes_are_the_rotation_columns(mg):
    rng = np.random.default_rng(7)
    n = 200
    t0 = rng.normal(size=(n, 3)); nrm = rng.normal(size=(n, 3))
    R = scenes.frames_from_axes(t0, nrm)
    q = scenes.rot_to_quat(R).astype(F)
    for scale in (1.0, 3.0):
        tu, tv, nn = mg.quat_axes(q * F(scale))
        assert np.allclose(tu, R[:, :, 0], atol=2e-6)
        assert np.allclose(tv, R[:, :, 1], atol=2e-6)
        assert np.allclose(nn, R[:, :, 2], atol=2e-6)
    tu, tv, nn = mg.quat_axes(np.array([[1, 0, 0, 0]], F))
    assert tu.tolist() == [[1, 0, 0]] and tv.tolist() == [[0, 1, 0]] and nn.tolist() == [[0, 0, 1]]
    h = F(math.sqrt(0.5))
    tu, tv, nn = mg.quat_axes(np.array([[h, 0, 0, h]], F))   # 90 degrees about z
    assert np.allclose(tu, [[0, 1, 0]], atol=3e-7) and np.allclose(tv, [[-1, 0, 0]], atol=3e-7)
    assert np.allclose(nn, [[0, 0, 1]], atol=3e-7)


# --- M5 ------------------------------------------------------------------------
def _hand_map():
    """Nine surfels, identity orientation (tangent axes x, y; normal z),
    scales 0.1 m.  Voxel (0, 0) of the xy plane holds 0..6 and 8:
      0 (0.1, 0.1, 0)   logit 2  -> the representative (largest alpha)
      1 (0.2, 0.1, 0)   u = 1, v = 0          -> r^2 = 1
      2 (0.4, 0.1, 0)   u = 3                 -> r^2 = 9
      3 (0.7, 0.1, 0)   u = 6                 -> r^2 = 36
      4 (0.9, 0.9, 0)   u = v = 8             -> r^2 = 128
      5 (0.3, 0.3, 0.5) h = 0.5 > slab        -> not a member
      6 (0.5, 0.5, 0)   a line (lambda = (1,0,0)): c = 0.55, not a candidate
      8 (0.6, 0.6, 0)   alpha = sigmoid(-6) < 0.005 -> opacity-pruned
    and 7 (1.5, 0.1, 0) is alone in voxel (1, 0)."""
    mean = np.array([[.1, .1, 0], [.2, .1, 0], [.4, .1, 0], [.7, .1, 0], [.9, .9, 0],
                     [.3, .3, .5], [.5, .5, 0], [1.5, .1, 0], [.6, .6, 0]], F)
    n = mean.shape[0]
    quat = np.tile(np.array([1, 0, 0, 0], F), (n, 1))
    ls = np.full((n, 2), math.log(0.1), F)
    logit = np.array([2, 1, 1, 1, 1, 1, 1, 1, -6], F)
    lam = np.tile(_lam([[1, 1, 0]]), (n, 1))
    lam[6] = [1, 0, 0]
    res = np.zeros(n, F)
    return mean, quat, ls, logit, lam, res


def test_cover_prune_by_hand(mg):
    mean, quat, ls, logit, lam, res = _hand_map()
    P = mg.Params(n_passes=1, q_cover=0.5, prune_cap=0.5, q_split=1.0, split_cap=0.0)
    # scales are the oracle's exp(log 0.1), within 1e-6 of 0.1: r^2 as listed
    out = mg.manage(mean, quat, ls, logit, lam, res, P)
    # m = 4 members (1, 2, 3, 4), k = ceil(0.5 * 4) = 2: the two closest go
    assert out["counts"].tolist() == [6, 1, 2, 0, 0, 0]
    assert out["src"].tolist() == [0, 3, 4, 5, 6, 7]
    assert np.array_equal(out["mean"], mean[[0, 3, 4, 5, 6, 7]])
    # q_cover = 1 covers all four; a cap of floor(0.5 * 8) = 4 lets them go
    out = mg.manage(mean, quat, ls, logit, lam, res, mg.Params(n_passes=1, q_cover=1.0, prune_cap=0.5,
                                                              q_split=1.0, split_cap=0.0))
    assert out["src"].tolist() == [0, 5, 6, 7]
    # a slab of 0.6 admits 5 (r^2 = 8): k = ceil(0.5 * 5) = 3 -> 1, 5, 2
    out = mg.manage(mean, quat, ls, logit, lam, res, mg.Params(n_passes=1, q_cover=0.5, slab=0.6,
                                                              prune_cap=0.5, q_split=1.0, split_cap=0.0))
    assert out["src"].tolist() == [0, 3, 4, 6, 7]


def test_cover_prune_cap_takes_the_most_planar_first(mg):
    """Residual 1 on surfels 1 and 2 (Q_0.95 of the residuals is then 1) gives
    them c = 0.15 while the other planes have c = 0; with q_plane = 0.8 they
    stay candidates (Q_0.8 of the survivors' c = 0.15).  All four members
    are covered (q_cover = 1) but the cap floor(0.25 * 8) = 2 keeps the two
    of lowest c: 3 and 4 go, 1 and 2 stay."""
    mean, quat, ls, logit, lam, res = _hand_map()
    res[[1, 2]] = 1
    P = mg.Params(n_passes=1, q_plane=0.8, q_cover=1.0, prune_cap=0.25, q_split=1.0, split_cap=0.0)
    out = mg.manage(mean, quat, ls, logit, lam, res, P)
    assert out["counts"].tolist() == [6, 1, 2, 0, 0, 0]
    assert out["src"].tolist() == [0, 1, 2, 5, 6, 7]


# --- M6 ------------------------------------------------------------------------
def test_split_by_hand(mg):
    """Zero residuals; surfel 3 a line (lambda (1, 0, 0): c = 0.55), 0 and 4
    lambda (1, 0.2, 0) (lin = 0.8: c = 0.44), 1 and 2 planes (c = 0).
    q_split = 0 makes every survivor with alpha >= alpha_min a candidate; the
    cap floor(0.4 * 5) = 2 keeps the two largest scores: 3, then 0 (the tie
    of 0 and 4 broken by index).  Surfel 3 is turned 90 degrees about z, so
    its children sit at mu +- 0.5 * 0.2 * (0, 1, 0)."""
    h = math.sqrt(0.5)
    mean = np.array([[1, 2, 3], [4, 5, 6], [7, 8, 9], [10, 11, 12], [13, 14, 15]], F)
    quat = np.array([[1, 0, 0, 0]] * 3 + [[h, 0, 0, h], [1, 0, 0, 0]], F)
    ls = np.array([[math.log(0.2), math.log(0.1)]] * 5, F)
    logit = np.array([1, 1, 1, 1, 1], F)
    lam = _lam([[1, 0.2, 0], [1, 1, 0], [1, 1, 0], [1, 0, 0], [1, 0.2, 0]])
    res = np.zeros(5, F)
    P = mg.Params(n_passes=0, q_split=0.0, split_cap=0.4, alpha_min=0.1)
    out = mg.manage(mean, quat, ls, logit, lam, res, P)
    assert out["counts"].tolist() == [7, 0, 0, 0, 0, 2]
    assert out["src"].tolist() == [0, 0, 1, 2, 3, 3, 4]
    assert out["role"].tolist() == [1, 2, 0, 0, 1, 2, 0]
    m = out["mean"].astype(np.float64)
    assert np.allclose(m[4], [10, 11.1, 12], atol=2e-6) and np.allclose(m[5], [10, 10.9, 12], atol=2e-6)
    assert np.allclose(m[0], [1.1, 2, 3], atol=2e-6) and np.allclose(m[1], [0.9, 2, 3], atol=2e-6)
    assert np.allclose(0.5 * (m[4] + m[5]), mean[3], atol=1e-6)
    ols = out["log_scale"].astype(np.float64)
    assert ols[0, 0] == pytest.approx(math.log(0.1), abs=1e-6) and ols[0, 1] == pytest.approx(math.log(0.1))
    assert np.array_equal(out["log_scale"][2], ls[1]) and np.array_equal(out["quat"][4], quat[3])
    assert np.array_equal(out["logit"], logit[out["src"]])


# --- M7 ------------------------------------------------------------------------
def _brute(mean, quat, ls, logit, lam, res, P, mg, oracle):
    """The same definition restated element by element: pairwise voxel
    comparison instead of grouping, a scan for the representative, Python
    sorts of tuples for quantiles and caps."""
    n = len(logit)
    c = mg.control_score(lam, res, P)          # pinned on its own (M1)
    f = F
    lt_p = mg.logit_threshold(P.alpha_prune); lt_m = mg.logit_threshold(P.alpha_min)
    alive = [bool(logit[i] >= lt_p) for i in range(n)]

    def q_lower(vals, q):
        s = sorted(vals, key=lambda v: (int(mg.order_key(np.array([v], F))[0])))
        return s[math.floor(float(F(q)) * (len(s) - 1))]

    def axes(i):
        w, x, y, z = (f(v) for v in quat[i])
        r = np.sqrt(f(f(f(w * w) + f(x * x)) + f(y * y)) + f(z * z))
        w, x, y, z = w / r, x / r, y / r, z / r
        tu = (f(1) - f(2) * (y * y + z * z), f(2) * (x * y + w * z), f(2) * (x * z - w * y))
        tv = (f(2) * (x * y - w * z), f(1) - f(2) * (x * x + z * z), f(2) * (y * z + w * x))
        nn = (f(2) * (x * z + w * y), f(2) * (y * z - w * x), f(1) - f(2) * (x * x + y * y))
        return tu, tv, nn

    def dot(a, b):
        return f(f(a[0] * b[0]) + f(a[1] * b[1])) + f(a[2] * b[2])

    def vox(v):
        return int(min(max(math.floor(f(v) / f(P.voxel)), -2 ** 30), 2 ** 30))

    for p in range(P.n_passes):
        a, b = ((0, 1), (1, 2), (2, 0))[p]     # planes xy, yz, zx
        live = [i for i in range(n) if alive[i]]
        if not live:
            continue
        qp = q_lower([c[i] for i in live], P.q_plane)
        cand = [i for i in live if c[i] <= qp and logit[i] >= lt_m]
        flagged = []
        for j in cand:
            mates = [k for k in cand if vox(mean[k][a]) == vox(mean[j][a]) and vox(mean[k][b]) == vox(mean[j][b])]
            r = mates[0]
            for k in mates:
                if mg.order_key(np.array([logit[k]], F))[0] > mg.order_key(np.array([logit[r]], F))[0]:
                    r = k
            if j == r:
                continue
            tu, tv, nn = axes(r)
            s = oracle.f32_exp_spec_n(np.asarray(ls[r], F))

            def meas(k):
                d = [f(mean[k][t] - mean[r][t]) for t in range(3)]
                u = dot(tu, d) / s[0]; v = dot(tv, d) / s[1]
                return abs(dot(nn, d)) <= f(P.slab), f(f(u * u) + f(v * v))
            inside, r2 = meas(j)
            if not inside:
                continue
            members = [meas(k)[1] for k in mates if k != r and meas(k)[0]]
            kk = math.ceil(float(F(P.q_cover)) * len(members))
            if sum(1 for m2 in members if m2.view(np.uint32) < r2.view(np.uint32)) < kk:
                flagged.append(j)
        cap = math.floor(float(F(P.prune_cap)) * len(live))
        flagged.sort(key=lambda i: (int(mg.order_key(np.array([c[i]], F))[0]), i))
        for i in flagged[:cap]:
            alive[i] = False
    live = [i for i in range(n) if alive[i]]
    split = set()
    if live:
        qs = q_lower([c[i] for i in live], P.q_split)
        cand = [i for i in live if c[i] >= qs and logit[i] >= lt_m]
        cand.sort(key=lambda i: (-int(mg.order_key(np.array([c[i]], F))[0]), i))
        split = set(cand[:math.floor(float(F(P.split_cap)) * len(live))])
    src = []
    for i in live:
        src += [i, i] if i in split else [i]
    return src


_clustered = scenes.manage_cluster


@pytest.mark.parametrize("seed,n", [(0, 40), (1, 90), (2, 150)])
def test_manage_equals_brute_force(mg, oracle, seed, n):
    mean, quat, ls, logit, lam, res = _clustered(seed, n)
    P = mg.Params(voxel=0.8, q_plane=0.6, q_cover=0.6, slab=0.05, prune_cap=0.3, q_split=0.8, split_cap=0.1)
    out = mg.manage(mean, quat, ls, logit, lam, res, P)
    assert out["src"].tolist() == _brute(mean, quat, ls, logit, lam, res, P, mg, oracle)
    assert out["counts"][2:5].sum() > 0 and out["counts"][5] > 0


@pytest.mark.parametrize("kw", [
    dict(voxel=0.3, q_plane=0.9, q_cover=0.5, slab=0.5, prune_cap=1.0, q_split=0.5, split_cap=1.0),   # no caps
    dict(voxel=2.5, q_plane=1.0, q_cover=1.0, slab=10.0, prune_cap=0.5, q_split=0.95, split_cap=0.02),
    dict(voxel=1.0, n_passes=2, q_plane=0.4, q_cover=0.3, slab=0.02, prune_cap=0.0, q_split=0.0, split_cap=0.05),
])
def test_manage_equals_brute_force_other_parameters(mg, oracle, kw):
    mean, quat, ls, logit, lam, res = _clustered(5, 120)
    P = mg.Params(**kw)
    out = mg.manage(mean, quat, ls, logit, lam, res, P)
    assert out["src"].tolist() == _brute(mean, quat, ls, logit, lam, res, P, mg, oracle)


# --- M8 ------------------------------------------------------------------------
def test_manage_invariants(mg):
    mean, quat, ls, logit, lam, res = _clustered(11, 3000)
    P = mg.Params(voxel=0.5, q_plane=0.5, q_cover=0.7, prune_cap=0.05, q_split=0.9, split_cap=0.02)
    out = mg.manage(mean, quat, ls, logit, lam, res, P)
    n = len(logit)
    cnt = out["counts"]
    src, role = out["src"], out["role"]
    assert cnt[0] == n - cnt[1:5].sum() + cnt[5] == src.size
    alive = logit >= mg.logit_threshold(P.alpha_prune)
    assert cnt[1] == n - alive.sum()
    na = alive.sum()
    for k in range(3):
        assert 0 < cnt[2 + k] <= math.floor(float(F(P.prune_cap)) * na)
        na -= cnt[2 + k]
    assert 0 < cnt[5] <= math.floor(float(F(P.split_cap)) * na)
    assert np.all(np.diff(src) >= 0)
    u, k = np.unique(src, return_counts=True)
    assert np.array_equal(k == 2, np.isin(u, src[role == 1]))
    assert np.all(role[::1][np.r_[np.diff(src) == 0, False]] == 1)
    c = out["score"]
    assert np.all(c[src[role == 1]] >= np.quantile(c[u], float(F(P.q_split)), method="lower"))
    assert np.array_equal(out["quat"], quat[src]) and np.array_equal(out["logit"], logit[src])
    keep = role == 0
    assert np.array_equal(out["mean"][keep], mean[src[keep]])
    assert np.array_equal(out["log_scale"][keep], ls[src[keep]])


def test_manage_empty_and_single(mg):
    z = np.zeros((0, 3), F)
    out = mg.manage(z, np.zeros((0, 4), F), np.zeros((0, 2), F), np.zeros(0, F), z, np.zeros(0, F))
    assert out["counts"].tolist() == [0] * 6 and out["src"].size == 0
    out = mg.manage(np.ones((1, 3), F), np.array([[1, 0, 0, 0]], F), np.zeros((1, 2), F), np.ones(1, F),
                    np.array([[1, 0, 0]], F), np.ones(1, F), mg.Params(split_cap=1.0))
    # one survivor: Q_q is its own score; split cap floor(1 * 1) = 1
    assert out["counts"].tolist() == [2, 0, 0, 0, 0, 1] and out["role"].tolist() == [1, 2]


def test_far_voxels_clip_to_the_last_index(mg):
    """Voxel indices are clipped to [-2^30, 2^30]: two surfels 1e12 m and 2e12
    m out on the x axis share the last voxel, so with q_cover = 1 and no cap
    the one of lower alpha is covered by the other."""
    mean = np.array([[1e12, 0.1, 0], [2e12, 0.1, 0]], F)
    quat = np.tile(np.array([1, 0, 0, 0], F), (2, 1))
    ls = np.zeros((2, 2), F)
    logit = np.array([1, 2], F)
    lam = np.tile(_lam([[1, 1, 0]]), (2, 1))
    P = mg.Params(n_passes=1, q_plane=1.0, q_cover=1.0, prune_cap=1.0, q_split=1.0, split_cap=0.0)
    out = mg.manage(mean, quat, ls, logit, lam, np.zeros(2, F), P)
    assert out["src"].tolist() == [1] and out["counts"].tolist() == [1, 0, 1, 0, 0, 0]
