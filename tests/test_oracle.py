"""Pins of the FP64 CPU oracle against what the paper's definitions and plain
mathematics fix (closed forms, invariants, brute force, finite differences),
so that a mistake in the oracle fails here before it is used to check the
CUDA path.  CPU only.

Definitions pinned (paper Sec. 3.1 map representation, Sec. 3.4 map
optimisation, Eqs. depthloss / normalloss / scaleloss / totalloss):
  P1 single surfel facing the ray: plane-intersection depth, A = alpha G
  P2 coaxial stack: A = 1 - prod(1 - a), T = prod(1 - a), truncation at 1e-4
  P3 tiled == brute-force all-pairs (bitwise) and no valid pair is un-binned
  P4 sorted lists: key order, index tie-break, ranges, counts
  P5 90-degree rotation about z == column shift by W/4 (azimuth seam)
  P6 analytic gradient == central finite differences (steps 1e-6 and 1e-4)
  P7 special-case derivatives of P1
  P8 loss closed forms and mask invariances
  P9 the N_surf term: plane closed form (orientation, masks, azimuth wrap,
     mean over Omega_D), column-shift invariance, finite differences
and the binary32 polynomial exp / sin / cos used by binning.
"""
import math

import numpy as np
import pytest

from paper_2607_04127_gb300 import scenes

EPS = 1e-6


def pixel_dir(frame, r, c):
    """Unit ray of pixel (r, c) by the pixel-grid definition (sensor frame)."""
    emin, emax = float(np.float32(frame.elev_min)), float(np.float32(frame.elev_max))
    th = emax - (r + 0.5) * (emax - emin) / frame.H
    ph = (c + 0.5) * 2 * math.pi / frame.W
    return np.array([math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), math.sin(th)])


def facing_surfels(specs):
    """Surfels with normal -d facing the sensor at identity pose.
    specs: list of (d, range, alpha, s_u, s_v, offset_u)."""
    means, quats, ls, lg = [], [], [], []
    for d, rho, alpha, su, sv, off in specs:
        n = -d
        t0 = np.cross(d, [0.0, 0.0, 1.0])
        if np.linalg.norm(t0) < 1e-6:
            t0 = np.cross(d, [1.0, 0.0, 0.0])
        Rm = scenes.frames_from_axes(t0[None], n[None])[0]
        tu = Rm[:, 0]
        means.append(rho * d + off * tu)
        quats.append(scenes.rot_to_quat(Rm[None])[0])
        ls.append([math.log(su), math.log(sv)])
        lg.append(math.log(alpha / (1 - alpha)))
    f = np.float32
    return scenes.Surfels(np.array(means, f), np.array(quats, f), np.array(ls, f), np.array(lg, f))


def sigmoid(x):
    return 1.0 / (1.0 + math.exp(-x))


FRAME = scenes.Frame(32, 64, 16, 16, -math.radians(30), math.radians(30))


# --------------------------------------------------------------------------
# binary32 polynomials of the binning definition
# --------------------------------------------------------------------------
def test_spec_exp_accuracy(oracle):
    for x in np.linspace(-20.0, 5.0, 2001):
        x32 = float(np.float32(x))
        assert abs(float(oracle.f32_exp_spec(x32)) / math.exp(x32) - 1.0) < 1e-6


def test_spec_sin_cos_accuracy(oracle):
    for x in np.linspace(-math.pi / 2, math.pi / 2, 2001):
        x32 = float(np.float32(x))
        assert abs(float(oracle.f32_sin_spec(x32)) - math.sin(x32)) < 3e-7
        assert abs(float(oracle.f32_cos_spec(x32)) - math.cos(x32)) < 3e-7


@pytest.mark.parametrize("W", [64, 512, 1000, 1024, 2048])
def test_spec_column_directions(oracle, W):
    for c in range(0, W, max(1, W // 97)):
        cs, sn = oracle.f32_col_dir(c, W)
        ph = (c + 0.5) * 2 * math.pi / W
        assert abs(float(cs) - math.cos(ph)) < 5e-7 and abs(float(sn) - math.sin(ph)) < 5e-7


# --------------------------------------------------------------------------
# P1: single surfel facing the ray
# --------------------------------------------------------------------------
def _run(oracle, surf, frame):
    b = oracle.bin_frame(surf, frame)
    fw = oracle.render_fwd(surf, frame, b["ranges"], b["vals"])
    return b, fw


@pytest.mark.parametrize("rho,alpha,su", [(5.0, 0.6, 0.3), (12.5, 0.9, 0.8), (2.0, 0.35, 0.1)])
def test_p1_facing_surfel_centre(oracle, rho, alpha, su):
    r, c = 13, 21
    d = pixel_dir(FRAME, r, c)
    surf = facing_surfels([(d, rho, alpha, su, su * 0.7, 0.0)])
    _, fw = _run(oracle, surf, FRAME)
    a = sigmoid(float(surf.logit[0]))
    assert fw["S_t"][r, c] / fw["A"][r, c] == pytest.approx(rho, rel=1e-7)   # t = |mu| exactly
    assert fw["A"][r, c] == pytest.approx(a, rel=1e-10)
    Dh = fw["S_t"][r, c] / (fw["A"][r, c] + EPS)
    assert Dh == pytest.approx(rho * a / (a + EPS), rel=1e-7)
    N = fw["S_n"][:, r, c] / np.linalg.norm(fw["S_n"][:, r, c])
    assert np.allclose(N, -d, atol=1e-6)
    assert fw["T_final"][r, c] == pytest.approx(1 - a, rel=1e-10)
    assert fw["n_contrib"][r, c] == 1


@pytest.mark.parametrize("off_sigma", [0.5, 1.2, 2.5])
def test_p1_facing_surfel_offset(oracle, off_sigma):
    """Centre shifted by delta along t_u inside the plane: the ray meets the
    plane at u = -delta/s_u, v = 0, so A = alpha exp(-delta^2 / (2 s_u^2))."""
    r, c = 9, 40
    d = pixel_dir(FRAME, r, c)
    su = 0.4
    surf = facing_surfels([(d, 8.0, 0.8, su, 0.5, off_sigma * su)])
    _, fw = _run(oracle, surf, FRAME)
    a = sigmoid(float(surf.logit[0]))
    s_u = math.exp(float(surf.log_scale[0, 0]))
    # the FP32 inputs round the offset; recompute it from the stored centre
    delta = np.linalg.norm(surf.mean[0].astype(np.float64) - 8.0 * d)
    assert fw["A"][r, c] == pytest.approx(a * math.exp(-0.5 * (delta / s_u) ** 2), rel=1e-6)


# --------------------------------------------------------------------------
# P2: coaxial stack
# --------------------------------------------------------------------------
def test_p2_coaxial_stack(oracle):
    r, c = 20, 5
    d = pixel_dir(FRAME, r, c)
    alpha = 0.7
    ranges = [3.0 + i for i in range(8)]
    surf = facing_surfels([(d, rho, alpha, 0.3, 0.3, 0.0) for rho in ranges])
    _, fw = _run(oracle, surf, FRAME)
    a = sigmoid(float(surf.logit[0]))
    # (1-a)^8 < 1e-4 <= (1-a)^7: seven contributors, the eighth stops the ray
    assert (1 - a) ** 8 < 1e-4 <= (1 - a) ** 7
    T = np.cumprod([1.0] + [1 - a] * 7)
    assert fw["n_contrib"][r, c] == 7
    assert fw["T_final"][r, c] == pytest.approx((1 - a) ** 7, rel=1e-9)
    assert fw["A"][r, c] == pytest.approx(1 - (1 - a) ** 7, rel=1e-9)
    St = sum(a * T[i] * ranges[i] for i in range(7))
    assert fw["S_t"][r, c] == pytest.approx(St, rel=1e-7)


def test_p2_transmittance_is_product(oracle):
    """Random stack of opacities: T_final = prod(1 - a_i), A = 1 - T_final."""
    rng = np.random.default_rng(3)
    r, c = 16, 33
    d = pixel_dir(FRAME, r, c)
    al = rng.uniform(0.05, 0.5, 6)
    surf = facing_surfels([(d, 4.0 + i, float(x), 0.5, 0.5, 0.0) for i, x in enumerate(al)])
    _, fw = _run(oracle, surf, FRAME)
    a = np.array([sigmoid(float(x)) for x in surf.logit])
    assert fw["T_final"][r, c] == pytest.approx(np.prod(1 - a), rel=1e-9)
    assert fw["A"][r, c] == pytest.approx(1 - np.prod(1 - a), rel=1e-9)


# --------------------------------------------------------------------------
# P3: tiled == brute force; binning conservative
# --------------------------------------------------------------------------
def _scenes_small():
    out = []
    s, f, _ = scenes.box_room()
    out.append(("box_room", s, f))
    s, f = scenes.random_shell(1, 400, frame=scenes.Frame(32, 64, 16, 16, -0.5, 0.5))
    out.append(("shell64", s, f))
    s, f = scenes.random_shell(2, 1500, frame=scenes.Frame(32, 512, 8, 8, -0.6, 0.3, scenes.pose_matrix(0.7)))
    out.append(("shell512", s, f))
    # near the sensor and near the poles: spheres containing the sensor or a pole
    s, f = scenes.random_shell(4, 300, r_range=(0.3, 4.0), scale_range=(0.05, 1.5),
                               frame=scenes.Frame(40, 72, 8, 8, -1.4, 1.4))
    out.append(("near_poles", s, f))
    # ragged tiles (H, W not multiples of the tile)
    s, f = scenes.random_shell(5, 500, frame=scenes.Frame(37, 100, 16, 16, -0.4, 0.4))
    out.append(("ragged", s, f))
    return out


@pytest.mark.parametrize("name,surf,frame", _scenes_small(), ids=lambda x: x if isinstance(x, str) else "")
def test_p3_tiled_equals_brute_force(oracle, name, surf, frame):
    b = oracle.bin_frame(surf, frame)
    fw = oracle.render_fwd(surf, frame, b["ranges"], b["vals"])
    r, v = oracle.brute_lists(surf, frame)
    fb = oracle.render_fwd(surf, frame, r, v)
    for k in ("A", "S_t", "S_n", "T_final", "n_valid"):
        assert np.array_equal(fw[k], fb[k]), k
    assert oracle.coverage_misses(surf, frame, b["ranges"], b["vals"]) == 0
    assert fw["A"].max() > 0.1   # the scene is actually seen


# --------------------------------------------------------------------------
# P4: sorted lists
# --------------------------------------------------------------------------
def test_p4_sorted_lists(oracle):
    surf, frame, _ = scenes.box_room()
    b = oracle.bin_frame(surf, frame)
    keys, vals, ranges = b["keys"], b["vals"], b["ranges"]
    assert len(keys) == b["n_pairs"] == int(b["count"].sum())
    # ascending (key, index)
    assert np.all((keys[1:] > keys[:-1]) | ((keys[1:] == keys[:-1]) & (vals[1:] > vals[:-1])))
    # low word = depth key of the listed surfel, high word = its tile
    assert np.array_equal((keys & 0xFFFFFFFF).astype(np.uint32), b["depth_bits"][vals])
    tiles = (keys >> 32).astype(np.int64)
    for t in range(ranges.shape[0]):
        s, e = ranges[t]
        assert np.all(tiles[s:e] == t)
    assert np.array_equal(np.bincount(vals, minlength=surf.n), b["count"])
    # the depth key orders like the value it encodes
    dv = b["depth_bits"].view(np.float32)
    o1 = np.argsort(dv, kind="stable"); o2 = np.argsort(b["depth_bits"], kind="stable")
    assert np.array_equal(o1, o2)


# --------------------------------------------------------------------------
# P5: azimuth seam / rotation invariance
# --------------------------------------------------------------------------
def test_p5_rotation_about_z_shifts_columns(oracle):
    surf, _ = scenes.random_shell(7, 800, frame=scenes.Frame(32, 64, 16, 16, -0.5, 0.5))
    f0 = scenes.Frame(32, 64, 16, 16, -0.5, 0.5)
    rot = np.array([0, -1, 0, 0, 1, 0, 0, 0, 0, 0, 1, 0], np.float32)  # R_z(90 deg), exact
    f1 = scenes.Frame(32, 64, 16, 16, -0.5, 0.5, rot)
    _, a = _run(oracle, surf, f0)
    _, b = _run(oracle, surf, f1)
    sh = 64 // 4
    for k in ("A", "S_t", "T_final"):
        assert np.allclose(b[k], np.roll(a[k], -sh, axis=1), rtol=1e-12, atol=1e-12), k


def test_p5_seam_surfel_in_first_and_last_column(oracle):
    frame = scenes.Frame(32, 64, 16, 16, -0.5, 0.5)
    d = np.array([1.0, 0.0, 0.0])                     # azimuth exactly 0
    surf = facing_surfels([(d, 6.0, 0.8, 0.3, 0.3, 0.0)])
    b = oracle.bin_frame(surf, frame)
    cols = {int(k >> 32) % 4 for k in b["keys"]}
    assert 0 in cols and 3 in cols
    _, fw = _run(oracle, surf, frame)
    assert fw["A"][:, 0].max() > 0.1 and fw["A"][:, -1].max() > 0.1


# --------------------------------------------------------------------------
# P6: analytic gradient vs central differences
# --------------------------------------------------------------------------
def _fd_scene():
    frame = scenes.Frame(16, 64, 16, 16, -0.5, 0.5, scenes.pose_matrix(0.3, (0.1, -0.2, 0.05)))
    surf, _ = scenes.random_shell(11, 60, r_range=(2.0, 6.0), scale_range=(0.2, 0.9), frame=frame)
    surf.log_scale[:4, 0] = math.log(1.4)            # exercise the scale regulariser
    tgt = scenes.targets_for(frame, surf, seed=2)
    return surf, frame, tgt


def _loss64(oracle, surf, frame, tgt, p64):
    L, fw, g, _ = oracle.forward_backward(surf, [frame], [(tgt.D, tgt.N)], params64=p64)
    return L, fw[0], g


@pytest.mark.parametrize("h,rtol", [(1e-6, 2e-5), (1e-4, 1e-3)])
def test_p6_gradient_matches_central_differences(oracle, h, rtol):
    surf, frame, tgt = _fd_scene()
    base = [np.ascontiguousarray(a, np.float64).copy() for a in
            (surf.mean, surf.quat, surf.log_scale, surf.logit)]
    L0, fw0, g = _loss64(oracle, surf, frame, tgt, base)
    gl = [g["mean"], g["quat"], g["log_scale"], g["logit"]]
    rng = np.random.default_rng(0)
    used = skipped = 0
    for _ in range(60):
        which = int(rng.integers(4))
        idx = tuple(int(rng.integers(s)) for s in base[which].shape)
        vals = []
        same = True
        for sgn in (1, -1):
            p = [a.copy() for a in base]
            p[which][idx] += sgn * h
            L, fw, _ = _loss64(oracle, surf, frame, tgt, p)
            vals.append(L)
            same &= np.array_equal(fw["n_valid"], fw0["n_valid"]) and np.array_equal(fw["n_contrib"], fw0["n_contrib"])
        if not same:
            skipped += 1
            continue
        fd = (vals[0] - vals[1]) / (2 * h)
        an = gl[which][idx]
        scale = max(abs(fd), 1e-3 * max(np.abs(x).max() for x in gl))
        assert abs(an - fd) <= rtol * scale + 1e-9, (which, idx, an, fd)
        used += 1
    assert used >= 40, (used, skipped)


# --------------------------------------------------------------------------
# P7: special-case derivatives of the facing surfel
# --------------------------------------------------------------------------
def test_p7_special_derivatives(oracle):
    frame = FRAME
    r, c = 13, 21
    d = pixel_dir(frame, r, c)
    surf = facing_surfels([(d, 7.0, 0.6, 0.3, 0.2, 0.0)])
    b, fw = _run(oracle, surf, frame)
    a = sigmoid(float(surf.logit[0]))
    H, W = frame.H, frame.W
    gA = np.zeros((H, W)); gSt = np.zeros((H, W)); gSn = np.zeros((3, H, W))
    gA[r, c] = 1.0
    g = oracle.render_bwd(surf, frame, b["ranges"], b["vals"], gA, gSt, gSn)
    assert g["logit"][0] == pytest.approx(a * (1 - a), rel=1e-9)        # dA/dlogit = alpha (1 - alpha)
    # gradient of D = S_t/(A+eps) at the pixel w.r.t. the centre: (a/(a+eps)) n/(n.d) = (a/(a+eps)) d
    A, St = fw["A"][r, c], fw["S_t"][r, c]
    gA[r, c] = -St / (A + EPS) ** 2
    gSt[r, c] = 1.0 / (A + EPS)
    g = oracle.render_bwd(surf, frame, b["ranges"], b["vals"], gA, gSt, gSn)
    assert np.allclose(g["mean"][0], a / (a + EPS) * d, rtol=1e-6, atol=1e-9)


# --------------------------------------------------------------------------
# P8: losses
# --------------------------------------------------------------------------
def _planes(H=3, W=5, seed=0):
    rng = np.random.default_rng(seed)
    D = rng.uniform(2, 20, (H, W)).astype(np.float32)
    D[0, 1] = 0.0
    D[2, 3] = 0.0
    N = rng.normal(size=(3, H, W))
    N /= np.linalg.norm(N, axis=0)
    N[:, 1, 1] = 0.0
    return D, N.astype(np.float32)


def test_p8_depth_term_is_uniform_offset(oracle):
    D, N = _planes()
    A = np.full(D.shape, 0.8)
    for delta in (0.0, 0.37, -1.25):
        St = (D.astype(np.float64) + delta) * (A + EPS)
        Sn = np.array(N, np.float64) * 5.0
        _, _, terms = oracle.loss_image(dict(A=A, S_t=St, S_n=Sn), D, N)
        assert terms[0] == pytest.approx(abs(delta), abs=1e-12)


def test_p8_alpha_and_normal_terms(oracle):
    D, N = _planes()
    k = 0.9
    A = np.full(D.shape, math.exp(-k) - EPS)
    St = D.astype(np.float64) * (A + EPS)
    theta = 0.4
    # S_n at angle theta from N_gicp inside the plane of N and a perpendicular
    perp = np.cross(N.transpose(1, 2, 0), [0.3, -0.5, 0.8]).transpose(2, 0, 1)
    perp /= np.maximum(np.linalg.norm(perp, axis=0), 1e-30)
    Sn = 7.0 * (math.cos(theta) * N + math.sin(theta) * perp)
    L, _, terms = oracle.loss_image(dict(A=A, S_t=St, S_n=Sn), D, N)
    assert terms[1] == pytest.approx(k, rel=1e-9)
    # N_gicp is binary32, so |N_gicp| = 1 only to ~1e-7
    assert terms[2] == pytest.approx(1 - math.cos(theta), rel=1e-6)
    assert L == pytest.approx(0.1 * k + 0.05 * (1 - math.cos(theta)), rel=1e-6)


def test_p8_masks(oracle):
    D, N = _planes()
    rng = np.random.default_rng(1)
    A = rng.uniform(0.2, 0.99, D.shape); St = rng.uniform(1, 20, D.shape); Sn = rng.normal(size=(3,) + D.shape)
    L0, g0, _ = oracle.loss_image(dict(A=A, S_t=St, S_n=Sn), D, N)
    # pixels without a return do not enter the loss; pixels without a normal do not enter L_n
    A2, St2, Sn2 = A.copy(), St.copy(), Sn.copy()
    A2[0, 1] = 0.01; St2[2, 3] = 99.0; Sn2[:, 0, 1] = 3.0; Sn2[:, 1, 1] = [1, 2, 3]
    L1, _, _ = oracle.loss_image(dict(A=A2, S_t=St2, S_n=Sn2), D, N)
    assert L1 == pytest.approx(L0, rel=1e-12)
    assert g0["dA"][0, 1] == 0 and g0["dS_t"][2, 3] == 0 and np.all(g0["dS_n"][:, 1, 1] == 0)
    Lz, _, tz = oracle.loss_image(dict(A=A, S_t=St, S_n=Sn), np.zeros_like(D), N)
    assert Lz == 0.0 and np.all(tz == 0.0)


def test_p8_loss_gradient_matches_finite_differences(oracle):
    D, N = _planes()
    rng = np.random.default_rng(2)
    A = rng.uniform(0.2, 0.99, D.shape); St = rng.uniform(1, 20, D.shape); Sn = rng.normal(size=(3,) + D.shape)
    _, g, _ = oracle.loss_image(dict(A=A, S_t=St, S_n=Sn), D, N)
    h = 1e-7
    for name, arr in (("dA", A), ("dS_t", St), ("dS_n", Sn)):
        for idx in np.ndindex(arr.shape):
            p, m = arr.copy(), arr.copy()
            p[idx] += h; m[idx] -= h
            args = lambda x: dict(A=x if name == "dA" else A, S_t=x if name == "dS_t" else St,
                                  S_n=x if name == "dS_n" else Sn)
            fd = (oracle.loss_image(args(p), D, N)[0] - oracle.loss_image(args(m), D, N)[0]) / (2 * h)
            assert g[name][idx] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_p8_scale_regulariser(oracle):
    s = np.array([[0.5, 0.2], [1.3, 0.4], [0.9, 1.75], [2.0, 2.0]])
    L = oracle.scale_reg(np.log(s), s_max=1.0, lam_s=1.0)
    assert L == pytest.approx(0.3 + 0.75 + 1.0, rel=1e-12)
    d = np.zeros((4, 2))
    oracle.scale_reg(np.log(s), s_max=1.0, lam_s=10.0, dls=d)
    assert np.allclose(d, [[0, 0], [13.0, 0], [0, 17.5], [20.0, 0]])


# --------------------------------------------------------------------------
# P9: the surface-normal term of Eq. normalloss (N_surf from rendered depth)
# --------------------------------------------------------------------------
def _plane_image(frame, m, rho, A0=0.85):
    """Rendered planes of the plane {X : m.X = rho} (m unit, rho > 0) seen
    from the origin: D_hat = rho / (m.d) exactly where m.d > 0.2, else no
    return.  Returns (A, S_t, valid, rays)."""
    H, W = frame.H, frame.W
    d = np.array([[pixel_dir(frame, r, c) for c in range(W)] for r in range(H)])   # [H, W, 3]
    md = d @ m
    valid = md > 0.2
    t = np.where(valid, rho / np.where(valid, md, 1.0), 0.0)
    A = np.full((H, W), A0)
    return A, t * (A + EPS), valid, t


def _perp(v, seed):
    rng = np.random.default_rng(seed)
    p = np.cross(v, rng.normal(size=v.shape))
    return p / np.linalg.norm(p, axis=-1, keepdims=True)


def test_p9_surface_normal_of_a_plane(oracle):
    """Back-projected rendered ranges of a plane are coplanar, so N_surf is
    the plane's normal turned towards the sensor; with N_hat at a known angle
    theta_p from it, L_ns = sum over the pixels that have a term (a return
    and a rendered surface there, at the next column -- column W-1 pairs with
    column 0 -- and at the next row) of (1 - cos theta_p), divided by
    |Omega_D|."""
    frame = scenes.Frame(6, 32, 16, 16, -0.35, 0.35)
    H, W = frame.H, frame.W
    m = np.array([1.0, 0.15, -0.25]); m /= np.linalg.norm(m)
    A, St, valid, t = _plane_image(frame, m, 5.0)
    D = np.where(valid, t, 0.0).astype(np.float32)
    assert valid[:, 0].all() and valid[:, W - 1].all()        # the seam lies on the plane
    D[2, 5] = 0.0; D[4, 30] = 0.0                               # holes in the scan
    A[3, 1] = 0.0; St[3, 1] = 0.0                               # a pixel that renders nothing
    ok = D > 0
    rend = ok & (A > 0)
    rng = np.random.default_rng(4)
    theta = rng.uniform(0.0, 0.6, (H, W))
    theta[1, W - 1] = math.pi                                   # one normal pointing away
    perp = _perp(np.broadcast_to(m, (H, W, 3)), 5)
    nh = np.cos(theta)[..., None] * (-m) + np.sin(theta)[..., None] * perp
    Sn = 3.0 * nh.transpose(2, 0, 1)
    N = np.zeros((3, H, W), np.float32)                         # no G-ICP normals
    has = np.zeros((H, W), bool)
    for r in range(H - 1):
        for c in range(W):
            has[r, c] = rend[r, c] and rend[r, (c + 1) % W] and rend[r + 1, c]
    assert has[1, W - 1] and not has[H - 1].any() and not has[2, 4] and not has[1, 5]
    assert not has[3, 1] and not has[3, 0] and not has[2, 1] and has[3, 2]
    expect = (1.0 - np.cos(theta))[has].sum() / ok.sum()
    fw = dict(A=A, S_t=St, S_n=Sn)
    L0, _, t0 = oracle.loss_image(fw, D, N)
    L, _, terms = oracle.loss_image(fw, D, N, lam_ns=0.01, frame=frame)
    assert t0[3] == 0.0
    assert terms[3] == pytest.approx(expect, rel=1e-9)
    assert L - L0 == pytest.approx(0.01 * expect, rel=1e-6)
    # N_hat facing the sensor everywhere: no loss
    _, _, tz = oracle.loss_image(dict(A=A, S_t=St, S_n=np.broadcast_to(-m[:, None, None], (3, H, W))), D, N,
                                 lam_ns=1.0, frame=frame)
    assert abs(tz[3]) < 1e-12


def test_p9_column_shift_invariance(oracle):
    """Rolling every plane by W/4 columns while turning S_n by +90 degrees
    about z is the same scene turned by 90 degrees: the same L_ns, and the
    gradients roll with it (the wrap at 2 pi is a pixel pair like any other)."""
    frame = scenes.Frame(5, 16, 16, 16, -0.4, 0.3)
    rng = np.random.default_rng(6)
    H, W = frame.H, frame.W
    A = rng.uniform(0.3, 0.95, (H, W)); St = rng.uniform(3, 8, (H, W)) * (A + EPS)
    Sn = rng.normal(size=(3, H, W))
    D = rng.uniform(3, 8, (H, W)).astype(np.float32); D[1, 3] = 0.0; D[3, 15] = 0.0
    N = np.zeros((3, H, W), np.float32)
    L, g, t = oracle.loss_image(dict(A=A, S_t=St, S_n=Sn), D, N, lam_ns=1.0, frame=frame)
    k = W // 4
    roll = lambda x: np.roll(x, k, axis=-1)
    Sn2 = np.stack([-Sn[1], Sn[0], Sn[2]])
    L2, g2, t2 = oracle.loss_image(dict(A=roll(A), S_t=roll(St), S_n=roll(Sn2)), roll(D), N, lam_ns=1.0,
                                   frame=frame)
    assert t2[3] == pytest.approx(t[3], rel=1e-12)
    assert np.allclose(g2["dA"], roll(g["dA"]), rtol=1e-9, atol=1e-14)
    assert np.allclose(g2["dS_t"], roll(g["dS_t"]), rtol=1e-9, atol=1e-14)
    gsn = np.stack([-g["dS_n"][1], g["dS_n"][0], g["dS_n"][2]])
    assert np.allclose(g2["dS_n"], roll(gsn), rtol=1e-9, atol=1e-14)


def test_p9_surface_normal_gradient_matches_finite_differences(oracle):
    frame = scenes.Frame(4, 6, 16, 16, -0.5, 0.5)
    rng = np.random.default_rng(7)
    H, W = frame.H, frame.W
    A = rng.uniform(0.3, 0.95, (H, W)); St = rng.uniform(3, 8, (H, W)) * (A + EPS)
    Sn = rng.normal(size=(3, H, W))
    D = (St / (A + EPS) + rng.choice([-1.0, 1.0], (H, W)) * rng.uniform(0.5, 1.0, (H, W))).astype(np.float32)
    D[2, 1] = 0.0
    N = rng.normal(size=(3, H, W)).astype(np.float32)
    f = lambda a, st, sn: oracle.loss_image(dict(A=a, S_t=st, S_n=sn), D, N, lam_ns=0.5, frame=frame)
    _, g, terms = f(A, St, Sn)
    assert terms[3] > 0
    h = 1e-6
    for name, arr in (("dA", A), ("dS_t", St), ("dS_n", Sn)):
        for idx in np.ndindex(arr.shape):
            p, m = arr.copy(), arr.copy()
            p[idx] += h; m[idx] -= h
            sel = lambda x: (x if name == "dA" else A, x if name == "dS_t" else St, x if name == "dS_n" else Sn)
            fd = (f(*sel(p))[0] - f(*sel(m))[0]) / (2 * h)
            assert g[name][idx] == pytest.approx(fd, rel=1e-5, abs=1e-8), (name, idx)


def test_oracle_constants(oracle):
    c = oracle.constants()
    assert c[0] == 0.2 and c[1] == 9.0 and c[2] == 1 / 255 and c[3] == 0.99 and c[4] == 1e-4


def test_p6_gradient_with_clamped_opacity(oracle):
    """Surfels with alpha = 0.999 facing the ray through a pixel centre: there
    a = min(alpha G, 0.99) is clamped (flat), at the neighbouring pixels it is
    not; the analytic gradient (zero through the clamp) matches central
    differences."""
    frame = scenes.Frame(16, 64, 16, 16, -0.5, 0.5)
    bg, _ = scenes.random_shell(14, 40, r_range=(6.0, 9.0), scale_range=(0.2, 0.9), frame=frame)
    fs = facing_surfels([(pixel_dir(frame, r, c), 4.0 + 0.3 * k, 0.999, 0.5, 0.4, 0.0)
                         for k, (r, c) in enumerate(((5, 9), (8, 30), (11, 50)))])
    surf = scenes.Surfels(*(np.concatenate([getattr(fs, k), getattr(bg, k)])
                            for k in ("mean", "quat", "log_scale", "logit")))
    tgt = scenes.targets_for(frame, surf, seed=3)
    base = [np.ascontiguousarray(a, np.float64).copy() for a in
            (surf.mean, surf.quat, surf.log_scale, surf.logit)]
    L0, fw0, g = _loss64(oracle, surf, frame, tgt, base)
    assert (fw0["flags"] & 16).sum() == 0            # no pixel near the clamp kink
    gl = [g["mean"], g["quat"], g["log_scale"], g["logit"]]
    h, used = 1e-6, 0
    for which in range(4):
        for i in range(3):                            # the clamped surfels
            for comp in range(base[which].shape[1] if base[which].ndim > 1 else 1):
                idx = (i, comp) if base[which].ndim > 1 else (i,)
                vals, same = [], True
                for sgn in (1, -1):
                    p = [a.copy() for a in base]
                    p[which][idx] += sgn * h
                    L, fw, _ = _loss64(oracle, surf, frame, tgt, p)
                    vals.append(L)
                    same &= np.array_equal(fw["n_valid"], fw0["n_valid"])
                if not same:
                    continue
                fd = (vals[0] - vals[1]) / (2 * h)
                scale = max(abs(fd), 1e-3 * max(np.abs(x).max() for x in gl))
                assert abs(gl[which][idx] - fd) <= 2e-5 * scale + 1e-9, (which, idx, gl[which][idx], fd)
                used += 1
    assert used >= 25


# --------------------------------------------------------------------------
# Adam of the mapping loop: closed forms
# --------------------------------------------------------------------------
def test_adam_first_step_is_signed_learning_rate(oracle):
    """At t = 1 the bias corrections give mhat = g, vhat = g^2, so every
    parameter moves by lr g / (|g| + eps): -lr sign(g) for |g| >> eps."""
    rng = np.random.default_rng(3)
    p0 = rng.normal(size=50)
    g = rng.normal(size=50) * 10.0 ** rng.uniform(-6, 2, 50)
    p1, m, v = oracle.adam(p0, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    assert np.allclose(p1, p0 - 1e-3 * g / (np.abs(g) + 1e-15), rtol=0, atol=1e-15)
    assert np.all(np.abs(p1 - (p0 - 1e-3 * np.sign(g))) <= 1e-3 * 1e-15 / np.abs(g) + 1e-15)
    assert np.allclose(m, 0.1 * g, rtol=1e-15) and np.allclose(v, 0.001 * g * g, rtol=1e-15)


def test_adam_constant_gradient_moves_linearly(oracle):
    """With a constant gradient the bias-corrected moments stay g and g^2, so
    k steps move every parameter by k lr sign(g); lr = 0 moves nothing."""
    rng = np.random.default_rng(4)
    p = p0 = rng.normal(size=20)
    g = rng.normal(size=20)
    m = v = np.zeros(20)
    for t in range(1, 8):
        p, m, v = oracle.adam(p, g, m, v, t, 5e-3)
    assert np.allclose(p, p0 - 7 * 5e-3 * np.sign(g), rtol=0, atol=1e-12)
    q, _, _ = oracle.adam(p0, g, np.zeros(20), np.zeros(20), 1, 0.0)
    assert np.array_equal(q, p0)


# --- P10 tracking-side targets (Sec. 3.2) ---------------------------------------
def _surfels_from_axes(tu, n, scales, alpha, means=None):
    k = len(scales)
    R = scenes.frames_from_axes(np.asarray(tu, float), np.asarray(n, float))
    q = scenes.rot_to_quat(R)
    mean = np.zeros((k, 3)) if means is None else np.asarray(means, float)
    return scenes.Surfels(mean.astype(np.float32), q.astype(np.float32),
                          np.log(np.asarray(scales, float)).astype(np.float32),
                          np.log(np.asarray(alpha) / (1 - np.asarray(alpha))).astype(np.float32)), R


def test_target_covariance_eigenstructure(oracle):
    """C = R diag(s_x^2, s_y^2, eps^2) R^T: the axes the surfel was built from
    are its eigenvectors with those eigenvalues (checked against the axes of
    the construction, not the oracle's rotation)."""
    rng = np.random.default_rng(3)
    k = 50
    tu, n = rng.normal(size=(k, 3)), rng.normal(size=(k, 3))
    scales = rng.uniform(0.02, 0.8, (k, 2))
    surf, R = _surfels_from_axes(tu, n, scales, np.full(k, 0.5))
    idx, _, cov, _ = oracle.trackable_targets(surf, np.ones(k), np.zeros(k, np.int32), 0, 0.1, thickness=0.01)
    assert np.array_equal(idx, np.arange(k))
    s = np.exp(surf.log_scale.astype(np.float64))
    for i in range(k):
        c = cov[i]
        C = np.array([[c[0], c[1], c[2]], [c[1], c[3], c[4]], [c[2], c[4], c[5]]])
        ax = R[i] / np.linalg.norm(R[i], axis=0)
        lam = (s[i, 0] ** 2, s[i, 1] ** 2, 1e-4)
        for j in range(3):
            assert np.allclose(C @ ax[:, j], lam[j] * ax[:, j], atol=2e-6 * max(lam))
        assert np.trace(C) == pytest.approx(sum(lam), rel=1e-9)


def test_target_weights_from_anisotropy(oracle):
    """kappa = s_0 / (s_1 + eps) normalised over the set: the least anisotropic
    surfel gets w_max = 10, the most anisotropic 1 / (1 + eps), the middle one
    1 / (1/2 + eps); the order of the two scales does not matter."""
    k = 3
    tu = np.tile([1.0, 0.0, 0.0], (k, 1))
    n = np.tile([0.0, 0.0, 1.0], (k, 1))
    scales = [[0.1, 0.1], [0.1, 0.2], [0.3, 0.1]]          # kappa ~ 1, 2, 3
    surf, _ = _surfels_from_axes(tu, n, scales, [0.5] * k)
    _, _, _, w = oracle.trackable_targets(surf, np.ones(k), np.zeros(k, np.int32), 0, 0.1)
    s = np.exp(surf.log_scale.astype(np.float64))
    kap = s.max(1) / (s.min(1) + 1e-6)
    assert np.argmin(kap) == 0 and np.argmax(kap) == 2
    assert w[0] == 10.0
    assert w[2] == pytest.approx(1.0 / (1.0 + 1e-6), rel=1e-12)
    mid = (kap[1] - kap[0]) / (kap[2] - kap[0])
    assert mid == pytest.approx(0.5, abs=1e-5)
    assert w[1] == pytest.approx(1.0 / (mid + 1e-6), rel=1e-12)
    # one anisotropy for all: nothing to normalise, every weight is w_max
    surf2, _ = _surfels_from_axes(tu, n, [[0.2, 0.1]] * 3, [0.5] * 3)
    _, _, _, w2 = oracle.trackable_targets(surf2, np.ones(3), np.zeros(3, np.int32), 0, 0.1)
    assert np.all(w2 == 10.0)


def test_trackable_selection_rule(oracle):
    """m_i = 1, k_i >= k_min, alpha_i >= alpha_min, in ascending index; an
    empty selection gives empty arrays."""
    alpha = [0.9, 0.9, 0.2, 0.9, 0.9, 0.6]
    mask = [1, 0, 1, 1, 1, 1]
    kf = [5, 5, 5, 2, 7, 3]
    k = len(alpha)
    surf, _ = _surfels_from_axes(np.tile([1.0, 0, 0], (k, 1)), np.tile([0, 0, 1.0], (k, 1)),
                                 [[0.1, 0.05]] * k, alpha, means=np.arange(3 * k).reshape(k, 3))
    idx, mean, _, _ = oracle.trackable_targets(surf, np.array(mask), np.array(kf, np.int32), 3, 0.5)
    assert idx.tolist() == [0, 4, 5]
    assert np.array_equal(mean, np.arange(3 * k).reshape(k, 3)[[0, 4, 5]])
    idx, mean, cov, w = oracle.trackable_targets(surf, np.zeros(k), np.array(kf, np.int32), 3, 0.5)
    assert idx.size == 0 and mean.shape == (0, 3) and cov.shape == (0, 6) and w.size == 0
