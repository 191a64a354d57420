"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars (the required tolerances): sort order, tile lists and tile ranges
bit-exact; expected depth and opacity within 1e-5 relative, normals within
1e-4; gradients within 1e-3 relative.  "Relative" has a floor,
tol * max(|y|, 1e-3 max|y|), and every bar adds the uncertainty the oracle
computes for a binary32 evaluation of the same inputs (no pixel or surfel is
dropped from the check):

  * forward: fp32_err_A / fp32_err_D -- the error implied by representing the
    sensor-frame geometry and the rays in binary32 (local coordinates known
    to ~2^-24 max(t,|mu|)/s, amplified by 1/|n.d| and |mu|/|n.mu|), plus the
    size of any contribution whose skip / stop decision lies within that
    uncertainty (or 0.1 %) of its threshold;
  * gradients: 1e-5 (168 binary32 ulps) of a majorant of the per-pixel
    contributions (every term and every product of the chain to the raw
    parameters in absolute value: the conditioning of the sums, whatever
    their order), plus "flip": twice the first-order change of each
    contribution under the binary32 uncertainties of its inputs (u, v, t,
    n.d, the transmittance before it, the suffix after it, near-threshold
    decisions of the pixel's other entries counted as whole opacities) and
    the would-be contribution of the surfel's own near-threshold decisions; a
    grazing decision makes a surfel's gradient undetermined (inf, counted:
    0.02 % of the street map's surfels, at most 0.75 % in the random test
    shells).

Beyond that, each case requires the share of values that meet the plain bar
(no allowance) measured for it on a GB300, less a small margin (PLAIN).
The allowance itself is pinned on the CPU (tests/test_fp32_allowance.py).

The loss and the backward are each checked on identical inputs: the oracle's
loss on the GPU's forward outputs, the oracle's backward with the GPU's
upstream gradients, so the L1 subgradient's jump at D = D_hat cannot mix
into the comparison of the kernels.
"""
import math

import numpy as np
import pytest

from paper_2607_04127_gb300 import scenes

pytestmark = pytest.mark.gpu

EPS = 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_04127_gb300 import build
    build.build()


def ratio(x, y, tol, extra=0.0):
    """|x - y| / (tol max(|y|, 1e-3 max|y|) + extra), element-wise."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    floor = 1e-3 * np.abs(y).max() if y.size else 0.0
    lim = tol * np.maximum(np.abs(y), floor) + extra + 1e-300
    return np.abs(x - y) / lim, float(np.mean(np.abs(x - y) <= tol * np.maximum(np.abs(y), floor)))


def cases():
    out = []
    s, f, t = scenes.box_room()
    out.append(("box_room_32x512", s, f, t))
    s, f = scenes.random_shell(1, 400, frame=scenes.Frame(32, 64, 16, 16, -0.5, 0.5))
    out.append(("shell_32x64", s, f, scenes.targets_for(f, s, 1)))
    s, f = scenes.random_shell(5, 700, frame=scenes.Frame(37, 100, 8, 8, -0.4, 0.4, scenes.pose_matrix(1.1)))
    out.append(("ragged_37x100_8x8", s, f, scenes.targets_for(f, s, 2)))
    s, f = scenes.random_shell(4, 300, r_range=(0.3, 4.0), scale_range=(0.05, 1.5),
                               frame=scenes.Frame(40, 72, 8, 4, -1.4, 1.4))
    out.append(("near_sensor_poles", s, f, scenes.targets_for(f, s, 3)))
    s, f = scenes.random_shell(8, 1200, frame=scenes.Frame(64, 256, 8, 32, -0.8, 0.8,
                                                           scenes.pose_matrix(2.0, (0.5, -0.3, 0.2), 0.1, -0.05)))
    out.append(("shell_64x256_8x32_pose", s, f, scenes.targets_for(f, s, 4)))
    # opacities up to 0.999: exercises the 0.99 clamp and its zero derivative
    s, f = scenes.random_shell(9, 500, frame=scenes.Frame(32, 128, 16, 16, -0.4, 0.4))
    s.logit[::3] = 6.0
    out.append(("clamped_opacity", s, f, scenes.targets_for(f, s, 6)))
    out.append(("grazing_ground_seam",) + grazing_ground_seam())
    return out


def grazing_ground_seam(seed=12):
    """Thin, anisotropic surfels on a ground plane 1.8 m below the sensor
    (seen at grazing incidence: footprints one or two rows tall, where the
    compositing kernels' 3-sigma-disc culling box is much tighter than the
    bounding sphere) plus a cluster straddling the 0 / 2 pi azimuth seam."""
    rng = np.random.default_rng(seed)
    n_g, n_s = 2500, 600
    xy = rng.uniform(-15.0, 15.0, (n_g, 2))
    ground = np.column_stack([xy, -1.8 + rng.normal(0.0, 0.01, n_g)])
    n_ground = np.column_stack([rng.normal(0.0, 0.05, (n_g, 2)), np.ones(n_g)])
    phi = rng.uniform(-0.12, 0.12, n_s)
    el = rng.uniform(-0.6, 0.6, n_s)
    r = rng.uniform(2.0, 9.0, n_s)
    seam = np.column_stack([r * np.cos(el) * np.cos(phi), r * np.cos(el) * np.sin(phi), r * np.sin(el)])
    mean = np.concatenate([ground, seam])
    nrm = np.concatenate([n_ground, rng.normal(size=(n_s, 3))])
    Rm = scenes.frames_from_axes(rng.normal(size=(n_g + n_s, 3)), nrm)
    scale = np.column_stack([rng.uniform(0.02, 0.3, n_g + n_s), rng.uniform(0.004, 0.05, n_g + n_s)])
    alpha = rng.uniform(0.3, 0.95, n_g + n_s)
    surf = scenes.Surfels(mean.astype(np.float32), scenes.rot_to_quat(Rm).astype(np.float32),
                          np.log(scale).astype(np.float32), np.log(alpha / (1 - alpha)).astype(np.float32))
    frame = scenes.Frame(64, 512, 8, 8, -math.radians(45), math.radians(45))
    return surf, frame, scenes.targets_for(frame, surf, 8)


CASES = cases()
IDS = [c[0] for c in CASES]

# Share of values that must meet the plain bar (without any allowance) and
# the largest share of undetermined surfel gradients, per case: the fractions
# measured on a GB300 (forward outputs are reproducible bit for bit; the
# gradients vary with the order of float atomics) less a small margin, 0.002
# for the forward and 0.001 for the gradients.  Measured (A, D, gradients):
#   box_room 0.9705 1.0000 0.99967   shell_32x64 0.9927 1.0000 0.99875
#   ragged 0.9887 0.9951 0.99857     near_sensor_poles 1.0000 1.0000 1.00000
#   shell_pose 0.9936 0.9990 0.99917 clamped_opacity 0.9973 0.9998 0.99933
#   grazing_seam 0.9614 0.9997 0.99839  street (200k) 0.9990 1.0000 0.99994
# The undetermined surfels (a grazing |n.d| decision within the binary32
# uncertainty of 1e-6 at some pixel) are those the oracle flags: 0 to 0.75 %.
PLAIN = {
    "box_room_32x512": (0.9685, 0.998, 0.9986, 0.0),
    "shell_32x64": (0.9907, 0.998, 0.9977, 0.0025),
    "ragged_37x100_8x8": (0.9867, 0.9931, 0.9975, 0.0043),
    "near_sensor_poles": (0.998, 0.998, 0.999, 0.0),
    "shell_64x256_8x32_pose": (0.9916, 0.997, 0.9981, 0.0075),
    "clamped_opacity": (0.9953, 0.9978, 0.9983, 0.0),
    "grazing_ground_seam": (0.9594, 0.9977, 0.9973, 0.0046),
    "street_full": (0.997, 0.9980, 0.9989, 0.0002),
}
# the other GPU tests (batches, tunings, long lists): the weakest measured
# case's bars; undetermined 1.8 % was measured for the random shell of the
# multi-map batch
DEFAULT_PLAIN = (0.959, 0.993, 0.997, 0.02)


@pytest.mark.parametrize("name,surf,frame,tgt", CASES, ids=IDS)
def test_bins_bit_exact(oracle, name, surf, frame, tgt):
    from tests import _gpu
    g = _gpu.run([surf], [frame], read_bins=True)
    tp, ip, rg, dk = g["bins"]
    o = oracle.bin_frame(surf, frame)
    assert np.array_equal(dk, o["depth_bits"])
    keys = (tp.astype(np.uint64) << np.uint64(32)) | dk[ip].astype(np.uint64)
    assert len(keys) == o["n_pairs"]
    assert np.array_equal(keys, o["keys"])
    assert np.array_equal(ip, o["vals"])
    assert np.array_equal(rg.astype(np.int64), o["ranges"])


def compare_forward(gf, of, tolA=1e-5, tolN=1e-4):
    """Returns dict of (worst ratio, fraction within the plain bar)."""
    out = {}
    out["A"] = ratio(gf["A"], of["A"], tolA, 2 * of["fp32_err_A"])
    Dg = gf["S_t"] / (gf["A"].astype(np.float64) + EPS)
    Do = of["S_t"] / (of["A"] + EPS)
    out["D"] = ratio(Dg, Do, tolA, 2 * of["fp32_err_D"])
    out["T"] = ratio(gf["T_final"], of["T_final"], tolA, 2 * of["fp32_err_A"])
    Ng = gf["S_n"] / np.sqrt((gf["S_n"].astype(np.float64) ** 2).sum(0) + EPS ** 2)
    No = of["S_n"] / np.sqrt((of["S_n"] ** 2).sum(0) + EPS ** 2)
    nerr = np.abs(Ng - No).max(0)
    ntol = tolN + 4 * of["fp32_err_A"] / np.maximum(of["A"], 1e-3)
    out["N"] = (nerr / ntol, float(np.mean(nerr <= tolN)))
    calm = of["flags"] == 0
    out["nc_equal"] = bool(np.array_equal(gf["n_contrib"][calm], of["n_contrib"][calm]))
    out["calm"] = float(calm.mean())
    return out


def assert_forward(r):
    for k in ("A", "D", "T", "N"):
        assert r[k][0].max() <= 1.0, (k, float(r[k][0].max()), r[k][1])
    assert r["nc_equal"]


@pytest.mark.parametrize("name,surf,frame,tgt", CASES, ids=IDS)
def test_forward_parity(oracle, name, surf, frame, tgt):
    from tests import _gpu
    g = _gpu.run([surf], [frame])
    o = oracle.bin_frame(surf, frame)
    of = oracle.render_fwd(surf, frame, o["ranges"], o["vals"])
    r = compare_forward(g["fwd"][0], of)
    assert_forward(r)
    # the case's measured share of pixels meets the plain bar without any
    # uncertainty term
    assert r["A"][1] >= PLAIN[name][0] and r["D"][1] >= PLAIN[name][1], (name, r["A"][1], r["D"][1])


def oracle_grads(oracle, surf, frames, ups, scale_reg=True):
    """Oracle backward of a window of frames with the given upstream planes
    (gA, gSt, gSn per frame), plus the scale regulariser."""
    n = surf.n
    g = dict(mean=np.zeros((n, 3)), quat=np.zeros((n, 4)), log_scale=np.zeros((n, 2)), logit=np.zeros(n),
             abs=np.zeros((n, 10)), flip=np.zeros((n, 10)))
    for frame, (gA, gSt, gSn) in zip(frames, ups):
        b = oracle.bin_frame(surf, frame)
        oracle.render_bwd(surf, frame, b["ranges"], b["vals"], gA, gSt, gSn, grads=g)
    if scale_reg:
        oracle.scale_reg(surf.log_scale, dls=g["log_scale"])
    return g


def compare_grads(gg, og, tol=1e-3):
    out = {}
    n = og["mean"].shape[0]
    off = 0
    undet = np.isinf(og["flip"]).any(1)
    for k, (name, w) in enumerate((("mean", 3), ("quat", 4), ("log_scale", 2), ("logit", 1))):
        x = np.asarray(gg[k], np.float64).reshape(n, -1)
        y = og[name].reshape(n, -1)
        extra = 1e-5 * og["abs"][:, off:off + w] + og["flip"][:, off:off + w]
        off += w
        r, plain = ratio(x, y, tol, extra)
        r = np.where(np.isinf(extra), 0.0, r)
        out[name] = (float(r.max()), plain)
    out["undetermined"] = float(undet.mean())
    return out


def assert_grads(r, case=None):
    """Every value within its bar; the case's share (or the default) within
    the plain bar; at most the case's share undetermined."""
    plain = PLAIN.get(case, DEFAULT_PLAIN)
    for name in ("mean", "quat", "log_scale", "logit"):
        assert r[name][0] <= 1.0, (name, r)
        assert r[name][1] >= plain[2], (name, case, r)
    assert r["undetermined"] <= plain[3], (case, r)


def gpu_upstream(g, f):
    u = g["upstream"][f]
    return (u["dA"].astype(np.float64), u["dS_t"].astype(np.float64), u["dS_n"].astype(np.float64))


def check_loss_on_gpu_forward(oracle, g, frames, targets, scales):
    """The oracle's loss evaluated on the GPU's forward outputs equals the
    GPU loss, and its upstream planes equal the GPU's (pixels whose depth is
    within 1e-5 of the target -- the L1 kink -- are skipped)."""
    total = 0.0
    for f, (frame, tgt) in enumerate(zip(frames, targets)):
        fw = {k: np.asarray(v, np.float64) for k, v in g["fwd"][f].items()}
        Lf, up, terms = oracle.loss_image(fw, tgt.D, tgt.N, scale=scales[f])
        total += Lf
        Dh = fw["S_t"] / (fw["A"] + EPS)
        kink = np.abs(Dh - tgt.D) <= 1e-5 * np.abs(tgt.D)
        for k, key in (("dA", "dA"), ("dS_t", "dS_t")):
            r, _ = ratio(np.where(kink, 0, g["upstream"][f][key]), np.where(kink, 0, up[key]), 1e-5)
            assert r.max() <= 1.0, (key, float(r.max()))
        # dL/dS_n = g/m - S (S.g)/m^3 cancels when N_hat is parallel to N_gicp:
        # its binary32 error scales with the terms, |g|/m, not with the result
        m = np.sqrt((fw["S_n"] ** 2).sum(0) + EPS ** 2)
        nn = max(int(((tgt.D > 0) & ((tgt.N.astype(np.float64) ** 2).sum(0) > 0)).sum()), 1)
        gterm = scales[f] * 1.0 * 0.05 / nn / m
        r, _ = ratio(g["upstream"][f]["dS_n"], up["dS_n"], 1e-5, 1e-5 * gterm[None])
        assert r.max() <= 1.0, ("dS_n", float(r.max()))
        assert np.allclose(g["loss"][1 + 4 * f: 5 + 4 * f], terms, rtol=1e-5, atol=1e-9)
    return total


@pytest.mark.parametrize("name,surf,frame,tgt", CASES, ids=IDS)
def test_loss_and_backward_parity(oracle, name, surf, frame, tgt):
    from tests import _gpu
    g = _gpu.run([surf], [frame], targets=[tgt])
    Limg = check_loss_on_gpu_forward(oracle, g, [frame], [tgt], [1.0])
    Ls = oracle.scale_reg(surf.log_scale)
    assert g["loss"][0] == pytest.approx(Limg + Ls, rel=1e-5)
    # end to end (oracle's own forward): the same loss to 1e-5
    Lo, _, _, _ = oracle.forward_backward(surf, [frame], [(tgt.D, tgt.N)])
    assert g["loss"][0] == pytest.approx(Lo, rel=1e-5)
    og = oracle_grads(oracle, surf, [frame], [gpu_upstream(g, 0)])
    assert_grads(compare_grads(g["grads"][0], og), name)


NS_CASES = [(c, lam) for c in CASES if c[0] in ("box_room_32x512", "ragged_37x100_8x8", "near_sensor_poles")
            for lam in (0.01, 1.0)]


@pytest.mark.parametrize("name,surf,frame,tgt,lam_ns", [c + (lam,) for c, lam in NS_CASES],
                         ids=[f"{c[0]}-{lam}" for c, lam in NS_CASES])
def test_surface_normal_term_parity(oracle, name, surf, frame, tgt, lam_ns):
    """The N_surf term of Eq. normalloss (normal of the rendered depth, image
    columns wrapping at 2 pi): on the GPU's forward outputs the oracle gives
    the same L_ns and upstream planes, within 1e-5 plus the oracle's bound
    on a binary32 evaluation of the term (cross products of differences of
    neighbouring back-projected ranges); the surfel gradients through those
    planes match as in the plain loss."""
    from tests import _gpu
    g = _gpu.run([surf], [frame], targets=[tgt], loss=dict(_gpu.LOSS, lambda_ns=lam_ns))
    fw = {k: np.asarray(v, np.float64) for k, v in g["fwd"][0].items()}
    err = {}
    Lf, up, terms = oracle.loss_image(fw, tgt.D, tgt.N, lam_ns=lam_ns, frame=frame, ns_err=err)
    _, up0, _ = oracle.loss_image(fw, tgt.D, tgt.N)
    assert terms[3] > 0.0
    # the term moves most planes' values by far more than the tolerance (it is exercised)
    moved = np.abs(up["dS_t"] - up0["dS_t"]) > 1e-3 * np.abs(up0["dS_t"])
    assert moved[tgt.D > 0].mean() > 0.3
    a = fw["A"] + EPS
    Dh = fw["S_t"] / a
    kink = np.abs(Dh - tgt.D) <= 1e-5 * np.abs(tgt.D)
    extra = dict(dA=err["dD"] * np.abs(fw["S_t"]) / a ** 2, dS_t=err["dD"] / a)
    for key in ("dA", "dS_t"):
        r, _ = ratio(np.where(kink, 0, g["upstream"][0][key]), np.where(kink, 0, up[key]), 1e-5, extra[key])
        assert r.max() <= 1.0, (key, float(r.max()))
    m = np.sqrt((fw["S_n"] ** 2).sum(0) + EPS ** 2)
    nn = max(int(((tgt.D > 0) & ((tgt.N.astype(np.float64) ** 2).sum(0) > 0)).sum()), 1)
    nd = max(int((tgt.D > 0).sum()), 1)
    gterm = (0.05 / nn + lam_ns / nd) / m
    r, _ = ratio(g["upstream"][0]["dS_n"], up["dS_n"], 1e-5, 1e-5 * gterm[None] + err["dS_n"][None])
    assert r.max() <= 1.0, ("dS_n", float(r.max()))
    gt = g["loss"][1:5]
    assert np.allclose(gt[:3], terms[:3], rtol=1e-5, atol=1e-9)
    assert abs(gt[3] - terms[3]) <= 1e-5 * terms[3] + err["L_ns"], (gt[3], terms[3], err["L_ns"])
    Ls = oracle.scale_reg(surf.log_scale)
    assert g["loss"][0] == pytest.approx(Lf + Ls, rel=1e-5)
    og = oracle_grads(oracle, surf, [frame], [gpu_upstream(g, 0)])
    assert_grads(compare_grads(g["grads"][0], og), name)


SINGLE_CASES = [c for c in CASES if c[0] in ("box_room_32x512", "ragged_37x100_8x8", "near_sensor_poles")]


@pytest.mark.parametrize("name,surf,frame,tgt", SINGLE_CASES, ids=[c[0] for c in SINGLE_CASES])
def test_single_map_calls(oracle, name, surf, frame, tgt):
    """The single-map calls of the boundary (lgs_bin_sort, lgs_render_fwd,
    lgs_loss, lgs_render_bwd) called directly through the C ABI: bins equal
    the oracle's bit for bit; forward outputs and the loss vector equal the
    batch calls' bit for bit (gradients up to the order of float atomics);
    forward and gradients match the oracle."""
    from tests import _gpu
    g1 = _gpu.run([surf], [frame], targets=[tgt], read_bins=True, single=True)
    gb = _gpu.run([surf], [frame], targets=[tgt])
    tp, ip, rg, dk = g1["bins"]
    o = oracle.bin_frame(surf, frame)
    keys = (tp.astype(np.uint64) << np.uint64(32)) | dk[ip].astype(np.uint64)
    assert np.array_equal(keys, o["keys"]) and np.array_equal(ip, o["vals"])
    assert np.array_equal(rg.astype(np.int64), o["ranges"])
    for k in ("A", "S_t", "S_n", "T_final", "n_contrib"):
        assert np.array_equal(g1["fwd"][0][k], gb["fwd"][0][k]), k
    assert np.array_equal(g1["loss"], gb["loss"])
    for a, b in zip(g1["grads"][0], gb["grads"][0]):
        assert np.allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max())
    of = oracle.render_fwd(surf, frame, o["ranges"], o["vals"])
    assert_forward(compare_forward(g1["fwd"][0], of))
    og = oracle_grads(oracle, surf, [frame], [gpu_upstream(g1, 0)])
    assert_grads(compare_grads(g1["grads"][0], og), name)


TUNINGS = ([dict(fwd_batch=0, bwd_batch=0, group=g, persistent=p) for g in (1, 2, 4, 16) for p in (0, 1)]
           + [dict(fwd_batch=b, bwd_batch=min(b, 256), group=1, persistent=p) for b in (64, 128, 256, 512)
              for p in (0, 1)])


def test_tuning_and_tile_shape_do_not_change_results(oracle):
    """Every compositing variant and tile shape gives bit-identical forward
    outputs (n_contrib, which indexes the tile's own list, within each tile
    shape) and loss; gradients agree up to the order of the float atomics."""
    surf, frame, tgt = scenes.box_room()
    from tests import _gpu
    ref = _gpu.run([surf], [frame], targets=[tgt], tuning=dict(fwd_batch=0, bwd_batch=0, group=16, persistent=0))
    gref = [np.asarray(x, np.float64) for x in ref["grads"][0]]
    for tile in ((8, 8), (16, 16), (8, 32), (32, 8)):
        # n_contrib indexes the tile's own list: compared within a tile shape
        ref_t = _gpu.run([surf], [frame.with_tiles(*tile)], targets=[tgt],
                         tuning=dict(fwd_batch=0, bwd_batch=0, group=16, persistent=0))
        for tun in TUNINGS:
            g = _gpu.run([surf], [frame.with_tiles(*tile)], targets=[tgt], tuning=tun)
            for k in ("A", "S_t", "S_n", "T_final"):
                assert np.array_equal(g["fwd"][0][k], ref["fwd"][0][k]), (tile, tun, k)
            assert np.array_equal(g["fwd"][0]["n_contrib"], ref_t["fwd"][0]["n_contrib"]), (tile, tun)
            assert np.array_equal(g["loss"], ref["loss"]), (tile, tun)
            for a, b in zip(g["grads"][0], gref):
                assert np.allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max()), (tile, tun)


def test_multi_frame_multi_map_batch(oracle):
    """Two maps, three frames (two render map 0 from different poses) in one
    call: each frame equals its oracle frame; each map's loss and gradient
    equal the oracle's for that map's own window (image terms averaged over
    the map's frames)."""
    from tests import _gpu
    s0, f0, t0 = scenes.box_room(seed=0)
    f0b = scenes.Frame(32, 512, 16, 16, f0.elev_min, f0.elev_max, scenes.pose_matrix(0.4, (1.0, 0.5, 2.3)))
    _, _, t0b = scenes.box_room(seed=0, yaw=0.4)
    s1, f1 = scenes.random_shell(3, 500, frame=scenes.Frame(32, 512, 16, 16, -0.3, 0.3, scenes.pose_matrix(-0.2)))
    t1 = scenes.targets_for(f1, s1, 5)
    frames, fmap, tg = [f0, f1, f0b], [0, 1, 0], [t0, t1, t0b]
    g = _gpu.run([s0, s1], frames, targets=tg, frame_map=fmap)
    for f, (frame, m) in enumerate(zip(frames, fmap)):
        surf = (s0, s1)[m]
        b = oracle.bin_frame(surf, frame)
        of = oracle.render_fwd(surf, frame, b["ranges"], b["vals"])
        assert_forward(compare_forward(g["fwd"][f], of))
    check_loss_on_gpu_forward(oracle, g, frames, tg, [0.5, 1.0, 0.5])
    L0, _, _, _ = oracle.forward_backward(s0, [f0, f0b], [(t0.D, t0.N), (t0b.D, t0b.N)])
    L1, _, _, _ = oracle.forward_backward(s1, [f1], [(t1.D, t1.N)])
    F = 3
    assert g["loss"][1 + 4 * F] == pytest.approx(L0, rel=1e-5)
    assert g["loss"][2 + 4 * F] == pytest.approx(L1, rel=1e-5)
    assert g["loss"][0] == pytest.approx(L0 + L1, rel=1e-5)
    og0 = oracle_grads(oracle, s0, [f0, f0b], [gpu_upstream(g, 0), gpu_upstream(g, 2)])
    og1 = oracle_grads(oracle, s1, [f1], [gpu_upstream(g, 1)])
    assert_grads(compare_grads(g["grads"][0], og0))
    assert_grads(compare_grads(g["grads"][1], og1))


def test_gradients_accumulate(oracle):
    from tests import _gpu
    surf, frame, tgt = scenes.box_room()
    g1 = _gpu.run([surf], [frame], targets=[tgt])
    g2 = _gpu.run([surf], [frame], targets=[tgt], grads_init=[g1["grads"][0]])
    # the backward sums with float atomics: equal up to summation order
    for a, b in zip(g2["grads"][0], g1["grads"][0]):
        assert np.allclose(a, 2 * b, rtol=1e-5, atol=1e-6 * np.abs(b).max())


@pytest.mark.parametrize("n,lo,hi", [(5000, 2048, 4096), (12000, 4096, 1 << 30), (40000, 16384, 1 << 30)])
def test_long_tile_bucket_bit_exact(oracle, n, lo, hi):
    """Buckets beyond the merge sort's 2048 keys take the long-bucket sort
    (8192-key chunks in shared memory, then merge passes through global
    memory: none for a bucket of at most 8192 keys, one pass up to 16384,
    two for the 40000-surfel cloud's bucket of about 18,500 keys, whose
    third chunk first has no run to merge with), and lists beyond 4096
    entries the entry-parallel compositing
    kernels: bins stay bit-exact, forward and gradients match the oracle."""
    from tests import _gpu
    rng = np.random.default_rng(11)
    frame = scenes.Frame(32, 512, 16, 16, -0.26, 0.26)
    az = 0.3 + rng.uniform(-0.035, 0.035, n)
    el = rng.uniform(-0.035, 0.035, n)
    r = rng.uniform(6.0, 12.0, n)
    mean = np.stack([r * np.cos(el) * np.cos(az), r * np.cos(el) * np.sin(az), r * np.sin(el)], 1)
    surf = scenes.Surfels(mean.astype(np.float32), rng.normal(size=(n, 4)).astype(np.float32),
                          np.log(rng.uniform(0.005, 0.02, (n, 2))).astype(np.float32),
                          rng.normal(size=n).astype(np.float32))
    tgt = scenes.targets_for(frame, surf, 7)
    g = _gpu.run([surf], [frame], targets=[tgt], read_bins=True)
    tp, ip, rg, dk = g["bins"]
    o = oracle.bin_frame(surf, frame)
    assert lo < (o["ranges"][:, 1] - o["ranges"][:, 0]).max() <= hi
    keys = (tp.astype(np.uint64) << np.uint64(32)) | dk[ip].astype(np.uint64)
    assert np.array_equal(keys, o["keys"]) and np.array_equal(ip, o["vals"])
    assert np.array_equal(rg.astype(np.int64), o["ranges"])
    of = oracle.render_fwd(surf, frame, o["ranges"], o["vals"])
    assert_forward(compare_forward(g["fwd"][0], of))
    # lists beyond 4096 entries take the entry-parallel per-pixel kernels
    og = oracle_grads(oracle, surf, [frame], [gpu_upstream(g, 0)])
    assert_grads(compare_grads(g["grads"][0], og))


def test_second_backward_of_a_long_list_forward():
    """Lists beyond 4096 entries take the chunked backward with per-chunk
    suffixes computed at backward time: a second backward of the same
    forward (same upstream planes) gives the same gradients as the first, up
    to the order of float atomics."""
    import torch
    from paper_2607_04127_gb300 import render
    rng = np.random.default_rng(11)
    n = 12000
    frame = scenes.Frame(32, 512, 16, 16, -0.26, 0.26)
    az = 0.3 + rng.uniform(-0.035, 0.035, n)
    el = rng.uniform(-0.035, 0.035, n)
    r = rng.uniform(6.0, 12.0, n)
    mean = np.stack([r * np.cos(el) * np.cos(az), r * np.cos(el) * np.sin(az), r * np.sin(el)], 1)
    surf = scenes.Surfels(mean.astype(np.float32), rng.normal(size=(n, 4)).astype(np.float32),
                          np.log(rng.uniform(0.005, 0.02, (n, 2))).astype(np.float32),
                          rng.normal(size=n).astype(np.float32))
    tgt = scenes.targets_for(frame, surf, 7)
    dev = torch.device("cuda", 0)
    params = render.map_tensors(surf, dev)
    targets = [render.target_tensors(tgt, dev)]
    rast = render.Rasterizer([frame], device=0)
    try:
        g1 = [[torch.zeros_like(p) for p in params]]
        S = rast.bin_sort([params], check=True)
        assert rast.counters()["n_pairs"] > 0
        rast.forward_loss([params], targets, None, S)
        rast.backward([params], g1, S=S)
        g2 = [[torch.zeros_like(p) for p in params]]
        rast.backward([params], g2, S=S)
        torch.cuda.synchronize()
        rast.session.check_status()
        for a, b in zip(g2[0], g1[0]):
            a, b = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
            assert np.abs(b).max() > 0
            assert np.allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max())
    finally:
        rast.close()


def test_empty_and_invisible_maps(oracle):
    from tests import _gpu
    frame = scenes.Frame(32, 64, 16, 16, -0.2, 0.2)
    empty = scenes.Surfels(np.zeros((0, 3), np.float32), np.zeros((0, 4), np.float32),
                           np.zeros((0, 2), np.float32), np.zeros(0, np.float32))
    g = _gpu.run([empty], [frame], targets=[scenes.targets_for(frame, empty, 0)])
    assert np.all(g["fwd"][0]["A"] == 0) and np.all(g["fwd"][0]["T_final"] == 1)
    assert g["counters"]["n_pairs"] == 0
    # surfels far above a narrow field of view cover no tile
    surf, _ = scenes.random_shell(2, 50, frame=scenes.Frame(32, 64, 16, 16, 1.2, 1.4))
    g = _gpu.run([surf], [frame], targets=[scenes.targets_for(frame, surf, 0)])
    assert g["counters"]["n_pairs"] == 0 and g["counters"]["n_visible"] == 0
    assert all(np.all(x == 0) for x in g["grads"][0])


def test_capacity_overflow_is_reported_and_recovered(oracle):
    import torch
    from paper_2607_04127_gb300 import lib
    from tests import _gpu
    surf, frame, _ = scenes.box_room()
    o = oracle.bin_frame(surf, frame, want_pairs=False)
    T = _gpu.to_dev(surf)
    S = lib.surfels_struct(*T)
    fr = [lib.frame_struct(frame)]
    sess = lib.Session()
    sess.reserve([surf.n], fr, [0], 100)
    lib.lgs_bin_sort_batch(sess.handle, [S], fr, [0], torch.cuda.current_stream().cuda_stream)
    st, req = lib.lgs_session_status(sess.handle)
    assert st == lib.LGS_ERR_CAPACITY and req == o["n_pairs"]
    sess.bin_sort([S], fr, [0])          # grows the workspace and bins again
    assert lib.lgs_session_pair_count(sess.handle) == o["n_pairs"]
    sess.close()


def test_invalid_arguments_are_rejected():
    from paper_2607_04127_gb300 import lib
    sess = lib.Session()
    bad = scenes.Frame(32, 64, 5, 5, -0.2, 0.2)         # 25 pixels: not a multiple of 32
    with pytest.raises(lib.LgsError):
        lib.lgs_session_workspace_size(sess.handle, 10, [lib.frame_struct(bad)], 10)
    bad = scenes.Frame(32, 64, 16, 16, 0.3, 0.2)        # empty elevation range
    with pytest.raises(lib.LgsError):
        lib.lgs_session_workspace_size(sess.handle, 10, [lib.frame_struct(bad)], 10)
    sess.close()


def test_full_size_street_frame(oracle):
    """The 200k-surfel 128 x 1024 street frame in the launch configuration the
    benchmark times (the renderer's default tile shape and tuning): bit-exact
    bins; forward, loss and gradients against the oracle run at full size."""
    from paper_2607_04127_gb300 import render
    from tests import _gpu
    surf, frame, tgt = scenes.street()
    frame = frame.with_tiles(*render.DEFAULT_TILE)
    g = _gpu.run([surf], [frame], targets=[tgt], read_bins=True)
    tp, ip, rg, dk = g["bins"]
    o = oracle.bin_frame(surf, frame)
    keys = (tp.astype(np.uint64) << np.uint64(32)) | dk[ip].astype(np.uint64)
    assert np.array_equal(keys, o["keys"]) and np.array_equal(ip, o["vals"])
    assert np.array_equal(rg.astype(np.int64), o["ranges"])
    of = oracle.render_fwd(surf, frame, o["ranges"], o["vals"])
    r = compare_forward(g["fwd"][0], of)
    assert_forward(r)
    assert r["A"][1] >= PLAIN["street_full"][0] and r["D"][1] >= PLAIN["street_full"][1], (r["A"][1], r["D"][1])
    Limg = check_loss_on_gpu_forward(oracle, g, [frame], [tgt], [1.0])
    assert g["loss"][0] == pytest.approx(Limg + oracle.scale_reg(surf.log_scale), rel=1e-5)
    og = oracle_grads(oracle, surf, [frame], [gpu_upstream(g, 0)])
    assert_grads(compare_grads(g["grads"][0], og), "street_full")


def _fused_vs_separate(maps, frames, fmap, targets, lambda_ns=0.0):
    """Forward + loss as two calls and as the one fused call on the same
    binning: every output plane, the loss vector and the scale-regulariser
    gradient, bit for bit."""
    import torch
    from paper_2607_04127_gb300 import render
    dev = torch.device("cuda")
    params = [render.map_tensors(m, dev) for m in maps]
    tg = [render.target_tensors(t, dev) for t in targets]
    rast = render.Rasterizer(frames, frame_map=fmap, device=0, loss=render.LossParams(lambda_ns=lambda_ns))
    res = []
    for fused in (False, True):
        grads = [[torch.zeros_like(p) for p in ps] for ps in params]
        S = rast.bin_sort(params, check=True)
        if fused:
            rast.forward_loss(params, tg, grads, S)
        else:
            rast.forward(params, S)
            rast.loss(params, tg, grads, S)
        torch.cuda.synchronize()
        planes = [[x.cpu().numpy().copy() for x in (o.A, o.S_t, o.S_n, o.T_final, o.n_contrib)] for o in rast.out]
        ups = [[x.cpu().numpy().copy() for x in u] for u in rast.up]
        res.append((planes, ups, rast.loss_out.cpu().numpy().copy(), [g[2].cpu().numpy().copy() for g in grads]))
    rast.close()
    (p0, u0, l0, s0), (p1, u1, l1, s1) = res
    for a, b in zip(p0, p1):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    for a, b in zip(u0, u1):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert np.array_equal(l0, l1), (l0, l1)
    for x, y in zip(s0, s1):
        assert np.array_equal(x, y)


def test_fused_forward_loss_equals_separate_calls():
    """The loss in the forward's epilogue (one call) equals the forward and
    loss calls: one frame, a multi-frame multi-map batch, a tile list beyond
    the entry-parallel threshold (the long-list forward's epilogue), and the
    N_surf term on (the call falls back to the two kernels)."""
    s0, f0, t0 = scenes.box_room(seed=0)
    _fused_vs_separate([s0], [f0], [0], [t0])
    f0b = scenes.Frame(32, 512, 16, 16, f0.elev_min, f0.elev_max, scenes.pose_matrix(0.4, (1.0, 0.5, 2.3)))
    _, _, t0b = scenes.box_room(seed=0, yaw=0.4)
    s1, f1 = scenes.random_shell(3, 500, frame=scenes.Frame(32, 512, 16, 16, -0.3, 0.3, scenes.pose_matrix(-0.2)))
    t1 = scenes.targets_for(f1, s1, 5)
    _fused_vs_separate([s0, s1], [f0, f1, f0b], [0, 1, 0], [t0, t1, t0b])
    rng = np.random.default_rng(11)
    n = 12000
    frame = scenes.Frame(32, 512, 16, 16, -0.26, 0.26)
    az = 0.3 + rng.uniform(-0.035, 0.035, n)
    el = rng.uniform(-0.035, 0.035, n)
    r = rng.uniform(6.0, 12.0, n)
    mean = np.stack([r * np.cos(el) * np.cos(az), r * np.cos(el) * np.sin(az), r * np.sin(el)], 1)
    surf = scenes.Surfels(mean.astype(np.float32), rng.normal(size=(n, 4)).astype(np.float32),
                          np.log(rng.uniform(0.005, 0.02, (n, 2))).astype(np.float32),
                          rng.normal(size=n).astype(np.float32))
    _fused_vs_separate([surf], [frame], [0], [scenes.targets_for(frame, surf, 7)])
    _fused_vs_separate([s0], [f0], [0], [t0], lambda_ns=0.01)
