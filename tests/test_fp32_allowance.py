"""Pins of the oracle's binary32 allowance (oracle/lgs_fp32_allowance.c).

Every GPU parity bar adds to its tolerance what a binary32 evaluation of the
same inputs may differ from the FP64 oracle by.  Those bounds are pinned here
against a plain binary32 restatement of the compositing arithmetic
(tests/_fp32.py), on the CPU:

* coverage: on every sampled (pixel, surfel) pair, pixel and contribution
  whose decisions are away from the thresholds, the binary32 value differs
  from the FP64 value by no more than the bound (local coordinates u, v and
  ray parameter t: fp32_unc; opacity: opacity_unc; accumulated opacity and
  depth: the pixel bounds eA, eD; transmittance: eT; a contribution to the
  raw-parameter gradient: twice contrib_unc, plus 1e-5 of the majorant where
  the suffix is binary32 too);
* not slack: the median of bound / observed error stays below a stated cap.
  Per pair 40: a bound must cover the worst pairs, whose errors reach 30 to
  50 times the median one (measured medians 16 to 30).  Per pixel 100: a sum
  over the contributors of bounds whose signed errors partly cancel
  (measured 39 to 66).  Per contribution 250: a sum of six first-order terms
  (measured about 160);
* closed forms for the parts that only act near a threshold: a single surfel
  just outside the 3-sigma cut-off (the flip term equals its would-be opacity
  and its would-be logit gradient) and a single facing surfel without
  cancellation (the majorant equals the gradient);
* decisions that a binary32 evaluation does take the other way (a surfel
  swept across the cut-off) stay inside the pixel bound;
* a mistake planted in each bound (a factor 10 or 1/10, compiled into a
  separate build of the oracle) fails at least one of these pins.
"""
import math
import os
import tempfile

import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_04127_gb300 import scenes
from tests import _fp32 as F

SLACK_PAIR, SLACK_PIXEL, SLACK_CONTRIB = 40.0, 100.0, 250.0


def _scenes(small=False):
    out = []
    s, f, t = scenes.box_room()
    out.append(("box_room", s, f, t))
    s, f = scenes.random_shell(5, 700, frame=scenes.Frame(37, 100, 8, 8, -0.4, 0.4, scenes.pose_matrix(1.1)))
    out.append(("ragged", s, f, scenes.targets_for(f, s, 2)))
    if small:
        return out
    s, f = scenes.random_shell(4, 300, r_range=(0.3, 4.0), scale_range=(0.05, 1.5),
                               frame=scenes.Frame(40, 72, 8, 4, -1.4, 1.4))
    out.append(("near_sensor_poles", s, f, scenes.targets_for(f, s, 3)))
    s, f = scenes.random_shell(8, 1200, frame=scenes.Frame(64, 256, 8, 32, -0.8, 0.8,
                                                           scenes.pose_matrix(2.0, (0.5, -0.3, 0.2), 0.1, -0.05)))
    out.append(("posed_shell", s, f, scenes.targets_for(f, s, 4)))
    s, f = scenes.random_shell(9, 500, frame=scenes.Frame(32, 128, 16, 16, -0.4, 0.4))
    s.logit[::3] = 6.0
    out.append(("clamped_opacity", s, f, scenes.targets_for(f, s, 6)))
    return out


def collect(lib=None, small=False, pixels=220, street_pixels=40, seed=0):
    """Observed binary32 errors next to the oracle's bounds over sampled
    pixels of the scenes (and of the 200k-surfel street frame): rows of
    (error, bound) per kind.  Upstream gradients are the loss's own."""
    rng = np.random.default_rng(seed)
    rows = {k: [] for k in ("u", "v", "t", "a", "A", "D", "T", "c_in", "c_full")}
    work = _scenes(small)
    if not small and street_pixels:
        s, f, t = scenes.street()
        work.append(("street", s, f.with_tiles(8, 8), t))
    for name, s, f, tg in work:
        b = O.bin_frame(s, f)
        p64 = O._params64(s)
        fw = O.render_fwd(s, f, b["ranges"], b["vals"], params64=p64)
        _, up, _ = O.loss_image(fw, tg.D, tg.N)
        cand = np.argwhere(fw["n_valid"] > 0)
        k = street_pixels if name == "street" else pixels
        for r, c in cand[rng.choice(len(cand), min(k, len(cand)), replace=False)]:
            gA, gSt, gSn = up["dA"][r, c], up["dS_t"][r, c], up["dS_n"][:, r, c]
            d = O.pixel_detail(s, f, b["ranges"], b["vals"], r, c, gA, gSt, gSn, params64=p64, lib=lib)
            idx = d["item"].astype(np.int64)
            rec = F.records(s, f, idx)
            e = F.evaluate(rec, F.rays(f, r, c))
            calm = (d["flags"] == 0) & d["valid"] & e["valid"]
            for key, bound in (("u", "eu"), ("v", "ev"), ("t", "dt"), ("a", "da")):
                err = np.abs(e[key].astype(np.float64) - d[key])
                rows[key].append(np.column_stack([err[calm], d[bound][calm]]))
            if d["pflags"] != 0:
                continue
            A, St, Sn, T, ck, cT = F.composite(e, rec, range(len(idx)))
            D32 = float(St) / (float(A) + 1e-6)
            D64 = d["S_t"] / (d["A"] + 1e-6)
            rows["A"].append(np.array([[abs(float(A) - d["A"]), d["eA"]]]))
            rows["D"].append(np.array([[abs(D32 - D64), d["eD"]]]))
            if len(ck) != d["nc"]:
                continue
            Ts, Ss = F.reverse(e, rec, ck, T, gA, gSt, gSn)
            for m, kk in enumerate(ck):
                rows["T"].append(np.array([[abs(float(Ts[m]) - d["T"][m]), d["eT"][m] * d["T"][m]]]))
                q7 = (e["den"][kk], e["t"][kk], e["u"][kk], e["v"][kk], e["G"][kk], e["a"][kk], e["araw"][kk])
                c_in = O.contrib_with(s, f, idx[kk], r, c, *q7, Ts[m], d["S"][m], gA, gSt, gSn, params64=p64, lib=lib)
                c_full = O.contrib_with(s, f, idx[kk], r, c, *q7, Ts[m], Ss[m], gA, gSt, gSn, params64=p64, lib=lib)
                rows["c_in"].append(np.column_stack([np.abs(c_in - d["grad"][m]), 2.0 * d["gunc"][m]]))
                rows["c_full"].append(np.column_stack([np.abs(c_full - d["grad"][m]),
                                                       2.0 * d["gunc"][m] + 1e-5 * d["gmaj"][m]]))
    return {k: np.concatenate(v) if v else np.zeros((0, 2)) for k, v in rows.items()}


def covered(x):
    """(violations, worst error / bound)."""
    err, bnd = x[:, 0], x[:, 1]
    return int((err > bnd).sum()), float((err / np.maximum(bnd, 1e-300)).max()) if len(err) else 0.0


def slack(x):
    """Median of bound / error over the entries with a nonzero error."""
    err, bnd = x[:, 0], x[:, 1]
    pos = err > 0
    return float(np.median(bnd[pos] / err[pos])) if pos.any() else 0.0


# pins as functions of a sample, so that a planted mistake can be run through them
def pin_pairs(R):
    for k in ("u", "v", "t", "a"):
        n, worst = covered(R[k])
        assert n == 0, (k, n, worst)
        assert slack(R[k]) <= SLACK_PAIR, (k, slack(R[k]))


def pin_pixels(R):
    for k in ("A", "D"):
        n, worst = covered(R[k])
        assert n == 0, (k, n, worst)
        assert slack(R[k]) <= SLACK_PIXEL, (k, slack(R[k]))


def pin_contributions(R):
    for k in ("T", "c_in", "c_full"):
        n, worst = covered(R[k])
        assert n == 0, (k, n, worst)
    assert slack(R["c_in"]) <= SLACK_CONTRIB, slack(R["c_in"])


@pytest.fixture(scope="module")
def sample():
    return collect()


def test_sample_is_large_enough(sample):
    """At least 10^4 calm (pixel, surfel) pairs, hundreds of calm pixels and
    thousands of contributions are compared."""
    assert len(sample["a"]) >= 10_000, len(sample["a"])
    assert len(sample["A"]) >= 500 and len(sample["c_in"]) >= 10_000, (len(sample["A"]), len(sample["c_in"]))


def test_local_coordinates_depth_and_opacity_within_the_pair_bounds(sample):
    """fp32_unc (u, v, t) and opacity_unc (a) bound a binary32 evaluation of
    every calm pair, with a median slack of at most 40."""
    pin_pairs(sample)


def test_pixel_opacity_and_depth_within_the_pixel_bounds(sample):
    """eA and eD bound the binary32 compositing of every calm pixel."""
    pin_pixels(sample)


def test_transmittance_and_contributions_within_their_bounds(sample):
    """eT bounds the transmittance recovered backwards from the final one;
    twice contrib_unc bounds a contribution evaluated from binary32 inputs
    (and, with 1e-5 of the majorant, from a binary32 suffix too)."""
    pin_contributions(sample)


# --- closed forms ---------------------------------------------------------------
def _single_surfel(q_target, alpha=0.6, s_u=0.1, s_v=0.07, rng_m=5.0, r=16, c=10):
    """One surfel facing the ray of pixel (r, c) of a 32 x 64 frame, its centre
    moved along its first tangent axis so that the ray meets its plane at
    u = -sqrt(q_target), v = 0 (so q = q_target up to the binary32 inputs)."""
    frame = scenes.Frame(32, 64, 16, 16, -0.5, 0.5)
    emin, emax = float(np.float32(frame.elev_min)), float(np.float32(frame.elev_max))
    th = emax - (r + 0.5) * (emax - emin) / frame.H
    ph = (c + 0.5) * 2.0 * math.pi / frame.W
    d = np.array([math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), math.sin(th)])
    tu = np.cross(d, [0.0, 0.0, 1.0])
    tu /= np.linalg.norm(tu)
    n = -d
    tv = np.cross(n, tu)
    mean = rng_m * d + math.sqrt(q_target) * s_u * tu
    R = np.column_stack([tu, tv, n])[None]
    surf = scenes.Surfels(mean[None].astype(np.float32), scenes.rot_to_quat(R).astype(np.float32),
                          np.log([[s_u, s_v]]).astype(np.float32),
                          np.array([math.log(alpha / (1 - alpha))], np.float32))
    return surf, frame


def test_flip_term_equals_the_would_be_contribution():
    """A surfel just outside the 3-sigma cut-off (q = 9 (1 + 1e-4), within the
    near-threshold band): the pixel's opacity bound is its would-be opacity
    alpha e^(-q/2) (to its own binary32 uncertainty, 1e-4 relative), and its logit
    gradient bound, with dL/dA = 1, is the would-be dA/dlogit =
    e^(-q/2) alpha (1 - alpha)."""
    check_flip_closed_form(None)


def check_flip_closed_form(lib):
    surf, frame = _single_surfel(9.0 * (1 + 1e-4))
    b = O.bin_frame(surf, frame)
    d = O.pixel_detail(surf, frame, b["ranges"], b["vals"], 16, 10, lib=lib)
    assert d["nc"] == 0 and len(d["item"]) == 1 and d["flags"][0] & 4, d     # FL_QCUT
    alpha = 1.0 / (1.0 + math.exp(-float(surf.logit[0])))
    G = math.exp(-0.5 * d["q"][0])
    assert d["eA"] == pytest.approx(alpha * G, rel=3e-4)
    gA = np.zeros((frame.H, frame.W))
    gA[16, 10] = 1.0
    g = O.render_bwd(surf, frame, b["ranges"], b["vals"], gA, np.zeros_like(gA), np.zeros((3,) + gA.shape),
                     params64=None, grads=None) if lib is None else _bwd_with(lib, surf, frame, b, gA)
    assert g["flip"][0, 9] == pytest.approx(G * alpha * (1 - alpha), rel=1e-9)


def _bwd_with(lib, surf, frame, b, gA):
    """render_bwd through a variant build of the oracle."""
    n = surf.n
    g = dict(mean=np.zeros((n, 3)), quat=np.zeros((n, 4)), log_scale=np.zeros((n, 2)), logit=np.zeros(n),
             abs=np.zeros((n, 10)), flip=np.zeros((n, 10)))
    m, q, ls, lg = O._params64(surf)
    fa = O._frame_args(frame)
    gSt = np.zeros_like(gA)
    gSn = np.zeros((3,) + gA.shape)
    lib.lgso_render_bwd(O._p(m), O._p(q), O._p(ls), O._p(lg), n, *fa[:6], O._p(fa[6]),
                        O._p(O._c(b["ranges"], np.int64)), O._p(O._c(b["vals"], np.uint32)),
                        O._p(O._c(gA, np.float64)), O._p(gSt), O._p(gSn), O._p(g["mean"]), O._p(g["quat"]),
                        O._p(g["log_scale"]), O._p(g["logit"]), O._p(g["abs"]), O._p(g["flip"]), 0)
    return g


def check_majorant_closed_form(lib):
    surf, frame = _single_surfel(0.25)
    b = O.bin_frame(surf, frame)
    gA = np.zeros((frame.H, frame.W))
    gA[16, 10] = 1.0
    g = _bwd_with(lib, surf, frame, b, gA) if lib is not None else O.render_bwd(
        surf, frame, b["ranges"], b["vals"], gA, np.zeros_like(gA), np.zeros((3,) + gA.shape))
    # the only upstream gradient is dL/dA = 1 at one pixel: the logit term has
    # no cancellation, so its majorant is the gradient itself
    assert g["logit"][0] > 0
    assert g["abs"][0, 9] == pytest.approx(g["logit"][0], rel=1e-12)
    # and the majorant never lies below the gradient it bounds
    raw = np.concatenate([g["mean"][0], g["quat"][0], g["log_scale"][0], [g["logit"][0]]])
    assert np.all(g["abs"][0] >= np.abs(raw) * (1 - 1e-12))


def test_majorant_equals_the_gradient_without_cancellation():
    """A single facing surfel with dL/dA = 1 at one pixel: its logit
    gradient is one positive product, which its majorant equals; every
    component's majorant is at least the gradient's magnitude."""
    check_majorant_closed_form(None)


def test_decisions_taken_the_other_way_stay_inside_the_pixel_bound():
    """A surfel swept across the 3-sigma cut-off in steps of 1e-7 of q:
    wherever the binary32 restatement keeps it while FP64 drops it (or the
    reverse), the pixel's opacity still differs by no more than eA."""
    flipped = 0
    for k in range(-60, 61):
        surf, frame = _single_surfel(9.0 * (1 + 1e-7 * k))
        b = O.bin_frame(surf, frame)
        d = O.pixel_detail(surf, frame, b["ranges"], b["vals"], 16, 10)
        rec = F.records(surf, frame, d["item"].astype(np.int64))
        e = F.evaluate(rec, F.rays(frame, 16, 10))
        A, _, _, _, _, _ = F.composite(e, rec, range(len(d["item"])))
        flipped += bool(e["valid"][0]) != bool(d["valid"][0])
        assert abs(float(A) - d["A"]) <= d["eA"], (k, float(A), d["A"], d["eA"])
    assert flipped > 0


# --- planted mistakes -------------------------------------------------------------
PLANTS = ["PLANT_EK", "PLANT_DT", "PLANT_OPA", "PLANT_EA", "PLANT_ED", "PLANT_CONTRIB", "PLANT_FLIP", "PLANT_MAJOR"]


def _fails(fn, *a):
    try:
        fn(*a)
    except AssertionError:
        return True
    return False


def test_a_planted_mistake_in_every_bound_is_caught():
    """Each bound scaled by 10 (too loose) and by 1/10 (too tight) in its own
    build of the oracle: some pin fails for every one of the 16 variants."""
    missed = []
    with tempfile.TemporaryDirectory() as tmp:
        for name in PLANTS:
            for factor in (10.0, 0.1):
                lib = O.variant([f"{name}={factor}"], os.path.join(tmp, f"v_{name}_{factor}.so"))
                if name == "PLANT_FLIP":
                    caught = _fails(check_flip_closed_form, lib)
                elif name == "PLANT_MAJOR":
                    caught = _fails(check_majorant_closed_form, lib)
                else:
                    R = collect(lib=lib, small=True, pixels=160, street_pixels=0, seed=1)
                    caught = (_fails(pin_pairs, R) or _fails(pin_pixels, R) or _fails(pin_contributions, R))
                if not caught:
                    missed.append((name, factor))
    assert not missed, missed
