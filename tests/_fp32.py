"""A plain binary32 restatement of the compositing arithmetic (test
infrastructure for the allowance pins).

Every operation is one binary32 rounding (NumPy float32 arithmetic), with a
fused multiply-add where the compositing kernels fuse explicitly (the dot
products with the ray, the local coordinates, u^2 + v^2, the running sums):
the kind of evaluation the oracle's binary32 allowance claims to bound.  It
follows the paper's representation (Sec. 3.1: a surfel's plane, its
Gaussian in the local coordinates, alpha compositing front to back) and the
readings the oracle states; it is written from those definitions, not from
either implementation, and it is not bit-exact to the GPU (whose compiler may
fuse other products), only a binary32 evaluation of the same inputs.
"""
from __future__ import annotations

import math

import numpy as np

f32 = np.float32


def fma(a, b, c):
    """a b + c with one rounding to binary32 (the product is exact in
    binary64; the sum is rounded there and then to binary32, which matches a
    true fused operation except in rare double-rounding ties)."""
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(f32)


def rays(frame, r, c):
    """Unit ray of pixel (r, c) in binary32: elevation emax - (r + 1/2)
    (emax - emin)/H, azimuth pi (2c + 1)/W, each trigonometric value the
    correctly rounded binary32 of its binary32 argument."""
    emin, emax = f32(frame.elev_min), f32(frame.elev_max)
    th = emax - (f32(r) + f32(0.5)) * ((emax - emin) / f32(frame.H))
    x = (f32(2.0) * f32(c) + f32(1.0)) / f32(frame.W)
    st, ct = f32(math.sin(float(th))), f32(math.cos(float(th)))
    sp, cp = f32(math.sin(math.pi * float(x))), f32(math.cos(math.pi * float(x)))
    return np.array([ct * cp, ct * sp, st], f32)


def records(surf, frame, idx):
    """Sensor-frame records of surfels idx in binary32: normal n, h = n.mu,
    a_u = t_u / s_u, b_u = t_u.mu / s_u, a_v, b_v, opacity alpha (the plane
    and local-coordinate form of the paper's surfel)."""
    P = np.asarray(frame.pose, f32).reshape(3, 4)
    R, o = P[:, :3], P[:, 3]
    m = np.asarray(surf.mean, f32)[idx]
    d = m - o
    # mu = R^T (m - o), summed left to right
    mu = np.stack([(R[0, k] * d[:, 0] + R[1, k] * d[:, 1]) + R[2, k] * d[:, 2] for k in range(3)], 1)
    q = np.asarray(surf.quat, f32)[idx]
    inv = f32(1.0) / np.sqrt((q * q).sum(1, dtype=f32))
    w, x, y, z = (q * inv[:, None]).T
    two = f32(2.0)
    one = f32(1.0)
    cols = [
        np.stack([one - two * (y * y + z * z), two * (x * y + w * z), two * (x * z - w * y)], 1),
        np.stack([two * (x * y - w * z), one - two * (x * x + z * z), two * (y * z + w * x)], 1),
        np.stack([two * (x * z + w * y), two * (y * z - w * x), one - two * (x * x + y * y)], 1),
    ]
    sens = [np.stack([(R[0, k] * c[:, 0] + R[1, k] * c[:, 1]) + R[2, k] * c[:, 2] for k in range(3)], 1)
            for c in cols]
    tu, tv, n = sens
    ls = np.asarray(surf.log_scale, f32)[idx]
    isu = np.exp(-ls[:, 0].astype(np.float64)).astype(f32)
    isv = np.exp(-ls[:, 1].astype(np.float64)).astype(f32)
    lg = np.asarray(surf.logit, f32)[idx]
    alpha = (f32(1.0) / (f32(1.0) + np.exp(-lg.astype(np.float64)).astype(f32))).astype(f32)

    def dot(a, b):
        return (a[:, 0] * b[:, 0] + a[:, 1] * b[:, 1]) + a[:, 2] * b[:, 2]
    return dict(n=n, h=dot(n, mu), au=tu * isu[:, None], bu=dot(tu, mu) * isu, av=tv * isv[:, None],
                bv=dot(tv, mu) * isv, alpha=alpha)


NEG_HALF_LOG2E = f32(-0.5 / math.log(2.0))


def evaluate(rec, d):
    """Plane intersection and Gaussian of every record with ray d:
    den = n.d, t = h / den, u = t (a_u.d) - b_u, v likewise, q = u^2 + v^2,
    G = 2^(q (-log2(e)/2)), a = min(alpha G, 0.99), and the skip rules."""
    def dotd(a):
        return fma(a[:, 2], d[2], fma(a[:, 1], d[1], a[:, 0] * d[0]))
    den = dotd(rec["n"])
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        t = rec["h"] * (f32(1.0) / den)
        ud, vd = dotd(rec["au"]), dotd(rec["av"])
        u = fma(t, ud, -rec["bu"])
        v = fma(t, vd, -rec["bv"])
        q = fma(u, u, v * v)
        G = np.exp2((q * NEG_HALF_LOG2E).astype(np.float64)).astype(f32)
    araw = rec["alpha"] * G
    a = np.minimum(araw, f32(0.99))
    valid = (np.abs(den) >= f32(1e-6)) & (t > f32(0.2)) & (q <= f32(9.0)) & (a >= f32(1.0 / 255.0))
    return dict(den=den, t=t, u=u, v=v, q=q, G=G, araw=araw, a=a, valid=valid)


def composite(e, rec, order):
    """Front-to-back compositing over the evaluated entries in list order:
    stop before T (1 - a) < 1e-4, else w = a T, A += w, S_t += w t,
    S_n += w (-sign(n.d)) n, T *= 1 - a.  Returns A, S_t, S_n, T and the
    contributors' positions with T before each."""
    T, A, St = f32(1.0), f32(0.0), f32(0.0)
    Sn = np.zeros(3, f32)
    ck, cT = [], []
    for k in order:
        if not e["valid"][k]:
            continue
        a = e["a"][k]
        Tn = T * (f32(1.0) - a)
        if Tn < f32(1e-4):
            break
        w = a * T
        A = A + w
        St = fma(w, e["t"][k], St)
        ws = -w if e["den"][k] > 0 else w
        Sn = fma(ws, rec["n"][k], Sn)
        ck.append(k)
        cT.append(T)
        T = Tn
    return A, St, Sn, T, ck, cT


def reverse(e, rec, ck, T_final, gA, gSt, gSn):
    """The transmittance before each contributor recovered from the final
    one, T_k = T_{k+1} / (1 - a_k), and the suffix over the later
    contributors S_k = sum_{j>k} w_j (g.c_j), in reverse order; returns
    (T_k, S_k) per contributor in list order."""
    T, S = f32(T_final), f32(0.0)
    Ts, Ss = [], []
    gA, gSt = f32(gA), f32(gSt)
    gS = np.asarray(gSn, f32)
    for k in reversed(ck):
        a = e["a"][k]
        iom = f32(1.0) / (f32(1.0) - a)
        Tk = T * iom
        sg = f32(-1.0) if e["den"][k] > 0 else f32(1.0)
        n = rec["n"][k]
        gc = gA + gSt * e["t"][k] + sg * ((gS[0] * n[0] + gS[1] * n[1]) + gS[2] * n[2])
        w = a * Tk
        Ts.append(Tk)
        Ss.append(S)
        S = fma(w, gc, S)
        T = Tk
    return Ts[::-1], Ss[::-1]
