"""The mapping loop (Sec. 3.4): Adam on the device against the oracle's Adam,
the autograd path against the fused path, convergence of a small window, and
the window's gradients against the oracle and its central differences on a
500-surfel subset of the street track."""
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


def test_adam_kernel_matches_oracle(oracle):
    import torch
    from paper_2607_04127_gb300 import render
    rng = np.random.default_rng(5)
    n = 3000
    shapes = [(n, 3), (n, 4), (n, 2), (n,)]
    p = [rng.normal(size=s).astype(np.float32) for s in shapes]
    m = np.concatenate([rng.normal(size=s).ravel() * 1e-3 for s in shapes]).astype(np.float32)
    v = np.concatenate([rng.uniform(0, 1e-5, size=s).ravel() for s in shapes]).astype(np.float32)
    lr = (1e-3, 2e-3, 5e-3, 7e-3)
    P = [torch.from_numpy(x).cuda() for x in p]
    M, V = torch.from_numpy(m).cuda(), torch.from_numpy(v).cuda()
    ref_p = [x.astype(np.float64) for x in p]
    moved = [np.zeros(x.shape) for x in p]          # sum of |update| per parameter
    ref_m, ref_v = m.astype(np.float64), v.astype(np.float64)
    for t in (1, 2, 3):
        g = [(rng.normal(size=s) * 10.0 ** rng.uniform(-4, 0, size=s)).astype(np.float32) for s in shapes]
        G = [torch.from_numpy(x).cuda() for x in g]
        render.adam_step(P, G, M, V, t, lr=lr)
        off = 0
        for k, s in enumerate(shapes):
            cnt = int(np.prod(s))
            sl = slice(off, off + cnt)
            # the kernel takes lr, the betas and eps as binary32: so does the oracle here
            f32 = lambda x: float(np.float32(x))
            pn, mn, vn = oracle.adam(ref_p[k].reshape(-1), g[k].reshape(-1).astype(np.float64), ref_m[sl],
                                     ref_v[sl], t, f32(lr[k]), f32(0.9), f32(0.999), f32(1e-15))
            moved[k] += np.abs(pn.reshape(s) - ref_p[k])
            ref_p[k], ref_m[sl], ref_v[sl] = pn.reshape(s), mn, vn
            off += cnt
        assert all(float(G[k].abs().max()) == 0.0 for k in range(4))   # zero_grad
    torch.cuda.synchronize()
    off = 0
    for k, s in enumerate(shapes):
        cnt = int(np.prod(s))
        gp = P[k].cpu().numpy().astype(np.float64)
        # binary32: each update to a few ulps of its size, each rounding of p
        assert np.all(np.abs(gp - ref_p[k]) <= 1e-5 * moved[k] + 3 * 2.0 ** -23 * (np.abs(ref_p[k]) + moved[k])), k
        off += cnt
    # moments: a few binary32 roundings of terms of at most their largest size
    assert np.allclose(M.cpu().numpy(), ref_m, rtol=1e-6, atol=1e-6 * np.abs(ref_m).max())
    assert np.allclose(V.cpu().numpy(), ref_v, rtol=1e-6, atol=1e-6 * np.abs(ref_v).max())


def test_adam_batch_equals_per_map_steps():
    """One fused launch over maps of uneven size, each at its own step count,
    gives bit-identical parameters, moments and zeroed gradients to one
    single-map launch per map (same binary32 arithmetic per element)."""
    import torch
    from paper_2607_04127_gb300 import render
    sizes, steps = (1000, 37, 5000, 1), (1, 4, 2, 9)
    lrs = [(1e-3, 2e-3, 5e-3, 7e-3), (2e-3, 1e-3, 1e-2, 5e-3), (1e-3, 1e-3, 5e-3, 5e-3), (3e-3, 3e-3, 3e-3, 3e-3)]
    runs = []
    for _ in range(2):
        items = []
        for n, t, lr in zip(sizes, steps, lrs):
            r = np.random.default_rng(n)
            P = [torch.from_numpy(r.normal(size=s).astype(np.float32)).cuda() for s in ((n, 3), (n, 4), (n, 2), (n,))]
            G = [torch.from_numpy(r.normal(size=x.shape).astype(np.float32)).cuda() for x in P]
            M = torch.from_numpy(r.normal(size=10 * n).astype(np.float32) * 1e-3).cuda()
            V = torch.from_numpy(r.uniform(0, 1e-5, size=10 * n).astype(np.float32)).cuda()
            items.append((P, G, M, V, t, lr))
        runs.append(items)
    render.adam_step_batch(runs[0], zero_grad=True)
    for P, G, M, V, t, lr in runs[1]:
        render.adam_step(P, G, M, V, t, lr=lr, zero_grad=True)
    torch.cuda.synchronize()
    for a, b in zip(*runs):
        for x, y in zip(a[0] + a[1] + [a[2], a[3]], b[0] + b[1] + [b[2], b[3]]):
            assert torch.equal(x, y)
        assert all(float(g.abs().max()) == 0.0 for g in a[1])


def _window():
    surf, f0, t0 = scenes.box_room(seed=0)
    f1 = scenes.Frame(32, 512, 16, 16, f0.elev_min, f0.elev_max, scenes.pose_matrix(0.4, (1.0, 0.5, 2.3)))
    _, _, t1 = scenes.box_room(seed=0, yaw=0.4)
    # start away from the optimum: shifted centres, shrunk scales, lower opacity
    rng = np.random.default_rng(8)
    start = surf.copy()
    start.mean = (surf.mean + rng.normal(0, 0.05, surf.mean.shape)).astype(np.float32)
    start.log_scale = (surf.log_scale - 0.3).astype(np.float32)
    start.logit = (surf.logit - 0.5).astype(np.float32)
    return start, [f0, f1], [t0, t1]


@pytest.mark.parametrize("lambda_ns", [0.0, 0.01])
def test_autograd_path_equals_fused_path(oracle, lambda_ns):
    from paper_2607_04127_gb300 import mapping, render
    surf, frames, targets = _window()
    lp = render.LossParams(lambda_ns=lambda_ns)
    a = mapping.MappingWindow(surf, frames, targets, autograd=True, loss=lp)
    b = mapping.MappingWindow(surf, frames, targets, autograd=False, loss=lp)
    La, ga = a.loss_and_grads()
    Lb, gb = b.loss_and_grads()
    assert float(La) == float(Lb)
    for x, y in zip(ga, gb):
        x, y = x.cpu().numpy(), y.cpu().numpy()
        assert np.allclose(x, y, rtol=1e-5, atol=1e-6 * np.abs(y).max())
    a.close()
    b.close()


@pytest.mark.parametrize("autograd", [True, False])
def test_window_loss_decreases(oracle, autograd):
    from paper_2607_04127_gb300 import mapping
    surf, frames, targets = _window()
    w = mapping.MappingWindow(surf, frames, targets, autograd=autograd)
    L = w.run(10).cpu().numpy()
    assert np.all(np.isfinite(L))
    assert L[-1] < 0.95 * L[0] and np.sum(np.diff(L) < 0) >= 8, L
    w.close()


def test_surface_normal_term_switched_on_mid_run(oracle):
    """The N_surf term enters once switched on (as after densification): every
    frame reports a positive L_ns and the loss keeps decreasing."""
    from paper_2607_04127_gb300 import mapping, render
    surf, frames, targets = _window()
    w = mapping.MappingWindow(surf, frames, targets, autograd=False)
    L0 = w.run(5).cpu().numpy()
    w.set_loss_params(render.LossParams(lambda_ns=0.01))
    L1 = w.run(10).cpu().numpy()
    terms = w.rast.loss_out.cpu().numpy()[1:9].reshape(2, 4)
    assert np.all(terms[:, 3] > 0)
    assert np.all(np.isfinite(L0)) and np.all(np.isfinite(L1))
    assert L1[-1] < L1[0] and np.sum(np.diff(L1) < 0) >= 7, L1
    w.close()


def test_track_subset_gradients_vs_oracle_and_differences(oracle):
    """500 surfels of the street track seen from two keyframes (128 x 1024,
    8 x 8 tiles): the window's gradient (autograd path) equals the oracle's
    within the parity bars, and the oracle's matches central differences
    (step 1e-4) of its FP64 loss on coordinates whose probes cross no
    discontinuity (contributor sets, the depth L1 kink)."""
    from paper_2607_04127_gb300 import mapping
    from tests.test_gpu_parity import compare_grads, assert_grads, oracle_grads
    surf, frames, targets = scenes.street_track(seed=1, n=40_000, n_keyframes=2, length=60.0)
    frames = [f.with_tiles(8, 8) for f in frames]
    # the subset: 500 surfels within 25 m of the first keyframe
    o = frames[0].pose.reshape(3, 4)[:, 3]
    near = np.flatnonzero(np.linalg.norm(surf.mean - o, axis=1) < 25.0)
    sub = surf.subset(np.sort(np.random.default_rng(2).choice(near, 500, replace=False)))
    w = mapping.MappingWindow(sub, frames, targets, autograd=True)
    L, g = w.loss_and_grads()
    gg = [x.detach().cpu().numpy() for x in g]
    # oracle with the GPU's own upstream planes (the loss is checked elsewhere)
    ups = [(u[0].cpu().numpy().astype(np.float64), u[1].cpu().numpy().astype(np.float64),
            u[2].cpu().numpy().astype(np.float64)) for u in w.rast.up]
    og = oracle_grads(oracle, sub, frames, ups)
    assert_grads(compare_grads(gg, og))
    Lo, _, go, _ = oracle.forward_backward(sub, frames, [(t.D, t.N) for t in targets])
    assert float(L) == pytest.approx(Lo, rel=1e-5)
    # central differences of the oracle's loss, step 1e-4
    base = [np.ascontiguousarray(a, np.float64).copy() for a in (sub.mean, sub.quat, sub.log_scale, sub.logit)]
    gl = [go["mean"], go["quat"], go["log_scale"], go["logit"]]
    _, fw0, _, _ = oracle.forward_backward(sub, frames, [(t.D, t.N) for t in targets], params64=base)
    def l1_sign(fw, tgt):
        # the side of the depth L1 kink of every measured pixel
        return np.sign(fw["S_t"] / (fw["A"] + 1e-6) - tgt.D) * (tgt.D > 0)

    rng = np.random.default_rng(3)
    used = 0
    mags = np.concatenate([np.abs(x).ravel() for x in gl])
    for _ in range(40):
        which = int(rng.integers(4))
        big = np.argwhere(np.abs(gl[which]) > 1e-2 * mags.max())
        if len(big) == 0:
            continue
        idx = tuple(big[int(rng.integers(len(big)))])
        fds, same = [], True
        for h in (1e-4, 5e-5):
            vals = []
            for sgn in (1, -1):
                p = [a.copy() for a in base]
                p[which][idx] += sgn * h
                Lp, fw, _, _ = oracle.forward_backward(sub, frames, [(t.D, t.N) for t in targets], params64=p)
                vals.append(Lp)
                same &= all(np.array_equal(a["n_contrib"], b["n_contrib"]) and
                            np.array_equal(a["n_valid"], b["n_valid"]) and
                            np.array_equal(l1_sign(a, t), l1_sign(b, t)) for a, b, t in zip(fw, fw0, targets))
            fds.append((vals[0] - vals[1]) / (2 * h))
        if not same:
            continue
        # the O(h^2) truncation of the step-1e-4 difference, estimated from
        # the half step, is part of the bar
        trunc = abs(fds[0] - fds[1]) * 4.0 / 3.0
        an = gl[which][idx]
        assert abs(an - fds[0]) <= 1e-3 * max(abs(fds[0]), 1e-3 * mags.max()) + trunc, (which, idx, an, fds)
        used += 1
    assert used >= 15, used
    w.close()


def test_window_grows_and_budgets_its_map_on_the_device(oracle):
    """A box-room window takes a keyframe scan of the room from another pose
    (lgs_keyframe_init: the new surfels join with zero Adam moments), then one
    map-management step (lgs_map_manage, lgs_map_gather): every row of the
    new map carries the moments of its source row, children start at zero,
    the source mapping equals the oracle's management of the same map and
    signals, and two more iterations give a finite loss with the session's
    status OK."""
    import torch
    from oracle import manage as omg
    from paper_2607_04127_gb300 import mapping
    surf, frame, tgt = scenes.box_room()
    win = mapping.MappingWindow(surf, [frame], [tgt], autograd=False)
    win.run(3)
    # a scan of the same room from 1 m aside, as points in its sensor frame
    rng = np.random.default_rng(3)
    pose = scenes.pose_matrix(0.3, (1.0, -0.5, 2.0))
    kf = scenes.Frame(32, 512, 16, 16, -math.radians(15), math.radians(15), pose)
    _, pw, _, valid = scenes.simulate_scan(scenes.Scene(room=(-10.0, 10.0, -10.0, 10.0, 0.0, 5.0)), kf, rng)
    P = np.asarray(pose, np.float64).reshape(3, 4)
    pts = ((pw.reshape(-1, 3)[valid.reshape(-1)] - P[:, 3]) @ P[:, :3]).astype(np.float32)
    n0 = win.n
    m0, v0 = win.m.clone(), win.v.clone()
    win.insert_keyframe(torch.from_numpy(pts).cuda(), P.reshape(-1))
    n1 = win.n
    assert n1 == n0 + len(pts)
    # the old rows keep their moments, the new ones start at zero
    for old, new in ((m0, win.m), (v0, win.v)):
        for a, b in zip(mapping.state_blocks(old, n0), mapping.state_blocks(new, n1)):
            assert torch.equal(b[:n0], a) and not b[n0:].any()
    win.run(1)
    # management with signals from the map's own neighbourhoods
    host = [p.detach().cpu().numpy() for p in win.params]
    lam, res = scenes.manage_signals(host[0])
    m1, v1 = win.m.clone(), win.v.clone()
    counts, src = win.manage(torch.from_numpy(lam).cuda(), torch.from_numpy(res).cuda())
    want = omg.manage(*host, lam, res, omg.Params())
    src = src.cpu().numpy()
    assert counts == want["counts"].tolist() and np.array_equal(src, want["src"])
    child = want["role"] != 0
    for old, new in ((m1, win.m), (v1, win.v)):
        for a, b in zip(mapping.state_blocks(old, n1), mapping.state_blocks(new, counts[0])):
            a, b = a.cpu().numpy(), b.cpu().numpy()
            assert np.array_equal(b[~child], a[src[~child]]) and not b[child].any()
    L = win.run(2)
    assert torch.isfinite(L).all()
    win.rast.session.check_status()
    win.close()
