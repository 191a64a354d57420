"""Run the CUDA path through the C ABI on seeded inputs and bring the results
back to NumPy (test helper; calls only the binding, never the oracle)."""
import numpy as np

from paper_2607_04127_gb300 import lib

LOSS = dict(lambda_alpha=0.1, lambda_n=1.0, lambda_ng=0.05, lambda_s=10.0, s_max=1.0)


def to_dev(surf):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
            for a in (surf.mean, surf.quat, surf.log_scale, surf.logit)]


def run(maps, frames, targets=None, frame_map=None, tuning=None, read_bins=False, loss=LOSS,
        grads_init=None, session=None, repeat_fwd=1, single=False):
    """maps: list of scenes.Surfels; frames: list of scenes.Frame; targets:
    list of scenes.Target (or None for forward only).  single: one map,
    through the single-map calls (lgs_bin_sort, lgs_render_fwd, lgs_loss,
    lgs_render_bwd) instead of their batch forms."""
    assert not single or len(maps) == 1
    import torch
    dev = torch.device("cuda")
    T = [to_dev(m) for m in maps]
    S = [lib.surfels_struct(*t) for t in T]
    fr = [lib.frame_struct(f) for f in frames]
    fm = list(frame_map) if frame_map is not None else [0] * len(frames)
    sess = session or lib.Session()
    lib.lgs_session_set_tuning(sess.handle, **(tuning or {}))
    stream = torch.cuda.current_stream().cuda_stream
    if single:
        sess.reserve([maps[0].n], fr, fm, max(1024, 4 * maps[0].n))
        lib.lgs_bin_sort(sess.handle, S[0], fr, stream)
        st, req = lib.lgs_session_status(sess.handle)
        if st == lib.LGS_ERR_CAPACITY:          # grow to what the device reported, bin again
            sess.reserve([maps[0].n], fr, fm, req + 1024)
            lib.lgs_bin_sort(sess.handle, S[0], fr, stream)
        sess.check_status()
    else:
        sess.bin_sort(S, fr, fm)
    outs = [lib.alloc_fwd(f, dev) for f in frames]
    for _ in range(repeat_fwd):
        if single:
            lib.lgs_render_fwd(sess.handle, S[0], fr, [o.struct() for o in outs], stream)
        else:
            lib.lgs_render_fwd_batch(sess.handle, S, fr, fm, [o.struct() for o in outs], stream)
    res = dict(fwd=[dict(A=o.A, S_t=o.S_t, S_n=o.S_n, T_final=o.T_final, n_contrib=o.n_contrib) for o in outs])
    if read_bins:
        n_items = sum(maps[fm[f]].n for f in range(len(frames)))
        n_tiles = sum((-(-f.H // f.tile_h)) * (-(-f.W // f.tile_w)) for f in frames)
        res["bins"] = lib.lgs_session_read_bins(sess.handle, n_items, n_tiles)
    if targets is not None:
        F, M = len(frames), len(maps)
        tg = [(torch.from_numpy(t.D).cuda(), torch.from_numpy(np.ascontiguousarray(t.N)).cuda()) for t in targets]
        gp = [dict(dA=torch.zeros(f.H, f.W, device=dev), dS_t=torch.zeros(f.H, f.W, device=dev),
                   dS_n=torch.zeros(3, f.H, f.W, device=dev)) for f in frames]
        loss_out = torch.zeros(1 + lib.LOSS_TERMS * F + M, device=dev)
        grads = []
        for k, t in enumerate(T):
            g = [torch.zeros_like(x) for x in t]
            if grads_init is not None:
                for a, b in zip(g, grads_init[k]):
                    a.copy_(torch.from_numpy(np.asarray(b, np.float32)))
            grads.append(g)
        lp = lib.lgs_loss_params(**loss)
        if single:
            lib.lgs_loss(sess.handle, S[0], fr, [o.struct() for o in outs],
                         [lib.lgs_target(d.data_ptr(), n.data_ptr()) for d, n in tg], lp,
                         [lib.lgs_fwd_grad_out(g["dA"].data_ptr(), g["dS_t"].data_ptr(), g["dS_n"].data_ptr())
                          for g in gp], lib.grad_struct(*grads[0]), loss_out.data_ptr(), stream)
            lib.lgs_render_bwd(sess.handle, S[0], fr, [o.struct() for o in outs],
                               [lib.lgs_fwd_grad(g["dA"].data_ptr(), g["dS_t"].data_ptr(), g["dS_n"].data_ptr())
                                for g in gp], lib.grad_struct(*grads[0]), stream)
        else:
            lib.lgs_loss_batch(sess.handle, S, fr, fm, [o.struct() for o in outs],
                               [lib.lgs_target(d.data_ptr(), n.data_ptr()) for d, n in tg], lp,
                               [lib.lgs_fwd_grad_out(g["dA"].data_ptr(), g["dS_t"].data_ptr(), g["dS_n"].data_ptr())
                                for g in gp],
                               [lib.grad_struct(*g) for g in grads], loss_out.data_ptr(), stream)
            lib.lgs_render_bwd_batch(sess.handle, S, fr, fm, [o.struct() for o in outs],
                                     [lib.lgs_fwd_grad(g["dA"].data_ptr(), g["dS_t"].data_ptr(),
                                                       g["dS_n"].data_ptr()) for g in gp],
                                     [lib.grad_struct(*g) for g in grads], stream)
        res["loss"] = loss_out
        res["upstream"] = gp
        res["grads"] = grads
    torch.cuda.synchronize()
    res["counters"] = lib.lgs_session_counters(sess.handle)
    sess.check_status()
    res = _np(res)
    if session is None:
        sess.close()
    return res


def _np(x):
    import torch
    if isinstance(x, torch.Tensor):
        return x.detach().cpu().numpy()
    if isinstance(x, dict):
        return {k: _np(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return type(x)(_np(v) for v in x)
    return x
