"""lgs_image_loss_noalloc (static scratch, no session, no workspace) against
the session loss lgs_loss on the same rendered frames: identical image terms
and gradient planes, on two calls in a row.  Collected last on purpose: it
must also pass after every other test has used the library."""
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


def _setup():
    import torch
    from paper_2607_04127_gb300 import lib
    from tests import _gpu
    surf, f0, t0 = scenes.box_room(seed=0)
    f1 = scenes.Frame(32, 512, 16, 16, f0.elev_min, f0.elev_max, scenes.pose_matrix(0.4, (1.0, 0.5, 2.3)))
    _, _, t1 = scenes.box_room(seed=0, yaw=0.4)
    frames, targets = [f0, f1], [t0, t1]
    dev = torch.device("cuda")
    T = _gpu.to_dev(surf)
    S = [lib.surfels_struct(*T)]
    fr = [lib.frame_struct(f) for f in frames]
    sess = lib.Session()
    sess.bin_sort(S, fr, [0, 0])
    outs = [lib.alloc_fwd(f, dev) for f in frames]
    stream = torch.cuda.current_stream().cuda_stream
    lib.lgs_render_fwd_batch(sess.handle, S, fr, [0, 0], [o.struct() for o in outs], stream)
    tg = [(torch.from_numpy(t.D).cuda(), torch.from_numpy(np.ascontiguousarray(t.N)).cuda()) for t in targets]
    return sess, S, fr, frames, outs, tg, stream


def _planes(frames, dev):
    import torch
    return [dict(dA=torch.full((f.H, f.W), 7.0, device=dev), dS_t=torch.full((f.H, f.W), 7.0, device=dev),
                 dS_n=torch.full((3, f.H, f.W), 7.0, device=dev)) for f in frames]


def test_noalloc_loss_equals_session_loss():
    import torch
    from paper_2607_04127_gb300 import lib
    from tests._gpu import LOSS
    sess, S, fr, frames, outs, tg, stream = _setup()
    dev = torch.device("cuda")
    F = len(frames)
    lp = lib.lgs_loss_params(**LOSS)
    targets = [lib.lgs_target(d.data_ptr(), n.data_ptr()) for d, n in tg]
    # the session loss
    gs = _planes(frames, dev)
    Ls = torch.zeros(1 + 4 * F + 1, device=dev)
    lib.lgs_loss_batch(sess.handle, S, fr, [0, 0], [o.struct() for o in outs], targets, lp,
                       [lib.lgs_fwd_grad_out(g["dA"].data_ptr(), g["dS_t"].data_ptr(), g["dS_n"].data_ptr())
                        for g in gs], None, Ls.data_ptr(), stream)
    torch.cuda.synchronize()
    for call in range(2):            # two calls in a row on the same scratch
        gn = _planes(frames, dev)
        Ln = torch.full((1 + 3 * F,), -1.0, device=dev)
        lib.lgs_image_loss_noalloc([(f.H, f.W) for f in frames], [o.struct() for o in outs], targets, lp,
                                   [lib.lgs_fwd_grad_out(g["dA"].data_ptr(), g["dS_t"].data_ptr(),
                                                         g["dS_n"].data_ptr()) for g in gn],
                                   Ln.data_ptr(), stream)
        torch.cuda.synchronize()
        ln, ls = Ln.cpu().numpy(), Ls.cpu().numpy()
        terms = ls[1:1 + 4 * F].reshape(F, 4)      # (L_depth, L_alpha, L_ng, L_ns): no N_surf term here
        assert np.array_equal(ln[1:].reshape(F, 3), terms[:, :3]) and np.all(terms[:, 3] == 0), call
        for a, b in zip(gn, gs):
            for k in ("dA", "dS_t", "dS_n"):
                assert torch.equal(a[k], b[k]), (call, k)
        t = terms[:, :3].astype(np.float64)
        img = np.mean(t[:, 0] + LOSS["lambda_alpha"] * t[:, 1] + LOSS["lambda_n"] * LOSS["lambda_ng"] * t[:, 2])
        assert ln[0] == pytest.approx(img, rel=1e-6), call
    sess.close()


def test_noalloc_rejects_more_frames_than_the_scratch_holds():
    import torch
    from paper_2607_04127_gb300 import lib
    n = 9
    dummy = torch.zeros(4, device="cuda")
    p = dummy.data_ptr()
    with pytest.raises(lib.LgsError, match="static scratch"):
        lib.lgs_image_loss_noalloc([(1, 1)] * n, [lib.lgs_fwd_out(p, p, p, p, p)] * n, [lib.lgs_target(p, p)] * n,
                                   lib.lgs_loss_params(0.1, 1.0, 0.05, 10.0, 1.0),
                                   [lib.lgs_fwd_grad_out(p, p, p)] * n, p, torch.cuda.current_stream().cuda_stream)
