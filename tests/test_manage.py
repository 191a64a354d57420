"""Map management on the device (control score, Sec. 3.3 Eq. controlscore;
opacity prune; multi-pass planar cover-and-prune and adaptive split, Sec.
3.5) against the oracle, through the C-ABI: every output bit-exact (the
decisions and the children's parameters are specified in binary32), on
clustered maps with ragged sizes, the street map, degenerate parameters and
the empty map; determinism across runs; carrying per-surfel arrays over."""
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
def mg():
    from oracle import manage, oracle
    oracle.build()
    return manage


def _run(arrays, **kw):
    import torch
    from paper_2607_04127_gb300 import manage
    dev = torch.device("cuda")
    mean, quat, ls, logit, lam, res = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in arrays)
    m = manage.MapManager(dev)
    out = m.launch([mean, quat, ls, logit], lam, res, manage.params(**kw))
    torch.cuda.synchronize()
    cnt = out["counts"].cpu().numpy()
    k = int(cnt[0])
    host = {key: out[key][:k].cpu().numpy() for key in ("mean", "quat", "log_scale", "logit", "src", "role")}
    host["score"] = out["score"][: len(arrays[3])].cpu().numpy()
    host["counts"] = cnt
    return host, m, out


def _compare(mg, arrays, **kw):
    got, _, _ = _run(arrays, **kw)
    P = mg.Params(**kw)
    want = mg.manage(*arrays, P)
    assert got["counts"].tolist() == want["counts"].tolist()
    assert np.array_equal(got["score"].view(np.uint32), want["score"].view(np.uint32))
    assert np.array_equal(got["src"], want["src"]) and np.array_equal(got["role"], want["role"])
    for key in ("mean", "quat", "log_scale", "logit"):
        assert np.array_equal(got[key].view(np.uint32), want[key].view(np.uint32)), key
    return want


@pytest.mark.parametrize("seed,n", [(0, 1), (1, 2), (2, 150), (3, 3001), (4, 40_000)])
def test_clustered_maps_bit_exact(mg, seed, n):
    want = _compare(mg, scenes.manage_cluster(seed, n), voxel=0.5, q_plane=0.5, q_cover=0.6, prune_cap=0.1,
                    q_split=0.9, split_cap=0.05)
    if n >= 3000:
        assert want["counts"][2:5].min() > 0 and want["counts"][5] > 0


def test_street_map_bit_exact(mg):
    """The 200k-surfel street map with signals from its own k-NN covariances
    and the library's default parameters."""
    surf, _, _ = scenes.street()
    lam, res = scenes.manage_signals(surf.mean)
    want = _compare(mg, (surf.mean, surf.quat, surf.log_scale, surf.logit, lam, res))
    assert want["counts"][2] > 0 and want["counts"][5] > 0


@pytest.mark.parametrize("kw", [
    dict(n_passes=0),
    dict(q_cover=0.0),
    dict(q_cover=1.0, prune_cap=1.0, slab=1e9),
    dict(prune_cap=0.0, split_cap=0.0),
    dict(q_plane=1.0, q_split=0.0, split_cap=1.0),
    dict(alpha_min=0.999, alpha_prune=0.9),
    dict(voxel=1e-3),
    dict(voxel=1e6, n_passes=1),
])
def test_degenerate_parameters(mg, kw):
    _compare(mg, scenes.manage_cluster(7, 2000), **kw)


def test_ties_and_duplicates(mg):
    """Equal scores, equal logits and coincident means: ties go by index on
    both sides."""
    mean, quat, ls, logit, lam, res = scenes.manage_cluster(8, 1500)
    mean[::3] = mean[0]
    logit[::2] = logit[1]
    lam[::4] = lam[2]
    res[::5] = 0.0
    _compare(mg, (mean, quat, ls, logit, lam, res), voxel=0.7, q_plane=0.8, q_cover=0.9, prune_cap=0.3,
             q_split=0.5, split_cap=0.2)


def test_empty_map(mg):
    z3 = np.zeros((0, 3), np.float32)
    got, _, _ = _run((z3, np.zeros((0, 4), np.float32), np.zeros((0, 2), np.float32), np.zeros(0, np.float32), z3,
                      np.zeros(0, np.float32)))
    assert got["counts"].tolist() == [0] * 6


def test_deterministic_and_gather(mg):
    """Two runs give identical bits; per-surfel arrays follow src, children's
    rows zeroed on request."""
    import torch
    arrays = scenes.manage_cluster(9, 20_000)
    kw = dict(voxel=0.5, q_plane=0.5, q_cover=0.6, prune_cap=0.1, q_split=0.8, split_cap=0.1)
    a, m, out = _run(arrays, **kw)
    b, _, _ = _run(arrays, **kw)
    for key in a:
        assert np.array_equal(a[key], b[key]), key
    n = len(arrays[3])
    mom = torch.arange(n * 10, dtype=torch.float32, device="cuda").reshape(n, 10)
    g0, g1 = m.gather(out, [mom, mom], zero_children=True)
    torch.cuda.synchronize()
    k = int(a["counts"][0])
    src, role = a["src"], a["role"]
    want = mom.cpu().numpy()[src]
    want[role != 0] = 0
    assert np.array_equal(g0[:k].cpu().numpy(), want)
    m.gather(out, [mom], zero_children=False)[0]
    g2 = m.gather(out, [mom], zero_children=False)[0]
    torch.cuda.synchronize()
    assert np.array_equal(g2[:k].cpu().numpy(), mom.cpu().numpy()[src])


def test_step_api_round_trip(mg):
    """MapManager.step returns the new map sliced to its size and the carried
    arrays, matching the oracle."""
    import torch
    from paper_2607_04127_gb300 import manage
    arrays = scenes.manage_cluster(10, 5000)
    dev = torch.device("cuda")
    t = [torch.from_numpy(x).to(dev) for x in arrays]
    new, carried, info = manage.MapManager(dev).step(t[:4], t[4], t[5], manage.params(q_split=0.8),
                                                     carry=[t[0].contiguous()])
    want = mg.manage(*arrays, mg.Params(q_split=0.8))
    assert info["counts"] == want["counts"].tolist()
    assert np.array_equal(new[0].cpu().numpy(), want["mean"])
    c = carried[0].cpu().numpy()
    keep = want["role"] == 0
    assert np.array_equal(c[keep], arrays[0][want["src"][keep]]) and np.all(c[~keep] == 0)
