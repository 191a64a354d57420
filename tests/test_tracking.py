"""Tracking-side targets on the device (paper Sec. 3.2, Eqs. trackable_select,
anisotropy, anisotropy_norm, weight_func) against the oracle: the selection
and the means bit-exact, covariances and weights within the binary32 bounds
derived in the test."""
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
def oracle():
    from oracle import oracle as O
    O.build()
    return O


def _check(oracle, surf, mask, kf, k_min, alpha_min):
    import torch
    from paper_2607_04127_gb300 import render, track
    dev = torch.device("cuda")
    params = render.map_tensors(surf, dev)
    idx, mean, cov, w = track.trackable_targets(params, torch.from_numpy(mask).to(dev), torch.from_numpy(kf).to(dev),
                                                k_min, alpha_min)
    oi, om, oc, ow = oracle.trackable_targets(surf, mask, kf, k_min, alpha_min)
    idx, mean, cov, w = (x.cpu().numpy() for x in (idx, mean, cov, w))
    assert np.array_equal(idx.astype(np.int64), oi)
    assert np.array_equal(mean, surf.mean[oi])
    if not len(oi):
        return
    # covariance: binary32 rotation and scales, each good to a few ulps of the
    # largest eigenvalue
    s = np.exp(surf.log_scale.astype(np.float64))[oi]
    lam = np.maximum(np.maximum(s[:, 0], s[:, 1]) ** 2, 1e-4)
    assert np.all(np.abs(cov - oc) <= 2e-6 * lam[:, None])
    # weight: kappa in binary32 (exp, division: a few ulps), through
    # kappa_bar = (kappa - kmin) / (kmax - kmin) and w = 1 / (kappa_bar + eps)
    kap = s.max(1) / (s.min(1) + 1e-6)
    kmin, kmax = kap.min(), kap.max()
    kb = (kap - kmin) / (kmax - kmin) if kmax > kmin else np.zeros_like(kap)
    dkb = 6e-7 * kmax / max(kmax - kmin, 1e-30)
    tol = ow * dkb / (np.maximum(kb, 0.0) + 1e-6) + 1e-6
    assert np.all(np.abs(w - ow) <= tol)


def test_street_map_targets(oracle):
    """The 200k-surfel street map with random masks, keyframe indices and the
    paper's weight cap; a threshold inside the opacity range."""
    surf, _, _ = scenes.street()
    rng = np.random.default_rng(0)
    mask = (rng.uniform(size=surf.n) < 0.8).astype(np.uint8)
    kf = rng.integers(0, 10, surf.n).astype(np.int32)
    _check(oracle, surf, mask, kf, 3, 0.5)


def test_edge_cases(oracle):
    """Nothing selected, everything selected, one surfel, equal anisotropy
    (every weight the cap) and sizes that leave ragged CTAs."""
    surf, _ = scenes.random_shell(2, 1000)
    ones, zeros = np.ones(surf.n, np.uint8), np.zeros(surf.n, np.int32)
    _check(oracle, surf, np.zeros(surf.n, np.uint8), zeros, 0, 0.2)
    _check(oracle, surf, ones, zeros, 0, 1e-6)
    one = surf.subset(slice(0, 1))
    _check(oracle, one, np.ones(1, np.uint8), np.zeros(1, np.int32), 0, 1e-6)
    same = surf.subset(slice(0, 300))
    same.log_scale[:] = np.log([0.2, 0.1])
    _check(oracle, same, np.ones(300, np.uint8), np.zeros(300, np.int32), 0, 1e-6)
    for n in (255, 257, 4097):
        sub = surf.subset(slice(0, min(n, surf.n)))
        if sub.n < n:
            sub = scenes.random_shell(3, n)[0]
        _check(oracle, sub, (np.arange(sub.n) % 3 != 0).astype(np.uint8), np.zeros(sub.n, np.int32), 0, 0.4)
