"""Host logic of growing and budgeting a mapping window's map (no device):
keyframe surfels are appended with zero Adam moments, and a map-management
step carries each surfel's moments to its new row (children start at zero),
in the Adam state's group-major layout [mean 3n | quat 4n | log-scale 2n |
logit n].  The device calls are replaced by CPU fakes with the same
contracts (their own parity is checked on the GPU elsewhere)."""
import torch

from paper_2607_04127_gb300 import keyframe, manage, mapping


def _window(n, autograd=False):
    w = object.__new__(mapping.MappingWindow)
    g = torch.Generator().manual_seed(n)
    w.device = torch.device("cpu")
    w.params = [torch.randn(n, 3, generator=g), torch.randn(n, 4, generator=g), torch.randn(n, 2, generator=g),
                torch.randn(n, generator=g)]
    w.m = torch.arange(10 * n, dtype=torch.float32) + 1
    w.v = -(torch.arange(10 * n, dtype=torch.float32) + 1)
    w.autograd = autograd
    w.t = 3
    w.grads = None if autograd else [torch.zeros_like(p) for p in w.params]
    w._check_next = False
    w._manager = None
    return w


def test_state_blocks_round_trip():
    s = torch.arange(50, dtype=torch.float32)
    b = mapping.state_blocks(s, 5)
    assert [tuple(x.shape) for x in b] == [(5, 3), (5, 4), (5, 2), (5, 1)]
    assert b[1][0].tolist() == [15, 16, 17, 18] and b[3][:, 0].tolist() == [45, 46, 47, 48, 49]
    assert torch.equal(mapping.state_from_blocks(b), s)


def test_insert_keyframe_appends_with_zero_moments(monkeypatch):
    n, k = 5, 3
    w = _window(n)
    old = [p.clone() for p in w.params]
    m0, v0 = w.m.clone(), w.v.clone()
    rows = k + 2          # the initialiser's buffers may be longer than k

    def fake_init(points, pose, p=None, stream=None, out=None, pairs=None):
        assert points.shape == (k, 3) and len(pose) == 12
        return dict(mean=torch.full((rows, 3), 7.0), quat=torch.full((rows, 4), 0.5),
                    log_scale=torch.full((rows, 2), -1.0), logit=torch.full((rows,), 0.25),
                    lam=torch.ones(rows, 3), u=torch.full((rows,), 0.75), knn=torch.zeros(rows, 20, dtype=torch.int32))
    monkeypatch.setattr(keyframe, "initialise", fake_init)
    lam, u = w.insert_keyframe(torch.zeros(k, 3), list(range(12)))
    assert lam.shape == (k, 3) and u.shape == (k,)
    assert w.n == n + k and w._check_next
    for p, o, fill in zip(w.params, old, (7.0, 0.5, -1.0, 0.25)):
        assert torch.equal(p[:n], o) and torch.all(p[n:] == fill)
    for state, ref in ((w.m, m0), (w.v, v0)):
        assert state.numel() == 10 * (n + k)
        for b_new, b_old in zip(mapping.state_blocks(state, n + k), mapping.state_blocks(ref, n)):
            assert torch.equal(b_new[:n], b_old) and torch.all(b_new[n:] == 0)
    assert [tuple(g.shape) for g in w.grads] == [tuple(p.shape) for p in w.params]


class _FakeManager:
    """The contracts of MapManager.launch / gather on the CPU."""
    src = torch.tensor([0, 2, 2, 3, 5], dtype=torch.int32)
    role = torch.tensor([0, 1, 2, 0, 0], dtype=torch.uint8)

    def __init__(self, device):
        pass

    def launch(self, surf, lam, res, p=None):
        k, cap = len(self.src), len(self.src) + 3
        pad = lambda t: torch.cat([t, torch.full((cap - t.shape[0],) + tuple(t.shape[1:]), float("nan"))])
        src = self.src.long()
        return dict(mean=pad(surf[0][src] + 1), quat=pad(surf[1][src]), log_scale=pad(surf[2][src]),
                    logit=pad(surf[3][src]), src=torch.cat([self.src, torch.zeros(3, dtype=torch.int32)]),
                    role=torch.cat([self.role, torch.zeros(3, dtype=torch.uint8)]),
                    counts=torch.tensor([k, 1, 0, 0, 0, 1]), capacity=cap, score=torch.zeros(surf[0].shape[0]))

    def gather(self, out, arrays, zero_children=True):
        res = []
        for a in arrays:
            o = torch.full((out["capacity"],) + tuple(a.shape[1:]), float("nan"))
            k = int(out["counts"][0])
            rows = a[out["src"][:k].long()].clone()
            if zero_children:
                rows[out["role"][:k] != 0] = 0
            o[:k] = rows
            res.append(o)
        return res


def test_manage_carries_moments(monkeypatch):
    n = 6
    w = _window(n)
    old = [p.clone() for p in w.params]
    m0, v0 = w.m.clone(), w.v.clone()
    monkeypatch.setattr(manage, "MapManager", _FakeManager)
    counts, src = w.manage(torch.zeros(n, 3), torch.zeros(n))
    k = 5
    assert counts == [k, 1, 0, 0, 0, 1] and src.tolist() == [0, 2, 2, 3, 5]
    assert w.n == k and w._check_next
    assert torch.equal(w.params[0], old[0][[0, 2, 2, 3, 5]] + 1)
    assert torch.equal(w.params[3], old[3][[0, 2, 2, 3, 5]])
    for state, ref in ((w.m, m0), (w.v, v0)):
        assert state.numel() == 10 * k
        for b_new, b_old in zip(mapping.state_blocks(state, k), mapping.state_blocks(ref, n)):
            assert torch.equal(b_new[[0, 3, 4]], b_old[[0, 3, 5]])    # copies keep their moments
            assert torch.all(b_new[[1, 2]] == 0)                      # the two children start at zero
    assert [tuple(g.shape) for g in w.grads] == [tuple(p.shape) for p in w.params]


def test_autograd_window_keeps_leaf_parameters(monkeypatch):
    w = _window(4, autograd=True)
    monkeypatch.setattr(manage, "MapManager", _FakeManager)
    _FakeManager.src = torch.tensor([0, 1, 3], dtype=torch.int32)
    _FakeManager.role = torch.tensor([0, 0, 0], dtype=torch.uint8)
    try:
        w.manage(torch.zeros(4, 3), torch.zeros(4))
    finally:
        _FakeManager.src = torch.tensor([0, 2, 2, 3, 5], dtype=torch.int32)
        _FakeManager.role = torch.tensor([0, 1, 2, 0, 0], dtype=torch.uint8)
    assert all(p.is_leaf and p.requires_grad for p in w.params) and w.grads is None


def test_first_step_of_an_inserted_row_at_a_late_step(oracle):
    """Rows that join the window (keyframe insertion, split children) start
    from zero Adam moments but share the window's step count t, so their
    bias correction is that of step t, not 1: their first update is
    lr (1 - b1) / (1 - b1^t) / sqrt((1 - b2) / (1 - b2^t)) (2.51 lr at
    t = 1000, sqrt(10) lr as t grows, for the default betas), where a fresh
    optimiser would move them by lr.  This is the behaviour the window has (a
    per-row step count would need a per-row bias correction in the Adam
    kernel)."""
    import math
    import numpy as np
    lr, g, b1, b2 = 1e-3, np.array([0.37, -2.0e-4, 5.0]), 0.9, 0.999
    for t in (1000, 100_000):
        p, _, _ = oracle.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), t, lr)
        step = lr * (1 - b1) / (1 - b1 ** t) / math.sqrt((1 - b2) / (1 - b2 ** t))
        assert np.allclose(np.abs(p), step, rtol=1e-9)
    assert step == np.float64(step) and abs(step / lr - math.sqrt(10.0)) < 1e-9
    p1, _, _ = oracle.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr)
    assert np.allclose(np.abs(p1), lr, rtol=1e-9)
