"""Batched uneven maps: one call per stage over every map's frame equals the
per-map launches; the persistent longest-first schedule and the CUDA-graph
replay change nothing; the autotuner returns a valid configuration."""
import numpy as np
import pytest

from paper_2607_04127_gb300 import scenes

pytestmark = pytest.mark.gpu

SIZES = [3000, 6000, 12000, 24000, 1500]
SHAPES = [(32, 256), (64, 512), (32, 512)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_04127_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def workload():
    return scenes.street_maps(3, SIZES, SHAPES, tile=(8, 8))


def _cpu(x):
    return x.detach().cpu().numpy()


def _compare(outs_a, outs_b):
    for a, b in zip(outs_a, outs_b):
        for k in ("A", "S_t", "S_n", "T_final", "n_contrib"):
            assert np.array_equal(_cpu(getattr(a, k)), _cpu(getattr(b, k))), k


def _grads_close(ga, gb):
    for xa, xb in zip(ga, gb):
        for a, b in zip(xa, xb):
            a, b = _cpu(a), _cpu(b)
            assert np.allclose(a, b, rtol=1e-5, atol=1e-6 * max(np.abs(b).max(), 1e-30))


def test_batched_equals_sequential(workload):
    import torch
    from paper_2607_04127_gb300 import batched
    maps, frames, targets = zip(*workload)
    B = batched.BatchedMaps(maps, frames, targets)
    S = batched.SequentialMaps(maps, frames, targets)
    LB = B.step(check=True).clone()
    S.step(check=True)
    torch.cuda.synchronize()
    _compare(B.outputs(), S.outputs())
    F, M = len(frames), len(maps)
    for m, r in enumerate(S.rasts):
        assert float(LB[1 + 4 * F + m]) == float(r.loss_out[0])
    _grads_close(B.grads, S.grads)
    B.close()
    S.close()


@pytest.mark.parametrize("tuning", [dict(persistent=1), dict(persistent=1, fwd_batch=0, bwd_batch=64),
                                    dict(fwd_batch=256, bwd_batch=128)])
def test_schedules_change_nothing(workload, tuning):
    import torch
    from paper_2607_04127_gb300 import batched
    maps, frames, targets = zip(*workload)
    ref = batched.BatchedMaps(maps, frames, targets)
    alt = batched.BatchedMaps(maps, frames, targets, tuning=tuning)
    L0 = ref.step(check=True).clone()
    L1 = alt.step(check=True).clone()
    torch.cuda.synchronize()
    _compare(ref.outputs(), alt.outputs())
    assert np.array_equal(_cpu(L0), _cpu(L1))
    _grads_close(alt.grads, ref.grads)
    ref.close()
    alt.close()


def test_graph_replay_equals_eager(workload):
    import torch
    from paper_2607_04127_gb300 import batched
    maps, frames, targets = zip(*workload)
    eager = batched.BatchedMaps(maps, frames, targets, tuning=dict(persistent=1))
    L0 = eager.step(check=True).clone()
    g = batched.BatchedMaps(maps, frames, targets, tuning=dict(persistent=1))
    g.capture()
    for _ in range(2):                    # replays are repeatable
        g.replay()
    torch.cuda.synchronize()
    g.rast.session.check_status()
    _compare(eager.outputs(), g.outputs())
    assert np.array_equal(_cpu(L0), _cpu(g.rast.loss_out))
    _grads_close(g.grads, eager.grads)
    eager.close()
    g.close()


def test_autotune_picks_a_valid_configuration(workload):
    from paper_2607_04127_gb300 import autotune, batched, lib
    maps, frames, targets = zip(*workload[:3])

    def make(tile, tun):
        return batched.BatchedMaps(maps, [f.with_tiles(*tile) for f in frames], targets, tuning=tun)

    tile, tun, log = autotune.autotune(make, steps=2)
    assert tile in autotune.TILES and len(log) >= len(autotune.TILES)
    s = lib.Session()
    lib.lgs_session_set_tuning(s.handle, **tun)       # accepted by the library
    s.close()
