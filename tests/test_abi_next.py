"""Host logic of the map-management and keyframe-initialisation entry points
(no device needed): default parameters equal to the oracles' defaults,
capacity and launch accounting, scratch sizes, and argument errors returned
before any device work."""
import ctypes
import math

import numpy as np
import pytest

F = np.float32
INVALID = 1


@pytest.fixture(scope="module")
def lgslib():
    from paper_2607_04127_gb300 import build, lib
    build.build()
    return lib


def test_manage_defaults_match_the_oracle(lgslib):
    from oracle import manage as om
    p = lgslib.lgs_manage_default_params()
    o = om.Params()
    for name, _ in p._fields_:
        got = getattr(p, name)
        want = getattr(o, name)
        assert (got == want) if isinstance(got, int) else (F(got) == F(want)), name


def test_init_defaults_match_the_oracle(lgslib):
    from oracle import init as oi
    p = lgslib.lgs_init_default_params()
    o = oi.Params()
    for name, _ in p._fields_:
        got = getattr(p, name)
        want = getattr(o, name)
        assert (got == want) if isinstance(got, int) else (F(got) == F(want)), name


def test_capacity_and_launch_accounting(lgslib):
    p = lgslib.lgs_manage_default_params()
    for n in (0, 1, 19, 20, 1000, 2_000_000):
        assert lgslib.lgs_manage_capacity(n, p) == n + math.floor(float(F(p.split_cap)) * n)
    bad = lgslib.lgs_manage_default_params()
    bad.split_cap = 1.5
    assert lgslib.lgs_manage_capacity(10, bad) == -1
    for passes in range(4):
        p.n_passes = passes
        # residual select (3 digits) + 2; 17 per pass; the split: 15
        assert lgslib.lgs_manage_launches(p) == 5 + 17 * passes + 15
    p.n_passes = 4
    assert lgslib.lgs_manage_launches(p) == -1
    L = lgslib.load()
    assert L.lgs_init_launches() == 11
    assert L.lgs_init_max_points() == 1 << 20


def test_scratch_sizes_grow(lgslib):
    a = [lgslib.lgs_manage_scratch_bytes(n) for n in (0, 1000, 100_000, 2_000_000)]
    assert all(x > 0 for x in a) and a == sorted(a)
    b = [lgslib.lgs_init_scratch_bytes(n) for n in (0, 1000, 100_000, 1 << 20)]
    assert all(x > 0 for x in b) and b == sorted(b)


def _surfels(lgslib, n, ptr=256):
    return lgslib.lgs_surfels(ptr, ptr, ptr, ptr, n)


def test_manage_argument_errors(lgslib):
    L = lgslib.load()
    P = ctypes.c_void_p
    p = lgslib.lgs_manage_default_params()
    out = lgslib.lgs_surfel_params_out(256, 256, 256, 256)
    n = 100
    cap = lgslib.lgs_manage_capacity(n, p)
    big = lgslib.lgs_manage_scratch_bytes(n)

    def call(surf=None, params=None, scratch=4096, sbytes=None, capacity=None, counts=256, o=out):
        s = surf if surf is not None else _surfels(lgslib, n)
        pr = params if params is not None else p
        return L.lgs_map_manage(ctypes.byref(s), P(256), P(256), ctypes.byref(pr), P(scratch),
                                big if sbytes is None else sbytes, P(256), ctypes.byref(o),
                                cap if capacity is None else capacity, P(256), P(256), P(counts), None)
    assert L.lgs_map_manage(None, None, None, None, None, 0, None, None, 0, None, None, None, None) == INVALID
    assert call(surf=_surfels(lgslib, (1 << 28) + 1)) == INVALID
    assert call(surf=_surfels(lgslib, -1)) == INVALID
    assert call(surf=lgslib.lgs_surfels(0, 256, 256, 256, n)) == INVALID
    assert call(capacity=cap - 1) == INVALID
    assert call(sbytes=big - 1) == INVALID
    assert call(scratch=4096 + 16) == INVALID                # not 256-byte aligned
    assert call(counts=0) == INVALID
    for field, value in (("alpha_prune", 0.0), ("alpha_min", 1.0), ("q_plane", 1.5), ("q_cover", -0.1),
                         ("prune_cap", 2.0), ("eps", 0.0), ("voxel", 0.0), ("voxel", float("inf")),
                         ("slab", -1.0), ("n_passes", 4), ("n_passes", -1), ("split_shift", float("nan"))):
        q = lgslib.lgs_manage_default_params()
        setattr(q, field, value)
        assert call(params=q) == INVALID, (field, value)
    assert L.lgs_map_gather(P(256), P(256), P(256), 10, P(256), P(256), 0, 1, None) == INVALID
    assert L.lgs_map_gather(P(256), P(256), P(256), -1, P(256), P(256), 1, 1, None) == INVALID
    assert L.lgs_map_gather(P(256), P(256), P(256), 10, P(258), P(256), 1, 1, None) == INVALID
    assert L.lgs_map_gather(P(256), P(256), None, 10, P(256), P(256), 1, 1, None) == INVALID


def test_keyframe_argument_errors(lgslib):
    L = lgslib.load()
    P = ctypes.c_void_p
    out = lgslib.lgs_surfel_params_out(256, 256, 256, 256)
    pose = (ctypes.c_float * 12)(*np.eye(3, 4).ravel())
    n = 1000
    need = lgslib.lgs_init_scratch_bytes(n)

    def call(params=None, n_=n, scratch=4096, sbytes=need, pz=pose, points=256):
        p = params if params is not None else lgslib.lgs_init_default_params()
        return L.lgs_keyframe_init(P(points), n_, pz, ctypes.byref(p), P(scratch), sbytes, P(256),
                                   ctypes.byref(out), P(256), P(256), None, None)
    assert call(n_=(1 << 20) + 1) == INVALID
    assert call(n_=-1) == INVALID
    assert call(points=0) == INVALID
    assert call(sbytes=need - 1) == INVALID
    assert call(scratch=4096 + 8) == INVALID                  # not 16-byte aligned
    bad_pose = (ctypes.c_float * 12)(*([float("nan")] + [0.0] * 11))
    assert call(pz=bad_pose) == INVALID
    for field, value in (("k", 2), ("k", 33), ("kappa", 0.0), ("s_min", 0.0), ("s_max", 1e-4), ("r0", 0.0),
                         ("c0", 1.0), ("eps", 0.0), ("alpha_min", 0.0), ("alpha_max", 1.0), ("alpha_max", 0.2)):
        q = lgslib.lgs_init_default_params()
        setattr(q, field, value)
        assert call(params=q) == INVALID, (field, value)
    q = lgslib.lgs_init_default_params()
    q.k = 20
    assert call(params=q, n_=19) == INVALID                   # k > n
