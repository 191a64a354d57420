"""The C-ABI library builds for sm_103a, loads on a host without a GPU, and
exports every entry point that include/lgs.h declares (no compute calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lgslib():
    from paper_2607_04127_gb300 import build, lib
    build.build()
    return lib


def header_functions():
    txt = open(os.path.join(ROOT, "include", "lgs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lgs_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lgslib):
    names = header_functions()
    assert len(names) >= 20
    dll = ctypes.CDLL(lgslib.LIB_PATH)
    missing = [n for n in names if not hasattr(dll, n)]
    assert not missing, missing
    assert set(names) == set(lgslib.EXPORTS)


def test_constants_match_the_oracle(lgslib, oracle):
    c = lgslib.lgs_constants()
    o = oracle.constants()
    assert np.array_equal(c[:12], o[:12].astype(np.float32))


def test_status_strings(lgslib):
    assert lgslib.lgs_status_string(0) == "ok"
    assert lgslib.lgs_status_string(2) == "pair capacity exceeded"
    assert "sm_103a" in lgslib.lgs_version()


def test_argument_errors_without_device(lgslib):
    """Validation happens before any device work: invalid arguments return
    LGS_ERR_INVALID_ARG (or an error) instead of crashing."""
    L = lgslib.load()
    assert L.lgs_session_workspace_size(None, 10, None, 1, 10, None) == 1
    assert L.lgs_session_set_workspace(None, None, 0) == 1
    assert L.lgs_adam_step(None, None, None, None, None, None, None, -1, 1, None, 0.9, 0.999, 1e-15, 0, None) == 1
    assert L.lgs_adam_step_batch(None, 1, 0.9, 0.999, 1e-15, 0, None) == 1
    assert L.lgs_adam_step_batch(None, 0, 0.9, 0.999, 1e-15, 0, None) == 1
