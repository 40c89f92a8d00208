"""The C-ABI library loads without a GPU, exports every symbol include/pty.h
declares, and its host-only grouping equals the oracle's, bit for bit."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import grouping
from paper_2205_04295_b300 import pty, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pty.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pty_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = pty.lib()
    names = declared_symbols()
    assert "pty_run_iterations" in names and "pty_init_problem" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert L.pty_abi_version() == 3


def _groups_equal(pos, W, max_group=0, order=None):
    got = pty.group_positions(pos, W, max_group, order)
    ref = grouping.greedy_groups(np.asarray(pos, np.float32).astype(np.float64), W, order, max_group)
    assert len(got) == len(ref)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
    return got


@pytest.mark.parametrize("seed,W,mg", [(0, 8, 0), (1, 32, 0), (2, 16, 5), (3, 64, 1)])
def test_grouping_matches_oracle_random(seed, W, mg):
    pos = np.random.default_rng(seed).uniform(0, 300, size=(400, 2)).astype(np.float32)
    _groups_equal(pos, W, mg)
    order = np.random.default_rng(seed + 1).permutation(len(pos))
    _groups_equal(pos, W, mg, order)


def test_grouping_matches_oracle_on_scan_geometries():
    for wl in (synth.plain_rpie_64(), synth.refine_128(), synth.spiral_256(n=3000)):
        gs = _groups_equal(wl.pos, wl.W)
        assert sum(len(g) for g in gs) == wl.N


def test_grouping_half_pixel_rounding_is_exact():
    # floor(p + 0.5): 7.5 -> 8 and 7.4999995 -> 7 (float32 values, computed in double)
    pos = np.array([[0, 0], [7.5, 0], [np.float32(7.4999995), 40]], np.float32)
    gs = _groups_equal(pos, 8)
    assert [g.tolist() for g in gs] == [[0, 1, 2]]


def test_grouping_errors():
    L = pty.lib()
    g = np.zeros(4, np.int32)
    n = ctypes.c_int(0)
    pos = np.array([[0, 0], [np.nan, 1]], np.float32)
    rc = L.pty_group_positions(pos.ctypes.data, 2, 8, 0, None, g.ctypes.data, g.ctypes.data, ctypes.byref(n))
    assert rc == pty.PTY_EDATA
    assert b"not finite" in L.pty_last_error()
    rc = L.pty_group_positions(pos.ctypes.data, 0, 8, 0, None, g.ctypes.data, g.ctypes.data, ctypes.byref(n))
    assert rc == pty.PTY_EINVAL
    bad = np.array([0, 0], np.int32)
    ok = np.zeros((2, 2), np.float32)
    rc = L.pty_group_positions(ok.ctypes.data, 2, 8, 0, bad.ctypes.data, g.ctypes.data, g.ctypes.data, ctypes.byref(n))
    assert rc == pty.PTY_EINVAL


def test_init_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    d = pty.ProblemDesc(64, 1, 10, 100, 100, None, pty.ALLOC_FN(), pty.FREE_FN(), None, 0, 0)
    h = ctypes.c_void_p()
    rc = pty.lib().pty_init_problem(ctypes.byref(d), ctypes.byref(h))
    assert rc != pty.PTY_OK and not h.value
    d.W = 100
    assert pty.lib().pty_init_problem(ctypes.byref(d), ctypes.byref(h)) == pty.PTY_EINVAL


def test_unknown_problem_flags_are_rejected_before_any_device_call():
    """pty_problem_desc.flags accepts PTY_FLAG_FP32_REGISTRATION only; any other
    bit fails with PTY_EINVAL during argument checking (no GPU needed)."""
    L = pty.lib()
    d = pty.ProblemDesc(64, 2, 4, 100, 100, None, pty.ALLOC_FN(), pty.FREE_FN(), None, 0, 4)
    h = ctypes.c_void_p()
    assert L.pty_init_problem(ctypes.byref(d), ctypes.byref(h)) == pty.PTY_EINVAL
    assert b"unknown flags" in L.pty_last_error()
    assert not h.value
