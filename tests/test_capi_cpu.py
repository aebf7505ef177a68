"""Host-side checks of the C ABI that need no GPU.

The library must build for sm_103a, load, export every symbol that
include/p2p.h declares, answer the workspace-size queries and reject invalid
arguments before touching the device.
"""
import ctypes
import os
import re

import pytest

from paper_2403_01596_gb300 import _capi as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "p2p.h")).read()
    return sorted(set(re.findall(r"P2P_API\s+[\w\s\*]+?\b(p2p_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return C.load()


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for required in ("p2p_bin_points", "p2p_build_neighbors", "p2p_plan_create", "p2p_apply", "p2p_apply_adjoint",
                     "p2p_grad_points", "p2p_plan_destroy", "p2p_last_async_status", "p2p_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_only_the_api_is_exported():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", C.library_path()], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    ours = {s for s in exported if s.startswith("p2p_")}
    assert ours == set(_declared_symbols())


def test_status_strings(lib):
    for s in range(7):
        assert lib.p2p_status_string(s)
    assert lib.p2p_version() >= 100


def test_workspace_queries_are_monotone():
    a = C.p2p_bin_workspace_size(1000)
    b = C.p2p_bin_workspace_size(1_000_000)
    assert 0 < a < b
    assert C.p2p_neighbors_workspace_size(0) > 0
    i = C.p2p_plan_workspace_size(1 << 20, 65622, 900_000, 14_500_000, C.P2P_LAYOUT_INDEXED, 1)
    r = C.p2p_plan_workspace_size(1 << 20, 65622, 900_000, 14_500_000, C.P2P_LAYOUT_REDUNDANT, 1)
    assert 0 < i < r
    assert C.p2p_plan_workspace_size(1 << 20, 65622, 900_000, 14_500_000, C.P2P_LAYOUT_INDEXED, 64) > i


def test_invalid_arguments_rejected_on_host(lib):
    nb = ctypes.c_int32(0)
    lo = (ctypes.c_double * 3)(0, 0, 0)
    # negative n, zero h, ng out of range
    assert lib.p2p_bin_points(None, -1, lo, 1.0, 8, None, None, None, None, ctypes.byref(nb), None, 0, None) == 1
    assert lib.p2p_bin_points(None, 10, lo, 0.0, 8, None, None, None, None, ctypes.byref(nb), None, 0, None) == 1
    assert lib.p2p_bin_points(None, 10, lo, 1.0, 0, None, None, None, None, ctypes.byref(nb), None, 0, None) == 1
    assert lib.p2p_bin_points(None, 10, lo, 1.0, (1 << 21) + 1, None, None, None, None, ctypes.byref(nb), None, 0,
                              None) == 1
    out = ctypes.c_size_t(0)
    assert lib.p2p_plan_workspace_size(100, 10, 50, 500, 7, 1, None, ctypes.byref(out)) == 1      # bad layout
    assert lib.p2p_plan_workspace_size(100, 10, 50, 500, 0, 0, None, ctypes.byref(out)) == 1      # nrhs 0
    assert lib.p2p_plan_workspace_size(100, 10, 50, 500, 0, 257, None, ctypes.byref(out)) == 1    # nrhs too big
    bad = C.p2p_tuning(48, 8, 128, 0)                                                               # chunk % 32
    assert lib.p2p_plan_workspace_size(100, 10, 50, 500, 0, 1, ctypes.byref(bad), ctypes.byref(out)) == 1
    bad = C.p2p_tuning(128, 17, 128, 0)                                                             # warps
    assert lib.p2p_plan_workspace_size(100, 10, 50, 500, 0, 1, ctypes.byref(bad), ctypes.byref(out)) == 1
    # null plan handles
    assert lib.p2p_apply(None, None, None, 1, 1, None) == 1
    assert lib.p2p_plan_info(None, None, None, None, None, None, None) == 1
    plan = ctypes.c_void_p(0)
    assert lib.p2p_plan_create(ctypes.byref(plan), None, 10, None, None, 0, None, None, 0, 0, 0, 1.0, 0, 1, None,
                               None, 0, None) == 1


def test_host_pipe_arguments_rejected_on_host(lib):
    out = ctypes.c_size_t(0)
    assert lib.p2p_host_pipe_workspace_size(0, 1, ctypes.byref(out)) == 1           # no points
    assert lib.p2p_host_pipe_workspace_size(100, 0, ctypes.byref(out)) == 1         # nrhs 0
    assert lib.p2p_host_pipe_workspace_size(100, 257, ctypes.byref(out)) == 1       # nrhs too big
    assert lib.p2p_host_pipe_workspace_size(1000, 4, ctypes.byref(out)) == 0
    assert out.value >= 4 * 1000 * 4 * 8                                             # 2 strength + 2 result slots
    pipe = ctypes.c_void_p(0)
    assert lib.p2p_host_pipe_create(ctypes.byref(pipe), 1000, 4, None, out.value) == 1          # no workspace
    assert lib.p2p_host_pipe_create(ctypes.byref(pipe), 1000, 4, ctypes.c_void_p(256), 16) == 2  # too small
    assert lib.p2p_host_pipe_create(ctypes.byref(pipe), 1000, 4, ctypes.c_void_p(8), out.value) == 1  # unaligned
    assert not pipe.value
    assert lib.p2p_apply_host(None, None, 1, None, None, None) == 1
    assert lib.p2p_host_pipe_destroy(None) == 0
