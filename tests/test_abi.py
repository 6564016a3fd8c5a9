"""The C-ABI library builds, loads and exports every symbol include/tcgs.h declares; host-side
argument validation answers without touching a GPU.  CPU only."""
import ctypes
import os
import re

import pytest

from paper_2505_24796_gb300 import _lib
from paper_2505_24796_gb300 import build as tbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"TCGS_API\s+[\w\s\*]+?\b(tcgs_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    tbuild.build()
    return _lib.load(build_if_needed=False)


def test_header_declares_the_pipeline():
    names = declared_symbols()
    for n in ["tcgs_project", "tcgs_bin_sort", "tcgs_bin_sort_workspace_size", "tcgs_render_fwd",
              "tcgs_render_bwd", "tcgs_status_string", "tcgs_version", "tcgs_frag2mat_beta"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in declared_symbols():
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, f"binding lacks {n}"


def test_status_strings(lib):
    assert lib.tcgs_status_string(0) == b"ok"
    assert b"capacity" in lib.tcgs_status_string(3)
    assert lib.tcgs_version() >= 100


def test_workspace_size_is_host_only_and_monotone(lib):
    a = lib.tcgs_bin_sort_workspace_size(1000, 10_000, 64)
    b = lib.tcgs_bin_sort_workspace_size(2000, 10_000, 64)
    c = lib.tcgs_bin_sort_workspace_size(2000, 20_000, 64)
    assert 0 < a < b < c
    assert c - b >= 3 * 4 * 10_000 - 3 * 256   # three splat-sized arrays, 256-byte aligned
    assert lib.tcgs_bin_sort_workspace_size(-1, 10, 1) == 0


def test_invalid_arguments_rejected_on_host(lib):
    cam = _lib.tcgs_camera()
    cam.width, cam.height, cam.fx, cam.fy = 0, 10, 1.0, 1.0   # invalid width
    V = None
    assert lib.tcgs_project(ctypes.byref(cam), 10, 0, *([V] * 11), None) == _lib.TCGS_ERR_INVALID
    cam.width = 16
    assert lib.tcgs_project(ctypes.byref(cam), 10, 4, *([V] * 11), None) == _lib.TCGS_ERR_INVALID  # degree > 3
    assert lib.tcgs_project(ctypes.byref(cam), 10, 0, *([V] * 11), None) == _lib.TCGS_ERR_INVALID  # null arrays
    assert lib.tcgs_project(ctypes.byref(cam), 0, 0, *([V] * 11), None) == _lib.TCGS_OK             # empty: no-op
    opts = _lib.tcgs_render_opts()
    opts.precision, opts.alpha_max = 9, 0.99
    assert lib.tcgs_render_fwd(ctypes.byref(cam), ctypes.byref(opts), *([V] * 10), None) == _lib.TCGS_ERR_INVALID
    assert lib.tcgs_bin_sort(ctypes.byref(cam), 10, V, V, V, 2 ** 33, V, 0, V, V, V, V, None) == \
        _lib.TCGS_ERR_INVALID
    assert lib.tcgs_bin_sort_exact(ctypes.byref(cam), 10, V, V, V, V, V, 100, V, 0, V, V, V, V, None) == \
        _lib.TCGS_ERR_INVALID   # conic and opacity required
    assert lib.tcgs_selftest_bounded_wait(V, 16, None) == _lib.TCGS_ERR_INVALID          # no status word
    assert lib.tcgs_selftest_bounded_wait(ctypes.c_void_p(256), 0, None) == _lib.TCGS_ERR_INVALID   # no polls
    assert lib.tcgs_microbench_ex2(V, 1, 1, None) == _lib.TCGS_ERR_INVALID
    assert lib.tcgs_microbench_ex2(ctypes.c_void_p(256), 0, 1, None) == _lib.TCGS_ERR_INVALID


def test_wave_query_reports_no_tc_device_without_a_gpu(lib):
    """tcgs_tc_wave_tiles answers 0 when the current device is not an sm_103 GPU (here: none)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present; the GPU tests check the wave size")
    assert lib.tcgs_tc_wave_tiles() == 0


def test_build_targets_sm103a_only():
    assert tbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
