"""The C-ABI library builds, loads and exports every entry point of include/vfmm.h."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vfmm.h")).read()
    return sorted(set(re.findall(r"^(?:int|const char \*)\s*(vfmm_\w+)\s*\(", src, re.M)))


def test_library_exports_all_declared_symbols():
    from paper_1110_2921_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name


def test_host_only_calls():
    from paper_1110_2921_gb300 import _native as nv
    cfg = nv.config_default()
    assert cfg.p == 10 and cfg.periodic_levels == 2 and abs(cfg.box - 6.283185307179586) < 1e-15
    assert nv.strerror(nv.VFMM_ERR_ARG) == "invalid argument"
    # argument validation happens before any device work
    bad = nv.config_default()
    bad.p = 1
    h = ctypes.c_void_p()
    assert nv.lib().vfmm_create(ctypes.byref(bad), ctypes.byref(h)) == nv.VFMM_ERR_ARG
    bad = nv.config_default()
    bad.p = 11
    assert nv.lib().vfmm_create(ctypes.byref(bad), ctypes.byref(h)) == nv.VFMM_ERR_UNSUPPORTED
    bad = nv.config_default()
    bad.dtype = nv.VFMM_F64   # FP64 data with a tensor-core M2L is rejected
    assert nv.lib().vfmm_create(ctypes.byref(bad), ctypes.byref(h)) == nv.VFMM_ERR_ARG
    assert nv.lib().vfmm_build_tree(None, 10, None) == nv.VFMM_ERR_ARG
    assert nv.lib().vfmm_sync(None) == nv.VFMM_ERR_ARG
    assert nv.lib().vfmm_set_wait_limit(None, 5) == nv.VFMM_ERR_ARG
    assert nv.lib().vfmm_energy_spectrum(None, 16, None, 8, None) == nv.VFMM_ERR_ARG
    assert nv.lib().vfmm_derivative_moments(None, 10, None, None) == nv.VFMM_ERR_ARG
    ops = ctypes.c_double(0.0)
    # argument checks of the peak probes come before any CUDA call
    assert nv.lib().vfmm_probe_peak(nv.VFMM_PROBE_FFMA, 0, None, None, ctypes.byref(ops)) == nv.VFMM_ERR_ARG
    assert nv.lib().vfmm_probe_peak(nv.VFMM_PROBE_FFMA, 10, None, None, None) == nv.VFMM_ERR_ARG
    assert cfg.concurrent_far == 1 and abs(cfg.rho_cut - 5.0) < 1e-15


def test_layout_matches_header():
    from paper_1110_2921_gb300 import _native as nv
    # vfmm_config: 4 ints, double, int, double, 4 ints, pointer, int (padded to 8)
    assert ctypes.sizeof(nv.vfmm_config) == 4 * 4 + 8 + 8 + 8 + 4 * 4 + 8 + 8
