"""The C ABI library loads and exports everything include/stem.h declares (CPU only),
and the host-side checks that return before any CUDA call behave as documented."""
import ctypes
import math
import os
import re

import pytest

from paper_1706_08563_b300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "stem.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stem_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    lib = _lib.load()
    names = header_functions()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert set(names) <= set(_lib.SIGNATURES)


def test_status_strings():
    for code in range(-5, 1):
        assert _lib.status_string(code)
    assert _lib.status_string(-4) == "unsupported size"


def _params(n=64, rings=10, slices=2):
    return _lib.StemParams((ctypes.c_double * 3)(10.0, 10.0, 4.0), n, slices, 2.0, 200.0, 20.0, 1.0, rings)


def test_plan_create_rejects_before_touching_the_gpu():
    lib = _lib.load()
    h = ctypes.c_void_p()
    assert lib.stem_plan_create(None, ctypes.byref(h)) == _lib.STEM_ERR_INVALID
    for n in (0, 4, 100, 4096):
        p = _params(n=n)
        assert lib.stem_plan_create(ctypes.byref(p), ctypes.byref(h)) == _lib.STEM_ERR_UNSUPPORTED
    for rings in (0, 3000):
        p = _params(rings=rings)
        assert lib.stem_plan_create(ctypes.byref(p), ctypes.byref(h)) == _lib.STEM_ERR_INVALID
    p = _params(slices=0)
    assert lib.stem_plan_create(ctypes.byref(p), ctypes.byref(h)) == _lib.STEM_ERR_INVALID
    assert lib.stem_plan_create(ctypes.byref(_params()), None) == _lib.STEM_ERR_INVALID


def test_fft2_argument_checks():
    lib = _lib.load()
    assert lib.stem_fft2(100, 1, 0, None, None) == _lib.STEM_ERR_UNSUPPORTED
    assert lib.stem_fft2(4, 1, 0, None, None) == _lib.STEM_ERR_UNSUPPORTED
    assert lib.stem_fft2(64, -1, 0, None, None) == _lib.STEM_ERR_INVALID
    assert lib.stem_fft2(64, 1, 0, None, None) == _lib.STEM_ERR_INVALID
    assert lib.stem_fft2(64, 70000, 0, ctypes.c_void_p(16), None) == _lib.STEM_ERR_INVALID
    assert lib.stem_fft2(64, 0, 0, None, None) == _lib.STEM_OK       # empty batch is a no-op


def test_null_plan_is_rejected_everywhere():
    lib = _lib.load()
    z = None
    assert lib.stem_multislice_scan(z, z, z, 0, 1, 1.0, z, z, 0, z) == _lib.STEM_ERR_INVALID
    assert lib.stem_prism_smatrix(z, z, 1, 0, 1, z, 0, z, 0, z) == _lib.STEM_ERR_INVALID
    assert lib.stem_prism_output(z, 1, 0, 0, z, z, 0, 1, 1.0, z, z, 0, z) == _lib.STEM_ERR_INVALID
    assert lib.stem_slice_potentials(z, z, z, 0, z, z, z, 0, z) == _lib.STEM_ERR_INVALID
    assert lib.stem_detector_readout(z, 1, z, 0, 1.0, z, z) == _lib.STEM_ERR_INVALID
    assert lib.stem_multislice_workspace(z, 4) == 0
    assert lib.stem_prism_smatrix_bytes(z, 1, 0) == 0


def test_footprint_multislice_is_stack_plus_batch_plus_rings():
    lib = _lib.load()
    p = _params(n=256, rings=100, slices=20)
    got = lib.stem_footprint_bytes(ctypes.byref(p), 0, 1, 0, 4096, 64)
    want = 20 * 256 * 256 * 8 + 64 * 256 * 256 * 8 + 4096 * 100 * 4
    assert got == want


def test_footprint_prism_counts_the_beams():
    """PRISM footprint grows with the S-matrix: f=1 needs about 16x the beams of f=4."""
    lib = _lib.load()
    p = _params(n=256, rings=100, slices=20)
    f1 = lib.stem_footprint_bytes(ctypes.byref(p), 1, 1, 0, 4096, 64)
    f4 = lib.stem_footprint_bytes(ctypes.byref(p), 1, 4, 0, 4096, 64)
    h16 = lib.stem_footprint_bytes(ctypes.byref(p), 1, 1, 1, 4096, 64)
    assert f1 > f4 > 0
    assert h16 < f1
    assert lib.stem_footprint_bytes(ctypes.byref(p), 1, 3, 0, 4096, 64) == 0   # f not a power of two


def test_footprint_streamed_replaces_the_stack_by_three_slices():
    lib = _lib.load()
    p = _params(n=256, rings=100, slices=20)
    plane = 256 * 256 * 8
    ms = lib.stem_footprint_bytes(ctypes.byref(p), 0, 1, 0, 4096, 64)
    ms_s = lib.stem_footprint_bytes(ctypes.byref(p), 2, 1, 0, 4096, 64)
    assert ms - ms_s == (20 - 3) * plane
    pr = lib.stem_footprint_bytes(ctypes.byref(p), 1, 4, 0, 4096, 64)
    pr_s = lib.stem_footprint_bytes(ctypes.byref(p), 3, 4, 0, 4096, 64)
    assert pr - pr_s == (20 - 3) * plane
    assert lib.stem_footprint_bytes(ctypes.byref(p), 4, 1, 0, 4096, 64) == 0


def test_memory_model_picks_single_then_streamed():
    """The paper's automatic choice of memory model from the footprint estimate."""
    import workloads as W
    from paper_1706_08563_b300 import api
    w = W.C3
    single = api.footprint_bytes(w, "ms", batch=256)
    streamed = api.footprint_bytes(w, "ms_streamed", batch=256)
    assert streamed < single
    assert api.memory_model(w, "ms", single, batch=256) == "single"
    assert api.memory_model(w, "ms", single - 1, batch=256) == "streamed"
    assert api.memory_model(w, "ms", streamed, batch=256) == "streamed"
    with pytest.raises(MemoryError):
        api.memory_model(w, "ms", streamed - 1, batch=256)


def test_streamed_entry_points_reject_bad_arguments():
    lib = _lib.load()
    z = None
    assert lib.stem_multislice_scan_streamed(z, z, z, 0, 1, 1.0, z, z, 0, z) == _lib.STEM_ERR_INVALID
    assert lib.stem_prism_smatrix_streamed(z, z, 1, 0, 1, z, 0, z, 0, z) == _lib.STEM_ERR_INVALID
    assert lib.stem_multislice_streamed_workspace(z, 4) == 0
    assert lib.stem_prism_smatrix_streamed_workspace(z, 4) == 0


def test_selftest_entry_point_rejects_bad_arguments():
    lib = _lib.load()
    assert lib.stem_selftest_bounded_wait(None, 1000, None) == _lib.STEM_ERR_INVALID
    assert lib.stem_selftest_fma_rate(0, 0, 1, ctypes.c_void_p(16), None) == _lib.STEM_ERR_INVALID
    assert lib.stem_selftest_fma_rate(1, 10, 0, ctypes.c_void_p(16), None) == _lib.STEM_ERR_INVALID
    assert lib.stem_selftest_fma_rate(0, 10, 1, None, None) == _lib.STEM_ERR_INVALID


def test_c_client_compiles_and_links_as_c99(repo_tmp):
    """The header is plain C and the library links without Python or PyTorch."""
    from conftest import build_c_client
    exe = build_c_client(repo_tmp)
    assert os.access(exe, os.X_OK)


def test_profile_read_argument_checks():
    lib = _lib.load()
    n, ms = ctypes.c_int64(), ctypes.c_double()
    assert lib.stem_profile_read(-1, ctypes.byref(n), ctypes.byref(ms)) == _lib.STEM_ERR_INVALID
    assert lib.stem_profile_read(4, ctypes.byref(n), ctypes.byref(ms)) == _lib.STEM_ERR_INVALID
    assert lib.stem_profile_read(0, None, ctypes.byref(ms)) == _lib.STEM_ERR_INVALID
    # nothing recorded yet: zero launches, no CUDA call needed
    assert lib.stem_profile_enable(1) == _lib.STEM_OK
    assert lib.stem_profile_read(0, ctypes.byref(n), ctypes.byref(ms)) == _lib.STEM_OK
    assert n.value == 0 and ms.value == 0.0
    assert lib.stem_profile_enable(0) == _lib.STEM_OK
