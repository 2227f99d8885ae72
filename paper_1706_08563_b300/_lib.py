"""ctypes loader for libstem.so (the C ABI declared in include/stem.h).

The library is built in-tree (``python -m paper_1706_08563_b300.build``).  There
is no fallback: if the shared library is missing or cannot be loaded, importing
the package's compute API raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int32, c_int64, c_size_t, c_void_p

# STEM_LIB may name another build of the same library (for example a tuning variant).
LIB_PATH = os.environ.get("STEM_LIB") or os.path.join(os.path.dirname(os.path.abspath(__file__)), "libstem.so")

STEM_OK = 0
# kernel families of stem_profile_read
STEM_PROF_ROW_SLICE = 0
STEM_PROF_COL_SLICE = 1
STEM_PROF_BEAM_SUM = 2
STEM_PROF_POTENTIALS = 3
STEM_ERR_INVALID = -1
STEM_ERR_NOMEM = -2
STEM_ERR_CUDA = -3
STEM_ERR_UNSUPPORTED = -4
STEM_ERR_TIMEOUT = -5

STORAGE = {"f32": 0, "f16": 1, "bf16": 2}
STEM_CROPPED = 16          # storage flag: Fourier-cropped S-matrix on the 3N/4 grid
ENGINE = {"auto": 0, "simt": 1, "tensor": 2}


class StemParams(ctypes.Structure):
    _fields_ = [("cell", c_double * 3), ("n", c_int32), ("n_slices", c_int32), ("slice_dz", c_double),
                ("energy_kev", c_double), ("alpha_mrad", c_double), ("ring_width_mrad", c_double),
                ("n_rings", c_int32), ("defocus_a", c_double), ("cs_a", c_double)]


class StemError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


# name -> (restype, argtypes)
SIGNATURES = {
    "stem_status_string": (c_char_p, [c_int32]),
    "stem_launch_count": (ctypes.c_uint64, []),
    "stem_profile_enable": (c_int32, [c_int32]),
    "stem_profile_read": (c_int32, [c_int32, POINTER(c_int64), POINTER(c_double)]),
    "stem_plan_create": (c_int32, [POINTER(StemParams), POINTER(c_void_p)]),
    "stem_plan_destroy": (None, [c_void_p]),
    "stem_plan_device_status": (c_int32, [c_void_p, POINTER(c_int32)]),
    "stem_selftest_bounded_wait": (c_int32, [c_void_p, c_int64, c_void_p]),
    "stem_selftest_fma_rate": (c_int32, [c_int32, c_int64, c_int32, c_void_p, c_void_p]),
    "stem_plan_constants": (c_int32, [c_void_p, POINTER(c_double), POINTER(c_double), POINTER(c_int32)]),
    "stem_slice_potentials_workspace": (c_size_t, [c_void_p, c_int64]),
    "stem_slice_potentials": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p,
                                        c_size_t, c_void_p]),
    "stem_multislice_workspace": (c_size_t, [c_void_p, c_int32]),
    "stem_multislice_scan": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_float, c_void_p,
                                       c_void_p, c_size_t, c_void_p]),
    "stem_multislice_scan_noalloc": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_float,
                                               c_void_p, c_void_p]),
    "stem_multislice_streamed_workspace": (c_size_t, [c_void_p, c_int32]),
    "stem_multislice_scan_streamed": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_float,
                                                c_void_p, c_void_p, c_size_t, c_void_p]),
    "stem_prism_smatrix_streamed_workspace": (c_size_t, [c_void_p, c_int32]),
    "stem_prism_smatrix_streamed": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_void_p, c_size_t,
                                              c_void_p, c_size_t, c_void_p]),
    "stem_multislice_scan_4d": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_float, c_void_p,
                                          c_void_p, c_size_t, c_void_p]),
    "stem_prism_output_4d": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_int64, c_int32,
                                       c_float, c_void_p, c_void_p, c_size_t, c_void_p]),
    "stem_plan_set_detector_edges": (c_int32, [c_void_p, c_int32, c_void_p]),
    "stem_prism_beams": (c_int32, [c_void_p, c_int32, POINTER(c_int32), c_void_p]),
    "stem_prism_smatrix_bytes": (c_size_t, [c_void_p, c_int32, c_int32]),
    "stem_prism_smatrix_workspace": (c_size_t, [c_void_p, c_int32]),
    "stem_prism_smatrix": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_void_p, c_size_t,
                                     c_void_p, c_size_t, c_void_p]),
    "stem_prism_smatrix_range": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32,
                                           c_void_p, c_size_t, c_void_p, c_size_t, c_void_p]),
    "stem_prism_output_workspace": (c_size_t, [c_void_p, c_int32, c_int32]),
    "stem_prism_output": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_int64, c_int32,
                                    c_float, c_void_p, c_void_p, c_size_t, c_void_p]),
    "stem_prism_windows": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_int64, c_void_p,
                                     c_void_p, c_size_t, c_void_p]),
    "stem_detector_readout": (c_int32, [c_void_p, c_int32, c_void_p, c_int64, c_float, c_void_p, c_void_p]),
    "stem_fft2": (c_int32, [c_int32, c_int64, c_int32, c_void_p, c_void_p]),
    "stem_footprint_bytes": (c_size_t, [POINTER(StemParams), c_int32, c_int32, c_int32, c_int64, c_int32]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libstem.so once and declare every function's C signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libstem.so not found at {path}; build it with "
                          "`python -m paper_1706_08563_b300.build` (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().stem_status_string(int(status)).decode()


def check(status: int, what: str) -> None:
    if status != STEM_OK:
        raise StemError(status, what)
