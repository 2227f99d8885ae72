"""B300-native multislice / PRISM STEM simulation (hot path of arXiv 1706.08563).

The compute lives in ``libstem.so`` (hand-written CUDA for sm_103a behind the C
ABI in ``include/stem.h``).  ``api`` is a thin PyTorch binding; ``serve`` is
the continuous-batching request loop.
"""
from ._lib import LIB_PATH, StemError, load  # noqa: F401


def __getattr__(name):
    # the torch-facing API is imported lazily so that ``build`` works without CUDA
    if name in ("Plan", "SMatrix", "fft2", "footprint_bytes"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
