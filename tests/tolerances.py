"""Parity tolerances shared by the GPU tests.

FP32 arithmetic is held to relative L2 <= 1e-4 over the whole [probe, ring]
array, and ring by ring: a ring whose RMS is at least FLOOR of the largest
ring's RMS must match to relative L2 <= tol; a darker ring must match to an
absolute RMS error <= tol * FLOOR * (largest ring RMS).  Rounding leaves every
Fourier pixel with an error set by the bright field, not by the ring's own
signal, so rings far below the bright field carry an error floor that no
relative bound can meet (their relative error grows like 1/sqrt(I) from the
cross term, then like 1/I).  FLOOR is 1e-5 for FP32 and 1e-4 for FP16/BF16
S-matrix storage (tol = 1e-2 there).

The intensity at which a dark ring's relative error reaches tol grows in
proportion to the rounding-noise energy, which grows with the number of
roundings along the chain: per slice two 2D FFTs of log2(N) radix stages each
plus the transmission and propagator products.  `fp32_floor` scales FLOOR by
that count relative to the 128^2, 10-slice case the 1e-5 was set on.
"""
import math

import numpy as np

from oracle import stem as O

FP32_TOL = 1e-4
LOWP_TOL = 1e-2
FP32_FLOOR = 1e-5
LOWP_FLOOR = 1e-4


def _chain(n, n_slices):
    return n_slices * (2 * math.log2(n) + 2)


def fp32_floor(n, n_slices):
    """FLOOR for an FP32 multislice of n_slices slices at N = n."""
    return FP32_FLOOR * max(1.0, _chain(n, n_slices) / _chain(128, 10))


def rel_l2(a, b):
    return O.rel_l2(np.asarray(a, np.float64), np.asarray(b, np.float64))


def check_rings(got, ref, tol, floor=None):
    floor = (FP32_FLOOR if tol <= FP32_TOL else LOWP_FLOOR) if floor is None else floor
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert got.shape == ref.shape
    assert np.all(np.isfinite(got))
    assert rel_l2(got, ref) <= tol, rel_l2(got, ref)
    norms = np.sqrt(np.mean(ref ** 2, axis=0))
    top = norms.max()
    for i in range(ref.shape[1]):
        err = np.sqrt(np.mean((got[:, i] - ref[:, i]) ** 2))
        bound = tol * max(norms[i], floor * top)
        assert err <= bound, (i, err / max(norms[i], 1e-300), norms[i] / top)
