"""FP64 CPU oracle for multislice and PRISM STEM simulation (test infrastructure).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / ``--impl reference`` legs may import it.  The
product path (``paper_1706_08563_b300``) never imports, calls or links it, and
this package shares no code with the CUDA path: the two are written
independently from the paper (Methods section, Eq. 1 and Eq. 2; "PRISM Probe
Simulations"; "Multislice Probe Simulations").  The only module both sides use is
``workloads`` (seeded input generation, no method arithmetic).

Every function is plain NumPy in float64 / complex128.  The FFT is NumPy's
(a library primitive used as one step); nothing is blocked, fused or reordered
beyond what the method states.

Pins (see ``tests/test_oracle_pins.py``): brute-force DFTs, textbook electron
wavelengths, a Jacobi-Anger closed form for a phase grating followed by Fresnel
propagation, a Gaussian-beam Fresnel closed form, V=0 closed forms for
multislice and PRISM rings, PRISM f=1 == multislice, norm bookkeeping
(Parseval), linearity, cyclic-shift covariance, analytic single-atom
potentials and the Gaussian sum rule; PRISM shift covariance in a cell with
Lx != Ly (fixes the window crop's axes); the Fourier-cropped S-matrix against
an explicit trigonometric sum over the band, its zero-padded inverse, f = 1
against multislice, the free-space closed form and shift covariance on the
cropped grid.

Every function above has at least one such pin.  What no pin bounds is the
approximation PRISM f > 1 itself makes (its distance from multislice, which
the paper describes only qualitatively for f = 4): the oracle computes the
same approximate algorithm in FP64, the GPU path is held to the oracle's
PRISM, and the distance to multislice is reported, not asserted.
"""
from .stem import *  # noqa: F401,F403
