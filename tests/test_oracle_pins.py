"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test checks the oracle against a closed form, a brute-force computation, a
physical invariant or an independent route to the same number, chosen so that a
plausible mistake (a dropped term, a wrong sign, a swapped x/y, a wrong
normalisation) fails at least one of them.  ``test_oracle_mutations.py`` plants
such mistakes in the oracle and checks that these pins catch them.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
import workloads as W
from oracle import stem as O


def small_params(n=32, cell=(10.0, 12.0, 4.0), slices=2, dz=2.0, e=200.0, alpha=20.0,
                 ring=5.0, rings=40):
    return O.Params(cell, n, slices, dz, e, alpha, ring, rings)


# --------------------------------------------------------------------------- FFT
@pytest.mark.parametrize("shape", [(8, 8), (8, 16), (16, 16)])
def test_fft_conventions_vs_bruteforce_dft(shape):
    """Forward FFT is sum x e^{-2 pi i (jm/N + il/M)}; inverse has e^{+} and 1/(NM)."""
    rng = np.random.default_rng(0)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ny, nx = shape
    fwd = np.zeros(shape, complex)
    inv = np.zeros(shape, complex)
    for l in range(ny):
        for m in range(nx):
            acc_f = 0j
            acc_i = 0j
            for i in range(ny):
                for j in range(nx):
                    ang = 2 * math.pi * (j * m / nx + i * l / ny)
                    acc_f += x[i, j] * complex(math.cos(ang), -math.sin(ang))
                    acc_i += x[i, j] * complex(math.cos(ang), math.sin(ang))
            fwd[l, m] = acc_f
            inv[l, m] = acc_i / (nx * ny)
    assert np.max(np.abs(np.fft.fft2(x) - fwd)) < 1e-12 * np.max(np.abs(fwd))
    assert np.max(np.abs(np.fft.ifft2(x) - inv)) < 1e-12 * np.max(np.abs(inv))


# --------------------------------------------------------------- physical constants
@pytest.mark.parametrize("kev", [80.0, 200.0, 300.0])
def test_wavelength_and_sigma_from_si_constants(kev):
    """lambda = h / p with p from special relativity, sigma = 2 pi m e lambda / h^2
    (relativistic mass), both in SI units: an independent route to the same values."""
    h = 6.62607015e-34
    m0 = 9.1093837015e-31
    e = 1.602176634e-19
    c = 299792458.0
    v = kev * 1e3
    p = math.sqrt(e * v * (2 * m0 * c * c + e * v)) / c
    lam_si = h / p
    m = m0 * (1 + e * v / (m0 * c * c))
    sigma_si = 2 * math.pi * m * e * lam_si / (h * h)      # rad / (V m)
    assert O.wavelength(kev) == pytest.approx(lam_si * 1e10, rel=2e-9)
    assert O.interaction_constant(kev) == pytest.approx(sigma_si * 1e-10, rel=2e-9)


def test_wavelength_textbook_values():
    """Textbook relativistic wavelengths (4 significant digits)."""
    assert O.wavelength(200.0) == pytest.approx(0.02508, abs=1e-5)
    assert O.wavelength(300.0) == pytest.approx(0.01969, abs=1e-5)
    assert O.wavelength(100.0) == pytest.approx(0.03701, abs=1e-5)


# ------------------------------------------------ Eq. 1 + Eq. 2 closed forms
def _grating_closed_form(p, g, h, v0, v1, nmax=40):
    """Jacobi-Anger: exp(i a cos th) = sum_n i^n J_n(a) e^{i n th}.  After one slice
    (transmit, then propagate with the band limit) the Fourier coefficient at
    (m, n) = (k g, l h) is N^2 i^(k+l) J_k(sigma v0) J_l(sigma v1) M P(m, n)."""
    n = p.n
    out = np.zeros((n, n), complex)
    s = p.sigma
    for k in range(-nmax, nmax + 1):
        for l in range(-nmax, nmax + 1):
            m, q = k * g, l * h
            if abs(m) >= n // 2 or abs(q) >= n // 2:
                continue
            if 9 * (m * m + q * q) > n * n:
                continue
            kx, ky = m / p.cell[0], q / p.cell[1]
            prop = complex(math.cos(math.pi * p.lam * p.slice_dz * (kx * kx + ky * ky)),
                           -math.sin(math.pi * p.lam * p.slice_dz * (kx * kx + ky * ky)))
            out[q % n, m % n] += n * n * (1j ** (k + l)) * special.jv(k, s * v0) * special.jv(l, s * v1) * prop
    return out


def test_phase_grating_one_slice_jacobi_anger():
    p = small_params(n=64, cell=(10.0, 13.0, 50.0), slices=1, dz=50.0)
    g, h = 1, 2
    v0, v1 = 900.0, 500.0   # sigma*v ~ 0.66 and 0.36 rad at 200 keV
    j = np.arange(p.n)
    v = v0 * np.cos(2 * math.pi * g * j[None, :] / p.n) + v1 * np.cos(2 * math.pi * h * j[:, None] / p.n)
    t = O.transmission(p, v[None])
    psi = np.ones((1, p.n, p.n), complex)
    got = O.multislice_k(p, t, psi)[0]
    want = _grating_closed_form(p, g, h, v0, v1)
    assert np.max(np.abs(got - want)) < 1e-9 * p.n * p.n


def test_gaussian_beam_fresnel_closed_form():
    """Free-space Fresnel propagation (Eq. 2, V=0) of exp(-r^2/(2 w^2)) over
    distance z gives (w^2/w'^2) exp(-r^2/(2 w'^2)) with w'^2 = w^2 + i lambda z/(2 pi)."""
    p = O.Params((40.0, 40.0, 100.0), 256, 5, 20.0, 200.0, 20.0, 1.0, 10)
    w = 1.5
    x = np.arange(p.n) * p.dx - 20.0
    y = np.arange(p.n) * p.dy - 20.0
    r2 = x[None, :] ** 2 + y[:, None] ** 2
    psi0 = np.exp(-r2 / (2 * w * w))[None].astype(complex)
    t = np.ones((p.n_slices, p.n, p.n), complex)
    out = np.fft.ifft2(O.multislice_k(p, t, psi0))[0]
    z = p.n_slices * p.slice_dz
    w2 = w * w + 1j * p.lam * z / (2 * math.pi)
    want = (w * w / w2) * np.exp(-r2 / (2 * w2))
    assert np.max(np.abs(out - want)) < 1e-10


def _dft2_bruteforce(a, inverse=False):
    n = a.shape[0]
    k = np.arange(n)
    sgn = 1.0 if inverse else -1.0
    w = np.exp(sgn * 2j * math.pi * np.outer(k, k) / n)
    out = w @ a @ w.T
    return out / (n * n) if inverse else out


def test_multislice_bruteforce_8x8():
    """Three slices on an 8x8 grid with explicit DFT matrices and a Python loop."""
    p = O.Params((4.0, 5.0, 6.0), 8, 3, 2.0, 80.0, 40.0, 10.0, 20)
    rng = np.random.default_rng(5)
    v = rng.random((3, 8, 8)) * 50.0
    t = O.transmission(p, v)
    psi = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
    m = [j if j < 4 else j - 8 for j in range(8)]
    prop = np.zeros((8, 8), complex)
    for a in range(8):          # row: y frequency
        for b in range(8):      # column: x frequency
            if 9 * (m[a] ** 2 + m[b] ** 2) <= 64:
                k2 = (m[b] / 4.0) ** 2 + (m[a] / 5.0) ** 2
                prop[a, b] = complex(math.cos(math.pi * p.lam * 2.0 * k2), -math.sin(math.pi * p.lam * 2.0 * k2))
    cur = psi.copy()
    for s in range(3):
        tr = np.array([[complex(math.cos(p.sigma * v[s, i, j]), math.sin(p.sigma * v[s, i, j]))
                        for j in range(8)] for i in range(8)])
        spec = prop * _dft2_bruteforce(tr * cur)
        if s < 2:
            cur = _dft2_bruteforce(spec, inverse=True)
    got = O.multislice_k(p, t, psi[None])[0]
    assert np.max(np.abs(got - spec)) < 1e-11 * np.max(np.abs(spec))


# ---------------------------------------------------------------- invariants
def _random_trans(p, seed=1, vmax=60.0):
    rng = np.random.default_rng(seed)
    return O.transmission(p, rng.random((p.n_slices, p.n, p.n)) * vmax)


def test_transmission_is_unitary():
    p = small_params()
    t = _random_trans(p)
    rng = np.random.default_rng(2)
    psi = rng.standard_normal((p.n, p.n)) + 1j * rng.standard_normal((p.n, p.n))
    assert np.linalg.norm(t[0] * psi) == pytest.approx(np.linalg.norm(psi), rel=1e-14)


def test_norm_loss_equals_masked_energy_parseval():
    p = small_params(slices=1)
    t = _random_trans(p, vmax=300.0)
    rng = np.random.default_rng(3)
    psi = rng.standard_normal((1, p.n, p.n)) + 1j * rng.standard_normal((1, p.n, p.n))
    spec = np.fft.fft2(t[0] * psi[0])
    lost = np.sum(np.abs(spec[~O.bandlimit_mask(p.n)]) ** 2) / p.n ** 2
    out = np.fft.ifft2(O.multislice_k(p, t, psi)[0])
    assert np.sum(np.abs(out) ** 2) == pytest.approx(np.sum(np.abs(psi) ** 2) - lost, rel=1e-12)
    assert lost > 1e-3 * np.sum(np.abs(psi) ** 2)   # the mask really removes something


def test_linearity():
    p = small_params(slices=3)
    t = _random_trans(p)
    rng = np.random.default_rng(4)
    a = rng.standard_normal((1, p.n, p.n)) + 1j * rng.standard_normal((1, p.n, p.n))
    b = rng.standard_normal((1, p.n, p.n)) + 1j * rng.standard_normal((1, p.n, p.n))
    lhs = O.multislice_k(p, t, (2 - 1j) * a + 0.5j * b)
    rhs = (2 - 1j) * O.multislice_k(p, t, a) + 0.5j * O.multislice_k(p, t, b)
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(lhs))


def test_probe_normalisation_and_free_space_rings():
    """V = 0: |Psi_hat| = |psi_hat| pixelwise, so ring i holds |A cap ring i| / |A|
    (counted here point by point over the integer lattice; Lx != Ly)."""
    lx, ly = 16.0, 20.0
    p = O.Params((lx, ly, 20.0), 64, 4, 5.0, 80.0, 20.0, 2.0, 40)
    t = np.ones((p.n_slices, p.n, p.n), complex)
    xy = np.array([[3.3, 7.1], [0.0, 0.0], [15.9, 1.2]])
    rings = O.multislice_rings(p, t, xy)
    counts = np.zeros(p.n_rings)
    n_ap = 0
    for a in range(-32, 32):          # x frequency index
        for b in range(-32, 32):      # y frequency index
            if 9 * (a * a + b * b) > 64 * 64:
                continue
            ang = p.lam * math.sqrt((a / lx) ** 2 + (b / ly) ** 2) * 1000.0
            if ang <= 20.0:
                n_ap += 1
                r = int(math.floor(ang / 2.0))
                if r < p.n_rings:
                    counts[r] += 1
    want = counts / n_ap
    for row in rings:
        assert np.max(np.abs(row - want)) < 1e-13
        assert row.sum() == pytest.approx(1.0, abs=1e-13)


def test_ring_table_orientation_hand_values():
    """A few pixels worked by hand (80 keV, lambda = 0.0417572 A, Lx = 16, Ly = 20 A,
    2 mrad rings): x frequency index 5 -> 13.05 mrad (ring 6), y index 5 -> 10.44
    mrad (ring 5), (m, n) = (-3, 4) -> 11.45 mrad (ring 5); outside the 2/3 band
    limit -> -1."""
    p = O.Params((16.0, 20.0, 20.0), 64, 4, 5.0, 80.0, 20.0, 2.0, 40)
    t = O.ring_table(p)
    assert t[0, 5] == 6
    assert t[5, 0] == 5
    assert t[4, 64 - 3] == 5
    assert t[0, 22] == -1          # 9 * 22^2 > 64^2
    assert t[0, 21] == int(0.0417572 * 21 / 16 * 1000 // 2)


def test_detector_total_never_exceeds_one():
    p = O.Params((16.0, 16.0, 20.0), 64, 5, 4.0, 80.0, 25.0, 4.0, 100)
    t = _random_trans(p, vmax=100.0)
    rings = O.multislice_rings(p, t, np.array([[4.0, 4.0], [8.5, 12.25]]))
    assert np.all(rings >= 0)
    assert np.all(rings.sum(axis=1) <= 1.0 + 1e-12)
    assert np.all(rings.sum(axis=1) > 0.5)


def test_cyclic_shift_covariance():
    """Moving every atom and the probe by a whole number of pixels leaves the rings unchanged."""
    p = O.Params((8.0, 8.0, 4.0), 64, 2, 2.0, 200.0, 20.0, 5.0, 30)
    rng = np.random.default_rng(6)
    xyz = rng.random((12, 3)) * np.array(p.cell)
    gauss = np.tile(np.array([5.0, 0.2, 2.0, 0.6], np.float32), (12, 1))
    shift = np.array([5 * p.dx, 11 * p.dy, 0.0])
    xyz2 = xyz + shift
    xyz2[:, 0] %= p.cell[0]
    xyz2[:, 1] %= p.cell[1]
    t1 = O.transmission(p, O.projected_potential(p, xyz, gauss))
    t2 = O.transmission(p, O.projected_potential(p, xyz2, gauss))
    xy = np.array([[1.1, 2.3], [6.0, 0.5]])
    r1 = O.multislice_rings(p, t1, xy)
    r2 = O.multislice_rings(p, t2, xy + shift[:2])
    assert np.max(np.abs(r1 - r2)) < 1e-10


# ---------------------------------------------------------------- potentials
def test_slice_assignment():
    p = O.Params((10.0, 10.0, 20.0), 32, 10, 2.0, 200.0, 20.0, 1.0, 10)
    z = np.array([0.0, 0.5, 1.999, 2.0, 3.9, 19.99, 20.0, 25.0])
    assert list(O.slice_index(p, z)) == [0, 0, 0, 1, 1, 9, 9, 9]


def test_potential_sum_rule_and_peak():
    """sum_r V dx dy = sum_atoms 2 pi (A1 s1^2 + A2 s2^2) (Gaussian integral; the grid
    sum of a smooth periodic function equals its integral up to e^{-2 pi^2 s^2/dx^2})."""
    p = O.Params((12.0, 10.0, 4.0), 160, 2, 2.0, 200.0, 20.0, 1.0, 10)
    xyz = np.array([[0.05, 9.97, 0.3],          # near a corner: periodic images
                    [6.0, 5.0, 3.0],            # exactly on pixel (80, 80)
                    [11.99, 4.2, 1.0]])
    gauss = np.tile(np.array([5.0, 0.2, 2.0, 0.6], np.float32), (3, 1))
    v = O.projected_potential(p, xyz, gauss)
    s1, s2 = float(np.float32(0.2)), float(np.float32(0.6))   # the parameters are float32
    per_atom = 2 * math.pi * (5.0 * s1 ** 2 + 2.0 * s2 ** 2)
    assert v[0].sum() * p.dx * p.dy == pytest.approx(2 * per_atom, rel=1e-9)
    assert v[1].sum() * p.dx * p.dy == pytest.approx(per_atom, rel=1e-9)
    # atom 2 sits on pixel (i=80, j=80) of slice 1: peak is A1 + A2 (plus the far
    # tail of atom 3 in the same slice, which is below 1e-9 there)
    assert v[1, 80, 80] == pytest.approx(7.0, rel=1e-9)


def test_potential_single_atom_profile():
    """One atom: V at a pixel offset (a, b) from it is 5 e^{-d^2/0.08} + 2 e^{-d^2/0.72}."""
    p = O.Params((10.0, 10.0, 4.0), 100, 1, 4.0, 200.0, 20.0, 1.0, 10)
    xyz = np.array([[5.0, 5.0, 1.0]])
    gauss = np.array([[5.0, 0.2, 2.0, 0.6]], np.float32)
    v = O.projected_potential(p, xyz, gauss)[0]
    for (a, b) in [(0, 0), (1, 0), (3, 4), (-7, 2), (20, -30)]:
        d2 = (a * 0.1) ** 2 + (b * 0.1) ** 2
        s1, s2 = float(np.float32(0.2)), float(np.float32(0.6))
        want = 5 * math.exp(-d2 / (2 * s1 * s1)) + 2 * math.exp(-d2 / (2 * s2 * s2))
        assert v[50 + b, 50 + a] == pytest.approx(want, rel=1e-7, abs=1e-15)


# -------------------------------------------------------------------- PRISM
def test_prism_f1_equals_multislice():
    """PRISM with f = 1 is multislice by linearity (the key PRISM pin)."""
    p = O.Params((8.0, 8.0, 6.0), 32, 3, 2.0, 200.0, 30.0, 4.0, 40)
    rng = np.random.default_rng(7)
    t = O.transmission(p, rng.random((3, 32, 32)) * 80.0)
    xy = np.array([[0.3, 0.7], [4.4, 2.25], [7.9, 7.9]])
    ms = O.multislice_rings(p, t, xy)
    beams = O.prism_beams(p, 1)
    pr = O.prism_rings(p, O.prism_smatrix(p, t, beams), beams, 1, xy)
    assert np.max(np.abs(ms - pr)) < 1e-12


@pytest.mark.parametrize("f", [2, 4])
def test_prism_free_space_closed_form(f):
    """V = 0, any f: S_b = P^S psi_b, each beam lands on one coarse pixel of the window
    FFT with weight W^4 |c_b|^2, so ring i holds |beams in ring i| / n_b."""
    p = O.Params((16.0, 16.0, 6.0), 64, 3, 2.0, 80.0, 30.0, 3.0, 40)
    t = np.ones((3, 64, 64), complex)
    beams = O.prism_beams(p, f)
    s = O.prism_smatrix(p, t, beams)
    xy = np.array([[1.0, 2.0], [9.3, 14.1]])
    rings = O.prism_rings(p, s, beams, f, xy)
    counts = np.zeros(p.n_rings)
    for (m, n) in beams:
        ang = p.lam * math.sqrt((m / 16.0) ** 2 + (n / 16.0) ** 2) * 1000.0
        r = int(math.floor(ang / 3.0))
        if r < p.n_rings:
            counts[r] += 1
    for row in rings:
        assert np.max(np.abs(row - counts / len(beams))) < 1e-12


def test_prism_beam_set_every_fth():
    p = O.Params((20.0, 20.0, 6.0), 128, 3, 2.0, 200.0, 20.0, 1.0, 40)
    b1 = {tuple(b) for b in O.prism_beams(p, 1)}
    b4 = {tuple(b) for b in O.prism_beams(p, 4)}
    assert b4 == {b for b in b1 if b[0] % 4 == 0 and b[1] % 4 == 0}
    assert (0, 0) in b4
    # symmetric under (m, n) -> (-m, -n) for a square cell
    assert all((-m, -n) in b1 for (m, n) in b1)


def test_prism_window_origin():
    p = O.Params((16.0, 16.0, 6.0), 64, 3, 2.0, 200.0, 20.0, 1.0, 40)
    xy = np.array([[0.0, 0.0], [0.125, 0.124], [15.9, 8.0]])   # dx = 0.25
    org = O.prism_window_origin(p, 4, xy)        # W = 16
    assert org.tolist() == [[56, 56], [57, 56], [(64 - 8) % 64, 24]]


@pytest.mark.parametrize("f", [2, 4])
def test_prism_shift_covariance_non_square_cell(f):
    """Moving every atom by whole pixels (a dx, b dy) with a != b in a cell with
    Lx != Ly and the probes by the same vector leaves the PRISM window waves
    unchanged: each exit wave becomes S_b(r - s) exp(2 pi i k_b . s), the
    coefficient picks up exp(-2 pi i k_b . s) and the window origin moves by
    (a, b) pixels.  This fixes which axis of the window crop follows x and
    which follows y (a crop with the axes exchanged moves the window by (b, a)
    and fails), which neither f = 1 nor free space can see."""
    p = O.Params((10.0, 13.0, 4.0), 32, 2, 2.0, 200.0, 30.0, 4.0, 40)
    rng = np.random.default_rng(61)
    xyz = rng.random((14, 3)) * np.array(p.cell)
    gauss = np.tile(np.array([5.0, 0.2, 2.0, 0.6], np.float32), (14, 1))
    a, b = 3, -5
    shift = np.array([a * p.dx, b * p.dy, 0.0])
    xyz2 = xyz + shift
    xyz2[:, 0] %= p.cell[0]
    xyz2[:, 1] %= p.cell[1]
    t1 = O.transmission(p, O.projected_potential(p, xyz, gauss))
    t2 = O.transmission(p, O.projected_potential(p, xyz2, gauss))
    beams = O.prism_beams(p, f)
    s1 = O.prism_smatrix(p, t1, beams)
    s2 = O.prism_smatrix(p, t2, beams)
    # probe positions a quarter pixel off the rounding boundary of the origin
    xy = np.array([[1.1 * p.dx, 2.3 * p.dy], [20.2 * p.dx, 7.9 * p.dy], [30.7 * p.dx, 25.4 * p.dy]])
    xy2 = xy + shift[:2]
    assert np.array_equal(O.prism_window_origin(p, f, xy2),
                          np.mod(O.prism_window_origin(p, f, xy) + np.array([a, b]), p.n))
    w1 = O.prism_window_waves(p, s1, beams, f, xy)
    w2 = O.prism_window_waves(p, s2, beams, f, xy2)
    assert np.max(np.abs(w1 - w2)) < 1e-10 * np.max(np.abs(w1))
    r1 = O.prism_rings(p, s1, beams, f, xy)
    r2 = O.prism_rings(p, s2, beams, f, xy2)
    assert np.max(np.abs(r1 - r2)) < 1e-10 * np.max(r1)
    # the shift does change the window waves at a fixed probe position
    assert np.max(np.abs(O.prism_window_waves(p, s2, beams, f, xy) - w1)) > 1e-3 * np.max(np.abs(w1))


# -------------------------------------------------------------- aberrations
def test_defocus_equals_free_propagation():
    """A probe with defocus C1 is the in-focus probe propagated by C1 with Eq. 2's
    propagator (a different code path of the oracle)."""
    p0 = O.Params((20.0, 24.0, 10.0), 128, 1, 37.0, 200.0, 25.0, 1.0, 30)
    p1 = O.Params((20.0, 24.0, 10.0), 128, 1, 37.0, 200.0, 25.0, 1.0, 30, defocus=37.0)
    xy = np.array([[3.1, 17.4]])
    got = O.probe_k(p1, xy)[0]
    want = O.probe_k(p0, xy)[0] * O.propagator(p0)      # propagate by dz = 37 A = C1
    assert np.max(np.abs(got - want)) < 1e-13


def test_spherical_aberration_hand_value():
    """Cs = 1 mm at 200 keV: chi at k = 0.5 1/A is (pi/2) Cs lambda^3 k^4
    = (pi/2) * 1e7 * 0.0250793^3 * 0.0625 = 15.486 rad (worked by hand)."""
    p = O.Params((20.0, 20.0, 10.0), 128, 1, 1.0, 200.0, 30.0, 1.0, 30, cs=1e7)
    assert O.aberration_chi(p, 0.5, 0.0) == pytest.approx(15.486, abs=2e-3)
    assert O.aberration_chi(p, 0.3, 0.4) == pytest.approx(15.486, abs=2e-3)   # depends on |k| only


def test_prism_f1_equals_multislice_with_aberrations():
    p = O.Params((8.0, 8.0, 6.0), 32, 3, 2.0, 200.0, 30.0, 4.0, 40, defocus=50.0, cs=2e6)
    rng = np.random.default_rng(9)
    t = O.transmission(p, rng.random((3, 32, 32)) * 80.0)
    xy = np.array([[0.3, 0.7], [4.4, 2.25]])
    beams = O.prism_beams(p, 1)
    ms = O.multislice_rings(p, t, xy)
    pr = O.prism_rings(p, O.prism_smatrix(p, t, beams), beams, 1, xy)
    assert np.max(np.abs(ms - pr)) < 1e-12
    # and the aberration changes the result
    p0 = O.Params((8.0, 8.0, 6.0), 32, 3, 2.0, 200.0, 30.0, 4.0, 40)
    assert np.max(np.abs(ms - O.multislice_rings(p0, t, xy))) > 1e-4


# ------------------------------------------------------ detectors, 4D output
def test_detector_edges_free_space_closed_form():
    """Annular detectors with arbitrary edges at V = 0: each holds the fraction of
    aperture pixels whose angle falls in it (counted point by point)."""
    p = O.Params((16.0, 20.0, 20.0), 64, 2, 5.0, 80.0, 20.0, 2.0, 40)
    edges = [0.0, 7.5, 13.25, 20.0, 41.0, 60.0]
    t = np.ones((2, 64, 64), complex)
    rings = O.multislice_rings(p, t, np.array([[1.0, 2.0]]), edges=edges)[0]
    counts = np.zeros(len(edges) - 1)
    n_ap = 0
    for a in range(-32, 32):
        for b in range(-32, 32):
            if 9 * (a * a + b * b) > 64 * 64:
                continue
            ang = p.lam * math.sqrt((a / 16.0) ** 2 + (b / 20.0) ** 2) * 1000.0
            if ang <= 20.0:
                n_ap += 1
                for i in range(len(edges) - 1):
                    if edges[i] <= ang < edges[i + 1]:
                        counts[i] += 1
    assert np.max(np.abs(rings - counts / n_ap)) < 1e-13
    assert rings[3:].sum() == pytest.approx(0.0, abs=1e-15)     # dark field is dark in vacuum


def test_4d_output_free_space_and_ring_sums():
    """V = 0: the diffraction pattern is 1/|A| on aperture pixels and 0 elsewhere;
    with a specimen, summing the pattern over a ring gives that ring's output."""
    p = O.Params((16.0, 16.0, 8.0), 64, 2, 4.0, 200.0, 25.0, 2.0, 40)
    xy = np.array([[3.3, 1.1], [9.0, 12.5]])
    dp0 = O.multislice_dp(p, np.ones((2, 64, 64), complex), xy)
    ap = O.aperture(p)
    assert np.max(np.abs(dp0 - ap[None] / ap.sum())) < 1e-14
    rng = np.random.default_rng(8)
    t = O.transmission(p, rng.random((2, 64, 64)) * 70.0)
    dp = O.multislice_dp(p, t, xy)
    rings = O.multislice_rings(p, t, xy)
    table = O.ring_table(p)
    for i in (0, 5, 17):
        assert np.allclose(dp[:, table == i].sum(axis=1), rings[:, i], rtol=1e-12, atol=1e-16)


def test_frozen_phonon_mean_of_translated_configurations():
    """Configurations that are whole-pixel translations of one structure: each
    one's rings equal the untranslated structure's rings at the probe moved the
    opposite way (exact: a whole-pixel shift moves the sampled potential and
    the probe's phase ramp together), so the frozen-phonon mean is the mean
    over moved probes.  Identical configurations reduce to one run, and the
    PRISM branch at f = 1 is multislice."""
    w = W.Workload("fp", (8.0, 8.0, 4.0), 6, 32, 2, 2.0, 200.0, 20.0, 0, 5.0, 10)
    p = O.params_from(w)
    xyz, gauss = W.atoms(w, seed=5)
    xy = W.random_positions(w, 3, seed=6)
    shifts = [(0, 0), (3, -2), (-5, 7)]
    configs = [xyz + np.array([a * p.dx, b * p.dy, 0.0]) for a, b in shifts]
    got = O.frozen_phonon_rings(p, configs, gauss, xy)
    t = O.transmission(p, O.projected_potential(p, xyz, gauss))
    moved = [O.multislice_rings(p, t, xy - np.array([a * p.dx, b * p.dy])) for a, b in shifts]
    assert np.allclose(got, np.mean(moved, axis=0), rtol=1e-9, atol=1e-14)
    assert not np.allclose(moved[0], moved[1], rtol=1e-3)          # the shifts do change the rings
    assert np.allclose(O.frozen_phonon_rings(p, [xyz, xyz], gauss, xy), O.multislice_rings(p, t, xy),
                       rtol=1e-12, atol=1e-15)
    assert np.allclose(O.frozen_phonon_rings(p, configs, gauss, xy, algo="prism", f=1), got,
                       rtol=1e-9, atol=1e-14)


def test_propagator_semigroup():
    """Free propagation composes: P(dz1) P(dz2) = P(dz1 + dz2) inside the band
    limit (and 0 outside), P(0) is the band-limit mask, and a free-space wave
    propagated through two half-thickness slices equals one full slice."""
    import dataclasses
    w = W.Workload("sg", (10.0, 14.0, 4.0), 0, 32, 2, 2.0, 200.0, 20.0, 0, 5.0, 8)
    p = O.params_from(w)
    pa = dataclasses.replace(p, slice_dz=0.7)
    pb = dataclasses.replace(p, slice_dz=1.9)
    pab = dataclasses.replace(p, slice_dz=2.6)
    p0 = dataclasses.replace(p, slice_dz=0.0)
    assert np.allclose(O.propagator(pa) * O.propagator(pb), O.propagator(pab), atol=1e-13)
    assert np.array_equal(O.propagator(p0), O.bandlimit_mask(p.n).astype(np.complex128))
    half = dataclasses.replace(p, n_slices=2, slice_dz=1.3)
    full = dataclasses.replace(p, n_slices=1, slice_dz=2.6)
    xy = np.array([[3.3, 7.1]])
    psi = O.probe_k(p, xy)
    a = O.multislice_k(half, np.ones((2, p.n, p.n), complex), psi)
    b = O.multislice_k(full, np.ones((1, p.n, p.n), complex), psi)
    assert np.allclose(a, b, atol=1e-12)


# ------------------------------------------------- Fourier-cropped S-matrix
def test_cropped_smatrix_samples_the_band_limited_wave():
    """S'_b on the cropped grid N' = 3N/4 is the band-limited exit wave S_b
    evaluated at the points (j Lx / N', i Ly / N'): checked against an explicit
    trigonometric sum over the band (Lx != Ly), and zero-padding its spectrum
    back to N reproduces S_b on the simulation grid."""
    p = O.Params((5.0, 6.0, 4.0), 16, 2, 2.0, 200.0, 60.0, 4.0, 40)
    n, n2 = 16, O.cropped_grid(16)
    assert n2 == 12
    t = _random_trans(p, seed=11, vmax=40.0)
    beams = O.prism_beams(p, 1)[::3]
    full = O.prism_smatrix(p, t, beams)
    crop = O.prism_smatrix_cropped(p, t, beams)
    assert crop.shape == (len(beams), n2, n2)
    band = [(m, k) for m in range(-n // 2, n // 2) for k in range(-n // 2, n // 2) if 9 * (m * m + k * k) <= n * n]
    jj = np.arange(n2)
    for b in range(len(beams)):
        spec = np.fft.fft2(full[b])
        want = np.zeros((n2, n2), complex)
        for (m, k) in band:
            want += spec[k % n, m % n] * np.exp(2j * math.pi * (m * jj[None, :] + k * jj[:, None]) / n2)
        want /= n * n
        assert np.max(np.abs(crop[b] - want)) < 1e-12 * np.max(np.abs(want))
        # zero-padded back to N: the band-limited wave itself
        sc = np.fft.fft2(crop[b]) * (n / n2) ** 2
        pad = np.zeros((n, n), complex)
        f2 = O.freq_index(n2)
        pad[np.ix_(np.mod(f2, n), np.mod(f2, n))] = sc
        assert np.max(np.abs(np.fft.ifft2(pad) - full[b])) < 1e-12 * np.max(np.abs(full[b]))


def test_prism_cropped_f1_equals_multislice():
    """With f = 1 the window is the whole cropped cell and its FFT holds the
    multislice exit spectrum on every in-band frequency: the rings are those of
    multislice."""
    p = O.Params((8.0, 9.0, 6.0), 32, 3, 2.0, 200.0, 30.0, 4.0, 40)
    rng = np.random.default_rng(12)
    t = O.transmission(p, rng.random((3, 32, 32)) * 80.0)
    xy = np.array([[0.3, 0.7], [4.4, 2.25], [7.9, 8.9]])
    beams = O.prism_beams(p, 1)
    s = O.prism_smatrix_cropped(p, t, beams)
    pr = O.prism_rings(p, s, beams, 1, xy, grid=O.cropped_grid(p.n))
    assert np.max(np.abs(pr - O.multislice_rings(p, t, xy))) < 1e-12


@pytest.mark.parametrize("f", [2, 4])
def test_prism_cropped_free_space_closed_form(f):
    """V = 0: each cropped exit wave is a plane wave sampled on the N' grid, whose
    window (W' = N'/f pixels over L/f) holds a whole number of its periods, so each
    beam lands on one window-FFT pixel: ring i holds |beams in ring i| / n_b."""
    p = O.Params((16.0, 16.0, 6.0), 64, 3, 2.0, 80.0, 30.0, 3.0, 40)
    t = np.ones((3, 64, 64), complex)
    beams = O.prism_beams(p, f)
    s = O.prism_smatrix_cropped(p, t, beams)
    xy = np.array([[1.0, 2.0], [9.3, 14.1]])
    rings = O.prism_rings(p, s, beams, f, xy, grid=O.cropped_grid(64))
    counts = np.zeros(p.n_rings)
    for (m, n) in beams:
        r = int(math.floor(p.lam * math.sqrt((m / 16.0) ** 2 + (n / 16.0) ** 2) * 1000.0 / 3.0))
        if r < p.n_rings:
            counts[r] += 1
    for row in rings:
        assert np.max(np.abs(row - counts / len(beams))) < 1e-12


def test_prism_cropped_shift_covariance_non_square_cell():
    """Atoms moved by (4, -8) pixels of the simulation grid = (3, -6) pixels of
    the cropped grid (Lx != Ly) and probes moved by the same vector: the cropped
    window waves are unchanged (fixes the crop orientation and the window origin
    on the cropped grid)."""
    p = O.Params((10.0, 13.0, 4.0), 32, 2, 2.0, 200.0, 30.0, 4.0, 40)
    n2 = O.cropped_grid(p.n)
    rng = np.random.default_rng(63)
    xyz = rng.random((14, 3)) * np.array(p.cell)
    gauss = np.tile(np.array([5.0, 0.2, 2.0, 0.6], np.float32), (14, 1))
    shift = np.array([4 * p.dx, -8 * p.dy, 0.0])
    xyz2 = xyz + shift
    xyz2[:, 0] %= p.cell[0]
    xyz2[:, 1] %= p.cell[1]
    t1 = O.transmission(p, O.projected_potential(p, xyz, gauss))
    t2 = O.transmission(p, O.projected_potential(p, xyz2, gauss))
    beams = O.prism_beams(p, 2)
    s1 = O.prism_smatrix_cropped(p, t1, beams)
    s2 = O.prism_smatrix_cropped(p, t2, beams)
    dxc, dyc = p.cell[0] / n2, p.cell[1] / n2
    xy = np.array([[1.1 * dxc, 2.3 * dyc], [15.2 * dxc, 7.9 * dyc], [22.7 * dxc, 19.4 * dyc]])
    w1 = O.prism_window_waves(p, s1, beams, 2, xy, n2)
    w2 = O.prism_window_waves(p, s2, beams, 2, xy + shift[:2], n2)
    assert np.max(np.abs(w1 - w2)) < 1e-10 * np.max(np.abs(w1))
    assert np.max(np.abs(O.prism_window_waves(p, s2, beams, 2, xy, n2) - w1)) > 1e-5 * np.max(np.abs(w1))
