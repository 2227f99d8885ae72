"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each.

Each case replaces one oracle function with a subtly wrong version and runs the
pins that should notice; the case passes when at least one of them fails.
"""
import math

import numpy as np
import pytest

from oracle import stem as O
import tests.test_oracle_pins as pins


def _fails(fn, *args):
    try:
        fn(*args)
    except AssertionError:
        return True
    return False


def _prop_flipped(p):
    return np.conj(O._orig_propagator(p))


def _prop_unmasked(p):
    m = O.freq_index(p.n).astype(np.float64)
    kx = m / p.cell[0]
    ky = m / p.cell[1]
    k2 = kx[None, :] ** 2 + ky[:, None] ** 2
    return np.exp(-1j * math.pi * p.lam * p.slice_dz * k2)


def _prop_xy_swapped(p):
    m = O.freq_index(p.n).astype(np.float64)
    kx = m / p.cell[1]
    ky = m / p.cell[0]
    k2 = kx[None, :] ** 2 + ky[:, None] ** 2
    return np.exp(-1j * math.pi * p.lam * p.slice_dz * k2) * O.bandlimit_mask(p.n)


def _trans_flipped(p, v):
    return np.exp(-1j * p.sigma * v)


def _angle_xy_swapped(p):
    m = O.freq_index(p.n).astype(np.float64)
    kx = m / p.cell[1]
    ky = m / p.cell[0]
    return p.lam * np.sqrt(kx[None, :] ** 2 + ky[:, None] ** 2) * 1000.0


def _probe_unnormalised(p, xy):
    return O._orig_probe_k(p, xy) * math.sqrt(int(O.aperture(p).sum()))


def _origin_round_down(p, f, xy, grid=None):
    n = p.n if grid is None else grid
    w = n // f
    xy = np.atleast_2d(xy)
    ox = np.floor(xy[:, 0] / (p.cell[0] / n)).astype(np.int64) - w // 2
    oy = np.floor(xy[:, 1] / (p.cell[1] / n)).astype(np.int64) - w // 2
    return np.stack([np.mod(ox, n), np.mod(oy, n)], axis=1)


def _coef_conj(p, beams, xy):
    return np.conj(O._orig_prism_coefficients(p, beams, xy))


def _slice_round(p, z):
    return np.clip(np.round(np.asarray(z) / p.slice_dz).astype(np.int64), 0, p.n_slices - 1)


def _potential_one_gaussian(p, xyz, gauss):
    g = np.array(gauss, dtype=np.float32).copy()
    g[:, 2] = 0.0
    return O._orig_projected_potential(p, xyz, g)


def _lambda_nonrel(e):
    return O.HC_KEV_A / math.sqrt(2.0 * O.MC2_KEV * e)


def _ms_last_slice_unpropagated(p, trans, psi):
    prop = O.propagator(p)
    psi = np.asarray(psi, dtype=np.complex128)
    for s in range(p.n_slices):
        if s < p.n_slices - 1:
            psi = np.fft.ifft2(prop * np.fft.fft2(trans[s] * psi, axes=(-2, -1)), axes=(-2, -1))
        else:
            return O.bandlimit_mask(p.n) * np.fft.fft2(trans[s] * psi, axes=(-2, -1))


def _chi_defocus_flipped(p, kx, ky):
    k2 = kx * kx + ky * ky
    return -math.pi * p.lam * p.defocus * k2 + 0.5 * math.pi * p.cs * p.lam ** 3 * k2 * k2


def _chi_cs_no_lambda_cubed(p, kx, ky):
    k2 = kx * kx + ky * ky
    return math.pi * p.lam * p.defocus * k2 + 0.5 * math.pi * p.cs * p.lam * k2 * k2


def _window_crop_axes_swapped(p, smatrix, beams, f, xy, grid=None):
    # the window's rows taken from the x origin and its columns from the y origin
    w = p.n // f
    org = O.prism_window_origin(p, f, xy)
    coef = O.prism_coefficients(p, beams, xy)
    out = np.empty((org.shape[0], w, w), dtype=np.complex128)
    u = np.arange(w)
    for i in range(org.shape[0]):
        rows = np.mod(org[i, 0] + u, p.n)
        cols = np.mod(org[i, 1] + u, p.n)
        out[i] = np.tensordot(coef[i], O._smatrix_crop(smatrix, rows, cols), axes=(0, 0))
    return out


def _cropped_unnormalised(p, trans, beams, chunk=16):
    # the inverse transform's 1/N'^2 left in place of 1/N^2
    return O._orig_prism_smatrix_cropped(p, trans, beams, chunk) * (p.n / float(O.cropped_grid(p.n))) ** 2


def _cropped_first_indices(p, trans, beams, chunk=16):
    # the first N' FFT indices kept instead of the N' signed frequencies
    n2 = O.cropped_grid(p.n)
    psi = O.plane_waves(p, beams)
    spec = O.multislice_k(p, trans, psi)[:, :n2, :n2]
    return np.fft.ifft2(spec, axes=(-2, -1)) * (float(n2) / p.n) ** 2


def _fp_first_config_only(p, configs, gauss, xy, algo="ms", f=1):
    # every configuration replaced by the first one
    return O._orig_frozen_phonon_rings(p, [configs[0]] * len(configs), gauss, xy, algo, f)


def _fp_sum_not_mean(p, configs, gauss, xy, algo="ms", f=1):
    return O._orig_frozen_phonon_rings(p, configs, gauss, xy, algo, f) * len(configs)


CASES = [
    ("propagator", _prop_flipped, [pins.test_phase_grating_one_slice_jacobi_anger,
                                   pins.test_gaussian_beam_fresnel_closed_form]),
    ("propagator", _prop_unmasked, [pins.test_norm_loss_equals_masked_energy_parseval]),
    ("propagator", _prop_xy_swapped, [pins.test_phase_grating_one_slice_jacobi_anger]),
    ("transmission", _trans_flipped, [pins.test_phase_grating_one_slice_jacobi_anger]),
    ("angle_mrad", _angle_xy_swapped, [pins.test_ring_table_orientation_hand_values]),
    ("probe_k", _probe_unnormalised, [pins.test_probe_normalisation_and_free_space_rings]),
    ("prism_window_origin", _origin_round_down, [pins.test_prism_window_origin]),
    ("prism_coefficients", _coef_conj, [pins.test_prism_f1_equals_multislice]),
    ("prism_window_waves", _window_crop_axes_swapped,
     [lambda: pins.test_prism_shift_covariance_non_square_cell(2),
      lambda: pins.test_prism_shift_covariance_non_square_cell(4)]),
    ("slice_index", _slice_round, [pins.test_slice_assignment]),
    ("prism_smatrix_cropped", _cropped_unnormalised, [pins.test_cropped_smatrix_samples_the_band_limited_wave,
                                                      pins.test_prism_cropped_f1_equals_multislice]),
    ("prism_smatrix_cropped", _cropped_first_indices, [pins.test_cropped_smatrix_samples_the_band_limited_wave,
                                                       pins.test_prism_cropped_f1_equals_multislice]),
    ("projected_potential", _potential_one_gaussian, [pins.test_potential_sum_rule_and_peak]),
    ("wavelength", _lambda_nonrel, [pins.test_wavelength_textbook_values]),
    ("multislice_k", _ms_last_slice_unpropagated, [pins.test_phase_grating_one_slice_jacobi_anger]),
    ("aberration_chi", _chi_defocus_flipped, [pins.test_defocus_equals_free_propagation]),
    ("aberration_chi", _chi_cs_no_lambda_cubed, [pins.test_spherical_aberration_hand_value]),
    ("frozen_phonon_rings", _fp_first_config_only, [pins.test_frozen_phonon_mean_of_translated_configurations]),
    ("frozen_phonon_rings", _fp_sum_not_mean, [pins.test_frozen_phonon_mean_of_translated_configurations]),
]


@pytest.mark.parametrize("name,mutant,checks", CASES, ids=[f"{c[0]}:{c[1].__name__}" for c in CASES])
def test_pins_catch_planted_mistake(monkeypatch, name, mutant, checks):
    monkeypatch.setattr(O, "_orig_" + name, getattr(O, name), raising=False)
    monkeypatch.setattr(O, name, mutant)
    caught = [getattr(c, "__name__", "check") for c in checks if _fails(c)]
    assert caught, f"no pin caught the mutation {mutant.__name__} of {name}"
