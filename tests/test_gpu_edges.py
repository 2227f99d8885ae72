"""Degenerate and extreme cases of the method, through the C ABI."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import stem as O

pytestmark = pytest.mark.gpu


def test_zero_aperture_is_a_plane_wave_and_one_beam():
    """alpha = 0: the aperture is the single pixel k = 0 (a plane wave), PRISM has one
    beam, and in vacuum all intensity stays in ring 0."""
    from paper_1706_08563_b300 import api
    w = W.Workload("z", (12.0, 12.0, 4.0), 0, 64, 2, 2.0, 200.0, 0.0, 2, 1.0, 10)
    plan = api.Plan.from_workload(w)
    assert plan.n_aperture == 1
    assert plan.prism_beams(1).tolist() == [[0, 0]]
    t = torch.ones((2, 64, 64), dtype=torch.complex64, device="cuda")
    xy = torch.tensor([[1.0, 2.0], [7.7, 0.3]], dtype=torch.float64, device="cuda")
    r = plan.multislice(t, xy).cpu().numpy()
    assert np.allclose(r[:, 0], 1.0, atol=1e-6) and np.allclose(r[:, 1:], 0.0, atol=1e-9)
    sm = plan.prism_smatrix(t, 1, "f32")
    assert sm.n_beams == 1
    r2 = plan.prism_output(sm, xy).cpu().numpy()
    assert np.allclose(r2, r, atol=1e-6)


def test_no_atoms_gives_unit_transmission():
    from paper_1706_08563_b300 import api
    w = W.scaled(W.C1, n=64, n_atoms=0, n_slices=3, slice_dz=4.0)
    plan = api.Plan.from_workload(w)
    t, v = plan.slice_potentials(torch.zeros((0, 3), dtype=torch.float64, device="cuda"),
                                 torch.zeros((0, 4), dtype=torch.float32, device="cuda"), want_v=True)
    assert float(v.abs().max()) == 0.0
    assert float((t - 1).abs().max()) == 0.0


@pytest.mark.parametrize("f", [8, 16])
def test_largest_f_smallest_window(f):
    """W = N / f down to 8 pixels (f = 16 at N = 128)."""
    from paper_1706_08563_b300 import api
    w = W.Workload("f", (24.0, 24.0, 4.0), 30, 128, 2, 2.0, 200.0, 25.0, 4, 2.0, 40)
    xyz, gauss = W.atoms(w, seed=f)
    plan = api.Plan.from_workload(w)
    p = O.params_from(w)
    t = O.transmission(p, O.projected_potential(p, xyz, gauss))
    beams = O.prism_beams(p, f)
    sm = plan.prism_smatrix(torch.from_numpy(t.astype(np.complex64)).cuda(), f, "f32", batch=8)
    xy = W.random_positions(w, 13, seed=1)
    got = plan.prism_output(sm, torch.from_numpy(xy).cuda(), chunk=5).cpu().numpy()
    ref = O.prism_rings(p, O.prism_smatrix(p, t, beams), beams, f, xy)
    assert O.rel_l2(got, ref) <= 1e-4


def test_single_ring_and_max_rings():
    from paper_1706_08563_b300 import api
    w = W.Workload("r", (16.0, 16.0, 4.0), 20, 64, 2, 2.0, 200.0, 20.0, 2, 500.0, 1)
    xyz, gauss = W.atoms(w, seed=2)
    plan = api.Plan.from_workload(w)
    p = O.params_from(w)
    t = O.transmission(p, O.projected_potential(p, xyz, gauss))
    xy = W.random_positions(w, 3, seed=3)
    got = plan.multislice(torch.from_numpy(t.astype(np.complex64)).cuda(), torch.from_numpy(xy).cuda()).cpu().numpy()
    assert got.shape == (3, 1)
    assert np.allclose(got[:, 0], O.multislice_rings(p, t, xy)[:, 0], rtol=1e-5)
    edges = np.linspace(0.0, 600.0, 2049)           # 2048 detectors, the maximum
    plan.set_detector_edges(edges)
    got2 = plan.multislice(torch.from_numpy(t.astype(np.complex64)).cuda(), torch.from_numpy(xy).cuda()).cpu().numpy()
    assert got2.shape == (3, 2048)
    assert np.allclose(got2.sum(axis=1), got[:, 0], rtol=1e-5)
    with pytest.raises(Exception):
        plan.set_detector_edges(np.linspace(0.0, 600.0, 2050))
