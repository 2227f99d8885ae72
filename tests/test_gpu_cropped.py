"""The Fourier-cropped S-matrix (STEM_CROPPED) through the C ABI against the
FP64 oracle: exit waves on the 3N/4 grid, PRISM output on W' = 3W/4 windows
(rings, window waves, 4D), both beam-sum engines, and the degenerate windows
of 6 and 12 pixels that take the direct-DFT path.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import stem as O
from tolerances import FP32_TOL, LOWP_TOL, check_rings

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1706_08563_b300 import api as A
    return A


def dev(x, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _case(n=128, f=2, slices=4, atoms=60, seed=21, cell=(24.0, 28.0, 8.0)):
    w = W.Workload("pc", cell, atoms, n, slices, 2.0, 200.0, 20.0, 8, 2.0, 60, f=(f,))
    xyz, gauss = W.atoms(w, seed=seed)
    p = O.params_from(w)
    return w, p, O.transmission(p, O.projected_potential(p, xyz, gauss))


@pytest.mark.parametrize("n,f", [(128, 1), (128, 4), (256, 2)])
def test_cropped_smatrix_beams_vs_oracle(api, n, f):
    w, p, tref = _case(n=n, f=f)
    plan = api.Plan.from_workload(w)
    beams = O.prism_beams(p, f)
    sm = plan.prism_smatrix(dev(tref, torch.complex64), f, "f32", batch=7, cropped=True)
    assert sm.cropped and sm.n == 3 * n // 4
    got = sm.beams_real_space().cpu().numpy()
    pick = np.unique(np.linspace(0, len(beams) - 1, 7).astype(int))
    ref = O.prism_smatrix_cropped(p, tref, beams[pick])
    for k, b in enumerate(pick):
        e = np.linalg.norm(got[b] - ref[k]) / np.linalg.norm(ref[k])
        assert e <= 2e-5, (b, e)


def test_cropped_smatrix_bytes(api):
    from paper_1706_08563_b300 import _lib
    w, p, _ = _case(n=256, f=4)
    plan = api.Plan.from_workload(w)
    lib = _lib.load()
    for st in (0, 1, 2):
        full = lib.stem_prism_smatrix_bytes(plan._h, 4, st)
        crop = lib.stem_prism_smatrix_bytes(plan._h, 4, st | _lib.STEM_CROPPED)
        nb = len(plan.prism_beams(4))
        nbp = (nb + 63) // 64 * 64
        head = (nbp * 4 + 255) // 256 * 256
        assert (crop - head) * 16 == (full - head) * 9
    assert lib.stem_prism_smatrix_bytes(plan._h, 4, 3) == 0                  # unknown element type


@pytest.mark.parametrize("f", [2, 4, 8])
def test_cropped_prism_output_vs_oracle(api, f):
    w, p, tref = _case(n=128, f=f)
    plan = api.Plan.from_workload(w)
    beams = O.prism_beams(p, f)
    n2 = O.cropped_grid(p.n)
    sm = plan.prism_smatrix(dev(tref, torch.complex64), f, "f32", batch=32, cropped=True)
    xy = np.concatenate([W.scan_positions(w, scan=6), W.random_positions(w, 7, seed=9)])
    got = plan.prism_output(sm, dev(xy), chunk=16).cpu().numpy()
    sref = O.prism_smatrix_cropped(p, tref, beams)
    check_rings(got, O.prism_rings(p, sref, beams, f, xy, grid=n2), FP32_TOL)
    # stage-wise: the window beam sum on the GPU's own cropped S-matrix
    s_gpu = sm.beams_real_space().cpu().numpy().astype(np.complex128)
    win = plan.prism_windows(sm, dev(xy[:5])).cpu().numpy()
    assert win.shape == (5, n2 // f, n2 // f)
    wref = O.prism_window_waves(p, s_gpu, beams, f, xy[:5], n2)
    assert np.linalg.norm(win - wref) / np.linalg.norm(wref) <= 1e-5


def test_cropped_f1_equals_multislice_on_gpu(api):
    w, p, tref = _case(n=64, f=1, slices=3)
    plan = api.Plan.from_workload(w)
    t = dev(tref, torch.complex64)
    xy = W.random_positions(w, 11, seed=5)
    sm = plan.prism_smatrix(t, 1, "f32", batch=64, cropped=True)
    pr = plan.prism_output(sm, dev(xy), chunk=5).cpu().numpy()
    check_rings(pr, O.multislice_rings(p, tref, xy), FP32_TOL)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("n,f", [(128, 2), (256, 4)])
def test_cropped_tensor_engine_vs_simt_and_oracle(api, storage, n, f):
    w, p, tref = _case(n=n, f=f)
    plan = api.Plan.from_workload(w)
    beams = O.prism_beams(p, f)
    sm = plan.prism_smatrix(dev(tref, torch.complex64), f, storage, batch=32, cropped=True)
    xy = np.concatenate([W.scan_positions(w, scan=7), W.random_positions(w, 150, seed=3)])
    d_xy = dev(xy)
    wt = plan.prism_windows(sm, d_xy, engine="tensor").cpu().numpy()
    ws = plan.prism_windows(sm, d_xy, engine="simt").cpu().numpy()
    eps = 2.0 ** -11 if storage == "f16" else 2.0 ** -8
    assert np.linalg.norm(wt - ws) / np.linalg.norm(ws) <= 4 * eps
    got = plan.prism_output(sm, d_xy, chunk=100, engine="tensor").cpu().numpy()
    ref = O.prism_rings(p, O.prism_smatrix_cropped(p, tref, beams), beams, f, xy, grid=O.cropped_grid(n))
    check_rings(got, ref, LOWP_TOL)
    assert plan.device_status() == 0


def test_cropped_4d_vs_oracle(api):
    w, p, tref = _case(n=128, f=4)
    plan = api.Plan.from_workload(w)
    beams = O.prism_beams(p, 4)
    n2 = O.cropped_grid(p.n)
    sm = plan.prism_smatrix(dev(tref, torch.complex64), 4, "f32", batch=32, cropped=True)
    xy = W.random_positions(w, 7, seed=5)
    dp = plan.prism_output_4d(sm, dev(xy), chunk=4).cpu().numpy()
    ref = O.prism_dp(p, O.prism_smatrix_cropped(p, tref, beams), beams, 4, xy, grid=n2)
    assert dp.shape == ref.shape == (7, n2 // 4, n2 // 4)
    assert np.linalg.norm(dp - ref) <= FP32_TOL * np.linalg.norm(ref)
    assert np.max(np.abs(dp - ref)) <= FP32_TOL * np.max(ref)


@pytest.mark.parametrize("f", [8, 4])
def test_cropped_small_windows_free_space(api, f):
    """N = 64 with f = 8 and 4: windows of W' = 6 and 12 pixels (direct DFTs);
    in free space every beam lands on one window pixel."""
    w = W.Workload("pf", (16.0, 16.0, 6.0), 0, 64, 3, 2.0, 80.0, 30.0, 4, 3.0, 40, f=(f,))
    plan = api.Plan.from_workload(w)
    p = O.params_from(w)
    t = torch.ones((3, 64, 64), dtype=torch.complex64, device="cuda")
    sm = plan.prism_smatrix(t, f, "f32", cropped=True)
    xy = W.random_positions(w, 6, seed=1)
    got = plan.prism_output(sm, dev(xy)).cpu().numpy()
    beams = O.prism_beams(p, f)
    ref = O.prism_rings(p, O.prism_smatrix_cropped(p, np.ones((3, 64, 64), complex), beams), beams, f, xy,
                        grid=O.cropped_grid(64))
    assert np.max(np.abs(got - ref)) <= 1e-5
    counts = np.zeros(p.n_rings)
    tab = O.ring_table(p)
    for m, n in beams:
        r = tab[n % 64, m % 64]
        if r >= 0:
            counts[r] += 1
    assert np.max(np.abs(got - counts[None] / len(beams))) <= 1e-5
