"""CUDA path (through the C ABI) vs the FP64 oracle, element by element.

The ring tolerances and their rationale are in tests/tolerances.py.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import stem as O

pytestmark = pytest.mark.gpu

from tolerances import FP32_FLOOR, FP32_TOL, LOWP_FLOOR, LOWP_TOL, check_rings, rel_l2  # noqa: F401


@pytest.fixture(scope="module")
def api():
    from paper_1706_08563_b300 import api as A
    return A


def dev(x, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


# ------------------------------------------------------------------------ FFT
@pytest.mark.parametrize("n,batch", [(8, 3), (16, 5), (32, 3), (64, 7), (128, 3), (256, 2), (512, 2),
                                     (1024, 2), (2048, 1)])
@pytest.mark.parametrize("inverse", [False, True])
def test_fft2_vs_numpy(api, n, batch, inverse):
    x = W.random_complex((batch, n, n), seed=n + batch)
    got = api.fft2(dev(x, torch.complex64), inverse=inverse).cpu().numpy()
    ref = np.fft.ifft2(x) * n * n if inverse else np.fft.fft2(x)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-6, err


# ---------------------------------------------------------------- potentials
def test_potentials_vs_oracle(api):
    w = W.scaled(W.C1, n_atoms=60)
    xyz, gauss = W.atoms(w, seed=11)
    xyz[0] = [0.01, 15.99, 0.5]            # periodic images along both axes
    xyz[1] = [8.0, 8.0, 19.999]            # last slice
    plan = api.Plan.from_workload(w)
    trans, v = plan.slice_potentials(dev(xyz), dev(gauss), want_v=True)
    p = O.params_from(w)
    vref = O.projected_potential(p, xyz, gauss)
    v = v.cpu().numpy()
    assert np.max(np.abs(v - vref)) <= 2e-6 * np.max(vref)
    tref = O.transmission(p, vref)
    assert np.max(np.abs(trans.cpu().numpy() - tref)) <= 2e-6


@pytest.mark.parametrize("n,cell,n_atoms", [
    (64, (6.0, 7.0, 4.0), 12),      # cutoff above half the cell: several periodic images per axis
    (512, (10.0, 12.0, 4.0), 80),   # 256 neighbour cells in reach (two cell groups), lists above 32 atoms
])
def test_potentials_large_cutoff_vs_oracle(api, n, cell, n_atoms):
    w = W.Workload("pl", cell, n_atoms, n, 2, 2.0, 200.0, 20.0, 4, 2.0, 40)
    xyz, gauss = W.atoms(w, seed=n)
    plan = api.Plan.from_workload(w)
    _, v = plan.slice_potentials(dev(xyz), dev(gauss), want_v=True)
    vref = O.projected_potential(O.params_from(w), xyz, gauss)
    assert np.max(np.abs(v.cpu().numpy() - vref)) <= 2e-6 * np.max(vref)


def test_potentials_repeatable(api):
    """The FP32 sums run in an order fixed by the input: two calls agree bit for bit."""
    w = W.scaled(W.C2, n_atoms=2000)
    xyz, gauss = W.atoms(w, seed=12)
    plan = api.Plan.from_workload(w)
    _, v1 = plan.slice_potentials(dev(xyz), dev(gauss), want_v=True)
    _, v2 = plan.slice_potentials(dev(xyz), dev(gauss), want_v=True)
    assert torch.equal(v1, v2)
    vref = O.projected_potential(O.params_from(w), xyz, gauss)
    assert np.max(np.abs(v1.cpu().numpy() - vref)) <= 2e-6 * np.max(vref)


# ------------------------------------------------------------------ detector
def test_detector_readout_vs_oracle(api):
    w = W.scaled(W.C1, n=64)
    plan = api.Plan.from_workload(w)
    p = O.params_from(w)
    for f in (1, 2, 4):
        x = W.random_complex((5, 64 // f, 64 // f), seed=f)
        got = plan.detector_readout(dev(x, torch.complex64), f=f, scale=0.5).cpu().numpy()
        table = O.ring_table(p) if f == 1 else O.coarse_ring_table(p, f)
        ref = 0.5 * O.detector_rings(table, p.n_rings, np.abs(x) ** 2)
        assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(ref)


# ---------------------------------------------------------------- multislice
def _oracle_trans(w, xyz, gauss):
    p = O.params_from(w)
    return p, O.transmission(p, O.projected_potential(p, xyz, gauss))


def test_multislice_c1_end_to_end(api):
    """Config 1 in full: 200 atoms, 128^2, 10 slices, 80 keV, 16x16 probes."""
    w = W.C1
    xyz, gauss = W.atoms(w)
    xy = W.scan_positions(w)
    plan = api.Plan.from_workload(w)
    trans = plan.slice_potentials(dev(xyz), dev(gauss))
    got = plan.multislice(trans, dev(xy), batch=w.batch).cpu().numpy()
    p, tref = _oracle_trans(w, xyz, gauss)
    ref = O.multislice_rings(p, tref, xy, chunk=64)
    check_rings(got, ref, FP32_TOL)
    # stage-wise: the same oracle transmission on both sides isolates propagation
    got2 = plan.multislice(dev(tref, torch.complex64), dev(xy), batch=w.batch).cpu().numpy()
    check_rings(got2, ref, FP32_TOL)


def test_multislice_ragged_batches_and_weight(api):
    """37 probes in launches of 16 (a ragged tail), N = 64, accumulation with weight."""
    w = W.scaled(W.C1, n=64, n_atoms=40, n_slices=4, slice_dz=5.0)
    xyz, gauss = W.atoms(w, seed=3)
    xy = W.random_positions(w, 37, seed=4)
    plan = api.Plan.from_workload(w)
    p, tref = _oracle_trans(w, xyz, gauss)
    t = dev(tref, torch.complex64)
    rings = torch.zeros((37, w.n_rings), dtype=torch.float32, device="cuda")
    plan.multislice(t, dev(xy), batch=16, rings=rings, weight=0.5)
    plan.multislice(t, dev(xy), batch=16, rings=rings, weight=0.5)     # accumulates (+=)
    ref = O.multislice_rings(p, tref, xy)
    check_rings(rings.cpu().numpy(), ref, FP32_TOL)
    one = plan.multislice(t, dev(xy), batch=37).cpu().numpy()
    many = plan.multislice(t, dev(xy), batch=1).cpu().numpy()
    check_rings(one, ref, FP32_TOL)
    check_rings(many, ref, FP32_TOL)


@pytest.mark.parametrize("n", [64, 256, 512, 1024, 2048])
def test_multislice_sizes(api, n):
    w = W.Workload("t", (20.0, 24.0, 8.0), 30, n, 4, 2.0, 200.0, 25.0, 3, 2.0, 60)
    xyz, gauss = W.atoms(w, seed=n)
    xy = W.random_positions(w, 5, seed=n + 1)
    plan = api.Plan.from_workload(w)
    p, tref = _oracle_trans(w, xyz, gauss)
    got = plan.multislice(dev(tref, torch.complex64), dev(xy), batch=4).cpu().numpy()
    check_rings(got, O.multislice_rings(p, tref, xy), FP32_TOL)


def test_multislice_free_space_closed_form(api):
    """V = 0: rings equal |A cap ring| / |A| at every probe position."""
    w = W.scaled(W.C1, n=128)
    plan = api.Plan.from_workload(w)
    p = O.params_from(w)
    t = torch.ones((w.n_slices, 128, 128), dtype=torch.complex64, device="cuda")
    xy = W.random_positions(w, 9, seed=2)
    got = plan.multislice(t, dev(xy), batch=9).cpu().numpy()
    ap = O.aperture(p)
    tab = O.ring_table(p)
    want = np.array([np.sum(ap & (tab == i)) for i in range(p.n_rings)]) / ap.sum()
    assert np.max(np.abs(got - want[None])) <= 1e-5


def test_multislice_empty_and_errors(api):
    from paper_1706_08563_b300 import _lib
    w = W.scaled(W.C1, n=64, n_slices=2)
    plan = api.Plan.from_workload(w)
    t = torch.ones((2, 64, 64), dtype=torch.complex64, device="cuda")
    r = plan.multislice(t, torch.zeros((0, 2), dtype=torch.float64, device="cuda"))
    assert r.shape == (0, w.n_rings)
    lib = _lib.load()
    ws = plan.multislice_workspace(4)
    xy = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    rings = torch.zeros((4, w.n_rings), device="cuda")
    assert lib.stem_multislice_scan(plan._h, t.data_ptr(), xy.data_ptr(), 4, 4, 1.0, rings.data_ptr(),
                                    ws.data_ptr(), 1024, None) == _lib.STEM_ERR_NOMEM
    assert lib.stem_multislice_scan(plan._h, t.data_ptr(), xy.data_ptr(), 4, 0, 1.0, rings.data_ptr(),
                                    ws.data_ptr(), ws.numel(), None) == _lib.STEM_ERR_INVALID
    torch.cuda.synchronize()


# --------------------------------------------------------------------- PRISM
def _small_prism_case(n=128, f=4, slices=4, atoms=60, seed=21):
    w = W.Workload("p", (24.0, 28.0, 8.0), atoms, n, slices, 2.0, 200.0, 20.0, 8, 2.0, 60, f=(f,))
    xyz, gauss = W.atoms(w, seed=seed)
    return w, xyz, gauss


def test_prism_beams_match_oracle(api):
    w, _, _ = _small_prism_case()
    plan = api.Plan.from_workload(w)
    p = O.params_from(w)
    for f in (1, 2, 4, 8):
        assert np.array_equal(plan.prism_beams(f), O.prism_beams(p, f).astype(np.int32))


@pytest.mark.parametrize("f", [1, 4])
def test_prism_smatrix_beams_vs_oracle(api, f):
    w, xyz, gauss = _small_prism_case(f=f)
    plan = api.Plan.from_workload(w)
    p, tref = _oracle_trans(w, xyz, gauss)
    beams = O.prism_beams(p, f)
    sm = plan.prism_smatrix(dev(tref, torch.complex64), f, "f32", batch=7)
    got = sm.beams_real_space().cpu().numpy()
    pick = np.unique(np.linspace(0, len(beams) - 1, 9).astype(int))
    ref = O.prism_smatrix(p, tref, beams[pick])
    for k, b in enumerate(pick):
        e = np.linalg.norm(got[b] - ref[k]) / np.linalg.norm(ref[k])
        assert e <= 2e-5, (b, e)


def test_prism_f1_equals_multislice_on_gpu(api):
    w, xyz, gauss = _small_prism_case(n=64, f=1, slices=3)
    plan = api.Plan.from_workload(w)
    p, tref = _oracle_trans(w, xyz, gauss)
    t = dev(tref, torch.complex64)
    xy = W.random_positions(w, 11, seed=5)
    sm = plan.prism_smatrix(t, 1, "f32", batch=64)
    pr = plan.prism_output(sm, dev(xy), chunk=5).cpu().numpy()
    ms = plan.multislice(t, dev(xy), batch=11).cpu().numpy()
    ref = O.multislice_rings(p, tref, xy)
    check_rings(pr, ref, FP32_TOL)
    check_rings(ms, ref, FP32_TOL)


@pytest.mark.parametrize("f", [2, 4, 8])
def test_prism_output_vs_oracle(api, f):
    w, xyz, gauss = _small_prism_case(f=f)
    plan = api.Plan.from_workload(w)
    p, tref = _oracle_trans(w, xyz, gauss)
    beams = O.prism_beams(p, f)
    sm = plan.prism_smatrix(dev(tref, torch.complex64), f, "f32", batch=32)
    xy = np.concatenate([W.scan_positions(w, scan=6), W.random_positions(w, 7, seed=9)])
    got = plan.prism_output(sm, dev(xy), chunk=16).cpu().numpy()
    sref = O.prism_smatrix(p, tref, beams)
    ref = O.prism_rings(p, sref, beams, f, xy)
    check_rings(got, ref, FP32_TOL)
    # stage-wise: the window beam sum on the GPU's own S-matrix
    s_gpu = sm.beams_real_space().cpu().numpy().astype(np.complex128)
    win = plan.prism_windows(sm, dev(xy[:5])).cpu().numpy()
    wref = O.prism_window_waves(p, s_gpu, beams, f, xy[:5])
    assert np.linalg.norm(win - wref) / np.linalg.norm(wref) <= 1e-5


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_prism_reduced_precision_storage(api, storage):
    w, xyz, gauss = _small_prism_case(f=4)
    plan = api.Plan.from_workload(w)
    p, tref = _oracle_trans(w, xyz, gauss)
    beams = O.prism_beams(p, 4)
    t = dev(tref, torch.complex64)
    sm = plan.prism_smatrix(t, 4, storage, batch=16)
    sc = sm.scales().cpu().numpy()
    assert np.all(sc[: sm.n_beams] > 0) and np.all(np.log2(sc) == np.round(np.log2(sc)))
    assert np.all(np.abs(sm.data().float().cpu().numpy()) <= 1.0)
    xy = W.scan_positions(w, scan=5)
    got = plan.prism_output(sm, dev(xy), chunk=25, engine="simt").cpu().numpy()
    ref = O.prism_rings(p, O.prism_smatrix(p, tref, beams), beams, 4, xy)
    check_rings(got, ref, LOWP_TOL)


def test_prism_free_space_closed_form(api):
    w, _, _ = _small_prism_case(n=128, f=4)
    plan = api.Plan.from_workload(w)
    p = O.params_from(w)
    t = torch.ones((w.n_slices, 128, 128), dtype=torch.complex64, device="cuda")
    sm = plan.prism_smatrix(t, 4, "f32")
    xy = W.random_positions(w, 6, seed=1)
    got = plan.prism_output(sm, dev(xy)).cpu().numpy()
    beams = O.prism_beams(p, 4)
    tab = O.ring_table(p)
    counts = np.zeros(p.n_rings)
    for m, n in beams:
        r = tab[n % 128, m % 128]
        if r >= 0:
            counts[r] += 1
    assert np.max(np.abs(got - counts[None] / len(beams))) <= 1e-5


# ------------------------------------------------------- tensor-core beam sum
def _device_status(plan):
    import ctypes
    from paper_1706_08563_b300 import _lib
    code = ctypes.c_int32(-99)
    assert _lib.load().stem_plan_device_status(plan._h, ctypes.byref(code)) == _lib.STEM_OK
    return code.value


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("n,f", [(128, 4), (256, 2)])
def test_prism_tensor_engine_vs_simt_and_oracle(api, storage, n, f):
    """tcgen05 complex GEMM beam sum: same windows as the CUDA-core engine on the
    same 16-bit S-matrix (both accumulate in FP32), and rings within the
    reduced-precision bound of the FP64 oracle."""
    w, xyz, gauss = _small_prism_case(n=n, f=f)
    plan = api.Plan.from_workload(w)
    p, tref = _oracle_trans(w, xyz, gauss)
    beams = O.prism_beams(p, f)
    sm = plan.prism_smatrix(dev(tref, torch.complex64), f, storage, batch=32)
    xy = np.concatenate([W.scan_positions(w, scan=7), W.random_positions(w, 150, seed=3)])
    d_xy = dev(xy)
    wt = plan.prism_windows(sm, d_xy, engine="tensor").cpu().numpy()
    ws = plan.prism_windows(sm, d_xy, engine="simt").cpu().numpy()
    assert _device_status(plan) == 0
    # both engines multiply 16-bit operands exactly and sum in FP32; the tensor
    # engine also rounds the coefficients to 16 bits
    eps = 2.0 ** -11 if storage == "f16" else 2.0 ** -8
    assert np.linalg.norm(wt - ws) / np.linalg.norm(ws) <= 4 * eps
    got = plan.prism_output(sm, d_xy, chunk=100, engine="tensor").cpu().numpy()
    ref = O.prism_rings(p, O.prism_smatrix(p, tref, beams), beams, f, xy)
    check_rings(got, ref, LOWP_TOL)
    assert _device_status(plan) == 0


@pytest.mark.parametrize("n,f,storage", [(1024, 8, "f32"), (1024, 4, "f16"), (2048, 16, "f32")])
def test_prism_smatrix_tiled_sizes(api, n, f, storage):
    """S-matrix at the sizes whose slice loop uses the 4-row tiled wave layout."""
    w = W.Workload("p", (24.0, 24.0, 4.0), 40, n, 2, 2.0, 200.0, 20.0, 4, 2.0, 40, f=(f,))
    xyz, gauss = W.atoms(w, seed=n + f)
    plan = api.Plan.from_workload(w)
    p, tref = _oracle_trans(w, xyz, gauss)
    beams = O.prism_beams(p, f)
    sm = plan.prism_smatrix(dev(tref, torch.complex64), f, storage, batch=5)
    got = sm.beams_real_space().cpu().numpy()
    pick = np.unique(np.linspace(0, len(beams) - 1, 4).astype(int))
    ref = O.prism_smatrix(p, tref, beams[pick])
    tol = 2e-5 if storage == "f32" else 2e-3
    for k, b in enumerate(pick):
        e = np.linalg.norm(got[b] - ref[k]) / np.linalg.norm(ref[k])
        assert e <= tol, (b, e)
    xy = W.random_positions(w, 6, seed=1)
    out = plan.prism_output(sm, dev(xy)).cpu().numpy()
    check_rings(out, O.prism_rings(p, O.prism_smatrix(p, tref, beams), beams, f, xy),
                FP32_TOL if storage == "f32" else LOWP_TOL)


# -------------------------------------------------------------- aberrations
@pytest.mark.parametrize("defocus,cs", [(80.0, 0.0), (-40.0, 5e5)])
def test_multislice_and_prism_with_aberrations(api, defocus, cs):
    w = W.Workload("ab", (20.0, 20.0, 6.0), 30, 128, 3, 2.0, 200.0, 25.0, 4, 2.0, 40, f=(2,),
                   defocus=defocus, cs=cs)
    xyz, gauss = W.atoms(w, seed=17)
    plan = api.Plan.from_workload(w)
    p, tref = _oracle_trans(w, xyz, gauss)
    assert p.defocus == defocus and p.cs == cs
    t = dev(tref, torch.complex64)
    xy = W.random_positions(w, 9, seed=2)
    ms = plan.multislice(t, dev(xy), batch=9).cpu().numpy()
    check_rings(ms, O.multislice_rings(p, tref, xy), FP32_TOL)
    beams = O.prism_beams(p, 2)
    sref = O.prism_smatrix(p, tref, beams)
    for storage, engine, tol in (("f32", "simt", FP32_TOL), ("f16", "tensor", LOWP_TOL)):
        sm = plan.prism_smatrix(t, 2, storage, batch=32)
        pr = plan.prism_output(sm, dev(xy), engine=engine).cpu().numpy()
        check_rings(pr, O.prism_rings(p, sref, beams, 2, xy), tol)


# --------------------------------------------- detectors with edges, 4D output
def test_detector_edges_multislice_and_prism(api):
    """A BF disc, an annular BF, two ADF rings and a HAADF-like ring."""
    w, xyz, gauss = _small_prism_case(n=128, f=2)
    plan = api.Plan.from_workload(w)
    edges = [0.0, 10.0, 20.0, 41.0, 80.0, 251.0]
    plan.set_detector_edges(edges)
    p, tref = _oracle_trans(w, xyz, gauss)
    t = dev(tref, torch.complex64)
    xy = W.random_positions(w, 11, seed=6)
    ms = plan.multislice(t, dev(xy), batch=11).cpu().numpy()
    assert ms.shape == (11, len(edges) - 1)
    check_rings(ms, O.multislice_rings(p, tref, xy, edges=edges), FP32_TOL)
    beams = O.prism_beams(p, 2)
    sm = plan.prism_smatrix(t, 2, "f32", batch=64)
    pr = plan.prism_output(sm, dev(xy), engine="simt").cpu().numpy()
    sref = O.prism_smatrix(p, tref, beams)
    win = O.prism_window_waves(p, sref, beams, 2, xy)
    spec = np.abs(np.fft.fft2(win)) ** 2 / (64.0 ** 4)
    ref = O.detector_rings(O.coarse_ring_table(p, 2, edges), len(edges) - 1, spec)
    check_rings(pr, ref, FP32_TOL)


def _check_dp(got, ref, tol):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert np.all(np.isfinite(got))
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    assert np.max(np.abs(got - ref)) <= tol * np.max(ref)


def test_multislice_4d_vs_oracle(api):
    w = W.Workload("d", (20.0, 24.0, 6.0), 30, 128, 3, 2.0, 200.0, 25.0, 4, 2.0, 40)
    xyz, gauss = W.atoms(w, seed=23)
    plan = api.Plan.from_workload(w)
    p, tref = _oracle_trans(w, xyz, gauss)
    xy = W.random_positions(w, 5, seed=3)
    dp = plan.multislice_4d(dev(tref, torch.complex64), dev(xy), batch=3).cpu().numpy()
    _check_dp(dp, O.multislice_dp(p, tref, xy), FP32_TOL)


@pytest.mark.parametrize("storage,engine,tol", [("f32", "simt", FP32_TOL), ("bf16", "tensor", LOWP_TOL)])
def test_prism_4d_vs_oracle(api, storage, engine, tol):
    w, xyz, gauss = _small_prism_case(n=128, f=4)
    plan = api.Plan.from_workload(w)
    p, tref = _oracle_trans(w, xyz, gauss)
    beams = O.prism_beams(p, 4)
    sm = plan.prism_smatrix(dev(tref, torch.complex64), 4, storage, batch=32)
    xy = W.random_positions(w, 7, seed=5)
    dp = plan.prism_output_4d(sm, dev(xy), chunk=4, engine=engine).cpu().numpy()
    _check_dp(dp, O.prism_dp(p, O.prism_smatrix(p, tref, beams), beams, 4, xy), tol)


def test_frozen_phonon_average_vs_oracle(api):
    """Frozen phonons: three configurations with i.i.d. displacements, each
    through the GPU's potentials and slice loop, accumulated with weight 1/C
    (multislice, and PRISM f = 2 with an S-matrix per configuration), against
    the oracle's frozen-phonon mean."""
    w = W.Workload("fpg", (16.0, 16.0, 6.0), 30, 64, 3, 2.0, 200.0, 20.0, 0, 2.0, 30, fp_configs=3, fp_sigma=0.08)
    xyz, gauss = W.atoms(w, seed=31)
    xy = W.random_positions(w, 11, seed=32)
    configs = [W.displaced(w, xyz, c) for c in range(w.fp_configs)]
    plan = api.Plan.from_workload(w)
    ms = torch.zeros((len(xy), w.n_rings), dtype=torch.float32, device="cuda")
    pr = torch.zeros_like(ms)
    for xc in configs:
        t = plan.slice_potentials(dev(xc), dev(gauss))
        plan.multislice(t, dev(xy), batch=8, rings=ms, weight=1.0 / len(configs))
        sm = plan.prism_smatrix(t, 2, "f32")
        plan.prism_output(sm, dev(xy), chunk=8, rings=pr, weight=1.0 / len(configs))
    p = O.params_from(w)
    check_rings(ms.cpu().numpy(), O.frozen_phonon_rings(p, configs, gauss, xy), FP32_TOL)
    check_rings(pr.cpu().numpy(), O.frozen_phonon_rings(p, configs, gauss, xy, algo="prism", f=2), FP32_TOL)


def test_probe_phase_far_from_the_origin(api):
    """Probe positions moved by whole multiples of the cell (up to 10^6 A away)
    give the rings of the original positions: the phase ramps (probe
    initialisation, PRISM coefficients) and the PRISM window origins are
    reduced in FP64 before anything is evaluated in FP32."""
    w = W.scaled(W.C1, n=64)
    xyz, gauss = W.atoms(w, seed=51)
    plan = api.Plan.from_workload(w)
    trans = plan.slice_potentials(dev(xyz), dev(gauss))
    xy = W.random_positions(w, 9, seed=52)
    lx, ly = w.cell[0], w.cell[1]
    far = xy + np.array([[62500.0 * lx, -31000.0 * ly]])
    near_ms = plan.multislice(trans, dev(xy), batch=4).cpu().numpy()
    far_ms = plan.multislice(trans, dev(far), batch=4).cpu().numpy()
    assert np.allclose(far_ms, near_ms, rtol=1e-5, atol=1e-9 * near_ms.max())
    sm = plan.prism_smatrix(trans, 2, "f32")
    near_pr = plan.prism_output(sm, dev(xy), chunk=4).cpu().numpy()
    far_pr = plan.prism_output(sm, dev(far), chunk=4).cpu().numpy()
    assert np.allclose(far_pr, near_pr, rtol=1e-5, atol=1e-9 * near_pr.max())


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_prism_smatrix_beam_ranges_sum_to_the_whole(api, storage):
    """Beams built in disjoint ranges into zeroed buffers (as ranks of the PRISM
    split do) sum, value by value in the stored type, to exactly the S-matrix
    built in one call; the last range also writes the padding beams."""
    w, xyz, gauss = _small_prism_case(n=128, f=2)
    plan = api.Plan.from_workload(w)
    p, tref = _oracle_trans(w, xyz, gauss)
    t = dev(tref, torch.complex64)
    whole = plan.prism_smatrix(t, 2, storage, batch=16)
    nb = whole.n_beams
    cuts = [0, 5, 5, nb // 2, nb]                  # includes an empty range
    parts = [plan.prism_smatrix(t, 2, storage, batch=16, beams=(a, b)) for a, b in zip(cuts[:-1], cuts[1:])]
    scales = sum(s.scales() for s in parts)
    data = sum(s.data().float() for s in parts).to(whole.data().dtype)
    assert torch.equal(scales, whole.scales())
    assert torch.equal(data, whole.data())
    # a range outside [0, n_beams] is refused
    from paper_1706_08563_b300 import _lib
    with pytest.raises(_lib.StemError):
        plan.prism_smatrix(t, 2, storage, beams=(3, nb + 1))
