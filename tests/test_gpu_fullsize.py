"""Parity at the benchmark sizes, in the launch configuration bench.py times,
on outputs the FP64 oracle can compute one by one.

* Batched multislice at 1024^2, 50 slices of 2 A, 200 keV, 50 000 atoms, in a
  launch of 256 probes: 64 sampled probes against the oracle end to end.
* PRISM f=8 at 2048^2, 100 slices of 1 A, 300 keV, 793 beams, FP16 S-matrix
  with the tcgen05 beam sum and chunks of 4096 probes: the potentials on
  sampled slices, two sampled S-matrix beams against the oracle (through all
  100 slices), and the output of 33 sampled probes computed by the oracle from
  the GPU's own S-matrix, read window by window (stage-wise: it isolates the
  output step).
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import stem as O
from tolerances import FP32_TOL, check_rings, fp32_floor

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_multislice_1024_launch_of_256_sampled(repo_tmp):
    """64 probes sampled from a launch of 256 (every fourth, so every part of
    the launch and of the scan row is covered), each against the FP64 oracle
    end to end (the oracle runs in a process pool)."""
    from oracle_pool import multislice_rings_pool
    from paper_1706_08563_b300 import api
    w = W.C3
    xyz, gauss = W.atoms(w)
    plan = api.Plan.from_workload(w)
    trans = plan.slice_potentials(torch.from_numpy(xyz).cuda(), torch.from_numpy(gauss).cuda())
    xy = W.scan_positions(w)[: w.batch]
    rings = plan.multislice(trans, torch.from_numpy(xy).cuda(), batch=w.batch).cpu().numpy()
    p = O.params_from(w)
    t = O.transmission(p, O.projected_potential(p, xyz, gauss))
    pick = np.arange(0, w.batch, 4)
    assert len(pick) == 64
    ref = multislice_rings_pool(p, t, xy[pick], repo_tmp)
    check_rings(rings[pick], ref, FP32_TOL, floor=fp32_floor(w.n, w.n_slices))


@pytest.fixture(scope="module")
def prism8():
    from paper_1706_08563_b300 import api
    w = W.C4
    xyz, gauss = W.atoms(w)
    plan = api.Plan.from_workload(w)
    trans, v = plan.slice_potentials(torch.from_numpy(xyz).cuda(), torch.from_numpy(gauss).cuda(), want_v=True)
    sm = plan.prism_smatrix(trans, 8, "f16", batch=w.batch)
    return w, xyz, gauss, plan, trans, v, sm


def test_prism8_potentials_sampled_slices(prism8):
    w, xyz, gauss, plan, trans, v, sm = prism8
    p = O.params_from(w)
    for s in (0, 57):
        sub = O.Params(p.cell, p.n, 1, p.slice_dz, p.energy_kev, p.alpha_mrad, p.ring_width_mrad, p.n_rings)
        keep = O.slice_index(p, xyz[:, 2]) == s
        ref = O.projected_potential(sub, np.c_[xyz[keep, :2], np.zeros(keep.sum())], gauss[keep])[0]
        got = v[s].cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(ref)


def test_prism8_smatrix_sampled_beams(prism8):
    """Two beams through all 100 slices at 2048^2 against the FP64 oracle; the
    stored FP16 values carry the 16-bit rounding on top."""
    w, xyz, gauss, plan, trans, v, sm = prism8
    p = O.params_from(w)
    beams = O.prism_beams(p, 8)
    assert sm.n_beams == len(beams) == 793
    t = trans.cpu().numpy().astype(np.complex128)      # the GPU's own t_n (checked above)
    sc = sm.scales().cpu().numpy()
    for b in (0, 396):
        ref = O.prism_smatrix(p, t, beams[b:b + 1])[0]
        d = sm.data()[:, :, :, b].float().cpu().numpy()
        got = (d[:, :, 0] + 1j * d[:, :, 1]) * sc[b]
        assert _rel(got, ref) <= 2e-3, b


def test_prism8_output_sampled_probes(prism8):
    """Rings of sampled probes (bench chunk of 4096, tcgen05 engine) against the
    oracle's output step (window crop, beam sum, window FFT, rings) applied to
    the GPU's own S-matrix, read window by window."""
    w, xyz, gauss, plan, trans, v, sm = prism8
    p = O.params_from(w)
    beams = O.prism_beams(p, 8)
    xy_all = W.scan_positions(w)[:4096]
    rings = plan.prism_output(sm, torch.from_numpy(xy_all).cuda(), chunk=4096).cpu().numpy()
    pick = np.array(list(range(0, 4096, 128)) + [4095])      # 33 probes over the chunk's 16 scan rows
    ref = O.prism_rings(p, sm, beams, 8, xy_all[pick])
    for k, i in enumerate(pick):
        assert _rel(rings[i], ref[k]) <= 1e-2, i
    check_rings(rings[pick], ref, 1e-2)


def test_prism8_cropped_sampled(prism8):
    """The Fourier-cropped S-matrix at the bench size (2048^2 -> 1536^2, FP16,
    tensor-core beam sum, windows of 192): one sampled beam through all 100
    slices against the oracle's cropped exit wave, and the rings of sampled
    probes of a 4096-probe chunk against the oracle's output step on the GPU's
    own cropped S-matrix, read window by window."""
    w, xyz, gauss, plan, trans, v, sm = prism8
    p = O.params_from(w)
    beams = O.prism_beams(p, 8)
    smc = plan.prism_smatrix(trans, 8, "f16", batch=w.batch, cropped=True)
    assert smc.n == 1536 and smc.n_beams == 793
    assert smc.buf.numel() < 0.57 * sm.buf.numel()
    t = trans.cpu().numpy().astype(np.complex128)
    ref = O.prism_smatrix_cropped(p, t, beams[396:397])[0]
    d = smc.data()[:, :, :, 396].double().cpu().numpy()
    got = (d[:, :, 0] + 1j * d[:, :, 1]) * float(smc.scales()[396])
    assert _rel(got, ref) <= 2e-3
    xy_all = W.scan_positions(w)[:4096]
    rings = plan.prism_output(smc, torch.from_numpy(xy_all).cuda(), chunk=4096).cpu().numpy()
    pick = np.array(list(range(0, 4096, 256)) + [4095])
    refr = O.prism_rings(p, smc, beams, 8, xy_all[pick], grid=1536)
    check_rings(rings[pick], refr, 1e-2)
    assert plan.device_status() == 0
