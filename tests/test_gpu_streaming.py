"""The streaming memory model ("Streaming Data for Very Large Simulations"):
the transmission stack stays in host memory and three slice buffers cycle on
the device.  It must give the single-transfer results."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from oracle import stem as O
from tolerances import FP32_TOL, check_rings

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    from paper_1706_08563_b300 import api
    w = W.C1                                           # 128^2, 10 slices
    xyz, gauss = W.atoms(w)
    plan = api.Plan.from_workload(w)
    trans = plan.slice_potentials(torch.from_numpy(xyz).cuda(), torch.from_numpy(gauss).cuda())
    return w, xyz, gauss, plan, trans


def test_multislice_streamed_equals_resident(case):
    """100 probes in launches of 37: 3 batches x 10 slices = 30 trips through 3 buffers."""
    w, xyz, gauss, plan, trans = case
    xy = torch.from_numpy(W.random_positions(w, 100, seed=5)).cuda()
    ref = plan.multislice(trans, xy, batch=37)
    for host in (trans.cpu().pin_memory(), trans.cpu()):          # pinned, then pageable
        got = plan.multislice_streamed(host, xy, batch=37)
        torch.cuda.synchronize()
        assert torch.allclose(got, ref, rtol=1e-6, atol=1e-12)
    p = O.params_from(w)
    t = O.transmission(p, O.projected_potential(p, xyz, gauss))
    check_rings(got.cpu().numpy(), O.multislice_rings(p, t, xy.cpu().numpy()), FP32_TOL)


def test_multislice_streamed_accepts_a_device_stack(case):
    from paper_1706_08563_b300 import _lib
    w, xyz, gauss, plan, trans = case
    lib = _lib.load()
    xy = torch.from_numpy(W.random_positions(w, 9, seed=6)).cuda()
    ref = plan.multislice(trans, xy, batch=4)
    rings = torch.zeros_like(ref)
    ws = torch.empty(lib.stem_multislice_streamed_workspace(plan._h, 4), dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert lib.stem_multislice_scan_streamed(plan._h, trans.data_ptr(), xy.data_ptr(), 9, 4, 1.0,
                                             rings.data_ptr(), ws.data_ptr(), ws.numel(), st) == 0
    torch.cuda.synchronize()
    assert torch.allclose(rings, ref, rtol=1e-6, atol=1e-12)
    # the workspace must hold the waves and three slice buffers
    short = lib.stem_multislice_workspace(plan._h, 4)
    assert lib.stem_multislice_scan_streamed(plan._h, trans.data_ptr(), xy.data_ptr(), 9, 4, 1.0,
                                             rings.data_ptr(), ws.data_ptr(), short, st) == _lib.STEM_ERR_NOMEM


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_smatrix_streamed_is_bit_identical(case, storage):
    w, xyz, gauss, plan, trans = case
    ref = plan.prism_smatrix(trans, 2, storage, batch=16)
    got = plan.prism_smatrix_streamed(trans.cpu().pin_memory(), 2, storage, batch=16)
    torch.cuda.synchronize()
    assert ref.n_beams == got.n_beams and ref.n_beams > 16
    assert torch.equal(ref.buf, got.buf)
