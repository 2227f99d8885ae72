"""The allocation-free multislice entry point, called through the C ABI.

stem_multislice_scan_noalloc serves callers that cannot allocate device memory
and cannot lend a workspace: it keeps the batch of waves in a fixed scratch
array inside the library.  It must give the same rings as stem_multislice_scan
with a caller workspace, on consecutive calls (the array keeps the previous
call's contents, here first filled by a call of another layout), and must
refuse a batch that does not fit or a plan made on another device.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from oracle import stem as O

pytestmark = pytest.mark.gpu

TOL = 1e-4
FLOOR = 1e-5


def _close(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert np.all(np.isfinite(got))
    assert O.rel_l2(got, ref) <= TOL
    norms = np.sqrt(np.mean(ref ** 2, axis=0))
    for i in range(ref.shape[1]):
        err = np.sqrt(np.mean((got[:, i] - ref[:, i]) ** 2))
        assert err <= TOL * max(norms[i], FLOOR * norms.max()), i


def _fill_scratch_with_other_data(lib, _lib, stream):
    """A call of another layout (1024^2, batch of 4 waves, free space) leaves
    the shared array full of waves unrelated to the next call's."""
    from paper_1706_08563_b300 import api
    w = W.scaled(W.C1, n=1024, n_slices=1, slice_dz=20.0)
    plan = api.Plan.from_workload(w)
    trans = torch.ones((1, 1024, 1024), dtype=torch.complex64, device="cuda")
    xy = torch.from_numpy(W.random_positions(w, 4, seed=77)).cuda()
    rings = torch.zeros((4, w.n_rings), dtype=torch.float32, device="cuda")
    assert lib.stem_multislice_scan_noalloc(plan._h, ctypes.c_void_p(trans.data_ptr()),
                                            ctypes.c_void_p(xy.data_ptr()), 4, 4, 1.0,
                                            ctypes.c_void_p(rings.data_ptr()), stream) == _lib.STEM_OK
    torch.cuda.synchronize()


def test_noalloc_matches_workspace_entry_point_twice():
    from paper_1706_08563_b300 import _lib, api
    lib = _lib.load()
    _fill_scratch_with_other_data(lib, _lib, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    w = W.C1
    xyz, gauss = W.atoms(w)
    xy = W.scan_positions(w)
    plan = api.Plan.from_workload(w)
    trans = plan.slice_potentials(torch.from_numpy(xyz).cuda(), torch.from_numpy(gauss).cuda())
    d_xy = torch.from_numpy(xy).cuda()
    n = xy.shape[0]
    batch = 96                      # ragged: 256 probes = 96 + 96 + 64
    ws = plan.multislice_workspace(batch)
    ref = torch.zeros((n, w.n_rings), dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.stem_multislice_scan(plan._h, ctypes.c_void_p(trans.data_ptr()), ctypes.c_void_p(d_xy.data_ptr()),
                                    n, batch, 1.0, ctypes.c_void_p(ref.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                    ws.numel(), stream) == _lib.STEM_OK
    outs = []
    for call in range(2):
        out = torch.zeros((n, w.n_rings), dtype=torch.float32, device="cuda")
        st = lib.stem_multislice_scan_noalloc(plan._h, ctypes.c_void_p(trans.data_ptr()),
                                              ctypes.c_void_p(d_xy.data_ptr()), n, batch, 1.0,
                                              ctypes.c_void_p(out.data_ptr()), stream)
        assert st == _lib.STEM_OK, (call, st)
        outs.append(out)
    torch.cuda.synchronize()
    r = ref.cpu().numpy()
    for out in outs:
        _close(out.cpu().numpy(), r)


def test_noalloc_rejects_batches_beyond_its_scratch():
    from paper_1706_08563_b300 import _lib, api
    lib = _lib.load()
    w = W.scaled(W.C1, n=1024, n_slices=1, slice_dz=20.0)
    plan = api.Plan.from_workload(w)
    trans = torch.ones((1, 1024, 1024), dtype=torch.complex64, device="cuda")
    xy = torch.zeros((5, 2), dtype=torch.float64, device="cuda")
    rings = torch.zeros((5, w.n_rings), dtype=torch.float32, device="cuda")
    before = lib.stem_launch_count()
    st = lib.stem_multislice_scan_noalloc(plan._h, ctypes.c_void_p(trans.data_ptr()), ctypes.c_void_p(xy.data_ptr()),
                                          5, 5, 1.0, ctypes.c_void_p(rings.data_ptr()), None)
    assert st == _lib.STEM_ERR_NOMEM          # 5 waves of 1024^2 = 40 MiB > 32 MiB
    assert lib.stem_launch_count() == before  # nothing launched
    assert float(rings.abs().sum()) == 0.0
    st = lib.stem_multislice_scan_noalloc(plan._h, ctypes.c_void_p(trans.data_ptr()), ctypes.c_void_p(xy.data_ptr()),
                                          5, 4, 1.0, ctypes.c_void_p(rings.data_ptr()), None)
    assert st == _lib.STEM_OK                 # 4 waves fit
    torch.cuda.synchronize()
    assert np.allclose(rings.sum(dim=1).cpu().numpy(), 1.0, atol=1e-4)   # V = 0: all intensity kept


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs two GPUs to make another device current")
def test_noalloc_refuses_a_plan_of_another_device():
    from paper_1706_08563_b300 import _lib, api
    lib = _lib.load()
    w = W.scaled(W.C1, n=64, n_slices=1)
    with torch.cuda.device(0):
        plan = api.Plan.from_workload(w, device="cuda:0")
        trans = torch.ones((1, 64, 64), dtype=torch.complex64, device="cuda:0")
        xy = torch.zeros((2, 2), dtype=torch.float64, device="cuda:0")
        rings = torch.zeros((2, w.n_rings), dtype=torch.float32, device="cuda:0")
    before = lib.stem_launch_count()
    with torch.cuda.device(1):
        st = lib.stem_multislice_scan_noalloc(plan._h, ctypes.c_void_p(trans.data_ptr()),
                                              ctypes.c_void_p(xy.data_ptr()), 2, 2, 1.0,
                                              ctypes.c_void_p(rings.data_ptr()), None)
    assert st == _lib.STEM_ERR_INVALID
    assert lib.stem_launch_count() == before
