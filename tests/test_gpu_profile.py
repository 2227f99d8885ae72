"""CUDA-event kernel timing (stem_profile_enable / stem_profile_read): it counts
the launches of each hot kernel family, reports positive device times, and
leaves the results unchanged."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1706_08563_b300 import api as A
    return A


@pytest.mark.parametrize("n", [256, 2048])
def test_profile_counts_slice_passes_and_keeps_results(api, n):
    slices, probes, batch = 3, 6, 4
    w = W.Workload("pr", (20.0, 20.0, 2.0 * slices), 40, n, slices, 2.0, 200.0, 20.0, 4, 2.0, 40, f=(4,))
    xyz, gauss = W.atoms(w, seed=3)
    plan = api.Plan.from_workload(w)
    trans = plan.slice_potentials(torch.from_numpy(xyz).cuda(), torch.from_numpy(gauss).cuda())
    xy = torch.from_numpy(W.random_positions(w, probes, seed=4)).cuda()
    plain = plan.multislice(trans, xy, batch=batch).cpu().numpy()
    api.profile_enable(True)
    try:
        timed = plan.multislice(trans, xy, batch=batch).cpu().numpy()
        sm = plan.prism_smatrix(trans, 4, "f16", batch=8)
        out = plan.prism_output(sm, xy, engine="tensor").cpu().numpy()
        rows, rows_ms = api.profile_read("row_slice")
        cols, cols_ms = api.profile_read("col_slice")
        sums, sums_ms = api.profile_read("beam_sum")
    finally:
        api.profile_enable(False)
    batches = -(-probes // batch)
    beam_batches = -(-sm.n_beams // 8)
    # multislice: a row pass per slice, a slice column pass per slice but the
    # last (the detector pass); the S-matrix: row and slice column passes on
    # every slice but the first (which starts from the transform of t_0)
    assert rows == batches * slices + beam_batches * (slices - 1)
    assert cols == batches * (slices - 1) + beam_batches * (slices - 1)
    assert sums >= 1
    assert rows_ms > 0 and cols_ms > 0 and sums_ms > 0
    np.testing.assert_allclose(timed, plain, rtol=1e-6, atol=1e-9)
    assert np.isfinite(out).all()
    # recording is off again: nothing new is counted
    api.profile_enable(True)
    api.profile_enable(False)
    plan.multislice(trans, xy, batch=batch)
    torch.cuda.synchronize()
    assert api.profile_read("row_slice")[0] == 0
