"""The C-ABI calls can be captured in a CUDA graph (no allocation, no host
synchronisation, no per-call setup after the first call): a captured
multislice scan and PRISM output replay to the results of plain calls.  For
small launches a graph removes most of the launch overhead of the 2 S + 1
slice-pass kernels (measured on 256^2 x 20 slices, 8 probes: 0.27 -> 0.18 ms)."""
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def test_multislice_and_prism_output_replay_from_a_cuda_graph():
    from paper_1706_08563_b300 import api
    w = W.Workload("g", (32.0, 32.0, 40.0), 400, 256, 20, 2.0, 200.0, 20.0, 0, 2.0, 50)
    xyz, gauss = W.atoms(w, seed=1)
    plan = api.Plan.from_workload(w)
    trans = plan.slice_potentials(torch.from_numpy(xyz).cuda(), torch.from_numpy(gauss).cuda())
    xy = torch.from_numpy(W.random_positions(w, 8, seed=2)).cuda()
    rings = torch.zeros((8, w.n_rings), device="cuda")
    ws = plan.multislice_workspace(8)
    sm = plan.prism_smatrix(trans, 4, "f16")
    ws_o = plan.prism_output_workspace(4, 8)
    rings_p = torch.zeros_like(rings)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):                  # plain calls first: one-time setup stays out of the graph
        plan.multislice(trans, xy, batch=8, rings=rings, workspace=ws)
        plan.prism_output(sm, xy, chunk=8, rings=rings_p, workspace=ws_o)
    torch.cuda.synchronize()
    ref, ref_p = rings.clone(), rings_p.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rings.zero_()
        rings_p.zero_()
        plan.multislice(trans, xy, batch=8, rings=rings, workspace=ws)
        plan.prism_output(sm, xy, chunk=8, rings=rings_p, workspace=ws_o)
    for _ in range(3):
        g.replay()
        torch.cuda.synchronize()
        assert torch.allclose(rings, ref, rtol=1e-6, atol=1e-12)          # float atomics: order only
        assert torch.allclose(rings_p, ref_p, rtol=1e-6, atol=1e-12)
    xy.copy_(torch.from_numpy(W.random_positions(w, 8, seed=3)).cuda())  # new inputs, same buffers
    g.replay()
    torch.cuda.synchronize()
    direct = torch.zeros_like(rings)
    plan.multislice(trans, xy, batch=8, rings=direct, workspace=ws)
    torch.cuda.synchronize()
    assert torch.allclose(rings, direct, rtol=1e-6, atol=1e-12)
