"""The C ABI from a plain C program (tests/c_client/stem_client.c): it
allocates its own device buffers with the CUDA runtime, runs the potentials
and the multislice scan, and must give the rings the Python binding gives for
the same inputs (and meet the parity bar against the FP64 oracle)."""
import os
import struct
import subprocess

import numpy as np
import pytest
import torch

import workloads as W
from oracle import stem as O
from tolerances import FP32_TOL, check_rings

pytestmark = pytest.mark.gpu


def test_c_client_matches_python_binding_and_oracle(repo_tmp):
    from conftest import build_c_client
    from paper_1706_08563_b300 import api
    exe = build_c_client(repo_tmp)
    w = W.Workload("cc", (16.0, 12.0, 8.0), 30, 64, 4, 2.0, 200.0, 20.0, 0, 2.0, 40)
    xyz, gauss = W.atoms(w, seed=21)
    xy = W.random_positions(w, 37, seed=22)
    inputs = os.path.join(repo_tmp, "inputs.bin")
    out = os.path.join(repo_tmp, "rings.bin")
    with open(inputs, "wb") as fh:
        fh.write(struct.pack("<5i", w.n, w.n_slices, w.n_rings, len(xyz), len(xy)))
        fh.write(struct.pack("<7d", *w.cell, w.slice_dz, w.energy_kev, w.alpha_mrad, w.ring_width_mrad))
        fh.write(np.ascontiguousarray(xyz, "<f8").tobytes())
        fh.write(np.ascontiguousarray(gauss, "<f4").tobytes())
        fh.write(np.ascontiguousarray(xy, "<f8").tobytes())
    r = subprocess.run([exe, inputs, out], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    got = np.fromfile(out, "<f4").reshape(len(xy), w.n_rings)

    plan = api.Plan.from_workload(w)
    trans = plan.slice_potentials(torch.from_numpy(xyz).cuda(), torch.from_numpy(gauss).cuda())
    ref = plan.multislice(trans, torch.from_numpy(xy).cuda(), batch=len(xy)).cpu().numpy()
    assert np.allclose(got, ref, rtol=1e-6, atol=1e-12)     # float atomics: order of additions only

    p = O.params_from(w)
    t = O.transmission(p, O.projected_potential(p, xyz, gauss))
    check_rings(got, O.multislice_rings(p, t, xy), FP32_TOL)
