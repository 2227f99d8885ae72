"""Small, named runs of the hot-path kernels, for profilers and quick timing.

    python -m paper_1706_08563_b300.profile_case CASE [--repeat R]

Each case runs the real C-ABI calls on a reduced problem (few slices, few
probes) whose working set is still larger than L2, so that a profiler can
capture individual launches of the bench kernels in a minute or two.  Prints
one JSON line with CUDA-event times per call.

Cases
  ms2048    multislice at the PRISM f=8 bench geometry (2048^2, 300 keV): 4 slices,
            16 probes in one launch  -> k_col_pass<2048,*>, k_row_pass<2048,*>
  ms1024    multislice at the 1024^2 bench geometry: 4 slices, 32 probes
  smat2048  S-matrix, 2048^2, f=8, FP16 storage, 2 slices (793 beams, batches of 128)
  out2048   PRISM f=8 output for 4096 probes from a 2-slice S-matrix (FP16)
  smat2048c, out2048c  the same with the Fourier-cropped S-matrix (1536^2, windows of 192)
  pot2048   projected potentials and transmission functions of the full PRISM f=8 bench
            specimen (50 000 atoms, 100 slices of 2048^2)  -> k_potential
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import torch  # noqa: E402

import workloads as W  # noqa: E402
from paper_1706_08563_b300 import api  # noqa: E402

CASES = ("ms2048", "ms1024", "smat2048", "out2048", "smat2048c", "out2048c", "pot2048")


def _timed(fn, repeat):
    s = torch.cuda.current_stream()
    out = []
    for _ in range(repeat):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        torch.cuda.synchronize()
        out.append(a.elapsed_time(b))
    return out


def run(case: str, repeat: int = 1) -> dict:
    dev = torch.device("cuda", torch.cuda.current_device())
    if case == "pot2048":
        w = W.C4
        xyz, gauss = W.atoms(w)
        plan = api.Plan.from_workload(w, device=dev)
        d_xyz, d_gauss = torch.from_numpy(xyz).to(dev), torch.from_numpy(gauss).to(dev)
        out = torch.empty((w.n_slices, w.n, w.n), dtype=torch.complex64, device=dev)
        ws = plan.potentials_workspace(w.n_atoms)
        return {"case": case, "grid": w.n, "slices": w.n_slices, "atoms": w.n_atoms,
                "ms_per_call": _timed(lambda: plan.slice_potentials(d_xyz, d_gauss, out=out, workspace=ws),
                                      repeat)}
    if case in ("ms2048", "smat2048", "out2048", "smat2048c", "out2048c"):
        base = W.C4
        slices = 4 if case == "ms2048" else 2
    else:
        base = W.C3
        slices = 4
    w = W.scaled(base, n_slices=slices, cell=(base.cell[0], base.cell[1], slices * base.slice_dz),
                 n_atoms=base.n_atoms * slices // base.n_slices)
    xyz, gauss = W.atoms(w)
    plan = api.Plan.from_workload(w, device=dev)
    trans = plan.slice_potentials(torch.from_numpy(xyz).to(dev), torch.from_numpy(gauss).to(dev))
    res = {"case": case, "grid": w.n, "slices": w.n_slices}
    if case.startswith("ms"):
        nprobe = 16 if w.n == 2048 else 32
        xy = torch.from_numpy(W.scan_positions(w)[:nprobe]).to(dev)
        ws = plan.multislice_workspace(nprobe)
        rings = torch.zeros((nprobe, w.n_rings), device=dev)
        res["ms_per_call"] = _timed(lambda: plan.multislice(trans, xy, batch=nprobe, rings=rings, workspace=ws),
                                    repeat)
        res["probes"] = nprobe
    else:
        f = 8
        ws = torch.empty(int(api._lib.load().stem_prism_smatrix_workspace(plan._h, 128)), dtype=torch.uint8,
                         device=dev)
        holder = {}

        cropped = case.endswith("c")

        def smat():
            holder["sm"] = plan.prism_smatrix(trans, f, "f16", batch=128, workspace=ws, cropped=cropped)
        t_s = _timed(smat, repeat if case.startswith("smat") else 1)
        if case.startswith("smat"):
            res["ms_per_call"] = t_s
            res["beams"] = holder["sm"].n_beams
        else:
            xy = torch.from_numpy(W.scan_positions(w)[:4096]).to(dev)
            wso = plan.prism_output_workspace(f, 4096)
            rings = torch.zeros((4096, w.n_rings), device=dev)
            res["ms_per_call"] = _timed(lambda: plan.prism_output(holder["sm"], xy, chunk=4096, rings=rings,
                                                                  workspace=wso), repeat)
            res["probes"] = 4096
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=CASES)
    ap.add_argument("--repeat", type=int, default=1)
    a = ap.parse_args()
    print(json.dumps(run(a.case, a.repeat)), flush=True)


if __name__ == "__main__":
    main()
