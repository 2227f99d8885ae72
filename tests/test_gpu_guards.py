"""Out-of-bounds writes, checked without a sanitiser: every output and
workspace handed to the library is the middle of a larger buffer whose guard
regions hold a known byte pattern, and the guards must be intact after the
call.  Covers the potentials, multislice (rings and 4D), the S-matrix, the
PRISM output (both engines, rings and 4D), the detector readout and the FFT,
on ragged sizes."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

GUARD_BYTES = 4096
PATTERN = 0xA5


class Guarded:
    """A device buffer of `nbytes` between two guard regions."""

    def __init__(self, nbytes: int, fill: int = 0):
        self.raw = torch.full((GUARD_BYTES + nbytes + GUARD_BYTES,), PATTERN, dtype=torch.uint8, device="cuda")
        self.raw[GUARD_BYTES:GUARD_BYTES + nbytes] = fill
        self.nbytes = nbytes

    def view(self, dtype=torch.uint8, shape=None) -> torch.Tensor:
        v = self.raw[GUARD_BYTES:GUARD_BYTES + self.nbytes].view(dtype)
        return v if shape is None else v.view(shape)

    def intact(self) -> bool:
        torch.cuda.synchronize()
        lo = self.raw[:GUARD_BYTES]
        hi = self.raw[GUARD_BYTES + self.nbytes:]
        return bool((lo == PATTERN).all()) and bool((hi == PATTERN).all())


def _case(n=128, slices=3, f=4):
    w = W.Workload("gd", (20.0, 18.0, 2.0 * slices), 40, n, slices, 2.0, 200.0, 20.0, 0, 2.0, 37)
    xyz, gauss = W.atoms(w, seed=41)
    xy = W.random_positions(w, 29, seed=42)                  # ragged against every batch size used
    return w, xyz, gauss, xy, f


def test_guards_intact_around_every_output_and_workspace():
    from paper_1706_08563_b300 import _lib, api
    w, xyz, gauss, xy_np, f = _case()
    lib = _lib.load()
    plan = api.Plan.from_workload(w)
    n, S, R, P = w.n, w.n_slices, w.n_rings, len(xy_np)
    xy = torch.from_numpy(xy_np).cuda()
    guards = []

    def g(nbytes, fill=0):
        b = Guarded(int(nbytes), fill)
        guards.append(b)
        return b

    # potentials
    t_buf = g(S * n * n * 8)
    pws = g(lib.stem_slice_potentials_workspace(plan._h, len(xyz)))
    trans = plan.slice_potentials(torch.from_numpy(xyz).cuda(), torch.from_numpy(gauss).cuda(),
                                  out=t_buf.view(torch.complex64, (S, n, n)), workspace=pws.view())
    # multislice rings and 4D, batch 8 (29 = 3 * 8 + 5)
    ws = g(lib.stem_multislice_workspace(plan._h, 8))
    rings = g(P * R * 4)
    plan.multislice(trans, xy, batch=8, rings=rings.view(torch.float32, (P, R)), workspace=ws.view())
    dp = g(P * n * n * 4)
    plan.multislice_4d(trans, xy, batch=8, dp=dp.view(torch.float32, (P, n, n)), workspace=ws.view())
    # S-matrix (FP16, batches of 16 beams) and PRISM output with both engines
    sbytes = lib.stem_prism_smatrix_bytes(plan._h, f, 1)
    sbuf = g(sbytes)
    sws = g(lib.stem_prism_smatrix_workspace(plan._h, 16))
    sm = plan.prism_smatrix(trans, f, "f16", batch=16, workspace=sws.view(), out=sbuf.view())
    ows = g(lib.stem_prism_output_workspace(plan._h, f, 8))
    for engine in ("simt", "tensor"):
        pr = g(P * R * 4)
        plan.prism_output(sm, xy, chunk=8, engine=engine, rings=pr.view(torch.float32, (P, R)), workspace=ows.view())
    wdw = n // f
    pdp = g(P * wdw * wdw * 4)
    plan.prism_output_4d(sm, xy, chunk=8, dp=pdp.view(torch.float32, (P, wdw, wdw)))
    # detector readout and FFT on odd batches
    psi = torch.from_numpy(W.random_complex((5, n, n), seed=43)).to(torch.complex64).cuda()
    dr = g(5 * R * 4)
    plan.detector_readout(psi, f=1, rings=dr.view(torch.float32, (5, R)))
    fb = g(5 * n * n * 8)
    fb.view(torch.complex64, (5, n, n)).copy_(psi)
    st = lib.stem_fft2(n, 5, 0, fb.view().data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    bad = [i for i, b in enumerate(guards) if not b.intact()]
    assert not bad, f"guard regions overwritten: buffers {bad}"
    assert torch.isfinite(rings.view(torch.float32)).all() and float(rings.view(torch.float32).sum()) > 0


def test_guards_intact_at_2048_with_the_tma_column_pass():
    """The TMA-fed column pass and the staged row pass at 2048 (multislice of 3
    probes, 2 slices, and an S-matrix of f = 16)."""
    from paper_1706_08563_b300 import _lib, api
    w = W.Workload("gd2", (100.0, 100.0, 2.0), 500, 2048, 2, 1.0, 300.0, 25.0, 0, 1.0, 64)
    xyz, gauss = W.atoms(w, seed=44)
    lib = _lib.load()
    plan = api.Plan.from_workload(w)
    trans = plan.slice_potentials(torch.from_numpy(xyz).cuda(), torch.from_numpy(gauss).cuda())
    xy = torch.from_numpy(W.random_positions(w, 3, seed=45)).cuda()
    ws = Guarded(lib.stem_multislice_workspace(plan._h, 3))
    rings = Guarded(3 * w.n_rings * 4)
    plan.multislice(trans, xy, batch=3, rings=rings.view(torch.float32, (3, w.n_rings)), workspace=ws.view())
    sbuf = Guarded(lib.stem_prism_smatrix_bytes(plan._h, 16, 1))
    sws = Guarded(lib.stem_prism_smatrix_workspace(plan._h, 5))
    plan.prism_smatrix(trans, 16, "f16", batch=5, workspace=sws.view(), out=sbuf.view())
    assert plan.device_status() == 0
    assert ws.intact() and rings.intact() and sbuf.intact() and sws.intact()
