#!/usr/bin/env python3
"""Benchmark of the multislice / PRISM hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Default workload: mixed-precision PRISM f=8 at paper scale (100 x 100 x 100 A
cell, 50 000 atoms, 2048^2 grid, 100 slices of 1 A, 300 keV, 25 mrad, 256 x 256
probes, S-matrix stored FP16 with per-beam scales).  One step is one whole
simulation: projected potentials -> compact S-matrix (793 beams through 100
slices) -> PRISM output for all 65 536 probes (beam sum, 256^2 window FFT, 100
annular rings).

Beside the timed steps the JSON line states (rank 0, N = 1 extras):
  error      relative L2 error of the step against the FP64 oracle, stage by
             stage: sampled S-matrix beams through all slices, and the
             oracle's output step on the GPU's own S-matrix for sampled probes
  fp32_path  the same step with an FP32 S-matrix and the CUDA-core beam sum,
             with its own probes/s and error
  roofline   HBM fraction of the S-matrix phase and the FP32 lane-operation
             fraction against a measured FMA rate
  multislice batched multislice at paper scale (1024^2, 50 slices, launches of
             256 probes) with its error on sampled probes
  serving    a Poisson stream drawn from the serving ranges (grids 256-2048,
             f 1-16, scans 16^2-256^2, 10-100 slices) through the server
  cpu_baseline  the oracle timed on all host cores on a bounded sample

Prints one JSON line.  Under torchrun (N > 1) every rank runs its own whole
simulation (weak scaling, no data-path collective); rank 0 prints.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import math
import multiprocessing as mp
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "probes/s for multislice and PRISM f=8 at stated error; p50/p99 solve latency"
# DRAM bytes per wave and slice (row + column pass, t_n excluded), measured
# with ncu (dram__bytes_read.sum + dram__bytes_write.sum) on launches of 16
# waves of 2048^2 and 32 waves of 1024^2 of the slice passes
SLICE_TRAFFIC_PER_WAVE = {2048: 83.06e6, 1024: 19.34e6}
HBM_FALLBACK_GBS = 6400.0
LOWP_TOL, FP32_TOL = 1e-2, 1e-4
LOWP_FLOOR, FP32_FLOOR = 1e-4, 1e-5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=W.C4.name, choices=sorted(W.WORKLOADS))
    ap.add_argument("--storage", default="f16", choices=["f32", "f16", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-error", action="store_true", help="skip the stated-error measurement against the oracle")
    ap.add_argument("--no-fp32-path", action="store_true", help="skip the FP32-storage / CUDA-core comparison leg")
    ap.add_argument("--no-cropped", action="store_true", help="skip the Fourier-cropped S-matrix leg")
    ap.add_argument("--prism-split", action="store_true",
                    help="one PRISM simulation split over the ranks (beams for the S-matrix, one all-reduce, then "
                         "probes; strong scaling) instead of one whole simulation per rank")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops", 1800.0)), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, 1800.0, "fallback"


def tensor_peaks():
    """(burst, sustained) dense bf16 TFLOP/s (FP16 runs at the same rate) and the source."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        burst = float(d["bf16_tflops"])
        return burst, float(d.get("bf16_tflops_sustained", burst)), "measured"
    except Exception:
        return 1800.0, 1400.0, "fallback"


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def spawn_pool(workers: int) -> cf.ProcessPoolExecutor:
    """Oracle workers; 'spawn' because the parent has initialised CUDA."""
    return cf.ProcessPoolExecutor(max(1, workers), mp_context=mp.get_context("spawn"))


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


# --------------------------------------------------------------------------- FP32 roofline
# Radix plan of the FFT kernels (first radix = elements per thread, then up to
# two more), as the kernels' FftShape table sets it.
FFT_PLAN = {8: (8,), 16: (4, 4), 32: (8, 4), 64: (8, 8), 128: (16, 8), 256: (16, 16), 512: (32, 16),
            1024: (32, 32), 2048: (16, 16, 8)}


def _dft_lane_ops(r: int) -> int:
    """FP32 lane operations of one in-register radix-r DFT as the kernels do it:
    radix-2 decimation in frequency, each butterfly a complex add and subtract
    (4), each twiddle exp(-2 pi i j / 64) a complex multiply (4) except j = 0 and
    16 (sign swaps, 0) and j = 8, 24 (an add and a multiply per part, 4)."""
    ops = 0
    span = r // 2
    while span >= 1:
        for _start in range(0, r, 2 * span):
            for k in range(span):
                ops += 4
                j = k * (64 // (2 * span))
                if j not in (0, 16):
                    ops += 4
        span //= 2
    return ops


def fft_lane_ops_per_element(n: int) -> float:
    """FP32 lane operations per element of one length-n transform: the radix-E
    stage, then for each later stage (r - 1) table twiddles (4 each) and the
    radix-r DFTs."""
    plan = FFT_PLAN[n]
    e = plan[0]
    ops = _dft_lane_ops(e)
    for r in plan[1:]:
        ops += (e // r) * ((r - 1) * 4 + _dft_lane_ops(r))
    return ops / e


def band_cols(n: int) -> int:
    """Columns the slice column pass visits: whole column tiles that touch the
    2/3 band limit |m| <= n/3 (tiles of 4 columns in the TMA passes at 1024 and
    2048, of up to 16 otherwise)."""
    c = 4 if n in (1024, 2048) else max(1, min(16, 256 // (n // FFT_PLAN[n][0])))
    mb = n // 3
    lo, hi0 = (mb + 1 + c - 1) // c, (n - mb) // c
    return (lo + n // c - hi0) * c if lo < hi0 else n


def smatrix_lane_ops(n: int, n_slices: int, n_beams: int) -> float:
    """FP32 lane operations of the S-matrix build: per beam, S - 1 slice row
    passes (2 transforms of every row + the transmission product, 4 per
    element) and S - 1 slice column passes over the column tiles inside the
    band limit (2 transforms + the propagator products, 8 per element); the
    first slice's column pass (1 transform + propagator, from the shared 2D
    transform of t_0) and the last row pass (1 inverse transform)."""
    cols = band_cols(n)
    per_fft = fft_lane_ops_per_element(n)
    row = n * n * (2 * per_fft + 4)
    col = cols * n * (2 * per_fft + 8)
    first = cols * n * (per_fft + 8)
    last = n * n * per_fft
    return float(n_beams) * ((n_slices - 1) * (row + col) + first + last)


def measure_fma_rate(lib, dev) -> dict:
    """Measured FP32 lane-operation rate of this GPU: independent FMA chains,
    scalar and packed f32x2, timed with CUDA events (libstem's probe kernel)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms * 8
    out = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {}
    for packed in (0, 1):
        lib.stem_selftest_fma_rate(packed, 1000, blocks, out.data_ptr(), None)
        torch.cuda.synchronize()
        iters = 1 << 20
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lib.stem_selftest_fma_rate(packed, iters, blocks, out.data_ptr(), None)
        b.record(stream)
        torch.cuda.synchronize()
        ops = blocks * 256 * iters * 8 * (2 if packed else 1)
        res["packed_f32x2" if packed else "scalar"] = ops / (a.elapsed_time(b) / 1e3) / 1e12
    res["peak_tops"] = max(res["scalar"], res["packed_f32x2"])
    return res


# --------------------------------------------------------------------------- oracle workers
def _oracle_beam(args):
    """Oracle exit wave of one S-matrix beam through every slice (FP64), on the
    simulation grid or Fourier-cropped."""
    from oracle import stem as O
    params, t_path, mn, cropped = args
    t = np.load(t_path, mmap_mode="r")
    fn = O.prism_smatrix_cropped if cropped else O.prism_smatrix
    return fn(params, t, np.asarray([mn], dtype=np.int64))[0]


def _oracle_ms_rings(args):
    from oracle import stem as O
    params, t_path, xy = args
    t = np.load(t_path, mmap_mode="r")
    return O.multislice_rings(params, t, xy)


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = math.sqrt(float(np.mean(b * b)))
    return math.sqrt(float(np.mean((a - b) ** 2))) / den if den > 0 else float("nan")


def ring_errors(got, ref, floor) -> dict:
    """Whole-array relative L2 and the largest per-ring relative L2 over the
    rings whose RMS is at least floor x the brightest ring's; darker rings are
    reported by their absolute error relative to the brightest ring."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    norms = np.sqrt(np.mean(ref ** 2, axis=0))
    top = float(norms.max())
    errs = np.sqrt(np.mean((got - ref) ** 2, axis=0))
    bright = norms >= floor * top
    return {"rel_l2": rel_l2(got, ref),
            "max_ring_rel_l2": float(np.max(errs[bright] / norms[bright])),
            "rings_above_floor": int(bright.sum()),
            "dark_rings_max_abs_err_over_top_ring": float(np.max(errs[~bright]) / top) if (~bright).any() else 0.0,
            "floor": floor}


def output_stage_error(p, sm, beams, f, xy, got, floor) -> dict:
    """The oracle's output step (window crop, beam sum, W x W FFT, rings) on the
    GPU's own S-matrix, read window by window, against the GPU's rings."""
    from oracle import stem as O
    ref = O.prism_rings(p, sm, beams, f, xy, grid=sm.n)
    return ring_errors(got, ref, floor)


def smatrix_stage_error(sm, picks, oracle_beams) -> list:
    """Relative L2 of stored beams (times their scale) against the oracle's."""
    out = []
    sc = sm.scales().cpu().numpy()
    for b, ref in zip(picks, oracle_beams):
        d = sm.data()[:, :, :, b].double().cpu().numpy()
        got = (d[:, :, 0] + 1j * d[:, :, 1]) * float(sc[b])
        out.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
    return out


# --------------------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1706_08563_b300 as P
    from paper_1706_08563_b300 import api

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    lib = P.load()
    w = W.WORKLOADS[args.workload]
    prism = bool(w.f)
    f = w.f[-1] if prism else 1
    xyz, gauss = W.atoms(w)
    if w.fp_sigma > 0:
        xyz = W.displaced(w, xyz, rank % max(w.fp_configs, 1))
    xy = W.scan_positions(w)
    n_probes = xy.shape[0]
    extras = rank == 0

    # pinned host inputs (the end-to-end leg copies them every step)
    h_xyz = torch.from_numpy(xyz).pin_memory()
    h_gauss = torch.from_numpy(gauss).pin_memory()
    h_xy = torch.from_numpy(xy).pin_memory()
    d_xyz = torch.empty_like(h_xyz, device=dev)
    d_gauss = torch.empty_like(h_gauss, device=dev)
    d_xy = torch.empty_like(h_xy, device=dev)
    d_xyz.copy_(h_xyz)
    d_gauss.copy_(h_gauss)
    d_xy.copy_(h_xy)

    plan = api.Plan.from_workload(w, device=dev)
    trans = torch.empty((w.n_slices, w.n, w.n), dtype=torch.complex64, device=dev)
    ws_pot = plan.potentials_workspace(w.n_atoms)
    total = args.warmup + args.steps
    rings = [torch.zeros((n_probes, w.n_rings), dtype=torch.float32, device=dev) for _ in range(total)]
    h_rings = torch.empty((n_probes, w.n_rings), dtype=torch.float32).pin_memory()
    holder = {}
    if prism:
        batch, chunk = w.batch, 4096
        sm_bytes = lib.stem_prism_smatrix_bytes(plan._h, f, _storage_code(args.storage))
        sm_buf = torch.empty(sm_bytes, dtype=torch.uint8, device=dev)
        ws_s = torch.empty(lib.stem_prism_smatrix_workspace(plan._h, batch), dtype=torch.uint8, device=dev)
        ws_o = plan.prism_output_workspace(f, chunk)
        n_beams = len(plan.prism_beams(f))
    else:
        batch = w.batch
        ws_m = plan.multislice_workspace(batch)
        n_beams = 0

    stream = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    split = prism and args.prism_split
    if split:
        from paper_1706_08563_b300.parallel import shard_range, sharded_smatrix, gather_rows
        sm_view = plan.prism_smatrix_view(sm_buf, f, args.storage)
        p0, p1 = shard_range(n_probes, rank, world)

    def step(i, copy_in):
        e = [ev() for _ in range(6)]
        e[0].record(stream)
        if copy_in:
            d_xyz.copy_(h_xyz, non_blocking=True)
            d_gauss.copy_(h_gauss, non_blocking=True)
            d_xy.copy_(h_xy, non_blocking=True)
        e[1].record(stream)
        plan.slice_potentials(d_xyz, d_gauss, out=trans, workspace=ws_pot)
        e[2].record(stream)
        if split:
            # beams of this rank into the zeroed S-matrix, one sum over the ranks,
            # then this rank's probes and one gather of the rings
            sharded_smatrix(n_beams, lambda b0, b1: plan.prism_smatrix(
                trans, f, args.storage, batch=batch, workspace=ws_s, out=sm_buf, beams=(b0, b1)),
                [sm_view.scales(), sm_view.data()])
            holder["sm"] = sm_view
            e[3].record(stream)
            part = plan.prism_output(sm_view, d_xy[p0:p1], chunk=chunk, workspace=ws_o)
            rings[i].copy_(gather_rows(part, n_probes) if world > 1 else part)
        elif prism:
            holder["sm"] = plan.prism_smatrix(trans, f, args.storage, batch=batch, workspace=ws_s, out=sm_buf)
            e[3].record(stream)
            plan.prism_output(holder["sm"], d_xy, chunk=chunk, rings=rings[i], workspace=ws_o)
        else:
            e[3].record(stream)
            plan.multislice(trans, d_xy, batch=batch, rings=rings[i], workspace=ws_m)
        e[4].record(stream)
        if copy_in:
            h_rings.copy_(rings[i], non_blocking=True)
        e[5].record(stream)
        return e

    for i in range(args.warmup):
        step(i, True)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()

    clocks = Clocks(local_rank)
    clocks.start()
    launches0 = lib.stem_launch_count()
    api.profile_enable(True)          # CUDA events around each hot kernel launch (roofline per kernel)
    t0 = time.perf_counter()
    evs = []
    for i in range(args.steps):
        evs.append(step(args.warmup + i, True))
        stream.synchronize()          # the result read-back is part of each end-to-end step
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = lib.stem_launch_count() - launches0
    try:
        kprof = {k: api.profile_read(k) for k in api.PROF_KINDS}
    except Exception as exc:          # an event call failed: keep the phase-level roofline only
        print(f"kernel timing unavailable: {exc}", file=sys.stderr)
        kprof = {k: (0, 0.0) for k in api.PROF_KINDS}
    api.profile_enable(False)
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()

    dev_ms = [e[1].elapsed_time(e[4]) for e in evs]          # inputs resident: compute only
    e2e_ms = [e[0].elapsed_time(e[5]) for e in evs]          # H2D + compute + D2H
    pot_ms = [e[1].elapsed_time(e[2]) for e in evs]
    sm_ms = [e[2].elapsed_time(e[3]) for e in evs]
    out_ms = [e[3].elapsed_time(e[4]) for e in evs]
    tot_dev = sum(dev_ms)
    tot_e2e = sum(e2e_ms)
    if world > 1:
        t = torch.tensor([tot_dev, tot_e2e], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        tot_dev, tot_e2e = float(t[0]), float(t[1])
    probes_all = n_probes * (1 if split else world) * args.steps
    res = {
        "metric": METRIC,
        "value": probes_all / (tot_dev / 1e3),
        "unit": "probes/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": tot_dev / args.steps,
        "higher_is_better": True,
        "scaling": "strong" if split else "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
    }
    cfg = {"workload": w.name, "algorithm": f"PRISM f={f}" if prism else "multislice",
           "cell_A": list(w.cell), "atoms": w.n_atoms, "grid": w.n, "slices": w.n_slices, "slice_dz_A": w.slice_dz,
           "kev": w.energy_kev, "alpha_mrad": w.alpha_mrad, "probes": n_probes, "rings": w.n_rings,
           "batch": batch, "l2": "no flush: inputs and working set far larger than L2 (126 MB)",
           "step": "potentials + " + ("S-matrix + PRISM output" if prism else "multislice scan"),
           "parallelism": (f"PRISM split over {world} ranks: beams, one all-reduce, probes, one gather" if split
                           else f"{world} independent simulations (one per rank)")}
    if prism:
        cfg.update({"f": f, "beams": n_beams, "smatrix_storage": args.storage, "chunk": chunk,
                    "beam_sum": "FP32 CUDA cores" if args.storage == "f32" else "tcgen05 complex GEMM (16-bit in, FP32 accumulate)"})
    res["config"] = cfg
    res["phases_ms"] = {"potentials": statistics.mean(pot_ms),
                        ("smatrix" if prism else "unused"): statistics.mean(sm_ms),
                        ("output" if prism else "multislice"): statistics.mean(out_ms)}
    res["latency"] = {"p50_ms": float(np.percentile(dev_ms, 50)), "p99_ms": float(np.percentile(dev_ms, 99)),
                      "what": "one whole simulation (device time)"}
    # the rate of each phase on its own
    rates = {"potential_slices_per_s": w.n_slices / (statistics.mean(pot_ms) / 1e3)}
    if prism:
        rates["smatrix_beams_per_s"] = n_beams / (statistics.mean(sm_ms) / 1e3)
        rates["output_probes_per_s"] = n_probes / (statistics.mean(out_ms) / 1e3)
    else:
        rates["multislice_probes_per_s"] = n_probes / (statistics.mean(out_ms) / 1e3)
    res["phase_rates"] = rates
    hbm, _, src = peaks()
    n2 = w.n * w.n
    # inside the slice loop only the columns within the 2/3 band limit hold data
    band = (2 * (w.n // 3) + 1) / w.n
    if prism:
        nbatches = math.ceil(n_beams / batch)
        esz = 4 if args.storage == "f32" else 2
        # per beam: 2 HBM round trips per slice (row + column pass) over the in-band
        # columns, the final row IFFT pass (in-band read, full write) and the
        # transposing store; t_n is read once per beam batch
        alg = (n_beams * (w.n_slices * 32.0 * band + 8.0 * band + 8.0 + 8.0 + 2.0 * esz) * n2
               + nbatches * w.n_slices * 8.0 * n2)
        ms = statistics.mean(sm_ms)
        kernel = {2048: "k_row_slice_pair_2048 + k_col_slice_tma<2048> (S-matrix slice passes)",
                  1024: "k_row_pass<1024> + k_col_slice_tma<1024> (S-matrix slice passes)"}.get(
                      w.n, f"k_row_pass/k_col_pass<{w.n}> (S-matrix slice passes)")
    else:
        nb = math.ceil(n_probes / batch)
        # per probe: init write, then per slice row + column pass, the last column
        # pass reads only (detector): 32 S B per in-band pixel; t_n once per batch
        alg = n_probes * w.n_slices * 32.0 * band * n2 + nb * w.n_slices * 8.0 * n2
        ms = statistics.mean(out_ms)
        kernel = {2048: "k_row_slice_pair_2048 + k_col_slice_tma<2048> (multislice slice passes)",
                  1024: "k_row_pass<1024> + k_col_slice_tma<1024> (multislice slice passes)"}.get(
                      w.n, f"k_row_pass/k_col_pass<{w.n}> (multislice slice passes)")
    ach = alg / (ms / 1e3) / 1e9
    per_wave = SLICE_TRAFFIC_PER_WAVE.get(w.n)
    waves = n_beams if prism else n_probes
    # the dominant kernels alone: the slice row and column passes, timed by CUDA
    # events around each of their launches over the timed steps.  Per step the
    # S-matrix runs S - 1 of each per beam (the first slice starts from the 2D
    # transform of t_0); multislice runs S row passes and S - 1 slice column
    # passes per probe (the last is the detector).
    (n_row, row_ms), (n_col, col_ms) = kprof["row_slice"], kprof["col_slice"]
    row_ws = waves * (w.n_slices - 1 if prism else w.n_slices)
    col_ws = waves * (w.n_slices - 1)
    k_alg = (row_ws + col_ws) * 16.0 * band * n2 + (n_row / args.steps) * 8.0 * n2
    # measured DRAM bytes per (row + column) pass pair, split evenly, plus t_n per row-pass launch
    traffic = (None if per_wave is None
               else per_wave / 2.0 * (row_ws + col_ws) + (n_row / args.steps) * 8.0 * n2)
    k_ms = (row_ms + col_ms) / args.steps
    k_ach = k_alg / (k_ms / 1e3) / 1e9 if k_ms > 0 else None
    if not k_ach:                     # no kernel timing: the phase-level figures stand in
        k_ach, k_alg = ach, alg
    res["roofline"] = {"bound": "hbm", "achieved": k_ach, "peak": hbm, "unit": "GB/s",
                       "frac": k_ach / hbm,
                       "traffic": traffic, "traffic_unit": "bytes per step (slice passes, scaled from a 16-wave capture)",
                       "kernel": kernel, "peak_source": src, "algorithmic_bytes_per_step": k_alg,
                       "what": "band-limited algorithmic bytes of the slice row and column passes / their summed "
                               "launch durations (CUDA events around every launch in the timed steps)",
                       "launches_per_step": {"row": n_row / args.steps, "col": n_col / args.steps},
                       "ms_per_launch": {"row": row_ms / max(n_row, 1), "col": col_ms / max(n_col, 1)},
                       "phase": {"achieved": ach, "frac": ach / hbm, "algorithmic_bytes_per_step": alg,
                                 "what": ("whole S-matrix phase" if prism else "whole multislice call")
                                 + " (first-slice, last-slice and store passes included) / phase time"}}
    if prism and extras:
        fma = measure_fma_rate(lib, dev)
        ops = smatrix_lane_ops(w.n, w.n_slices, n_beams)
        ach_ops = ops / (ms / 1e3) / 1e12
        # the slice passes alone: row pass 2 transforms + transmission per element,
        # column pass 2 transforms + propagator products on the in-band columns
        per_fft = fft_lane_ops_per_element(w.n)
        k_ops = (row_ws * n2 * (2 * per_fft + 4) + col_ws * band_cols(w.n) * w.n * (2 * per_fft + 8))
        k_ach_ops = k_ops / (k_ms / 1e3) / 1e12 if k_ms > 0 else ach_ops
        res["roofline"]["fp32"] = {
            "bound": "alu", "achieved": k_ach_ops, "peak": fma["peak_tops"], "unit": "T lane-ops/s",
            "frac": k_ach_ops / fma["peak_tops"], "lane_ops_per_step": k_ops,
            "lane_ops_per_element_per_fft": per_fft,
            "peak_source": "measured in this run: independent FMA chains (scalar "
                           f"{fma['scalar']:.1f}, packed f32x2 {fma['packed_f32x2']:.1f} T lane-ops/s)",
            "what": "FP32 lane operations of the slice row and column passes counted from the kernels' radix "
                    "plan (transforms, twiddles, transmission and propagator products) / their summed launch "
                    "durations",
            "phase": {"achieved": ach_ops, "frac": ach_ops / fma["peak_tops"], "lane_ops_per_step": ops,
                      "what": "the whole S-matrix phase's lane operations / S-matrix phase time"}}
    n_sum, sum_ms = kprof["beam_sum"]
    if prism and n_sum > 0 and args.storage != "f32":
        # useful work of the window beam sums: a complex multiply-add (8 flops)
        # per probe, window pixel and beam; the kernel runs inside a long step,
        # so the sustained tensor rate is the denominator
        burst, sustained, tsrc = tensor_peaks()
        flop = float(n_probes) * (w.n // f) ** 2 * n_beams * 8.0
        t_ach = flop / (sum_ms / args.steps / 1e3) / 1e12
        res["roofline"]["beam_sum"] = {
            "bound": "tensor", "achieved": t_ach, "peak": sustained, "unit": "TFLOP/s", "frac": t_ach / sustained,
            "frac_of_burst": t_ach / burst, "peak_source": tsrc + " (bf16 sustained; FP16 has the same dense rate)",
            "kernel": "k_beam_sum_umma (tcgen05, FP16 S-matrix)", "flop_per_step": flop,
            "launches_per_step": n_sum / args.steps, "ms_per_launch": sum_ms / n_sum,
            "what": "useful flops of the window beam sums / the beam-sum launches' summed durations"}
    res["kernel_ms_per_step"] = {k: v[1] / args.steps for k, v in kprof.items()}
    res["e2e"] = {"value": probes_all / (tot_e2e / 1e3), "unit": "probes/s",
                  "h2d_bytes_per_step": int(h_xyz.numel() * 8 + h_gauss.numel() * 4 + h_xy.numel() * 8),
                  "d2h_bytes_per_step": int(h_rings.numel() * 4)}
    res["gpu_launches"] = int(launches)
    res["clocks"] = clk
    res["wall_s_timed"] = wall
    if not extras:
        return res

    # ---- stated error (stage by stage against the FP64 oracle), FP32 path, side measurements
    from oracle import stem as O
    p = O.params_from(w)
    tmp = tempfile.mkdtemp(prefix="stem_bench_")
    pool = None
    try:
        cores = host_cores()
        beam_futs, ms_job = [], None
        if prism and not args.no_error:
            beams_o = O.prism_beams(p, f)
            picks = sorted({0, len(beams_o) // 2, len(beams_o) - 1})
            t_path = os.path.join(tmp, "trans.npy")
            np.save(t_path, trans.cpu().numpy())
            pool = spawn_pool(min(cores, 2 * len(picks) + 4))
            beam_futs = [pool.submit(_oracle_beam, (p, t_path, beams_o[b], False)) for b in picks]
            crop_futs = [pool.submit(_oracle_beam, (p, t_path, beams_o[b], True)) for b in picks]
        if prism:
            res["multislice"], ms_job = measure_multislice(args, dev, hbm, src, pool, tmp)
        if prism and not args.no_error:
            sample = np.unique(np.linspace(0, n_probes - 1, 8).astype(np.int64))
            got = rings[args.warmup + args.steps - 1].cpu().numpy()[sample]
            err_out = output_stage_error(p, holder["sm"], beams_o, f, xy[sample], got, LOWP_FLOOR)
            err_out["probes"] = int(len(sample))
        fp32, sm32 = None, None
        if prism and not args.no_fp32_path and args.storage != "f32":
            fp32, sm32, rings32 = measure_fp32_path(plan, trans, d_xyz, d_gauss, d_xy, w, f, batch, chunk, ws_pot,
                                                    ws_o, n_probes)
            if not args.no_error:
                fp32["error"] = {"bound": FP32_TOL, "output_stage": output_stage_error(
                    p, sm32, beams_o, f, xy[sample], rings32[sample], FP32_FLOOR) | {"probes": int(len(sample))}}
        crop, smc = None, None
        if prism and args.storage != "f32" and not args.no_cropped:
            crop, smc, rings_c = measure_cropped(plan, trans, d_xyz, d_gauss, d_xy, w, f, batch, chunk, ws_pot, ws_o,
                                                 n_probes, args.storage, sm_bytes)
            if not args.no_error:
                crop["error"] = {"bound": LOWP_TOL, "output_stage": output_stage_error(
                    p, smc, beams_o, f, xy[sample], rings_c[sample], LOWP_FLOOR) | {"probes": int(len(sample))}}
        if not args.no_serving:
            res["serving"] = measure_serving(dev)
        if prism and not args.no_error:
            oracle_beams = [fu.result(timeout=3600) for fu in beam_futs]
            e_s = smatrix_stage_error(holder["sm"], picks, oracle_beams)
            tol = LOWP_TOL if args.storage != "f32" else FP32_TOL
            res["error"] = {
                "metric": "relative L2, RMS(diff) / RMS(ref), against the FP64 oracle",
                "bound": tol,
                "smatrix_stage": {"beams": [int(b) for b in picks], "rel_l2": e_s,
                                  "what": "sampled beams through all slices: the oracle on the GPU's t_n vs the "
                                          "stored beams times their scale"},
                "output_stage": err_out | {"what": "the oracle's output step (window crop, beam sum, window FFT, "
                                                   "rings) on the GPU's own S-matrix, read window by window, vs the "
                                                   "timed step's rings for the sampled probes"},
                "composed_first_order": err_out["rel_l2"] + 2.0 * max(e_s),
                "composed_what": "output-stage error + 2 x the largest S-matrix beam error (a ring is quadratic "
                                 "in the beams: first-order bound of the end-to-end ring error)"}
            if sm32 is not None:
                s32 = smatrix_stage_error(sm32, picks, oracle_beams)
                fp32["error"]["smatrix_stage"] = {"beams": [int(b) for b in picks], "rel_l2": s32}
                fp32["error"]["composed_first_order"] = fp32["error"]["output_stage"]["rel_l2"] + 2.0 * max(s32)
            if smc is not None:
                c_beams = [fu.result(timeout=3600) for fu in crop_futs]
                sc = smatrix_stage_error(smc, picks, c_beams)
                crop["error"]["smatrix_stage"] = {"beams": [int(b) for b in picks], "rel_l2": sc}
                crop["error"]["composed_first_order"] = crop["error"]["output_stage"]["rel_l2"] + 2.0 * max(sc)
        del sm32, smc
        if fp32 is not None:
            res["fp32_path"] = fp32
        if crop is not None:
            res["cropped"] = crop
        if ms_job is not None:
            fut_list, got_ms, xy_ms, floor_ms = ms_job
            ref_ms = np.concatenate([fu.result(timeout=3600) for fu in fut_list], axis=0)
            res["multislice"]["error"] = ring_errors(got_ms, ref_ms, floor_ms) | {
                "probes": int(len(xy_ms)), "bound": FP32_TOL,
                "what": "sampled probes of the timed launch end to end against the oracle on the GPU's t_n"}
    finally:
        if pool is not None:
            pool.shutdown(cancel_futures=True)
        shutil.rmtree(tmp, ignore_errors=True)
    return res


def _storage_code(s):
    return {"f32": 0, "f16": 1, "bf16": 2}[s]


def measure_fp32_path(plan, trans, d_xyz, d_gauss, d_xy, w, f, batch, chunk, ws_pot, ws_o, n_probes):
    """The same whole step with an FP32 S-matrix and the CUDA-core beam sum.
    Returns (result, its S-matrix, rings of the last step on the host)."""
    import torch
    from paper_1706_08563_b300 import _lib
    lib = _lib.load()
    dev = trans.device
    buf = torch.empty(lib.stem_prism_smatrix_bytes(plan._h, f, 0), dtype=torch.uint8, device=dev)
    ws_s = torch.empty(lib.stem_prism_smatrix_workspace(plan._h, batch), dtype=torch.uint8, device=dev)
    rings = torch.zeros((n_probes, w.n_rings), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    holder = {}

    def one():
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        rings.zero_()
        e[0].record(stream)
        plan.slice_potentials(d_xyz, d_gauss, out=trans, workspace=ws_pot)
        e[1].record(stream)
        holder["sm"] = plan.prism_smatrix(trans, f, "f32", batch=batch, workspace=ws_s, out=buf)
        e[2].record(stream)
        plan.prism_output(holder["sm"], d_xy, chunk=chunk, engine="simt", rings=rings, workspace=ws_o)
        e[3].record(stream)
        return e
    one()
    torch.cuda.synchronize()
    evs = [one() for _ in range(2)]
    torch.cuda.synchronize()
    tot = [e[0].elapsed_time(e[3]) for e in evs]
    out = {"value": n_probes / (statistics.mean(tot) / 1e3), "unit": "probes/s", "ms_per_step": statistics.mean(tot),
           "steps": 2, "warmup": 1, "smatrix_storage": "f32", "beam_sum": "FP32 CUDA cores (SIMT tiled complex GEMM)",
           "phases_ms": {"potentials": statistics.mean(e[0].elapsed_time(e[1]) for e in evs),
                         "smatrix": statistics.mean(e[1].elapsed_time(e[2]) for e in evs),
                         "output": statistics.mean(e[2].elapsed_time(e[3]) for e in evs)}}
    return out, holder["sm"], rings.cpu().numpy()


def measure_cropped(plan, trans, d_xyz, d_gauss, d_xy, w, f, batch, chunk, ws_pot, ws_o, n_probes, storage,
                    full_bytes):
    """The same whole step with the Fourier-cropped S-matrix (3N/4 grid, W' = 3W/4
    windows).  Returns (result, its S-matrix, rings of the last step on the host)."""
    import torch
    from paper_1706_08563_b300 import _lib
    lib = _lib.load()
    dev = trans.device
    code = {"f16": 1, "bf16": 2}[storage] | _lib.STEM_CROPPED
    buf = torch.empty(lib.stem_prism_smatrix_bytes(plan._h, f, code), dtype=torch.uint8, device=dev)
    ws_s = torch.empty(lib.stem_prism_smatrix_workspace(plan._h, batch), dtype=torch.uint8, device=dev)
    rings = torch.zeros((n_probes, w.n_rings), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    holder = {}

    def one():
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        rings.zero_()
        e[0].record(stream)
        plan.slice_potentials(d_xyz, d_gauss, out=trans, workspace=ws_pot)
        e[1].record(stream)
        holder["sm"] = plan.prism_smatrix(trans, f, storage, batch=batch, workspace=ws_s, out=buf, cropped=True)
        e[2].record(stream)
        plan.prism_output(holder["sm"], d_xy, chunk=chunk, rings=rings, workspace=ws_o)
        e[3].record(stream)
        return e
    one()
    torch.cuda.synchronize()
    evs = [one() for _ in range(2)]
    torch.cuda.synchronize()
    tot = [e[0].elapsed_time(e[3]) for e in evs]
    sm = holder["sm"]
    out = {"value": n_probes / (statistics.mean(tot) / 1e3), "unit": "probes/s", "ms_per_step": statistics.mean(tot),
           "steps": 2, "warmup": 1, "smatrix_storage": storage + " Fourier-cropped",
           "grid": sm.n, "window": sm.n // f, "smatrix_bytes": int(buf.numel()),
           "smatrix_bytes_uncropped": int(full_bytes),
           "phases_ms": {"potentials": statistics.mean(e[0].elapsed_time(e[1]) for e in evs),
                         "smatrix": statistics.mean(e[1].elapsed_time(e[2]) for e in evs),
                         "output": statistics.mean(e[2].elapsed_time(e[3]) for e in evs)},
           "what": "S-matrix stored on the 3N/4 grid that holds the 2/3 band exactly; windows of 3W/4 pixels over "
                   "the same L/f; a different (Fourier-interpolated) sampling, checked against its own oracle"}
    return out, sm, rings.cpu().numpy()


def measure_multislice(args, dev, hbm, src, pool, tmp):
    """Batched multislice at paper scale: launches of 256 probes, 1024^2, 50 slices.
    Returns the result and, when an oracle pool is given, the pending error job."""
    import torch
    from paper_1706_08563_b300 import api
    w = W.C3
    xyz, gauss = W.atoms(w)
    plan = api.Plan.from_workload(w, device=dev)
    trans = plan.slice_potentials(torch.from_numpy(xyz).to(dev), torch.from_numpy(gauss).to(dev))
    xy_h = W.scan_positions(w)[: w.batch]
    xy = torch.from_numpy(xy_h).to(dev)
    ws = plan.multislice_workspace(w.batch)
    rings = torch.zeros((w.batch, w.n_rings), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        plan.multislice(trans, xy, batch=w.batch, rings=rings, workspace=ws)
    torch.cuda.synchronize()
    k = max(3, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rings.zero_()
    e0.record(stream)
    for _ in range(k):
        plan.multislice(trans, xy, batch=w.batch, rings=rings, workspace=ws)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / k
    got = rings.cpu().numpy() / k
    job = None
    if pool is not None:
        from oracle import stem as O
        t_path = os.path.join(tmp, "trans_ms.npy")
        np.save(t_path, trans.cpu().numpy())
        pick = np.arange(0, w.batch, 16)
        parts = np.array_split(pick, 4)
        p = O.params_from(w)
        futs = [pool.submit(_oracle_ms_rings, (p, t_path, xy_h[c])) for c in parts]
        # the ring floor grows with the rounding chain (slices x FFT stages), as in the parity tests
        chain = w.n_slices * (2 * math.log2(w.n) + 2) / (10 * (2 * math.log2(128) + 2))
        job = (futs, got[pick], xy_h[pick], FP32_FLOOR * max(1.0, chain))
    n2 = w.n * w.n
    band = (2 * (w.n // 3) + 1) / w.n
    alg = w.batch * w.n_slices * 32.0 * band * n2 + w.n_slices * 8.0 * n2
    ach = alg / (ms / 1e3) / 1e9
    # the same launches under the streaming memory model (stack in pinned host memory)
    host = trans.cpu().pin_memory()
    ws_s = torch.empty(api._lib.load().stem_multislice_streamed_workspace(plan._h, w.batch), dtype=torch.uint8,
                       device=dev)
    for _ in range(2):
        plan.multislice_streamed(host, xy, batch=w.batch, rings=rings, workspace=ws_s)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(k):
        plan.multislice_streamed(host, xy, batch=w.batch, rings=rings, workspace=ws_s)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1) / k
    return ({"workload": w.name, "value": w.batch / (ms / 1e3), "unit": "probes/s", "ms_per_launch": ms,
             "batch": w.batch, "grid": w.n, "slices": w.n_slices,
             "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                          "peak_source": src, "kernel": "k_row_pass<1024> + k_col_slice_tma<1024>"},
             "streamed": {"value": w.batch / (ms_s / 1e3), "unit": "probes/s", "ms_per_launch": ms_s,
                          "footprint_bytes": api.footprint_bytes(w, "ms_streamed", batch=w.batch),
                          "footprint_bytes_single": api.footprint_bytes(w, "ms", batch=w.batch),
                          "h2d_bytes_per_launch": w.n_slices * n2 * 8}}, job)


# Per-request work caps of the serving stream (about a second of GPU time each):
# wave-pixel-slices of a slice loop, and useful flop of a PRISM beam sum.
SERVE_CAP_PIXEL_SLICES = 2.0e11
SERVE_CAP_SUM_FLOP = 5.0e13


def serving_mix(recipes, dev):
    """Bound each recipe's work with the library's own beam counts: a PRISM
    recipe whose S-matrix build is above the cap takes the next larger f; the
    scan side of each recipe's requests is capped so that one request stays
    within the caps.  Returns (recipes, max scan side per recipe)."""
    import dataclasses
    from paper_1706_08563_b300 import api
    out, max_scan = [], []
    for r in recipes:
        w = r.workload
        n2 = w.n * w.n
        if r.algo == "prism":
            plan = api.Plan.from_workload(w, device=dev)
            f = r.f
            while len(plan.prism_beams(f)) * w.n_slices * n2 > SERVE_CAP_PIXEL_SLICES and w.n // (2 * f) >= 8:
                f *= 2
            nb = len(plan.prism_beams(f))
            plan.close()
            r = dataclasses.replace(r, f=f)
            probes = SERVE_CAP_SUM_FLOP / (8.0 * (w.n // f) ** 2 * nb)
        else:
            probes = SERVE_CAP_PIXEL_SLICES / (w.n_slices * n2)
        out.append(r)
        max_scan.append(int(max(1.0, math.sqrt(probes))))
    return out, max_scan


def measure_serving(dev, n_requests=24, rate_hz=4.0, load=0.6):
    """Seeded Poisson stream of mixed multislice / PRISM requests (settings drawn
    from the serving ranges: grids 256-2048, f 1-16, 10-100 slices, scans
    16^2-256^2) through the continuous-batching server, against the same
    requests run one at a time."""
    import threading
    import torch
    from paper_1706_08563_b300 import api
    from paper_1706_08563_b300.serve import Server, SimRequest, run_serial
    budget = 160 << 30
    recipes, max_scan = serving_mix(W.serving_recipes(grids=(256, 512, 1024, 2048), fs=(1, 2, 4, 8, 16),
                                                      slices=(10, 100), count=8), dev)
    stream = W.serving_requests(recipes, n_requests, rate_hz, scans=(16, 32, 64, 128, 256), max_scan=max_scan)
    atoms = {r.specimen: W.atoms(r.workload, seed=r.seed) for r in recipes}

    def make(k, xy):
        r = recipes[k]
        xyz, gauss = atoms[r.specimen]
        return SimRequest(r.specimen, r.workload, xyz, gauss, xy, r.algo, r.f, r.storage)

    # recipes whose resident footprint exceeds the budget are refused at admission
    fits = {k: api.footprint_bytes(r.workload, "prism" if r.algo == "prism" else "ms", f=r.f, storage=r.storage,
                                   batch=64) <= budget for k, r in enumerate(recipes)}
    reqs = [make(k, xy) for _, k, xy in stream if fits[k]]
    probes = sum(r.probe_xy.shape[0] for r in reqs)
    run_serial(reqs[:2], device=dev)                 # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run_serial(reqs, device=dev)
    torch.cuda.synchronize()
    t_serial = time.perf_counter() - t0
    # capacity: the requests queued at once (fresh server, no resident lanes)
    kept = [(t, k, xy) for t, k, xy in stream if fits[k]]
    burst = [make(k, xy) for _, k, xy in kept]
    srv2 = Server(budget, batch=64, prism_chunk=1024, arena=65536, device=dev)
    futs2 = [srv2.submit(r) for r in burst]
    t0 = time.perf_counter()
    srv2.start()
    for fu in futs2:
        fu.result(timeout=1800)
    t_burst = time.perf_counter() - t0
    srv2.stop()
    # latency: Poisson arrivals offering about `load` of that capacity (the same
    # seeded draws, times rescaled), results as soon as their probes are done
    rate = load * len(reqs) / t_burst
    kept = [(t, k, xy) for t, k, xy in W.serving_requests(recipes, n_requests, rate, scans=(16, 32, 64, 128, 256),
                                                           max_scan=max_scan) if fits[k]]
    srv = Server(budget, batch=64, prism_chunk=1024, arena=65536, device=dev)
    srv.start()
    futs = []
    t_start = time.perf_counter()

    def feeder():
        for (t_arr, k, xy), r in zip(kept, [make(k, xy) for _, k, xy in kept]):
            delay = t_start + t_arr - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            futs.append(srv.submit(r))
    th = threading.Thread(target=feeder)
    th.start()
    th.join()
    for fu in futs:
        fu.result(timeout=1800)
    srv.stop()
    lat = np.array(srv.latencies) * 1e3
    return {"requests": len(reqs), "requests_drawn": n_requests,
            "refused_by_footprint": int(sum(1 for _, k, _ in stream if not fits[k])),
            "probes": probes, "arrival_rate_hz": rate, "offered_load": load, "memory_budget_bytes": budget,
            "recipes": [f"{r.algo} N={r.workload.n} S={r.workload.n_slices}" + (f" f={r.f} {r.storage}" if r.algo == "prism" else "")
                        for r in recipes],
            "work_caps": {"wave_pixel_slices": SERVE_CAP_PIXEL_SLICES, "beam_sum_flop": SERVE_CAP_SUM_FLOP},
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "burst_probes_s": probes / t_burst, "serial_probes_s": probes / t_serial,
            "speedup_vs_serial": t_serial / t_burst, "launches_poisson": srv.launches, "launches_burst": srv2.launches,
            "what": ("p50/p99: arrival to result on the host under Poisson arrivals at the offered load (fraction of "
                     "the burst capacity); burst: all requests queued at "
                     "once through the server; serial: the same requests one at a time, no overlap, no resident "
                     "potentials.  Scan sides are drawn from 16-256 and halved while a request's work is above "
                     "the caps (multislice: probes x slices x N^2; PRISM output: 8 W^2 n_beams flop per probe); "
                     "a PRISM recipe whose S-matrix build (beams x slices x N^2) is above the cap takes the "
                     "next larger f")}


# --------------------------------------------------------------------------- oracle timing
def _time_task(args):
    """One timed piece of the oracle's work in a worker process (seconds)."""
    from oracle import stem as O
    kind, params, payload = args
    rng = np.random.default_rng(0)
    n = params.n
    if kind == "pot":
        xyz, gauss = payload
        t0 = time.perf_counter()
        O.projected_potential(params, xyz, gauss)
        return time.perf_counter() - t0
    # a phase-only transmission of the sampled slices (the timing does not depend on the values)
    t = np.exp(1j * rng.random((params.n_slices, n, n)))
    if kind == "beam":
        t0 = time.perf_counter()
        O.prism_smatrix(params, t, np.asarray([payload], dtype=np.int64))
        return time.perf_counter() - t0
    if kind == "ms":
        t0 = time.perf_counter()
        O.multislice_rings(params, t, payload)
        return time.perf_counter() - t0
    # kind == "out": the output step with every beam, S-matrix windows served from one random crop
    beams, f, xy = payload
    w = n // f

    shape = (len(beams), w, w)
    arr = (rng.random(shape, dtype=np.float32) + 1j * rng.random(shape, dtype=np.float32)).astype(np.complex64)

    class Crops:

        def crop(self, rows, cols):
            return arr[:, np.mod(rows, w)][:, :, np.mod(cols, w)]
    t0 = time.perf_counter()
    O.prism_rings(params, Crops(), beams, f, xy)
    return time.perf_counter() - t0


def oracle_rate(w, cores: int, pool=None):
    """The FP64 oracle's probes/s on this host: a bounded sample of workload w
    run by `cores` worker processes at once (one task per worker per phase),
    extrapolated linearly in slices, beams and probes."""
    from oracle import stem as O
    p = O.params_from(w)
    xyz, gauss = W.atoms(w)
    xy = W.scan_positions(w)
    slices_sample = 2
    sub = O.Params(p.cell, p.n, slices_sample, p.slice_dz, p.energy_kev, p.alpha_mrad, p.ring_width_mrad, p.n_rings)
    own = pool is None
    pool = pool or spawn_pool(cores)
    try:
        list(pool.map(abs, range(cores)))       # workers up before any timing
        sl = O.slice_index(p, xyz[:, 2])

        def phase(tasks):
            t0 = time.perf_counter()
            list(pool.map(_time_task, tasks))
            return time.perf_counter() - t0
        # potentials: one slice per worker
        pot_tasks = [("pot", O.Params(p.cell, p.n, 1, p.slice_dz, p.energy_kev, p.alpha_mrad, p.ring_width_mrad,
                                      p.n_rings), (np.c_[xyz[sl == s, :2], np.zeros((sl == s).sum())],
                                                   gauss[sl == s])) for s in range(min(cores, p.n_slices))]
        t_pot = phase(pot_tasks) * p.n_slices / len(pot_tasks)
        if w.f:
            f = w.f[-1]
            beams = O.prism_beams(p, f)
            t_beam = phase([("beam", sub, beams[i % len(beams)]) for i in range(cores)])
            t_smat = t_beam * (len(beams) / cores) * (p.n_slices / slices_sample)
            per = 1
            n_out = min(cores, 4)
            t_o = phase([("out", p, (beams, f, xy[i * per:(i + 1) * per])) for i in range(n_out)])
            t_out = t_o * len(xy) / (n_out * per)
            total = t_pot + t_smat + t_out
            sample = (f"{cores} worker processes: potentials of {len(pot_tasks)}/{p.n_slices} slices; S-matrix "
                      f"{cores} beams x {slices_sample}/{p.n_slices} slices (of {len(beams)} beams); output step "
                      f"of {n_out * per}/{len(xy)} probes with all {len(beams)} beams on {n_out} workers; "
                      "extrapolated linearly")
        else:
            per = 2
            t_m = phase([("ms", sub, xy[i * per:(i + 1) * per]) for i in range(cores)])
            t_ms = t_m * (len(xy) / (cores * per)) * (p.n_slices / slices_sample)
            total = t_pot + t_ms
            sample = (f"{cores} worker processes: potentials of {len(pot_tasks)}/{p.n_slices} slices; multislice "
                      f"of {cores * per}/{len(xy)} probes x {slices_sample}/{p.n_slices} slices; extrapolated "
                      "linearly")
    finally:
        if own:
            pool.shutdown()
    return len(xy) / total, sample


def run_reference(args, rank, world):
    if rank != 0:
        return None
    w = W.WORKLOADS[args.workload]
    cores = host_cores()
    vals = []
    sample = ""
    with spawn_pool(cores) as pool:
        for i in range(args.warmup + args.steps):
            v, sample = oracle_rate(w, cores, pool)
            if i >= args.warmup:
                vals.append(v)
    val = statistics.mean(vals)
    return {"metric": METRIC, "value": val, "unit": "probes/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * w.n_probes / val, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name},
            "cpu_baseline": {"value": val, "unit": "probes/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "probes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    res = run_ours(args, rank, world, local_rank)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        w = W.WORKLOADS[args.workload]
        cores = host_cores()
        v, sample = oracle_rate(w, cores)
        res["cpu_baseline"] = {"value": v, "unit": "probes/s", "cores": cores, "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
