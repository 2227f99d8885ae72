#!/usr/bin/env python3
"""Benchmark of the multislice / PRISM hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Default workload: mixed-precision PRISM f=8 at paper scale (100 x 100 x 100 A
cell, 50 000 atoms, 2048^2 grid, 100 slices of 1 A, 300 keV, 25 mrad, 256 x 256
probes, S-matrix stored FP16 with per-beam scales).  One step is one whole
simulation: projected potentials -> compact S-matrix (793 beams through 100
slices) -> PRISM output for all 65 536 probes (beam sum, 256^2 window FFT, 100
annular rings).  A secondary measurement times batched multislice at paper
scale (1024^2, 50 slices of 2 A, 200 keV, launches of 256 probes).

Prints one JSON line.  Under torchrun (N > 1) every rank runs its own whole
simulation (weak scaling, no data-path collective); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import math
import os
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
# waves of 2048^2 and 32 waves of 1024^2 of the current slice passes
SLICE_TRAFFIC_PER_WAVE = {2048: 83.09e6, 1024: 19.33e6}
HBM_FALLBACK_GBS = 6400.0


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
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops", 1800.0)), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, 1800.0, "fallback"


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
        if prism:
            sm = plan.prism_smatrix(trans, f, args.storage, batch=batch, workspace=ws_s, out=sm_buf)
            e[3].record(stream)
            plan.prism_output(sm, d_xy, chunk=chunk, rings=rings[i], workspace=ws_o)
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
    t0 = time.perf_counter()
    evs = []
    for i in range(args.steps):
        evs.append(step(args.warmup + i, True))
        stream.synchronize()          # the result read-back is part of each end-to-end step
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = lib.stem_launch_count() - launches0
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
    probes_all = n_probes * world * args.steps
    res = {
        "metric": METRIC,
        "value": probes_all / (tot_dev / 1e3),
        "unit": "probes/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": tot_dev / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
    }
    cfg = {"workload": w.name, "algorithm": f"PRISM f={f}" if prism else "multislice",
           "cell_A": list(w.cell), "atoms": w.n_atoms, "grid": w.n, "slices": w.n_slices, "slice_dz_A": w.slice_dz,
           "kev": w.energy_kev, "alpha_mrad": w.alpha_mrad, "probes": n_probes, "rings": w.n_rings,
           "batch": batch, "l2": "no flush: inputs and working set far larger than L2 (126 MB)",
           "step": "potentials + " + ("S-matrix + PRISM output" if prism else "multislice scan")}
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
        # row + column pass per beam and slice: read + write of the wave each; t_n once per batch
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
    batches = math.ceil(n_beams / batch) if prism else math.ceil(n_probes / batch)
    traffic = None if per_wave is None else per_wave * waves * w.n_slices + batches * w.n_slices * 8.0 * n2
    res["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                       "traffic": traffic, "traffic_unit": "bytes per step (slice passes, scaled from a 16-wave capture)",
                       "kernel": kernel, "peak_source": src, "algorithmic_bytes_per_step": alg}
    res["e2e"] = {"value": probes_all / (tot_e2e / 1e3), "unit": "probes/s",
                  "h2d_bytes_per_step": int(h_xyz.numel() * 8 + h_gauss.numel() * 4 + h_xy.numel() * 8),
                  "d2h_bytes_per_step": int(h_rings.numel() * 4)}
    res["gpu_launches"] = int(launches)
    res["clocks"] = clk
    res["wall_s_timed"] = wall
    if prism and rank == 0:
        res["multislice"] = measure_multislice(args, dev, hbm, src)
    if rank == 0 and not args.no_serving:
        res["serving"] = measure_serving(dev)
    return res


def _storage_code(s):
    return {"f32": 0, "f16": 1, "bf16": 2}[s]


def measure_multislice(args, dev, hbm, src):
    """Batched multislice at paper scale: launches of 256 probes, 1024^2, 50 slices."""
    import torch
    from paper_1706_08563_b300 import api
    w = W.C3
    xyz, gauss = W.atoms(w)
    plan = api.Plan.from_workload(w, device=dev)
    trans = plan.slice_potentials(torch.from_numpy(xyz).to(dev), torch.from_numpy(gauss).to(dev))
    xy = torch.from_numpy(W.scan_positions(w)[: w.batch]).to(dev)
    ws = plan.multislice_workspace(w.batch)
    rings = torch.zeros((w.batch, w.n_rings), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        plan.multislice(trans, xy, batch=w.batch, rings=rings, workspace=ws)
    torch.cuda.synchronize()
    k = max(3, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(k):
        plan.multislice(trans, xy, batch=w.batch, rings=rings, workspace=ws)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / k
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
    return {"workload": w.name, "value": w.batch / (ms / 1e3), "unit": "probes/s", "ms_per_launch": ms,
            "batch": w.batch, "grid": w.n, "slices": w.n_slices,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                         "peak_source": src, "kernel": "k_row_pass/k_col_pass<1024>"},
            "streamed": {"value": w.batch / (ms_s / 1e3), "unit": "probes/s", "ms_per_launch": ms_s,
                         "footprint_bytes": api.footprint_bytes(w, "ms_streamed", batch=w.batch),
                         "footprint_bytes_single": api.footprint_bytes(w, "ms", batch=w.batch),
                         "h2d_bytes_per_launch": w.n_slices * n2 * 8}}


def measure_serving(dev, n_requests=40, rate_hz=40.0):
    """Seeded Poisson stream of mixed multislice / PRISM requests through the
    continuous-batching server, against the same requests run one at a time."""
    import threading
    import torch
    from paper_1706_08563_b300.serve import Server, SimRequest, run_serial
    recipes = W.serving_recipes()
    atoms = {r.specimen: W.atoms(r.workload, seed=r.seed) for r in recipes}
    stream = W.serving_requests(recipes, n_requests, rate_hz)

    def make(k, xy):
        r = recipes[k]
        xyz, gauss = atoms[r.specimen]
        return SimRequest(r.specimen, r.workload, xyz, gauss, xy, r.algo, r.f, r.storage)

    reqs = [make(k, xy) for _, k, xy in stream]
    probes = sum(r.probe_xy.shape[0] for r in reqs)
    run_serial(reqs[:3], device=dev)                 # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run_serial(reqs, device=dev)
    torch.cuda.synchronize()
    t_serial = time.perf_counter() - t0
    # latency: Poisson arrivals, results as soon as their probes are done
    srv = Server(64 << 30, batch=64, prism_chunk=1024, arena=8192, device=dev)
    srv.start()
    futs = []
    t_start = time.perf_counter()

    def feeder():
        for (t_arr, k, xy), r in zip(stream, reqs):
            delay = t_start + t_arr - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            futs.append(srv.submit(r))
    th = threading.Thread(target=feeder)
    th.start()
    th.join()
    for fu in futs:
        fu.result(timeout=600)
    srv.stop()
    lat = np.array(srv.latencies) * 1e3
    # capacity: the same requests queued at once (fresh server, no resident lanes)
    burst = [make(k, xy) for _, k, xy in stream]
    srv2 = Server(64 << 30, batch=64, prism_chunk=1024, arena=8192, device=dev)
    futs2 = [srv2.submit(r) for r in burst]
    t0 = time.perf_counter()
    srv2.start()
    for fu in futs2:
        fu.result(timeout=600)
    t_burst = time.perf_counter() - t0
    srv2.stop()
    return {"requests": n_requests, "probes": probes, "arrival_rate_hz": rate_hz,
            "recipes": [f"{r.algo} N={r.workload.n} S={r.workload.n_slices}" + (f" f={r.f} {r.storage}" if r.algo == "prism" else "")
                        for r in recipes],
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "burst_probes_s": probes / t_burst, "serial_probes_s": probes / t_serial,
            "speedup_vs_serial": t_serial / t_burst, "launches_poisson": srv.launches, "launches_burst": srv2.launches,
            "what": ("p50/p99: arrival to result on the host under Poisson arrivals; burst: all requests queued at "
                     "once through the server; serial: the same requests one at a time, no overlap, no resident "
                     "potentials")}


# --------------------------------------------------------------------------- oracle
def oracle_sample(w, beams_sample=2, slices_sample=4, probes_sample=8, out_beams=16):
    """Time the FP64 oracle on a bounded sample of workload w and extrapolate to
    probes/s for the whole simulation (time is linear in beams, slices and probes)."""
    from oracle import stem as O
    xyz, gauss = W.atoms(w)
    xy = W.scan_positions(w)
    p = O.params_from(w)
    sub = O.Params(p.cell, p.n, slices_sample, p.slice_dz, p.energy_kev, p.alpha_mrad, p.ring_width_mrad,
                   p.n_rings)
    keep = xyz[:, 2] < slices_sample * p.slice_dz
    t0 = time.perf_counter()
    v = O.projected_potential(sub, xyz[keep], gauss[keep])
    t_pot = (time.perf_counter() - t0) * (p.n_slices / slices_sample)
    trans = O.transmission(sub, v)
    prism = bool(w.f)
    n = p.n
    if prism:
        f = w.f[-1]
        beams = O.prism_beams(p, f)
        t0 = time.perf_counter()
        O.prism_smatrix(sub, trans, beams[:beams_sample])
        t_s = (time.perf_counter() - t0) * (len(beams) / beams_sample) * (p.n_slices / slices_sample)
        rng = np.random.default_rng(0)
        fake = (rng.standard_normal((out_beams, n, n)) + 1j * rng.standard_normal((out_beams, n, n)))
        t0 = time.perf_counter()
        O.prism_rings(p, fake, beams[:out_beams], f, xy[:probes_sample])
        t_o = (time.perf_counter() - t0) * (len(beams) / out_beams) * (len(xy) / probes_sample)
        total = t_pot + t_s + t_o
        sample = (f"potentials of {slices_sample}/{p.n_slices} slices; S-matrix of {beams_sample}/{len(beams)} "
                  f"beams x {slices_sample}/{p.n_slices} slices; output of {probes_sample}/{len(xy)} probes with "
                  f"{out_beams}/{len(beams)} beams; extrapolated linearly")
    else:
        t0 = time.perf_counter()
        O.multislice_rings(sub, trans, xy[:probes_sample])
        t_m = (time.perf_counter() - t0) * (len(xy) / probes_sample) * (p.n_slices / slices_sample)
        total = t_pot + t_m
        sample = (f"potentials of {slices_sample}/{p.n_slices} slices; multislice of {probes_sample}/{len(xy)} "
                  f"probes x {slices_sample}/{p.n_slices} slices; extrapolated linearly")
    return len(xy) / total, sample


def run_reference(args, rank, world):
    if rank != 0:
        return None
    w = W.WORKLOADS[args.workload]
    vals = []
    sample = ""
    for i in range(args.warmup + args.steps):
        v, sample = oracle_sample(w, beams_sample=1, slices_sample=2, probes_sample=2, out_beams=8)
        if i >= args.warmup:
            vals.append(v)
    val = statistics.mean(vals)
    return {"metric": METRIC, "value": val, "unit": "probes/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * w.n_probes / val, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name},
            "cpu_baseline": {"value": val, "unit": "probes/s", "cores": 1, "kind": "oracle", "sample": sample},
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
    if rank == 0 and not args.no_cpu_baseline:
        w = W.WORKLOADS[args.workload]
        v, sample = oracle_sample(w)
        res["cpu_baseline"] = {"value": v, "unit": "probes/s", "cores": 1, "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
