"""Continuous-batching server: every result is the same alone and in the mix.

Requests of several specimens (multislice and PRISM, different grids, slice
counts, f and scan sizes) are served one at a time and then all together
through one server, where probes of compatible requests share launches and
lanes overlap on separate streams.  Results must agree to float32 rounding
(the ring sums use float atomics, so the order of additions may differ).
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import stem as O

pytestmark = pytest.mark.gpu

MIX_TOL = 1e-5


def _requests():
    from paper_1706_08563_b300.serve import SimRequest
    specs = {
        "A": (W.Workload("A", (16.0, 16.0, 8.0), 40, 64, 4, 2.0, 200.0, 20.0, 8, 2.0, 40), "ms", 1, "f32"),
        "B": (W.Workload("B", (24.0, 24.0, 6.0), 60, 128, 3, 2.0, 300.0, 25.0, 8, 2.0, 50), "prism", 2, "f16"),
        "C": (W.Workload("C", (20.0, 20.0, 10.0), 50, 64, 5, 2.0, 80.0, 20.0, 8, 1.0, 60), "ms", 1, "f32"),
        "D": (W.Workload("D", (24.0, 24.0, 6.0), 60, 128, 3, 2.0, 300.0, 25.0, 8, 2.0, 50), "prism", 4, "f32"),
    }
    atoms = {k: W.atoms(v[0], seed=100 + i) for i, (k, v) in enumerate(specs.items())}
    reqs = []
    sizes = [37, 64, 5, 120, 1, 80, 33, 17]
    for i, size in enumerate(sizes):
        k = "ABCD"[i % 4]
        w, algo, f, st = specs[k]
        xyz, gauss = atoms[k]
        xy = W.random_positions(w, size, seed=500 + i)
        reqs.append(SimRequest(k, w, xyz, gauss, xy, algo, f, st))
    return reqs


def _close(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    assert a.shape == b.shape
    assert np.linalg.norm(a - b) <= MIX_TOL * np.linalg.norm(b)


def test_results_alone_equal_results_in_the_mix():
    from paper_1706_08563_b300.serve import Server, run_serial
    reqs = _requests()
    serial = run_serial(reqs, batch=32, prism_chunk=64)
    alone = []
    for r in reqs:
        with Server(8 << 30, batch=32, prism_chunk=64) as srv:
            alone.append(srv.submit(r).result(timeout=300))
    srv = Server(8 << 30, batch=32, prism_chunk=64, arena=512)
    futs = [srv.submit(r) for r in reqs]          # all queued before the loop starts
    srv.start()
    try:
        mixed = [f.result(timeout=300) for f in futs]
    finally:
        srv.stop()
    # probes of several requests shared launches: fewer launches than serving
    # each request on its own
    alone_launches = sum(-(-r.probe_xy.shape[0] // (64 if r.algo == "prism" else 32)) for r in reqs)
    assert srv.launches < alone_launches
    for a, m, s in zip(alone, mixed, serial):
        _close(m, a)
        _close(s, a)


def test_mix_matches_oracle_for_a_multislice_request():
    from paper_1706_08563_b300.serve import Server
    reqs = _requests()
    with Server(8 << 30, batch=32, prism_chunk=64, arena=512) as srv:
        futs = [srv.submit(r) for r in reqs]
        res = [f.result(timeout=300) for f in futs]
    r = reqs[0]
    p = O.params_from(r.workload)
    t = O.transmission(p, O.projected_potential(p, r.xyz, r.gauss))
    ref = O.multislice_rings(p, t, r.probe_xy)
    assert O.rel_l2(res[0], ref) <= 1e-4


def test_admission_by_footprint_and_eviction():
    from paper_1706_08563_b300.serve import Server, ServerError
    reqs = _requests()
    ms = [r for r in reqs if r.algo == "ms"]
    # a budget that holds one multislice lane at a time: lanes are evicted when idle
    srv = Server(1, batch=32, prism_chunk=64, arena=256)
    need = max(srv.footprint(r, 256) for r in ms)
    srv = Server(need + 1024, batch=32, prism_chunk=64, arena=256)
    with srv:
        futs = [srv.submit(r) for r in ms]
        out = [f.result(timeout=300) for f in futs]
    assert all(o.shape == (r.probe_xy.shape[0], r.workload.n_rings) for o, r in zip(out, ms))
    assert srv.used <= need + 1024
    # a request larger than the whole budget is refused, the others still run
    with Server(1 << 20, batch=32) as small:
        with pytest.raises(ServerError):
            small.submit(ms[0]).result(timeout=60)
