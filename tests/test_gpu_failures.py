"""Failure detection without a GPU fault.

* Serving: failures are injected on the host (a malformed request, a request
  cancelled before admission, an allocation failure while a lane is created,
  an exception while a lane launches); each fails only its own request and
  the other requests still return the results they return alone.
* Bounded waits: the self-test kernel waits on a barrier that nothing arrives
  at with a 2 ms limit; the timeout must show up in the plan's status word and
  the context must stay usable.
"""
import dataclasses
import os
import time

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _requests():
    from paper_1706_08563_b300.serve import SimRequest
    specs = {
        "A": (W.Workload("A", (16.0, 16.0, 8.0), 40, 64, 4, 2.0, 200.0, 20.0, 8, 2.0, 40), "ms", 1, "f32"),
        "B": (W.Workload("B", (24.0, 24.0, 6.0), 60, 128, 3, 2.0, 300.0, 25.0, 8, 2.0, 50), "prism", 2, "f16"),
        "C": (W.Workload("C", (20.0, 20.0, 10.0), 50, 64, 5, 2.0, 80.0, 20.0, 8, 1.0, 60), "ms", 1, "f32"),
        "D": (W.Workload("D", (24.0, 24.0, 6.0), 60, 128, 3, 2.0, 300.0, 25.0, 8, 2.0, 50), "prism", 4, "f32"),
    }
    out = []
    for i, (k, (w, algo, f, st)) in enumerate(specs.items()):
        xyz, gauss = W.atoms(w, seed=300 + i)
        out.append(SimRequest(k, w, xyz, gauss, W.random_positions(w, 20 + 7 * i, seed=900 + i), algo, f, st))
    return out


def _same(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    assert a.shape == b.shape
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)


def test_malformed_requests_are_refused_and_others_complete():
    from paper_1706_08563_b300.serve import Server, ServerError, run_serial
    good = _requests()[:2]
    ref = run_serial(good)
    a, b = good
    bad = [
        dataclasses.replace(a, probe_xy=np.zeros((4, 3))),                    # wrong shape
        dataclasses.replace(a, probe_xy=np.array([[np.nan, 1.0]])),          # non-finite position
        dataclasses.replace(a, probe_xy=a.probe_xy.astype(np.float32)),      # wrong dtype
        dataclasses.replace(a, gauss=a.gauss[:-1]),                          # atom arrays disagree
        dataclasses.replace(b, algo="tomography"),                           # unknown algorithm
        dataclasses.replace(b, f=3),                                         # f not a power of two
        dataclasses.replace(b, storage="f8"),                                # unknown storage
    ]
    log = []
    with Server(4 << 30, batch=32, prism_chunk=64, arena=512, log=log.append) as srv:
        futs_good = [srv.submit(a)]
        futs_bad = [srv.submit(r) for r in bad]
        futs_good.append(srv.submit(b))
        for f in futs_bad:
            assert f.done()
            with pytest.raises(ServerError):
                f.result()
        for f, r in zip(futs_good, ref):
            _same(f.result(timeout=300), r)
        srv.drain(timeout=300)
    # one log line per request: refusals with their reason, completions with times
    assert sorted(r["status"] for r in log) == ["done"] * 2 + ["refused"] * len(bad)
    for r in log:
        if r["status"] == "done":
            assert r["latency_ms"] > 0 and r["admitted_s"] >= r["arrival_s"] and r["lane_bytes"] > 0
        else:
            assert r["error"] and r["finished_s"] is None


def test_cancelled_request_is_dropped_and_others_complete():
    from paper_1706_08563_b300.serve import Server, run_serial
    reqs = _requests()[:3]
    ref = run_serial(reqs)
    srv = Server(4 << 30, batch=32, prism_chunk=64, arena=512)
    futs = [srv.submit(r) for r in reqs]
    assert futs[1].cancel()                     # before the server has seen it
    with srv:
        _same(futs[0].result(timeout=300), ref[0])
        _same(futs[2].result(timeout=300), ref[2])
        srv.drain(timeout=300)
    assert futs[1].cancelled()


def test_lane_failures_fail_only_their_own_requests(monkeypatch):
    """An allocation failure while lane C is created and an exception while lane
    D launches: C's and D's requests fail, A's and B's complete unchanged, and
    the server keeps serving afterwards."""
    from paper_1706_08563_b300 import serve
    from paper_1706_08563_b300.serve import Server, ServerError, run_serial
    reqs = _requests()
    ref = run_serial(reqs[:2])
    real_init, real_launch = serve._Lane.__init__, serve._Lane.launch

    def init(self, key, req, *args, **kw):
        if req.specimen == "C":
            raise torch.cuda.OutOfMemoryError("injected allocation failure")
        real_init(self, key, req, *args, **kw)

    def launch(self, max_inflight):
        if self.key[0] == "D":
            raise RuntimeError("injected launch failure")
        return real_launch(self, max_inflight)

    monkeypatch.setattr(serve._Lane, "__init__", init)
    monkeypatch.setattr(serve._Lane, "launch", launch)
    with Server(4 << 30, batch=32, prism_chunk=64, arena=512) as srv:
        futs = [srv.submit(r) for r in reqs]
        _same(futs[0].result(timeout=300), ref[0])
        _same(futs[1].result(timeout=300), ref[1])
        with pytest.raises(torch.cuda.OutOfMemoryError):
            futs[2].result(timeout=300)
        with pytest.raises(ServerError):
            futs[3].result(timeout=300)
        assert not any(k[0] == "D" for k in srv.lanes)          # the failed lane is gone
        again = srv.submit(reqs[0])                              # and the server still serves
        _same(again.result(timeout=300), ref[0])


def test_bounded_wait_times_out_and_the_context_survives():
    from paper_1706_08563_b300 import _lib, api
    w = W.scaled(W.C1, n=64)
    xyz, gauss = W.atoms(w, seed=4)
    plan = api.Plan.from_workload(w)
    trans = plan.slice_potentials(torch.from_numpy(xyz).cuda(), torch.from_numpy(gauss).cuda())
    xy = torch.from_numpy(W.random_positions(w, 9, seed=5)).cuda()
    before = plan.multislice(trans, xy, batch=4).clone()
    assert plan.device_status() == 0
    t0 = time.perf_counter()
    plan.selftest_bounded_wait(2_000_000)        # 2 ms on a barrier nothing arrives at
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 5.0
    assert plan.device_status() == _lib.STEM_ERR_TIMEOUT
    assert plan.device_status() == 0             # reading clears the word
    after = plan.multislice(trans, xy, batch=4)
    torch.cuda.synchronize()
    assert torch.allclose(after, before, rtol=1e-6, atol=1e-12)
    with pytest.raises(Exception):
        plan.selftest_bounded_wait(0)


def test_smatrix_checkpoint_round_trip(repo_tmp):
    """An S-matrix saved to a file and loaded into a fresh plan gives the same
    bytes and the same output; a file for other parameters or another
    specimen is refused."""
    from paper_1706_08563_b300 import api
    w = W.Workload("ck", (24.0, 24.0, 6.0), 60, 128, 3, 2.0, 300.0, 25.0, 8, 2.0, 50)
    xyz, gauss = W.atoms(w, seed=8)
    plan = api.Plan.from_workload(w)
    trans = plan.slice_potentials(torch.from_numpy(xyz).cuda(), torch.from_numpy(gauss).cuda())
    sm = plan.prism_smatrix(trans, 4, "f16")
    xy = torch.from_numpy(W.random_positions(w, 11, seed=9)).cuda()
    ref = plan.prism_output(sm, xy, chunk=8)
    path = os.path.join(repo_tmp, "smatrix.npz")
    sm.save(path, plan, tag="specimen-8")
    fresh = api.Plan.from_workload(w)
    back = fresh.load_smatrix(path, tag="specimen-8")
    assert torch.equal(back.buf, sm.buf)
    # the ring sums use float atomics: equal up to the order of additions
    assert torch.allclose(fresh.prism_output(back, xy, chunk=8), ref, rtol=1e-6, atol=1e-12)
    with pytest.raises(ValueError):
        fresh.load_smatrix(path, tag="another specimen")
    other = api.Plan.from_workload(W.scaled(w, n_slices=4))
    with pytest.raises(ValueError):
        other.load_smatrix(path, tag="specimen-8")
