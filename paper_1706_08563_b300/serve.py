"""Continuous-batching request loop for STEM simulations on one GPU.

Requests (a specimen's atoms, simulation parameters and a list of probe
positions) arrive at any time.  The server keeps each specimen's transmission
functions (and, for PRISM, its compact S-matrix) resident on the device in a
*lane*.  Every lane owns a device arena of probe positions and ring outputs:
an admitted request gets a contiguous range of it, so consecutive requests of
the same lane sit side by side and one launch of the slice or beam-sum kernels
covers probes of several requests ("compatible probes batched across
requests").  Lanes run on their own CUDA streams, so work of different
specimens overlaps on the device.  New requests are admitted whenever the
device-memory budget (footprints from ``stem_footprint_bytes``, the paper's
memory estimate) and arena space allow; finished probes free arena space and
idle lanes are evicted least-recently-used when memory is needed.

Failures stay with the request that caused them: a malformed request is
refused at ``submit``, a request cancelled before admission is dropped, and
an exception while creating or running a lane fails that lane's requests
only (the lane is dropped) while the other lanes go on.

All arithmetic runs in libstem's kernels through the C ABI; this module only
schedules, moves pointers and copies results back.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import json
import threading
import time
from typing import Dict, List, Optional

import numpy as np
import torch

from . import _lib
from .api import Plan, SMatrix, _ptr


@dataclasses.dataclass
class SimRequest:
    """One simulation request.  Requests with the same ``specimen`` key must carry
    the same atoms; they then share the resident potentials / S-matrix."""
    specimen: str
    workload: object            # workloads.Workload: cell, grid, slices, optics, detector
    xyz: np.ndarray             # float64 [n, 3]
    gauss: np.ndarray           # float32 [n, 4]
    probe_xy: np.ndarray        # float64 [P, 2]
    algo: str = "ms"            # "ms" or "prism"
    f: int = 1
    storage: str = "f32"
    arrival: float = 0.0        # filled by submit
    admitted: float = 0.0
    finished: float = 0.0


class ServerError(RuntimeError):
    pass


@dataclasses.dataclass
class _Active:
    req: SimRequest
    fut: cf.Future
    lane: "_Lane"
    start: int
    count: int
    host: Optional[torch.Tensor] = None
    event: Optional[torch.cuda.Event] = None


class _Lane:
    """Resident state of one (specimen, parameters, algorithm) combination."""

    def __init__(self, key, req: SimRequest, device, capacity: int, batch: int, chunk: int):
        w = req.workload
        self.key = key
        self.device = device
        self.algo = req.algo
        self.f = req.f
        self.storage = req.storage
        self.capacity = capacity
        self.batch = batch
        self.chunk = chunk
        self.stream = torch.cuda.Stream(device=device)
        self.n_rings = w.n_rings
        self.last_used = time.perf_counter()
        with torch.cuda.stream(self.stream):
            self.plan = Plan.from_workload(w, device=device)
            self.trans = self.plan.slice_potentials(torch.from_numpy(req.xyz).to(device, non_blocking=True),
                                                    torch.from_numpy(req.gauss).to(device, non_blocking=True))
            self.smat: Optional[SMatrix] = None
            if self.algo == "prism":
                self.smat = self.plan.prism_smatrix(self.trans, self.f, self.storage, batch=min(batch, 128))
                self.ws = self.plan.prism_output_workspace(self.f, chunk)
            else:
                self.ws = self.plan.multislice_workspace(batch)
            self.xy = torch.empty((capacity, 2), dtype=torch.float64, device=device)
            self.rings = torch.zeros((capacity, self.n_rings), dtype=torch.float32, device=device)
        self.filled = 0       # arena slots handed to requests
        self.launched = 0     # slots whose kernels are enqueued
        self.done = 0         # slots whose kernels have completed
        self.inflight: collections.deque = collections.deque()   # (event, end)
        self.requests: List[_Active] = []

    def idle(self) -> bool:
        return not self.requests and not self.inflight

    def room(self) -> int:
        return self.capacity - self.filled

    def reset_if_empty(self):
        if not self.requests and not self.inflight and self.launched == self.filled:
            self.filled = self.launched = self.done = 0

    def enqueue(self, act: _Active, xy: np.ndarray):
        with torch.cuda.stream(self.stream):
            self.xy[act.start:act.start + act.count].copy_(torch.from_numpy(xy), non_blocking=True)
            self.rings[act.start:act.start + act.count].zero_()

    def launch(self, max_inflight: int) -> int:
        """Enqueue kernels for the next batch of queued probes (any requests)."""
        n = 0
        while self.launched < self.filled and len(self.inflight) < max_inflight:
            step = self.chunk if self.algo == "prism" else self.batch
            a, b = self.launched, min(self.filled, self.launched + step)
            with torch.cuda.stream(self.stream):
                xy = self.xy[a:b]
                rings = self.rings[a:b]
                if self.algo == "prism":
                    self.plan.prism_output(self.smat, xy, chunk=b - a, rings=rings, workspace=self.ws)
                else:
                    self.plan.multislice(self.trans, xy, batch=b - a, rings=rings, workspace=self.ws)
                ev = torch.cuda.Event()
                ev.record(self.stream)
            self.inflight.append((ev, b))
            self.launched = b
            n += 1
        return n

    def poll(self):
        while self.inflight and self.inflight[0][0].query():
            _, end = self.inflight.popleft()
            self.done = end


class Server:
    """Continuous-batching STEM server on one CUDA device.

    ``submit`` returns a Future resolving to a float32 [P, n_rings] array.
    ``max_bytes`` bounds the device memory of resident lanes (footprint of the
    transmission stack, S-matrix, workspaces and arenas).
    """

    def __init__(self, max_bytes: int, batch: int = 64, prism_chunk: int = 1024, arena: int = 16384,
                 max_inflight: int = 2, device=None, log=None):
        self.lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.max_bytes = int(max_bytes)
        self.batch = batch
        self.prism_chunk = prism_chunk
        self.arena = arena
        self.max_inflight = max_inflight
        self.lanes: Dict[tuple, _Lane] = {}
        self.lane_bytes: Dict[tuple, int] = {}
        self.used = 0
        self._in: "collections.deque" = collections.deque()
        self._lock = threading.Lock()
        self._pending: List[tuple] = []
        self._active: List[_Active] = []
        self._stop = threading.Event()
        self._thread: Optional[threading.Thread] = None
        self.latencies: List[float] = []
        self.launches = 0
        self.copy_stream = torch.cuda.Stream(device=self.device)
        # per-request log: a path (JSON lines appended) or a callable taking a dict
        self._log = log
        self._t0 = time.perf_counter()

    # ------------------------------------------------------------------ API
    def _record(self, req: SimRequest, status: str, lane_bytes: int = 0, error: str = ""):
        """One log line per request: what it was, when it arrived, was admitted
        and finished (seconds since the server was created), and its outcome."""
        if self._log is None:
            return
        rec = dict(specimen=req.specimen, algo=req.algo, f=req.f if req.algo == "prism" else 1,
                   storage=req.storage if req.algo == "prism" else "f32",
                   probes=int(getattr(req.probe_xy, "shape", (0,))[0]), status=status,
                   arrival_s=req.arrival - self._t0,
                   admitted_s=(req.admitted - self._t0) if req.admitted else None,
                   finished_s=(req.finished - self._t0) if req.finished else None,
                   latency_ms=1e3 * (req.finished - req.arrival) if req.finished else None,
                   lane_bytes=int(lane_bytes), error=error)
        if callable(self._log):
            self._log(rec)
        else:
            with open(self._log, "a") as fh:
                fh.write(json.dumps(rec) + "\n")

    @staticmethod
    def validate(req: SimRequest) -> Optional[str]:
        """Why the request cannot be served, or None."""
        def arr(x, dt, cols):
            return isinstance(x, np.ndarray) and x.dtype == dt and x.ndim == 2 and x.shape[1] == cols
        if not arr(req.probe_xy, np.float64, 2):
            return "probe_xy must be a float64 array [P, 2]"
        if not np.all(np.isfinite(req.probe_xy)):
            return "probe_xy holds non-finite positions"
        if not arr(req.xyz, np.float64, 3) or not arr(req.gauss, np.float32, 4):
            return "atoms must be float64 xyz [n, 3] and float32 gauss [n, 4]"
        if req.xyz.shape[0] != req.gauss.shape[0]:
            return "xyz and gauss describe different numbers of atoms"
        if not (np.all(np.isfinite(req.xyz)) and np.all(np.isfinite(req.gauss))):
            return "atoms hold non-finite values"
        if req.algo not in ("ms", "prism"):
            return f"unknown algorithm {req.algo!r}"
        if req.algo == "prism":
            from ._lib import STORAGE
            if not (isinstance(req.f, int) and req.f >= 1 and req.f & (req.f - 1) == 0):
                return "f must be a power of two"
            if req.storage not in STORAGE:
                return f"unknown storage {req.storage!r}"
        return None

    def submit(self, req: SimRequest) -> cf.Future:
        """Queue a request; the Future resolves to float32 [P, n_rings] rings,
        or raises ServerError.  Cancelling it before it is admitted drops it."""
        fut: cf.Future = cf.Future()
        req.arrival = time.perf_counter()
        why = self.validate(req)
        if why is not None:
            fut.set_exception(ServerError(why))
            self._record(req, "refused", error=why)
            return fut
        with self._lock:
            self._in.append((req, fut))
        return fut

    def start(self):
        self._thread = threading.Thread(target=self._loop, name="stem-server", daemon=True)
        self._thread.start()
        return self

    def stop(self):
        self._stop.set()
        if self._thread:
            self._thread.join()

    def __enter__(self):
        return self.start()

    def __exit__(self, *exc):
        self.stop()

    # ------------------------------------------------------------- internals
    @staticmethod
    def lane_key(req: SimRequest) -> tuple:
        w = req.workload
        return (req.specimen, tuple(w.cell), w.n, w.n_slices, w.slice_dz, w.energy_kev, w.alpha_mrad,
                w.ring_width_mrad, w.n_rings, getattr(w, "defocus", 0.0), getattr(w, "cs", 0.0), req.algo, req.f if req.algo == "prism" else 1,
                req.storage if req.algo == "prism" else "f32")

    def footprint(self, req: SimRequest, capacity: int) -> int:
        from ._lib import STORAGE, StemParams
        import ctypes
        w = req.workload
        p = StemParams((ctypes.c_double * 3)(*[float(c) for c in w.cell]), int(w.n), int(w.n_slices),
                       float(w.slice_dz), float(w.energy_kev), float(w.alpha_mrad), float(w.ring_width_mrad),
                       int(w.n_rings))
        algo = 0 if req.algo == "ms" else 1
        b = self.lib.stem_footprint_bytes(ctypes.byref(p), algo, req.f if algo else 1,
                                          STORAGE[req.storage] if algo else 0, capacity,
                                          self.batch if algo == 0 else min(self.batch, 128))
        return int(b) + capacity * 16

    def _admit(self, req: SimRequest, fut: cf.Future) -> bool:
        if fut.cancelled():
            return True
        key = self.lane_key(req)
        n = int(req.probe_xy.shape[0])
        lane = self.lanes.get(key)
        if lane is None:
            cap = max(self.arena, n)
            need = self.footprint(req, cap)
            if need == 0:
                fut.set_exception(ServerError("unsupported request parameters"))
                self._record(req, "refused", error="unsupported request parameters")
                return True
            if need > self.max_bytes:
                why = f"request needs {need} bytes, more than the budget {self.max_bytes}"
                fut.set_exception(ServerError(why))
                self._record(req, "refused", error=why)
                return True
            while self.used + need > self.max_bytes:
                if not self._evict_one():
                    return False
            lane = _Lane(key, req, self.device, cap, self.batch, self.prism_chunk)
            self.lanes[key] = lane
            self.lane_bytes[key] = need
            self.used += need
        lane.reset_if_empty()
        if lane.room() < n:
            return False
        if not fut.set_running_or_notify_cancel():
            return True
        act = _Active(req, fut, lane, lane.filled, n)
        lane.filled += n
        lane.enqueue(act, req.probe_xy)
        lane.requests.append(act)
        lane.last_used = time.perf_counter()
        req.admitted = time.perf_counter()
        return True

    def _drop_lane(self, key):
        lane = self.lanes.pop(key)
        lane.plan.close()
        self.used -= self.lane_bytes.pop(key)

    def _evict_one(self) -> bool:
        idle = [k for k, l in self.lanes.items() if l.idle()]
        if not idle:
            return False
        self._drop_lane(min(idle, key=lambda k: self.lanes[k].last_used))
        return True

    def _fail_lane(self, key, err: Exception):
        """A lane whose launch or copy-back raised: fail its requests, drop it.
        Its stream is synchronised first so that nothing it queued is still
        running when its buffers are released."""
        lane = self.lanes[key]
        try:
            lane.stream.synchronize()
        except Exception:
            pass
        for act in lane.requests:
            if not act.fut.done():
                act.fut.set_exception(ServerError(f"lane failed: {err!r}"))
                self._record(act.req, "failed", self.lane_bytes.get(key, 0), repr(err))
        lane.requests = []
        lane.inflight.clear()
        self._drop_lane(key)

    def _finish(self, lane: _Lane):
        keep = []
        for act in lane.requests:
            if act.host is None and lane.done >= act.start + act.count:
                # the kernels covering this range have completed (their event was
                # observed), so the copy-back does not queue behind later batches
                with torch.cuda.stream(self.copy_stream):
                    act.host = torch.empty((act.count, lane.n_rings), dtype=torch.float32).pin_memory()
                    act.host.copy_(lane.rings[act.start:act.start + act.count], non_blocking=True)
                    act.event = torch.cuda.Event()
                    act.event.record(self.copy_stream)
            if act.event is not None and act.event.query():
                act.req.finished = time.perf_counter()
                self.latencies.append(act.req.finished - act.req.arrival)
                act.fut.set_result(act.host.numpy().copy())
                self._record(act.req, "done", self.lane_bytes.get(lane.key, 0))
                continue
            keep.append(act)
        lane.requests = keep

    def step(self) -> bool:
        """One scheduling pass; returns True if anything happened."""
        busy = False
        with self._lock:
            while self._in:
                self._pending.append(self._in.popleft())
        still = []
        for req, fut in self._pending:
            try:
                ok = self._admit(req, fut)
            except Exception as e:     # a failing request must not stop the others
                fut.set_exception(e)
                self._record(req, "failed", error=repr(e))
                ok = True
            if ok:
                busy = True
            else:
                still.append((req, fut))
        self._pending = still
        for key, lane in list(self.lanes.items()):
            try:
                lane.poll()
                n = lane.launch(self.max_inflight)
                self.launches += n
                busy |= n > 0
                before = len(lane.requests)
                self._finish(lane)
                busy |= len(lane.requests) != before
            except Exception as e:     # this lane's failure must not stop the others
                self._fail_lane(key, e)
                busy = True
        return busy

    def _loop(self):
        torch.cuda.set_device(self.device)
        while not self._stop.is_set():
            if not self.step():
                time.sleep(0.0005)

    def pending(self) -> int:
        with self._lock:
            n = len(self._in)
        return n + len(self._pending) + sum(len(l.requests) for l in self.lanes.values())

    def drain(self, timeout: float = 600.0):
        t0 = time.perf_counter()
        while self.pending():
            if time.perf_counter() - t0 > timeout:
                raise TimeoutError("server did not drain")
            time.sleep(0.001)


def run_serial(reqs: List[SimRequest], device=None, batch: int = 64, prism_chunk: int = 1024) -> List[np.ndarray]:
    """The same requests one at a time, no overlap (the comparison point)."""
    out = []
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index or 0)
    for r in reqs:
        plan = Plan.from_workload(r.workload, device=dev)
        t = plan.slice_potentials(torch.from_numpy(r.xyz).to(dev), torch.from_numpy(r.gauss).to(dev))
        xy = torch.from_numpy(r.probe_xy).to(dev)
        if r.algo == "prism":
            sm = plan.prism_smatrix(t, r.f, r.storage, batch=min(batch, 128))
            rings = plan.prism_output(sm, xy, chunk=prism_chunk)
        else:
            rings = plan.multislice(t, xy, batch=batch)
        out.append(rings.cpu().numpy())
        plan.close()
    return out
