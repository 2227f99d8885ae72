"""PyTorch-facing binding of libstem (argument marshalling only).

Every computation runs in libstem's CUDA kernels; this module checks tensor
devices, dtypes and shapes, allocates outputs and workspaces with PyTorch (the
device-memory provider) and passes raw pointers plus the current CUDA stream
through the C ABI.
"""
from __future__ import annotations

import ctypes
import json
from dataclasses import dataclass
from typing import Optional, Tuple

import numpy as np
import torch

from . import _lib
from ._lib import ENGINE, STEM_CROPPED, STORAGE, StemParams, check


def _stream(device: torch.device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _need(t: torch.Tensor, dtype: torch.dtype, name: str, shape=None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.contiguous()


def _need_host(t: torch.Tensor, dtype: torch.dtype, name: str, shape=None) -> torch.Tensor:
    """A host tensor for the streaming memory model (page-locked memory lets the
    copies overlap the passes; a pageable tensor works, slower)."""
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise ValueError(f"{name} must be a host (CPU) tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.contiguous()


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


@dataclass
class SMatrix:
    """A compact S-matrix buffer filled by ``Plan.prism_smatrix``."""
    buf: torch.Tensor          # uint8, stem_prism_smatrix_bytes
    f: int
    storage: str
    n_beams: int
    nbp: int
    data_offset: int
    n: int                     # side of the grid it is stored on (N, or 3N/4 when cropped)
    cropped: bool = False

    @property
    def code(self) -> int:
        """The storage code of the C ABI (element type, with STEM_CROPPED when cropped)."""
        return STORAGE[self.storage] | (STEM_CROPPED if self.cropped else 0)

    def scales(self) -> torch.Tensor:
        return self.buf[: 4 * self.nbp].view(torch.float32)

    def data(self) -> torch.Tensor:
        """[n, n, 2, nbp] view of the stored values (S_b / s_b)."""
        dt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[self.storage]
        esz = 4 if self.storage == "f32" else 2
        raw = self.buf[self.data_offset: self.data_offset + self.n * self.n * 2 * self.nbp * esz]
        return raw.view(dt).view(self.n, self.n, 2, self.nbp)

    def beams_real_space(self) -> torch.Tensor:
        """S_b(y, x) as complex64 [n_beams, n, n] (scaled back)."""
        d = self.data().float() * self.scales()[None, None, None, :]
        c = torch.complex(d[:, :, 0, :], d[:, :, 1, :])
        return c.permute(2, 0, 1)[: self.n_beams].contiguous()

    def crop(self, rows, cols) -> np.ndarray:
        """S_b(y, x) over the given rows and columns, copied to the host as
        complex128 [n_beams, len(rows), len(cols)] (stored values times s_b).
        An inspection accessor: it reads one window at a time, for checks of
        the output step against an independent implementation, without
        holding the whole S-matrix on the host."""
        d = self.data()
        r = torch.as_tensor(np.asarray(rows, dtype=np.int64), device=d.device)
        c = torch.as_tensor(np.asarray(cols, dtype=np.int64), device=d.device)
        sub = d.index_select(0, r).index_select(1, c)[..., : self.n_beams].double()
        sub = sub * self.scales()[: self.n_beams].double()[None, None, None, :]
        return torch.complex(sub[:, :, 0, :], sub[:, :, 1, :]).permute(2, 0, 1).contiguous().cpu().numpy()

    def save(self, path: str, plan: "Plan", tag: str = "") -> None:
        """Checkpoint the S-matrix to a file (.npz): the raw buffer plus the plan
        parameters it depends on, so that ``Plan.load_smatrix`` can refuse a
        mismatched plan.  ``tag`` names the specimen (the plan does not know
        the atoms); loading with a different tag is refused too."""
        meta = dict(version=SMATRIX_FILE_VERSION, f=self.f, storage=self.storage, n_beams=self.n_beams,
                    nbp=self.nbp, data_offset=self.data_offset, n=self.n, cropped=self.cropped,
                    plan=plan.smatrix_key(), tag=tag)
        np.savez(path, buf=self.buf.cpu().numpy(), meta=np.array(json.dumps(meta)))


SMATRIX_FILE_VERSION = 1


class Plan:
    """A stem_plan: grid, optics and detector tables on the current CUDA device."""

    def __init__(self, cell, n, n_slices, slice_dz, energy_kev, alpha_mrad, ring_width_mrad, n_rings,
                 device=None, defocus=0.0, cs=0.0):
        lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.params = StemParams((ctypes.c_double * 3)(*[float(c) for c in cell]), int(n), int(n_slices),
                                 float(slice_dz), float(energy_kev), float(alpha_mrad),
                                 float(ring_width_mrad), int(n_rings), float(defocus), float(cs))
        handle = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(lib.stem_plan_create(ctypes.byref(self.params), ctypes.byref(handle)), "stem_plan_create")
        self._h = handle
        self.n = int(n)
        self.n_slices = int(n_slices)
        self.n_rings = int(n_rings)
        lam, sig, nap = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
        check(lib.stem_plan_constants(self._h, ctypes.byref(lam), ctypes.byref(sig), ctypes.byref(nap)),
              "stem_plan_constants")
        self.lam, self.sigma, self.n_aperture = lam.value, sig.value, nap.value

    @classmethod
    def from_workload(cls, w, device=None) -> "Plan":
        return cls(w.cell, w.n, w.n_slices, w.slice_dz, w.energy_kev, w.alpha_mrad, w.ring_width_mrad,
                   w.n_rings, device=device, defocus=getattr(w, "defocus", 0.0), cs=getattr(w, "cs", 0.0))

    def device_status(self) -> int:
        """Read and clear the plan's device status word (0, or STEM_ERR_TIMEOUT
        after a bounded wait gave up); synchronous."""
        code = ctypes.c_int32()
        check(_lib.load().stem_plan_device_status(self._h, ctypes.byref(code)), "stem_plan_device_status")
        return int(code.value)

    def selftest_bounded_wait(self, limit_ns: int) -> None:
        """Launch the bounded-wait self-test on the current stream."""
        check(_lib.load().stem_selftest_bounded_wait(self._h, int(limit_ns), _stream(self.device)),
              "stem_selftest_bounded_wait")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.load().stem_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ potentials
    def potentials_workspace(self, n_atoms: int) -> torch.Tensor:
        return _workspace(_lib.load().stem_slice_potentials_workspace(self._h, n_atoms), self.device)

    def slice_potentials(self, xyz: torch.Tensor, gauss: torch.Tensor, want_v: bool = False,
                         out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None):
        """t_n = exp(i sigma V_n) as complex64 [S, N, N] (and V_n float32 if want_v)."""
        lib = _lib.load()
        xyz = _need(xyz, torch.float64, "xyz")
        gauss = _need(gauss, torch.float32, "gauss")
        na = xyz.shape[0]
        if xyz.shape != (na, 3) or gauss.shape != (na, 4):
            raise ValueError("xyz must be [n,3] and gauss [n,4]")
        shape = (self.n_slices, self.n, self.n)
        trans = out if out is not None else torch.empty(shape, dtype=torch.complex64, device=self.device)
        trans = _need(trans, torch.complex64, "out", shape)
        v = torch.empty(shape, dtype=torch.float32, device=self.device) if want_v else None
        ws = workspace if workspace is not None else self.potentials_workspace(na)
        check(lib.stem_slice_potentials(self._h, _ptr(xyz), _ptr(gauss), na, _ptr(v), _ptr(trans), _ptr(ws),
                                        ws.numel(), _stream(self.device)), "stem_slice_potentials")
        return (trans, v) if want_v else trans

    # ------------------------------------------------------------------ multislice
    def multislice_workspace(self, batch: int) -> torch.Tensor:
        return _workspace(_lib.load().stem_multislice_workspace(self._h, batch), self.device)

    def multislice(self, trans: torch.Tensor, probe_xy: torch.Tensor, batch: int = 256,
                   rings: Optional[torch.Tensor] = None, weight: float = 1.0,
                   workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
        lib = _lib.load()
        trans = _need(trans, torch.complex64, "trans", (self.n_slices, self.n, self.n))
        probe_xy = _need(probe_xy, torch.float64, "probe_xy")
        npr = probe_xy.shape[0]
        if rings is None:
            rings = torch.zeros((npr, self.n_rings), dtype=torch.float32, device=self.device)
        else:
            rings = _need(rings, torch.float32, "rings", (npr, self.n_rings))
        batch = int(max(1, min(batch, max(npr, 1))))
        ws = workspace if workspace is not None else self.multislice_workspace(batch)
        check(lib.stem_multislice_scan(self._h, _ptr(trans), _ptr(probe_xy), npr, batch, float(weight),
                                       _ptr(rings), _ptr(ws), ws.numel(), _stream(self.device)),
              "stem_multislice_scan")
        return rings

    def multislice_streamed(self, trans_host: torch.Tensor, probe_xy: torch.Tensor, batch: int = 256,
                            rings: Optional[torch.Tensor] = None, weight: float = 1.0,
                            workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Multislice under the streaming memory model: the transmission stack
        stays in host memory (pin it for overlap) and three slice buffers cycle
        on the device.  The host tensor must not change until the call's work
        on the current stream has finished."""
        lib = _lib.load()
        trans_host = _need_host(trans_host, torch.complex64, "trans_host", (self.n_slices, self.n, self.n))
        probe_xy = _need(probe_xy, torch.float64, "probe_xy")
        npr = probe_xy.shape[0]
        if rings is None:
            rings = torch.zeros((npr, self.n_rings), dtype=torch.float32, device=self.device)
        else:
            rings = _need(rings, torch.float32, "rings", (npr, self.n_rings))
        batch = int(max(1, min(batch, max(npr, 1))))
        ws = workspace if workspace is not None else _workspace(
            lib.stem_multislice_streamed_workspace(self._h, batch), self.device)
        check(lib.stem_multislice_scan_streamed(self._h, trans_host.data_ptr(), _ptr(probe_xy), npr, batch,
                                                float(weight), _ptr(rings), _ptr(ws), ws.numel(),
                                                _stream(self.device)), "stem_multislice_scan_streamed")
        return rings

    def multislice_4d(self, trans: torch.Tensor, probe_xy: torch.Tensor, batch: int = 64,
                      dp: Optional[torch.Tensor] = None, weight: float = 1.0,
                      workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Whole diffraction pattern per probe, float32 [P, N, N] in FFT order."""
        lib = _lib.load()
        trans = _need(trans, torch.complex64, "trans", (self.n_slices, self.n, self.n))
        probe_xy = _need(probe_xy, torch.float64, "probe_xy")
        npr = probe_xy.shape[0]
        if dp is None:
            dp = torch.zeros((npr, self.n, self.n), dtype=torch.float32, device=self.device)
        else:
            dp = _need(dp, torch.float32, "dp", (npr, self.n, self.n))
        batch = int(max(1, min(batch, max(npr, 1))))
        ws = workspace if workspace is not None else self.multislice_workspace(batch)
        check(lib.stem_multislice_scan_4d(self._h, _ptr(trans), _ptr(probe_xy), npr, batch, float(weight), _ptr(dp),
                                          _ptr(ws), ws.numel(), _stream(self.device)), "stem_multislice_scan_4d")
        return dp

    def set_detector_edges(self, edges_mrad) -> None:
        """Annular detectors [edges[i], edges[i+1]) in mrad instead of uniform rings."""
        lib = _lib.load()
        e = np.ascontiguousarray(np.asarray(edges_mrad, dtype=np.float64))
        check(lib.stem_plan_set_detector_edges(self._h, len(e), e.ctypes.data_as(ctypes.c_void_p)),
              "stem_plan_set_detector_edges")
        self.n_rings = len(e) - 1

    # ------------------------------------------------------------------ PRISM
    def prism_beams(self, f: int) -> np.ndarray:
        lib = _lib.load()
        nb = ctypes.c_int32()
        check(lib.stem_prism_beams(self._h, f, ctypes.byref(nb), None), "stem_prism_beams")
        out = np.zeros((nb.value, 2), dtype=np.int32)
        check(lib.stem_prism_beams(self._h, f, ctypes.byref(nb), out.ctypes.data_as(ctypes.c_void_p)),
              "stem_prism_beams")
        return out

    def prism_smatrix(self, trans: torch.Tensor, f: int, storage: str = "f32", batch: int = 128,
                      workspace: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
                      beams: Optional[Tuple[int, int]] = None, cropped: bool = False) -> SMatrix:
        """The compact S-matrix; with beams=(b0, b1) only beams [b0, b1) are
        built into a zeroed buffer (a buffer passed as `out` must be zeroed by
        the caller), so that buffers of disjoint ranges sum to the whole.
        cropped: store it Fourier-cropped on the 3N/4 grid."""
        lib = _lib.load()
        trans = _need(trans, torch.complex64, "trans", (self.n_slices, self.n, self.n))
        st = STORAGE[storage] | (STEM_CROPPED if cropped else 0)
        nbytes = lib.stem_prism_smatrix_bytes(self._h, f, st)
        if nbytes == 0:
            raise ValueError(f"unsupported f={f} or storage={storage}")
        nb = len(self.prism_beams(f))
        batch = int(max(1, min(batch, nb)))
        alloc = torch.zeros if beams is not None else torch.empty
        buf = out if out is not None else alloc(nbytes, dtype=torch.uint8, device=self.device)
        ws = workspace if workspace is not None else _workspace(
            lib.stem_prism_smatrix_workspace(self._h, batch), self.device)
        if beams is None:
            check(lib.stem_prism_smatrix(self._h, _ptr(trans), f, st, batch, _ptr(buf), buf.numel(), _ptr(ws),
                                         ws.numel(), _stream(self.device)), "stem_prism_smatrix")
        else:
            check(lib.stem_prism_smatrix_range(self._h, _ptr(trans), f, st, batch, int(beams[0]), int(beams[1]),
                                               _ptr(buf), buf.numel(), _ptr(ws), ws.numel(), _stream(self.device)),
                  "stem_prism_smatrix_range")
        nbp = (nb + 63) // 64 * 64
        return SMatrix(buf, f, storage, nb, nbp, (nbp * 4 + 255) // 256 * 256,
                       3 * self.n // 4 if cropped else self.n, cropped)

    def prism_smatrix_view(self, buf: torch.Tensor, f: int, storage: str, cropped: bool = False) -> SMatrix:
        """An S-matrix handle on an existing buffer (e.g. one assembled from
        beam ranges built on several devices)."""
        lib = _lib.load()
        if buf.numel() < lib.stem_prism_smatrix_bytes(self._h, f, STORAGE[storage] | (STEM_CROPPED if cropped else 0)):
            raise ValueError("buffer smaller than the S-matrix")
        nb = len(self.prism_beams(f))
        nbp = (nb + 63) // 64 * 64
        return SMatrix(buf, f, storage, nb, nbp, (nbp * 4 + 255) // 256 * 256,
                       3 * self.n // 4 if cropped else self.n, cropped)

    def prism_smatrix_streamed(self, trans_host: torch.Tensor, f: int, storage: str = "f32", batch: int = 128,
                               workspace: Optional[torch.Tensor] = None,
                               out: Optional[torch.Tensor] = None) -> SMatrix:
        """The S-matrix built with the transmission stack streamed from host memory."""
        lib = _lib.load()
        trans_host = _need_host(trans_host, torch.complex64, "trans_host", (self.n_slices, self.n, self.n))
        st = STORAGE[storage]
        nbytes = lib.stem_prism_smatrix_bytes(self._h, f, st)
        if nbytes == 0:
            raise ValueError(f"unsupported f={f} or storage={storage}")
        nb = len(self.prism_beams(f))
        batch = int(max(1, min(batch, nb)))
        buf = out if out is not None else torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        ws = workspace if workspace is not None else _workspace(
            lib.stem_prism_smatrix_streamed_workspace(self._h, batch), self.device)
        check(lib.stem_prism_smatrix_streamed(self._h, trans_host.data_ptr(), f, st, batch, _ptr(buf), buf.numel(),
                                              _ptr(ws), ws.numel(), _stream(self.device)),
              "stem_prism_smatrix_streamed")
        nbp = (nb + 63) // 64 * 64
        return SMatrix(buf, f, storage, nb, nbp, (nbp * 4 + 255) // 256 * 256, self.n)

    def smatrix_key(self) -> dict:
        """The plan parameters an S-matrix depends on (grid, slices, optics)."""
        p = self.params
        return dict(cell=[float(c) for c in p.cell], n=int(p.n), n_slices=int(p.n_slices),
                    slice_dz=float(p.slice_dz), energy_kev=float(p.energy_kev), alpha_mrad=float(p.alpha_mrad),
                    defocus=float(p.defocus_a), cs=float(p.cs_a))

    def load_smatrix(self, path: str, tag: str = "") -> SMatrix:
        """Resume from ``SMatrix.save``: checks the file against this plan and
        the tag, then uploads the buffer to this plan's device."""
        with np.load(path, allow_pickle=False) as z:
            meta = json.loads(str(z["meta"]))
            raw = z["buf"]
        if meta.get("version") != SMATRIX_FILE_VERSION:
            raise ValueError(f"{path}: unknown S-matrix file version {meta.get('version')}")
        if meta["plan"] != self.smatrix_key():
            raise ValueError(f"{path}: S-matrix was computed for other plan parameters")
        if meta["tag"] != tag:
            raise ValueError(f"{path}: S-matrix belongs to specimen {meta['tag']!r}, not {tag!r}")
        lib = _lib.load()
        cropped = bool(meta.get("cropped", False))
        nbytes = lib.stem_prism_smatrix_bytes(self._h, meta["f"],
                                              STORAGE[meta["storage"]] | (STEM_CROPPED if cropped else 0))
        nb = len(self.prism_beams(meta["f"]))
        if raw.dtype != np.uint8 or raw.size != nbytes or nb != meta["n_beams"]:
            raise ValueError(f"{path}: buffer size or beam count does not match this plan")
        buf = torch.from_numpy(raw).to(self.device)
        return SMatrix(buf, meta["f"], meta["storage"], meta["n_beams"], meta["nbp"], meta["data_offset"],
                       meta["n"], cropped)

    def prism_output_workspace(self, f: int, chunk: int) -> torch.Tensor:
        return _workspace(_lib.load().stem_prism_output_workspace(self._h, f, chunk), self.device)

    def prism_output(self, smat: SMatrix, probe_xy: torch.Tensor, chunk: int = 4096, engine: str = "auto",
                     rings: Optional[torch.Tensor] = None, weight: float = 1.0,
                     workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
        lib = _lib.load()
        probe_xy = _need(probe_xy, torch.float64, "probe_xy")
        npr = probe_xy.shape[0]
        if rings is None:
            rings = torch.zeros((npr, self.n_rings), dtype=torch.float32, device=self.device)
        else:
            rings = _need(rings, torch.float32, "rings", (npr, self.n_rings))
        chunk = int(max(1, min(chunk, max(npr, 1), 65535)))
        ws = workspace if workspace is not None else self.prism_output_workspace(smat.f, chunk)
        check(lib.stem_prism_output(self._h, smat.f, smat.code, ENGINE[engine], _ptr(smat.buf),
                                    _ptr(probe_xy), npr, chunk, float(weight), _ptr(rings), _ptr(ws), ws.numel(),
                                    _stream(self.device)), "stem_prism_output")
        return rings

    def prism_output_4d(self, smat: SMatrix, probe_xy: torch.Tensor, chunk: int = 1024, engine: str = "auto",
                        dp: Optional[torch.Tensor] = None, weight: float = 1.0) -> torch.Tensor:
        """PRISM diffraction patterns on the window grid, float32 [P, W, W] (FFT order, / W^4)."""
        lib = _lib.load()
        probe_xy = _need(probe_xy, torch.float64, "probe_xy")
        npr = probe_xy.shape[0]
        w = smat.n // smat.f
        if dp is None:
            dp = torch.zeros((npr, w, w), dtype=torch.float32, device=self.device)
        chunk = int(max(1, min(chunk, max(npr, 1), 65535)))
        ws = self.prism_output_workspace(smat.f, chunk)
        check(lib.stem_prism_output_4d(self._h, smat.f, smat.code, ENGINE[engine], _ptr(smat.buf),
                                       _ptr(probe_xy), npr, chunk, float(weight), _ptr(dp), _ptr(ws), ws.numel(),
                                       _stream(self.device)), "stem_prism_output_4d")
        return dp

    def prism_windows(self, smat: SMatrix, probe_xy: torch.Tensor, engine: str = "auto") -> torch.Tensor:
        lib = _lib.load()
        probe_xy = _need(probe_xy, torch.float64, "probe_xy")
        npr = probe_xy.shape[0]
        w = smat.n // smat.f
        out = torch.empty((npr, w, w), dtype=torch.complex64, device=self.device)
        ws = self.prism_output_workspace(smat.f, max(npr, 1))
        check(lib.stem_prism_windows(self._h, smat.f, smat.code, ENGINE[engine], _ptr(smat.buf),
                                     _ptr(probe_xy), npr, _ptr(out), _ptr(ws), ws.numel(), _stream(self.device)),
              "stem_prism_windows")
        return out

    # ------------------------------------------------------------------ detector
    def detector_readout(self, psi_k: torch.Tensor, f: int = 1, scale: float = 1.0,
                         rings: Optional[torch.Tensor] = None) -> torch.Tensor:
        lib = _lib.load()
        w = self.n // f
        psi_k = _need(psi_k, torch.complex64, "psi_k")
        if psi_k.dim() != 3 or psi_k.shape[1:] != (w, w):
            raise ValueError(f"psi_k must be [batch, {w}, {w}]")
        b = psi_k.shape[0]
        if rings is None:
            rings = torch.zeros((b, self.n_rings), dtype=torch.float32, device=self.device)
        check(lib.stem_detector_readout(self._h, f, _ptr(psi_k), b, float(scale), _ptr(rings), _stream(self.device)),
              "stem_detector_readout")
        return rings


def fft2(x: torch.Tensor, inverse: bool = False) -> torch.Tensor:
    """Batched 2D FFT of complex64 [batch, n, n] with libstem's kernels (unnormalised)."""
    lib = _lib.load()
    x = _need(x, torch.complex64, "x").clone()
    if x.dim() != 3 or x.shape[1] != x.shape[2]:
        raise ValueError("x must be [batch, n, n]")
    check(lib.stem_fft2(x.shape[1], x.shape[0], 1 if inverse else 0, _ptr(x), _stream(x.device)), "stem_fft2")
    return x


ALGO = {"ms": 0, "prism": 1, "ms_streamed": 2, "prism_streamed": 3}


def footprint_bytes(w, algo: str = "ms", f: int = 1, storage: str = "f32", batch: int = 256,
                    cropped: bool = False) -> int:
    """Device bytes a simulation of workload ``w`` needs (admission control).
    algo: "ms", "prism", or their "_streamed" forms (transmission stack in host memory);
    cropped: a PRISM S-matrix stored Fourier-cropped."""
    lib = _lib.load()
    p = StemParams((ctypes.c_double * 3)(*[float(c) for c in w.cell]), int(w.n), int(w.n_slices),
                   float(w.slice_dz), float(w.energy_kev), float(w.alpha_mrad), float(w.ring_width_mrad),
                   int(w.n_rings), float(getattr(w, "defocus", 0.0)), float(getattr(w, "cs", 0.0)))
    return int(lib.stem_footprint_bytes(ctypes.byref(p), ALGO[algo], f,
                                        STORAGE[storage] | (STEM_CROPPED if cropped else 0), w.n_probes, batch))


def memory_model(w, algo: str, budget_bytes: int, f: int = 1, storage: str = "f32", batch: int = 256) -> str:
    """The paper's automatic choice between the single-transfer and the
    streaming memory model: "single" if the resident footprint fits the
    budget, else "streamed" if that fits, else raise MemoryError."""
    if footprint_bytes(w, algo, f, storage, batch) <= budget_bytes:
        return "single"
    if footprint_bytes(w, algo + "_streamed", f, storage, batch) <= budget_bytes:
        return "streamed"
    raise MemoryError(f"{w.name}: needs more than {budget_bytes} device bytes even when streamed")


# kernel families of profile_read (stem_prof_kind)
PROF_KINDS = {"row_slice": _lib.STEM_PROF_ROW_SLICE, "col_slice": _lib.STEM_PROF_COL_SLICE,
              "beam_sum": _lib.STEM_PROF_BEAM_SUM, "potentials": _lib.STEM_PROF_POTENTIALS}


def profile_enable(on: bool = True) -> None:
    """Start (clearing earlier records) or stop CUDA-event timing of the hot kernel families."""
    check(_lib.load().stem_profile_enable(1 if on else 0), "stem_profile_enable")


def profile_read(kind: str) -> Tuple[int, float]:
    """(launches, summed device milliseconds) of one family since profile_enable(True)."""
    n, ms = ctypes.c_int64(), ctypes.c_double()
    check(_lib.load().stem_profile_read(PROF_KINDS[kind], ctypes.byref(n), ctypes.byref(ms)), "stem_profile_read")
    return n.value, ms.value
