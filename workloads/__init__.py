"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only *generates inputs*: atom coordinates, per-atom Gaussian
potential parameters, frozen-phonon displacements, scan positions and request
arrival times.  It holds none of the method's arithmetic (no wavelength, no
interaction constant, no FFT, no propagator) so that the oracle and the CUDA
path stay independent of each other.

The workloads stand in for the amorphous-carbon cells of the paper's benchmarks
(Benchmarks section, "Algorithm Comparison" and "Hardware Scaling"): atoms are
i.i.d. uniform in an orthorhombic cell, each with a projected potential that is
a sum of two isotropic Gaussians (5 V*A at sigma 0.2 A, 2 V*A at sigma 0.6 A).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Tuple

import numpy as np

ATOM_SEED = 1706          # atom positions
PHONON_SEED_BASE = 1707   # frozen-phonon configuration c uses PHONON_SEED_BASE + c
ARRIVAL_SEED = 2017       # serving-stream arrivals

# Two-Gaussian projected potential per atom: (A1 [V*A], s1 [A], A2 [V*A], s2 [A]).
GAUSS_PARAMS = (5.0, 0.2, 2.0, 0.6)


@dataclasses.dataclass(frozen=True)
class Workload:
    """Sizes of one simulation (everything a request needs except the atoms)."""
    name: str
    cell: Tuple[float, float, float]   # Lx, Ly, Lz in Angstrom
    n_atoms: int
    n: int                             # grid side (nx == ny), power of two
    n_slices: int
    slice_dz: float                    # Angstrom
    energy_kev: float
    alpha_mrad: float                  # probe convergence semi-angle
    scan: int                          # scan is scan x scan probes over the whole cell
    ring_width_mrad: float
    n_rings: int
    batch: int = 256                   # probes (or beams) per launch
    f: Tuple[int, ...] = ()            # PRISM interpolation factors exercised
    fp_configs: int = 1                # frozen-phonon configurations
    fp_sigma: float = 0.0              # per-axis displacement std (A)
    defocus: float = 0.0               # probe defocus C1 (A)
    cs: float = 0.0                    # spherical aberration Cs (A)

    @property
    def n_probes(self) -> int:
        return self.scan * self.scan


# c1: plain FP32 multislice vs the FP64 oracle (small; the oracle finishes in seconds)
C1 = Workload("ms_128_16A", (16.0, 16.0, 20.0), 200, 128, 10, 2.0, 80.0, 20.0, 16,
              1.0, 112, batch=256)
# c2: PRISM f=4 and f=1 vs multislice
C2 = Workload("prism_256_32A", (32.0, 32.0, 40.0), 800, 256, 20, 2.0, 200.0, 20.0, 64,
              1.0, 100, batch=256, f=(1, 4))
# c3: batched multislice at paper scale, 8 frozen-phonon configurations
C3 = Workload("ms_1024_100A", (100.0, 100.0, 100.0), 50000, 1024, 50, 2.0, 200.0, 20.0,
              128, 1.0, 100, batch=256, fp_configs=8, fp_sigma=0.08)
# c4: mixed-precision PRISM f=8 at paper scale
C4 = Workload("prism8_2048_100A", (100.0, 100.0, 100.0), 50000, 2048, 100, 1.0, 300.0,
              25.0, 256, 1.0, 100, batch=128, f=(8,))

WORKLOADS = {w.name: w for w in (C1, C2, C3, C4)}


def scaled(w: Workload, **changes) -> Workload:
    """A copy of ``w`` with some fields replaced (used for small parity cases)."""
    return dataclasses.replace(w, **changes)


def atoms(w: Workload, seed: int = ATOM_SEED) -> Tuple[np.ndarray, np.ndarray]:
    """Uniform random atoms in the cell.

    Returns ``xyz`` float64 [n,3] in Angstrom (x, y in [0, L), z in [0, Lz)) and
    ``gauss`` float32 [n,4] = (A1, s1, A2, s2) per atom.
    """
    rng = np.random.default_rng(seed)
    xyz = rng.random((w.n_atoms, 3)) * np.asarray(w.cell, dtype=np.float64)
    gauss = np.tile(np.asarray(GAUSS_PARAMS, dtype=np.float32), (w.n_atoms, 1))
    return xyz, gauss


def displaced(w: Workload, xyz: np.ndarray, config: int) -> np.ndarray:
    """Frozen-phonon configuration ``config``: i.i.d. N(0, fp_sigma^2) per axis.

    x and y wrap into [0, L); z is clipped into [0, Lz).
    """
    if w.fp_sigma == 0.0:
        return xyz.copy()
    rng = np.random.default_rng(PHONON_SEED_BASE + config)
    out = xyz + rng.normal(0.0, w.fp_sigma, size=xyz.shape)
    lx, ly, lz = w.cell
    out[:, 0] = np.mod(out[:, 0], lx)
    out[:, 1] = np.mod(out[:, 1], ly)
    out[:, 2] = np.clip(out[:, 2], 0.0, np.nextafter(lz, 0.0))
    return out


def scan_positions(w: Workload, scan: Optional[int] = None) -> np.ndarray:
    """Regular scan grid covering the whole periodic cell.

    Probe p = iy * scan + ix sits at (ix * Lx / scan, iy * Ly / scan).
    Returns float64 [scan*scan, 2] holding (x, y) in Angstrom.
    """
    s = w.scan if scan is None else scan
    ix = np.arange(s, dtype=np.float64)
    xs = ix * (w.cell[0] / s)
    ys = ix * (w.cell[1] / s)
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    return np.stack([xx.ravel(), yy.ravel()], axis=1)


def random_positions(w: Workload, count: int, seed: int) -> np.ndarray:
    """``count`` probe positions uniform in the cell (float64 [count, 2])."""
    rng = np.random.default_rng(seed)
    return rng.random((count, 2)) * np.asarray(w.cell[:2], dtype=np.float64)


def random_complex(shape, seed: int, dtype=np.complex128) -> np.ndarray:
    """Standard complex normal array (used for FFT and beam-sum unit parity)."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return a.astype(dtype)


@dataclasses.dataclass
class Recipe:
    """A specimen plus fixed simulation settings that several requests share."""
    specimen: str
    workload: Workload
    algo: str
    f: int
    storage: str
    seed: int


def serving_recipes(grids: Tuple[int, ...] = (256, 512), cell: float = 50.0, n_atoms: int = 6000,
                    seed: int = ARRIVAL_SEED, count: int = 6, fs: Tuple[int, ...] = (4, 8, 16),
                    slices: Tuple[int, int] = (10, 40)) -> List[Recipe]:
    """Seeded mix of multislice and PRISM settings (grid, slice count in the
    inclusive range `slices`, f from `fs` with the window W = N / f kept at 8 or
    more, storage)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(grids))
        n_sl = int(rng.integers(slices[0], slices[1] + 1))
        algo = "prism" if i % 2 else "ms"
        f = int(rng.choice(fs)) if algo == "prism" else 1
        while n // f < 8:
            f //= 2
        storage = str(rng.choice(("f16", "bf16", "f32"))) if algo == "prism" else "f32"
        w = Workload(f"spec{i}", (cell, cell, n_sl * 1.0), n_atoms * n_sl // 40, n, n_sl, 1.0, 200.0,
                     20.0, 16, 1.0, 100)
        out.append(Recipe(f"spec{i}", w, algo, f, storage, seed + 1 + i))
    return out


def serving_requests(recipes: List[Recipe], n_requests: int, rate_hz: float, seed: int = ARRIVAL_SEED,
                     scans: Tuple[int, ...] = (8, 16, 32), max_scan: Optional[List[int]] = None):
    """Poisson arrivals; each request scans a random square region of one recipe's
    specimen (side drawn from `scans`, halved while above max_scan[recipe] when
    given).  Returns [(arrival_s, recipe_index, probe_xy float64 [P, 2])]."""
    rng = np.random.default_rng(seed + 99)
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        k = int(rng.integers(len(recipes)))
        w = recipes[k].workload
        s = int(rng.choice(scans))
        while max_scan is not None and s > max(1, max_scan[k]):
            s //= 2
        step = w.cell[0] / 64.0
        x0, y0 = rng.random(2) * np.asarray(w.cell[:2])
        g = np.arange(s) * step
        yy, xx = np.meshgrid(y0 + g, x0 + g, indexing="ij")
        xy = np.stack([np.mod(xx.ravel(), w.cell[0]), np.mod(yy.ravel(), w.cell[1])], axis=1)
        out.append((t, k, xy))
    return out
