"""FP64 oracle for the multislice / PRISM hot path (test infrastructure only).

Grid convention: arrays are indexed [y][x] (row i <-> y_i = i*dy, column
j <-> x_j = j*dx, dx = Lx/N, dy = Ly/N, origin at pixel 0).  A 2D FFT index
j maps to the signed frequency index m = j for j < N/2 and m = j - N
otherwise; the spatial frequency is (m/Lx, n/Ly) in 1/A.

Readings of the paper that this file fixes (where the paper is silent or leaves a choice):
* lambda and sigma are the relativistic electron wavelength and interaction
  constant (the paper defers to Kirkland for both, Methods, text after Eq. 1
  and Eq. 2).
* Forward FFT is e^{-}, unnormalised; inverse is e^{+} with 1/N^2.
* The 2/3 band limit is circular in index space: M(m,n) = 1 iff
  9 (m^2 + n^2) <= N^2, applied with the propagator on every slice and not to
  the transmission function.
* Every slice does Eq. 1 (transmit) and then Eq. 2 (propagate), the last one
  included; the detector sees |M P FFT(t_{S-1} psi)|^2.
* Angles are small-angle, alpha = lambda |k|, in mrad; ring i covers
  [i, i+1) * ring_width.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence, Tuple

import numpy as np

# CODATA 2018: h*c = 12.398419843320026 keV*A, m_e c^2 = 510.99895000 keV.
HC_KEV_A = 12.398419843320026
MC2_KEV = 510.99895000


def wavelength(energy_kev: float) -> float:
    """Relativistic electron wavelength in A: lambda = hc / sqrt(E (2 m c^2 + E))."""
    e = float(energy_kev)
    return HC_KEV_A / math.sqrt(e * (2.0 * MC2_KEV + e))


def interaction_constant(energy_kev: float) -> float:
    """sigma of Eq. 1 in rad / (V*A): (2 pi / (lambda V)) (m c^2 + eV) / (2 m c^2 + eV)."""
    e = float(energy_kev)
    lam = wavelength(e)
    return (2.0 * math.pi / (lam * e * 1000.0)) * (MC2_KEV + e) / (2.0 * MC2_KEV + e)


@dataclasses.dataclass(frozen=True)
class Params:
    cell: Tuple[float, float, float]
    n: int
    n_slices: int
    slice_dz: float
    energy_kev: float
    alpha_mrad: float
    ring_width_mrad: float
    n_rings: int
    defocus: float = 0.0      # C1 in A
    cs: float = 0.0           # spherical aberration C3 in A

    @property
    def lam(self) -> float:
        return wavelength(self.energy_kev)

    @property
    def sigma(self) -> float:
        return interaction_constant(self.energy_kev)

    @property
    def dx(self) -> float:
        return self.cell[0] / self.n

    @property
    def dy(self) -> float:
        return self.cell[1] / self.n


def params_from(w) -> Params:
    """Params from a ``workloads.Workload``."""
    return Params(tuple(float(c) for c in w.cell), int(w.n), int(w.n_slices),
                  float(w.slice_dz), float(w.energy_kev), float(w.alpha_mrad),
                  float(w.ring_width_mrad), int(w.n_rings), float(getattr(w, "defocus", 0.0)),
                  float(getattr(w, "cs", 0.0)))


def aberration_chi(p: Params, kx, ky):
    """Aberration phase chi(k) = pi lambda C1 |k|^2 + (pi/2) Cs lambda^3 |k|^4 (rad).
    The probe's Fourier coefficients carry exp(-i chi): with this sign a positive
    defocus C1 equals free propagation by C1 under Eq. 2."""
    k2 = kx * kx + ky * ky
    return math.pi * p.lam * p.defocus * k2 + 0.5 * math.pi * p.cs * p.lam ** 3 * k2 * k2


# ----------------------------------------------------------------------------
# Fourier-space tables
# ----------------------------------------------------------------------------

def freq_index(n: int) -> np.ndarray:
    """Signed FFT frequency index per array index (int64)."""
    j = np.arange(n, dtype=np.int64)
    return np.where(j < n // 2, j, j - n)


def bandlimit_mask(n: int) -> np.ndarray:
    """2/3 band limit M[n_y, m_x] = 9 (m^2 + n^2) <= N^2 (exact integers)."""
    m = freq_index(n)
    return 9 * (m[None, :] ** 2 + m[:, None] ** 2) <= n * n


def angle_mrad(p: Params) -> np.ndarray:
    """Small-angle scattering angle lambda*|k| in mrad on the N x N FFT grid [y][x]."""
    m = freq_index(p.n).astype(np.float64)
    kx = m / p.cell[0]
    ky = m / p.cell[1]
    k = np.sqrt(kx[None, :] * kx[None, :] + ky[:, None] * ky[:, None])
    return (p.lam * k) * 1000.0


def aperture(p: Params) -> np.ndarray:
    """Probe aperture A(k): inside the band limit and lambda |k| <= alpha."""
    return bandlimit_mask(p.n) & (angle_mrad(p) <= p.alpha_mrad)


def ring_table(p: Params, edges: Optional[Sequence[float]] = None) -> np.ndarray:
    """Ring index per FFT pixel (int64), -1 outside the band limit or beyond the last
    ring.  Uniform rings of ring_width_mrad, or annuli [edges[i], edges[i+1]) (mrad)."""
    ang = angle_mrad(p)
    if edges is None:
        r = np.floor(ang / p.ring_width_mrad).astype(np.int64)
        r[r >= p.n_rings] = -1
    else:
        e = np.asarray(edges, dtype=np.float64)
        r = np.searchsorted(e, ang, side="right").astype(np.int64) - 1
        r[r >= len(e) - 1] = -1
    r[~bandlimit_mask(p.n)] = -1
    return r


def coarse_ring_table(p: Params, f: int, edges: Optional[Sequence[float]] = None,
                      w: Optional[int] = None) -> np.ndarray:
    """Ring table of a W x W window FFT (W = N/f unless given): the window spans
    L/f, so coarse frequency (nu, mu) is the fine frequency (f nu, f mu) and the
    table is the fine one sampled every f-th signed index."""
    w = p.n // f if w is None else w
    fine = ring_table(p, edges)
    mu = freq_index(w)
    idx = np.mod(f * mu, p.n)
    return fine[np.ix_(idx, idx)]


def propagator(p: Params) -> np.ndarray:
    """Eq. 2 with the band limit: M * exp(-i pi lambda dz |k|^2), [y][x]."""
    m = freq_index(p.n).astype(np.float64)
    kx = m / p.cell[0]
    ky = m / p.cell[1]
    k2 = kx[None, :] * kx[None, :] + ky[:, None] * ky[:, None]
    return np.exp(-1j * math.pi * p.lam * p.slice_dz * k2) * bandlimit_mask(p.n)


# ----------------------------------------------------------------------------
# Projected potential and transmission (Methods, "Calculation of the Projected
# Potentials"; the 2-Gaussian atom model replaces the Kirkland table)
# ----------------------------------------------------------------------------

def slice_index(p: Params, z: np.ndarray) -> np.ndarray:
    """Slice of each atom: floor(z / dz), clamped into [0, S-1] (whole atom, no split)."""
    s = np.floor(np.asarray(z, dtype=np.float64) / p.slice_dz).astype(np.int64)
    return np.clip(s, 0, p.n_slices - 1)


def projected_potential(p: Params, xyz: np.ndarray, gauss: np.ndarray) -> np.ndarray:
    """V_n[y][x] in V*A: for every atom in slice n, every periodic image and both
    Gaussians, A_g exp(-d^2 / (2 s_g^2)).

    Support: terms with |x_j - x_atom| <= Rc and |y_i - y_atom| <= Rc, where
    Rc = 8 max(s1, s2) (the neglected terms are below A e^{-32}).  Image sums
    come from wrapping pixel indices modulo N.
    """
    n = p.n
    dx, dy = p.dx, p.dy
    v = np.zeros((p.n_slices, n, n), dtype=np.float64)
    sl = slice_index(p, xyz[:, 2])
    g = np.asarray(gauss, dtype=np.float64)
    for a in range(xyz.shape[0]):
        x, y = float(xyz[a, 0]), float(xyz[a, 1])
        a1, s1, a2, s2 = g[a]
        rc = 8.0 * max(s1, s2)
        jx = np.arange(math.ceil((x - rc) / dx), math.floor((x + rc) / dx) + 1)
        iy = np.arange(math.ceil((y - rc) / dy), math.floor((y + rc) / dy) + 1)
        ddx = jx * dx - x
        ddy = iy * dy - y
        keepx = np.abs(ddx) <= rc
        keepy = np.abs(ddy) <= rc
        jx, ddx = jx[keepx], ddx[keepx]
        iy, ddy = iy[keepy], ddy[keepy]
        vals = (a1 * np.outer(np.exp(-ddy * ddy / (2 * s1 * s1)), np.exp(-ddx * ddx / (2 * s1 * s1)))
                + a2 * np.outer(np.exp(-ddy * ddy / (2 * s2 * s2)), np.exp(-ddx * ddx / (2 * s2 * s2))))
        rows = np.mod(iy, n)
        cols = np.mod(jx, n)
        if len(np.unique(rows)) == len(rows) and len(np.unique(cols)) == len(cols):
            v[sl[a]][np.ix_(rows, cols)] += vals
        else:
            np.add.at(v[sl[a]], (rows[:, None], cols[None, :]), vals)
    return v


def transmission(p: Params, v: np.ndarray) -> np.ndarray:
    """Eq. 1 transmission function t_n = exp(i sigma V_n) (complex128)."""
    return np.exp(1j * p.sigma * v)


# ----------------------------------------------------------------------------
# Multislice (Methods, Eq. 1 and Eq. 2; "Multislice Probe Simulations")
# ----------------------------------------------------------------------------

def probe_k(p: Params, xy: np.ndarray) -> np.ndarray:
    """Converged probes in Fourier space, [P, N, N]:
    psi_hat_p(m, n) = A(m, n) exp(-i chi(k)) exp(-2 pi i (m x_p / Lx + n y_p / Ly)) / sqrt(|A|)."""
    ap = aperture(p)
    norm = 1.0 / math.sqrt(int(ap.sum()))
    m = freq_index(p.n).astype(np.float64)
    chi = aberration_chi(p, (m / p.cell[0])[None, :], (m / p.cell[1])[:, None])
    xy = np.atleast_2d(np.asarray(xy, dtype=np.float64))
    out = np.zeros((xy.shape[0], p.n, p.n), dtype=np.complex128)
    for i, (x, y) in enumerate(xy):
        ph = m[None, :] * x / p.cell[0] + m[:, None] * y / p.cell[1]
        out[i] = np.where(ap, np.exp(-2j * math.pi * ph - 1j * chi) * norm, 0.0)
    return out


def probe_real(p: Params, xy: np.ndarray) -> np.ndarray:
    """psi_p in real space with FFT(psi_p) = psi_hat_p (so sum_k |psi_hat|^2 = 1)."""
    return np.fft.ifft2(probe_k(p, xy), axes=(-2, -1))


def multislice_k(p: Params, trans: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Run every slice on real-space waves psi [B, N, N]; return the exit wave in
    Fourier space, Psi_hat = M P FFT(t_{S-1} psi_{S-1})."""
    prop = propagator(p)
    psi = np.asarray(psi, dtype=np.complex128)
    psi_k = None
    for s in range(p.n_slices):
        psi_k = prop * np.fft.fft2(trans[s] * psi, axes=(-2, -1))
        if s < p.n_slices - 1:
            psi = np.fft.ifft2(psi_k, axes=(-2, -1))
    return psi_k


def detector_rings(table: np.ndarray, n_rings: int, intensity: np.ndarray) -> np.ndarray:
    """I[b, i] = sum of intensity[b] over pixels whose ring index is i."""
    flat = intensity.reshape(intensity.shape[0], -1)
    t = table.ravel()
    keep = t >= 0
    out = np.zeros((flat.shape[0], n_rings), dtype=np.float64)
    for b in range(flat.shape[0]):
        out[b] = np.bincount(t[keep], weights=flat[b, keep], minlength=n_rings)[:n_rings]
    return out


def multislice_dp(p: Params, trans: np.ndarray, xy: np.ndarray) -> np.ndarray:
    """4D output: |Psi_hat|^2 per probe, [P, N, N] in FFT order."""
    return np.abs(multislice_k(p, trans, probe_real(p, xy))) ** 2


def multislice_rings(p: Params, trans: np.ndarray, xy: np.ndarray, chunk: int = 16,
                     edges: Optional[Sequence[float]] = None) -> np.ndarray:
    """Annular-ring output [P, n_rings] of multislice at probe positions xy [P, 2]
    (uniform rings, or the annuli between consecutive `edges` in mrad)."""
    xy = np.atleast_2d(np.asarray(xy, dtype=np.float64))
    table = ring_table(p, edges)
    n_out = p.n_rings if edges is None else len(edges) - 1
    out = np.zeros((xy.shape[0], n_out))
    for c0 in range(0, xy.shape[0], chunk):
        psi = probe_real(p, xy[c0:c0 + chunk])
        psi_k = multislice_k(p, trans, psi)
        out[c0:c0 + chunk] = detector_rings(table, n_out, np.abs(psi_k) ** 2)
    return out


# ----------------------------------------------------------------------------
# PRISM (Methods, "Description of Algorithms" and "PRISM Probe Simulations")
# ----------------------------------------------------------------------------

def prism_beams(p: Params, f: int) -> np.ndarray:
    """Every f-th Fourier component in x and y inside the probe aperture (and the
    band limit): int64 [n_b, 2] of (m, n), ordered by n, then m (ascending)."""
    ap = aperture(p)
    m = freq_index(p.n)
    nn, mm = np.meshgrid(m, m, indexing="ij")
    sel = ap & (np.mod(mm, f) == 0) & (np.mod(nn, f) == 0)
    beams = np.stack([mm[sel], nn[sel]], axis=1)
    order = np.lexsort((beams[:, 0], beams[:, 1]))
    return beams[order]


def plane_waves(p: Params, beams: np.ndarray) -> np.ndarray:
    """psi_b(x_j, y_i) = exp(2 pi i (m x_j / Lx + n y_i / Ly)) = exp(2 pi i (m j + n i) / N)."""
    n = p.n
    j = np.arange(n, dtype=np.int64)
    out = np.empty((beams.shape[0], n, n), dtype=np.complex128)
    for b, (m, nb) in enumerate(beams):
        k = np.mod(m * j[None, :] + nb * j[:, None], n)
        out[b] = np.exp(2j * math.pi * k / n)
    return out


def prism_smatrix(p: Params, trans: np.ndarray, beams: np.ndarray, chunk: int = 16) -> np.ndarray:
    """Compact S-matrix: each plane wave through every slice, exit wave kept in real
    space, [n_b, N, N] complex128."""
    out = np.empty((beams.shape[0], p.n, p.n), dtype=np.complex128)
    for c0 in range(0, beams.shape[0], chunk):
        psi = plane_waves(p, beams[c0:c0 + chunk])
        out[c0:c0 + chunk] = np.fft.ifft2(multislice_k(p, trans, psi), axes=(-2, -1))
    return out


def cropped_grid(n: int) -> int:
    """Side of the Fourier-cropped S-matrix grid: 3 N / 4, the size 3 * 2^k just
    above the 2/3 band (2 floor(N/3) + 1 frequencies per axis)."""
    return 3 * n // 4


def prism_smatrix_cropped(p: Params, trans: np.ndarray, beams: np.ndarray, chunk: int = 16) -> np.ndarray:
    """Fourier-cropped compact S-matrix ("Description of Algorithms": the output
    probe is a Fourier interpolation of the plane waves).  Each exit wave is
    band-limited (9 (m^2 + n^2) <= N^2), so its spectrum fits on the grid of
    signed frequencies |m|, |n| < N'/2, N' = 3 N / 4; the inverse transform
    there samples the same band-limited wave at the N' x N' points
    (j Lx / N', i Ly / N'): S'_b = (1 / N^2) sum_k Psi_hat_b(k) e^{2 pi i k.r}.
    Returns [n_b, N', N'] complex128."""
    n2 = cropped_grid(p.n)
    idx = np.mod(freq_index(n2), p.n)          # positions of the N' signed frequencies in N-point order
    out = np.empty((beams.shape[0], n2, n2), dtype=np.complex128)
    for c0 in range(0, beams.shape[0], chunk):
        psi = plane_waves(p, beams[c0:c0 + chunk])
        spec = multislice_k(p, trans, psi)[:, idx][:, :, idx]
        out[c0:c0 + chunk] = np.fft.ifft2(spec, axes=(-2, -1)) * (float(n2) / p.n) ** 2
    return out


def prism_window_origin(p: Params, f: int, xy: np.ndarray, grid: Optional[int] = None) -> np.ndarray:
    """Window origin per probe (int64 [P, 2] of (ox, oy)) on a grid of `grid`
    pixels per side (the simulation grid N unless given): the pixel nearest the
    probe (round half up) minus W/2, W = grid / f, wrapped modulo grid."""
    n = p.n if grid is None else grid
    w = n // f
    dx = p.cell[0] / n
    dy = p.cell[1] / n
    xy = np.atleast_2d(np.asarray(xy, dtype=np.float64))
    ox = np.floor(xy[:, 0] / dx + 0.5).astype(np.int64) - w // 2
    oy = np.floor(xy[:, 1] / dy + 0.5).astype(np.int64) - w // 2
    return np.stack([np.mod(ox, n), np.mod(oy, n)], axis=1)


def prism_coefficients(p: Params, beams: np.ndarray, xy: np.ndarray) -> np.ndarray:
    """c[p, b] = exp(-i chi(k_b)) exp(-2 pi i (m_b x_p / Lx + n_b y_p / Ly)) / sqrt(n_b)."""
    xy = np.atleast_2d(np.asarray(xy, dtype=np.float64))
    mb = beams[:, 0].astype(np.float64)
    nb = beams[:, 1].astype(np.float64)
    chi = aberration_chi(p, mb / p.cell[0], nb / p.cell[1])
    ph = xy[:, 0:1] * mb[None, :] / p.cell[0] + xy[:, 1:2] * nb[None, :] / p.cell[1]
    return np.exp(-2j * math.pi * ph - 1j * chi[None, :]) / math.sqrt(beams.shape[0])


def _smatrix_crop(smatrix, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """S_b on the given rows (y) and columns (x) of the grid, [n_b, len(rows), len(cols)].
    `smatrix` is an array [n_b, N, N], or any object whose crop(rows, cols) returns
    that sub-array (an S-matrix too large to hold whole, read window by window)."""
    if hasattr(smatrix, "crop"):
        return np.asarray(smatrix.crop(rows, cols), dtype=np.complex128)
    return smatrix[:, rows][:, :, cols]


def prism_window_waves(p: Params, smatrix, beams: np.ndarray, f: int,
                       xy: np.ndarray, grid: Optional[int] = None) -> np.ndarray:
    """Psi_p(v, u) = sum_b c[p, b] S_b((o_p + (u, v)) mod n), [P, W, W] (rows v, cols u),
    for an S-matrix on a grid of n = `grid` pixels per side (N unless given), W = n / f."""
    n = p.n if grid is None else grid
    w = n // f
    org = prism_window_origin(p, f, xy) if grid is None else prism_window_origin(p, f, xy, grid)
    coef = prism_coefficients(p, beams, xy)
    out = np.empty((org.shape[0], w, w), dtype=np.complex128)
    u = np.arange(w)
    for i in range(org.shape[0]):
        rows = np.mod(org[i, 1] + u, n)
        cols = np.mod(org[i, 0] + u, n)
        crop = _smatrix_crop(smatrix, rows, cols)            # [n_b, W, W]
        out[i] = np.tensordot(coef[i], crop, axes=(0, 0))
    return out


def prism_dp(p: Params, smatrix, beams: np.ndarray, f: int, xy: np.ndarray,
             grid: Optional[int] = None) -> np.ndarray:
    """PRISM 4D output on the window grid: |FFT_W(Psi_p)|^2 / W^4 inside the band
    limit (coarse (mu, nu) standing for (f mu, f nu), so the limit is
    9 (f mu)^2 + 9 (f nu)^2 <= N^2), [P, W, W] in FFT order, W = grid / f."""
    n = p.n if grid is None else grid
    w = n // f
    args = () if grid is None else (grid,)
    spec = np.fft.fft2(prism_window_waves(p, smatrix, beams, f, xy, *args), axes=(-2, -1))
    mu = freq_index(w)
    mask = 9 * f * f * (mu[None, :] ** 2 + mu[:, None] ** 2) <= p.n * p.n
    return np.abs(spec) ** 2 / float(w) ** 4 * mask[None]


def prism_rings(p: Params, smatrix, beams: np.ndarray, f: int,
                xy: np.ndarray, chunk: int = 64, grid: Optional[int] = None) -> np.ndarray:
    """PRISM annular-ring output [P, n_rings]: window beam sum, W x W FFT, |.|^2 / W^4,
    binned on the coarse grid (S-matrix on a grid of `grid` pixels per side, N
    unless given; W = grid / f)."""
    n = p.n if grid is None else grid
    w = n // f
    table = coarse_ring_table(p, f, w=w)
    xy = np.atleast_2d(np.asarray(xy, dtype=np.float64))
    out = np.zeros((xy.shape[0], p.n_rings))
    args = () if grid is None else (grid,)
    for c0 in range(0, xy.shape[0], chunk):
        win = prism_window_waves(p, smatrix, beams, f, xy[c0:c0 + chunk], *args)
        spec = np.fft.fft2(win, axes=(-2, -1))
        out[c0:c0 + chunk] = detector_rings(table, p.n_rings, np.abs(spec) ** 2) / float(w) ** 4
    return out


# ----------------------------------------------------------------------------
# Frozen phonons and error metric
# ----------------------------------------------------------------------------

def frozen_phonon_rings(p: Params, configs: Sequence[np.ndarray], gauss: np.ndarray,
                        xy: np.ndarray, algo: str = "ms", f: int = 1) -> np.ndarray:
    """Mean ring output over frozen-phonon atom configurations."""
    acc = None
    for xyz in configs:
        t = transmission(p, projected_potential(p, xyz, gauss))
        if algo == "ms":
            r = multislice_rings(p, t, xy)
        else:
            beams = prism_beams(p, f)
            r = prism_rings(p, prism_smatrix(p, t, beams), beams, f, xy)
        acc = r if acc is None else acc + r
    return acc / len(configs)


def rel_l2(test: np.ndarray, ref: np.ndarray) -> float:
    """Relative RMS error RMS(test - ref) / RMS(ref) (the AET section's metric)."""
    ref = np.asarray(ref, dtype=np.float64)
    d = np.asarray(test, dtype=np.float64) - ref
    den = math.sqrt(float(np.mean(ref * ref)))
    return math.sqrt(float(np.mean(d * d))) / den if den > 0 else math.sqrt(float(np.mean(d * d)))
