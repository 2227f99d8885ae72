// potential.cu - projected potential slices and transmission functions.
//
// Methods, "Calculation of the Projected Potentials": atoms are assigned whole
// to the slice floor(z / dz) and each slice's projected potential is the sum
// of the atoms' projected potentials.  Here every atom carries two isotropic
// Gaussians, A1 exp(-d^2/(2 s1^2)) + A2 exp(-d^2/(2 s2^2)), summed over
// periodic images on the square support |dx|, |dy| <= Rc = 8 max(s1, s2).
// Eq. 1's transmission function t_n = exp(i sigma V_n) is written alongside.
//
// Layout of the work: atoms are counting-sorted by (slice, 32 x 32 pixel cell
// of their centre).  A CTA owns one pixel tile and walks the slices; for each
// slice it visits the cells within reach of the largest cutoff and adds every
// atom there to the pixels it owns.  Sums are accumulated in 2^-32 fixed point
// (64-bit integers), so the result does not depend on the order in which the
// counting sort placed the atoms.
#include "internal.h"

namespace stem {

struct AtomRec {
  int jx, iy;      // pixel of the atom position, floor(x / dx) mod N
  float fx, fy;    // fractional pixel offset in [0, 1)
  float a1, a2;
  float e1x, e2x;  // dx^2 / (2 s^2): Gaussian exponent per squared pixel along x
  float e1y, e2y;  // ... along y
  float rcx, rcy;  // cutoff in pixels
};

constexpr int kTile = 32;
constexpr int kPotThreads = 256;
constexpr float kFix = 4294967296.0f;   // 2^32

struct PotWs {
  size_t recs, key, sorted, counts, offsets, reach, total;
};

static size_t al(size_t x) { return (x + 255) / 256 * 256; }

static PotWs pot_layout(int64_t n_atoms, int n, int n_slices) {
  const size_t na = (size_t)(n_atoms > 0 ? n_atoms : 1);
  const size_t keys = (size_t)n_slices * (n / kTile) * (n / kTile);
  PotWs L;
  size_t off = 0;
  L.recs = off;    off += al(na * sizeof(AtomRec));
  L.key = off;     off += al(na * sizeof(int));
  L.sorted = off;  off += al(na * sizeof(int));
  L.counts = off;  off += al(keys * sizeof(int));
  L.offsets = off; off += al((keys + 1) * sizeof(int));
  L.reach = off;   off += al(2 * sizeof(int));
  L.total = off;
  return L;
}

__global__ void k_atom_prep(const double* __restrict__ xyz, const float* __restrict__ gauss, int64_t n_atoms,
                            int n, int n_slices, double dz, double dx, double dy, AtomRec* __restrict__ out,
                            int* __restrict__ key, int* __restrict__ counts, int* __restrict__ reach) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= n_atoms) return;
  const double x = xyz[3 * a], y = xyz[3 * a + 1], z = xyz[3 * a + 2];
  long long s = (long long)floor(z / dz);
  s = s < 0 ? 0 : (s > n_slices - 1 ? n_slices - 1 : s);
  const double u = x / dx, v = y / dy;
  const double ju = floor(u), iv = floor(v);
  AtomRec r;
  r.jx = (int)(((long long)ju % n + n) % n);
  r.iy = (int)(((long long)iv % n + n) % n);
  r.fx = (float)(u - ju);
  r.fy = (float)(v - iv);
  const float a1 = gauss[4 * a], s1 = gauss[4 * a + 1], a2 = gauss[4 * a + 2], s2 = gauss[4 * a + 3];
  const float fdx = (float)dx, fdy = (float)dy;
  r.a1 = a1;
  r.a2 = a2;
  r.e1x = fdx * fdx / (2.0f * s1 * s1);
  r.e2x = fdx * fdx / (2.0f * s2 * s2);
  r.e1y = fdy * fdy / (2.0f * s1 * s1);
  r.e2y = fdy * fdy / (2.0f * s2 * s2);
  const float rc = 8.0f * fmaxf(s1, s2);
  r.rcx = rc / fdx;
  r.rcy = rc / fdy;
  out[a] = r;
  const int cells = n / kTile;
  const int k = ((int)s * cells + r.iy / kTile) * cells + r.jx / kTile;
  key[a] = k;
  atomicAdd(counts + k, 1);
  // reach in cells: a pixel of a tile can be touched by atoms whose centre cell
  // is up to ceil((rc + 1) / 32) cells away
  atomicMax(reach, (int)ceilf((r.rcx + 1.0f) / (float)kTile));
  atomicMax(reach + 1, (int)ceilf((r.rcy + 1.0f) / (float)kTile));
}

// Exclusive scan of counts into offsets; counts become zeroed fill cursors.
__global__ void k_pot_scan(int* __restrict__ counts, int n_keys, int* __restrict__ offsets) {
  __shared__ int s_a[1024];
  const int per = (n_keys + blockDim.x - 1) / blockDim.x;
  const int lo = min((int)threadIdx.x * per, n_keys), hi = min(lo + per, n_keys);
  int a = 0;
  for (int i = lo; i < hi; ++i) a += counts[i];
  s_a[threadIdx.x] = a;
  __syncthreads();
  for (int d = 1; d < (int)blockDim.x; d <<= 1) {
    const int va = threadIdx.x >= d ? s_a[threadIdx.x - d] : 0;
    __syncthreads();
    s_a[threadIdx.x] += va;
    __syncthreads();
  }
  a = s_a[threadIdx.x] - a;
  for (int i = lo; i < hi; ++i) {
    offsets[i] = a;
    a += counts[i];
    counts[i] = 0;
  }
  if (threadIdx.x == blockDim.x - 1) offsets[n_keys] = s_a[threadIdx.x];
}

__global__ void k_pot_fill(const int* __restrict__ key, int64_t n_atoms, const int* __restrict__ offsets,
                           int* __restrict__ cursor, int* __restrict__ sorted) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= n_atoms) return;
  const int k = key[a];
  sorted[offsets[k] + atomicAdd(cursor + k, 1)] = (int)a;
}

// Sum over periodic images of the two Gaussians along one axis (pixel units).
// dj = pixel index - atom pixel index (integer), f = the atom's fractional
// offset.  The integer offset is wrapped into [-n/2, n/2) before f is taken off,
// so that f keeps its full FP32 precision next to the cell edge.
__device__ __forceinline__ void axis_terms(int dj, float f, float rc, float e1, float e2, int n, float& g1,
                                           float& g2) {
  if (dj >= n / 2) dj -= n;
  if (dj < -(n / 2)) dj += n;
  const float d0 = (float)dj - f;
  g1 = 0.0f;
  g2 = 0.0f;
  const int kmax = (int)ceilf(rc / (float)n);
  for (int k = -kmax; k <= kmax; ++k) {
    const float d = d0 + (float)(k * n);
    if (fabsf(d) <= rc) {
      const float d2 = d * d;
      g1 += expf(-d2 * e1);
      g2 += expf(-d2 * e2);
    }
  }
}

__global__ void __launch_bounds__(kPotThreads) k_potential(const AtomRec* __restrict__ recs,
                                                           const int* __restrict__ sorted,
                                                           const int* __restrict__ offsets,
                                                           const int* __restrict__ reach, int n, int n_slices,
                                                           float sigma, float* __restrict__ v_out,
                                                           float2* __restrict__ t_out) {
  constexpr int PX = kTile * kTile / kPotThreads;   // pixels per thread (one column, PX rows)
  const int cells = n / kTile;
  const int cx = blockIdx.x % cells, cy = blockIdx.x / cells;
  const int j = cx * kTile + (threadIdx.x % kTile);
  const int i0 = cy * kTile + threadIdx.x / kTile;
  const int rx = __ldg(reach), ry = __ldg(reach + 1);
  // distinct neighbour cells only (small grids wrap onto themselves)
  const int nx = min(2 * rx + 1, cells), ny = min(2 * ry + 1, cells);
  for (int s = 0; s < n_slices; ++s) {
    long long acc[PX];
#pragma unroll
    for (int q = 0; q < PX; ++q) acc[q] = 0;
    for (int oy = 0; oy < ny; ++oy) {
      const int ccy = ((cy - ry + oy) % cells + cells) % cells;
      for (int ox = 0; ox < nx; ++ox) {
        const int ccx = ((cx - rx + ox) % cells + cells) % cells;
        const int k = (s * cells + ccy) * cells + ccx;
        const int b = __ldg(offsets + k), e = __ldg(offsets + k + 1);
        for (int idx = b; idx < e; ++idx) {
          const AtomRec at = recs[__ldg(sorted + idx)];
          float gx1, gx2;
          axis_terms(j - at.jx, at.fx, at.rcx, at.e1x, at.e2x, n, gx1, gx2);
          if (gx1 == 0.0f && gx2 == 0.0f) continue;
#pragma unroll
          for (int q = 0; q < PX; ++q) {
            const int i = i0 + q * (kPotThreads / kTile);
            float gy1, gy2;
            axis_terms(i - at.iy, at.fy, at.rcy, at.e1y, at.e2y, n, gy1, gy2);
            const float v = at.a1 * gx1 * gy1 + at.a2 * gx2 * gy2;
            acc[q] += __float2ll_rn(v * kFix);
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < PX; ++q) {
      const int i = i0 + q * (kPotThreads / kTile);
      const size_t idx = ((size_t)s * n + i) * n + j;
      const float v = (float)((double)acc[q] * (1.0 / 4294967296.0));
      if (v_out) v_out[idx] = v;
      if (t_out) {
        float sn, cs;
        sincosf(sigma * v, &sn, &cs);
        t_out[idx] = make_float2(cs, sn);
      }
    }
  }
}

size_t potential_workspace(int64_t n_atoms, int n, int n_slices) { return pot_layout(n_atoms, n, n_slices).total; }

cudaError_t launch_potentials(const stem_params& p, double sigma, const double* xyz, const float* gauss,
                              int64_t n_atoms, float* v_out, float2* t_out, void* ws, cudaStream_t s) {
  const int n = p.n;
  const PotWs L = pot_layout(n_atoms, n, p.n_slices);
  char* base = static_cast<char*>(ws);
  AtomRec* recs = reinterpret_cast<AtomRec*>(base + L.recs);
  int* key = reinterpret_cast<int*>(base + L.key);
  int* sorted = reinterpret_cast<int*>(base + L.sorted);
  int* counts = reinterpret_cast<int*>(base + L.counts);
  int* offsets = reinterpret_cast<int*>(base + L.offsets);
  int* reach = reinterpret_cast<int*>(base + L.reach);
  const int n_keys = p.n_slices * (n / kTile) * (n / kTile);
  cudaError_t e;
  if ((e = cudaMemsetAsync(counts, 0, n_keys * sizeof(int), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(reach, 0, 2 * sizeof(int), s)) != cudaSuccess) return e;
  if (n_atoms > 0) {
    const unsigned blocks = (unsigned)((n_atoms + 255) / 256);
    note_launch(), k_atom_prep<<<blocks, 256, 0, s>>>(xyz, gauss, n_atoms, n, p.n_slices, p.slice_dz, p.cell[0] / n, p.cell[1] / n,
                                       recs, key, counts, reach);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  note_launch(), k_pot_scan<<<1, 1024, 0, s>>>(counts, n_keys, offsets);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (n_atoms > 0) {
    note_launch(), k_pot_fill<<<(unsigned)((n_atoms + 255) / 256), 256, 0, s>>>(key, n_atoms, offsets, counts, sorted);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  note_launch(), k_potential<<<(n / kTile) * (n / kTile), kPotThreads, 0, s>>>(recs, sorted, offsets, reach, n, p.n_slices,
                                                                (float)sigma, v_out, t_out);
  return cudaGetLastError();
}

}  // namespace stem
