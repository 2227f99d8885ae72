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
// of their centre).  A CTA owns one 64 x 64 pixel tile of one slice; it visits
// the cells within reach of the largest cutoff and adds every atom there to
// the pixels it owns.  Sums are accumulated in FP32 in an order
// fixed by the input alone (cells in a fixed order, the atoms of a cell by
// ascending index), so that repeated runs give identical bits.
#include <algorithm>

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
constexpr int kScanThreads = 1024;   // the key scan: threads per chunk
constexpr int kScanPer = 4;          // keys per thread
constexpr int kScanChunk = kScanThreads * kScanPer;
constexpr int kPotThreads = 256;

struct PotWs {
  size_t recs, key, filled, sorted, counts, offsets, chunks, reach, total;
};

static size_t al(size_t x) { return (x + 255) / 256 * 256; }

static PotWs pot_layout(int64_t n_atoms, int n, int n_slices) {
  const size_t na = (size_t)(n_atoms > 0 ? n_atoms : 1);
  const size_t keys = (size_t)n_slices * (n / kTile) * (n / kTile);
  PotWs L;
  size_t off = 0;
  L.recs = off;    off += al(na * sizeof(AtomRec));
  L.key = off;     off += al(na * sizeof(int));
  L.filled = off;  off += al(na * sizeof(int));
  L.sorted = off;  off += al(na * sizeof(int));
  L.counts = off;  off += al(keys * sizeof(int));
  L.offsets = off; off += al((keys + 1) * sizeof(int));
  L.chunks = off;  off += al((keys + kScanChunk - 1) / kScanChunk * sizeof(int));
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

// Exclusive scan of counts into offsets in two launches over chunks of
// kScanChunk keys: k_pot_scan_local scans each chunk on its own and records the
// chunk's total; k_pot_scan_add adds the totals of the chunks before it.
// counts become zeroed fill cursors.
// Exclusive scan of v over the CTA (blockDim.x == kScanThreads); returns the
// CTA total through *total.
__device__ __forceinline__ int block_exclusive_scan(int v, int* s_warp, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int o = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int w = s_warp[lane];
    int wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int o = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += o;
    }
    s_warp[lane] = wi - w;
    if (lane == 31) s_warp[32] = wi;
  }
  __syncthreads();
  *total = s_warp[32];
  return s_warp[warp] + incl - v;
}

__global__ void __launch_bounds__(kScanThreads) k_pot_scan_local(int* __restrict__ counts, int n_keys,
                                                                 int* __restrict__ offsets,
                                                                 int* __restrict__ chunk_sum) {
  __shared__ int s_warp[33];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanPer;
  int c[kScanPer], run = 0;
#pragma unroll
  for (int u = 0; u < kScanPer; ++u) {
    c[u] = base + u < n_keys ? counts[base + u] : 0;
    run += c[u];
  }
  int total;
  int first = block_exclusive_scan(run, s_warp, &total);
#pragma unroll
  for (int u = 0; u < kScanPer; ++u)
    if (base + u < n_keys) {
      offsets[base + u] = first;
      counts[base + u] = 0;
      first += c[u];
    }
  if (threadIdx.x == 0) chunk_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_pot_scan_add(int* __restrict__ offsets, int n_keys,
                                                               const int* __restrict__ chunk_sum) {
  __shared__ int s_warp[33];
  int part = 0;
  for (int c = threadIdx.x; c < (int)blockIdx.x; c += kScanThreads) part += chunk_sum[c];
  int carry;
  block_exclusive_scan(part, s_warp, &carry);
  const int64_t base = (int64_t)blockIdx.x * kScanChunk;
  for (int u = threadIdx.x; u < kScanChunk; u += kScanThreads)
    if (base + u < n_keys) offsets[base + u] += carry;
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) offsets[n_keys] = carry + chunk_sum[blockIdx.x];
}

__global__ void k_pot_fill(const int* __restrict__ key, int64_t n_atoms, const int* __restrict__ offsets,
                           int* __restrict__ cursor, int* __restrict__ filled) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= n_atoms) return;
  const int k = key[a];
  filled[offsets[k] + atomicAdd(cursor + k, 1)] = (int)a;
}

// The fill above places a cell's atoms in arrival order; this pass puts them
// in ascending atom index (each atom's rank among its cell's atoms), so that
// the FP32 sums of k_potential run in an order fixed by the input alone.
__global__ void k_pot_order(const int* __restrict__ key, int64_t n_atoms, const int* __restrict__ offsets,
                            const int* __restrict__ filled, int* __restrict__ sorted) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= n_atoms) return;
  const int k = key[a];
  const int b = offsets[k], e = offsets[k + 1];
  int rank = 0;
  for (int i = b; i < e; ++i) rank += filled[i] < (int)a;
  sorted[b + rank] = (int)a;
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
  if (rc < 0.5f * (float)n - 1.0f) {
    // d0 lies in [-n/2 - 1, n/2), so every other image d0 +- k n is at least
    // n/2 - 1 > rc away
    if (fabsf(d0) <= rc) {
      const float d2 = d0 * d0;
      g1 = expf(-d2 * e1);
      g2 = expf(-d2 * e2);
    }
    return;
  }
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

// One CTA per (64 x 64 pixel tile, slice).  Each atom's Gaussians are
// separable, A exp(-dx^2/2s^2) exp(-dy^2/2s^2), so for a batch of the slice's
// atoms within reach the CTA first tabulates the x factors of the tile's 64
// columns and the y factors of its 64 rows (periodic images included) in
// shared memory; then every thread adds the products to its own pixels (one
// column, PX consecutive rows, read from the y table as float4) in FP32, in
// list order.  Atoms whose factors vanish over
// all the tile's columns or all its rows are skipped by the whole CTA (they
// would add exact zeros).
constexpr int kPotTile = 64;    // pixels per CTA side (2 x 2 sort cells)
constexpr int kPotBatch = 32;   // atoms tabulated at a time
constexpr int kPotCells = 128;  // neighbour cells flattened into one atom list at a time

__global__ void __launch_bounds__(kPotThreads, 5) k_potential(const AtomRec* __restrict__ recs,
                                                           const int* __restrict__ sorted,
                                                           const int* __restrict__ offsets,
                                                           const int* __restrict__ reach, int n, int n_slices,
                                                           float sigma, float* __restrict__ v_out,
                                                           float2* __restrict__ t_out) {
  constexpr int T = kPotTile;
  constexpr int SUB = T / kTile;                    // sort cells per tile side
  constexpr int PX = T * T / kPotThreads;           // pixels per thread (one column, PX consecutive rows)
  static_assert(PX % 4 == 0, "float4 reads of the y table");
  static_assert(kPotCells == 4 * 32 && kPotBatch <= kPotThreads, "cell scan: 4 cells per lane of one warp");
  static_assert(T % 32 == 0 && T % kTile == 0, "whole warps per (atom, axis) row of the tables");
  __shared__ __align__(16) float s_g[kPotBatch][2][2][T];   // [atom][axis x/y][Gaussian 1/2][pixel]
  __shared__ float s_amp[kPotBatch][2];
  __shared__ int s_nz[kPotBatch];                   // bit axis * (T / 32) + w: a factor is nonzero in pixels [32 w, 32 w + 32)
  __shared__ int s_atom[kPotBatch];
  __shared__ int s_first[kPotCells + 1];            // running atom count over the group's cells
  __shared__ int s_begin[kPotCells];                // each cell's first entry of `sorted`
  const int cells = n / kTile, tiles = n / T;
  const int tx = blockIdx.x % tiles, ty = blockIdx.x / tiles;
  const int lane = threadIdx.x & 31;
  const int col = threadIdx.x % T, row0 = threadIdx.x / T;
  const int j = tx * T + col;
  const int rx = __ldg(reach), ry = __ldg(reach + 1);
  // distinct neighbour cells only (small grids wrap onto themselves)
  const int nx = min(2 * rx + SUB, cells), ny = min(2 * ry + SUB, cells);
  const int nc = nx * ny;
  for (int s = blockIdx.y; s < n_slices; s += gridDim.y) {
    float acc[PX];
#pragma unroll
    for (int q = 0; q < PX; ++q) acc[q] = 0.0f;
    for (int g0 = 0; g0 < nc; g0 += kPotCells) {
      const int ng = min(kPotCells, nc - g0);
      // the group's cells as one atom list [0, total): warp 0 scans 4 cells per lane
      if (threadIdx.x < 32) {
        int cnt[4], run = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = 4 * lane + u;
          cnt[u] = 0;
          if (c < ng) {
            const int oy = (g0 + c) / nx, ox = (g0 + c) % nx;
            const int ccy = ((ty * SUB - ry + oy) % cells + cells) % cells;
            const int ccx = ((tx * SUB - rx + ox) % cells + cells) % cells;
            const int k = (s * cells + ccy) * cells + ccx;
            s_begin[c] = __ldg(offsets + k);
            cnt[u] = __ldg(offsets + k + 1) - s_begin[c];
          }
          run += cnt[u];
        }
        int incl = run;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int o = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += o;
        }
        int first = incl - run;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = 4 * lane + u;
          if (c < ng) s_first[c] = first;
          first += cnt[u];
        }
        if (lane == 31) s_first[ng] = incl;
      }
      __syncthreads();
      const int total = s_first[ng];
      for (int t0 = 0; t0 < total; t0 += kPotBatch) {
        const int nb = min(kPotBatch, total - t0);
        if (threadIdx.x < nb) {
          // the cell holding list entry t: the last c with s_first[c] <= t
          const int t = t0 + threadIdx.x;
          int lo = 0, hi = ng - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_first[mid] <= t) lo = mid;
            else hi = mid - 1;
          }
          s_atom[threadIdx.x] = __ldg(sorted + s_begin[lo] + (t - s_first[lo]));
          s_nz[threadIdx.x] = 0;
        }
        __syncthreads();
        // tabulate: entries e = (atom, axis, pixel); each warp pass covers 32
        // pixels of one (atom, axis) row
        for (int e = threadIdx.x; e < nb * 2 * T; e += kPotThreads) {
          const int a = e / (2 * T), axis = (e / T) & 1, pos = e % T;
          const AtomRec& at = recs[s_atom[a]];
          float g1, g2;
          if (axis == 0) axis_terms(tx * T + pos - at.jx, at.fx, at.rcx, at.e1x, at.e2x, n, g1, g2);
          else axis_terms(ty * T + pos - at.iy, at.fy, at.rcy, at.e1y, at.e2y, n, g1, g2);
          s_g[a][axis][0][pos] = g1;
          s_g[a][axis][1][pos] = g2;
          const unsigned nz = __ballot_sync(0xffffffffu, g1 != 0.0f || g2 != 0.0f);
          if (lane == 0) {
            if (nz) atomicOr(&s_nz[a], 1 << (axis * (T / 32) + pos / 32));
            if (axis == 0 && pos == 0) {
              s_amp[a][0] = at.a1;
              s_amp[a][1] = at.a2;
            }
          }
        }
        __syncthreads();
        for (int a = 0; a < nb; ++a) {
          constexpr int kAxisBits = (1 << (T / 32)) - 1;
          const int nz = s_nz[a];
          if (!(nz & kAxisBits) || !(nz >> (T / 32))) continue;
          const float gx1 = s_amp[a][0] * s_g[a][0][0][col], gx2 = s_amp[a][1] * s_g[a][0][1][col];
          const float4* gy1 = reinterpret_cast<const float4*>(&s_g[a][1][0][row0 * PX]);
          const float4* gy2 = reinterpret_cast<const float4*>(&s_g[a][1][1][row0 * PX]);
#pragma unroll
          for (int q4 = 0; q4 < PX / 4; ++q4) {
            const float4 y1 = gy1[q4], y2 = gy2[q4];
            float* c = acc + 4 * q4;
            c[0] = fmaf(gx2, y2.x, fmaf(gx1, y1.x, c[0]));
            c[1] = fmaf(gx2, y2.y, fmaf(gx1, y1.y, c[1]));
            c[2] = fmaf(gx2, y2.z, fmaf(gx1, y1.z, c[2]));
            c[3] = fmaf(gx2, y2.w, fmaf(gx1, y1.w, c[3]));
          }
        }
        __syncthreads();
      }
      __syncthreads();   // the next group rewrites s_first / s_begin
    }
#pragma unroll
    for (int q = 0; q < PX; ++q) {
      const int i = ty * T + row0 * PX + q;
      const size_t idx = ((size_t)s * n + i) * n + j;
      const float v = acc[q];
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
  int* filled = reinterpret_cast<int*>(base + L.filled);
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
  const unsigned chunks = (unsigned)((n_keys + kScanChunk - 1) / kScanChunk);
  int* chunk_sum = reinterpret_cast<int*>(base + L.chunks);
  note_launch(), k_pot_scan_local<<<chunks, kScanThreads, 0, s>>>(counts, n_keys, offsets, chunk_sum);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  note_launch(), k_pot_scan_add<<<chunks, kScanThreads, 0, s>>>(offsets, n_keys, chunk_sum);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (n_atoms > 0) {
    const unsigned blocks = (unsigned)((n_atoms + 255) / 256);
    note_launch(), k_pot_fill<<<blocks, 256, 0, s>>>(key, n_atoms, offsets, counts, filled);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    note_launch(), k_pot_order<<<blocks, 256, 0, s>>>(key, n_atoms, offsets, filled, sorted);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const dim3 grid((unsigned)((n / kPotTile) * (n / kPotTile)), (unsigned)std::min(p.n_slices, 65535));
  ProfScope prof(STEM_PROF_POTENTIALS, s);
  note_launch(), k_potential<<<grid, kPotThreads, 0, s>>>(recs, sorted, offsets, reach, n, p.n_slices, (float)sigma,
                                                         v_out, t_out);
  return cudaGetLastError();
}

}  // namespace stem
