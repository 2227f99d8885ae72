// potential.cu - projected potential slices and transmission functions.
//
// Methods, "Calculation of the Projected Potentials": atoms are assigned whole
// to the slice floor(z / dz) and each slice's projected potential is the sum
// of the atoms' projected potentials.  Here every atom carries two isotropic
// Gaussians, A1 exp(-d^2/(2 s1^2)) + A2 exp(-d^2/(2 s2^2)), summed over
// periodic images on the square support |dx|, |dy| <= Rc = 8 max(s1, s2).
// Eq. 1's transmission function t_n = exp(i sigma V_n) is written alongside.
//
// Deterministic gather: a CTA owns a 32 x 32 pixel tile and a chunk of 8
// slices; it streams the atom list, compacts (in atom order) the atoms of its
// slices whose support touches the tile, and every thread adds them, in that
// order, to the pixels it owns.
#include "internal.h"

namespace stem {

struct AtomRec {
  int slice;
  int jx, iy;      // pixel of the atom position, floor(x / dx) mod N
  float fx, fy;    // fractional pixel offset in [0, 1)
  float a1, a2;
  float inv2s1x, inv2s2x;   // dx^2 / (2 s^2): Gaussian exponent per squared pixel along x
  float inv2s1y, inv2s2y;   // ... along y
  float rcx, rcy;  // cutoff in pixels
};

constexpr int kTile = 32;
constexpr int kSliceChunk = 8;
constexpr int kPotThreads = 256;

__global__ void k_atom_prep(const double* __restrict__ xyz, const float* __restrict__ gauss, int64_t n_atoms,
                            int n, int n_slices, double dz, double dx, double dy, AtomRec* __restrict__ out) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= n_atoms) return;
  const double x = xyz[3 * a], y = xyz[3 * a + 1], z = xyz[3 * a + 2];
  long long s = (long long)floor(z / dz);
  s = s < 0 ? 0 : (s > n_slices - 1 ? n_slices - 1 : s);
  const double u = x / dx, v = y / dy;
  const double ju = floor(u), iv = floor(v);
  AtomRec r;
  r.slice = (int)s;
  r.jx = (int)(((long long)ju % n + n) % n);
  r.iy = (int)(((long long)iv % n + n) % n);
  r.fx = (float)(u - ju);
  r.fy = (float)(v - iv);
  const float a1 = gauss[4 * a], s1 = gauss[4 * a + 1], a2 = gauss[4 * a + 2], s2 = gauss[4 * a + 3];
  const float fdx = (float)dx, fdy = (float)dy;
  r.a1 = a1;
  r.a2 = a2;
  r.inv2s1x = fdx * fdx / (2.0f * s1 * s1);
  r.inv2s2x = fdx * fdx / (2.0f * s2 * s2);
  r.inv2s1y = fdy * fdy / (2.0f * s1 * s1);
  r.inv2s2y = fdy * fdy / (2.0f * s2 * s2);
  const float rc = 8.0f * fmaxf(s1, s2);
  r.rcx = rc / fdx;
  r.rcy = rc / fdy;
  out[a] = r;
}

// Does [c - r, c + r] (pixel units, any periodic image) touch [lo, lo + len - 1]?
// Widened by one pixel on each side; the exact support test is per pixel.
__device__ __forceinline__ bool touches(float c, float r, int lo, int len, int n) {
  const float a = (float)lo - c - r - 1.0f;
  const float b = (float)(lo + len - 1) - c + r + 1.0f;
  return floorf(b / (float)n) * (float)n >= a;
}

// Sum over periodic images of the two Gaussians along one axis (pixel units).
__device__ __forceinline__ void axis_terms(float d0, float rc, float i1, float i2, int n, float& g1, float& g2) {
  d0 -= (float)n * rintf(d0 / (float)n);
  g1 = 0.0f;
  g2 = 0.0f;
  const int kmax = (int)ceilf(rc / (float)n);
  for (int k = -kmax; k <= kmax; ++k) {
    const float d = d0 + (float)(k * n);
    if (fabsf(d) <= rc) {
      const float d2 = d * d;
      g1 += expf(-d2 * i1);
      g2 += expf(-d2 * i2);
    }
  }
}

__global__ void __launch_bounds__(kPotThreads) k_potential(const AtomRec* __restrict__ atoms, int64_t n_atoms, int n,
                                                           int n_slices, float sigma, float* __restrict__ v_out,
                                                           float2* __restrict__ t_out) {
  __shared__ float acc[kSliceChunk][kTile * kTile];
  __shared__ AtomRec list[kPotThreads];
  __shared__ int warp_count[kPotThreads / 32];
  __shared__ int n_list;
  const int tiles_x = n / kTile;
  const int tx0 = (blockIdx.x % tiles_x) * kTile;
  const int ty0 = (blockIdx.x / tiles_x) * kTile;
  const int s0 = blockIdx.y * kSliceChunk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  for (int i = threadIdx.x; i < kSliceChunk * kTile * kTile; i += kPotThreads) (&acc[0][0])[i] = 0.0f;

  // thread owns column tid % 32 and rows tid / 32 + 8 q, q < 4
  const int j = tx0 + (threadIdx.x % kTile);
  for (int64_t base = 0; base < n_atoms; base += kPotThreads) {
    const int64_t a = base + threadIdx.x;
    bool keep = false;
    AtomRec r;
    if (a < n_atoms) {
      r = atoms[a];
      keep = r.slice >= s0 && r.slice < s0 + kSliceChunk &&
             touches((float)r.jx + r.fx, r.rcx, tx0, kTile, n) &&
             touches((float)r.iy + r.fy, r.rcy, ty0, kTile, n);
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) warp_count[warp] = __popc(ballot);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < kPotThreads / 32; ++w) {
      before += (w < warp) ? warp_count[w] : 0;
      total += warp_count[w];
    }
    if (keep) list[before + __popc(ballot & ((1u << lane) - 1u))] = r;
    if (threadIdx.x == 0) n_list = total;
    __syncthreads();
    const int cnt = n_list;
    for (int k = 0; k < cnt; ++k) {
      const AtomRec& at = list[k];
      float* out = acc[at.slice - s0];
      float gx1, gx2;
      axis_terms((float)(j - at.jx) - at.fx, at.rcx, at.inv2s1x, at.inv2s2x, n, gx1, gx2);
      if (gx1 == 0.0f && gx2 == 0.0f) continue;
#pragma unroll
      for (int q = 0; q < kTile * kTile / kPotThreads; ++q) {
        const int p = threadIdx.x + q * kPotThreads;
        const int i = ty0 + (p / kTile);
        float gy1, gy2;
        axis_terms((float)(i - at.iy) - at.fy, at.rcy, at.inv2s1y, at.inv2s2y, n, gy1, gy2);
        out[p] += at.a1 * gx1 * gy1 + at.a2 * gx2 * gy2;
      }
    }
    __syncthreads();
  }

  for (int sl = 0; sl < kSliceChunk && s0 + sl < n_slices; ++sl) {
    for (int p = threadIdx.x; p < kTile * kTile; p += kPotThreads) {
      const int jj = tx0 + (p % kTile), i = ty0 + (p / kTile);
      const size_t idx = ((size_t)(s0 + sl) * n + i) * n + jj;
      const float v = acc[sl][p];
      if (v_out) v_out[idx] = v;
      if (t_out) {
        float s, c;
        sincosf(sigma * v, &s, &c);
        t_out[idx] = make_float2(c, s);
      }
    }
  }
}

size_t potential_workspace(int64_t n_atoms) { return (size_t)(n_atoms > 0 ? n_atoms : 1) * sizeof(AtomRec); }

cudaError_t launch_potentials(const stem_params& p, double sigma, const double* xyz, const float* gauss,
                              int64_t n_atoms, float* v_out, float2* t_out, void* ws, cudaStream_t s) {
  const int n = p.n;
  AtomRec* atoms = static_cast<AtomRec*>(ws);
  if (n_atoms > 0) {
    const int threads = 256;
    const unsigned blocks = (unsigned)((n_atoms + threads - 1) / threads);
    k_atom_prep<<<blocks, threads, 0, s>>>(xyz, gauss, n_atoms, n, p.n_slices, p.slice_dz, p.cell[0] / n,
                                           p.cell[1] / n, atoms);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  dim3 grid((n / kTile) * (n / kTile), (p.n_slices + kSliceChunk - 1) / kSliceChunk);
  k_potential<<<grid, kPotThreads, 0, s>>>(atoms, n_atoms, n, p.n_slices, (float)sigma, v_out, t_out);
  return cudaGetLastError();
}

}  // namespace stem
