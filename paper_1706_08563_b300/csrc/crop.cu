// crop.cu - the Fourier-cropped S-matrix ("Description of Algorithms": the
// PRISM output probe is a Fourier interpolation of the plane waves).
//
// Every exit wave is band-limited by the 2/3 limit 9 (m^2 + n^2) <= N^2, so its
// spectrum fits on the grid of signed frequencies |m|, |n| < N'/2 with
// N' = 3 N / 4, and the inverse transform there samples the same wave at the
// N' x N' points (j Lx / N', i Ly / N').  The S-matrix is stored on that grid
// (0.5625 of the bytes), the output windows have W' = N' / f pixels over the
// same L / f, and their W' x W' transforms carry the same coarse frequencies.
//
// S-matrix finish, in place in each wave buffer [N][N] after the last column
// pass has left the spectrum (k_x, k_y) / N^2 in the in-band columns:
//   k_crop_cols: every in-band column k_x: the N' entries of the signed k_y,
//                inverse transform of length N', written to rows 0 .. N'-1;
//   k_crop_rows: every row y' < N': the N' signed k_x entries (zero outside the
//                band), inverse transform, written to columns 0 .. N'-1, and
//                the beam's largest |Re|, |Im| for the 16-bit scale.
// Output windows: k_win_rows (forward transform of every row of every window)
// and k_win_cols (columns, then rings or the 4D pattern).
#include "fft3.cuh"
#include "internal.h"

namespace stem {

constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

// Lines (rows or columns) per CTA: as many as fit in 384 threads (192 for the
// long transforms, whose ~100 registers would otherwise leave one CTA per SM)
// with the CTA a whole number of warps (the ring sums use warp primitives).
template <int M> struct LineCta {
  using C = Fft3Cfg<M>;
  static constexpr int STEP = 32 / gcd_c(C::THREADS, 32);   // lines per whole number of warps
  static constexpr int G0 = ((M >= 256 ? 192 : 384) / C::THREADS) / STEP * STEP;
  static constexpr int G = G0 > 0 ? G0 : STEP;
  static constexpr int THREADS = G * C::THREADS;
  static constexpr size_t SMEM = ((size_t)G * C::LINE + C::TW) * sizeof(float2);
  static_assert(THREADS % 32 == 0, "whole warps");
};

__device__ __forceinline__ int sfreq(int j, int n) { return j < (n >> 1) ? j : j - n; }

template <int M>
__device__ __forceinline__ void line_setup(float2* smem, float2*& tw) {
  using K = LineCta<M>;
  tw = smem + (size_t)K::G * K::C::LINE;
  if constexpr (!K::C::DIRECT) build_twiddles<M>(tw, threadIdx.x, K::THREADS);
  __syncthreads();
}

// ---------------------------------------------------------------------------
// S-matrix finish
// ---------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(LineCta<M>::THREADS) k_crop_cols(float2* __restrict__ wave, int n, int nband,
                                                                   int n_lines) {
  using K = LineCta<M>;
  using C = typename K::C;
  constexpr int L = C::L, G = K::G;
  extern __shared__ float2 smem[];
  float2* tw;
  line_setup<M>(smem, tw);
  const int g = threadIdx.x / C::THREADS, lt = threadIdx.x % C::THREADS;
  const int base = blockIdx.x * G;
  const int nb3 = n / 3;
  // consecutive threads take consecutive lines (neighbouring columns) of a row;
  // K::THREADS is a multiple of G, so a thread always serves the same line
  const int gl = threadIdx.x % G, line = base + gl;
  const bool valid = line < n_lines;
  const int w = line / nband, cb = line % nband;
  const int col = cb <= nb3 ? cb : n - (nband - cb);
  float2* colp = wave + (size_t)w * n * n + col;
  // loads batched ahead of their shared-memory stores (no wait per element)
#pragma unroll 8
  for (int i = threadIdx.x; i < G * L; i += K::THREADS) {
    const int j = i / G;
    smem[gl * C::LINE + j] = valid ? colp[(size_t)((sfreq(j, L) + n) & (n - 1)) * n] : make_float2(0.0f, 0.0f);
  }
  __syncthreads();
  fft3m_line<M, true>(smem + g * C::LINE, smem + g * C::LINE, tw, lt, [] { __syncthreads(); });
  if (valid)
    for (int i = threadIdx.x; i < G * L; i += K::THREADS) {
      const int j = i / G;
      colp[(size_t)j * n] = smem[gl * C::LINE + j];
    }
}

template <int M>
__global__ void __launch_bounds__(LineCta<M>::THREADS) k_crop_rows(float2* __restrict__ wave, int n, int n_lines,
                                                                   unsigned* __restrict__ beam_max) {
  using K = LineCta<M>;
  using C = typename K::C;
  constexpr int L = C::L, G = K::G;
  extern __shared__ float2 smem[];
  __shared__ unsigned s_max[G];
  float2* tw;
  line_setup<M>(smem, tw);
  if (threadIdx.x < G) s_max[threadIdx.x] = 0u;
  const int g = threadIdx.x / C::THREADS, lt = threadIdx.x % C::THREADS;
  const int base = blockIdx.x * G;
  const int nb3 = n / 3;
  // the CTA walks its lines one after the other, consecutive threads on
  // consecutive entries of the row (line-wide indices computed once per line)
  for (int gl = 0; gl < G; ++gl) {
    const int line = base + gl;
    const bool valid = line < n_lines;
    const float2* src = wave + ((size_t)(line / L) * n + line % L) * n;
#pragma unroll 8
    for (int j0 = 0; j0 < L; j0 += K::THREADS) {
      const int j = j0 + threadIdx.x;
      if (j < L) {
        const int m = sfreq(j, L);
        smem[gl * C::LINE + j] = valid && m <= nb3 && m >= -nb3 ? src[(m + n) & (n - 1)] : make_float2(0.0f, 0.0f);
      }
    }
  }
  __syncthreads();
  fft3m_line<M, true>(smem + g * C::LINE, smem + g * C::LINE, tw, lt, [] { __syncthreads(); });
  for (int gl = 0; gl < G; ++gl) {
    const int line = base + gl;
    const bool valid = line < n_lines;
    float2* dst = wave + ((size_t)(line / L) * n + line % L) * n;
    for (int j0 = 0; j0 < L; j0 += K::THREADS) {
      const int j = j0 + threadIdx.x;
      float mx = 0.0f;
      if (valid && j < L) {
        const float2 v = smem[gl * C::LINE + j];
        dst[j] = v;
        mx = fmaxf(fabsf(v.x), fabsf(v.y));
      }
      // every lane takes part (uniform trip count); one atomic per warp
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if ((threadIdx.x & 31) == 0 && valid) atomicMax(s_max + gl, __float_as_uint(mx));
    }
  }
  __syncthreads();
  if (threadIdx.x < G && base + (int)threadIdx.x < n_lines)
    atomicMax(beam_max + (base + threadIdx.x) / L, s_max[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// Output windows of side W' = 3M
// ---------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(LineCta<M>::THREADS) k_win_rows(float2* __restrict__ win, int n_lines) {
  using K = LineCta<M>;
  using C = typename K::C;
  constexpr int L = C::L, G = K::G;
  extern __shared__ float2 smem[];
  float2* tw;
  line_setup<M>(smem, tw);
  const int g = threadIdx.x / C::THREADS, lt = threadIdx.x % C::THREADS;
  const size_t base = (size_t)blockIdx.x * G;
  // loads batched ahead of their shared-memory stores (no wait per element)
#pragma unroll 8
  for (int i = threadIdx.x; i < G * L; i += K::THREADS) {
    const int gl = i / L, j = i % L;
    smem[gl * C::LINE + j] = base + gl < (size_t)n_lines ? win[(base + gl) * L + j] : make_float2(0.0f, 0.0f);
  }
  __syncthreads();
  fft3m_line<M, false>(smem + g * C::LINE, smem + g * C::LINE, tw, lt, [] { __syncthreads(); });
  for (int i = threadIdx.x; i < G * L; i += K::THREADS) {
    const int gl = i / L, j = i % L;
    if (base + gl < (size_t)n_lines) win[(base + gl) * L + j] = smem[gl * C::LINE + j];
  }
}

// One CTA per window: columns G at a time, forward transform, then either the
// rings (lut: the window's coarse ring table, warp_run_add into shared rings,
// one flush per window) or the 4D pattern inside the band limit
// 9 (mu^2 + nu^2) <= band_w2 (= (N / f)^2: coarse mu stands for f mu).
template <int M, bool DP>
__global__ void __launch_bounds__(LineCta<M>::THREADS)
    k_win_cols(const float2* __restrict__ win, const uint16_t* __restrict__ lut, int n_rings, float scale,
               float* __restrict__ rings, float* __restrict__ dp, int band_w2) {
  using K = LineCta<M>;
  using C = typename K::C;
  constexpr int L = C::L, G = K::G;
  extern __shared__ float2 smem[];
  float2* tw;
  line_setup<M>(smem, tw);
  float* ring_acc = reinterpret_cast<float*>(tw + C::TW);
  const int g = threadIdx.x / C::THREADS, lt = threadIdx.x % C::THREADS;
  const size_t p = blockIdx.x;
  const float2* src = win + p * L * L;
  if constexpr (!DP)
    for (int i = threadIdx.x; i < n_rings; i += K::THREADS) ring_acc[i] = 0.0f;
  for (int u0 = 0; u0 < L; u0 += G) {
    // loads batched ahead of their shared-memory stores (no wait per element)
#pragma unroll 8
    for (int i = threadIdx.x; i < G * L; i += K::THREADS) {
      const int gl = i % G, j = i / G, u = u0 + gl;
      smem[gl * C::LINE + j] = u < L ? src[(size_t)j * L + u] : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    fft3m_line<M, false>(smem + g * C::LINE, smem + g * C::LINE, tw, lt, [] { __syncthreads(); });
    // consecutive threads walk down a column, along which the ring changes rarely
    constexpr int ITER = (G * L + K::THREADS - 1) / K::THREADS;
    for (int it = 0; it < ITER; ++it) {
      const int i = threadIdx.x + it * K::THREADS;
      const int gl = i / L, j = i % L, u = u0 + gl;
      const bool in = i < G * L && u < L;
      const float v = in ? cabs2(smem[gl * C::LINE + j]) : 0.0f;
      if constexpr (DP) {
        const int mu = sfreq(u, L), nu = sfreq(j, L);
        if (in && 9 * (mu * mu + nu * nu) <= band_w2) dp[(p * L + j) * L + u] += v * scale;
      } else {
        const int r = in ? (__ldg(lut + (size_t)j * L + u) & kLutNoRing) : kLutNoRing;
        warp_run_add(ring_acc, r, v, kLutNoRing);
      }
    }
    __syncthreads();
  }
  if constexpr (!DP) {
    float* out = rings + p * n_rings;
    for (int i = threadIdx.x; i < n_rings; i += K::THREADS) {
      const float acc = ring_acc[i];
      if (acc != 0.0f) atomicAdd(out + i, acc * scale);
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <class Kern>
static cudaError_t opt_in(Kern k, size_t smem) {
  return smem > 48 * 1024 ? cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                          : cudaSuccess;
}

template <int M>
static cudaError_t crop_finish_m(float2* wave, int batch, int n, unsigned* beam_max, cudaStream_t s) {
  using K = LineCta<M>;
  const int nband = 2 * (n / 3) + 1;
  cudaError_t e = opt_in(k_crop_cols<M>, K::SMEM);
  if (e != cudaSuccess) return e;
  int lines = nband * batch;
  note_launch(), k_crop_cols<M><<<(lines + K::G - 1) / K::G, K::THREADS, K::SMEM, s>>>(wave, n, nband, lines);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = opt_in(k_crop_rows<M>, K::SMEM)) != cudaSuccess) return e;
  lines = 3 * M * batch;
  note_launch(), k_crop_rows<M><<<(lines + K::G - 1) / K::G, K::THREADS, K::SMEM, s>>>(wave, n, lines, beam_max);
  return cudaGetLastError();
}

cudaError_t launch_crop_finish(float2* wave, int batch, int n, unsigned* beam_max, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  switch (n) {
    case 64: return crop_finish_m<16>(wave, batch, n, beam_max, s);
    case 128: return crop_finish_m<32>(wave, batch, n, beam_max, s);
    case 256: return crop_finish_m<64>(wave, batch, n, beam_max, s);
    case 512: return crop_finish_m<128>(wave, batch, n, beam_max, s);
    case 1024: return crop_finish_m<256>(wave, batch, n, beam_max, s);
    case 2048: return crop_finish_m<512>(wave, batch, n, beam_max, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int M>
static cudaError_t win_fft_m(float2* win, int np, const uint16_t* lut, int n_rings, float scale, float* rings,
                             float* dp, int band_w2, cudaStream_t s) {
  using K = LineCta<M>;
  cudaError_t e = opt_in(k_win_rows<M>, K::SMEM);
  if (e != cudaSuccess) return e;
  const int lines = 3 * M * np;
  note_launch(), k_win_rows<M><<<(lines + K::G - 1) / K::G, K::THREADS, K::SMEM, s>>>(win, lines);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (dp) {
    if ((e = opt_in(k_win_cols<M, true>, K::SMEM)) != cudaSuccess) return e;
    note_launch(), k_win_cols<M, true><<<np, K::THREADS, K::SMEM, s>>>(win, lut, n_rings, scale, rings, dp, band_w2);
  } else {
    const size_t smem = K::SMEM + (size_t)n_rings * sizeof(float);
    if ((e = opt_in(k_win_cols<M, false>, K::SMEM + kMaxRings * sizeof(float))) != cudaSuccess) return e;
    note_launch(), k_win_cols<M, false><<<np, K::THREADS, smem, s>>>(win, lut, n_rings, scale, rings, dp, band_w2);
  }
  return cudaGetLastError();
}

cudaError_t launch_window_fft3(int w, float2* win, int np, const uint16_t* lut, int n_rings, float scale,
                               float* rings, float* dp, int band_w2, cudaStream_t s) {
  if (np <= 0) return cudaSuccess;
  switch (w) {
    case 6: return win_fft_m<2>(win, np, lut, n_rings, scale, rings, dp, band_w2, s);
    case 12: return win_fft_m<4>(win, np, lut, n_rings, scale, rings, dp, band_w2, s);
    case 24: return win_fft_m<8>(win, np, lut, n_rings, scale, rings, dp, band_w2, s);
    case 48: return win_fft_m<16>(win, np, lut, n_rings, scale, rings, dp, band_w2, s);
    case 96: return win_fft_m<32>(win, np, lut, n_rings, scale, rings, dp, band_w2, s);
    case 192: return win_fft_m<64>(win, np, lut, n_rings, scale, rings, dp, band_w2, s);
    case 384: return win_fft_m<128>(win, np, lut, n_rings, scale, rings, dp, band_w2, s);
    case 768: return win_fft_m<256>(win, np, lut, n_rings, scale, rings, dp, band_w2, s);
    case 1536: return win_fft_m<512>(win, np, lut, n_rings, scale, rings, dp, band_w2, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stem
