// fft_core.cuh - register/shared-memory radix FFT building blocks (sm_103a).
//
// One length-N transform is spread over T = N / E threads; each thread keeps E
// complex values in registers.  The transform is a Stockham autosort
// Cooley-Tukey FFT: stage s (radix R_s, sub-transform length Ns = R_0...R_{s-1})
// reads, for butterfly j, the inputs x[j + r N / R_s], multiplies input r by
// w^(r (j mod Ns)) with w = exp(-+2 pi i / (Ns R_s)), runs a radix-R_s DFT in
// registers and writes output k to (j / Ns) Ns R_s + (j mod Ns) + k Ns.  The
// first stage has radix E and needs no twiddles; stages exchange data through
// shared memory.
//
// Register convention at entry and exit: thread t holds element t + T*q in
// v[q], q in [0, E).  So a forward transform can feed an inverse one (or a
// point-wise multiply) without a shared-memory round trip.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace stem {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// exp(-2 pi i j / 32) for j in [0, 16): the twiddles of radix-2 decimation in
// frequency for every transform length up to 32.
__device__ __forceinline__ float2 w32(int j) {
  switch (j) {
    case 1: return make_float2(9.807852804e-01f, -1.950903220e-01f);
    case 2: return make_float2(9.238795325e-01f, -3.826834324e-01f);
    case 3: return make_float2(8.314696123e-01f, -5.555702330e-01f);
    case 4: return make_float2(7.071067812e-01f, -7.071067812e-01f);
    case 5: return make_float2(5.555702330e-01f, -8.314696123e-01f);
    case 6: return make_float2(3.826834324e-01f, -9.238795325e-01f);
    case 7: return make_float2(1.950903220e-01f, -9.807852804e-01f);
    case 9: return make_float2(-1.950903220e-01f, -9.807852804e-01f);
    case 10: return make_float2(-3.826834324e-01f, -9.238795325e-01f);
    case 11: return make_float2(-5.555702330e-01f, -8.314696123e-01f);
    case 12: return make_float2(-7.071067812e-01f, -7.071067812e-01f);
    case 13: return make_float2(-8.314696123e-01f, -5.555702330e-01f);
    case 14: return make_float2(-9.238795325e-01f, -3.826834324e-01f);
    case 15: return make_float2(-9.807852804e-01f, -1.950903220e-01f);
    default: return make_float2(1.0f, 0.0f);
  }
}

// d * w^j (forward) or d * conj(w)^j (inverse), w = exp(-2 pi i / 32), j < 16.
template <bool INV>
__device__ __forceinline__ float2 tw32(float2 d, int j) {
  if (j == 0) return d;
  if (j == 8) return INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
  if (j == 4 || j == 12) {
    // forward: w = h (sx - i);  d w = h (sx d.x + d.y, sx d.y - d.x)
    // inverse: w = h (sx + i);  d w = h (sx d.x - d.y, sx d.y + d.x)
    const float h = 7.071067812e-01f;
    const float sx = (j == 4) ? 1.0f : -1.0f;
    return INV ? make_float2(h * (sx * d.x - d.y), h * (sx * d.y + d.x))
               : make_float2(h * (sx * d.x + d.y), h * (sx * d.y - d.x));
  }
  float2 w = w32(j);
  if (INV) w.y = -w.y;
  return cmul(d, w);
}

__host__ __device__ constexpr int bitrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}
__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

// In-register radix-R DFT (R = 1..32, power of two), natural order in and out:
// X[k] = sum_r x[r] exp(-+2 pi i r k / R).  Radix-2 decimation in frequency,
// then the bit-reversal permutation as a register rename.
template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v) {
  if constexpr (R > 1) {
#pragma unroll
    for (int span = R / 2; span >= 1; span >>= 1) {
#pragma unroll
      for (int start = 0; start < R; start += 2 * span) {
#pragma unroll
        for (int k = 0; k < span; ++k) {
          const float2 a = v[start + k];
          const float2 b = v[start + k + span];
          v[start + k] = cadd(a, b);
          v[start + k + span] = tw32<INV>(csub(a, b), k * (32 / (2 * span)));
        }
      }
    }
    float2 tmp[R];
#pragma unroll
    for (int i = 0; i < R; ++i) tmp[i] = v[i];
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = tmp[bitrev(i, ilog2(R))];
  }
}

// exp(-+2 pi i p / L) for 0 <= p < L (L a power of two), via the hardware
// sine/cosine on an argument reduced into [-pi, pi].
template <bool INV>
__device__ __forceinline__ float2 twiddle(int p, int L) {
  const int pp = (2 * p > L) ? p - L : p;
  const float ang = (INV ? 6.283185307179586f : -6.283185307179586f) * (float)pp / (float)L;
  float s, c;
  __sincosf(ang, &s, &c);
  return make_float2(c, s);
}

// Stage radices for each transform length: first radix E (elements per thread),
// then up to two more.
template <int N> struct FftShape;
template <> struct FftShape<8>    { static constexpr int E = 8,  R1 = 1,  R2 = 1; };
template <> struct FftShape<16>   { static constexpr int E = 4,  R1 = 4,  R2 = 1; };
template <> struct FftShape<32>   { static constexpr int E = 8,  R1 = 4,  R2 = 1; };
template <> struct FftShape<64>   { static constexpr int E = 8,  R1 = 8,  R2 = 1; };
template <> struct FftShape<128>  { static constexpr int E = 16, R1 = 8,  R2 = 1; };
template <> struct FftShape<256>  { static constexpr int E = 16, R1 = 16, R2 = 1; };
template <> struct FftShape<512>  { static constexpr int E = 32, R1 = 16, R2 = 1; };
template <> struct FftShape<1024> { static constexpr int E = 32, R1 = 32, R2 = 1; };
template <> struct FftShape<2048> { static constexpr int E = 32, R1 = 8,  R2 = 8; };

// Shared-memory view of one transform: element idx lives at
// base[(idx + idx / E) * STRIDE] (one pad slot per E elements keeps the
// stage-0 scatter free of bank conflicts).
template <int E, int STRIDE>
struct SmemView {
  float2* base;
  __device__ __forceinline__ float2& at(int idx) const { return base[(idx + idx / E) * STRIDE]; }
};

// Stage s >= 1 on values already gathered: v[i*R + r] = in[j_i + r N/R] with
// j_i = t + i T.  Applies twiddles and the radix-R DFTs.
template <int N, int E, int R, int NS, bool INV>
__device__ __forceinline__ void stage_compute(float2 (&v)[E], int t) {
  constexpr int T = N / E;
#pragma unroll
  for (int i = 0; i < E / R; ++i) {
    const int j = t + i * T;
    const int q = j & (NS - 1);
#pragma unroll
    for (int r = 1; r < R; ++r) v[i * R + r] = cmul(v[i * R + r], twiddle<INV>(r * q, NS * R));
    dft<R, INV>(&v[i * R]);
  }
}

template <int N, int E, int R, int NS, class View>
__device__ __forceinline__ void stage_store(const float2 (&v)[E], const View& sm, int t) {
  constexpr int T = N / E;
#pragma unroll
  for (int i = 0; i < E / R; ++i) {
    const int j = t + i * T;
    const int q = j & (NS - 1);
    const int base = (j / NS) * NS * R + q;
#pragma unroll
    for (int k = 0; k < R; ++k) sm.at(base + k * NS) = v[i * R + k];
  }
}

template <int N, int E, int R, class View>
__device__ __forceinline__ void stage_load(float2 (&v)[E], const View& sm, int t) {
  constexpr int T = N / E;
#pragma unroll
  for (int i = 0; i < E / R; ++i) {
#pragma unroll
    for (int r = 0; r < R; ++r) v[i * R + r] = sm.at(t + i * T + r * (N / R));
  }
}

// After the last stage (radix R): butterfly i output k is element t + T (i + k E/R).
template <int E, int R>
__device__ __forceinline__ void stage_rename(float2 (&v)[E]) {
  if constexpr (R < E) {
    float2 tmp[E];
#pragma unroll
    for (int i = 0; i < E; ++i) tmp[i] = v[i];
#pragma unroll
    for (int i = 0; i < E / R; ++i)
#pragma unroll
      for (int k = 0; k < R; ++k) v[i + k * (E / R)] = tmp[i * R + k];
  }
}

// Full length-N transform over the T threads that share `sm`.  `sync` is
// called around every shared-memory exchange (a warp or block barrier).
template <int N, bool INV, class View, class Sync>
__device__ __forceinline__ void fft_dist(float2 (&v)[FftShape<N>::E], const View& sm, int t, Sync sync) {
  using S = FftShape<N>;
  constexpr int E = S::E;
  dft<E, INV>(v);                                   // stage 0, butterfly j = t
  if constexpr (S::R1 > 1) {
    sync();
#pragma unroll
    for (int k = 0; k < E; ++k) sm.at(t * E + k) = v[k];
    sync();
    stage_load<N, E, S::R1>(v, sm, t);
    stage_compute<N, E, S::R1, E, INV>(v, t);
    if constexpr (S::R2 > 1) {
      sync();
      stage_store<N, E, S::R1, E>(v, sm, t);
      sync();
      stage_load<N, E, S::R2>(v, sm, t);
      stage_compute<N, E, S::R2, E * S::R1, INV>(v, t);
      stage_rename<E, S::R2>(v);
    } else {
      stage_rename<E, S::R1>(v);
    }
  }
}

}  // namespace stem
