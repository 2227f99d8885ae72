// fft3.cuh - transforms of length L = 3 M (M a power of two) for the
// Fourier-cropped grid N' = 3 N / 4 and its PRISM windows W' = 3 W / 4.
//
// Decimation in time by 3: with Y_r = FFT_M(x[3 j + r]) for r = 0, 1, 2,
//   X[k + M s] = sum_r (w^(r k) Y_r[k]) exp(-+2 pi i r s / 3),  w = exp(-+2 pi i / L).
// The three length-M transforms run side by side on three groups of TM = M / E
// threads (fft_dist, registers and shared memory as in fft_core.cuh); then each
// thread combines whole triples (k, k + M, k + 2 M) in place in shared memory
// with one radix-3 butterfly.  Lengths with M < 8 (L = 6, 12, 24... below 24)
// use a direct DFT with the exponent reduced exactly in integers.
//
// A line lives in shared memory in natural order on entry and on exit; every
// thread of the CTA must call the transform (it synchronises the CTA).
#pragma once

#include "fft_core.cuh"

namespace stem {

template <int M> struct Fft3Cfg {
  static constexpr bool DIRECT = M < 8;
  static constexpr int L = 3 * M;
  static constexpr int E = DIRECT ? 1 : FftShape<(M < 8 ? 8 : M)>::E;
  static constexpr int TM = DIRECT ? 1 : M / E;
  static constexpr int THREADS = DIRECT ? 32 : 3 * TM;       // threads per line
  static constexpr int XCH = DIRECT ? 0 : M + M / E;          // exchange buffer of one sub-transform
  // float2 of shared memory per line: the line and the three exchange buffers
  // share it (the line is read into registers before the sub-transforms'
  // first exchange and written back after their last one)
  static constexpr int LINE = L > 3 * XCH ? L : 3 * XCH;
  static constexpr int TW = DIRECT ? 0 : TwLayout<(M < 8 ? 8 : M)>::TOTAL;
};

// sqrt(3) / 2
constexpr float kHalfSqrt3 = 0.8660254037844386f;

// One length-3M transform of the line x (shared memory, natural order), in
// place; exch: 3 * XCH float2 for the sub-transforms' exchanges, which may be
// x itself; tw: the CTA's table (build_twiddles<M>); tid: thread index within
// the line's THREADS.
template <int M, bool INV, class Sync>
__device__ __forceinline__ void fft3m_line(float2* x, float2* exch, const float2* tw, int tid, Sync sync) {
  using C = Fft3Cfg<M>;
  constexpr int L = C::L;
  if constexpr (C::DIRECT) {
    constexpr int PER = (L + 31) / 32;
    float2 out[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int k = tid + 32 * i;
      float2 acc = make_float2(0.0f, 0.0f);
      if (k < L) {
        for (int j = 0; j < L; ++j) {
          const int e = (j * k) % L;
          float s, c;
          sincospif((INV ? 2.0f : -2.0f) * (float)e / (float)L, &s, &c);
          acc = cadd(acc, cmul(x[j], make_float2(c, s)));
        }
      }
      out[i] = acc;
    }
    sync();
#pragma unroll
    for (int i = 0; i < PER; ++i)
      if (tid + 32 * i < L) x[tid + 32 * i] = out[i];
    sync();
  } else {
    constexpr int E = C::E, TM = C::TM;
    const int r = tid / TM, t = tid % TM;
    float2 v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = x[3 * (t + TM * q) + r];
    sync();   // the line is in registers before any exchange overwrites it
    const SmemView<E, 1> view{exch + r * C::XCH};
    fft_dist<M, INV>(v, view, t, sync, tw);
    sync();   // every thread has read its inputs from x (fft_dist<8> has no barrier of its own)
#pragma unroll
    for (int q = 0; q < E; ++q) x[r * M + t + TM * q] = v[q];
    sync();
    for (int k = tid; k < M; k += C::THREADS) {
      float s, c;
      sincospif((INV ? 2.0f : -2.0f) * (float)k / (float)L, &s, &c);
      const float2 w1 = make_float2(c, s), w2 = cmul(w1, w1);
      const float2 a0 = x[k], a1 = cmul(x[M + k], w1), a2 = cmul(x[2 * M + k], w2);
      const float2 t1 = cadd(a1, a2);
      const float2 t2 = make_float2(fmaf(-0.5f, t1.x, a0.x), fmaf(-0.5f, t1.y, a0.y));
      const float2 d = csub(a1, a2);
      // forward: -i sqrt(3)/2 d; inverse: +i sqrt(3)/2 d
      const float2 rd = INV ? make_float2(-kHalfSqrt3 * d.y, kHalfSqrt3 * d.x)
                            : make_float2(kHalfSqrt3 * d.y, -kHalfSqrt3 * d.x);
      x[k] = cadd(a0, t1);
      x[M + k] = cadd(t2, rd);
      x[2 * M + k] = csub(t2, rd);
    }
    sync();
  }
}

}  // namespace stem
