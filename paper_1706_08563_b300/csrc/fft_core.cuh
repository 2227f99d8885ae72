// fft_core.cuh - register/shared-memory radix FFT building blocks (sm_103a).
//
// One length-N transform is spread over T = N / E threads; each thread keeps E
// complex values in registers.  The transform is a Stockham autosort
// Cooley-Tukey FFT: stage s (radix R_s, sub-transform length Ns = R_0...R_{s-1})
// reads, for butterfly j, the inputs x[j + r N / R_s], multiplies input r by
// w^(r (j mod Ns)) with w = exp(-+2 pi i / (Ns R_s)), runs a radix-R_s DFT in
// registers and writes output k to (j / Ns) Ns R_s + (j mod Ns) + k Ns.  The
// first stage has radix E and needs no twiddles; stages exchange data through
// shared memory, and the later stages read their twiddles from a per-block
// shared-memory table.
//
// Register convention at entry and exit: thread t holds element t + T*q in
// v[q], q in [0, E).  So a forward transform can feed an inverse one (or a
// point-wise multiply) without a shared-memory round trip.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>


namespace stem {

// Complex add and subtract as one packed FP32 pair instruction each (the
// f32x2 forms of sm_100 and later; same IEEE rounding as two scalar ops).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "add.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// exp(-2 pi i j / 64) for j in [0, 32): the twiddles of radix-2 decimation in
// frequency for every transform length up to 64.
__device__ __forceinline__ float2 w64(int j) {
  switch (j) {
    case 1: return make_float2(9.951847267e-01f, -9.801714033e-02f);
    case 2: return make_float2(9.807852804e-01f, -1.950903220e-01f);
    case 3: return make_float2(9.569403357e-01f, -2.902846773e-01f);
    case 4: return make_float2(9.238795325e-01f, -3.826834324e-01f);
    case 5: return make_float2(8.819212643e-01f, -4.713967368e-01f);
    case 6: return make_float2(8.314696123e-01f, -5.555702330e-01f);
    case 7: return make_float2(7.730104534e-01f, -6.343932842e-01f);
    case 9: return make_float2(6.343932842e-01f, -7.730104534e-01f);
    case 10: return make_float2(5.555702330e-01f, -8.314696123e-01f);
    case 11: return make_float2(4.713967368e-01f, -8.819212643e-01f);
    case 12: return make_float2(3.826834324e-01f, -9.238795325e-01f);
    case 13: return make_float2(2.902846773e-01f, -9.569403357e-01f);
    case 14: return make_float2(1.950903220e-01f, -9.807852804e-01f);
    case 15: return make_float2(9.801714033e-02f, -9.951847267e-01f);
    case 17: return make_float2(-9.801714033e-02f, -9.951847267e-01f);
    case 18: return make_float2(-1.950903220e-01f, -9.807852804e-01f);
    case 19: return make_float2(-2.902846773e-01f, -9.569403357e-01f);
    case 20: return make_float2(-3.826834324e-01f, -9.238795325e-01f);
    case 21: return make_float2(-4.713967368e-01f, -8.819212643e-01f);
    case 22: return make_float2(-5.555702330e-01f, -8.314696123e-01f);
    case 23: return make_float2(-6.343932842e-01f, -7.730104534e-01f);
    case 25: return make_float2(-7.730104534e-01f, -6.343932842e-01f);
    case 26: return make_float2(-8.314696123e-01f, -5.555702330e-01f);
    case 27: return make_float2(-8.819212643e-01f, -4.713967368e-01f);
    case 28: return make_float2(-9.238795325e-01f, -3.826834324e-01f);
    case 29: return make_float2(-9.569403357e-01f, -2.902846773e-01f);
    case 30: return make_float2(-9.807852804e-01f, -1.950903220e-01f);
    case 31: return make_float2(-9.951847267e-01f, -9.801714033e-02f);
    default: return make_float2(1.0f, 0.0f);
  }
}

// d * w^j (forward) or d * conj(w)^j (inverse), w = exp(-2 pi i / 64), j < 32.
template <bool INV>
__device__ __forceinline__ float2 tw64(float2 d, int j) {
  if (j == 0) return d;
  if (j == 16) return INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
  if (j == 8 || j == 24) {
    // forward: w = h (sx - i);  d w = h (sx d.x + d.y, sx d.y - d.x)
    // inverse: w = h (sx + i);  d w = h (sx d.x - d.y, sx d.y + d.x)
    const float h = 7.071067812e-01f;
    const float sx = (j == 8) ? 1.0f : -1.0f;
    return INV ? make_float2(h * (sx * d.x - d.y), h * (sx * d.y + d.x))
               : make_float2(h * (sx * d.x + d.y), h * (sx * d.y - d.x));
  }
  float2 w = w64(j);
  if (INV) w.y = -w.y;
  return cmul(d, w);
}

__host__ __device__ constexpr int bitrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}
__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

// In-register radix-R DFT (R = 1..64, power of two), natural order in and out:
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
          v[start + k + span] = tw64<INV>(csub(a, b), k * (64 / (2 * span)));
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

// Stage radices for each transform length: first radix E (elements per thread),
// then up to two more.
template <int E_, int R1_, int R2_> struct ShapeOf {
  static constexpr int E = E_, R1 = R1_, R2 = R2_;
};
#ifndef STEM_FFT2048_E
#define STEM_FFT2048_E 16
#define STEM_FFT2048_R1 16
#define STEM_FFT2048_R2 8
#endif
template <int N> struct FftShape;
template <> struct FftShape<8>    : ShapeOf<8, 1, 1> {};
template <> struct FftShape<16>   : ShapeOf<4, 4, 1> {};
template <> struct FftShape<32>   : ShapeOf<8, 4, 1> {};
template <> struct FftShape<64>   : ShapeOf<8, 8, 1> {};
template <> struct FftShape<128>  : ShapeOf<16, 8, 1> {};
template <> struct FftShape<256>  : ShapeOf<16, 16, 1> {};
template <> struct FftShape<512>  : ShapeOf<32, 16, 1> {};
template <> struct FftShape<1024> : ShapeOf<32, 32, 1> {};
template <> struct FftShape<2048> : ShapeOf<STEM_FFT2048_E, STEM_FFT2048_R1, STEM_FFT2048_R2> {};

// Shared-memory view of one transform: element idx lives at
// base[(idx + idx / E) * STRIDE] (one pad slot per E elements keeps the
// stage-0 scatter free of bank conflicts).
template <int E, int STRIDE>
struct SmemView {
  float2* base;
  __device__ __forceinline__ float2& at(int idx) const { return base[(idx + idx / E) * STRIDE]; }
};

// Twiddle tables of the stages after the first, kept in shared memory: stage
// (NS, R) needs w^(r q), w = exp(-2 pi i / (NS R)), for r in [1, R) and q in
// [0, NS), stored at [(r - 1) NS + q] so that lanes with consecutive q read
// consecutive words.  The inverse transform multiplies by the conjugate.
template <int N> struct TwLayout {
  using S = FftShape<N>;
  static constexpr int NS1 = S::E, R1 = S::R1;
  static constexpr int NS2 = S::E * S::R1, R2 = S::R2;
  static constexpr int SIZE1 = R1 > 1 ? (R1 - 1) * NS1 : 0;
  static constexpr int SIZE2 = R2 > 1 ? (R2 - 1) * NS2 : 0;
  static constexpr int OFF2 = SIZE1;
  static constexpr int TOTAL = SIZE1 + SIZE2;
};

// Fill the table with exp(-2 pi i p / L): the argument 2 p / L is exact in FP32
// (L is a power of two) and sincospif is accurate to about one ulp.
template <int N>
__device__ __forceinline__ void build_twiddles(float2* tw, int tid, int nthreads) {
  using L = TwLayout<N>;
  for (int i = tid; i < L::TOTAL; i += nthreads) {
    int r, q, len;
    if (i < L::SIZE1) {
      r = i / L::NS1 + 1; q = i % L::NS1; len = L::NS1 * L::R1;
    } else {
      const int k = i - L::SIZE1;
      r = k / L::NS2 + 1; q = k % L::NS2; len = L::NS2 * L::R2;
    }
    const int p = (r * q) % len;
    float sn, cs;
    sincospif(-2.0f * (float)p / (float)len, &sn, &cs);
    tw[i] = make_float2(cs, sn);
  }
}

// Stage s >= 1 on values already gathered: v[i*R + r] = in[j_i + r N/R] with
// j_i = t + i T.  Applies the table's twiddles and the radix-R DFTs.
template <int N, int E, int R, int NS, bool INV>
__device__ __forceinline__ void stage_compute(float2 (&v)[E], int t, const float2* tw) {
  constexpr int T = N / E;
#pragma unroll
  for (int i = 0; i < E / R; ++i) {
    const int j = t + i * T;
    const int q = j & (NS - 1);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const float2 w = tw[(r - 1) * NS + q];
      v[i * R + r] = INV ? cmulc(v[i * R + r], w) : cmul(v[i * R + r], w);
    }
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
// called around every shared-memory exchange (a warp or block barrier); `tw`
// is the block's twiddle table (build_twiddles<N>).
//
// FIRST_SYNC = false drops the barrier before the first exchange write, for
// callers that have synchronised the threads since their last read of `sm`.
template <int N, bool INV, bool FIRST_SYNC = true, class View, class Sync>
__device__ __forceinline__ void fft_dist(float2 (&v)[FftShape<N>::E], const View& sm, int t, Sync sync,
                                         const float2* tw) {
  using S = FftShape<N>;
  using L = TwLayout<N>;
  constexpr int E = S::E;
  dft<E, INV>(v);                                   // stage 0, butterfly j = t
  if constexpr (S::R1 > 1) {
    if constexpr (FIRST_SYNC) sync();
#pragma unroll
    for (int k = 0; k < E; ++k) sm.at(t * E + k) = v[k];
    sync();
    stage_load<N, E, S::R1>(v, sm, t);
    stage_compute<N, E, S::R1, E, INV>(v, t, tw);
    if constexpr (S::R2 > 1) {
      sync();
      stage_store<N, E, S::R1, E>(v, sm, t);
      sync();
      stage_load<N, E, S::R2>(v, sm, t);
      stage_compute<N, E, S::R2, E * S::R1, INV>(v, t, tw + L::OFF2);
      stage_rename<E, S::R2>(v);
    } else {
      stage_rename<E, S::R1>(v);
    }
  }
}

// Twiddles of one stage held in registers: when a thread's butterflies j = t + i T
// have tile-independent q = j mod NS (always, since t is fixed per thread), a
// kernel can load them once (load_stage_twiddles) and save the shared-memory
// reads of every later transform.  wr[i][r - 1] = w^(r q_i).
template <int N, int E, int R, int NS>
__device__ __forceinline__ void load_stage_twiddles(float2 (&wr)[E / R][R - 1], int t, const float2* tw) {
  constexpr int T = N / E;
#pragma unroll
  for (int i = 0; i < E / R; ++i) {
    const int q = (t + i * T) & (NS - 1);
#pragma unroll
    for (int r = 1; r < R; ++r) wr[i][r - 1] = tw[(r - 1) * NS + q];
  }
}

template <int N, int E, int R, bool INV>
__device__ __forceinline__ void stage_compute_reg(float2 (&v)[E], const float2 (&wr)[E / R][R - 1]) {
#pragma unroll
  for (int i = 0; i < E / R; ++i) {
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const float2 w = wr[i][r - 1];
      v[i * R + r] = INV ? cmulc(v[i * R + r], w) : cmul(v[i * R + r], w);
    }
    dft<R, INV>(&v[i * R]);
  }
}

// Registers that hold the twiddles of stage 1 (W1) and stage 2 (W2) of a
// three-stage transform, for fft_dist_x2 with TW1 / TW2 set.
template <int N> struct StageTwiddles {
  using S = FftShape<N>;
  float2 w1[S::R1 > 1 ? S::E / S::R1 : 1][S::R1 > 1 ? S::R1 - 1 : 1];
  float2 w2[S::R2 > 1 ? S::E / S::R2 : 1][S::R2 > 1 ? S::R2 - 1 : 1];
};

// Two independent transforms of the same length (rows a and b) stage by stage,
// sharing the barriers: the instructions of one fill the latencies of the
// other, and a row costs half the barriers.  sa and sb are separate exchange
// buffers.  Same register conventions (and FIRST_SYNC) as fft_dist.
template <int N, bool INV, bool TW1 = false, bool TW2 = false, bool FIRST_SYNC = true, class View, class Sync>
__device__ __forceinline__ void fft_dist_x2(float2 (&va)[FftShape<N>::E], float2 (&vb)[FftShape<N>::E],
                                            const View& sa, const View& sb, int t, Sync sync, const float2* tw,
                                            const StageTwiddles<N>* reg = nullptr) {
  using S = FftShape<N>;
  using L = TwLayout<N>;
  constexpr int E = S::E;
  dft<E, INV>(va);
  dft<E, INV>(vb);
  if constexpr (S::R1 > 1) {
    if constexpr (FIRST_SYNC) sync();
#pragma unroll
    for (int k = 0; k < E; ++k) {
      sa.at(t * E + k) = va[k];
      sb.at(t * E + k) = vb[k];
    }
    sync();
    stage_load<N, E, S::R1>(va, sa, t);
    stage_load<N, E, S::R1>(vb, sb, t);
    if constexpr (TW1) {
      stage_compute_reg<N, E, S::R1, INV>(va, reg->w1);
      stage_compute_reg<N, E, S::R1, INV>(vb, reg->w1);
    } else {
      stage_compute<N, E, S::R1, E, INV>(va, t, tw);
      stage_compute<N, E, S::R1, E, INV>(vb, t, tw);
    }
    if constexpr (S::R2 > 1) {
      sync();
      stage_store<N, E, S::R1, E>(va, sa, t);
      stage_store<N, E, S::R1, E>(vb, sb, t);
      sync();
      stage_load<N, E, S::R2>(va, sa, t);
      stage_load<N, E, S::R2>(vb, sb, t);
      if constexpr (TW2) {
        stage_compute_reg<N, E, S::R2, INV>(va, reg->w2);
        stage_compute_reg<N, E, S::R2, INV>(vb, reg->w2);
      } else {
        stage_compute<N, E, S::R2, E * S::R1, INV>(va, t, tw + L::OFF2);
        stage_compute<N, E, S::R2, E * S::R1, INV>(vb, t, tw + L::OFF2);
      }
      stage_rename<E, S::R2>(va);
      stage_rename<E, S::R2>(vb);
    } else {
      stage_rename<E, S::R1>(va);
      stage_rename<E, S::R1>(vb);
    }
  }
}

// Ring accumulation with warp primitives: each of the 32 lanes of a warp adds
// v into acc[key].  Lanes whose keys form a run of equal values in lane order
// are summed first by a segmented inclusive scan over shuffles, and the last
// lane of each run issues the one shared-memory atomic of that run (keys equal
// to skip_key are dropped).  Any arrangement of keys gives the right sums; runs
// make it cheap, and along a column or row of an FFT grid the ring index is
// monotonic on each half, so neighbouring lanes mostly share a ring.  All 32
// lanes must call it together.
__device__ __forceinline__ void warp_run_add(float* acc, int key, float v, int skip_key) {
  const unsigned lane = threadIdx.x & 31u;
  const int prev = __shfl_up_sync(0xffffffffu, key, 1);
  const unsigned heads = __ballot_sync(0xffffffffu, lane == 0u || prev != key);
  // first lane of this lane's run: the highest head at or below it
  const int start = 31 - __clz(heads & (0xffffffffu >> (31u - lane)));
  float s = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float u = __shfl_up_sync(0xffffffffu, s, o);
    if ((int)lane - o >= start) s += u;
  }
  const bool tail = lane == 31u || ((heads >> (lane + 1u)) & 1u);
  if (tail && key != skip_key) atomicAdd(acc + key, s);
}

}  // namespace stem
