// passes.cu - fused row / column FFT passes of the multislice slice loop.
//
// One slice (Eq. 1 then Eq. 2) of a batch of waves is two passes over HBM:
//   row pass:    [row IFFT] -> x t_n (Eq. 1) -> row FFT
//   column pass: col FFT -> x M P / N^2 (Eq. 2, 2/3 band limit) -> col IFFT
// so the wave is read and written twice per slice (32 bytes per pixel).  The
// first row pass of a probe follows the column pass that builds the probe
// (Fourier-space aperture and phase ramp, then a column IFFT); the last column
// pass of multislice squares |FFT| and bins it into rings instead of storing
// (|P| = 1, so the last propagator phase does not change intensities).
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "async_copy.cuh"
#include "fft_core.cuh"
#include "internal.h"

namespace stem {

// Threads per row-pass CTA, columns per column-pass CTA and the minimum number
// of resident CTAs asked of the compiler, per transform length.
#ifndef STEM_ROW_THREADS_BIG
#define STEM_ROW_THREADS_BIG 128
#endif
#ifndef STEM_COL_C_2048
#define STEM_COL_C_2048 4
#endif
#ifndef STEM_MINB_1024
#define STEM_MINB_1024 2
#endif
#ifndef STEM_MINB_2048
#define STEM_MINB_2048 1
#endif
#ifndef STEM_PREFETCH
#define STEM_PREFETCH 1
#endif

template <int N> constexpr int min_blocks() { return N == 2048 ? STEM_MINB_2048 : (N == 1024 ? STEM_MINB_1024 : 1); }

// Ask L2 to fetch bytes that this CTA will read on its next tile, so that the
// next tile's loads are served from L2 while this tile is being transformed.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <int N> struct RowCfg {
  static constexpr int E = FftShape<N>::E;
  static constexpr int T = N / E;
  static constexpr int THR = N >= 1024 ? STEM_ROW_THREADS_BIG : 256;
  static constexpr int ROWS = (THR / T) < N ? (THR / T) : N;
  static constexpr int THREADS = ROWS * T;
  static constexpr int ROWBUF = N + N / E;
  // t_n rows of the tile, staged by one bulk copy (large transforms)
  static constexpr bool T_STAGED = N >= 1024;
  static constexpr size_t SMEM = ((size_t)ROWS * ROWBUF + TwLayout<N>::TOTAL + (T_STAGED ? (size_t)ROWS * N : 0)) *
                                     sizeof(float2) + (T_STAGED ? 16 : 0);
  static constexpr int MINB = min_blocks<N>();
};

template <int N> struct ColCfg {
  static constexpr int E = FftShape<N>::E;
  static constexpr int T = N / E;
  static constexpr int C0 = N == 2048 ? STEM_COL_C_2048 : ((256 / T) > 16 ? 16 : (256 / T));
  static constexpr int C = C0 < 1 ? 1 : (C0 > N ? N : C0);
  static constexpr int THREADS = C * T;
  static constexpr size_t FFT_SMEM = ((size_t)(N + N / E) * C + TwLayout<N>::TOTAL) * sizeof(float2);
  static constexpr int MINB = min_blocks<N>();
  // the detector pass at N <= 256 (PRISM windows, small multislice grids) runs
  // three CTAs per SM (80 registers, no spills): 1210 -> 922 us per 4096
  // windows of 256^2
  static constexpr int minb(int mode) { return (mode == COL_DET && N <= 256) ? 3 : MINB; }
  // Column tiles inside the 2/3 band limit, |m| <= N/3 (columns [0, MB] and
  // [N - MB, N)).  Outside it the propagator's mask zeroes whole columns, so
  // the slice loop never reads or writes them.
  static constexpr int MB = N / 3;
  static constexpr int LO = (MB + 1 + C - 1) / C;     // tiles covering columns 0..MB
  static constexpr int HI0 = (N - MB) / C;            // first tile touching columns N-MB..N-1
  static constexpr bool SKIP = LO < HI0;
  static constexpr int BAND_TILES = SKIP ? LO + N / C - HI0 : N / C;
  __device__ static int band_tile(int k) { return (SKIP && k >= LO) ? k - LO + HI0 : k; }
};

// Is FFT column index x inside the 2/3 band limit (|m| <= N/3)?
template <int N>
__device__ __forceinline__ bool in_band(int x) { return x <= N / 3 || x >= N - N / 3; }

// Are all indices t + T q (0 <= t < T) outside the band limit?  With q known
// after unrolling this is a constant, so the zeros it implies reach the first
// FFT stage and the unused outputs of the last one are dropped.
template <int N, int T>
__device__ __forceinline__ constexpr bool all_out_of_band(int q) {
  return q * T > N / 3 && q * T + T - 1 < N - N / 3;
}

__device__ __forceinline__ int signed_freq(int j, int n) { return j < (n >> 1) ? j : j - n; }

// ---------------------------------------------------------------------------
// Row pass: persistent CTAs over tiles of ROWS rows of one wave.  Tile index
// runs over the waves fastest and each CTA takes a contiguous block of tiles,
// so consecutive tiles of a CTA are the same rows of different waves.  For
// N >= 1024 the rows of t_n are copied into shared memory by one bulk copy
// when the tile's rows change (issued at the start of the tile, waited for
// after the inverse transform; bounded wait, timeout recorded in the status
// word).
// ---------------------------------------------------------------------------
template <int N, int MODE>
__global__ void __launch_bounds__(RowCfg<N>::THREADS, RowCfg<N>::MINB) k_row_pass(const PassArgs a, int n_tiles) {
  using Cfg = RowCfg<N>;
  constexpr int E = Cfg::E, T = Cfg::T;
  extern __shared__ float2 smem[];
  float2* tw = smem + Cfg::ROWS * Cfg::ROWBUF;
  constexpr bool T_BULK = Cfg::T_STAGED && MODE == ROW_SLICE;
  float2* tbuf = tw + TwLayout<N>::TOTAL;                                 // [ROWS][N] when T_BULK
  uint64_t* tbar = reinterpret_cast<uint64_t*>(tbuf + (Cfg::T_STAGED ? Cfg::ROWS * N : 0));
  if constexpr (T_BULK) {
    if (threadIdx.x == 0) {
      mbar_init(smem_u32(tbar), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  build_twiddles<N>(tw, threadIdx.x, Cfg::THREADS);
  __syncthreads();
  const int t = threadIdx.x % T;
  const int rl = threadIdx.x / T;
  const SmemView<E, 1> view{smem + rl * Cfg::ROWBUF};
  auto sync = [] {
    if constexpr (T > 32 || Cfg::THREADS <= 32) __syncthreads();
    else __syncwarp();
  };
  const int per = (n_tiles + gridDim.x - 1) / gridDim.x;
  const int tile_end = min(n_tiles, (int)(blockIdx.x + 1) * per);
  int staged_row0 = -1;
  uint32_t tphase = 0;

  for (int tile = blockIdx.x * per; tile < tile_end; ++tile) {
    const int wave = tile % a.batch;
    const int row0 = (tile / a.batch) * Cfg::ROWS;
    const int row = row0 + rl;
    float2* w = a.wave + (size_t)wave * N * N + (size_t)row * N;
    const bool fresh = T_BULK && row0 != staged_row0;
    if constexpr (T_BULK) {
      if (fresh) {
        __syncthreads();   // every thread has read the previous rows of t_n
        if (threadIdx.x == 0) {
          fence_proxy_async();
          const uint32_t bar = smem_u32(tbar);
          mbar_arrive_expect_tx(bar, Cfg::ROWS * N * (uint32_t)sizeof(float2));
          bulk_load(smem_u32(tbuf), a.trans + (size_t)row0 * N, Cfg::ROWS * N * (uint32_t)sizeof(float2), bar);
        }
      }
    }

    // slice-loop rows in the (k_x, y) domain hold zeros outside the band limit:
    // they are neither read from nor written to memory
    constexpr bool BAND_IN = MODE == ROW_SLICE || MODE == ROW_IFFT_MAX;
    constexpr bool BAND_OUT = MODE == ROW_SLICE;
    float2 v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int x = t + q * T;
      v[q] = (!BAND_IN || (!all_out_of_band<N, T>(q) && in_band<N>(x))) ? w[x] : make_float2(0.0f, 0.0f);
    }
#if STEM_PREFETCH
    {
      const int nt = tile + 1;
      if (t == 0 && nt < tile_end) {
        const int nrow = (nt / a.batch) * Cfg::ROWS + rl;
        const float2* nr = a.wave + (size_t)(nt % a.batch) * N * N + (size_t)nrow * N;
        if constexpr (BAND_IN) {
          // the two in-band segments, widened to 16-byte boundaries
          constexpr int lo = ((N / 3 + 1) + 1) & ~1, hi = (N - N / 3) & ~1;
          prefetch_l2_bulk(nr, lo * sizeof(float2));
          prefetch_l2_bulk(nr + hi, (N - hi) * sizeof(float2));
        } else {
          prefetch_l2_bulk(nr, N * sizeof(float2));
        }
      }
    }
#endif

    if constexpr (MODE == ROW_SLICE || MODE == ROW_IFFT_MAX || MODE == ROW_IFFT)
      fft_dist<N, true>(v, view, t, sync, tw);

    if constexpr (T_BULK) {
      if (fresh) {
        const bool ok = mbar_wait(smem_u32(tbar), tphase);
        tphase ^= 1u;
        staged_row0 = row0;
        if (__syncthreads_or(!ok)) {
          if (threadIdx.x == 0) {
            if (a.status) atomicExch(a.status, (int)STEM_ERR_TIMEOUT);
            mbar_wait(smem_u32(tbar), tphase ^ 1u);   // let the copy land before the CTA exits
          }
          return;
        }
      }
      const float2* tr = tbuf + rl * N;
#pragma unroll
      for (int q = 0; q < E; ++q) v[q] = cmul(v[q], tr[t + q * T]);
    } else if constexpr (MODE == ROW_SLICE) {
      const float2* tr = a.trans + (size_t)row * N;
#pragma unroll
      for (int q = 0; q < E; ++q) v[q] = cmul(v[q], __ldg(tr + t + q * T));
    }

    if constexpr (MODE == ROW_SLICE || MODE == ROW_FFT)
      fft_dist<N, false>(v, view, t, sync, tw);

#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int x = t + q * T;
      if (!BAND_OUT || (!all_out_of_band<N, T>(q) && in_band<N>(x))) w[x] = v[q];
    }

    if constexpr (MODE == ROW_IFFT_MAX) {
      float m = 0.0f;
#pragma unroll
      for (int q = 0; q < E; ++q) m = fmaxf(m, fmaxf(fabsf(v[q].x), fabsf(v[q].y)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if ((threadIdx.x & 31) == 0) atomicMax(a.beam_max + wave, __float_as_uint(m));
    }
  }
}

// ---------------------------------------------------------------------------
// Slice row pass at N = 2048 on pairs of waves: a tile is one row of two
// neighbouring waves, transformed together (fft_dist_x2) against one staged
// row of t_n.  The in-band part of the tile's two rows (x in [0, 684) and
// [1364, 2048): two 5 472-byte bulk copies per row) reaches shared memory one
// tile ahead: thread 0 issues the next tile's copies as soon as every thread
// has taken the current tile into registers, so the transform never waits on
// a global load.  The stage-2 twiddles live in registers (computed once per
// CTA), which leaves room in shared memory for the row stage at three CTAs
// per SM.
// ---------------------------------------------------------------------------
// Stage-2 twiddles of the pair's transforms held in registers: a thread's
// butterflies have the same twiddles in every tile, so the 14 complex values
// are computed once per CTA: 164 registers, three CTAs per SM (the register
// bound of __launch_bounds__(128, 3) would force 168 and spill), 1.3% off the
// slice loop at 2048; the stage-1 ones as well would leave two CTAs per SM
// (no gain).
struct RowPairCfg {
  static constexpr int N = 2048, E = FftShape<N>::E, T = N / E, THREADS = T;
  static constexpr int ROWBUF = N + N / E;
  // in-band segments of a row, widened to 16-byte multiples: [0, SEG) and [N - SEG, N)
  static constexpr int SEG = ((N / 3 + 1) + 1) & ~1;                 // 684
  static constexpr uint32_t SEG_BYTES = SEG * sizeof(float2);         // 5 472
  static constexpr int TW1 = TwLayout<N>::SIZE1;                      // stage-1 table in shared memory
  static constexpr size_t SMEM =
      ((size_t)2 * ROWBUF + TW1 + N + 2 * 2 * SEG) * sizeof(float2) + 2 * sizeof(uint64_t);
  static_assert(SEG_BYTES % 16 == 0 && ((N - SEG) * sizeof(float2)) % 16 == 0, "bulk copy alignment");
  static_assert(((2 * ROWBUF + TW1) * sizeof(float2)) % 16 == 0, "t_n row buffer alignment");
  // shared-memory slot of in-band element x of a staged row
  __device__ static int seg_slot(int x) { return x < SEG ? x : x - (N - 2 * SEG); }
};

// The stage-1 part of build_twiddles<2048> (the stage-2 twiddles are computed
// into registers by row_pair_stage2_twiddles).
__device__ __forceinline__ void build_twiddles_stage1(float2* tw, int tid, int nthreads) {
  using L = TwLayout<2048>;
  for (int i = tid; i < L::SIZE1; i += nthreads) {
    const int r = i / L::NS1 + 1, q = i % L::NS1, len = L::NS1 * L::R1;
    const int p = (r * q) % len;
    float sn, cs;
    sincospif(-2.0f * (float)p / (float)len, &sn, &cs);
    tw[i] = make_float2(cs, sn);
  }
}

// The values load_stage_twiddles would read from a full table, computed the
// way build_twiddles computes them (bit for bit).
__device__ __forceinline__ void row_pair_stage2_twiddles(StageTwiddles<2048>& reg, int t) {
  using S = FftShape<2048>;
  using L = TwLayout<2048>;
  constexpr int E = S::E, R = S::R2, NS = L::NS2, T = 2048 / E, len = NS * R;
#pragma unroll
  for (int i = 0; i < E / R; ++i) {
    const int q = (t + i * T) & (NS - 1);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const int p = (r * q) % len;
      float sn, cs;
      sincospif(-2.0f * (float)p / (float)len, &sn, &cs);
      reg.w2[i][r - 1] = make_float2(cs, sn);
    }
  }
}

__global__ void __launch_bounds__(RowPairCfg::THREADS, 2) k_row_slice_pair_2048(const PassArgs a, int n_tiles) {
  using Cfg = RowPairCfg;
  constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T, SEG = Cfg::SEG;
  static_assert(FftShape<N>::R2 > 1, "three-stage transform");
  extern __shared__ float2 smem[];
  float2* xa = smem;
  float2* xb = smem + Cfg::ROWBUF;
  float2* tw = smem + 2 * Cfg::ROWBUF;
  float2* tbuf = tw + Cfg::TW1;                     // [N]: the tile's row of t_n
  float2* stg = tbuf + N;                           // [2][2 SEG]: the tile's in-band rows
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg + 4 * SEG);
  const uint32_t tbar = smem_u32(bars), sbar = smem_u32(bars + 1);
  if (threadIdx.x == 0) {
    mbar_init(tbar, 1);
    mbar_init(sbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  build_twiddles_stage1(tw, threadIdx.x, Cfg::THREADS);
  const int t = threadIdx.x;
  StageTwiddles<N> reg;
  row_pair_stage2_twiddles(reg, t);
  __syncthreads();
  const SmemView<E, 1> va{xa}, vb{xb};
  auto sync = [] { __syncthreads(); };
  const int pairs = (a.batch + 1) / 2;
  const int per = (n_tiles + gridDim.x - 1) / gridDim.x;
  const int tile_begin = blockIdx.x * per;
  const int tile_end = min(n_tiles, (int)(blockIdx.x + 1) * per);

  // the in-band segments of tile's rows into the stage (thread 0)
  auto issue_rows = [&](int tile) {
    const int row = tile / pairs, k = tile % pairs;
    const int nw = 2 * k + 1 < a.batch ? 2 : 1;
    mbar_arrive_expect_tx(sbar, 2u * nw * Cfg::SEG_BYTES);
    for (int j = 0; j < nw; ++j) {
      const float2* src = a.wave + (size_t)(2 * k + j) * N * N + (size_t)row * N;
      const uint32_t dst = smem_u32(stg + j * 2 * SEG);
      bulk_load(dst, src, Cfg::SEG_BYTES, sbar);
      bulk_load(dst + Cfg::SEG_BYTES, src + (N - SEG), Cfg::SEG_BYTES, sbar);
    }
  };
  if (threadIdx.x == 0 && tile_begin < tile_end) issue_rows(tile_begin);

  int staged_row = -1;
  uint32_t tphase = 0, sphase = 0;
  bool t_pending = false;
  for (int tile = tile_begin; tile < tile_end; ++tile) {
    const int row = tile / pairs, k = tile % pairs;
    const int wa = 2 * k, wb = 2 * k + 1;
    const bool has_b = wb < a.batch;
    float2* pa = a.wave + (size_t)wa * N * N + (size_t)row * N;
    float2* pb = a.wave + (size_t)(has_b ? wb : wa) * N * N + (size_t)row * N;
    const bool fresh = row != staged_row;
    if (fresh) {
      __syncthreads();   // every thread has read the previous row of t_n
      if (threadIdx.x == 0) {
        fence_proxy_async();
        mbar_arrive_expect_tx(tbar, N * (uint32_t)sizeof(float2));
        bulk_load(smem_u32(tbuf), a.trans + (size_t)row * N, N * (uint32_t)sizeof(float2), tbar);
      }
      t_pending = true;
    }
    const bool ok = mbar_wait(sbar, sphase);
    sphase ^= 1u;
    float2 A[E], B[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int x = t + q * T;
      const bool in = !all_out_of_band<N, T>(q) && in_band<N>(x);
      A[q] = in ? stg[Cfg::seg_slot(x)] : make_float2(0.0f, 0.0f);
      B[q] = (in && has_b) ? stg[2 * SEG + Cfg::seg_slot(x)] : make_float2(0.0f, 0.0f);
    }
    // every thread holds its values (and agrees on the wait): the stage takes the next tile
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        if (a.status) atomicExch(a.status, (int)STEM_ERR_TIMEOUT);
        if (t_pending) mbar_wait(tbar, tphase);   // let the copies land before the CTA exits
      }
      return;
    }
    if (threadIdx.x == 0 && tile + 1 < tile_end) {
      fence_proxy_async();
      issue_rows(tile + 1);
    }
    // the tile barrier above follows the previous tile's last reads of xa / xb
    fft_dist_x2<N, true, false, true, false>(A, B, va, vb, t, sync, tw, &reg);
    if (fresh) {
      const bool tok = mbar_wait(tbar, tphase);
      tphase ^= 1u;
      t_pending = false;
      staged_row = row;
      if (__syncthreads_or(!tok)) {
        if (threadIdx.x == 0) {
          if (a.status) atomicExch(a.status, (int)STEM_ERR_TIMEOUT);
          mbar_wait(tbar, tphase ^ 1u);                                  // the t_n copy
          if (tile + 1 < tile_end) mbar_wait(sbar, sphase);             // the next tile's rows
        }
        return;
      }
    }
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const float2 tv = tbuf[t + q * T];
      A[q] = cmul(A[q], tv);
      B[q] = cmul(B[q], tv);
    }
    fft_dist_x2<N, false, false, true>(A, B, va, vb, t, sync, tw, &reg);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int x = t + q * T;
      if (!all_out_of_band<N, T>(q) && in_band<N>(x)) {
        pa[x] = A[q];
        if (has_b) pb[x] = B[q];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Column pass: persistent CTAs over tiles of C columns of one wave.  Thread
// (c, t) = threadIdx c + C t holds column elements t + T q; neighbouring lanes
// read neighbouring columns, so every global access is C * 8 contiguous bytes.
// ---------------------------------------------------------------------------
template <int N, int MODE, bool BAND>
__global__ void __launch_bounds__(ColCfg<N>::THREADS, ColCfg<N>::minb(MODE)) k_col_pass(const PassArgs a, int n_tiles) {
  using Cfg = ColCfg<N>;
  constexpr int E = Cfg::E, T = Cfg::T, C = Cfg::C;
  extern __shared__ float2 smem[];
  float2* tw = smem + (N + N / E) * C;
  float* ring_acc = reinterpret_cast<float*>(tw + TwLayout<N>::TOTAL);
  build_twiddles<N>(tw, threadIdx.x, Cfg::THREADS);
  __syncthreads();
  const int c = threadIdx.x % C;
  const int t = threadIdx.x / C;
  const SmemView<E, C> view{smem + c};
  auto sync = [] { __syncthreads(); };
  constexpr int col_tiles = BAND ? Cfg::BAND_TILES : N / C;
  // The detector pass takes a contiguous block of tiles, so that consecutive
  // tiles are mostly columns of the same wave: its rings stay in shared memory
  // across them and reach global memory once per wave (and CTA), not once per
  // tile.  The other modes stride over the tiles.
  constexpr bool DET = MODE == COL_DET;
  const int per = DET ? (n_tiles + gridDim.x - 1) / gridDim.x : 0;
  const int tile_begin = DET ? blockIdx.x * per : blockIdx.x;
  const int tile_end = DET ? min(n_tiles, (int)(blockIdx.x + 1) * per) : n_tiles;
  const int tile_step = DET ? 1 : gridDim.x;
  int acc_wave = -1;   // the wave whose rings ring_acc holds (detector pass)
  auto flush_rings = [&](bool zero) {
    // every thread has finished adding into ring_acc (callers synchronise)
    if (acc_wave >= 0) {
      float* out = a.rings + (size_t)acc_wave * a.n_rings;
      for (int i = threadIdx.x; i < a.n_rings; i += Cfg::THREADS) {
        const float acc = ring_acc[i];
        if (acc != 0.0f) atomicAdd(out + i, acc * a.ring_scale);
        if (zero) ring_acc[i] = 0.0f;
      }
    } else if (zero) {
      for (int i = threadIdx.x; i < a.n_rings; i += Cfg::THREADS) ring_acc[i] = 0.0f;
    }
  };

  for (int tile = tile_begin; tile < tile_end; tile += tile_step) {
    const int wave = tile / col_tiles;
    const int ct = tile % col_tiles;
    const int col = (BAND ? Cfg::band_tile(ct) : ct) * C + c;
    float2* w = a.wave + (size_t)wave * N * N + col;

    if constexpr (DET) {
      if (wave != acc_wave) {
        __syncthreads();   // the previous tile's sums are in ring_acc
        flush_rings(true);
        acc_wave = wave;
      }
    }

    float2 v[E];
    if constexpr (MODE == COL_PROBE_INIT) {
      // psi_hat(m, n) = A(m, n) exp(-2 pi i (m x_p / Lx + n y_p / Ly)) / (sqrt|A| N^2);
      // the phase is reduced in FP64, then evaluated in FP32.
      const double xp = a.probe_xy[2 * wave], yp = a.probe_xy[2 * wave + 1];
      const double thx = (double)signed_freq(col, N) * xp * a.inv_lx;
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const int ky = t + q * T;
        const uint16_t l = __ldg(a.lut + (size_t)ky * N + col);
        float2 val = make_float2(0.0f, 0.0f);
        if (l & kLutAperture) {
          const int n = signed_freq(ky, N);
          double th = thx + (double)n * yp * a.inv_ly;
          if (a.chi_c1 != 0.0 || a.chi_c3 != 0.0) {
            // aberrations exp(-i chi(k)), chi / (2 pi) = chi_c1 |k|^2 + chi_c3 |k|^4
            const double kx = (double)signed_freq(col, N) * a.inv_lx, kyy = (double)n * a.inv_ly;
            const double k2 = kx * kx + kyy * kyy;
            th += a.chi_c1 * k2 + a.chi_c3 * k2 * k2;
          }
          th -= rint(th);
          float s, cth;
          sincospif(-2.0f * (float)th, &s, &cth);
          val = make_float2(cth * a.probe_norm, s * a.probe_norm);
        }
        v[q] = val;
      }
    } else if constexpr (MODE == COL_BEAM0 || MODE == COL_BEAM0_SPEC) {
      // the first slice of beam (m, n): the 2D transform of t_0 times the plane
      // wave exp(2 pi i (m x + n y) / N) is the transform of t_0 shifted by (m, n)
      const int2 mn = a.beams[wave];
      const float2* src = a.t0hat + ((col - mn.x) & (N - 1));
#pragma unroll
      for (int q = 0; q < E; ++q) v[q] = __ldg(src + (size_t)((t + q * T - mn.y) & (N - 1)) * N);
    } else {
#pragma unroll
      for (int q = 0; q < E; ++q) v[q] = w[(size_t)(t + q * T) * N];
    }
#if STEM_PREFETCH
    if constexpr (MODE != COL_PROBE_INIT && MODE != COL_BEAM0 && MODE != COL_BEAM0_SPEC) {
      // one prefetch per 32-byte sector of the next tile's column strip
      const int nt = tile + gridDim.x;
      if (nt < n_tiles && (c % (C < 4 ? C : 4)) == 0) {
        const int nct = nt % col_tiles;
        const float2* nw = a.wave + (size_t)(nt / col_tiles) * N * N + (BAND ? Cfg::band_tile(nct) : nct) * C + c;
#pragma unroll
        for (int q = 0; q < E; ++q) prefetch_l2(nw + (size_t)(t + q * T) * N);
      }
    }
#endif

    if constexpr (MODE == COL_SLICE || MODE == COL_DET || MODE == COL_FFT || MODE == COL_DP || MODE == COL_SPEC)
      fft_dist<N, false>(v, view, t, sync, tw);

    // COL_SPEC (the last slice of a cropped S-matrix) stores the propagated
    // spectrum M P FFT(.) / N^2 without the inverse transform
    if constexpr (MODE == COL_SLICE || MODE == COL_SPEC || MODE == COL_BEAM0 || MODE == COL_BEAM0_SPEC) {
      const int m = signed_freq(col, N);
      const float2 px = cscale(__ldg(a.prop_x + col), a.prop_scale);
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const int ky = t + q * T;
        const int n = signed_freq(ky, N);
        const bool keep = !all_out_of_band<N, T>(q) && 9 * (m * m + n * n) <= N * N;
        v[q] = keep ? cmul(v[q], cmul(px, __ldg(a.prop_y + ky))) : make_float2(0.0f, 0.0f);
      }
    }

    if constexpr (MODE == COL_SLICE || MODE == COL_PROBE_INIT || MODE == COL_IFFT || MODE == COL_BEAM0)
      fft_dist<N, true>(v, view, t, sync, tw);

    if constexpr (MODE == COL_DET) {
      __syncthreads();   // ring_acc zeroed; every thread is done with the exchange buffer
      if constexpr (Cfg::THREADS >= 32) {
        // (|psi|^2, ring) of the tile, column by column in row order, in the
        // exchange buffer (row stride S keeps the scattered writes free of bank
        // conflicts); then each warp takes runs of 32 consecutive rows of one
        // column, along which the ring index changes rarely (warp_run_add)
        constexpr int S = N + 16 / C;
        float2* pk = smem;
#pragma unroll
        for (int q = 0; q < E; ++q) {
          const int ky = t + q * T;
          const int r = __ldg(a.lut + (size_t)ky * N + col) & kLutNoRing;
          pk[c * S + ky] = make_float2(cabs2(v[q]), __int_as_float(r));
        }
        __syncthreads();
        constexpr int NW = Cfg::THREADS / 32;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 4
        for (int i = 0; i < E; ++i) {        // C * N / 32 runs of 32 elements, E per warp
          const int idx = (warp + NW * i) * 32 + lane;
          const float2 e = pk[(idx / N) * S + idx % N];
          warp_run_add(ring_acc, __float_as_int(e.y), e.x, kLutNoRing);
        }
      } else {
#pragma unroll
        for (int q = 0; q < E; ++q) {
          const int ky = t + q * T;
          const int r = __ldg(a.lut + (size_t)ky * N + col) & kLutNoRing;
          if (r != kLutNoRing) atomicAdd(ring_acc + r, cabs2(v[q]));
        }
      }
    } else if constexpr (MODE == COL_DP) {
      // 4D output: the whole diffraction pattern of the wave inside the 2/3
      // band limit (pixels outside it, including stale out-of-band columns of a
      // band tile, are left untouched)
      float* out = a.dp + (size_t)wave * N * N + col;
      const int m = signed_freq(col, N);
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const int ky = t + q * T;
        const int n = signed_freq(ky, N);
        if (9 * (m * m + n * n) <= N * N) out[(size_t)ky * N] += cabs2(v[q]) * a.ring_scale;
      }
    } else {
#pragma unroll
      for (int q = 0; q < E; ++q) w[(size_t)(t + q * T) * N] = v[q];
    }
  }
  if constexpr (DET) {
    __syncthreads();   // the last tile's sums are in ring_acc
    flush_rings(false);
  }
}

// ---------------------------------------------------------------------------
// Slice-loop column pass of the large transforms (N = 1024, 2048) moved by the
// tensor memory accelerator.  A tile (C = 4 columns x N rows, 64 KB at 2048)
// reaches shared memory as N / 256 2D tensor copies of 256 rows, one tile
// ahead of the transform (two buffers, one "full" mbarrier each), and leaves
// it the same way: the transformed tile is written back into its buffer and
// stored by N / 256 bulk tensor copies, after which the buffer takes the tile
// after next.  The slice pass is warp-specialised: C x T transform threads
// (synchronised among themselves by named barrier 1) and one copy warp whose
// lane 0 issues every tensor copy.  When the transform threads have written a
// tile back they arrive on the buffer's "done" mbarrier; the copy thread
// stores the tile, waits until the store has read the buffer and refills it,
// while the transform threads go on with the other buffer.  The threads issue
// no global loads or stores for the wave.  Every mbarrier wait is bounded; on
// timeout the kernel records STEM_ERR_TIMEOUT in the status word, waits
// (bounded) for its copies in flight and returns.  The detector variant (DET),
// the last pass of a multislice run, loads tiles the same way (all its threads
// compute; thread 0 issues the copies), squares the forward transform and sums
// it into the rings instead of storing anything.
// ---------------------------------------------------------------------------
#ifndef STEM_COL_TMA_MINB_1024
#define STEM_COL_TMA_MINB_1024 2
#endif
#ifndef STEM_COL_TMA_C_1024
#define STEM_COL_TMA_C_1024 4
#endif
template <int N_> struct ColTmaCfg {
  static constexpr int N = N_, E = FftShape<N>::E, T = N / E;
  static constexpr int C = N == 2048 ? 4 : STEM_COL_TMA_C_1024, THREADS = C * T;
  static constexpr int MINB = N == 2048 ? 1 : STEM_COL_TMA_MINB_1024;
  static constexpr int BOX_ROWS = 256, BOXES = N / BOX_ROWS;
  static constexpr uint32_t STAGE_BYTES = (uint32_t)N * C * sizeof(float2);   // 64 KB
  static constexpr uint32_t BOX_BYTES = STAGE_BYTES / BOXES;
  static constexpr size_t XBUF = (size_t)(N + N / E) * C * sizeof(float2);
  static constexpr size_t TW = (size_t)TwLayout<N>::TOTAL * sizeof(float2);
  static constexpr size_t SMEM = 1024 + 2 * (size_t)STAGE_BYTES + XBUF + TW + 64;
  static constexpr size_t SMEM_DET = SMEM + (size_t)kMaxRings * sizeof(float);   // + the tile's rings
  static constexpr int MB = N / 3;
  static constexpr int LO = (MB + 1 + C - 1) / C, HI0 = (N - MB) / C;
  static constexpr int BAND_TILES = LO + N / C - HI0;
  __device__ static int band_tile(int k) { return k >= LO ? k - LO + HI0 : k; }
  // threads per CTA: the slice pass adds the copy warp
  static constexpr int threads(bool det) { return det ? THREADS : THREADS + 32; }
};

template <int N_, bool DET>
__global__ void __launch_bounds__(ColTmaCfg<N_>::threads(DET), ColTmaCfg<N_>::MINB)
    k_col_slice_tma(const PassArgs a, const __grid_constant__ CUtensorMap map, int n_tiles) {
  using Cfg = ColTmaCfg<N_>;
  constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T, C = Cfg::C;
  constexpr int NT = Cfg::THREADS;   // transform threads
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  float2* stage = reinterpret_cast<float2*>(base);                        // [2][N][C]
  float2* xbuf = reinterpret_cast<float2*>(base + 2 * (size_t)Cfg::STAGE_BYTES);
  float2* tw = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(xbuf) + Cfg::XBUF);
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(tw) + Cfg::TW);
  // bars[0..1]: buffer full (tensor load landed); bars[2..3]: buffer done
  // (transformed tile written back; slice pass); bars[4] (an int): abort flag
  int* s_abort = reinterpret_cast<int*>(bars + 4);
  float* ring_acc = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(bars) + 64);   // DET only
  const int tid = threadIdx.x;
  const int c = tid % C, t = (tid / C) % T;
  const SmemView<E, C> view{xbuf + c};

  auto issue = [&](int tile, int b) {
    const int wave = tile / Cfg::BAND_TILES;
    const int col0 = Cfg::band_tile(tile % Cfg::BAND_TILES) * C;
    const uint32_t bar = smem_u32(bars + b);
    const uint32_t dst = smem_u32(stage + (size_t)b * N * C);
    mbar_arrive_expect_tx(bar, Cfg::STAGE_BYTES);
#pragma unroll
    for (int y = 0; y < Cfg::BOXES; ++y)
      tma_load_3d(dst + y * Cfg::BOX_BYTES, &map, 2 * col0, y * Cfg::BOX_ROWS, wave, bar);
  };

  if (tid == 0) {
    // full: one arrival (the copy thread's expect_tx); done: one per transform warp
    for (int i = 0; i < 4; ++i) mbar_init(smem_u32(bars + i), i < 2 ? 1 : NT / 32);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  build_twiddles<N>(tw, tid, Cfg::threads(DET));
  __syncthreads();
  // the copy thread: thread 0 of the detector variant, lane 0 of the copy warp otherwise
  const bool copier = DET ? tid == 0 : tid == NT;
  if (copier) {
    if (blockIdx.x < n_tiles) issue(blockIdx.x, 0);
    if (blockIdx.x + gridDim.x < n_tiles) issue(blockIdx.x + gridDim.x, 1);
  }

  if constexpr (!DET) {
    if (tid >= NT) {
      // ------------------------------------------------------------ copy warp
      if (tid == NT) {
        int k = 0;
        bool failed = false;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++k) {
          const int b = k & 1;
          if (!mbar_wait(smem_u32(bars + 2 + b), (uint32_t)(k >> 1) & 1u)) { failed = true; break; }
          if (*reinterpret_cast<volatile int*>(s_abort)) { failed = true; break; }
          const int wave = tile / Cfg::BAND_TILES;
          const int col0 = Cfg::band_tile(tile % Cfg::BAND_TILES) * C;
          const uint32_t src = smem_u32(stage + (size_t)b * N * C);
#pragma unroll
          for (int y = 0; y < Cfg::BOXES; ++y)
            tma_store_3d(&map, 2 * col0, y * Cfg::BOX_ROWS, wave, src + y * Cfg::BOX_BYTES);
          bulk_commit();
          if (tile + 2 * gridDim.x < n_tiles) {
            bulk_wait_read();   // buffer b is read out: refill it with the tile after next
            issue(tile + 2 * gridDim.x, b);
          }
        }
        bulk_wait_all();
        if (failed) {
          if (a.status) atomicExch(a.status, (int)STEM_ERR_TIMEOUT);
          // let the loads already issued into this CTA's buffers land before it
          // exits: tiles k and k + 1 may still be in flight
          int tile = blockIdx.x + k * gridDim.x;
          for (int j = 0; j < 2 && tile < n_tiles; ++j, ++k, tile += gridDim.x)
            mbar_wait(smem_u32(bars + (k & 1)), (uint32_t)(k >> 1) & 1u);
        }
      }
      return;
    }
    // -------------------------------------------------------- transform threads
    auto sync = [] { named_sync(1, NT); };
    int k = 0;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++k) {
      const int b = k & 1;
      const bool ok = mbar_wait(smem_u32(bars + b), (uint32_t)(k >> 1) & 1u);
      if (named_sync_or(1, NT, !ok)) {
        // hand the outcome to the copy thread, which records it and drains
        if (tid == 0) *s_abort = 1;
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive_one(smem_u32(bars + 2 + b));
        break;
      }
      float2* st = stage + (size_t)b * N * C;
      float2 v[E];
#pragma unroll
      for (int q = 0; q < E; ++q) v[q] = st[(t + q * T) * C + c];
      const int col = Cfg::band_tile(tile % Cfg::BAND_TILES) * C + c;
      // the barrier that ended the previous tile follows its last reads of xbuf
      fft_dist<N, false, false>(v, view, t, sync, tw);
      const int m = signed_freq(col, N);
      const float2 px = cscale(__ldg(a.prop_x + col), a.prop_scale);
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const int ky = t + q * T;
        const int n = signed_freq(ky, N);
        const bool keep = !all_out_of_band<N, T>(q) && 9 * (m * m + n * n) <= N * N;
        v[q] = keep ? cmul(v[q], cmul(px, __ldg(a.prop_y + ky))) : make_float2(0.0f, 0.0f);
      }
      fft_dist<N, true>(v, view, t, sync, tw);
#pragma unroll
      for (int q = 0; q < E; ++q) st[(t + q * T) * C + c] = v[q];
      fence_proxy_async();   // these writes before the tensor store reads them
      __syncwarp();
      // one arrival per transform warp (the next tile's barrier orders the
      // reuse of xbuf)
      if ((tid & 31) == 0) mbar_arrive_one(smem_u32(bars + 2 + b));
    }
  } else {
    auto sync = [] { __syncthreads(); };
    int k = 0;
    bool aborted = false;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++k) {
      const int b = k & 1;
      const bool ok = mbar_wait(smem_u32(bars + b), (uint32_t)(k >> 1) & 1u);
      if (__syncthreads_or(!ok)) {
        aborted = true;
        break;
      }
      float2* st = stage + (size_t)b * N * C;
      float2 v[E];
#pragma unroll
      for (int q = 0; q < E; ++q) v[q] = st[(t + q * T) * C + c];
      const int wave = tile / Cfg::BAND_TILES;
      const int col0 = Cfg::band_tile(tile % Cfg::BAND_TILES) * C;
      // nothing is stored back, so the buffer takes the tile after next as
      // soon as every thread holds its values; the rings of the previous tile
      // have been flushed, so they can be cleared
      __syncthreads();
      if (tid == 0 && tile + 2 * gridDim.x < n_tiles) issue(tile + 2 * gridDim.x, b);
      for (int i = tid; i < a.n_rings; i += NT) ring_acc[i] = 0.0f;
      fft_dist<N, false>(v, view, t, sync, tw);
      // |Psi_hat|^2 of each pixel, column by column in row order (row stride S
      // keeps the scattered writes free of bank conflicts); each warp then sums
      // runs of 32 consecutive rows of one column (warp_run_add), reading their
      // rings from the transposed table in one contiguous 64-byte load
      constexpr int S = N + 32 / C;
      float* pk = reinterpret_cast<float*>(xbuf);
      __syncthreads();
#pragma unroll
      for (int q = 0; q < E; ++q) pk[c * S + t + q * T] = cabs2(v[q]);
      __syncthreads();
      constexpr int NW = NT / 32;
      const int lane = tid & 31, warp = tid >> 5;
#pragma unroll 4
      for (int i = 0; i < E; ++i) {
        const int idx = (warp + NW * i) * 32 + lane;
        const int cc = idx / N, row = idx % N;
        const int r = __ldg(a.lut_t + (size_t)(col0 + cc) * N + row) & kLutNoRing;
        warp_run_add(ring_acc, r, pk[cc * S + row], kLutNoRing);
      }
      __syncthreads();
      float* out = a.rings + (size_t)wave * a.n_rings;
      for (int i = tid; i < a.n_rings; i += NT) {
        const float acc = ring_acc[i];
        if (acc != 0.0f) atomicAdd(out + i, acc * a.ring_scale);
      }
    }
    if (aborted && tid == 0) {
      if (a.status) atomicExch(a.status, (int)STEM_ERR_TIMEOUT);
      // let the copies already issued into this CTA's buffers land before it exits
      int tile = blockIdx.x + k * gridDim.x;
      for (int j = 0; j < 2 && tile < n_tiles; ++j, ++k, tile += gridDim.x)
        mbar_wait(smem_u32(bars + (k & 1)), (uint32_t)(k >> 1) & 1u);
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers.  The dynamic shared-memory opt-in is set once per kernel in this
// process (the library drives the device that was current at plan creation).
// ---------------------------------------------------------------------------
template <class K>
static cudaError_t set_smem(K kernel, size_t bytes, std::once_flag& flag) {
  cudaError_t err = cudaSuccess;
  std::call_once(flag, [&] {
    err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  });
  return err;
}

// Persistent grid: as many CTAs as fit on the device at once, capped by the
// number of tiles.
template <class K>
static int resident_ctas(K kernel, int threads, size_t smem, std::once_flag& flag, int& cached) {
  std::call_once(flag, [&] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
    cached = (sms > 0 ? sms : 148) * (per > 0 ? per : 1);
  });
  return cached;
}

template <int N, int MODE>
static cudaError_t row_launch(const PassArgs& a, cudaStream_t s) {
  using Cfg = RowCfg<N>;
  static std::once_flag flag, occ_flag;
  static int occ = 0;
  cudaError_t e = set_smem(k_row_pass<N, MODE>, Cfg::SMEM, flag);
  if (e != cudaSuccess) return e;
  const int n_tiles = a.batch * (N / Cfg::ROWS);
  const int grid = std::min(n_tiles, resident_ctas(k_row_pass<N, MODE>, Cfg::THREADS, Cfg::SMEM, occ_flag, occ));
  ProfScope prof(MODE == ROW_SLICE ? STEM_PROF_ROW_SLICE : -1, s);
  note_launch(), k_row_pass<N, MODE><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(a, n_tiles);
  return cudaGetLastError();
}

template <int N, int MODE, bool BAND>
static cudaError_t col_launch(const PassArgs& a, cudaStream_t s) {
  using Cfg = ColCfg<N>;
  const size_t smem = Cfg::FFT_SMEM + (MODE == COL_DET ? kMaxRings * sizeof(float) : 0);
  static std::once_flag flag, occ_flag;
  static int occ = 0;
  cudaError_t e = set_smem(k_col_pass<N, MODE, BAND>, smem, flag);
  if (e != cudaSuccess) return e;
  const int n_tiles = a.batch * (BAND ? Cfg::BAND_TILES : N / Cfg::C);
  const int grid = std::min(n_tiles, resident_ctas(k_col_pass<N, MODE, BAND>, Cfg::THREADS, smem, occ_flag, occ));
  ProfScope prof(MODE == COL_SLICE ? STEM_PROF_COL_SLICE : -1, s);
  note_launch(), k_col_pass<N, MODE, BAND><<<grid, Cfg::THREADS, smem, s>>>(a, n_tiles);
  return cudaGetLastError();
}

static cudaError_t row_slice_pair_2048(const PassArgs& a, cudaStream_t s) {
  using Cfg = RowPairCfg;
  static std::once_flag flag, occ_flag;
  static int occ = 0;
  // the bulk copies read rows of the waves and of t_n from 16-byte boundaries
  if (reinterpret_cast<uintptr_t>(a.wave) % 16 || reinterpret_cast<uintptr_t>(a.trans) % 16)
    return cudaErrorInvalidValue;
  cudaError_t e = set_smem(k_row_slice_pair_2048, Cfg::SMEM, flag);
  if (e != cudaSuccess) return e;
  const int n_tiles = ((a.batch + 1) / 2) * Cfg::N;
  const int grid = std::min(n_tiles, resident_ctas(k_row_slice_pair_2048, Cfg::THREADS, Cfg::SMEM, occ_flag, occ));
  ProfScope prof(STEM_PROF_ROW_SLICE, s);
  note_launch(), k_row_slice_pair_2048<<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(a, n_tiles);
  return cudaGetLastError();
}

template <int N>
static cudaError_t row_dispatch(int mode, const PassArgs& a, cudaStream_t s) {
  if constexpr (N == 2048)
    if (mode == ROW_SLICE) return row_slice_pair_2048(a, s);
  switch (mode) {
    case ROW_FFT: return row_launch<N, ROW_FFT>(a, s);
    case ROW_IFFT: return row_launch<N, ROW_IFFT>(a, s);
    default: break;
  }
  if constexpr (N >= 64) {
    switch (mode) {
      case ROW_SLICE: return row_launch<N, ROW_SLICE>(a, s);
      case ROW_IFFT_MAX: return row_launch<N, ROW_IFFT_MAX>(a, s);
      default: break;
    }
  }
  return cudaErrorInvalidValue;
}

#ifndef STEM_COL_TMA
#define STEM_COL_TMA 1
#endif
#ifndef STEM_COL_TMA_1024
#define STEM_COL_TMA_1024 1
#endif
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag flag;
  std::call_once(flag, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// The waves [batch][N][N] of complex64 as a 3D FP32 tensor (2N, N, batch),
// boxes of C complex columns x 256 rows.
template <int N>
static cudaError_t wave_tensor_map(const PassArgs& a, CUtensorMap* map) {
  using Cfg = ColTmaCfg<N>;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  if (reinterpret_cast<uintptr_t>(a.wave) % 16) return cudaErrorInvalidValue;
  const cuuint64_t dims[3] = {2ull * Cfg::N, (cuuint64_t)Cfg::N, (cuuint64_t)a.batch};
  const cuuint64_t strides[2] = {2ull * Cfg::N * sizeof(float), 2ull * Cfg::N * Cfg::N * sizeof(float)};
  const cuuint32_t box[3] = {2u * Cfg::C, (cuuint32_t)Cfg::BOX_ROWS, 1u};
  const cuuint32_t estride[3] = {1u, 1u, 1u};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.wave, dims, strides, box, estride,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int N, bool DET>
static cudaError_t col_slice_tma(const PassArgs& a, cudaStream_t s) {
  using Cfg = ColTmaCfg<N>;
  static std::once_flag flag, occ_flag;
  static int occ = 0;
  cudaError_t e = set_smem(k_col_slice_tma<N, DET>, DET ? Cfg::SMEM_DET : Cfg::SMEM, flag);
  if (e != cudaSuccess) return e;
  CUtensorMap map;
  if ((e = wave_tensor_map<N>(a, &map)) != cudaSuccess) return e;
  const int n_tiles = a.batch * Cfg::BAND_TILES;
  int grid;
  size_t smem = Cfg::SMEM;
  if constexpr (DET) {
    // the detector variant holds only this plan's rings, so that more CTAs fit
    smem += ((size_t)a.n_rings * sizeof(float) + 15) / 16 * 16;
    int dev = 0, sms = 148, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_col_slice_tma<N, DET>, Cfg::threads(DET), smem);
    grid = std::min(n_tiles, sms * std::max(per, 1));
  } else {
    grid = std::min(n_tiles, resident_ctas(k_col_slice_tma<N, DET>, Cfg::threads(DET), smem, occ_flag, occ));
  }
  ProfScope prof(DET ? -1 : STEM_PROF_COL_SLICE, s);
  note_launch(), k_col_slice_tma<N, DET><<<grid, Cfg::threads(DET), smem, s>>>(a, map, n_tiles);
  return cudaGetLastError();
}

// Slice-loop column passes visit only the column tiles inside the band limit;
// the detector pass does so when it ends a multislice run (a.band), not when
// it reads PRISM windows or other full fields.
template <int N>
static cudaError_t col_dispatch(int mode, const PassArgs& a, cudaStream_t s) {
#if STEM_COL_TMA
  // the detector pass that ends a slice loop reads only in-band column tiles
  if constexpr (N == 2048 || N == 1024)
    if (mode == COL_DET && a.band) return col_slice_tma<N, true>(a, s);
#endif
  switch (mode) {
    case COL_DET: return a.band ? col_launch<N, COL_DET, true>(a, s) : col_launch<N, COL_DET, false>(a, s);
    case COL_DP: return a.band ? col_launch<N, COL_DP, true>(a, s) : col_launch<N, COL_DP, false>(a, s);
    case COL_FFT: return col_launch<N, COL_FFT, false>(a, s);
    case COL_IFFT: return col_launch<N, COL_IFFT, false>(a, s);
    default: break;
  }
#if STEM_COL_TMA
  if constexpr (N == 2048)
    if (mode == COL_SLICE) return col_slice_tma<2048, false>(a, s);
#endif
#if STEM_COL_TMA_1024
  if constexpr (N == 1024)
    if (mode == COL_SLICE) return col_slice_tma<1024, false>(a, s);
#endif
  if constexpr (N >= 64) {
    switch (mode) {
      case COL_SLICE: return col_launch<N, COL_SLICE, true>(a, s);
      case COL_PROBE_INIT: return col_launch<N, COL_PROBE_INIT, true>(a, s);
      case COL_SPEC: return col_launch<N, COL_SPEC, true>(a, s);
      case COL_BEAM0: return col_launch<N, COL_BEAM0, true>(a, s);
      case COL_BEAM0_SPEC: return col_launch<N, COL_BEAM0_SPEC, true>(a, s);
      default: break;
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_row_pass(int n, int mode, const PassArgs& a, cudaStream_t s) {
  if (a.batch <= 0) return cudaSuccess;
  switch (n) {
    case 8: return row_dispatch<8>(mode, a, s);
    case 16: return row_dispatch<16>(mode, a, s);
    case 32: return row_dispatch<32>(mode, a, s);
    case 64: return row_dispatch<64>(mode, a, s);
    case 128: return row_dispatch<128>(mode, a, s);
    case 256: return row_dispatch<256>(mode, a, s);
    case 512: return row_dispatch<512>(mode, a, s);
    case 1024: return row_dispatch<1024>(mode, a, s);
    case 2048: return row_dispatch<2048>(mode, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_col_pass(int n, int mode, const PassArgs& a, cudaStream_t s) {
  if (a.batch <= 0) return cudaSuccess;
  switch (n) {
    case 8: return col_dispatch<8>(mode, a, s);
    case 16: return col_dispatch<16>(mode, a, s);
    case 32: return col_dispatch<32>(mode, a, s);
    case 64: return col_dispatch<64>(mode, a, s);
    case 128: return col_dispatch<128>(mode, a, s);
    case 256: return col_dispatch<256>(mode, a, s);
    case 512: return col_dispatch<512>(mode, a, s);
    case 1024: return col_dispatch<1024>(mode, a, s);
    case 2048: return col_dispatch<2048>(mode, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stem
