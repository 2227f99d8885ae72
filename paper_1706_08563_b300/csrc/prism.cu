// prism.cu - PRISM: S-matrix storage, probe coefficients, window bookkeeping and
// the FP32 CUDA-core beam sum.
//
// "PRISM Probe Simulations": the compact S-matrix holds every selected plane
// wave's exit wave in real space, stored so that the beams of one pixel are
// contiguous (the paper's layout, beams along the fastest axis).  The output of
// a probe is the coefficient-weighted beam sum over a W x W window (W = N/f)
// around the probe ("Description of Algorithms", PRISM paragraph).
//
// The beam sum is organised as a complex GEMM over absolute pixels: a 16 x 8
// pixel tile of the S-matrix ([128 pixels] x [beams]) times the coefficients of
// every probe whose window touches that tile ([beams] x [probes]).  A pixel of a
// window is computed exactly once (by the tile that contains it), with the full
// sum over beams in a fixed order.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fft_core.cuh"
#include "internal.h"

namespace stem {

constexpr int kTileX = 16, kTileY = 8, kTilePix = kTileX * kTileY;

SmatLayout smatrix_layout(int n, int n_beams, int storage) {
  SmatLayout L;
  L.n_beams = n_beams;
  L.nbp = ((n_beams + 63) / 64) * 64;
  L.elem_bytes = storage == STEM_F32 ? 4 : 2;
  L.data_offset = ((size_t)L.nbp * 4 + 255) / 256 * 256;
  L.total = L.data_offset + (size_t)n * n * 2 * L.nbp * L.elem_bytes;
  return L;
}

template <int S> struct Elem;
template <> struct Elem<STEM_F32> {
  using T = float;
  __device__ static T from(float x) { return x; }
  __device__ static float to(T x) { return x; }
};
template <> struct Elem<STEM_F16> {
  using T = __half;
  __device__ static T from(float x) { return __float2half_rn(x); }
  __device__ static float to(T x) { return __half2float(x); }
};
template <> struct Elem<STEM_BF16> {
  using T = __nv_bfloat16;
  __device__ static T from(float x) { return __float2bfloat16_rn(x); }
  __device__ static float to(T x) { return __bfloat162float(x); }
};

// ---------------------------------------------------------------------------
// S-matrix store: waves [nb][N*N] (real-space exit waves of beams b0..b0+nb)
// -> data[R][re|im][b], divided by the per-beam power-of-two scale.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float pow2_scale(unsigned max_bits, int storage) {
  if (storage == STEM_F32) return 1.0f;
  const float m = __uint_as_float(max_bits);
  if (!(m > 0.0f)) return 1.0f;
  int e;
  frexpf(m, &e);          // m = frac * 2^e, frac in [0.5, 1)
  return ldexpf(1.0f, e);
}

template <int S>
__global__ void k_smatrix_store(const float2* __restrict__ waves, int nb, int n, int n_out, int b0,
                                const unsigned* __restrict__ beam_max, int nbp, float* __restrict__ scales,
                                typename Elem<S>::T* __restrict__ data) {
  __shared__ float2 tile[32][33];
  __shared__ float inv_scale[32];
  const int pix0 = blockIdx.x * 32;
  const int bl0 = blockIdx.y * 32;          // local beam index within this batch
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
  if (threadIdx.x < 32) {
    const int bl = bl0 + threadIdx.x;
    float sc = 1.0f;
    if (bl < nb) {
      sc = pow2_scale(beam_max[bl], S);
      if (blockIdx.x == 0) scales[b0 + bl] = sc;
    }
    inv_scale[threadIdx.x] = 1.0f / sc;
  }
  for (int k = ty; k < 32; k += 8) {
    const int bl = bl0 + k;
    const int pix = pix0 + tx;   // pixel (pix / n_out, pix % n_out) of the stored grid
    tile[k][tx] = bl < nb ? waves[(size_t)bl * n * n + (size_t)(pix / n_out) * n + pix % n_out]
                          : make_float2(0.0f, 0.0f);
  }
  __syncthreads();
  const int bl = bl0 + tx;
  if (bl < nb) {
    for (int k = ty; k < 32; k += 8) {
      const size_t r = (size_t)(pix0 + k);
      const float2 v = tile[tx][k];
      data[r * 2 * nbp + b0 + bl] = Elem<S>::from(v.x * inv_scale[tx]);
      data[r * 2 * nbp + nbp + b0 + bl] = Elem<S>::from(v.y * inv_scale[tx]);
    }
  }
}

// zero the padded beams [n_beams, nbp) and give them scale 1
template <int S>
__global__ void k_smatrix_pad(int npix, int n_beams, int nbp, float* scales, typename Elem<S>::T* data) {
  const int pad = nbp - n_beams;
  const size_t total = (size_t)npix * 2 * pad;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t r = i / (2 * pad);
    const int rem = (int)(i % (2 * pad));
    const int plane = rem / pad, b = n_beams + rem % pad;
    data[r * 2 * nbp + plane * nbp + b] = Elem<S>::from(0.0f);
  }
  if (blockIdx.x == 0)
    for (int b = n_beams + threadIdx.x; b < nbp; b += blockDim.x) scales[b] = 1.0f;
}

template <int S>
static void store_typed(const float2* waves, int nb, int n, int n_out, int b0, int n_beams_total,
                        const unsigned* beam_max, const SmatLayout& L, float* scales, char* data, cudaStream_t s) {
  using T = typename Elem<S>::T;
  const int npix = n_out * n_out;
  dim3 grid(npix / 32, (nb + 31) / 32);
  note_launch(), k_smatrix_store<S><<<grid, 256, 0, s>>>(waves, nb, n, n_out, b0, beam_max, L.nbp, scales,
                                                        reinterpret_cast<T*>(data));
  if (b0 + nb >= n_beams_total && L.nbp > n_beams_total)
    note_launch(), k_smatrix_pad<S><<<1024, 256, 0, s>>>(npix, n_beams_total, L.nbp, scales, reinterpret_cast<T*>(data));
}

cudaError_t launch_smatrix_store(const float2* waves, int nb, int n, int n_out, int b0, int n_beams_total,
                                 const unsigned* beam_max, int storage, const SmatLayout& L, void* smatrix,
                                 cudaStream_t s) {
  float* scales = static_cast<float*>(smatrix);
  char* data = static_cast<char*>(smatrix) + L.data_offset;
  switch (storage) {
    case STEM_F32: store_typed<STEM_F32>(waves, nb, n, n_out, b0, n_beams_total, beam_max, L, scales, data, s); break;
    case STEM_F16: store_typed<STEM_F16>(waves, nb, n, n_out, b0, n_beams_total, beam_max, L, scales, data, s); break;
    case STEM_BF16: store_typed<STEM_BF16>(waves, nb, n, n_out, b0, n_beams_total, beam_max, L, scales, data, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Output-step workspace
// ---------------------------------------------------------------------------
static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

OutputWs output_workspace_layout(int n, int f, int chunk, int nbp) {
  OutputWs L;
  const int w = n / f;
  const size_t ntx = (size_t)(n / kTileX), nty = (size_t)(n / kTileY);
  const size_t n_tiles = ntx * nty;
  const size_t tx = (size_t)((w + kTileX - 1) / kTileX + 1), ty = (size_t)((w + kTileY - 1) / kTileY + 1);
  const size_t per_probe = (tx < ntx ? tx : ntx) * (ty < nty ? ty : nty);
  size_t off = 0;
  L.coef = off;    off += align256((size_t)chunk * 2 * nbp * sizeof(float));
  L.origin = off;  off += align256((size_t)chunk * sizeof(int2));
  L.counts = off;  off += align256(n_tiles * sizeof(int));
  L.offsets = off; off += align256((n_tiles + 1) * sizeof(int));
  L.work = off;    off += align256((n_tiles + 1) * sizeof(int));
  // items: at most one partial group per tile plus chunk * per_probe / 64 full ones
  L.items = off;   off += align256((n_tiles + (size_t)chunk * per_probe / 64 + 1) * sizeof(int));
  L.list = off;    off += align256((size_t)chunk * per_probe * sizeof(int));
  L.windows = off; off += align256((size_t)chunk * w * w * sizeof(float2));
  L.total = off;
  return L;
}

// c[p][re|im][b] = exp(-i chi(k_b)) exp(-2 pi i (m_b x_p / Lx + n_b y_p / Ly)) * norm * s_b;
// the phase (in turns) is reduced modulo 1 in FP64 before the FP32 sine/cosine.
__global__ void k_coefficients(const double* __restrict__ xy, const int2* __restrict__ beams,
                               const double* __restrict__ turns, int n_beams, int nbp,
                               const float* __restrict__ scales, double inv_lx, double inv_ly, float norm,
                               float* __restrict__ coef) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (b >= nbp) return;
  float re = 0.0f, im = 0.0f;
  if (b < n_beams) {
    const int2 mn = beams[b];
    double th = (double)mn.x * xy[2 * p] * inv_lx + (double)mn.y * xy[2 * p + 1] * inv_ly + turns[b];
    th -= rint(th);
    float s, c;
    sincospif(-2.0f * (float)th, &s, &c);
    const float g = norm * scales[b];
    re = c * g;
    im = s * g;
  }
  coef[(size_t)p * 2 * nbp + b] = re;
  coef[(size_t)p * 2 * nbp + nbp + b] = im;
}

__device__ __forceinline__ void tile_span(int2 o, int n, int w, int& cx, int& cy) {
  const int ntx = n / kTileX, nty = n / kTileY;
  cx = (o.x + w - 1) / kTileX - o.x / kTileX + 1;
  cy = (o.y + w - 1) / kTileY - o.y / kTileY + 1;
  cx = cx > ntx ? ntx : cx;
  cy = cy > nty ? nty : cy;
}

// Window origin of each probe (round half up, minus W/2, modulo N).
__global__ void k_origins(const double* __restrict__ xy, int np, int n, int w, double dx, double dy,
                          int2* __restrict__ origin) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const long long ox = (long long)floor(xy[2 * p] / dx + 0.5) - w / 2;
  const long long oy = (long long)floor(xy[2 * p + 1] / dy + 0.5) - w / 2;
  const int2 o = make_int2((int)((ox % n + n) % n), (int)((oy % n + n) % n));
  origin[p] = o;
}

// One warp per probe: count the probe in every pixel tile its window touches
// (a window of W = 256 touches about 560 tiles; the lanes share them).
__global__ void k_count_tiles(const int2* __restrict__ origin, int np, int n, int w, int* __restrict__ counts) {
  const int p = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (p >= np) return;
  const int2 o = origin[p];
  const int ntx = n / kTileX, nty = n / kTileY;
  int cx, cy;
  tile_span(o, n, w, cx, cy);
  for (int i = lane; i < cx * cy; i += 32) {
    const int iy = i / cx, ix = i % cx;
    const int tx = (o.x / kTileX + ix) % ntx, ty = (o.y / kTileY + iy) % nty;
    atomicAdd(counts + ty * ntx + tx, 1);
  }
}

// Exclusive scans of the tiles' probe counts (offsets into the probe lists)
// and of their work items (ceil(count / group)) in one CTA of 1024 threads:
// chunks of 4096 tiles, 4 consecutive tiles per thread (coalesced), a
// shuffle scan per warp, the warps' totals scanned by warp 0, and a running
// carry across chunks.  counts become zeroed fill cursors.
__global__ void __launch_bounds__(1024) k_scan_tiles(int* __restrict__ counts, int n_tiles, int group,
                                                     int* __restrict__ offsets, int* __restrict__ work) {
  __shared__ int s_wa[32], s_wb[32], s_carry[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry[0] = s_carry[1] = 0;
  for (int base = 0; base < n_tiles; base += 4 * 1024) {
    const int i0 = base + 4 * threadIdx.x;
    int c[4], a = 0, b = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      c[u] = i0 + u < n_tiles ? counts[i0 + u] : 0;
      a += c[u];
      b += (c[u] + group - 1) / group;
    }
    int ia = a, ib = b;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int oa = __shfl_up_sync(0xffffffffu, ia, d), ob = __shfl_up_sync(0xffffffffu, ib, d);
      if (lane >= d) { ia += oa; ib += ob; }
    }
    __syncthreads();   // s_carry from the previous chunk is final; s_wa/s_wb free
    if (lane == 31) { s_wa[warp] = ia; s_wb[warp] = ib; }
    __syncthreads();
    if (warp == 0) {
      int wa = s_wa[lane], wb = s_wb[lane];
      const int xa = wa, xb = wb;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int oa = __shfl_up_sync(0xffffffffu, wa, d), ob = __shfl_up_sync(0xffffffffu, wb, d);
        if (lane >= d) { wa += oa; wb += ob; }
      }
      s_wa[lane] = wa - xa;   // exclusive prefix of the warps' totals
      s_wb[lane] = wb - xb;
    }
    __syncthreads();
    int fa = s_carry[0] + s_wa[warp] + ia - a, fb = s_carry[1] + s_wb[warp] + ib - b;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i0 + u < n_tiles) {
        offsets[i0 + u] = fa;
        work[i0 + u] = fb;
        counts[i0 + u] = 0;
        fa += c[u];
        fb += (c[u] + group - 1) / group;
      }
    __syncthreads();   // every thread has read s_carry
    if (threadIdx.x == 1023) { s_carry[0] = fa; s_carry[1] = fb; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    offsets[n_tiles] = s_carry[0];
    work[n_tiles] = s_carry[1];
  }
}

// items[g] = t for every work item g of tile t (a direct look-up instead of a
// search over the item offsets)
__global__ void k_item_tiles(const int* __restrict__ work, int n_tiles, int* __restrict__ items) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  for (int g = work[t]; g < work[t + 1]; ++g) items[g] = t;
}

// One warp per probe: append the probe to the list of every tile its window
// touches (list order within a tile is arbitrary; every window pixel is still
// computed once, with its full beam sum in a fixed order).
__global__ void k_fill_tiles(const int2* __restrict__ origin, int np, int n, int w, const int* __restrict__ offsets,
                             int* __restrict__ cursor, int* __restrict__ list) {
  const int p = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (p >= np) return;
  const int2 o = origin[p];
  const int ntx = n / kTileX, nty = n / kTileY;
  int cx, cy;
  tile_span(o, n, w, cx, cy);
  for (int i = lane; i < cx * cy; i += 32) {
    const int iy = i / cx, ix = i % cx;
    const int t = ((o.y / kTileY + iy) % nty) * ntx + (o.x / kTileX + ix) % ntx;
    list[offsets[t] + atomicAdd(cursor + t, 1)] = p;
  }
}

// ---------------------------------------------------------------------------
// FP32 CUDA-core beam sum.  Work item = (pixel tile, group of up to 64 probes
// of that tile's list).  256 threads; a thread owns 4 pixels x 8 probes.
// ---------------------------------------------------------------------------
constexpr int kGroup = 64;
constexpr int kKb = 16;

template <int S>
__global__ void __launch_bounds__(256) k_beam_sum_simt(
    const typename Elem<S>::T* __restrict__ sdata, int n, int w, int nbp, const float* __restrict__ coef,
    const int2* __restrict__ origin, const int* __restrict__ offsets, const int* __restrict__ work,
    const int* __restrict__ items, const int* __restrict__ list, int n_tiles, float2* __restrict__ windows) {
  __shared__ float2 s_sm[kKb][kTilePix];
  __shared__ float2 c_sm[kKb][kGroup];
  __shared__ int p_sm[kGroup];
  const int total = __ldg(work + n_tiles);
  const int ntx = n / kTileX;
  const int pxg = threadIdx.x & 31;        // pixels 4 pxg .. 4 pxg + 3
  const int prg = threadIdx.x >> 5;        // probes 8 prg .. 8 prg + 7
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int tile = __ldg(items + item);
    const int g0 = (item - __ldg(work + tile)) * kGroup;
    const int first = __ldg(offsets + tile);
    const int cnt = min(kGroup, __ldg(offsets + tile + 1) - first - g0);
    const int x0 = (tile % ntx) * kTileX, y0 = (tile / ntx) * kTileY;
    __syncthreads();
    if (threadIdx.x < kGroup) p_sm[threadIdx.x] = (int)threadIdx.x < cnt ? __ldg(list + first + g0 + threadIdx.x) : -1;
    float2 acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = make_float2(0.0f, 0.0f);
    for (int k0 = 0; k0 < nbp; k0 += kKb) {
      __syncthreads();
      for (int i = threadIdx.x; i < kTilePix * kKb; i += 256) {
        const int b = i % kKb, px = i / kKb;
        const size_t r = (size_t)(y0 + px / kTileX) * n + x0 + px % kTileX;
        const float re = Elem<S>::to(sdata[r * 2 * nbp + k0 + b]);
        const float im = Elem<S>::to(sdata[r * 2 * nbp + nbp + k0 + b]);
        s_sm[b][px] = make_float2(re, im);
      }
      for (int i = threadIdx.x; i < kGroup * kKb; i += 256) {
        const int b = i % kKb, pl = i / kKb;
        const int p = p_sm[pl];
        c_sm[b][pl] = p >= 0 ? make_float2(coef[(size_t)p * 2 * nbp + k0 + b], coef[(size_t)p * 2 * nbp + nbp + k0 + b])
                             : make_float2(0.0f, 0.0f);
      }
      __syncthreads();
#pragma unroll 4
      for (int b = 0; b < kKb; ++b) {
        float2 sv[4], cv[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) sv[i] = s_sm[b][4 * pxg + i];
#pragma unroll
        for (int j = 0; j < 8; ++j) cv[j] = c_sm[b][8 * prg + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            acc[i][j].x = fmaf(sv[i].x, cv[j].x, fmaf(-sv[i].y, cv[j].y, acc[i][j].x));
            acc[i][j].y = fmaf(sv[i].x, cv[j].y, fmaf(sv[i].y, cv[j].x, acc[i][j].y));
          }
      }
    }
    // scatter into the probes' windows
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int p = p_sm[8 * prg + j];
      if (p < 0) continue;
      const int2 o = __ldg(origin + p);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int px = 4 * pxg + i;
        const int gx = x0 + px % kTileX, gy = y0 + px / kTileX;
        const int u = (gx - o.x + n) % n, v = (gy - o.y + n) % n;
        if (u < w && v < w) windows[((size_t)p * w + v) * w + u] = acc[i][j];
      }
    }
  }
}

cudaError_t prism_windows_chunk(const OutputArgs& o, const double* probe_xy, int np, float2* windows, char* ws,
                                const OutputWs& L, cudaStream_t s) {
  float* coef = reinterpret_cast<float*>(ws + L.coef);
  int2* origin = reinterpret_cast<int2*>(ws + L.origin);
  int* counts = reinterpret_cast<int*>(ws + L.counts);
  int* offsets = reinterpret_cast<int*>(ws + L.offsets);
  int* work = reinterpret_cast<int*>(ws + L.work);
  int* items = reinterpret_cast<int*>(ws + L.items);
  int* list = reinterpret_cast<int*>(ws + L.list);
  const int n = o.n, w = o.w;
  const int n_tiles = (n / kTileX) * (n / kTileY);
  const bool tensor = o.engine == STEM_SUM_TENSOR;
  const int group = tensor ? umma_group() : kGroup;
  cudaError_t e;

  dim3 cg((o.nbp + 127) / 128, np);
  if (!tensor) {
    note_launch(), k_coefficients<<<cg, 128, 0, s>>>(probe_xy, o.beams, o.beam_turns, o.n_beams, o.nbp, o.scales,
                                                    1.0 / o.lx, 1.0 / o.ly, o.coef_norm, coef);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = cudaMemsetAsync(counts, 0, n_tiles * sizeof(int), s)) != cudaSuccess) return e;
  note_launch(), k_origins<<<(np + 127) / 128, 128, 0, s>>>(probe_xy, np, n, w, o.dx, o.dy, origin);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const unsigned warp_blocks = (unsigned)(((size_t)np * 32 + 255) / 256);   // one warp per probe
  note_launch(), k_count_tiles<<<warp_blocks, 256, 0, s>>>(origin, np, n, w, counts);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  note_launch(), k_scan_tiles<<<1, 1024, 0, s>>>(counts, n_tiles, group, offsets, work);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  note_launch(), k_fill_tiles<<<warp_blocks, 256, 0, s>>>(origin, np, n, w, offsets, counts, list);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  note_launch(), k_item_tiles<<<(n_tiles + 255) / 256, 256, 0, s>>>(work, n_tiles, items);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  if (tensor)
    return launch_beam_sum_umma(o, np, probe_xy, coef, origin, offsets, work, items, list, n_tiles, windows, s);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)sms * 4;
  ProfScope prof(STEM_PROF_BEAM_SUM, s);
  switch (o.storage) {
    case STEM_F32:
      note_launch(), k_beam_sum_simt<STEM_F32><<<grid, 256, 0, s>>>(static_cast<const float*>(o.sdata), n, w, o.nbp, coef, origin,
                                                     offsets, work, items, list, n_tiles, windows);
      break;
    case STEM_F16:
      note_launch(), k_beam_sum_simt<STEM_F16><<<grid, 256, 0, s>>>(static_cast<const __half*>(o.sdata), n, w, o.nbp, coef, origin,
                                                     offsets, work, items, list, n_tiles, windows);
      break;
    case STEM_BF16:
      note_launch(), k_beam_sum_simt<STEM_BF16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(o.sdata), n, w, o.nbp, coef,
                                                      origin, offsets, work, items, list, n_tiles, windows);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace stem
