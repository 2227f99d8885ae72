// umma.cu - PRISM beam sum as a complex GEMM on the 5th-generation tensor cores.
//
// "Description of Algorithms" (PRISM paragraph) and "PRISM Probe Simulations"
// (last paragraph): every output probe is the coefficient-weighted sum of the
// S-matrix beams over its window.  For a 16 x 8 pixel tile of the S-matrix and
// a group of up to 128 probes whose windows touch the tile, this is
//   D[pixel][2p + h] = sum_k A[pixel][k] B[2p + h][k],   k in [0, 2 nbp)
// with A = [Re S | Im S] (the stored S-matrix row of the pixel, K-major) and
// B rows (p, re) = [Re c, -Im c], (p, im) = [Im c, Re c]: one real GEMM gives
// the real and imaginary parts.  M = 128 pixels, N = 256, K = 16 per
// tcgen05.mma (kind::f16, FP16 or BF16 in, FP32 accumulate in tensor memory).
//
// Per CTA (512 threads, one CTA per SM): all threads stage 64-wide K chunks of
// A and B into shared memory with cp.async in the 128-byte swizzled K-major
// layout (more loading warps keep more bytes in flight: 128 -> 256 -> 512
// threads took a 4096-probe output call at 2048^2 from 9.4 to 7.2 to 6.4 ms);
// thread 0 issues the MMAs and commits them to an mbarrier per stage; four
// stages keep the tensor pipe fed.  After the last chunk the warps read the
// accumulators with tcgen05.ld (a warp may read only the 32 lanes of its
// quarter, warp mod 4; the warps sharing a quarter split its columns) and
// scatter the pixels into the probes' windows.  Every wait is bounded (2 s of %globaltimer); on timeout the
// kernel records STEM_ERR_TIMEOUT in the plan's status word, drains its copies,
// frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "async_copy.cuh"
#include "internal.h"

namespace stem {

#ifndef STEM_UMMA_THREADS
#define STEM_UMMA_THREADS 512
#endif
constexpr int kUmmaThreads = STEM_UMMA_THREADS;   // 128 or 256: loaders; the epilogue splits columns
static_assert(kUmmaThreads == 128 || kUmmaThreads == 256 || kUmmaThreads == 512, "4, 8 or 16 warps");
constexpr int kUmmaStages = 4;
constexpr int kUmmaGroup = 128;                 // probes per work item (N = 256)
constexpr int kTileX = 16, kTileY = 8;          // must match prism.cu
constexpr int kAStage = 128 * 128;              // bytes: 128 rows x 64 halves
constexpr int kBStage = 256 * 128;              // bytes: 256 rows x 64 halves
constexpr int kStageBytes = kAStage + kBStage;
constexpr int kTmemCols = 256;

size_t umma_smem_bytes() { return (size_t)kUmmaStages * kStageBytes + 1024 + 2048; }
int umma_group() { return kUmmaGroup; }


__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }


// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator, A and B of the same
// 16-bit type (0 = FP16, 1 = BF16), both K-major, N = 256, M = 128.
__host__ __device__ constexpr uint32_t umma_idesc(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 64 consecutive accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&r)[64]) {
  uint32_t* u = reinterpret_cast<uint32_t*>(r);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
      "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
      "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
        "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]),
        "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]),
        "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31]),
        "=r"(u[32]), "=r"(u[33]), "=r"(u[34]), "=r"(u[35]), "=r"(u[36]), "=r"(u[37]), "=r"(u[38]), "=r"(u[39]),
        "=r"(u[40]), "=r"(u[41]), "=r"(u[42]), "=r"(u[43]), "=r"(u[44]), "=r"(u[45]), "=r"(u[46]), "=r"(u[47]),
        "=r"(u[48]), "=r"(u[49]), "=r"(u[50]), "=r"(u[51]), "=r"(u[52]), "=r"(u[53]), "=r"(u[54]), "=r"(u[55]),
        "=r"(u[56]), "=r"(u[57]), "=r"(u[58]), "=r"(u[59]), "=r"(u[60]), "=r"(u[61]), "=r"(u[62]), "=r"(u[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ int find_item_tile(const int* __restrict__ work, int n_tiles, int item) {
  int lo = 0, hi = n_tiles;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(work + mid) <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// Coefficients as the B operand: row (p, h) of length K = 2 nbp, 16-bit.
template <typename T>
__global__ void k_coefficients_umma(const double* __restrict__ xy, const int2* __restrict__ beams,
                                    const double* __restrict__ turns, int n_beams, int nbp,
                                    const float* __restrict__ scales, double inv_lx, double inv_ly, float norm,
                                    T* __restrict__ coef) {
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
  const size_t k2 = 2 * (size_t)nbp;
  T* r0 = coef + (size_t)p * 2 * k2;   // (p, re): [Re c | -Im c]
  T* r1 = r0 + k2;                     // (p, im): [Im c |  Re c]
  if constexpr (sizeof(T) == 2 && std::is_same<T, __half>::value) {
    r0[b] = __float2half_rn(re); r0[nbp + b] = __float2half_rn(-im);
    r1[b] = __float2half_rn(im); r1[nbp + b] = __float2half_rn(re);
  } else {
    r0[b] = __float2bfloat16_rn(re); r0[nbp + b] = __float2bfloat16_rn(-im);
    r1[b] = __float2bfloat16_rn(im); r1[nbp + b] = __float2bfloat16_rn(re);
  }
}

template <typename T>
__global__ void __launch_bounds__(kUmmaThreads, 1) k_beam_sum_umma(
    const T* __restrict__ sdata, const T* __restrict__ coef, int n, int w, int nbp,
    const int2* __restrict__ origin, const int* __restrict__ offsets, const int* __restrict__ work,
    const int* __restrict__ list, int n_tiles, float2* __restrict__ windows, int* __restrict__ status) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* tail = smem + kUmmaStages * kStageBytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(tail);                       // kUmmaStages mbarriers
  uint32_t* s_taddr = reinterpret_cast<uint32_t*>(tail + 64);
  int* s_abort = reinterpret_cast<int*>(tail + 68);
  int* s_probe = reinterpret_cast<int*>(tail + 128);                        // kUmmaGroup probe ids
  int2* s_org = reinterpret_cast<int2*>(tail + 128 + 4 * kUmmaGroup);       // their window origins

  const int tid = threadIdx.x, warp = tid >> 5;
  const int K = 2 * nbp, KC = K / 64;
  const uint32_t idesc = umma_idesc(std::is_same<T, __half>::value ? 0u : 1u);
  const uint32_t sbase = smem_u32(smem);

  if (tid == 0) {
    for (int s = 0; s < kUmmaStages; ++s) mbar_init(smem_u32(bars + s), 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_taddr)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *s_taddr;

  const int total = __ldg(work + n_tiles);
  const int ntx = n / kTileX;
  uint32_t chunk_counter = 0;     // chunks committed so far by this CTA (same on every thread)
  bool aborted = false;

  for (int item = blockIdx.x; item < total && !aborted; item += gridDim.x) {
    const int tile = find_item_tile(work, n_tiles, item);
    const int first = __ldg(offsets + tile);
    const int g0 = (item - __ldg(work + tile)) * kUmmaGroup;
    const int cnt = min(kUmmaGroup, __ldg(offsets + tile + 1) - first - g0);
    const int x0 = (tile % ntx) * kTileX, y0 = (tile / ntx) * kTileY;
    for (int i = tid; i < kUmmaGroup; i += kUmmaThreads) {
      const int p = i < cnt ? __ldg(list + first + g0 + i) : -1;
      s_probe[i] = p;
      s_org[i] = p >= 0 ? __ldg(origin + p) : make_int2(0, 0);
    }
    __syncthreads();

    // loads of one K chunk into stage st: A rows = the tile's pixels, B rows = (probe, re|im)
    auto load_chunk = [&](int kc, int st) {
      const uint32_t a_s = sbase + st * kStageBytes, b_s = a_s + kAStage;
      const int k0 = kc * 64;
#pragma unroll
      for (int i = 0; i < 1024 / kUmmaThreads; ++i) {
        const int idx = tid + i * kUmmaThreads;
        const int r = idx >> 3, c = idx & 7;
        const size_t pix = (size_t)(y0 + r / kTileX) * n + x0 + (r % kTileX);
        cp_async16(a_s + r * 128 + ((c ^ (r & 7)) << 4), sdata + pix * K + k0 + c * 8, 16);
      }
#pragma unroll
      for (int i = 0; i < 2048 / kUmmaThreads; ++i) {
        const int idx = tid + i * kUmmaThreads;
        const int r = idx >> 3, c = idx & 7;
        const int p = s_probe[r >> 1];
        const T* src = p >= 0 ? coef + ((size_t)p * 2 + (r & 1)) * K + k0 + c * 8 : coef;
        cp_async16(b_s + r * 128 + ((c ^ (r & 7)) << 4), src, p >= 0 ? 16 : 0);
      }
    };

    for (int s = 0; s < kUmmaStages - 1; ++s) {
      if (s < KC) load_chunk(s, (chunk_counter + s) % kUmmaStages);
      cp_async_commit();
    }
    for (int kc = 0; kc < KC; ++kc) {
      const uint32_t g = chunk_counter + kc;
      const int st = g % kUmmaStages;
      cp_async_wait<kUmmaStages - 2>();
      fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a_s = sbase + st * kStageBytes, b_s = a_s + kAStage;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          umma_f16(taddr, sw128_desc(a_s + kk * 32), sw128_desc(b_s + kk * 32), idesc, (kc > 0 || kk > 0) ? 1u : 0u);
        umma_commit(smem_u32(bars + st));
        // the stage about to be refilled was read by the previous chunk's MMAs
        if (kc >= 1) {
          const uint32_t gp = g - 1;
          if (!mbar_wait(smem_u32(bars + gp % kUmmaStages), (gp / kUmmaStages) & 1u)) *s_abort = 1;
        }
      }
      __syncthreads();
      if (*s_abort) { aborted = true; break; }
      const int kn = kc + kUmmaStages - 1;
      if (kn < KC) load_chunk(kn, (chunk_counter + kn) % kUmmaStages);
      cp_async_commit();
    }
    if (aborted) break;
    if (tid == 0) {
      const uint32_t gl = chunk_counter + KC - 1;
      if (!mbar_wait(smem_u32(bars + gl % kUmmaStages), (gl / kUmmaStages) & 1u)) *s_abort = 1;
    }
    chunk_counter += KC;
    __syncthreads();
    if (*s_abort) { aborted = true; break; }
    tc_fence_after();

    // epilogue: lane r of warp w holds pixel 32 (w mod 4) + r of the tile; with
    // eight warps, warps w and w + 4 share a lane quarter and split its columns
    constexpr int WARPS = kUmmaThreads / 32, BLKS = 4 / (WARPS / 4);
    const int quarter = warp % 4;
    const int r = quarter * 32 + (tid & 31);
    const int gx = x0 + r % kTileX, gy = y0 + r / kTileX;
    for (int b = 0; b < BLKS; ++b) {
      const int blk = (warp / 4) * BLKS + b;
      float v[64];
      tmem_ld64(taddr + ((uint32_t)(quarter * 32) << 16) + blk * 64, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int pl = blk * 32 + j;
        const int p = s_probe[pl];
        if (p < 0) continue;
        const int2 o = s_org[pl];
        const int u = (gx - o.x + n) % n, vv = (gy - o.y + n) % n;
        if (u < w && vv < w) windows[((size_t)p * w + vv) * w + u] = make_float2(v[2 * j], v[2 * j + 1]);
      }
    }
    tc_fence_before();
    __syncthreads();
  }

  if (aborted && tid == 0) atomicExch(status, (int)STEM_ERR_TIMEOUT);
  cp_async_wait_all();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols) : "memory");
  }
}

cudaError_t launch_beam_sum_umma(const OutputArgs& o, int np, const double* probe_xy, void* coef,
                                 const int2* origin, const int* offsets, const int* work, const int* list,
                                 int n_tiles, float2* windows, cudaStream_t s) {
  const double inv_lx = 1.0 / o.lx, inv_ly = 1.0 / o.ly;
  dim3 cg((o.nbp + 127) / 128, np);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = umma_smem_bytes();
  cudaError_t e;
  if (o.storage == STEM_F16) {
    note_launch(), k_coefficients_umma<__half><<<cg, 128, 0, s>>>(probe_xy, o.beams, o.beam_turns, o.n_beams, o.nbp, o.scales,
                                                                 inv_lx, inv_ly, o.coef_norm, static_cast<__half*>(coef));
    if ((e = cudaFuncSetAttribute(k_beam_sum_umma<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
      return e;
    note_launch(), k_beam_sum_umma<__half><<<sms, kUmmaThreads, smem, s>>>(
        static_cast<const __half*>(o.sdata), static_cast<const __half*>(coef), o.n, o.w, o.nbp, origin, offsets,
        work, list, n_tiles, windows, o.status);
  } else if (o.storage == STEM_BF16) {
    note_launch(), k_coefficients_umma<__nv_bfloat16><<<cg, 128, 0, s>>>(
        probe_xy, o.beams, o.beam_turns, o.n_beams, o.nbp, o.scales, inv_lx, inv_ly, o.coef_norm,
        static_cast<__nv_bfloat16*>(coef));
    if ((e = cudaFuncSetAttribute(k_beam_sum_umma<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
      return e;
    note_launch(), k_beam_sum_umma<__nv_bfloat16><<<sms, kUmmaThreads, smem, s>>>(
        static_cast<const __nv_bfloat16*>(o.sdata), static_cast<const __nv_bfloat16*>(coef), o.n, o.w, o.nbp,
        origin, offsets, work, list, n_tiles, windows, o.status);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace stem
