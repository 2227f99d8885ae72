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
// One persistent CTA per SM, warp-specialised, the roles synchronised by
// mbarriers only:
//   warp 0        one thread issues the MMAs of each 64-wide K chunk as soon as
//                 its stage is full, commits them to the stage's "empty"
//                 barrier, and after an item's last chunk to the item's
//                 accumulator barrier;
//   warps 1 - 11  producers: stage the chunks of A and B into shared memory in
//                 the 128-byte swizzled K-major layout with cp.async, each
//                 thread arriving on the stage's "full" barrier when its copies
//                 land (cp.async.mbarrier.arrive.noinc); four stages;
//   warps 12 - 15 epilogue: read an item's accumulator with tcgen05.ld (warp w
//                 reads the lane quarter w mod 4) and scatter the pixels into
//                 the probes' windows, then release the accumulator.
// The accumulator is double-buffered in tensor memory (2 x 256 columns), so the
// MMAs of one item run while the epilogue drains the previous one, and the
// producers stage the next item's chunks while the current one finishes.
// Every wait is bounded (2 s of %globaltimer); on timeout the kernel records
// STEM_ERR_TIMEOUT in the plan's status word, lets its copies and MMAs land,
// frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "async_copy.cuh"
#include "internal.h"

namespace stem {

constexpr int kUmmaThreads = 512;
constexpr int kProducerWarp0 = 1, kProducerWarps = 11;   // warps 1 .. 11
constexpr int kProducers = 32 * kProducerWarps;           // 352 threads
constexpr int kEpilogueWarp0 = 12;                        // warps 12 .. 15 (lane quarters 0 .. 3)
constexpr int kUmmaStages = 4;
constexpr int kUmmaGroup = 128;                 // probes per work item (N = 256)
constexpr int kTileX = 16, kTileY = 8;          // must match prism.cu
constexpr int kAStage = 128 * 128;              // bytes: 128 rows x 64 halves
constexpr int kBStage = 256 * 128;              // bytes: 256 rows x 64 halves
constexpr int kStageBytes = kAStage + kBStage;
constexpr int kAccCols = 256;                   // one accumulator: 128 lanes x 256 FP32 columns
constexpr int kTmemCols = 2 * kAccCols;         // double-buffered
constexpr int kACopies = (1024 + kProducers - 1) / kProducers;   // 16-byte copies per producer per chunk
constexpr int kBCopies = (2048 + kProducers - 1) / kProducers;

size_t umma_smem_bytes() { return (size_t)kUmmaStages * kStageBytes + 1024 + 256 + 12 * kUmmaGroup + 16; }
int umma_group() { return kUmmaGroup; }


__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// Arrive on the barrier once this thread's earlier cp.async copies have landed
// (the barrier's expected count includes this arrival).
__device__ __forceinline__ void cp_async_arrive(uint32_t bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

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

// The work item of a CTA's k-th turn: pixel tile and group of its probe list.
struct UmmaItem {
  int first, g0, cnt, x0, y0;
};
__device__ __forceinline__ UmmaItem umma_item(const int* __restrict__ offsets, const int* __restrict__ work,
                                              const int* __restrict__ items, int ntx, int item) {
  UmmaItem it;
  const int tile = __ldg(items + item);
  it.first = __ldg(offsets + tile);
  it.g0 = (item - __ldg(work + tile)) * kUmmaGroup;
  it.cnt = min(kUmmaGroup, __ldg(offsets + tile + 1) - it.first - it.g0);
  it.x0 = (tile % ntx) * kTileX;
  it.y0 = (tile / ntx) * kTileY;
  return it;
}

template <typename T>
__global__ void __launch_bounds__(kUmmaThreads, 1) k_beam_sum_umma(
    const T* __restrict__ sdata, const T* __restrict__ coef, int n, int w, int nbp,
    const int2* __restrict__ origin, const int* __restrict__ offsets, const int* __restrict__ work,
    const int* __restrict__ items, const int* __restrict__ list, int n_tiles, float2* __restrict__ windows,
    int* __restrict__ status) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kUmmaStages * kStageBytes);
  uint64_t* full = bars;                                  // [kUmmaStages]: stage staged
  uint64_t* empty = bars + kUmmaStages;                   // [kUmmaStages]: stage read by its MMAs
  uint64_t* acc_full = bars + 2 * kUmmaStages;            // [2]: accumulator complete
  uint64_t* acc_empty = bars + 2 * kUmmaStages + 2;       // [2]: accumulator read out
  uint32_t* s_taddr = reinterpret_cast<uint32_t*>(bars + 2 * kUmmaStages + 4);
  int* s_abort = reinterpret_cast<int*>(s_taddr + 1);
  int* e_flag = s_abort + 1;                                       // epilogue: accumulator ready
  int2* e_org = reinterpret_cast<int2*>(bars + 2 * kUmmaStages + 6);   // [kUmmaGroup] epilogue's item
  int* e_probe = reinterpret_cast<int*>(e_org + kUmmaGroup);           // [kUmmaGroup]

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = 2 * nbp, KC = K / 64;
  const uint32_t sbase = smem_u32(smem);
  const int total = __ldg(work + n_tiles);
  const int ntx = n / kTileX;

  if (tid == 0) {
    for (int s = 0; s < kUmmaStages; ++s) {
      mbar_init(smem_u32(full + s), kProducers);
      mbar_init(smem_u32(empty + s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(acc_full + b), 1);
      mbar_init(smem_u32(acc_empty + b), 1);
    }
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
  auto abort_now = [&] { return *reinterpret_cast<volatile int*>(s_abort) != 0; };

  if (warp == 0) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = umma_idesc(std::is_same<T, __half>::value ? 0u : 1u);
      uint32_t g = 0;
      int it = 0;
      for (int item = blockIdx.x; item < total; item += gridDim.x, ++it) {
        const int b = it & 1;
        if (it >= 2 && !mbar_wait(smem_u32(acc_empty + b), ((it >> 1) - 1) & 1u)) { *s_abort = 1; break; }
        tc_fence_after();
        const uint32_t acc = taddr + (uint32_t)(b * kAccCols);
        bool ok = true;
        for (int kc = 0; kc < KC; ++kc, ++g) {
          const int st = g % kUmmaStages;
          if (!mbar_wait(smem_u32(full + st), (g / kUmmaStages) & 1u) || abort_now()) { ok = false; break; }
          // the producers' cp.async writes (generic proxy) before the MMAs read them (async proxy)
          fence_proxy_async();
          tc_fence_after();
          const uint32_t a_s = sbase + st * kStageBytes, b_s = a_s + kAStage;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            umma_f16(acc, sw128_desc(a_s + kk * 32), sw128_desc(b_s + kk * 32), idesc, (kc > 0 || kk > 0) ? 1u : 0u);
          umma_commit(smem_u32(empty + st));
        }
        if (!ok) { *s_abort = 1; break; }
        umma_commit(smem_u32(acc_full + b));
      }
      // every MMA issued has landed before the tensor memory is freed
      if (g > 0) mbar_wait(smem_u32(empty + (g - 1) % kUmmaStages), ((g - 1) / kUmmaStages) & 1u);
    }
  } else if (warp < kEpilogueWarp0) {
    // ---------------------------------------------------------------- producers
    const int pt = tid - 32 * kProducerWarp0;
    // the probe ids of this thread's B rows for an item (loads issued one item
    // ahead, so that their latency hides behind the chunks of the current item)
    auto probe_ids = [&](const UmmaItem& itm, int (&pid)[kBCopies]) {
#pragma unroll
      for (int i = 0; i < kBCopies; ++i) {
        const int idx = pt + i * kProducers;
        const int pl = ((idx < 2048 ? idx : 0) >> 3) >> 1;
        pid[i] = pl < itm.cnt ? __ldg(list + itm.first + itm.g0 + pl) : -1;
      }
    };
    uint32_t g = 0;
    int item = blockIdx.x;
    UmmaItem itm{};
    int pid[kBCopies];
    if (item < total) {
      itm = umma_item(offsets, work, items, ntx, item);
      probe_ids(itm, pid);
    }
    for (; item < total && !abort_now(); item += gridDim.x) {
      // this thread's copies of every chunk of the item: source rows and swizzled destinations
      const T* a_src[kACopies];
      uint32_t a_dst[kACopies];
#pragma unroll
      for (int i = 0; i < kACopies; ++i) {
        const int idx = pt + i * kProducers;
        const int r = (idx < 1024 ? idx : 0) >> 3, c = idx & 7;
        const size_t pix = (size_t)(itm.y0 + r / kTileX) * n + itm.x0 + (r % kTileX);
        a_src[i] = sdata + pix * K + c * 8;
        a_dst[i] = r * 128 + ((c ^ (r & 7)) << 4);
      }
      const T* b_src[kBCopies];
      uint32_t b_dst[kBCopies];
#pragma unroll
      for (int i = 0; i < kBCopies; ++i) {
        const int idx = pt + i * kProducers;
        const int r = (idx < 2048 ? idx : 0) >> 3, c = idx & 7;
        b_src[i] = pid[i] >= 0 ? coef + ((size_t)pid[i] * 2 + (r & 1)) * K + c * 8 : nullptr;
        b_dst[i] = kAStage + r * 128 + ((c ^ (r & 7)) << 4);
      }
      // the next item's tile and probe ids, in flight while this item's chunks stream
      const int next = item + gridDim.x;
      if (next < total) {
        itm = umma_item(offsets, work, items, ntx, next);
        probe_ids(itm, pid);
      }
      bool ok = true;
      for (int kc = 0; kc < KC; ++kc, ++g) {
        const int st = g % kUmmaStages;
        if (g >= kUmmaStages && !mbar_wait(smem_u32(empty + st), ((g / kUmmaStages) - 1) & 1u)) { ok = false; break; }
        const uint32_t base = sbase + st * kStageBytes;
        const int k0 = kc * 64;
#pragma unroll
        for (int i = 0; i < kACopies; ++i)
          if (pt + i * kProducers < 1024) cp_async16(base + a_dst[i], a_src[i] + k0, 16);
#pragma unroll
        for (int i = 0; i < kBCopies; ++i)
          if (pt + i * kProducers < 2048) {
            // probes past the group's count read zeros (a zero-byte copy from any valid address)
            if (b_src[i]) cp_async16(base + b_dst[i], b_src[i] + k0, 16);
            else cp_async16(base + b_dst[i], coef, 0);
          }
        cp_async_arrive(smem_u32(full + st));
      }
      if (!ok) { *s_abort = 1; break; }
    }
    cp_async_wait_all();
  } else {
    // ---------------------------------------------------------------- epilogue
    const int quarter = warp % 4;
    const int et = tid - 32 * kEpilogueWarp0;            // 0 .. 127
    const int r = quarter * 32 + lane;                   // this lane's pixel of the tile
    auto epi_sync = [] { asm volatile("bar.sync 1, 128;" ::: "memory"); };   // the four epilogue warps
    int it = 0;
    for (int item = blockIdx.x; item < total; item += gridDim.x, ++it) {
      const int b = it & 1;
      // the item's probes and window origins, one per epilogue thread, staged
      // while its MMAs may still run
      const UmmaItem itm = umma_item(offsets, work, items, ntx, item);
      {
        const int p = et < itm.cnt ? __ldg(list + itm.first + itm.g0 + et) : -1;
        e_probe[et] = p;
        e_org[et] = p >= 0 ? __ldg(origin + p) : make_int2(0, 0);
      }
      // one thread waits; the named barrier hands all 128 the same outcome
      if (et == 0) *e_flag = mbar_wait(smem_u32(acc_full + b), (it >> 1) & 1u) && !abort_now();
      epi_sync();
      if (!*reinterpret_cast<volatile int*>(e_flag)) { *s_abort = 1; break; }
      tc_fence_after();
      const int gx = itm.x0 + r % kTileX, gy = itm.y0 + r / kTileX;
      for (int blk = 0; blk < 4; ++blk) {
        float v[64];
        tmem_ld64(taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * kAccCols + blk * 64), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int pl = blk * 32 + j;
          const int p = e_probe[pl];
          if (p < 0) break;
          const int2 o = e_org[pl];
          const int du = gx - o.x, dv = gy - o.y;    // in (-n, n): wrap into [0, n)
          const int u = du < 0 ? du + n : du, vv = dv < 0 ? dv + n : dv;
          if (u < w && vv < w) windows[((size_t)p * w + vv) * w + u] = make_float2(v[2 * j], v[2 * j + 1]);
        }
      }
      tc_fence_before();
      epi_sync();   // every epilogue thread is done with e_probe / e_org and the accumulator
      if (et == 0) mbar_arrive(smem_u32(acc_empty + b));
    }
  }

  __syncthreads();
  if (tid == 0 && *s_abort) atomicExch(status, (int)STEM_ERR_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols) : "memory");
  }
}

cudaError_t launch_beam_sum_umma(const OutputArgs& o, int np, const double* probe_xy, void* coef,
                                 const int2* origin, const int* offsets, const int* work, const int* items,
                                 const int* list, int n_tiles, float2* windows, cudaStream_t s) {
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
    ProfScope prof(STEM_PROF_BEAM_SUM, s);
    note_launch(), k_beam_sum_umma<__half><<<sms, kUmmaThreads, smem, s>>>(
        static_cast<const __half*>(o.sdata), static_cast<const __half*>(coef), o.n, o.w, o.nbp, origin, offsets,
        work, items, list, n_tiles, windows, o.status);
  } else if (o.storage == STEM_BF16) {
    note_launch(), k_coefficients_umma<__nv_bfloat16><<<cg, 128, 0, s>>>(
        probe_xy, o.beams, o.beam_turns, o.n_beams, o.nbp, o.scales, inv_lx, inv_ly, o.coef_norm,
        static_cast<__nv_bfloat16*>(coef));
    if ((e = cudaFuncSetAttribute(k_beam_sum_umma<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
      return e;
    ProfScope prof(STEM_PROF_BEAM_SUM, s);
    note_launch(), k_beam_sum_umma<__nv_bfloat16><<<sms, kUmmaThreads, smem, s>>>(
        static_cast<const __nv_bfloat16*>(o.sdata), static_cast<const __nv_bfloat16*>(coef), o.n, o.w, o.nbp,
        origin, offsets, work, items, list, n_tiles, windows, o.status);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace stem
