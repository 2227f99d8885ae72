// selftest.cu - diagnostics with no counterpart in the paper:
//   stem_selftest_bounded_wait exercises the bounded-wait path that the TMA and
//   tensor-core kernels share, so that the timeout handling can be tested on a
//   GPU without a fault or a hang;
//   stem_selftest_fma_rate runs independent FP32 FMA chains, the measured
//   denominator of the FFT passes' FP32 roofline.
#include "async_copy.cuh"
#include "internal.h"

namespace stem {

// One thread waits on a shared-memory barrier that nothing arrives at; after
// limit_ns it records STEM_ERR_TIMEOUT in the status word and returns.
__global__ void k_selftest_wait(unsigned long long limit_ns, int* status) {
  __shared__ uint64_t bar;
  mbar_init(smem_u32(&bar), 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait(smem_u32(&bar), 0u, limit_ns)) atomicExch(status, (int)STEM_ERR_TIMEOUT);
}

// kFmaChains independent FMA chains per thread, `iters` rounds.  Scalar:
// a = a * b + c (one lane operation per FMA).  Packed: the f32x2 FMA of sm_100
// and later on a pair (two lane operations per instruction).  The operands keep
// every value finite; one sum per thread is stored so nothing is dropped.
constexpr int kFmaChains = 8;
constexpr int kFmaThreads = 256;

template <bool PACKED>
__global__ void __launch_bounds__(kFmaThreads) k_fma_rate(long long iters, float seed, float* out) {
  const float b = 0.999999f, c = 1.0e-7f * seed;
  float acc = 0.0f;
  if constexpr (!PACKED) {
    float a[kFmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) a[k] = seed + (float)(threadIdx.x + k);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kFmaChains; ++k) a[k] = fmaf(a[k], b, c);
    }
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) acc += a[k];
  } else {
    unsigned long long a[kFmaChains];
    unsigned long long bb, cc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
    asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) {
      const float lo = seed + (float)(threadIdx.x + k), hi = lo + 0.5f;
      asm("mov.b64 %0, {%1, %2};" : "=l"(a[k]) : "f"(lo), "f"(hi));
    }
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kFmaChains; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(bb), "l"(cc));
    }
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) {
      float lo, hi;
      asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[k]));
      acc += lo + hi;
    }
  }
  out[blockIdx.x * kFmaThreads + threadIdx.x] = acc;
}

}  // namespace stem

extern "C" stem_status stem_selftest_fma_rate(int32_t packed, int64_t iters, int32_t blocks, float* out,
                                              void* stream) {
  if (iters < 1 || blocks < 1 || blocks > 1 << 20 || !out) return STEM_ERR_INVALID;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (packed)
    stem::note_launch(), stem::k_fma_rate<true><<<blocks, stem::kFmaThreads, 0, s>>>(iters, 1.0f, out);
  else
    stem::note_launch(), stem::k_fma_rate<false><<<blocks, stem::kFmaThreads, 0, s>>>(iters, 1.0f, out);
  return cudaGetLastError() == cudaSuccess ? STEM_OK : STEM_ERR_CUDA;
}

extern "C" stem_status stem_selftest_bounded_wait(stem_plan pl, int64_t limit_ns, void* stream) {
  if (!pl || limit_ns < 1 || limit_ns > 1000000000ll) return STEM_ERR_INVALID;
  stem::note_launch(), stem::k_selftest_wait<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(
                           (unsigned long long)limit_ns, pl->status);
  return cudaGetLastError() == cudaSuccess ? STEM_OK : STEM_ERR_CUDA;
}
