// selftest.cu - exercise of the bounded-wait path that the TMA and
// tensor-core kernels share (stem_selftest_bounded_wait).  The paper has no
// counterpart: it exists so that the timeout handling can be tested on a GPU
// without a fault or a hang.
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

}  // namespace stem

extern "C" stem_status stem_selftest_bounded_wait(stem_plan pl, int64_t limit_ns, void* stream) {
  if (!pl || limit_ns < 1 || limit_ns > 1000000000ll) return STEM_ERR_INVALID;
  stem::note_launch(), stem::k_selftest_wait<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(
                           (unsigned long long)limit_ns, pl->status);
  return cudaGetLastError() == cudaSuccess ? STEM_OK : STEM_ERR_CUDA;
}
