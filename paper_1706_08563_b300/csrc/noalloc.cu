// noalloc.cu - multislice for callers that cannot supply scratch memory.
//
// stem_multislice_scan needs a caller-provided workspace (the batch of waves).
// Some callers cannot allocate device memory and have no buffer to lend: a
// plugin inside a host application that owns the device's memory and hands the
// plugin only its input and output buffers, or a loop whose memory budget is
// fixed at start-up and must not call cudaMalloc (which, as the paper notes in
// its computational model, also synchronises the device).  For them this file
// keeps a fixed scratch array in the library's own device image and runs the
// same multislice kernels on it.  Nothing here allocates.
#include <mutex>

#include "internal.h"

namespace {

// 32 MiB of scratch, held on every device that loads the library until the
// process exits.  Enough for batch * n * n * 8 bytes of waves (for example
// 512 waves of 256^2, 4 of 1024^2, 1 of 2048^2).
constexpr size_t kNoAllocScratchBytes = 32u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per
// device (in host code the array's name is only a host-side stand-in).
stem_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return STEM_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return STEM_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return STEM_OK;
}

}  // namespace

extern "C" stem_status stem_multislice_scan_noalloc(stem_plan plan, const void* trans, const double* probe_xy,
                                                    int64_t n_probes, int32_t batch, float weight,
                                                    float* rings_out, void* stream) {
  if (!plan || batch < 1) return STEM_ERR_INVALID;
  // The plan's tables live on the device that was current at stem_plan_create,
  // and the scratch address looked up below belongs to the current device:
  // with another device current the kernels would mix memory of two devices.
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return STEM_ERR_CUDA;
  if (dev != plan->device) return STEM_ERR_INVALID;
  const size_t need = stem_multislice_workspace(plan, batch);
  if (need == 0) return STEM_ERR_INVALID;
  if (need > kNoAllocScratchBytes) return STEM_ERR_NOMEM;
  void* scratch = nullptr;
  const stem_status st = scratch_address(&scratch);
  if (st != STEM_OK) return st;
  // No clearing between calls is needed: the probe-initialisation pass writes
  // every in-band column of each wave, and the out-of-band columns, which keep
  // whatever an earlier call left there, are masked to zero by every pass that
  // reads them.
  return stem_multislice_scan(plan, trans, probe_xy, n_probes, batch, weight, rings_out, scratch,
                              kNoAllocScratchBytes, stream);
}
