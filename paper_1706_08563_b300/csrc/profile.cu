// profile.cu - optional CUDA-event timing of the hot kernel families
// (stem_profile_enable / stem_profile_read), for measuring a kernel's own
// launch duration inside a running workload.  While recording is off (the
// default) a ProfScope costs one relaxed atomic load.
#include <atomic>
#include <mutex>
#include <vector>

#include "internal.h"

namespace stem {

namespace {

struct Pair {
  cudaEvent_t start = nullptr, stop = nullptr;
};

struct ProfState {
  std::mutex m;
  std::vector<Pair> ev[STEM_PROF_KINDS];   // event pairs, reused across enable() calls
  size_t used[STEM_PROF_KINDS] = {};
  bool failed = false;
};

ProfState& prof() {
  static ProfState s;
  return s;
}

std::atomic<bool> g_prof_on{false};

}  // namespace

ProfScope::ProfScope(int kind, cudaStream_t s) {
  if (!g_prof_on.load(std::memory_order_relaxed) || kind < 0 || kind >= STEM_PROF_KINDS) return;
  ProfState& p = prof();
  std::lock_guard<std::mutex> lock(p.m);
  std::vector<Pair>& v = p.ev[kind];
  if (p.used[kind] == v.size()) {
    Pair e;
    if (cudaEventCreate(&e.start) != cudaSuccess || cudaEventCreate(&e.stop) != cudaSuccess) {
      if (e.start) cudaEventDestroy(e.start);
      p.failed = true;
      return;
    }
    v.push_back(e);
  }
  Pair& e = v[p.used[kind]];
  if (cudaEventRecord(e.start, s) != cudaSuccess) {
    p.failed = true;
    return;
  }
  stop_ = e.stop;
  stream_ = s;
  ++p.used[kind];
}

ProfScope::~ProfScope() {
  if (!stop_) return;
  if (cudaEventRecord(stop_, stream_) != cudaSuccess) {
    std::lock_guard<std::mutex> lock(prof().m);
    prof().failed = true;
  }
}

}  // namespace stem

using namespace stem;

extern "C" stem_status stem_profile_enable(int32_t on) {
  ProfState& p = prof();
  std::lock_guard<std::mutex> lock(p.m);
  if (on) {
    for (int k = 0; k < STEM_PROF_KINDS; ++k) p.used[k] = 0;
    p.failed = false;
  }
  g_prof_on.store(on != 0, std::memory_order_relaxed);
  return STEM_OK;
}

extern "C" stem_status stem_profile_read(int32_t kind, int64_t* launches, double* total_ms) {
  if (kind < 0 || kind >= STEM_PROF_KINDS || !launches || !total_ms) return STEM_ERR_INVALID;
  ProfState& p = prof();
  std::lock_guard<std::mutex> lock(p.m);
  if (p.failed) return STEM_ERR_CUDA;
  double sum = 0.0;
  for (size_t i = 0; i < p.used[kind]; ++i) {
    const Pair& e = p.ev[kind][i];
    float ms = 0.0f;
    if (cudaEventSynchronize(e.stop) != cudaSuccess || cudaEventElapsedTime(&ms, e.start, e.stop) != cudaSuccess)
      return STEM_ERR_CUDA;
    sum += ms;
  }
  *launches = (int64_t)p.used[kind];
  *total_ms = sum;
  return STEM_OK;
}
