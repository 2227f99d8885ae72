// api.cu - the C ABI of libstem (declared in include/stem.h).
//
// Host code here validates arguments, builds the plan's small tables (FP64
// decisions of aperture, band limit and ring membership; propagator factors;
// PRISM beam lists) and sequences the kernels on the caller's stream.  No
// simulation arithmetic runs on the host.
#include <algorithm>
#include <vector>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>

#include "internal.h"

using namespace stem;

namespace stem {
static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace stem

namespace {

// CODATA 2018: h*c in keV*A and the electron rest energy in keV.
constexpr double kHcKevA = 12.398419843320026;
constexpr double kMc2Kev = 510.99895000;

double wavelength_a(double e_kev) { return kHcKevA / std::sqrt(e_kev * (2.0 * kMc2Kev + e_kev)); }

double interaction_sigma(double e_kev) {
  const double lam = wavelength_a(e_kev);
  return (2.0 * M_PI / (lam * e_kev * 1000.0)) * (kMc2Kev + e_kev) / (2.0 * kMc2Kev + e_kev);
}

int freq(int j, int n) { return j < n / 2 ? j : j - n; }

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

int log2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

constexpr int kStreamBufs = 3;

// Supplies the transmission function t_n to a slice loop.
//
// Resident: a pointer into the device stack [S][n][n].
// Streamed (the paper's streaming memory model, "Streaming Data for Very Large
// Simulations"): the stack stays in host memory and kStreamBufs slice buffers
// take turns.  Each buffer is refilled by an asynchronous copy on a second
// stream as soon as the row pass that read it has finished, so the copies of
// the next slices run while the passes of the current one do.  The stream and
// events live for one call; destroying them with work still queued is allowed
// (CUDA releases them when that work completes).
class SliceSource {
 public:
  SliceSource(const float2* device_stack, size_t plane) : dev_(device_stack), plane_(plane) {}
  SliceSource(const float2* host_stack, size_t plane, float2* bufs) : host_(host_stack), plane_(plane) {
    for (int k = 0; k < kStreamBufs; ++k) buf_[k] = bufs + k * plane;
  }
  SliceSource(const SliceSource&) = delete;
  SliceSource& operator=(const SliceSource&) = delete;
  ~SliceSource() {
    if (copy_) cudaStreamDestroy(copy_);
    for (cudaEvent_t ev : ready_) if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : done_) if (ev) cudaEventDestroy(ev);
    if (start_) cudaEventDestroy(start_);
  }

  // Streamed: make the copy stream start after the work already queued on s
  // (an earlier call may still read the buffers).
  cudaError_t begin(cudaStream_t s) {
    if (!host_) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&copy_, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&start_, cudaEventDisableTiming);
    for (int k = 0; k < kStreamBufs && e == cudaSuccess; ++k) {
      e = cudaEventCreateWithFlags(&ready_[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done_[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventRecord(start_, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(copy_, start_, 0);
    return e;
  }

  // t_n for the next row pass, ordered before it on s.
  cudaError_t acquire(int slice, cudaStream_t s, const float2** t) {
    if (!host_) {
      *t = dev_ + (size_t)slice * plane_;
      return cudaSuccess;
    }
    const int k = (int)(step_ % kStreamBufs);
    cudaError_t e = cudaSuccess;
    if (step_ >= kStreamBufs) e = cudaStreamWaitEvent(copy_, done_[k], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(buf_[k], host_ + (size_t)slice * plane_, plane_ * sizeof(float2), cudaMemcpyDefault, copy_);
    if (e == cudaSuccess) e = cudaEventRecord(ready_[k], copy_);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ready_[k], 0);
    *t = buf_[k];
    return e;
  }

  // After the row pass that read the buffer has been queued on s.
  cudaError_t release(cudaStream_t s) {
    if (!host_) return cudaSuccess;
    const int k = (int)(step_++ % kStreamBufs);
    return cudaEventRecord(done_[k], s);
  }

 private:
  const float2* dev_ = nullptr;
  const float2* host_ = nullptr;
  size_t plane_ = 0;
  float2* buf_[kStreamBufs] = {};
  cudaStream_t copy_ = nullptr;
  cudaEvent_t start_ = nullptr;
  cudaEvent_t ready_[kStreamBufs] = {};
  cudaEvent_t done_[kStreamBufs] = {};
  int64_t step_ = 0;
};

stem_status cuda_status(cudaError_t e) { return e == cudaSuccess ? STEM_OK : STEM_ERR_CUDA; }

stem_status check_params(const stem_params* p) {
  if (!p) return STEM_ERR_INVALID;
  if (!is_pow2(p->n) || p->n < 8 || p->n > 2048) return STEM_ERR_UNSUPPORTED;
  if (!(p->cell[0] > 0.0) || !(p->cell[1] > 0.0) || p->n_slices < 1 || !(p->slice_dz > 0.0) ||
      !(p->energy_kev > 0.0) || !(p->alpha_mrad >= 0.0) || !(p->ring_width_mrad > 0.0) || p->n_rings < 1 ||
      p->n_rings > kMaxRings || !std::isfinite(p->defocus_a) || !std::isfinite(p->cs_a))
    return STEM_ERR_INVALID;
  return STEM_OK;
}

// f must be a power of two with W = n / f >= 8.
bool f_ok(const stem_plan_s* pl, int f) { return is_pow2(f) && f <= pl->n / 8; }

// Storage code = element type (STEM_F32, _F16, _BF16), optionally with the
// STEM_CROPPED flag; false for anything else.
bool decode_storage(int storage, int* elem, bool* cropped) {
  const int e = storage & ~(int)STEM_CROPPED;
  if (e < STEM_F32 || e > STEM_BF16) return false;
  *elem = e;
  *cropped = (storage & (int)STEM_CROPPED) != 0;
  return true;
}

// Side of the grid the S-matrix is stored on: N, or N' = 3N/4 when cropped.
int smatrix_grid(int n, bool cropped) { return cropped ? 3 * n / 4 : n; }

// Number of beams of the FP64 aperture test for a given f (used by the footprint query).
int count_beams(const stem_params* p, int f, double lam) {
  const int n = p->n;
  int nb = 0;
  for (int nn = -n / 2; nn < n / 2; ++nn) {
    if (((nn % f) + f) % f) continue;
    for (int mm = -n / 2; mm < n / 2; ++mm) {
      if (((mm % f) + f) % f) continue;
      if (9LL * ((long long)mm * mm + (long long)nn * nn) > (long long)n * n) continue;
      const double kx = (double)mm / p->cell[0], ky = (double)nn / p->cell[1];
      if ((lam * std::sqrt(kx * kx + ky * ky)) * 1000.0 <= p->alpha_mrad) ++nb;
    }
  }
  return nb;
}


// Ring of scattering angle `ang` (mrad): uniform rings of ring_width_mrad, or
// [edges[i], edges[i+1]) when detector edges are set; -1 outside every ring.
int ring_of(double ang, const stem_params& p, const std::vector<double>& edges) {
  if (edges.empty()) {
    const double r = std::floor(ang / p.ring_width_mrad);
    return r < (double)p.n_rings ? (int)r : -1;
  }
  const int i = (int)(std::upper_bound(edges.begin(), edges.end(), ang) - edges.begin()) - 1;
  return (i >= 0 && i < (int)edges.size() - 1) ? i : -1;
}

// Fine look-up table (aperture bit, ring index) decided in FP64; returns |A|.
int build_fine_lut(const stem_params& p, double lam, const std::vector<double>& edges, std::vector<uint16_t>& lut) {
  const int n = p.n;
  const double lx = p.cell[0], ly = p.cell[1];
  lut.assign((size_t)n * n, kLutNoRing);
  int n_ap = 0;
  for (int i = 0; i < n; ++i) {
    const int nn = freq(i, n);
    const double ky = (double)nn / ly;
    for (int j = 0; j < n; ++j) {
      const int mm = freq(j, n);
      const double kx = (double)mm / lx;
      const bool mask = 9LL * ((long long)mm * mm + (long long)nn * nn) <= (long long)n * n;
      const double k = std::sqrt(kx * kx + ky * ky);
      const double ang = (lam * k) * 1000.0;
      uint16_t v = kLutNoRing;
      if (mask) {
        const int r = ring_of(ang, p, edges);
        if (r >= 0) v = (uint16_t)r;
        if (ang <= p.alpha_mrad) {
          v |= kLutAperture;
          ++n_ap;
        }
      }
      lut[(size_t)i * n + j] = v;
    }
  }
  return n_ap;
}

// The fine table transposed, [x][y]: column-wise reads become contiguous.
std::vector<uint16_t> transpose_lut(const std::vector<uint16_t>& lut, int n) {
  std::vector<uint16_t> t((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) t[(size_t)j * n + i] = lut[(size_t)i * n + j];
  return t;
}

// Window table for f: a window spans L / f, so window frequency (mu, nu) is
// the fine frequency (f mu, f nu); w = n / f, or 3n / (4f) on the cropped grid.
std::vector<uint16_t> coarse_lut(const std::vector<uint16_t>& lut, int n, int f, int w) {
  std::vector<uint16_t> coarse((size_t)w * w);
  for (int v = 0; v < w; ++v) {
    const int fi = ((f * freq(v, w)) % n + n) % n;
    for (int u = 0; u < w; ++u) {
      const int fj = ((f * freq(u, w)) % n + n) % n;
      coarse[(size_t)v * w + u] = lut[(size_t)fi * n + fj];
    }
  }
  return coarse;
}

}  // namespace

extern "C" {

uint64_t stem_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

const char* stem_status_string(stem_status s) {
  switch (s) {
    case STEM_OK: return "ok";
    case STEM_ERR_INVALID: return "invalid argument";
    case STEM_ERR_NOMEM: return "out of memory or workspace too small";
    case STEM_ERR_CUDA: return "CUDA error";
    case STEM_ERR_UNSUPPORTED: return "unsupported size";
    case STEM_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

void stem_plan_destroy(stem_plan pl) {
  if (!pl) return;
  cudaFree(pl->status);
  cudaFree(pl->prop_x);
  cudaFree(pl->prop_y);
  for (int i = 0; i <= kMaxLog2F; ++i) {
    cudaFree(pl->lut[i]);
    cudaFree(pl->lut_crop[i]);
    if (i == 0) cudaFree(pl->lut_t);
    cudaFree(pl->beams[i]);
    cudaFree(pl->beam_turns[i]);
  }
  delete pl;
}

stem_status stem_plan_create(const stem_params* params, stem_plan* out) {
  if (!out) return STEM_ERR_INVALID;
  *out = nullptr;
  stem_status st = check_params(params);
  if (st != STEM_OK) return st;
  stem_plan_s* pl = new (std::nothrow) stem_plan_s;
  if (!pl) return STEM_ERR_NOMEM;
  pl->p = *params;
  const int n = params->n;
  pl->n = n;
  pl->lam = wavelength_a(params->energy_kev);
  pl->sigma = interaction_sigma(params->energy_kev);
  cudaGetDevice(&pl->device);
  const double lx = params->cell[0], ly = params->cell[1];

  // Fine look-up table: aperture bit and ring index, decided in FP64.
  std::vector<uint16_t> lut;
  pl->n_aperture = build_fine_lut(*params, pl->lam, pl->edges, lut);

  // Propagator factors exp(-i pi lambda dz (m/L)^2) per axis (Eq. 2 is separable).
  std::vector<float2> px(n), py(n);
  for (int j = 0; j < n; ++j) {
    const double kx = (double)freq(j, n) / lx, ky = (double)freq(j, n) / ly;
    const double ax = -M_PI * pl->lam * params->slice_dz * kx * kx;
    const double ay = -M_PI * pl->lam * params->slice_dz * ky * ky;
    px[j] = make_float2((float)std::cos(ax), (float)std::sin(ax));
    py[j] = make_float2((float)std::cos(ay), (float)std::sin(ay));
  }

  cudaError_t e = cudaSuccess;
  auto upload = [&](void** dst, const void* src, size_t bytes) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(dst, bytes > 0 ? bytes : 16);
    if (e == cudaSuccess && bytes > 0) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  const int zero = 0;
  upload(reinterpret_cast<void**>(&pl->status), &zero, sizeof(int));
  upload(reinterpret_cast<void**>(&pl->prop_x), px.data(), n * sizeof(float2));
  upload(reinterpret_cast<void**>(&pl->prop_y), py.data(), n * sizeof(float2));

  {
    const std::vector<uint16_t> lt = transpose_lut(lut, n);
    upload(reinterpret_cast<void**>(&pl->lut_t), lt.data(), lt.size() * sizeof(uint16_t));
  }
  for (int lf = 0; lf <= kMaxLog2F; ++lf) {
    const int f = 1 << lf;
    if (f > n / 8) break;
    const std::vector<uint16_t> coarse = coarse_lut(lut, n, f, n / f);
    upload(reinterpret_cast<void**>(&pl->lut[lf]), coarse.data(), coarse.size() * sizeof(uint16_t));
    if (n >= 64) {
      const std::vector<uint16_t> crop = coarse_lut(lut, n, f, smatrix_grid(n, true) / f);
      upload(reinterpret_cast<void**>(&pl->lut_crop[lf]), crop.data(), crop.size() * sizeof(uint16_t));
    }
    // PRISM beams: aperture pixels on every f-th frequency, ordered by n then m.
    std::vector<int2>& bl = pl->h_beams[lf];
    for (int nn = -n / 2; nn < n / 2; ++nn) {
      if (((nn % f) + f) % f) continue;
      for (int mm = -n / 2; mm < n / 2; ++mm) {
        if (((mm % f) + f) % f) continue;
        const int i = (nn + n) % n, j = (mm + n) % n;
        if (lut[(size_t)i * n + j] & kLutAperture) bl.push_back(make_int2(mm, nn));
      }
    }
    pl->n_beams[lf] = (int)bl.size();
    upload(reinterpret_cast<void**>(&pl->beams[lf]), bl.data(), bl.size() * sizeof(int2));
    // aberration phase of each beam in turns, chi(k_b) / (2 pi) reduced mod 1 in FP64
    std::vector<double> turns(bl.size());
    for (size_t b = 0; b < bl.size(); ++b) {
      const double kx = (double)bl[b].x / lx, ky = (double)bl[b].y / ly;
      const double k2 = kx * kx + ky * ky;
      const double t = 0.5 * pl->lam * params->defocus_a * k2 +
                       0.25 * params->cs_a * pl->lam * pl->lam * pl->lam * k2 * k2;
      turns[b] = t - std::floor(t);
    }
    upload(reinterpret_cast<void**>(&pl->beam_turns[lf]), turns.data(), turns.size() * sizeof(double));
  }
  if (e != cudaSuccess) {
    stem_plan_destroy(pl);
    return e == cudaErrorMemoryAllocation ? STEM_ERR_NOMEM : STEM_ERR_CUDA;
  }
  *out = pl;
  return STEM_OK;
}

stem_status stem_plan_device_status(stem_plan pl, int32_t* code) {
  if (!pl || !code) return STEM_ERR_INVALID;
  int v = 0;
  if (cudaMemcpy(&v, pl->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return STEM_ERR_CUDA;
  const int zero = 0;
  if (v != 0 && cudaMemcpy(pl->status, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return STEM_ERR_CUDA;
  *code = v;
  return STEM_OK;
}

stem_status stem_plan_constants(stem_plan pl, double* lambda_a, double* sigma, int32_t* n_aperture) {
  if (!pl) return STEM_ERR_INVALID;
  if (lambda_a) *lambda_a = pl->lam;
  if (sigma) *sigma = pl->sigma;
  if (n_aperture) *n_aperture = pl->n_aperture;
  return STEM_OK;
}

stem_status stem_plan_set_detector_edges(stem_plan pl, int32_t n_edges, const double* edges_mrad) {
  if (!pl || n_edges < 2 || n_edges - 1 > kMaxRings || !edges_mrad) return STEM_ERR_INVALID;
  for (int i = 0; i < n_edges; ++i) {
    if (!std::isfinite(edges_mrad[i]) || edges_mrad[i] < 0.0) return STEM_ERR_INVALID;
    if (i > 0 && !(edges_mrad[i] > edges_mrad[i - 1])) return STEM_ERR_INVALID;
  }
  std::vector<double> edges(edges_mrad, edges_mrad + n_edges);
  stem_params p = pl->p;
  p.n_rings = n_edges - 1;
  std::vector<uint16_t> lut;
  build_fine_lut(p, pl->lam, edges, lut);
  {
    const std::vector<uint16_t> lt = transpose_lut(lut, pl->n);
    if (cudaMemcpy(pl->lut_t, lt.data(), lt.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess)
      return STEM_ERR_CUDA;
  }
  for (int lf = 0; lf <= kMaxLog2F; ++lf) {
    const int f = 1 << lf;
    if (f > pl->n / 8 || !pl->lut[lf]) break;
    const std::vector<uint16_t> coarse = coarse_lut(lut, pl->n, f, pl->n / f);
    if (cudaMemcpy(pl->lut[lf], coarse.data(), coarse.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return STEM_ERR_CUDA;
    if (pl->lut_crop[lf]) {
      const std::vector<uint16_t> crop = coarse_lut(lut, pl->n, f, smatrix_grid(pl->n, true) / f);
      if (cudaMemcpy(pl->lut_crop[lf], crop.data(), crop.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) !=
          cudaSuccess)
        return STEM_ERR_CUDA;
    }
  }
  pl->edges = edges;
  pl->p.n_rings = p.n_rings;
  return STEM_OK;
}

// ----------------------------------------------------------------------------- potentials
size_t stem_slice_potentials_workspace(stem_plan pl, int64_t n_atoms) {
  if (!pl || n_atoms < 0 || pl->n < 64) return 0;
  return potential_workspace(n_atoms, pl->n, pl->p.n_slices);
}

stem_status stem_slice_potentials(stem_plan pl, const double* xyz, const float* gauss, int64_t n_atoms, float* v_out,
                                  void* trans_out, void* ws, size_t ws_bytes, void* stream) {
  if (!pl || n_atoms < 0 || (n_atoms > 0 && (!xyz || !gauss)) || (!v_out && !trans_out) || !ws)
    return STEM_ERR_INVALID;
  if (pl->n < 64) return STEM_ERR_UNSUPPORTED;
  if (ws_bytes < potential_workspace(n_atoms, pl->n, pl->p.n_slices)) return STEM_ERR_NOMEM;
  return cuda_status(launch_potentials(pl->p, pl->sigma, xyz, gauss, n_atoms, v_out,
                                       static_cast<float2*>(trans_out), ws, as_stream(stream)));
}

// ----------------------------------------------------------------------------- multislice
size_t stem_multislice_workspace(stem_plan pl, int32_t batch) {
  if (!pl || batch < 1) return 0;
  return (size_t)batch * pl->n * pl->n * sizeof(float2);
}

// The slice loop of Eq. 1 and Eq. 2 over batches of probes; the last column
// pass bins |Psi_hat|^2 into rings (dp == NULL) or accumulates the whole
// diffraction pattern into dp.
static stem_status run_multislice(stem_plan pl, const void* trans, bool streamed, const double* probe_xy,
                                  int64_t n_probes, int32_t batch, float weight, float* rings_out, float* dp_out,
                                  void* ws, size_t ws_bytes, void* stream) {
  if (!pl || !trans || n_probes < 0 || (n_probes > 0 && (!probe_xy || (!rings_out && !dp_out))) || batch < 1 ||
      batch > 65535 || !ws)
    return STEM_ERR_INVALID;
  const int n = pl->n;
  if (n < 64) return STEM_ERR_UNSUPPORTED;
  const size_t waves = stem_multislice_workspace(pl, batch);
  if (ws_bytes < (streamed ? stem_multislice_streamed_workspace(pl, batch) : waves)) return STEM_ERR_NOMEM;
  cudaStream_t s = as_stream(stream);
  const size_t plane = (size_t)n * n;
  const float2* t = static_cast<const float2*>(trans);
  float2* bufs = reinterpret_cast<float2*>(static_cast<char*>(ws) + waves);
  std::unique_ptr<SliceSource> src(streamed ? new (std::nothrow) SliceSource(t, plane, bufs)
                                             : new (std::nothrow) SliceSource(t, plane));
  if (!src) return STEM_ERR_NOMEM;
  if (n_probes > 0 && src->begin(s) != cudaSuccess) return STEM_ERR_CUDA;
  PassArgs a;
  a.wave = static_cast<float2*>(ws);
  a.prop_x = pl->prop_x;
  a.prop_y = pl->prop_y;
  a.prop_scale = 1.0f / (float)plane;
  a.lut = pl->lut[0];
  a.lut_t = pl->lut_t;
  a.n_rings = pl->p.n_rings;
  a.ring_scale = weight;
  a.inv_lx = 1.0 / pl->p.cell[0];
  a.inv_ly = 1.0 / pl->p.cell[1];
  a.probe_norm = (float)(1.0 / (std::sqrt((double)std::max(pl->n_aperture, 1)) * (double)plane));
  a.band = 1;   // the last column pass reads waves whose out-of-band columns were never written
  a.chi_c1 = 0.5 * pl->lam * pl->p.defocus_a;
  a.chi_c3 = 0.25 * pl->p.cs_a * pl->lam * pl->lam * pl->lam;
  a.status = pl->status;
  const int last = dp_out ? COL_DP : COL_DET;
  for (int64_t p0 = 0; p0 < n_probes; p0 += batch) {
    a.batch = (int)std::min<int64_t>(batch, n_probes - p0);
    a.probe_xy = probe_xy + 2 * p0;
    if (rings_out) a.rings = rings_out + p0 * pl->p.n_rings;
    if (dp_out) a.dp = dp_out + p0 * plane;
    cudaError_t e = launch_col_pass(n, COL_PROBE_INIT, a, s);
    for (int sl = 0; sl < pl->p.n_slices && e == cudaSuccess; ++sl) {
      e = src->acquire(sl, s, &a.trans);
      if (e == cudaSuccess) e = launch_row_pass(n, ROW_SLICE, a, s);
      if (e == cudaSuccess) e = src->release(s);
      if (e == cudaSuccess) e = launch_col_pass(n, sl + 1 < pl->p.n_slices ? COL_SLICE : last, a, s);
    }
    if (e != cudaSuccess) return STEM_ERR_CUDA;
  }
  return STEM_OK;
}

stem_status stem_multislice_scan(stem_plan pl, const void* trans, const double* probe_xy, int64_t n_probes,
                                 int32_t batch, float weight, float* rings_out, void* ws, size_t ws_bytes,
                                 void* stream) {
  if (n_probes > 0 && !rings_out) return STEM_ERR_INVALID;
  return run_multislice(pl, trans, false, probe_xy, n_probes, batch, weight, rings_out, nullptr, ws, ws_bytes, stream);
}

size_t stem_multislice_streamed_workspace(stem_plan pl, int32_t batch) {
  if (!pl || batch < 1) return 0;
  return stem_multislice_workspace(pl, batch) + (size_t)kStreamBufs * pl->n * pl->n * sizeof(float2);
}

stem_status stem_multislice_scan_streamed(stem_plan pl, const void* trans_host, const double* probe_xy,
                                          int64_t n_probes, int32_t batch, float weight, float* rings_out, void* ws,
                                          size_t ws_bytes, void* stream) {
  if (n_probes > 0 && !rings_out) return STEM_ERR_INVALID;
  return run_multislice(pl, trans_host, true, probe_xy, n_probes, batch, weight, rings_out, nullptr, ws, ws_bytes,
                        stream);
}

stem_status stem_multislice_scan_4d(stem_plan pl, const void* trans, const double* probe_xy, int64_t n_probes,
                                    int32_t batch, float weight, float* dp_out, void* ws, size_t ws_bytes,
                                    void* stream) {
  if (n_probes > 0 && !dp_out) return STEM_ERR_INVALID;
  return run_multislice(pl, trans, false, probe_xy, n_probes, batch, weight, nullptr, dp_out, ws, ws_bytes, stream);
}

// ----------------------------------------------------------------------------- PRISM S-matrix
stem_status stem_prism_beams(stem_plan pl, int32_t f, int32_t* n_beams, int32_t* mn_host) {
  if (!pl || !n_beams || !f_ok(pl, f)) return STEM_ERR_INVALID;
  const int lf = log2i(f);
  *n_beams = pl->n_beams[lf];
  if (mn_host)
    for (int b = 0; b < pl->n_beams[lf]; ++b) {
      mn_host[2 * b] = pl->h_beams[lf][b].x;
      mn_host[2 * b + 1] = pl->h_beams[lf][b].y;
    }
  return STEM_OK;
}

size_t stem_prism_smatrix_bytes(stem_plan pl, int32_t f, stem_storage storage) {
  int elem;
  bool crop;
  if (!pl || !f_ok(pl, f) || !decode_storage(storage, &elem, &crop) || (crop && pl->n < 64)) return 0;
  return smatrix_layout(smatrix_grid(pl->n, crop), pl->n_beams[log2i(f)], elem).total;
}

static size_t smatrix_ws_waves(int n, int batch) { return ((size_t)batch * n * n * sizeof(float2) + 255) / 256 * 256; }

// S-matrix workspace: the batch's waves, the beams' maxima, the 2D transform
// of t_0
static size_t smatrix_ws_t0hat(int n, int batch) {
  return smatrix_ws_waves(n, batch) + ((size_t)batch * sizeof(unsigned) + 255) / 256 * 256;
}

size_t stem_prism_smatrix_workspace(stem_plan pl, int32_t batch) {
  if (!pl || batch < 1) return 0;
  return smatrix_ws_t0hat(pl->n, batch) + (size_t)pl->n * pl->n * sizeof(float2);
}

size_t stem_prism_smatrix_streamed_workspace(stem_plan pl, int32_t batch) {
  if (!pl || batch < 1) return 0;
  return (stem_prism_smatrix_workspace(pl, batch) + 255) / 256 * 256 +
         (size_t)kStreamBufs * pl->n * pl->n * sizeof(float2);
}

// Beams [b_begin, b_end) of the S-matrix (b_end < 0: to the last beam).
static stem_status run_smatrix(stem_plan pl, const void* trans, bool streamed, int32_t f, stem_storage storage,
                               int32_t batch, void* smatrix, size_t smatrix_bytes, void* ws, size_t ws_bytes,
                               void* stream, int32_t b_begin = 0, int32_t b_end = -1) {
  int elem;
  bool crop;
  if (!pl || !trans || !smatrix || !ws || !f_ok(pl, f) || !decode_storage(storage, &elem, &crop) || batch < 1 ||
      batch > 65535)
    return STEM_ERR_INVALID;
  const int n = pl->n;
  if (n < 64) return STEM_ERR_UNSUPPORTED;
  const int lf = log2i(f);
  const int nb = pl->n_beams[lf];
  if (b_end < 0) b_end = nb;
  if (b_begin < 0 || b_begin > b_end || b_end > nb) return STEM_ERR_INVALID;
  const int n_out = smatrix_grid(n, crop);
  const SmatLayout L = smatrix_layout(n_out, nb, elem);
  const size_t need = streamed ? stem_prism_smatrix_streamed_workspace(pl, batch) : stem_prism_smatrix_workspace(pl, batch);
  if (smatrix_bytes < L.total || ws_bytes < need) return STEM_ERR_NOMEM;
  if (reinterpret_cast<uintptr_t>(smatrix) % 256) return STEM_ERR_INVALID;
  cudaStream_t s = as_stream(stream);
  const size_t plane = (size_t)n * n;
  const float2* t = static_cast<const float2*>(trans);
  float2* bufs = reinterpret_cast<float2*>(static_cast<char*>(ws) +
                                           (stem_prism_smatrix_workspace(pl, batch) + 255) / 256 * 256);
  std::unique_ptr<SliceSource> src(streamed ? new (std::nothrow) SliceSource(t, plane, bufs)
                                             : new (std::nothrow) SliceSource(t, plane));
  if (!src) return STEM_ERR_NOMEM;
  if (src->begin(s) != cudaSuccess) return STEM_ERR_CUDA;
  PassArgs a;
  a.wave = static_cast<float2*>(ws);
  a.prop_x = pl->prop_x;
  a.prop_y = pl->prop_y;
  a.prop_scale = 1.0f / (float)plane;
  a.beam_max = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + smatrix_ws_waves(n, batch));
  a.status = pl->status;
  // The first slice of every beam starts from the 2D transform of t_0: the
  // transform of t_0 times a plane wave (m, n) is that transform shifted by
  // (m, n), so one transform per call replaces a row pass and a column
  // transform per beam.
  float2* t0hat = reinterpret_cast<float2*>(static_cast<char*>(ws) + smatrix_ws_t0hat(n, batch));
  {
    const float2* t0 = nullptr;
    cudaError_t e = src->acquire(0, s, &t0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t0hat, t0, plane * sizeof(float2), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = src->release(s);
    PassArgs a0 = a;
    a0.wave = t0hat;
    a0.batch = 1;
    a0.band = 0;
    if (e == cudaSuccess) e = launch_row_pass(n, ROW_FFT, a0, s);
    if (e == cudaSuccess) e = launch_col_pass(n, COL_FFT, a0, s);
    if (e != cudaSuccess) return STEM_ERR_CUDA;
  }
  a.t0hat = t0hat;
  for (int b0 = b_begin; b0 < b_end; b0 += batch) {
    a.batch = std::min(batch, b_end - b0);
    a.beams = pl->beams[lf] + b0;
    cudaError_t e = cudaMemsetAsync(a.beam_max, 0, a.batch * sizeof(unsigned), s);
    for (int sl = 0; sl < pl->p.n_slices && e == cudaSuccess; ++sl) {
      const bool last = sl + 1 == pl->p.n_slices;
      // cropped: the last column pass leaves the spectrum for the crop
      if (sl == 0) {
        e = launch_col_pass(n, crop && last ? COL_BEAM0_SPEC : COL_BEAM0, a, s);
        continue;
      }
      e = src->acquire(sl, s, &a.trans);
      if (e == cudaSuccess) e = launch_row_pass(n, ROW_SLICE, a, s);
      if (e == cudaSuccess) e = src->release(s);
      if (e == cudaSuccess) e = launch_col_pass(n, crop && last ? COL_SPEC : COL_SLICE, a, s);
    }
    if (e == cudaSuccess)
      e = crop ? launch_crop_finish(a.wave, a.batch, n, a.beam_max, s) : launch_row_pass(n, ROW_IFFT_MAX, a, s);
    if (e == cudaSuccess)
      e = launch_smatrix_store(a.wave, a.batch, n, n_out, b0, nb, a.beam_max, elem, L, smatrix, s);
    if (e != cudaSuccess) return STEM_ERR_CUDA;
  }
  return STEM_OK;
}

stem_status stem_prism_smatrix(stem_plan pl, const void* trans, int32_t f, stem_storage storage, int32_t batch,
                               void* smatrix, size_t smatrix_bytes, void* ws, size_t ws_bytes, void* stream) {
  return run_smatrix(pl, trans, false, f, storage, batch, smatrix, smatrix_bytes, ws, ws_bytes, stream);
}

stem_status stem_prism_smatrix_range(stem_plan pl, const void* trans, int32_t f, stem_storage storage, int32_t batch,
                                     int32_t b_begin, int32_t b_end, void* smatrix, size_t smatrix_bytes, void* ws,
                                     size_t ws_bytes, void* stream) {
  if (b_end < 0) return STEM_ERR_INVALID;
  return run_smatrix(pl, trans, false, f, storage, batch, smatrix, smatrix_bytes, ws, ws_bytes, stream, b_begin,
                     b_end);
}

stem_status stem_prism_smatrix_streamed(stem_plan pl, const void* trans_host, int32_t f, stem_storage storage,
                                        int32_t batch, void* smatrix, size_t smatrix_bytes, void* ws,
                                        size_t ws_bytes, void* stream) {
  return run_smatrix(pl, trans_host, true, f, storage, batch, smatrix, smatrix_bytes, ws, ws_bytes, stream);
}

// ----------------------------------------------------------------------------- PRISM output
size_t stem_prism_output_workspace(stem_plan pl, int32_t f, int32_t chunk) {
  if (!pl || !f_ok(pl, f) || chunk < 1) return 0;
  const SmatLayout L = smatrix_layout(pl->n, pl->n_beams[log2i(f)], STEM_F32);
  return output_workspace_layout(pl->n, f, chunk, L.nbp).total;
}

static stem_status output_common(stem_plan pl, int32_t f, stem_storage storage, int32_t engine, const void* smatrix,
                                 OutputArgs& o) {
  int elem;
  bool crop;
  if (!pl || !smatrix || !f_ok(pl, f) || !decode_storage(storage, &elem, &crop)) return STEM_ERR_INVALID;
  if (engine < STEM_SUM_AUTO || engine > STEM_SUM_TENSOR) return STEM_ERR_INVALID;
  if (pl->n < 64) return STEM_ERR_UNSUPPORTED;
  const int lf = log2i(f);
  const int ng = smatrix_grid(pl->n, crop);
  const SmatLayout L = smatrix_layout(ng, pl->n_beams[lf], elem);
  o.n = ng;
  o.f = f;
  o.w = ng / f;
  o.cropped = crop;
  o.storage = elem;
  o.engine = engine == STEM_SUM_AUTO ? (elem == STEM_F32 ? STEM_SUM_SIMT : STEM_SUM_TENSOR) : engine;
  if (o.engine == STEM_SUM_TENSOR && elem == STEM_F32) return STEM_ERR_UNSUPPORTED;
  o.status = pl->status;
  o.n_beams = L.n_beams;
  o.nbp = L.nbp;
  o.beams = pl->beams[lf];
  o.beam_turns = pl->beam_turns[lf];
  o.smatrix = smatrix;
  o.scales = static_cast<const float*>(smatrix);
  o.sdata = static_cast<const char*>(smatrix) + L.data_offset;
  o.lx = pl->p.cell[0];
  o.ly = pl->p.cell[1];
  o.dx = pl->p.cell[0] / ng;
  o.dy = pl->p.cell[1] / ng;
  o.coef_norm = (float)(1.0 / std::sqrt((double)std::max(L.n_beams, 1)));
  return STEM_OK;
}

stem_status stem_prism_windows(stem_plan pl, int32_t f, stem_storage storage, int32_t engine, const void* smatrix,
                               const double* probe_xy, int64_t n_probes, void* windows_out, void* ws, size_t ws_bytes,
                               void* stream) {
  OutputArgs o;
  stem_status st = output_common(pl, f, storage, engine, smatrix, o);
  if (st != STEM_OK) return st;
  if (n_probes < 0 || n_probes > 65535 || (n_probes > 0 && (!probe_xy || !windows_out)) || !ws)
    return STEM_ERR_INVALID;
  if (n_probes == 0) return STEM_OK;
  const OutputWs L = output_workspace_layout(o.n, f, (int)n_probes, o.nbp);
  if (ws_bytes < L.total) return STEM_ERR_NOMEM;
  return cuda_status(prism_windows_chunk(o, probe_xy, (int)n_probes, static_cast<float2*>(windows_out),
                                         static_cast<char*>(ws), L, as_stream(stream)));
}

static stem_status run_prism_output(stem_plan pl, int32_t f, stem_storage storage, int32_t engine, const void* smatrix,
                                    const double* probe_xy, int64_t n_probes, int32_t chunk, float weight,
                                    float* rings_out, float* dp_out, void* ws, size_t ws_bytes, void* stream) {
  OutputArgs o;
  stem_status st = output_common(pl, f, storage, engine, smatrix, o);
  if (st != STEM_OK) return st;
  if (n_probes < 0 || (n_probes > 0 && (!probe_xy || (!rings_out && !dp_out))) || chunk < 1 || chunk > 65535 || !ws)
    return STEM_ERR_INVALID;
  const OutputWs L = output_workspace_layout(o.n, f, chunk, o.nbp);
  if (ws_bytes < L.total) return STEM_ERR_NOMEM;
  cudaStream_t s = as_stream(stream);
  char* base = static_cast<char*>(ws);
  float2* windows = reinterpret_cast<float2*>(base + L.windows);
  const int lf = log2i(f);
  const double w4 = std::pow((double)o.w, 4.0);
  for (int64_t c0 = 0; c0 < n_probes; c0 += chunk) {
    const int np = (int)std::min<int64_t>(chunk, n_probes - c0);
    cudaError_t e = prism_windows_chunk(o, probe_xy + 2 * c0, np, windows, base, L, s);
    PassArgs a;
    a.wave = windows;
    a.batch = np;
    a.lut = pl->lut[lf];
    a.n_rings = pl->p.n_rings;
    if (rings_out) a.rings = rings_out + c0 * pl->p.n_rings;
    if (dp_out) a.dp = dp_out + c0 * (size_t)o.w * o.w;
    a.ring_scale = (float)(weight / w4);
    if (o.cropped) {
      // W' = 3N / (4f) windows; the band limit in coarse units is (N / f)^2
      const int wf = pl->n / f;
      if (e == cudaSuccess)
        e = launch_window_fft3(o.w, windows, np, pl->lut_crop[lf], a.n_rings, a.ring_scale, a.rings, a.dp, wf * wf, s);
    } else {
      if (e == cudaSuccess) e = launch_row_pass(o.w, ROW_FFT, a, s);
      if (e == cudaSuccess) e = launch_col_pass(o.w, dp_out ? COL_DP : COL_DET, a, s);
    }
    if (e != cudaSuccess) return STEM_ERR_CUDA;
  }
  return STEM_OK;
}

stem_status stem_prism_output(stem_plan pl, int32_t f, stem_storage storage, int32_t engine, const void* smatrix,
                              const double* probe_xy, int64_t n_probes, int32_t chunk, float weight,
                              float* rings_out, void* ws, size_t ws_bytes, void* stream) {
  if (n_probes > 0 && !rings_out) return STEM_ERR_INVALID;
  return run_prism_output(pl, f, storage, engine, smatrix, probe_xy, n_probes, chunk, weight, rings_out, nullptr, ws,
                          ws_bytes, stream);
}

stem_status stem_prism_output_4d(stem_plan pl, int32_t f, stem_storage storage, int32_t engine, const void* smatrix,
                                 const double* probe_xy, int64_t n_probes, int32_t chunk, float weight,
                                 float* dp_out, void* ws, size_t ws_bytes, void* stream) {
  if (n_probes > 0 && !dp_out) return STEM_ERR_INVALID;
  return run_prism_output(pl, f, storage, engine, smatrix, probe_xy, n_probes, chunk, weight, nullptr, dp_out, ws,
                          ws_bytes, stream);
}

// ----------------------------------------------------------------------------- detector, FFT
stem_status stem_detector_readout(stem_plan pl, int32_t f, const void* psi_k, int64_t batch, float scale,
                                  float* rings_out, void* stream) {
  if (!pl || !f_ok(pl, f) || batch < 0 || batch > 65535 || (batch > 0 && (!psi_k || !rings_out)))
    return STEM_ERR_INVALID;
  return cuda_status(launch_readout(pl->n / f, static_cast<const float2*>(psi_k), batch, pl->lut[log2i(f)],
                                    pl->p.n_rings, scale, rings_out, as_stream(stream)));
}

stem_status stem_fft2(int32_t n, int64_t batch, int32_t inverse, void* data, void* stream) {
  if (!is_pow2(n) || n < 8 || n > 2048) return STEM_ERR_UNSUPPORTED;
  if (batch < 0 || batch > 65535 || (batch > 0 && !data)) return STEM_ERR_INVALID;
  PassArgs a;
  a.wave = static_cast<float2*>(data);
  a.batch = (int)batch;
  cudaStream_t s = as_stream(stream);
  cudaError_t e = launch_row_pass(n, inverse ? ROW_IFFT : ROW_FFT, a, s);
  if (e == cudaSuccess) e = launch_col_pass(n, inverse ? COL_IFFT : COL_FFT, a, s);
  return cuda_status(e);
}

// ----------------------------------------------------------------------------- footprint
size_t stem_footprint_bytes(const stem_params* p, int32_t algo, int32_t f, stem_storage storage, int64_t n_probes,
                            int32_t batch) {
  if (check_params(p) != STEM_OK || batch < 1) return 0;
  const size_t n = (size_t)p->n, plane = n * n;
  const size_t trans = (size_t)p->n_slices * plane * sizeof(float2);
  const size_t rings = (size_t)std::max<int64_t>(n_probes, 0) * p->n_rings * sizeof(float);
  if (algo < 0 || algo > 3) return 0;
  const size_t stack = algo >= 2 ? (size_t)kStreamBufs * plane * sizeof(float2) : trans;
  if (algo == 0 || algo == 2) return stack + (size_t)batch * plane * sizeof(float2) + rings;
  if (!is_pow2(f) || f > p->n / 8) return 0;
  int elem;
  bool crop;
  if (!decode_storage(storage, &elem, &crop) || (crop && p->n < 64)) return 0;
  const int nb = count_beams(p, f, wavelength_a(p->energy_kev));
  const SmatLayout L = smatrix_layout(smatrix_grid(p->n, crop), nb, elem);
  const int chunk = (int)std::min<int64_t>(std::max<int64_t>(n_probes, 1), 4096);
  // S-matrix workspace (waves, beam maxima, row transforms of t_0), S-matrix, output workspace
  return stack + L.total + (size_t)batch * plane * sizeof(float2) + ((size_t)batch * 4 + 255) / 256 * 256 +
         plane * sizeof(float2) + output_workspace_layout(p->n, f, chunk, L.nbp).total + rings;
}

}  // extern "C"
