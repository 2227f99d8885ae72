// internal.h - shared declarations of libstem's CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/stem.h"

namespace stem {

constexpr int kMaxLog2F = 11;      // f = 1 .. 2048
constexpr int kMaxRings = 2048;
constexpr uint16_t kLutNoRing = 0x7FFF;
constexpr uint16_t kLutAperture = 0x8000;

// Arguments of the fused row / column FFT passes.  Waves are [batch][N][N]
// complex64, contiguous.
struct PassArgs {
  float2* wave = nullptr;
  int batch = 0;
  const float2* trans = nullptr;     // t_n [N][N] of the current slice (row passes)
  const float2* prop_x = nullptr;    // exp(-i pi lambda dz (m/Lx)^2), [N]
  const float2* prop_y = nullptr;    // exp(-i pi lambda dz (n/Ly)^2), [N]
  float prop_scale = 1.0f;           // 1/N^2 folds the inverse-FFT normalisation in
  const uint16_t* lut = nullptr;     // [N][N]: bit 15 aperture, bits 0..14 ring or 0x7FFF
  const uint16_t* lut_t = nullptr;   // the same table transposed, [x][y] (column-wise reads)
  int n_rings = 0;
  float* rings = nullptr;            // [batch][n_rings] (offset to the batch's first wave)
  float ring_scale = 1.0f;
  const double* probe_xy = nullptr;  // [batch][2] (offset)
  double inv_lx = 0.0, inv_ly = 0.0;
  float probe_norm = 0.0f;           // 1 / (sqrt(|A|) N^2)
  const int2* beams = nullptr;       // [batch] (m, n) (offset)
  const float2* t0hat = nullptr;     // COL_BEAM0*: the 2D transform of t_0, [N][N]
  unsigned* beam_max = nullptr;      // [batch] float bits of max(|Re|, |Im|)
  int band = 0;                      // COL_DET ends a slice loop: only in-band columns hold data
  double chi_c1 = 0.0, chi_c3 = 0.0; // aberration phase in turns: chi_c1 |k|^2 + chi_c3 |k|^4
  float* dp = nullptr;               // COL_DP: [batch][N][N] intensities, += ring_scale |psi|^2
  int* status = nullptr;             // plan status word (bounded waits record timeouts), or null
};

enum RowMode { ROW_SLICE = 0, ROW_IFFT_MAX = 2, ROW_FFT = 3, ROW_IFFT = 4 };
// COL_BEAM0 / COL_BEAM0_SPEC: the first slice of the S-matrix build, from the
// 2D transform of t_0 shifted by each beam (then as COL_SLICE / COL_SPEC
// without the forward transform)
enum ColMode {
  COL_SLICE = 0, COL_DET = 1, COL_PROBE_INIT = 2, COL_FFT = 3, COL_IFFT = 4, COL_DP = 5, COL_SPEC = 6,
  COL_BEAM0 = 7, COL_BEAM0_SPEC = 8
};

// Counts this library's kernel launches (stem_launch_count); called at every launch site.
void note_launch();

// Brackets the kernel launch that follows it, in the same scope, with a pair of
// CUDA events on stream s while stem_profile_enable(1) is in force
// (profile.cu); kind is a stem_prof_kind.
class ProfScope {
 public:
  ProfScope(int kind, cudaStream_t s);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  cudaEvent_t stop_ = nullptr;
  cudaStream_t stream_ = nullptr;
};

cudaError_t launch_row_pass(int n, int mode, const PassArgs& a, cudaStream_t s);
cudaError_t launch_col_pass(int n, int mode, const PassArgs& a, cudaStream_t s);

// Potentials (potential.cu)
size_t potential_workspace(int64_t n_atoms, int n, int n_slices);
cudaError_t launch_potentials(const stem_params& p, double sigma, const double* xyz, const float* gauss,
                              int64_t n_atoms, float* v_out, float2* t_out, void* ws, cudaStream_t s);

// PRISM helpers (prism.cu)
struct SmatLayout {
  int n_beams = 0;
  int nbp = 0;            // beams padded to 64
  size_t data_offset = 0; // bytes
  size_t elem_bytes = 4;
  size_t total = 0;
};
SmatLayout smatrix_layout(int n, int n_beams, int storage);

// waves [nb][n][n]; the stored pixels are the top-left n_out x n_out of each
// wave (n_out = n, or N' = 3n/4 for the Fourier-cropped S-matrix)
cudaError_t launch_smatrix_store(const float2* waves, int nb, int n, int n_out, int b0, int n_beams_total,
                                 const unsigned* beam_max, int storage, const SmatLayout& L,
                                 void* smatrix, cudaStream_t s);

// Fourier-cropped S-matrix (crop.cu): from the spectra / N^2 in the in-band
// columns of each wave [n][n] to the exit waves on the N' = 3n/4 grid in the
// top-left N' x N' of the same buffer, with each beam's largest |Re|, |Im|.
cudaError_t launch_crop_finish(float2* wave, int batch, int n, unsigned* beam_max, cudaStream_t s);
// W' x W' transforms (W' = 3 * 2^k) of PRISM windows [np][W'][W'] in place, then
// rings (lut: the window's coarse ring table) or, with dp, the 4D pattern inside
// 9 (mu^2 + nu^2) <= band_w2.
cudaError_t launch_window_fft3(int w, float2* win, int np, const uint16_t* lut, int n_rings, float scale,
                               float* rings, float* dp, int band_w2, cudaStream_t s);

struct OutputWs {
  size_t coef = 0, origin = 0, counts = 0, offsets = 0, work = 0, items = 0, list = 0, windows = 0, total = 0;
};
OutputWs output_workspace_layout(int n, int f, int chunk, int nbp);

struct OutputArgs {
  int n = 0, f = 0, w = 0, storage = 0, engine = 0;   // n, w: the S-matrix grid and window (cropped or not)
  bool cropped = false;
  int n_beams = 0, nbp = 0;
  const int2* beams = nullptr;
  const double* beam_turns = nullptr;   // chi(k_b) / (2 pi) per beam, reduced mod 1
  const void* smatrix = nullptr;
  const float* scales = nullptr;
  const void* sdata = nullptr;
  double lx = 0, ly = 0, dx = 0, dy = 0;
  float coef_norm = 0.0f;
  int* status = nullptr;    // plan's device status word (bounded waits record timeouts here)
};
// tcgen05 beam sum (umma.cu)
int umma_group();
size_t umma_smem_bytes();
// items[i]: the pixel tile of work item i (items of tile t are work[t] .. work[t+1]-1)
cudaError_t launch_beam_sum_umma(const OutputArgs& o, int np, const double* probe_xy, void* coef, const int2* origin,
                                 const int* offsets, const int* work, const int* items, const int* list, int n_tiles,
                                 float2* windows, cudaStream_t s);

cudaError_t prism_windows_chunk(const OutputArgs& o, const double* probe_xy, int np, float2* windows,
                                char* ws, const OutputWs& L, cudaStream_t s);

// detector readout on a standalone k-space batch (detector.cu)
cudaError_t launch_readout(int w, const float2* psi_k, int64_t batch, const uint16_t* lut, int n_rings,
                           float scale, float* rings, cudaStream_t s);

}  // namespace stem

// Plan object (library-owned device tables).
struct stem_plan_s {
  stem_params p{};
  double lam = 0.0, sigma = 0.0;
  int n = 0;
  int n_aperture = 0;
  int device = 0;
  float2* prop_x = nullptr;
  float2* prop_y = nullptr;
  uint16_t* lut[stem::kMaxLog2F + 1] = {};
  uint16_t* lut_crop[stem::kMaxLog2F + 1] = {};   // window tables W' x W' of the cropped S-matrix
  uint16_t* lut_t = nullptr;                       // lut[0] transposed (the multislice detector pass)
  int2* beams[stem::kMaxLog2F + 1] = {};
  int n_beams[stem::kMaxLog2F + 1] = {};
  double* beam_turns[stem::kMaxLog2F + 1] = {};   // chi(k_b) / (2 pi) mod 1 per beam
  std::vector<int2> h_beams[stem::kMaxLog2F + 1];
  int* status = nullptr;   // device status word, 0 = ok
  std::vector<double> edges;   // detector edges (mrad) when set, else uniform rings
};
