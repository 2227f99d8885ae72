// detector.cu - annular-ring readout of Fourier-space waves.
//
// Methods, "Description of Algorithms": the simulated output is the probe's
// intensity in Fourier space summed over virtual detectors; here an array of
// annular rings (the 3D output).  The ring of each Fourier pixel comes from the
// plan's look-up table (decided once in FP64 on the host); a CTA sums |psi|^2
// into shared-memory rings, a warp's run of equal rings by shuffles first
// (warp_run_add), and adds them to the output once.
#include "fft_core.cuh"
#include "internal.h"

namespace stem {

constexpr int kReadThreads = 256;
constexpr int kReadPix = 4096;   // pixels per CTA

__global__ void __launch_bounds__(kReadThreads) k_readout(const float2* __restrict__ psi, int64_t npix,
                                                          const uint16_t* __restrict__ lut, int n_rings, float scale,
                                                          float* __restrict__ rings) {
  extern __shared__ float acc[];
  const int64_t b = blockIdx.y;
  for (int i = threadIdx.x; i < n_rings; i += kReadThreads) acc[i] = 0.0f;
  __syncthreads();
  const float2* src = psi + b * npix;
  const int64_t p0 = (int64_t)blockIdx.x * kReadPix;
  // consecutive lanes take consecutive pixels of a row, whose rings form runs
  for (int64_t p = p0 + threadIdx.x; p < p0 + kReadPix; p += kReadThreads) {
    const bool in = p < npix;
    const int r = in ? (__ldg(lut + p) & kLutNoRing) : kLutNoRing;
    warp_run_add(acc, r, in ? cabs2(src[p]) : 0.0f, kLutNoRing);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_rings; i += kReadThreads)
    if (acc[i] != 0.0f) atomicAdd(rings + b * n_rings + i, acc[i] * scale);
}

cudaError_t launch_readout(int w, const float2* psi_k, int64_t batch, const uint16_t* lut, int n_rings, float scale,
                           float* rings, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  const int64_t npix = (int64_t)w * w;
  dim3 grid((unsigned)((npix + kReadPix - 1) / kReadPix), (unsigned)batch);
  note_launch(), k_readout<<<grid, kReadThreads, n_rings * sizeof(float), s>>>(psi_k, npix, lut, n_rings, scale, rings);
  return cudaGetLastError();
}

}  // namespace stem
