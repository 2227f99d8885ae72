/*
 * stem_client.c - a plain C (C99) client of libstem: no Python, no PyTorch.
 * Used by the tests to show that the C ABI stands on its own.
 *
 *   stem_client <inputs.bin> <rings.bin>
 *
 * inputs.bin (little endian): int32 n, n_slices, n_rings, n_atoms, n_probes;
 * float64 cell[3], slice_dz, energy_kev, alpha_mrad, ring_width_mrad;
 * float64 xyz[n_atoms][3]; float32 gauss[n_atoms][4]; float64 probe_xy[n_probes][2].
 * The client builds the plan, the potentials and the multislice rings with
 * device buffers it allocates itself, and writes float32 rings[n_probes][n_rings].
 * Exit status 0 on success; a message on stderr otherwise.
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "stem.h"

#define CHECK_CUDA(x)                                                            \
  do {                                                                           \
    cudaError_t e_ = (x);                                                        \
    if (e_ != cudaSuccess) {                                                     \
      fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));                   \
      return 2;                                                                  \
    }                                                                            \
  } while (0)
#define CHECK_STEM(x)                                                            \
  do {                                                                           \
    stem_status s_ = (x);                                                        \
    if (s_ != STEM_OK) {                                                         \
      fprintf(stderr, "%s: %s\n", #x, stem_status_string(s_));                   \
      return 3;                                                                  \
    }                                                                            \
  } while (0)

static int read_all(FILE* f, void* dst, size_t bytes) { return fread(dst, 1, bytes, f) == bytes; }

int main(int argc, char** argv) {
  if (argc != 3) {
    fprintf(stderr, "usage: %s inputs.bin rings.bin\n", argv[0]);
    return 1;
  }
  FILE* in = fopen(argv[1], "rb");
  if (!in) return 1;
  int32_t hdr[5];
  double geo[7];
  if (!read_all(in, hdr, sizeof hdr) || !read_all(in, geo, sizeof geo)) return 1;
  const int n = hdr[0], n_slices = hdr[1], n_rings = hdr[2], n_atoms = hdr[3], n_probes = hdr[4];
  double* xyz = malloc((size_t)n_atoms * 3 * sizeof(double));
  float* gauss = malloc((size_t)n_atoms * 4 * sizeof(float));
  double* xy = malloc((size_t)n_probes * 2 * sizeof(double));
  float* rings = malloc((size_t)n_probes * n_rings * sizeof(float));
  if (!xyz || !gauss || !xy || !rings) return 1;
  if (!read_all(in, xyz, (size_t)n_atoms * 3 * sizeof(double)) ||
      !read_all(in, gauss, (size_t)n_atoms * 4 * sizeof(float)) ||
      !read_all(in, xy, (size_t)n_probes * 2 * sizeof(double)))
    return 1;
  fclose(in);

  stem_params p;
  memset(&p, 0, sizeof p);
  p.cell[0] = geo[0];
  p.cell[1] = geo[1];
  p.cell[2] = geo[2];
  p.n = n;
  p.n_slices = n_slices;
  p.slice_dz = geo[3];
  p.energy_kev = geo[4];
  p.alpha_mrad = geo[5];
  p.ring_width_mrad = geo[6];
  p.n_rings = n_rings;
  stem_plan plan;
  CHECK_STEM(stem_plan_create(&p, &plan));

  const size_t plane = (size_t)n * n;
  double *d_xyz, *d_xy;
  float *d_gauss, *d_v, *d_rings;
  void *d_trans, *d_ws, *d_pws;
  const int batch = n_probes < 64 ? n_probes : 64;
  const size_t ws_bytes = stem_multislice_workspace(plan, batch);
  const size_t pws_bytes = stem_slice_potentials_workspace(plan, n_atoms);
  CHECK_CUDA(cudaMalloc((void**)&d_xyz, (size_t)n_atoms * 3 * sizeof(double) + 16));
  CHECK_CUDA(cudaMalloc((void**)&d_gauss, (size_t)n_atoms * 4 * sizeof(float) + 16));
  CHECK_CUDA(cudaMalloc((void**)&d_xy, (size_t)n_probes * 2 * sizeof(double)));
  CHECK_CUDA(cudaMalloc((void**)&d_v, (size_t)n_slices * plane * sizeof(float)));
  CHECK_CUDA(cudaMalloc(&d_trans, (size_t)n_slices * plane * 8));
  CHECK_CUDA(cudaMalloc((void**)&d_rings, (size_t)n_probes * n_rings * sizeof(float)));
  CHECK_CUDA(cudaMalloc(&d_ws, ws_bytes));
  CHECK_CUDA(cudaMalloc(&d_pws, pws_bytes));
  CHECK_CUDA(cudaMemcpy(d_xyz, xyz, (size_t)n_atoms * 3 * sizeof(double), cudaMemcpyHostToDevice));
  CHECK_CUDA(cudaMemcpy(d_gauss, gauss, (size_t)n_atoms * 4 * sizeof(float), cudaMemcpyHostToDevice));
  CHECK_CUDA(cudaMemcpy(d_xy, xy, (size_t)n_probes * 2 * sizeof(double), cudaMemcpyHostToDevice));
  CHECK_CUDA(cudaMemset(d_rings, 0, (size_t)n_probes * n_rings * sizeof(float)));

  CHECK_STEM(stem_slice_potentials(plan, d_xyz, d_gauss, n_atoms, d_v, d_trans, d_pws, pws_bytes, NULL));
  CHECK_STEM(stem_multislice_scan(plan, d_trans, d_xy, n_probes, batch, 1.0f, d_rings, d_ws, ws_bytes, NULL));
  CHECK_CUDA(cudaDeviceSynchronize());
  int32_t code = 0;
  CHECK_STEM(stem_plan_device_status(plan, &code));
  if (code != 0) {
    fprintf(stderr, "device status %d\n", code);
    return 4;
  }
  CHECK_CUDA(cudaMemcpy(rings, d_rings, (size_t)n_probes * n_rings * sizeof(float), cudaMemcpyDeviceToHost));

  FILE* out = fopen(argv[2], "wb");
  if (!out || fwrite(rings, sizeof(float), (size_t)n_probes * n_rings, out) != (size_t)n_probes * n_rings) return 1;
  fclose(out);
  printf("stem_client: %d probes x %d rings, launches %llu\n", n_probes, n_rings,
         (unsigned long long)stem_launch_count());
  stem_plan_destroy(plan);
  cudaFree(d_xyz); cudaFree(d_gauss); cudaFree(d_xy); cudaFree(d_v); cudaFree(d_trans);
  cudaFree(d_rings); cudaFree(d_ws); cudaFree(d_pws);
  free(xyz); free(gauss); free(xy); free(rings);
  return 0;
}
