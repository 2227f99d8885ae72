/*
 * stem.h - C ABI of libstem: multislice and PRISM STEM simulation on one B300 (sm_103a).
 *
 * The operations follow the method of "Prismatic: a streaming multi-GPU
 * implementation of the PRISM and multislice algorithms" (arXiv 1706.08563):
 *   - projected potentials per slice ........ Methods, "Calculation of the Projected Potentials"
 *   - multislice: transmit (Eq. 1), propagate (Eq. 2), repeat over slices,
 *     then |FFT|^2 into annular rings ........ Methods, Eq. 1, Eq. 2 and "Multislice Probe Simulations"
 *   - PRISM compact S-matrix ................. "PRISM Probe Simulations" (first paragraph)
 *   - PRISM output: phase-shifted beam sum in a window cropped by f, FFT,
 *     |.|^2 into rings ....................... "Description of Algorithms" (PRISM paragraph)
 *                                              and "PRISM Probe Simulations" (last paragraph)
 *
 * Conventions shared by every call
 *   - All array pointers are DEVICE pointers owned by the caller unless a
 *     comment says "host".  Every call is asynchronous on `stream` (a
 *     cudaStream_t passed as void*; NULL = the legacy default stream).
 *   - Complex arrays are interleaved single precision (re, im) = "complex64".
 *   - Real-space arrays are [y][x] (row = y).  Fourier arrays use FFT order:
 *     index j holds signed frequency m = j for j < N/2 and m = j - N otherwise;
 *     the spatial frequency is (m / Lx, n / Ly).
 *   - Ring outputs are float32 [n_probes][n_rings] and are ACCUMULATED:
 *     rings_out += weight * I.  Frozen-phonon averaging zeroes once and passes
 *     weight = 1 / n_configs.  Accumulation uses float atomics, so the last
 *     bits of a ring value may differ from run to run.
 *   - Errors are returned, never thrown.  STEM_ERR_INVALID / _UNSUPPORTED /
 *     _NOMEM are returned before anything is launched.  STEM_ERR_CUDA means a
 *     launch failed (the sticky CUDA error is left for the caller to inspect).
 *   - No call allocates device memory except stem_plan_create.  Scratch
 *     memory ("workspace") is passed in by the caller; each call has a
 *     *_workspace query giving the bytes it needs.
 *   - The compute calls can be captured into a CUDA graph once they have run
 *     once plainly (their one-time kernel attribute setup then stays out of
 *     the capture): they neither allocate nor synchronise with the host.  Not
 *     capturable: stem_plan_create / _destroy / _set_detector_edges /
 *     _device_status (synchronous) and the *_streamed calls (they create a
 *     stream and events).
 */
#ifndef STEM_H_
#define STEM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  STEM_OK = 0,
  STEM_ERR_INVALID = -1,      /* bad argument or NULL pointer; nothing launched */
  STEM_ERR_NOMEM = -2,        /* workspace too small or plan allocation failed */
  STEM_ERR_CUDA = -3,         /* a CUDA runtime call or kernel launch failed */
  STEM_ERR_UNSUPPORTED = -4,  /* size outside the supported set (see stem_params) */
  STEM_ERR_TIMEOUT = -5       /* a bounded device-side wait gave up */
} stem_status;

/* Storage of the compact S-matrix.  F16 / BF16 store each beam divided by a
 * per-beam power-of-two scale s_b (its largest |Re| or |Im| rounded up to a
 * power of two); the beam sum multiplies the coefficient by s_b and accumulates
 * in FP32. */
typedef enum { STEM_F32 = 0, STEM_F16 = 1, STEM_BF16 = 2, STEM_CROPPED = 16 } stem_storage;
/* STEM_CROPPED, OR-ed into the element type, selects the Fourier-cropped
 * S-matrix ("Description of Algorithms": the PRISM output probe is a Fourier
 * interpolation of the plane waves).  Every exit wave is band-limited by the
 * 2/3 limit 9 (m^2 + n^2) <= N^2, so its spectrum fits on the grid of signed
 * frequencies |m|, |n| < N'/2 with N' = 3N/4, and the inverse transform there
 * samples the same wave at the N' x N' points (j Lx / N', i Ly / N'):
 *   S'_b(r') = (1 / N^2) sum_{k in band} Psi_hat_b(k) exp(2 pi i k . r').
 * The S-matrix is stored on that grid (9/16 of the bytes) and the output uses
 * windows of W' = N' / f = 3W/4 pixels over the same L / f, their W' x W'
 * transforms giving the same coarse frequencies (mu, nu) <-> (f mu, f nu).
 * It needs n >= 64.  Every call that takes a storage code accepts the flag;
 * an S-matrix must be read back with the code it was built with. */

/* Beam-sum engine for stem_prism_output. */
typedef enum {
  STEM_SUM_AUTO = 0,     /* tensor cores for F16/BF16 storage, CUDA cores for F32 */
  STEM_SUM_SIMT = 1,     /* FP32 CUDA-core tiled complex GEMM (any storage) */
  STEM_SUM_TENSOR = 2    /* tcgen05 complex GEMM, F16/BF16 storage only */
} stem_sum_engine;

/* Simulation parameters (Methods; Benchmarks give the values used there).
 *   n          grid side, nx == ny == n, a power of two in [8, 2048]
 *              (potentials, multislice and the S-matrix need n >= 64)
 *   cell       Lx, Ly, Lz in Angstrom
 *   n_slices   slices along the beam; atoms go to slice floor(z / slice_dz)
 *              clamped to [0, n_slices - 1]
 *   energy_kev beam energy; lambda and sigma are the relativistic values
 *   alpha_mrad probe convergence semi-angle (aperture: lambda |k| <= alpha)
 *   ring_width_mrad, n_rings  ring i collects lambda |k| in [i, i+1) * width,
 *              1 <= n_rings <= 2048, inside the 2/3 band limit 9 (m^2+n^2) <= N^2
 *   defocus_a, cs_a  probe aberrations C1 and Cs in Angstrom ("Description of
 *              Algorithms": the probe coefficients carry the coherent wave
 *              aberrations); the probe's Fourier coefficients and the PRISM
 *              coefficients are multiplied by exp(-i chi(k)),
 *              chi = pi lambda C1 |k|^2 + (pi/2) Cs lambda^3 |k|^4, so that a
 *              positive C1 equals free propagation by C1 under Eq. 2. */
typedef struct {
  double cell[3];
  int32_t n;
  int32_t n_slices;
  double slice_dz;
  double energy_kev;
  double alpha_mrad;
  double ring_width_mrad;
  int32_t n_rings;
  double defocus_a;
  double cs_a;
} stem_params;

/* Opaque plan: device-resident tables derived from stem_params (propagator
 * factors, ring/aperture look-up tables for every power-of-two f, PRISM beam
 * lists).  Library-owned. */
typedef struct stem_plan_s* stem_plan;

/* Build a plan (allocates its tables with cudaMalloc and fills them with
 * synchronous copies on the calling thread's current device).  Returns
 * STEM_ERR_UNSUPPORTED for n outside the set above, STEM_ERR_INVALID for
 * non-positive sizes, STEM_ERR_NOMEM if an allocation fails. */
stem_status stem_plan_create(const stem_params* params, stem_plan* out);
void stem_plan_destroy(stem_plan plan);

/* lambda (Angstrom) and sigma (rad / (V*A)) of Eq. 1 and Eq. 2, and the number
 * of aperture pixels |A| (host outputs; any may be NULL). */
stem_status stem_plan_constants(stem_plan plan, double* lambda_a, double* sigma,
                                int32_t* n_aperture);

/* Replace the uniform rings by annular detectors with arbitrary edges (host
 * array, mrad, strictly increasing, >= 0): detector i collects lambda |k| in
 * [edges[i], edges[i+1]) inside the band limit; n_rings becomes n_edges - 1
 * (<= 2048).  Covers 2D virtual detectors such as an ADF ring (two edges).
 * Rebuilds the plan's tables with synchronous copies. */
stem_status stem_plan_set_detector_edges(stem_plan plan, int32_t n_edges, const double* edges_mrad);

/* Device status word of the plan: kernels whose waits are bounded (the
 * tensor-core beam sum, the TMA-fed column passes, the row passes' bulk copy
 * of t_n) record STEM_ERR_TIMEOUT there instead of hanging.  Copies it to
 * *code (host) and clears it; synchronous (waits for the copy). */
stem_status stem_plan_device_status(stem_plan plan, int32_t* code);

/* Self-test of that bounded-wait path; the paper has no counterpart.  Launches
 * one thread that waits on a shared-memory barrier nothing arrives at, with
 * the wait routine the kernels above use but a limit of limit_ns (1 .. 1e9).
 * When the limit passes it records STEM_ERR_TIMEOUT in the plan's status word
 * and returns, leaving the context usable.  Asynchronous on `stream`;
 * STEM_ERR_INVALID for a null plan or a limit out of range. */
stem_status stem_selftest_bounded_wait(stem_plan plan, int64_t limit_ns, void* stream);

/* FP32 arithmetic rate probe; the paper has no counterpart.  It gives the
 * measured denominator of the FP32 roofline of the FFT passes.  Launches
 * `blocks` CTAs of 256 threads; each thread runs `iters` rounds of 8
 * independent FMA chains: scalar FMAs (packed = 0; one lane operation each)
 * or the packed f32x2 FMA (packed = 1; two lane operations each).  Lane
 * operations per launch = blocks * 256 * iters * 8 * (packed ? 2 : 1); the
 * caller times the launch on `stream`.  out: float32 [blocks * 256] device
 * buffer (written with one sum per thread).  STEM_ERR_INVALID for iters < 1,
 * blocks outside [1, 2^20] or a NULL out; asynchronous. */
stem_status stem_selftest_fma_rate(int32_t packed, int64_t iters, int32_t blocks, float* out, void* stream);

/* ---------------------------------------------------------------------------
 * Projected potentials (Methods, "Calculation of the Projected Potentials").
 * The paper's Kirkland look-up table is replaced by a sum of two isotropic
 * Gaussians per atom:  V_n(r) = sum_{atoms in slice n} sum_{periodic images}
 *   A1 exp(-d^2 / (2 s1^2)) + A2 exp(-d^2 / (2 s2^2)),
 * over the square support |dx|, |dy| <= 8 max(s1, s2).
 *   atoms_xyz  float64 [n_atoms][3]  (x, y, z) in Angstrom, any values
 *              (x, y are taken periodically)
 *   gauss      float32 [n_atoms][4]  (A1 [V*A], s1 [A], A2 [V*A], s2 [A]), s > 0
 *   v_out      float32 [n_slices][n][n] in V*A, or NULL
 *   trans_out  complex64 [n_slices][n][n]: t_n = exp(i sigma V_n) (Eq. 1), or NULL
 *   workspace  >= stem_slice_potentials_workspace(plan, n_atoms) bytes
 * Each pixel's sum runs in FP32 in an order fixed by the input (atoms by index
 * within each 32 x 32 pixel cell), so repeated calls give identical bits;
 * permuting the atoms may change the last bits.  Needs n >= 64
 * (STEM_ERR_UNSUPPORTED otherwise); asynchronous on `stream`.
 * ------------------------------------------------------------------------ */
size_t stem_slice_potentials_workspace(stem_plan plan, int64_t n_atoms);
stem_status stem_slice_potentials(stem_plan plan, const double* atoms_xyz, const float* gauss,
                                  int64_t n_atoms, float* v_out, void* trans_out,
                                  void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Multislice STEM (Eq. 1, Eq. 2; "Multislice Probe Simulations").
 * For each probe p at (x_p, y_p):
 *   psi_hat_p(k) = A(k) exp(-i chi(k)) exp(-2 pi i k . r_p) / sqrt(|A|);  psi = IFFT(psi_hat)
 *   for every slice n: psi <- IFFT( M P FFT(t_n psi) ),  P = exp(-i pi lambda dz |k|^2)
 *   (after the last slice the Fourier-space wave is kept)
 *   I_i(p) = sum_{k in ring i} |Psi_hat(k)|^2   (fraction of the incident intensity)
 *   trans      complex64 [n_slices][n][n] (from stem_slice_potentials or the caller)
 *   probe_xy   float64 [n_probes][2] (x, y) in Angstrom
 *   batch      probes propagated together (1 .. 65535)
 *   rings_out  float32 [n_probes][n_rings], += weight * I
 *   workspace  >= stem_multislice_workspace(plan, batch) bytes (the batch of waves)
 * ------------------------------------------------------------------------ */
size_t stem_multislice_workspace(stem_plan plan, int32_t batch);
stem_status stem_multislice_scan(stem_plan plan, const void* trans, const double* probe_xy,
                                 int64_t n_probes, int32_t batch, float weight, float* rings_out,
                                 void* workspace, size_t workspace_bytes, void* stream);

/* 4D output of multislice ("Description of Algorithms": the whole probe
 * diffraction pattern per probe position): dp_out float32 [n_probes][n][n] in
 * FFT order, dp_out += weight * |Psi_hat|^2 inside the 2/3 band limit (other
 * pixels are not written).  Otherwise as stem_multislice_scan. */
stem_status stem_multislice_scan_4d(stem_plan plan, const void* trans, const double* probe_xy,
                                    int64_t n_probes, int32_t batch, float weight, float* dp_out,
                                    void* workspace, size_t workspace_bytes, void* stream);

/* Multislice without a workspace argument, for callers that cannot allocate
 * device memory and have no scratch buffer to lend (for example a plugin whose
 * host application owns all device memory and passes it only its inputs and
 * outputs, or a loop whose memory budget is fixed at start-up).  There is no
 * counterpart in the paper.  Same arguments and results as
 * stem_multislice_scan, minus the workspace: the batch of waves lives in a
 * 32 MiB array inside the library's device image (held on every device that
 * loads the library until the process exits).  batch * n * n * 8 bytes must
 * fit in it, else STEM_ERR_NOMEM and nothing is launched.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current); make that first call before any stream capture.  Every call
 * shares the array: calls that overlap on the GPU (other streams, other host
 * threads) race and corrupt each other's waves; serialise them.  No call
 * allocates, and nothing in the array needs clearing between calls.  The
 * device current at the call must be the plan's device (the one current at
 * stem_plan_create), else STEM_ERR_INVALID and nothing is launched. */
stem_status stem_multislice_scan_noalloc(stem_plan plan, const void* trans, const double* probe_xy,
                                         int64_t n_probes, int32_t batch, float weight,
                                         float* rings_out, void* stream);

/* ---------------------------------------------------------------------------
 * Streaming memory model ("Streaming Data for Very Large Simulations"): the
 * transmission stack stays in HOST memory and only a few slices are on the
 * device at a time.
 *   trans_host  complex64 [n_slices][n][n] in host memory (page-locked memory,
 *               e.g. cudaHostAlloc, lets the copies overlap the passes;
 *               pageable memory works but the copies then stall the host).
 *               A device pointer is accepted too (the copies become
 *               device-to-device).  It must stay valid and unchanged until the
 *               work queued on `stream` has finished.
 *   workspace   >= stem_multislice_streamed_workspace(plan, batch) bytes: the
 *               batch of waves followed by 3 slice buffers of n*n*8 bytes.
 * Each slice is copied into the next free buffer by an asynchronous copy on a
 * stream the call creates (ordered after the work already queued on `stream`)
 * as soon as the row pass that read that buffer's previous slice has
 * finished; the row pass of a slice waits for its copy.  Every batch of
 * probes copies all n_slices slices again (the price of the smaller
 * footprint).  Results equal stem_multislice_scan's.  Calls that overlap on
 * the GPU must use different workspaces.
 * ------------------------------------------------------------------------ */
size_t stem_multislice_streamed_workspace(stem_plan plan, int32_t batch);
stem_status stem_multislice_scan_streamed(stem_plan plan, const void* trans_host, const double* probe_xy,
                                          int64_t n_probes, int32_t batch, float weight, float* rings_out,
                                          void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * PRISM compact S-matrix ("Description of Algorithms", PRISM paragraph;
 * "PRISM Probe Simulations").  Beams: every f-th Fourier component in x and y
 * inside the probe aperture, psi_b(r) = exp(2 pi i k_b . r), ordered by n then
 * m (ascending signed indices).  Each beam goes through every slice as in
 * multislice and its exit wave is kept in real space.
 *
 * S-matrix buffer layout (stem_prism_smatrix_bytes bytes, 256-byte aligned):
 *   float32 scale[nbp]              s_b (1 for F32 storage), nbp = n_beams rounded up to 64
 *   then at byte offset 256 * ceil(4 nbp / 256):
 *   elem data[n][n][2][nbp]          [y][x][re|im][beam], elem = float / half / bfloat16,
 *                                    stored value = S_b(x, y) / s_b; padded beams are 0.
 * ------------------------------------------------------------------------ */
stem_status stem_prism_beams(stem_plan plan, int32_t f, int32_t* n_beams, int32_t* mn_host);
size_t stem_prism_smatrix_bytes(stem_plan plan, int32_t f, stem_storage storage);
size_t stem_prism_smatrix_workspace(stem_plan plan, int32_t batch);
stem_status stem_prism_smatrix(stem_plan plan, const void* trans, int32_t f, stem_storage storage,
                               int32_t batch, void* smatrix, size_t smatrix_bytes,
                               void* workspace, size_t workspace_bytes, void* stream);

/* Beams [b_begin, b_end) only (0 <= b_begin <= b_end <= n_beams), for an
 * S-matrix whose beams are built on several devices ("PRISM Probe
 * Simulations": every plane wave is propagated independently).  Writes those
 * beams' values and scales, and the padding beams when b_end == n_beams;
 * nothing else in the buffer is touched.  With the buffer zeroed beforehand on
 * every device, summing the buffers of devices that built disjoint ranges
 * covering [0, n_beams) gives exactly the whole S-matrix (each sum adds only
 * zeros), which is how an all-reduce assembles it.  Otherwise as
 * stem_prism_smatrix; STEM_ERR_INVALID for a range outside [0, n_beams]. */
stem_status stem_prism_smatrix_range(stem_plan plan, const void* trans, int32_t f, stem_storage storage,
                                     int32_t batch, int32_t b_begin, int32_t b_end, void* smatrix,
                                     size_t smatrix_bytes, void* workspace, size_t workspace_bytes, void* stream);

/* The S-matrix built under the streaming memory model: trans_host as for
 * stem_multislice_scan_streamed (host stack, copied slice by slice into 3
 * device buffers; every batch of beams copies all slices); workspace >=
 * stem_prism_smatrix_streamed_workspace(plan, batch).  The S-matrix itself is
 * written to device memory as by stem_prism_smatrix, with identical bytes. */
size_t stem_prism_smatrix_streamed_workspace(stem_plan plan, int32_t batch);
stem_status stem_prism_smatrix_streamed(stem_plan plan, const void* trans_host, int32_t f,
                                        stem_storage storage, int32_t batch, void* smatrix,
                                        size_t smatrix_bytes, void* workspace, size_t workspace_bytes,
                                        void* stream);

/* ---------------------------------------------------------------------------
 * PRISM output ("Description of Algorithms", PRISM paragraph; "PRISM Probe
 * Simulations", last paragraph).  W = n / f.  For each probe:
 *   origin o_p = (floor(x_p/dx + 0.5), floor(y_p/dy + 0.5)) - W/2  (mod n)
 *   c_{p,b}   = exp(-i chi(k_b)) exp(-2 pi i (m_b x_p / Lx + n_b y_p / Ly)) / sqrt(n_beams)
 *               (phase reduced in FP64 on the device)
 *   Psi_p(u, v) = sum_b c_{p,b} S_b((o_p + (u, v)) mod n),  u, v in [0, W)
 *   I_i(p) = sum_{coarse k in ring i} |FFT_W(Psi_p)|^2 / W^4,
 *   the coarse frequency (mu, nu) being the fine frequency (f mu, f nu).
 *   smatrix    a buffer filled by stem_prism_smatrix with the same f and storage
 *   chunk      probes handled per internal step (1 .. 65535; bounds the workspace)
 *   engine     stem_sum_engine
 *   workspace  >= stem_prism_output_workspace(plan, f, chunk) bytes
 * ------------------------------------------------------------------------ */
size_t stem_prism_output_workspace(stem_plan plan, int32_t f, int32_t chunk);
stem_status stem_prism_output(stem_plan plan, int32_t f, stem_storage storage, int32_t engine,
                              const void* smatrix, const double* probe_xy, int64_t n_probes,
                              int32_t chunk, float weight, float* rings_out,
                              void* workspace, size_t workspace_bytes, void* stream);

/* 4D output of PRISM: dp_out float32 [n_probes][W][W] in FFT order on the
 * window's coarse grid, dp_out += weight * |FFT_W(Psi_p)|^2 / W^4 inside the
 * band limit (9 (mu^2 + nu^2) <= W^2).  Otherwise as stem_prism_output. */
stem_status stem_prism_output_4d(stem_plan plan, int32_t f, stem_storage storage, int32_t engine,
                                 const void* smatrix, const double* probe_xy, int64_t n_probes,
                                 int32_t chunk, float weight, float* dp_out,
                                 void* workspace, size_t workspace_bytes, void* stream);

/* Stage of stem_prism_output exposed for stage-wise checks: the window waves
 * Psi_p (before the FFT) of n_probes probes (<= 65535), complex64
 * [n_probes][W][W]; workspace >= stem_prism_output_workspace(plan, f, n_probes). */
stem_status stem_prism_windows(stem_plan plan, int32_t f, stem_storage storage, int32_t engine,
                               const void* smatrix, const double* probe_xy, int64_t n_probes,
                               void* windows_out, void* workspace, size_t workspace_bytes,
                               void* stream);

/* ---------------------------------------------------------------------------
 * Detector readout (Methods, "Description of Algorithms": annular ring virtual
 * detectors).  psi_k complex64 [batch][W][W] in FFT order with W = n / f, the
 * coarse frequency (mu, nu) standing for (f mu, f nu); batch <= 65535:
 *   rings_out[b][i] += scale * sum_{k in ring i} |psi_k[b](k)|^2
 * ------------------------------------------------------------------------ */
stem_status stem_detector_readout(stem_plan plan, int32_t f, const void* psi_k, int64_t batch,
                                  float scale, float* rings_out, void* stream);

/* ---------------------------------------------------------------------------
 * Batched 2D FFT with the path's FFT kernels (the transform used by Eq. 2 and
 * the detector).  data complex64 [batch][n][n], in place; n a power of two in
 * [8, 2048]; batch <= 65535.  inverse = 0: forward e^{-}, unnormalised;
 * inverse = 1: e^{+}, unnormalised (divide by n^2 for the inverse DFT).
 * ------------------------------------------------------------------------ */
stem_status stem_fft2(int32_t n, int64_t batch, int32_t inverse, void* data, void* stream);

/* ---------------------------------------------------------------------------
 * Device bytes a request needs (admission control for serving; the paper's
 * memory estimate of "Streaming Data for Very Large Simulations").
 *   algo 0 = multislice (transmission stack + one batch of waves + rings),
 *   algo 1 = PRISM (transmission stack + S-matrix + S-matrix workspace +
 *            output workspace for chunks of up to 4096 probes + rings),
 *   algo 2 = multislice, streamed (3 slice buffers instead of the stack),
 *   algo 3 = PRISM with the S-matrix built streamed (3 slice buffers instead
 *            of the stack; the S-matrix itself stays resident)
 * ------------------------------------------------------------------------ */
size_t stem_footprint_bytes(const stem_params* params, int32_t algo, int32_t f,
                            stem_storage storage, int64_t n_probes, int32_t batch);

/* Number of CUDA kernels this library has launched in this process (all
 * devices, all streams); for launch accounting in benchmarks. */
uint64_t stem_launch_count(void);

/* ---------------------------------------------------------------------------
 * Kernel timing, for measuring a hot kernel's own launch duration inside a
 * running workload (the roofline of one kernel rather than of a whole phase).
 * While enabled, the library brackets every launch of the kernel families
 * below with two CUDA events recorded on the launch's stream (two event
 * records per launch, nothing else changes); stem_profile_read waits for the
 * family's last launch and returns the number of launches recorded since
 * stem_profile_enable(1) and their summed device time in milliseconds.
 *   STEM_PROF_ROW_SLICE   slice-loop row pass (Eq. 1 and the row transforms)
 *   STEM_PROF_COL_SLICE   slice-loop column pass (Eq. 2 and the column transforms)
 *   STEM_PROF_BEAM_SUM    PRISM beam sum (tcgen05 or CUDA-core engine)
 *   STEM_PROF_POTENTIALS  projected potentials (the per-tile sum)
 * stem_profile_enable(1) starts recording and clears earlier records,
 * stem_profile_enable(0) stops it.  Process-wide, thread-safe; the events
 * belong to the device current at each launch.  Errors: STEM_ERR_INVALID for
 * an unknown family or NULL outputs, STEM_ERR_CUDA if an event call failed.
 * ------------------------------------------------------------------------ */
typedef enum {
  STEM_PROF_ROW_SLICE = 0,
  STEM_PROF_COL_SLICE = 1,
  STEM_PROF_BEAM_SUM = 2,
  STEM_PROF_POTENTIALS = 3,
  STEM_PROF_KINDS = 4
} stem_prof_kind;
stem_status stem_profile_enable(int32_t on);
stem_status stem_profile_read(int32_t kind, int64_t* launches, double* total_ms);

const char* stem_status_string(stem_status status);

#ifdef __cplusplus
}
#endif

#endif /* STEM_H_ */
