/*
 * adc_gb300_diag.h -- diagnostics of the GB300 ADC library's contraction
 * kernels (no counterpart in arXiv:2511.21640; used by the tests and the
 * benchmark to check and time the building blocks in isolation).
 */
#ifndef ADC_GB300_DIAG_H
#define ADC_GB300_DIAG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* the context type of adc_gb300.h */
typedef struct adc_ctx adc_ctx_opaque;

/* Random complex A [M][K] and B [N][K] (seeded, uniform in [-1,1) per
 * component) are multiplied as C = A B^T by the kernel `which`
 * (0 = FP64 CUDA-core GEMM, 1 = BF16x3 tensor-core GEMM, 2 = the same product
 * as one job of the grouped persistent tensor-core launch with an autotuned
 * tile width, 3 = three jobs of different shapes in one grouped launch:
 * (M, N, K), (M/2+37, max(1, N/3), K/2+11) and (129, 3, 2K+5), the last one
 * long and narrow so that it is split along K; rel_err is then the largest of
 * the three), 4 = the six-product (BF16x6) tensor-core GEMM, 5 = the sliced
 * FP64-accurate tensor-core product of ADC_PREC_SLICED, including the slicing
 * of both operands, 6 = the setup's route: zgemm as the sliced product with
 * about 48 bits, in operand chunks (adc_diag_set_sliced_cap)) and compared with
 * the FP64 GEMM. Outputs: rel_err = ||C - C_fp64||_F / ||C_fp64||_F,
 * ms = average time of one launch sequence over `reps` repetitions (CUDA
 * events, after one warm-up). Allocates and frees its own device memory.
 * Returns ADC_OK or a negative ADC_ERR_* code. */
int adc_diag_gemm(int which, int64_t M, int64_t N, int64_t K, uint64_t seed, int reps,
                  double *rel_err, double *ms);

/* Per-kernel timing of one context. adc_profile_enable(ctx, 1) clears the
 * record and starts recording a CUDA event pair around every GEMM launch on
 * the context's stream (0 stops). adc_profile_read() synchronises the stream
 * and returns one entry per kernel and sigma term ("tc_gemm_bf16x3/ladder",
 * "zgemm_fp64/ring", ...): launches, total device milliseconds, the
 * algorithmic flops of those launches (8 per complex multiply-add, no
 * padding) and their algorithmic device-memory bytes (operands read once,
 * results written once; 0 where not recorded). *n receives the number of
 * entries (at most max). */
typedef struct {
  char name[48];
  int64_t launches;
  double total_ms;
  double flops;
  double bytes;
} adc_kernel_stat;

int adc_profile_enable(adc_ctx_opaque *ctx, int on);
int adc_profile_read(adc_ctx_opaque *ctx, adc_kernel_stat *out, int max, int *n);

/* Device memory of one context: the bytes its allocations hold now and the
 * largest amount they held at once since adc_init (the context's own buffers,
 * not the CUDA runtime's). Host-side counters only, no device work.
 * ADC_ERR_STATE for a NULL context, ADC_ERR_ARG for NULL outputs. */
int adc_memory(const adc_ctx_opaque *ctx, int64_t *in_use, int64_t *peak);

/* Test hook for the failure path of the tensor-core kernels: sets the limit
 * (nanoseconds of %globaltimer) of their pipeline waits on the current device,
 * 0 = the default of 2 s. With a limit far below a kernel's run time a wait
 * gives up: the kernel records the error, waits (with its own fixed 2 s
 * limit) for the copies and MMAs it has in flight, frees its tensor memory
 * and returns, and the call that launched it returns ADC_ERR_TIMEOUT. Affects
 * every context of the process on that device until it is set again. */
int adc_diag_set_wait_ns(uint64_t ns);

/* Test hook: the size (complex elements) of one chunk of the setup's chunked
 * intermediates (the IP third-order coupling's (ea|fk) block, formed in chunks
 * of its first virtual index); <= 0 restores the default of 2^28. Process-wide,
 * host only; affects contexts initialised afterwards. Returns ADC_OK. */
int adc_diag_set_setup_chunk(int64_t elems);

/* Test hook: bytes of one operand chunk of the sliced product behind the
 * setup's large contractions (the digit planes of A row blocks and B column
 * blocks; when one 128-row tile would exceed it, the inner index is split and
 * the FP64-accurate partial products add up). <= 0 restores the rule of an
 * eighth of the free memory (1 to 16 GiB). Process-wide. Returns ADC_OK. */
int adc_diag_set_sliced_cap(int64_t bytes);

/* 1 when the context forms its EA ladder integrals inside every product
 * (opts.ladder), else 0. ADC_ERR_STATE for a NULL context. */
int adc_ladder_mode(const adc_ctx_opaque *ctx, int *direct);

/* Routes of the complex products adc_init issued for this context: how many
 * ran as the sliced tensor-core product (opts.setup = ADC_PREC_SLICED, inner
 * size at least 512 and at least 2^24 flops) and how many on the FP64 CUDA
 * cores, with their algorithmic flops (8 per complex multiply-add). Host-side
 * counters only. ADC_ERR_STATE for a NULL context, ADC_ERR_ARG for NULL
 * outputs. */
int adc_setup_routes(const adc_ctx_opaque *ctx, int64_t *n_sliced, int64_t *n_fp64, double *flops_sliced,
                     double *flops_fp64);

/* Davidson block kernels alone (blockops.cu), against the FP64 GEMM:
 *   which 0: gram, G[m][nb] = sum_k conj(A[m][k]) B[nb][k] for A [m][n],
 *            B [nb][n] (the subspace projections V^H T);
 *   which 1: combine, Y[nb][n] = sum_i C[i][r] V[i][n] for C [m][nb],
 *            V [m][n] (Ritz vectors and Gram-Schmidt updates).
 * Operands are seeded uniform random complex numbers. rel_err =
 * ||out - out_zgemm||_F / ||out_zgemm||_F, ms = average time of one call over
 * `reps` repetitions (CUDA events, after one warm-up). Allocates and frees
 * its own device memory. */
int adc_diag_blockops(int which, int64_t m, int64_t nb, int64_t n, uint64_t seed, int reps,
                      double *rel_err, double *ms);

/* The small Hermitian eigensolvers of the Davidson's Rayleigh-Ritz step on a
 * host matrix A [n][n] (row-major, Hermitian): which 0 = FP64 cyclic Jacobi,
 * 1 = FP32 Jacobi start refined in FP64 (n <= 128, else
 * ADC_ERR_UNSUPPORTED). Eigenvalues ascending into w [n], eigenvectors as the
 * columns of V [n][n] (host). ms = CUDA-event time of one solve after a
 * warm-up (NULL allowed); *steps (NULL allowed) = refinement steps taken, -1
 * when the refinement handed the matrix to the FP64 Jacobi, 0 for which 0.
 * Allocates and frees its own device memory. */
int adc_diag_eigh(int which, const adc_c128 *A, int n, double *w, adc_c128 *V, double *ms, int *steps);

/* FP64 FMA throughput of the device: every thread of a grid of `blocks`
 * blocks of 256 threads runs 16 independent fused multiply-add chains of
 * `iters` steps each (2 flops per FMA). tflops = flops / CUDA-event time. A
 * plain probe for the FP64 roofline; changes no device setting. */
int adc_diag_fp64_peak(int blocks, int64_t iters, double *tflops, double *ms);

/* Number of CUDA kernels this library has launched in the process so far. */
int64_t adc_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif
