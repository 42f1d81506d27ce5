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

/* Random complex A [M][K] and B [N][K] (seeded, uniform in [-1,1) per
 * component) are multiplied as C = A B^T by the kernel `which`
 * (0 = FP64 CUDA-core GEMM, 1 = BF16x3 tensor-core GEMM) and compared with
 * the FP64 GEMM. Outputs: rel_err = ||C - C_fp64||_F / ||C_fp64||_F,
 * ms = average time of one launch sequence over `reps` repetitions (CUDA
 * events, after one warm-up). Allocates and frees its own device memory.
 * Returns ADC_OK or a negative ADC_ERR_* code. */
int adc_diag_gemm(int which, int64_t M, int64_t N, int64_t K, uint64_t seed, int reps,
                  double *rel_err, double *ms);

#ifdef __cplusplus
}
#endif

#endif
