// FP64 tall-skinny block kernels of the Davidson solver (see blockops.cu).
#pragma once
#include "tensor.cuh"

namespace adc {
// G[a][b] = alpha * sum_k conj(A[a][k]) B[b][k], a < na, b < nb, k < n
void gram(Exec &ex, const cplx *A, int64_t lda, int na, const cplx *B, int64_t ldb, int nb, int64_t n, cplx alpha,
          cplx *G, int64_t ldg);
// Y[r][k] = alpha * sum_i C[i][r] V[i][k] + beta * Y[r][k], r < nr, i < m, k < n
void combine(Exec &ex, const cplx *C, int64_t ldc, int m, int nr, const cplx *V, int64_t ldv, int64_t n,
             cplx alpha, cplx beta, cplx *Y, int64_t ldy);
}  // namespace adc
