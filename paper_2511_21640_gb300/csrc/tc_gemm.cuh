// Split-precision (BF16x3) complex GEMM on tcgen05; see tc_gemm.cu.
#pragma once
#include "tensor.cuh"

struct adc_ctx;

namespace adc {

// An operand in the real embedding, split into BF16 hi and lo planes of shape
// [rows][2*kp] (kp = K rounded up to 64). For A, rows = M; for B, rows = 2N.
struct TcMat {
  DBuf hi, lo;
  int64_t rows = 0, kp = 0, kreal = 0;
};

// A[m][k] = op(src[m*s_m + k*s_k]) (op = conj when conj is set)
void tc_pack_A(Exec &ex, TcMat &dst, const cplx *src, int64_t M, int64_t K, int64_t s_m, int64_t s_k, bool conj);
// B[n][k] = op(src[(n / n_in)*s_nh + (n % n_in)*s_nl + k*s_k]), Nc complex rows
void tc_pack_B(Exec &ex, TcMat &dst, const cplx *src, int64_t Nc, int64_t K, int64_t s_nh, int64_t s_nl,
               int64_t n_in, int64_t s_k, bool conj);
// B operand of the ring term, gathered from the packed satellite block of X
void tc_pack_B_ring(Exec &ex, TcMat &dst, const adc_ctx *c, const cplx *X, int64_t k);
// out[m][n] (n = nh*n_in + nl at m*s_m + nh*s_nh + nl*s_nl) = alpha * A B^T + beta * out
void tc_gemm(Exec &ex, const TcMat &A, const TcMat &B, int64_t M, int64_t N, cplx alpha, cplx beta, cplx *out,
             int64_t s_m, int64_t s_nh, int64_t s_nl, int64_t n_in, int *err);

struct TcCache {
  TcMat Glad, W, Cpl, CplT;  // static operators (A side)
  TcMat Bx;                  // per-call B operand
  DBuf err;                  // device error word of the tensor-core kernels
  bool ready = false;
};

}  // namespace adc
