// FP64-accurate complex GEMM from integer BF16 slices on the tensor cores; see tc_slice.cu.
#pragma once

#include <vector>

#include "tc_gemm.cuh"

namespace adc {

// slicing of an inner size K: padded kp, digit width b (4..7 bits), slices ns
// for about `bits` significant bits, k-blocks of 64 per exact FP32 split
struct SlParams {
  int64_t kp = 0;
  int b = 0, ns = 0, kb_split = 0;
};
SlParams sl_params(int64_t K, int bits);

// An operand as ns BF16 planes of integer digits, [rows][2*kp] each, and one
// power-of-two exponent per row (A: per row; B: per complex row, shared by its
// two embedded rows).
struct SlMat {
  DBuf planes, exps;
  std::vector<TcMat> s;  // views of the planes (one hi plane each)
  int ns = 0, bits = 0, kb_split = 0;
  int64_t rows = 0, kp = 0, kreal = 0;
};

// scratch of sl_gemm: raw FP32 products of the slice pairs and the grouped launch state
struct SlWork {
  DBuf part;
  TcGroup grp;
};

// sliced copies of a context's static operators (built on first use) and the per-call B operand
struct SlCache {
  int bits = 0;
  SlMat Glad, W, Cpl, CplT, Bx;
  SlWork w;
  DBuf err;
  bool ready = false;
};

// A[m][k] = op(src[m*s_m + k*s_k]); digits for about `bits` significant bits
void sl_pack_A(Exec &ex, SlMat &dst, const cplx *src, int64_t M, int64_t K, int64_t s_m, int64_t s_k, bool conj,
               int bits);
// B[n][k] = op(src[(n / n_in)*s_nh + (n % n_in)*s_nl + k*s_k]), sliced like the A operand `like`
// bits > 0: only the leading digits for about that many significant bits (the
// product then uses the same leading slices of A)
void sl_pack_B(Exec &ex, SlMat &dst, const cplx *src, int64_t Nc, int64_t K, int64_t s_nh, int64_t s_nl,
               int64_t n_in, int64_t s_k, bool conj, const SlMat &like, int bits = 0);
// B operand of the ring term, gathered from the packed satellite block of X
void sl_pack_B_ring(Exec &ex, SlMat &dst, const adc_ctx *c, const cplx *X, int64_t k, const SlMat &like,
                    int bits = 0);
// zgemm's contract (tensor.cuh) computed as the sliced product with ex.sliced_bits bits
void zgemm_sliced(Exec &ex, int64_t M, int64_t N, int64_t K, int64_t batch, cplx alpha, const cplx *A, int64_t sAb,
                  int64_t sAm, int64_t sAk, bool conjA, const cplx *B, int64_t sBb, int64_t sBk, int64_t sBn,
                  bool conjB, cplx beta, cplx *C, int64_t sCb, int64_t sCm, int64_t sCn);
// out = alpha A B^T + beta out, addressing as tc_gemm
void sl_gemm(Exec &ex, const SlMat &A, const SlMat &B, int64_t M, int64_t N, cplx alpha, cplx beta, cplx *out,
             int64_t s_m, int64_t s_nh, int64_t s_nl, int64_t n_in, int *err, SlWork &w);

// test hook: bytes per operand chunk of zgemm_sliced (0 restores the free-memory rule)
void set_sliced_cap_bytes(size_t bytes);

}  // namespace adc
