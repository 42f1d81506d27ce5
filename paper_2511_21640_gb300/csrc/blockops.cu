// FP64 block kernels of the Davidson solver for "tall-skinny" operands: a
// handful of long vectors (length N, up to 10^8) against a subspace of at most
// a few hundred. A general GEMM tile (64 x 64) would waste most of its FP64
// throughput on such shapes; these kernels keep every loaded vector element
// busy for all the short indices it meets.
#include "blockops.cuh"

namespace adc {

namespace {

constexpr int GA = 64;   // rows of A per CTA (gram)
constexpr int GB = 16;   // rows of B per CTA (gram)
constexpr int GK = 32;   // K staged per step (gram)

// part[chunk][a][b] = sum_{k in chunk} conj(A[a][k]) B[b][k]
__global__ void __launch_bounds__(256)
k_gram(const cplx *__restrict__ A, int64_t lda, int na, const cplx *__restrict__ B, int64_t ldb, int nb,
       int64_t n, int64_t chunk, cplx *part) {
  __shared__ cplx As[GK][GA + 1];
  __shared__ cplx Bs[GK][GB + 1];
  const int t = threadIdx.x;
  const int al = t & 63, bg = t >> 6;
  const int a0 = blockIdx.y * GA, b0 = blockIdx.z * GB;
  const int64_t k_beg = (int64_t)blockIdx.x * chunk;
  const int64_t k_end = min(n, k_beg + chunk);
  cplx acc[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) acc[j] = cmake(0.0, 0.0);
  for (int64_t k0 = k_beg; k0 < k_end; k0 += GK) {
#pragma unroll
    for (int s = 0; s < (GA * GK) / 256; ++s) {
      const int e = t + 256 * s;
      const int ai = e / GK, kk = e % GK;
      const int64_t k = k0 + kk;
      cplx v = cmake(0.0, 0.0);
      if (a0 + ai < na && k < k_end) v = A[(int64_t)(a0 + ai) * lda + k];
      As[kk][ai] = v;
    }
#pragma unroll
    for (int s = 0; s < (GB * GK) / 256; ++s) {
      const int e = t + 256 * s;
      const int bi = e / GK, kk = e % GK;
      const int64_t k = k0 + kk;
      cplx v = cmake(0.0, 0.0);
      if (b0 + bi < nb && k < k_end) v = B[(int64_t)(b0 + bi) * ldb + k];
      Bs[kk][bi] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GK; ++kk) {
      const cplx a = cconj(As[kk][al]);
#pragma unroll
      for (int j = 0; j < 4; ++j) cfma(acc[j], a, Bs[kk][bg * 4 + j]);
    }
    __syncthreads();
  }
  const int a = a0 + al;
  if (a < na) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = b0 + bg * 4 + j;
      if (b < nb) part[((int64_t)blockIdx.x * na + a) * nb + b] = acc[j];
    }
  }
}

__global__ void k_gram_reduce(const cplx *__restrict__ part, int nchunk, int na, int nb, cplx alpha, cplx *G,
                              int64_t ldg) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= na * nb) return;
  cplx s = cmake(0.0, 0.0);
  for (int c = 0; c < nchunk; ++c) s = cadd(s, part[(int64_t)c * na * nb + idx]);
  G[(int64_t)(idx / nb) * ldg + idx % nb] = cmul(alpha, s);
}

constexpr int CR_ROWS = 16;  // output rows per CTA (combine)
constexpr int CI = 64;       // subspace rows staged per step (combine)

// Y[r][k] = alpha sum_i C[i][r] V[i][k] + beta Y[r][k], r in this CTA's group of 16
__global__ void __launch_bounds__(256)
k_combine(const cplx *__restrict__ C, int64_t ldc, int m, int nr, const cplx *__restrict__ V, int64_t ldv,
          int64_t n, cplx alpha, cplx beta, cplx *Y, int64_t ldy) {
  __shared__ cplx Cs[CI][CR_ROWS];
  const int r0 = blockIdx.y * CR_ROWS;
  const int rn = min(CR_ROWS, nr - r0);
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  cplx acc[CR_ROWS];
#pragma unroll
  for (int r = 0; r < CR_ROWS; ++r) acc[r] = cmake(0.0, 0.0);
  for (int i0 = 0; i0 < m; i0 += CI) {
    const int ni = min(CI, m - i0);
    for (int e = threadIdx.x; e < CI * CR_ROWS; e += blockDim.x) {
      const int i = e / CR_ROWS, r = e % CR_ROWS;
      Cs[i][r] = (i < ni && r < rn) ? C[(int64_t)(i0 + i) * ldc + r0 + r] : cmake(0.0, 0.0);
    }
    __syncthreads();
    if (k < n) {
      for (int i = 0; i < ni; ++i) {
        const cplx v = V[(int64_t)(i0 + i) * ldv + k];
#pragma unroll
        for (int r = 0; r < CR_ROWS; ++r) cfma(acc[r], Cs[i][r], v);
      }
    }
    __syncthreads();
  }
  if (k >= n) return;
  const bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
#pragma unroll
  for (int r = 0; r < CR_ROWS; ++r) {
    if (r < rn) {
      cplx *dst = Y + (int64_t)(r0 + r) * ldy + k;
      cplx val = cmul(alpha, acc[r]);
      if (use_beta) val = cadd(val, cmul(beta, *dst));
      *dst = val;
    }
  }
}

int g_sms_blockops = 0;

}  // namespace

void gram(Exec &ex, const cplx *A, int64_t lda, int na, const cplx *B, int64_t ldb, int nb, int64_t n, cplx alpha,
          cplx *G, int64_t ldg) {
  if (na <= 0 || nb <= 0) return;
  if (!g_sms_blockops) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms_blockops, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms_blockops <= 0) g_sms_blockops = 148;
  }
  const int gy = (na + GA - 1) / GA, gz = (nb + GB - 1) / GB;
  int64_t nchunk = std::max<int64_t>(1, (4 * (int64_t)g_sms_blockops) / (gy * gz));
  nchunk = std::min<int64_t>(nchunk, std::max<int64_t>(1, n / (4 * GK)));
  int64_t chunk = (n + nchunk - 1) / nchunk;
  chunk = (chunk + GK - 1) / GK * GK;
  nchunk = std::max<int64_t>(1, (n + chunk - 1) / chunk);
  ADC_REQUIRE(nchunk < (1ll << 31) && gy <= 65535 && gz <= 65535, ADC_ERR_UNSUPPORTED, "gram: shape");
  DBuf part = cbuf(ex, nchunk * (int64_t)na * nb);
  int pr = ex.prof_begin("gram_fp64", 8.0 * (double)na * nb * (double)n);
  k_gram<<<dim3((unsigned)nchunk, gy, gz), 256, 0, ex.stream>>>(A, lda, na, B, ldb, nb, n, chunk, part.c());
  ADC_CHECK_LAUNCH();
  k_gram_reduce<<<(na * nb + 255) / 256, 256, 0, ex.stream>>>(part.c(), (int)nchunk, na, nb, alpha, G, ldg);
  ADC_CHECK_LAUNCH();
  ex.prof_end(pr);
}

void combine(Exec &ex, const cplx *C, int64_t ldc, int m, int nr, const cplx *V, int64_t ldv, int64_t n,
             cplx alpha, cplx beta, cplx *Y, int64_t ldy) {
  if (nr <= 0 || n <= 0) return;
  const int64_t gx = (n + 255) / 256;
  const int gy = (nr + CR_ROWS - 1) / CR_ROWS;
  ADC_REQUIRE(gx < (1ll << 31) && gy <= 65535, ADC_ERR_UNSUPPORTED, "combine: shape");
  int pr = ex.prof_begin("combine_fp64", 8.0 * (double)nr * m * (double)n);
  k_combine<<<dim3((unsigned)gx, gy), 256, 0, ex.stream>>>(C, ldc, m, nr, V, ldv, n, alpha, beta, Y, ldy);
  ADC_CHECK_LAUNCH();
  ex.prof_end(pr);
}

}  // namespace adc
