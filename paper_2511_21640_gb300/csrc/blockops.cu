// FP64 block kernels of the Davidson solver for "tall-skinny" operands: a
// handful of long vectors (length N, up to 10^8) against a subspace of at most
// a few hundred. A general GEMM tile (64 x 64) would waste most of its FP64
// throughput on such shapes; these kernels keep every loaded vector element
// busy for all the short indices it meets.
#include "blockops.cuh"

namespace adc {

namespace {

constexpr int GK = 16;   // K staged per step (gram)

// part[chunk][a][b] = sum_{k in chunk} conj(A[a][k]) B[b][k], GA rows of A
// (64, or 32 for short subspaces) and GB rows of B per CTA. Three FP64
// products per complex product (3M): with a' = conj(a), T1 = a'r br,
// T2 = a'i bi, T3 = (a'r + a'i)(br + bi); the sums are formed once per staged
// element.
template <int GA, int GB>
__global__ void __launch_bounds__(256)
k_gram(const cplx *__restrict__ A, int64_t lda, int na, const cplx *__restrict__ B, int64_t ldb, int nb,
       int64_t n, int64_t chunk, cplx *part) {
  constexpr int NG = 256 / GA;  // groups of threads sharing a row of A
  constexpr int PB = GB / NG;   // b rows per thread
  __shared__ double Ar[GK][GA + 1], Ai[GK][GA + 1], As[GK][GA + 1];
  __shared__ double Br[GK][GB + 1], Bi[GK][GB + 1], Bs[GK][GB + 1];
  const int t = threadIdx.x;
  const int al = t % GA, bg = t / GA;
  const int a0 = blockIdx.y * GA, b0 = blockIdx.z * GB;
  const int64_t k_beg = (int64_t)blockIdx.x * chunk;
  const int64_t k_end = min(n, k_beg + chunk);
  double t1[PB], t2[PB], t3[PB];
#pragma unroll
  for (int j = 0; j < PB; ++j) t1[j] = t2[j] = t3[j] = 0.0;
  for (int64_t k0 = k_beg; k0 < k_end; k0 += GK) {
#pragma unroll
    for (int s = 0; s < (GA * GK) / 256; ++s) {
      const int e = t + 256 * s;
      const int ai = e / GK, kk = e % GK;
      const int64_t k = k0 + kk;
      cplx v = cmake(0.0, 0.0);
      if (a0 + ai < na && k < k_end) v = A[(int64_t)(a0 + ai) * lda + k];
      Ar[kk][ai] = v.x;
      Ai[kk][ai] = -v.y;
      As[kk][ai] = v.x - v.y;
    }
    for (int e = t; e < GB * GK; e += 256) {
      const int bi = e / GK, kk = e % GK;
      const int64_t k = k0 + kk;
      cplx v = cmake(0.0, 0.0);
      if (b0 + bi < nb && k < k_end) v = B[(int64_t)(b0 + bi) * ldb + k];
      Br[kk][bi] = v.x;
      Bi[kk][bi] = v.y;
      Bs[kk][bi] = v.x + v.y;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GK; ++kk) {
      const double ar = Ar[kk][al], ai = Ai[kk][al], as = As[kk][al];
#pragma unroll
      for (int j = 0; j < PB; ++j) {
        const int bj = bg * PB + j;
        t1[j] = fma(ar, Br[kk][bj], t1[j]);
        t2[j] = fma(ai, Bi[kk][bj], t2[j]);
        t3[j] = fma(as, Bs[kk][bj], t3[j]);
      }
    }
    __syncthreads();
  }
  const int a = a0 + al;
  if (a < na) {
#pragma unroll
    for (int j = 0; j < PB; ++j) {
      const int b = b0 + bg * PB + j;
      if (b < nb) part[((int64_t)blockIdx.x * na + a) * nb + b] = cmake(t1[j] - t2[j], t3[j] - t1[j] - t2[j]);
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

constexpr int CI = 64;  // subspace rows staged per step (combine)

// Y[r][k] = alpha sum_i C[i][r] V[i][k] + beta Y[r][k], r in this CTA's group
// of RR rows; 3M products as in k_gram
template <int RR>
__global__ void __launch_bounds__(256)
k_combine(const cplx *__restrict__ C, int64_t ldc, int m, int nr, const cplx *__restrict__ V, int64_t ldv,
          int64_t n, cplx alpha, cplx beta, cplx *Y, int64_t ldy) {
  __shared__ double Cr[CI][RR], Cim[CI][RR], Cs[CI][RR];
  const int r0 = blockIdx.y * RR;
  const int rn = min(RR, nr - r0);
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double t1[RR], t2[RR], t3[RR];
#pragma unroll
  for (int r = 0; r < RR; ++r) t1[r] = t2[r] = t3[r] = 0.0;
  for (int i0 = 0; i0 < m; i0 += CI) {
    const int ni = min(CI, m - i0);
    for (int e = threadIdx.x; e < CI * RR; e += blockDim.x) {
      const int i = e / RR, r = e % RR;
      const cplx cv = (i < ni && r < rn) ? C[(int64_t)(i0 + i) * ldc + r0 + r] : cmake(0.0, 0.0);
      Cr[i][r] = cv.x;
      Cim[i][r] = cv.y;
      Cs[i][r] = cv.x + cv.y;
    }
    __syncthreads();
    if (k < n) {
      for (int i = 0; i < ni; ++i) {
        const cplx v = V[(int64_t)(i0 + i) * ldv + k];
        const double vs = v.x + v.y;
#pragma unroll
        for (int r = 0; r < RR; ++r) {
          t1[r] = fma(Cr[i][r], v.x, t1[r]);
          t2[r] = fma(Cim[i][r], v.y, t2[r]);
          t3[r] = fma(Cs[i][r], vs, t3[r]);
        }
      }
    }
    __syncthreads();
  }
  if (k >= n) return;
  const bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
#pragma unroll
  for (int r = 0; r < RR; ++r) {
    if (r < rn) {
      cplx *dst = Y + (int64_t)(r0 + r) * ldy + k;
      cplx val = cmul(alpha, cmake(t1[r] - t2[r], t3[r] - t1[r] - t2[r]));
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
  const int GB = nb <= 8 ? 8 : 16;
  const int GA = na <= 32 ? 32 : 64;
  const int gy = (na + GA - 1) / GA, gz = (nb + GB - 1) / GB;
  int64_t nchunk = std::max<int64_t>(1, (4 * (int64_t)g_sms_blockops) / (gy * gz));
  nchunk = std::min<int64_t>(nchunk, std::max<int64_t>(1, n / (4 * GK)));
  int64_t chunk = (n + nchunk - 1) / nchunk;
  chunk = (chunk + GK - 1) / GK * GK;
  nchunk = std::max<int64_t>(1, (n + chunk - 1) / chunk);
  ADC_REQUIRE(nchunk < (1ll << 31) && gy <= 65535 && gz <= 65535, ADC_ERR_UNSUPPORTED, "gram: shape");
  DBuf part = cbuf(ex, nchunk * (int64_t)na * nb);
  int pr = ex.prof_begin("gram_fp64", 8.0 * (double)na * nb * (double)n);
  const dim3 grid((unsigned)nchunk, gy, gz);
  if (GA == 32 && GB == 8)
    k_gram<32, 8><<<grid, 256, 0, ex.stream>>>(A, lda, na, B, ldb, nb, n, chunk, part.c());
  else if (GA == 32)
    k_gram<32, 16><<<grid, 256, 0, ex.stream>>>(A, lda, na, B, ldb, nb, n, chunk, part.c());
  else if (GB == 8)
    k_gram<64, 8><<<grid, 256, 0, ex.stream>>>(A, lda, na, B, ldb, nb, n, chunk, part.c());
  else
    k_gram<64, 16><<<grid, 256, 0, ex.stream>>>(A, lda, na, B, ldb, nb, n, chunk, part.c());
  ADC_CHECK_LAUNCH();
  k_gram_reduce<<<(na * nb + 255) / 256, 256, 0, ex.stream>>>(part.c(), (int)nchunk, na, nb, alpha, G, ldg);
  ADC_CHECK_LAUNCH();
  ex.prof_end(pr);
}

void combine(Exec &ex, const cplx *C, int64_t ldc, int m, int nr, const cplx *V, int64_t ldv, int64_t n,
             cplx alpha, cplx beta, cplx *Y, int64_t ldy) {
  if (nr <= 0 || n <= 0) return;
  const int64_t gx = (n + 255) / 256;
  const int RR = nr <= 8 ? 8 : 16;
  const int gy = (nr + RR - 1) / RR;
  ADC_REQUIRE(gx < (1ll << 31) && gy <= 65535, ADC_ERR_UNSUPPORTED, "combine: shape");
  int pr = ex.prof_begin("combine_fp64", 8.0 * (double)nr * m * (double)n);
  if (RR == 8)
    k_combine<8><<<dim3((unsigned)gx, gy), 256, 0, ex.stream>>>(C, ldc, m, nr, V, ldv, n, alpha, beta, Y, ldy);
  else
    k_combine<16><<<dim3((unsigned)gx, gy), 256, 0, ex.stream>>>(C, ldc, m, nr, V, ldv, n, alpha, beta, Y, ldy);
  ADC_CHECK_LAUNCH();
  ex.prof_end(pr);
}

}  // namespace adc
