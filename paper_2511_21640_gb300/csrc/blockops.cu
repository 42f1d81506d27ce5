// FP64 block kernels of the Davidson solver for "tall-skinny" operands: a
// handful of long vectors (length N, up to 10^8) against a subspace of at most
// a few hundred. On GB300 the FP64 units execute two fused multiply-adds per
// clock per SM, so these products are bound by the FP64 pipe, never by HBM
// (about 3 flops per byte against a ridge near 0.2): the only thing that
// matters is that every issued FP64 operation is useful. The tile shapes are
// therefore chosen per call from the actual numbers of rows on both sides, so
// that no FMA is spent on padding, and the K dimension is split across the
// threads of a CTA (reduced by warp shuffles) instead of padding the tile.
//
// Complex products use three real products (3M): for conj(a) b,
//   T1 = ar br, T2 = ai bi, T3 = (ar - ai)(br + bi),
//   Re = T1 + T2, Im = T3 - T1 + T2,
// with the sums ar - ai and br + bi formed once per staged element.
#include <algorithm>
#include <climits>

#include "blockops.cuh"

namespace adc {

namespace {

// ---------------------------------------------------------------- gram
// smallest stride >= g (in doubles) with stride % q == r
__host__ __device__ constexpr int stride_mod(int g, int q, int r) { return g + ((r - g % q) + q) % q; }

// part[chunk][a][b] = sum_{k in chunk} conj(A[a][k]) B[b][k] for one (GA x GB)
// output tile per CTA. 256 threads: TA x TB register tiles of RA x RB outputs
// (rows a0 + ta + TA i, columns b0 + tb + TB j), and KS = 256 / (TA TB)
// adjacent lanes per register tile, each taking every KS-th staged k; their
// sums meet by warp shuffles at the end. The staged rows are padded (in
// doubles) so that the 16 lanes of a half-warp, which read from KS different
// k rows, fall on distinct banks: an odd stride when a half-warp is one
// register tile (KS >= 16), 2 mod 4 when it is two (KS = 8), 4 mod 8 when it
// is four (KS = 4); the B side, read by one column group, takes an odd stride.
template <int GA, int GB, int RA, int RB, int GK>
__global__ void __launch_bounds__(256)
k_gram(const cplx *__restrict__ A, int64_t lda, int na, const cplx *__restrict__ B, int64_t ldb, int nb,
       int64_t n, int64_t chunk, cplx *part) {
  constexpr int TA = GA / RA, TB = GB / RB, KS = 256 / (TA * TB);
  static_assert(TA * TB * KS == 256 && KS >= 4 && KS <= 32 && GK % KS == 0 && TA >= 8, "gram tile");
  constexpr int SA = KS >= 16 ? stride_mod(GA, 2, 1) : KS == 8 ? stride_mod(GA, 4, 2) : stride_mod(GA, 8, 4);
  constexpr int SB = stride_mod(GB, 2, 1);
  static_assert(3 * GK * (SA + SB) * 8 <= 48 * 1024, "gram staging exceeds 48 KB");
  __shared__ double sA[3][GK * SA];  // re, im, re - im of conj-side rows
  __shared__ double sB[3][GK * SB];  // re, im, re + im
  const int t = threadIdx.x;
  const int ks = t % KS, tile = t / KS;
  const int ta = tile % TA, tb = tile / TA;
  const int a0 = blockIdx.y * GA, b0 = blockIdx.z * GB;
  const int64_t k_beg = (int64_t)blockIdx.x * chunk;
  const int64_t k_end = min(n, k_beg + chunk);
  double t1[RA][RB], t2[RA][RB], t3[RA][RB];
#pragma unroll
  for (int i = 0; i < RA; ++i)
#pragma unroll
    for (int j = 0; j < RB; ++j) t1[i][j] = t2[i][j] = t3[i][j] = 0.0;
  for (int64_t k0 = k_beg; k0 < k_end; k0 += GK) {
    for (int e = t; e < GA * GK; e += 256) {
      const int ai = e / GK, kk = e % GK;
      const int64_t k = k0 + kk;
      cplx v = cmake(0.0, 0.0);
      if (a0 + ai < na && k < k_end) v = A[(int64_t)(a0 + ai) * lda + k];
      sA[0][kk * SA + ai] = v.x;
      sA[1][kk * SA + ai] = v.y;
      sA[2][kk * SA + ai] = v.x - v.y;
    }
    for (int e = t; e < GB * GK; e += 256) {
      const int bi = e / GK, kk = e % GK;
      const int64_t k = k0 + kk;
      cplx v = cmake(0.0, 0.0);
      if (b0 + bi < nb && k < k_end) v = B[(int64_t)(b0 + bi) * ldb + k];
      sB[0][kk * SB + bi] = v.x;
      sB[1][kk * SB + bi] = v.y;
      sB[2][kk * SB + bi] = v.x + v.y;
    }
    __syncthreads();
    for (int kk = ks; kk < GK; kk += KS) {
      double ar[RA], ai[RA], as[RA], br[RB], bi[RB], bs[RB];
#pragma unroll
      for (int i = 0; i < RA; ++i) {
        ar[i] = sA[0][kk * SA + ta + TA * i];
        ai[i] = sA[1][kk * SA + ta + TA * i];
        as[i] = sA[2][kk * SA + ta + TA * i];
      }
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        br[j] = sB[0][kk * SB + tb + TB * j];
        bi[j] = sB[1][kk * SB + tb + TB * j];
        bs[j] = sB[2][kk * SB + tb + TB * j];
      }
#pragma unroll
      for (int i = 0; i < RA; ++i)
#pragma unroll
        for (int j = 0; j < RB; ++j) {
          t1[i][j] = fma(ar[i], br[j], t1[i][j]);
          t2[i][j] = fma(ai[i], bi[j], t2[i][j]);
          t3[i][j] = fma(as[i], bs[j], t3[i][j]);
        }
    }
    __syncthreads();
  }
  // sum over the KS lanes of each register tile
#pragma unroll
  for (int i = 0; i < RA; ++i)
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      double re = t1[i][j] + t2[i][j];
      double im = t3[i][j] - t1[i][j] + t2[i][j];
#pragma unroll
      for (int off = KS / 2; off > 0; off >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, off);
        im += __shfl_xor_sync(0xffffffffu, im, off);
      }
      const int a = a0 + ta + TA * i, b = b0 + tb + TB * j;
      if (ks == 0 && a < na && b < nb) part[((int64_t)blockIdx.x * na + a) * nb + b] = cmake(re, im);
    }
}

// G[a][b] = alpha sum_c part[c][a][b]; with trans, part holds the transposed
// product (part[c][b][a] = sum conj(B_b) A_a) and G[a][b] = alpha conj(.)
__global__ void k_gram_reduce(const cplx *__restrict__ part, int nchunk, int na, int nb, int trans, cplx alpha,
                              cplx *G, int64_t ldg) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= na * nb) return;
  const int a = idx / nb, b = idx % nb;
  const int src = trans ? b * na + a : idx;
  cplx s = cmake(0.0, 0.0);
  for (int c = 0; c < nchunk; ++c) s = cadd(s, part[(int64_t)c * na * nb + src]);
  if (trans) s = cconj(s);
  G[(int64_t)a * ldg + b] = cmul(alpha, s);
}

typedef void (*GramFn)(const cplx *, int64_t, int, const cplx *, int64_t, int, int64_t, int64_t, cplx *);

struct GramCfg {
  int ga, gb, gk;
  GramFn fn;
};

// register tiles: RB = 4 for 16 columns, else min(GB, 2); RA = 4 for 32 or 64
// rows, 2 for 16, 1 for 8 (so that 4 to 32 lanes share a register tile); GK
// staged k per step so that the staged triples stay within 48 KB
#define GRAM_CFG(GA, GB, RA, RB, GK) {GA, GB, GK, &k_gram<GA, GB, RA, RB, GK>}
const GramCfg kGramCfgs[] = {
    GRAM_CFG(8, 1, 1, 1, 64),   GRAM_CFG(8, 2, 1, 2, 64),   GRAM_CFG(8, 4, 1, 2, 64),
    GRAM_CFG(8, 8, 1, 2, 64),   GRAM_CFG(8, 16, 1, 4, 32),  GRAM_CFG(16, 1, 2, 1, 64),
    GRAM_CFG(16, 2, 2, 2, 64),  GRAM_CFG(16, 4, 2, 2, 64),  GRAM_CFG(16, 8, 2, 2, 32),
    GRAM_CFG(16, 16, 2, 4, 32), GRAM_CFG(32, 1, 4, 1, 32),  GRAM_CFG(32, 2, 4, 2, 32),
    GRAM_CFG(32, 4, 4, 2, 32),  GRAM_CFG(32, 8, 4, 2, 32),  GRAM_CFG(32, 16, 4, 4, 32),
    GRAM_CFG(64, 1, 4, 1, 16),  GRAM_CFG(64, 2, 4, 2, 16),  GRAM_CFG(64, 4, 4, 2, 16),
    GRAM_CFG(64, 8, 4, 2, 16),  GRAM_CFG(64, 16, 4, 4, 16),
};
#undef GRAM_CFG

// FP64 operations per staged k of the whole product with this tile: 3 FMAs per
// padded output plus one add per staged element of each side, per tile
int64_t gram_ops(int na, int nb, int ga, int gb) {
  const int64_t ta = (na + ga - 1) / ga, tb = (nb + gb - 1) / gb;
  return ta * tb * (3LL * ga * gb + ga + gb);
}

// ---------------------------------------------------------------- combine
constexpr int CI = 64;  // subspace rows staged per step

// Y[r][k] = alpha sum_i C[i][r] V[i][k] + beta Y[r][k], r in this CTA's group
// of RR rows; 3M products (as in k_gram, without the conjugate)
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

int sm_count() { return device_sm_count(); }

}  // namespace

void gram(Exec &ex, const cplx *A, int64_t lda, int na, const cplx *B, int64_t ldb, int nb, int64_t n, cplx alpha,
          cplx *G, int64_t ldg) {
  if (na <= 0 || nb <= 0) return;
  if (n <= 0) {
    for (int a = 0; a < na; ++a) ADC_CUDA(cudaMemsetAsync(G + (int64_t)a * ldg, 0, nb * sizeof(cplx), ex.stream));
    return;
  }
  int pr = ex.prof_begin("gram_fp64", 8.0 * (double)na * nb * (double)n,
                         16.0 * ((double)(na + nb) * (double)n + (double)na * nb));
  // one row against many: the transposed product has the long side in rows
  const bool trans = (na < 8 && nb > na);
  const cplx *P = trans ? B : A, *R = trans ? A : B;
  const int64_t ldp = trans ? ldb : lda, ldr = trans ? lda : ldb;
  const int np = trans ? nb : na, nr = trans ? na : nb;
  const GramCfg *best = nullptr;
  int64_t best_ops = LLONG_MAX;
  for (const GramCfg &g : kGramCfgs) {
    const int64_t ops = gram_ops(np, nr, g.ga, g.gb);
    // ties go to the larger tile (fewer staged re-reads)
    if (ops < best_ops || (ops == best_ops && g.ga * g.gb > best->ga * best->gb)) {
      best_ops = ops;
      best = &g;
    }
  }
  const int gy = (np + best->ga - 1) / best->ga, gz = (nr + best->gb - 1) / best->gb;
  // enough CTAs for four per SM, each chunk at least four staged steps
  int64_t nchunk = std::max<int64_t>(1, (4 * (int64_t)sm_count() + gy * gz - 1) / (gy * gz));
  nchunk = std::min<int64_t>(nchunk, std::max<int64_t>(1, n / (4 * best->gk)));
  int64_t chunk = (n + nchunk - 1) / nchunk;
  chunk = (chunk + best->gk - 1) / best->gk * best->gk;
  nchunk = std::max<int64_t>(1, (n + chunk - 1) / chunk);
  ADC_REQUIRE(nchunk < (1ll << 31) && gy <= 65535 && gz <= 65535, ADC_ERR_UNSUPPORTED, "gram: shape");
  DBuf part = cbuf(ex, nchunk * (int64_t)na * nb);
  const dim3 grid((unsigned)nchunk, gy, gz);
  best->fn<<<grid, 256, 0, ex.stream>>>(P, ldp, np, R, ldr, nr, n, chunk, part.c());
  ADC_CHECK_LAUNCH();
  k_gram_reduce<<<(na * nb + 255) / 256, 256, 0, ex.stream>>>(part.c(), (int)nchunk, na, nb, trans ? 1 : 0, alpha,
                                                               G, ldg);
  ADC_CHECK_LAUNCH();
  ex.prof_end(pr);
}

void combine(Exec &ex, const cplx *C, int64_t ldc, int m, int nr, const cplx *V, int64_t ldv, int64_t n,
             cplx alpha, cplx beta, cplx *Y, int64_t ldy) {
  if (nr <= 0 || n <= 0) return;
  const int64_t gx = (n + 255) / 256;
  // rows per CTA: the smallest group that covers nr in as few padded rows as
  // possible (16 for more than 8)
  const int RR = nr >= 9 ? 16 : nr >= 5 ? 8 : nr >= 3 ? 4 : nr;
  const int gy = (nr + RR - 1) / RR;
  ADC_REQUIRE(gx < (1ll << 31) && gy <= 65535, ADC_ERR_UNSUPPORTED, "combine: shape");
  const bool rd = (beta.x != 0.0 || beta.y != 0.0);
  int pr = ex.prof_begin("combine_fp64", 8.0 * (double)nr * m * (double)n,
                         16.0 * ((double)m + (rd ? 2.0 : 1.0) * nr) * (double)n);
  const dim3 grid((unsigned)gx, gy);
  switch (RR) {
    case 1: k_combine<1><<<grid, 256, 0, ex.stream>>>(C, ldc, m, nr, V, ldv, n, alpha, beta, Y, ldy); break;
    case 2: k_combine<2><<<grid, 256, 0, ex.stream>>>(C, ldc, m, nr, V, ldv, n, alpha, beta, Y, ldy); break;
    case 4: k_combine<4><<<grid, 256, 0, ex.stream>>>(C, ldc, m, nr, V, ldv, n, alpha, beta, Y, ldy); break;
    case 8: k_combine<8><<<grid, 256, 0, ex.stream>>>(C, ldc, m, nr, V, ldv, n, alpha, beta, Y, ldy); break;
    default: k_combine<16><<<grid, 256, 0, ex.stream>>>(C, ldc, m, nr, V, ldv, n, alpha, beta, Y, ldy); break;
  }
  ADC_CHECK_LAUNCH();
  ex.prof_end(pr);
}

}  // namespace adc
