// FP64-accurate complex GEMM from BF16 slices on the tensor cores.
//
// out[m][n] = alpha * sum_k A[m][k] B[n][k] + beta * out[m][n]   (complex)
//
// The operands use the real embedding of tc_gemm.cu (an A row is [Re | Im], a
// complex B row n becomes [Re | -Im] and [Im | Re]). Every row of an operand
// is scaled by a power of two, 2^E with max |row| < 2^E, and each scaled value
// y (|y| < 1) is written as a sum of slices y = sum_i d_i 2^(-b i), i = 1..ns,
// with integer digits d_i = rint((y - d_1 2^-b - ... - d_(i-1) 2^(-b (i-1))) 2^(b i)),
// so |d_1| <= 2^b and |d_i| <= 2^(b-1) for i >= 2: integers of at most b + 1
// bits, exact in BF16 for b <= 7. The product of slice i of A and slice j of B
// over K2 embedded terms is a sum of integers whose partial sums stay below
// K2 2^(2b); with K2 <= 2^(24 - 2b) (longer inner sizes are split) every
// partial sum is an integer below 2^24 and the tensor cores' FP32 accumulator
// holds it exactly. The pairs i + j <= ns + 1 run as one grouped tcgen05 launch
// (tc_gemm_grouped, one product per tile, raw FP32 outputs) and a combine
// kernel forms, in FP64, sum over pairs and splits of 2^(E_m + F_n - b (i + j)) P_ij.
// The error comes only from the dropped slice digits and pairs, about 2^(-b ns)
// relative to the row and column maxima, whatever K is: an error-free
// splitting of the products in the manner of Ozaki, Ogita, Oishi and Rump
// ("Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication", Numer. Algorithms 59, 2012), on BF16
// tensor cores with integer digits.
#include <cuda_bf16.h>

#include <cmath>

#include "ctx.cuh"
#include "tc_gemm.cuh"
#include "tc_slice.cuh"

namespace adc {

namespace {

constexpr int SL_MAXPAIRS = 160;

__device__ __forceinline__ double amax2(cplx x) { return fmax(fabs(x.x), fabs(x.y)); }

// block-wide maximum (blockDim.x a multiple of 32, at most 1024)
__device__ double block_max(double v) {
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
  }
  return v;  // valid in thread 0
}

// exponent E with max < 2^E (0 for an all-zero row)
__device__ __forceinline__ int exp_above(double amax) {
  if (!(amax > 0.0)) return 0;
  int e;
  frexp(amax, &e);  // amax = f 2^e, f in [0.5, 1)
  return e;
}

// E[m] for the rows of A (element (m, k) at src[m*s_m + k*s_k]), one block per row
__global__ void k_sl_exp_A(const cplx *__restrict__ src, int64_t M, int64_t K, int64_t s_m, int64_t s_k, int *E) {
  for (int64_t m = blockIdx.x; m < M; m += gridDim.x) {
    double v = 0.0;
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x) v = fmax(v, amax2(src[m * s_m + k * s_k]));
    v = block_max(v);
    if (threadIdx.x == 0) E[m] = exp_above(v);
    __syncthreads();
  }
}

// F[n] for the complex rows of B, one block per row
__global__ void k_sl_exp_B(BSrc src, int64_t Nc, int64_t K, int *F) {
  for (int64_t n = blockIdx.x; n < Nc; n += gridDim.x) {
    double v = 0.0;
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x) v = fmax(v, amax2(src.get(n, k)));
    v = block_max(v);
    if (threadIdx.x == 0) F[n] = exp_above(v);
    __syncthreads();
  }
}

// Digits in integer arithmetic (the FP64 pipe is the scarce one): the value
// y = x 2^-E (|y| < 1) as the integer R = round(y 2^(b ns)) (at most 61 bits),
// then ns signed digits of b bits, each rounded to nearest with the remainder
// carried to the next (|d_1| <= 2^b, |d_i| <= 2^(b-1) after it), so that
// y = sum_i d_i 2^(-b i) to within 2^(-b ns - 1).
__device__ __forceinline__ long long fixed_of(double x, int E, int bns) { return llrint(ldexp(x, bns - E)); }
__device__ __forceinline__ int next_digit(long long &R, int sh) {
  const long long d = (sh > 0) ? ((R + (1LL << (sh - 1))) >> sh) : R;
  R -= d * (1LL << sh);
  return (int)d;
}

// A rows [Re | Im] (conj negates Im), padded to kp with zeros. One thread per
// 8 consecutive k of a row, 16-byte stores of every slice
__global__ void k_sl_slice_A(const cplx *__restrict__ src, int64_t M, int64_t K, int64_t s_m, int64_t s_k, int conj,
                             int64_t kp, const int *__restrict__ E, int ns, int b, __nv_bfloat16 *base, int64_t pe) {
  const int64_t kq = kp >> 3;
  const int64_t total = M * kq;
  const int bns = b * ns;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = idx / kq, k0 = (idx - m * kq) << 3;
    const cplx *row = src + m * s_m;
    const int e = E[m];
    long long Rr[8], Ri[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t k = k0 + j;
      cplx x = cmake(0.0, 0.0);
      if (k < K) x = row[k * s_k];
      Rr[j] = fixed_of(x.x, e, bns);
      Ri[j] = fixed_of(conj ? -x.y : x.y, e, bns);
    }
    const int64_t r0 = m * 2 * kp + k0;
    for (int i = 1; i <= ns; ++i) {
      const int sh = b * (ns - i);
      __align__(16) __nv_bfloat16 dr[8], di[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        dr[j] = __int2bfloat16_rn(next_digit(Rr[j], sh));
        di[j] = __int2bfloat16_rn(next_digit(Ri[j], sh));
      }
      __nv_bfloat16 *pl = base + (int64_t)(i - 1) * pe;
      *(uint4 *)(pl + r0) = *(const uint4 *)dr;
      *(uint4 *)(pl + r0 + kp) = *(const uint4 *)di;
    }
  }
}

// B rows: row 2n = [Re | -Im], row 2n+1 = [Im | Re] (conj negates Im first).
// One thread per 8 consecutive k of a row; every slice's digits of the 8
// elements go out as 16-byte stores (the digits of -Im are the negated digits of Im)
__global__ void k_sl_slice_B(BSrc src, int64_t Nc, int64_t K, int conj, int64_t kp, const int *__restrict__ F,
                             int ns, int b, __nv_bfloat16 *base, int64_t pe) {
  const int64_t kq = kp >> 3;
  const int64_t total = Nc * kq;
  const int bns = b * ns;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = idx / kq, k0 = (idx - n * kq) << 3;
    cplx x[8];
    src.get8(n, k0, K, x);
    const int e = F[n];
    long long Rr[8], Ri[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      Rr[j] = fixed_of(x[j].x, e, bns);
      Ri[j] = fixed_of(conj ? -x[j].y : x[j].y, e, bns);
    }
    const int64_t r0 = (2 * n) * 2 * kp + k0, r1 = (2 * n + 1) * 2 * kp + k0;
    for (int i = 1; i <= ns; ++i) {
      const int sh = b * (ns - i);
      __align__(16) __nv_bfloat16 dr[8], di[8], dn[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int a = next_digit(Rr[j], sh), c = next_digit(Ri[j], sh);
        dr[j] = __int2bfloat16_rn(a);
        di[j] = __int2bfloat16_rn(c);
        dn[j] = __int2bfloat16_rn(-c);
      }
      __nv_bfloat16 *pl = base + (int64_t)(i - 1) * pe;
      *(uint4 *)(pl + r0) = *(const uint4 *)dr;
      *(uint4 *)(pl + r0 + kp) = *(const uint4 *)dn;
      *(uint4 *)(pl + r1) = *(const uint4 *)di;
      *(uint4 *)(pl + r1 + kp) = *(const uint4 *)dr;
    }
  }
}

struct SlCombine {
  int npair, ksplit;
  int sh[SL_MAXPAIRS];     // b (i + j) of each pair; pairs ordered by i + j
  double sc[SL_MAXPAIRS];  // 2^-sh (exact)
};

// out[m][n] = alpha 2^(E_m + F_n) sum_p sum_s 2^-sh_p P[p][s][m][2n..2n+1] + beta out.
// Every P is an integer below 2^24 held exactly in FP32; the pairs of one
// shift (same i + j) and their K splits are summed exactly as 64-bit integers,
// and only one FP64 conversion and product per shift remains (the FP64 pipe is
// the scarce one).
__global__ void k_sl_combine(const float *__restrict__ P, SlCombine cfg, int64_t M, int64_t N2,
                             const int *__restrict__ E, const int *__restrict__ F, cplx alpha, cplx beta, cplx *out,
                             int64_t s_m, int64_t s_nh, int64_t s_nl, int64_t n_in) {
  const int64_t Nc = N2 / 2, total = M * Nc, per = M * N2;
  const bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = idx % Nc, m = idx / Nc;
    const float *base = P + m * N2 + 2 * n;
    double re = 0.0, im = 0.0;
    long long ar = 0, ai = 0;
    for (int p = cfg.npair - 1; p >= 0; --p) {  // smallest terms first
      for (int s = 0; s < cfg.ksplit; ++s) {
        const float2 v = *(const float2 *)(base + ((int64_t)p * cfg.ksplit + s) * per);
        ar += __float2int_rn(v.x);
        ai += __float2int_rn(v.y);
      }
      if (p == 0 || cfg.sh[p - 1] != cfg.sh[p]) {  // last pair of this shift
        re = fma((double)ar, cfg.sc[p], re);
        im = fma((double)ai, cfg.sc[p], im);
        ar = 0;
        ai = 0;
      }
    }
    const int e = E[m] + F[n];
    const cplx val0 = cmake(ldexp(re, e), ldexp(im, e));
    const int64_t nh = n / n_in, nl = n - nh * n_in;
    cplx *dst = out + m * s_m + nh * s_nh + nl * s_nl;
    cplx val = cmul(alpha, val0);
    if (use_beta) val = cadd(val, cmul(beta, *dst));
    *dst = val;
  }
}

int ceil_log2(int64_t x) {
  int l = 0;
  while ((1ll << l) < x) ++l;
  return l;
}

void set_views(SlMat &d) {
  const int64_t pe = d.rows * 2 * d.kp;
  d.s.resize(d.ns);
  for (int i = 0; i < d.ns; ++i) {
    TcMat &t = d.s[i];
    t.hi.ex = nullptr;  // a view into d.planes
    t.hi.p = (__nv_bfloat16 *)d.planes.p + (int64_t)i * pe;
    t.hi.bytes = (size_t)pe * sizeof(__nv_bfloat16);
    t.planes = 1;
    t.rows = d.rows;
    t.kp = d.kp;
    t.kreal = d.kreal;
  }
}

void alloc_sl(Exec &ex, SlMat &d, int64_t rows, int64_t expn) {
  const size_t bytes = (size_t)d.ns * rows * 2 * d.kp * sizeof(__nv_bfloat16);
  if (d.planes.bytes < bytes) {
    d.s.clear();
    d.planes.reset();
    d.planes = DBuf(ex, bytes);
  }
  if (d.exps.bytes < (size_t)expn * sizeof(int)) {
    d.exps.reset();
    d.exps = DBuf(ex, (size_t)std::max<int64_t>(expn, 1) * sizeof(int));
  }
  d.rows = rows;
  set_views(d);
}

}  // namespace

SlParams sl_params(int64_t K, int bits) {
  SlParams p;
  p.kp = (K + 63) / 64 * 64;
  if (p.kp == 0) p.kp = 64;
  const int64_t K2 = 2 * p.kp;
  int b = (24 - ceil_log2(K2)) / 2;
  b = std::max(4, std::min(7, b));
  p.b = b;
  p.ns = (bits + b - 1) / b;
  p.kb_split = (int)((1ll << (24 - 2 * b)) / 64);
  return p;
}

void sl_pack_A(Exec &ex, SlMat &dst, const cplx *src, int64_t M, int64_t K, int64_t s_m, int64_t s_k, bool conj,
               int bits) {
  const SlParams p = sl_params(K, bits);
  dst.kp = p.kp;
  dst.kreal = K;
  dst.ns = p.ns;
  dst.bits = p.b;
  dst.kb_split = p.kb_split;
  alloc_sl(ex, dst, M, M);
  if (M <= 0) return;
  k_sl_exp_A<<<(unsigned)std::min<int64_t>(M, 65535), 256, 0, ex.stream>>>(src, M, K, s_m, s_k, (int *)dst.exps.p);
  ADC_CHECK_LAUNCH();
  k_sl_slice_A<<<grid1d(M * (dst.kp / 8), 256), 256, 0, ex.stream>>>(src, M, K, s_m, s_k, conj ? 1 : 0, dst.kp,
                                                               (const int *)dst.exps.p, dst.ns, dst.bits,
                                                               (__nv_bfloat16 *)dst.planes.p, M * 2 * dst.kp);
  ADC_CHECK_LAUNCH();
}

static void sl_pack_B_impl(Exec &ex, SlMat &dst, const BSrc &s, int64_t Nc, int64_t K, bool conj, const SlMat &like,
                           int bits) {
  ADC_REQUIRE(like.kreal == K, ADC_ERR_ARG, "sl_pack_B: inner size differs from the A operand");
  dst.kp = like.kp;
  dst.kreal = K;
  // fewer significant bits: the leading digits of the same width (the product
  // then runs over the common leading slices of both operands)
  dst.ns = bits > 0 ? std::min(like.ns, (bits + like.bits - 1) / like.bits) : like.ns;
  dst.bits = like.bits;
  dst.kb_split = like.kb_split;
  alloc_sl(ex, dst, 2 * Nc, Nc);
  if (Nc <= 0) return;
  k_sl_exp_B<<<(unsigned)std::min<int64_t>(Nc, 65535), 256, 0, ex.stream>>>(s, Nc, K, (int *)dst.exps.p);
  ADC_CHECK_LAUNCH();
  k_sl_slice_B<<<grid1d(Nc * (dst.kp / 8), 256), 256, 0, ex.stream>>>(s, Nc, K, conj ? 1 : 0, dst.kp,
                                                                (const int *)dst.exps.p, dst.ns, dst.bits,
                                                                (__nv_bfloat16 *)dst.planes.p, 2 * Nc * 2 * dst.kp);
  ADC_CHECK_LAUNCH();
}

void sl_pack_B(Exec &ex, SlMat &dst, const cplx *src, int64_t Nc, int64_t K, int64_t s_nh, int64_t s_nl,
               int64_t n_in, int64_t s_k, bool conj, const SlMat &like, int bits) {
  BSrc s{src, 0, s_nh, s_nl, n_in, s_k, 0, 0, 0, 0};
  sl_pack_B_impl(ex, dst, s, Nc, K, conj, like, bits);
}

void sl_pack_B_ring(Exec &ex, SlMat &dst, const adc_ctx *c, const cplx *X, int64_t k, const SlMat &like, int bits) {
  BSrc s{X, c->kind == ADC_EA ? 1 : 2, 0, 0, 1, 0, c->o, c->v, c->N, c->n1};
  const int64_t Nc = (c->kind == ADC_EA) ? k * c->v : k * c->o;
  sl_pack_B_impl(ex, dst, s, Nc, c->o * c->v, false, like, bits);
}

void sl_gemm(Exec &ex, const SlMat &A, const SlMat &B, int64_t M, int64_t N, cplx alpha, cplx beta, cplx *out,
             int64_t s_m, int64_t s_nh, int64_t s_nl, int64_t n_in, int *err, SlWork &w) {
  ADC_REQUIRE(A.kp == B.kp && A.bits == B.bits, ADC_ERR_ARG, "sl_gemm: operands sliced differently");
  const int ns = std::min(A.ns, B.ns);  // the common leading slices
  ADC_REQUIRE(A.rows >= M && B.rows >= 2 * N, ADC_ERR_ARG, "sl_gemm: operand rows");
  if (M <= 0 || N <= 0) return;
  if (n_in <= 0) n_in = 1;
  const int64_t N2 = 2 * N;
  const int kps = (int)(2 * A.kp / 64);
  const int kbs = std::min(A.kb_split, kps);
  const int ksplit = (kps + kbs - 1) / kbs;
  SlCombine cfg{};
  std::vector<std::pair<int, int>> pairs;
  for (int g = 2; g <= ns + 1; ++g)
    for (int i = 1; i < g; ++i)
      if (i <= ns && g - i <= ns) pairs.push_back({i, g - i});
  ADC_REQUIRE((int)pairs.size() <= SL_MAXPAIRS, ADC_ERR_UNSUPPORTED, "sl_gemm: too many slice pairs");
  cfg.npair = (int)pairs.size();
  cfg.ksplit = ksplit;
  for (size_t q = 0; q < pairs.size(); ++q) {
    cfg.sh[q] = A.bits * (pairs[q].first + pairs[q].second);
    cfg.sc[q] = std::ldexp(1.0, -cfg.sh[q]);
  }
  // output rows in chunks whose FP32 pair products stay within about 2 GiB
  const size_t per_row = (size_t)ksplit * N2 * pairs.size() * sizeof(float);
  const size_t budget = (size_t)2 << 30;
  int64_t mc = M;
  if ((size_t)M * per_row > budget) mc = std::max<int64_t>(128, (int64_t)(budget / per_row) / 128 * 128);
  const size_t need = per_row * (size_t)std::min(mc, M);
  if (w.part.bytes < need) {
    w.part.reset();
    w.part = DBuf(ex, need);
  }
  const int bn = N2 <= 32 ? 32 : N2 <= 64 ? 64 : N2 <= 128 ? 128 : 256;
  std::vector<TcMat> av(ns);
  for (int64_t m0 = 0; m0 < M; m0 += mc) {
    const int64_t mm = std::min(mc, M - m0);
    const size_t per = (size_t)ksplit * mm * N2;
    for (int i = 0; i < ns; ++i) {  // views of rows m0 .. m0 + mm of the A slices used
      TcMat &t = av[i];
      t.hi.ex = nullptr;
      t.hi.p = (__nv_bfloat16 *)A.s[i].hi.p + m0 * 2 * A.kp;
      t.hi.bytes = (size_t)mm * 2 * A.kp * sizeof(__nv_bfloat16);
      t.planes = 1;
      t.rows = mm;
      t.kp = A.kp;
      t.kreal = A.kreal;
    }
    std::vector<TcJobDesc> jobs(pairs.size());
    for (size_t q = 0; q < pairs.size(); ++q) {
      TcJobDesc &d = jobs[q];
      d.A = &av[pairs[q].first - 1];
      d.B = &B.s[pairs[q].second - 1];
      d.M = mm;
      d.N = N;
      d.nseg = 1;
      d.out32 = (float *)w.part.p + q * per;
      d.kb_split = kbs;
      d.bn = bn;
    }
    tc_gemm_grouped(ex, jobs, w.grp, err, false);
    int pr = ex.prof_begin("sl_combine", 0.0);
    k_sl_combine<<<grid1d(mm * N, 256), 256, 0, ex.stream>>>((const float *)w.part.p, cfg, mm, N2,
                                                             (const int *)A.exps.p + m0, (const int *)B.exps.p,
                                                             alpha, beta, out + m0 * s_m, s_m, s_nh, s_nl, n_in);
    ADC_CHECK_LAUNCH();
    ex.prof_end(pr);
    for (auto &t : av) { t.hi.p = nullptr; t.hi.bytes = 0; }
  }
  for (auto &t : av) { t.hi.p = nullptr; t.hi.bytes = 0; }
}

// zgemm's operands and output (element strides, conj flags, batch) through
// the sliced product: used for large contractions when Exec::sliced_bits > 0
// > 0: fixed bytes per operand chunk of zgemm_sliced instead of the free-memory rule (test hook)
static size_t g_sliced_cap = 0;
void set_sliced_cap_bytes(size_t bytes) { g_sliced_cap = bytes; }

void zgemm_sliced(Exec &ex, int64_t M, int64_t N, int64_t K, int64_t batch, cplx alpha, const cplx *A, int64_t sAb,
                  int64_t sAm, int64_t sAk, bool conjA, const cplx *B, int64_t sBb, int64_t sBk, int64_t sBn,
                  bool conjB, cplx beta, cplx *C, int64_t sCb, int64_t sCm, int64_t sCn) {
  SlMat Sa, Sb;
  SlWork w;
  DBuf err(ex, sizeof(int));
  fill_zero(ex, err.p, sizeof(int));
  // the digit planes take 4 ns kp bytes per row of A and 8 ns kp per column
  // of B (ns slices of the real embedding): rows and columns in chunks whose
  // planes stay within an eighth of the free device memory per operand
  // (between 1 and 16 GiB), so that B is sliced once where it fits. When even
  // one 128-row tile of A or 64 columns of B would exceed that, the inner
  // index is split as well: the partial products (each FP64-accurate) add up
  // in the output.
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    fr = (size_t)32 << 30;
  }
  const size_t cap =
      g_sliced_cap ? g_sliced_cap : std::min<size_t>((size_t)16 << 30, std::max<size_t>((size_t)1 << 30, fr / 8));
  int64_t kc = K;
  {
    const SlParams sp = sl_params(K, ex.sliced_bits);
    const size_t per = (size_t)4 * sp.ns * sp.kp * 128;  // one A row tile (B: 64 columns, the same bytes)
    if (per > cap) kc = std::max<int64_t>(512, (int64_t)((double)K * (double)cap / (double)per) / 64 * 64);
  }
  for (int64_t k0 = 0; k0 < K; k0 += kc) {
    const int64_t kk = std::min(kc, K - k0);
    const cplx beta_k = (k0 == 0) ? beta : C1();
    const SlParams sp = sl_params(kk, ex.sliced_bits);
    const int64_t mc = std::min<int64_t>(M, std::max<int64_t>(128, (int64_t)(cap / ((size_t)4 * sp.ns * sp.kp))));
    const int64_t nc = std::min<int64_t>(N, std::max<int64_t>(64, (int64_t)(cap / ((size_t)8 * sp.ns * sp.kp))));
    for (int64_t b = 0; b < batch; ++b) {
      const cplx *Ab = A + b * sAb + k0 * sAk, *Bb = B + b * sBb + k0 * sBk;
      for (int64_t m0 = 0; m0 < M; m0 += mc) {
        const int64_t mm = std::min(mc, M - m0);
        sl_pack_A(ex, Sa, Ab + m0 * sAm, mm, kk, sAm, sAk, conjA, ex.sliced_bits);
        for (int64_t n0 = 0; n0 < N; n0 += nc) {
          const int64_t nn = std::min(nc, N - n0);
          // B once per batch entry and inner chunk when it fits in one chunk
          if (nc < N || m0 == 0) sl_pack_B(ex, Sb, Bb + n0 * sBn, nn, kk, sBn, 0, 1, sBk, conjB, Sa);
          sl_gemm(ex, Sa, Sb, mm, nn, alpha, beta_k, C + b * sCb + m0 * sCm + n0 * sCn, sCm, sCn, 0, 1,
                  (int *)err.p, w);
        }
      }
    }
  }
  int h = 0;
  ADC_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, ex.stream));
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
  ADC_REQUIRE(h == 0, ADC_ERR_TIMEOUT, "sliced GEMM: a tensor-core wait gave up (code " + std::to_string(h) + ")");
}

}  // namespace adc
