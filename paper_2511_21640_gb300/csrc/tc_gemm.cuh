// Split-precision (BF16x3) complex GEMM on tcgen05; see tc_gemm.cu.
#pragma once
#include <cuda.h>

#include <vector>

#include "tensor.cuh"

struct adc_ctx;

namespace adc {

// value of B[n][k] for the three gather patterns of the B operands:
// strided, the EA ring and the IP ring gathered from the packed satellite block
struct BSrc {
  const cplx *p;
  int mode;        // 0 strided, 1 EA ring from packed X2, 2 IP ring from packed X2
  int64_t s_nh, s_nl, n_in, s_k;
  int64_t o, v, N, n1;
  __device__ __forceinline__ cplx get(int64_t n, int64_t k) const {
    if (mode == 0) {
      const int64_t nh = n / n_in, nl = n - nh * n_in;
      return p[nh * s_nh + nl * s_nl + k * s_k];
    }
    if (mode == 1) {  // n = (vec, b), k = (kk, c): Xf[vec][kk][c][b]
      const int64_t vec = n / v, b = n - vec * v;
      const int64_t kk = k / v, cc = k - kk * v;
      if (cc == b) return cmake(0.0, 0.0);
      const int64_t lo_ = cc < b ? cc : b, hi_ = cc < b ? b : cc;
      cplx x = p[n1 + vec * N + kk * (v * (v - 1) / 2) + pair_index(lo_, hi_, v)];
      return cc < b ? x : cmake(-x.x, -x.y);
    }
    // mode 2: n = (vec, i), k = (kp_, b): Xf[vec][i][kp_][b]
    const int64_t vec = n / o, i = n - vec * o;
    const int64_t kq = k / v, b = k - kq * v;
    if (kq == i) return cmake(0.0, 0.0);
    const int64_t lo_ = i < kq ? i : kq, hi_ = i < kq ? kq : i;
    cplx x = p[n1 + vec * N + pair_index(lo_, hi_, o) * v + b];
    return i < kq ? x : cmake(-x.x, -x.y);
  }
  // B[n][k0 .. k0 + 7] (zero past K): the row's index arithmetic once, the
  // inner index walked incrementally
  __device__ __forceinline__ void get8(int64_t n, int64_t k0, int64_t K, cplx (&x)[8]) const {
    if (mode == 0) {
      const int64_t nh = n / n_in, nl = n - nh * n_in;
      const cplx *base = p + nh * s_nh + nl * s_nl;
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = (k0 + j < K) ? base[(k0 + j) * s_k] : cmake(0.0, 0.0);
      return;
    }
    if (mode == 1) {  // n = (vec, b), k = (kk, c)
      const int64_t vec = n / v, b = n - vec * v;
      int64_t kk = k0 / v, cc = k0 - kk * v;
      const cplx *row = p + n1 + vec * N;
      const int64_t pv = v * (v - 1) / 2;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        cplx r = cmake(0.0, 0.0);
        if (k0 + j < K && cc != b) {
          const int64_t lo_ = cc < b ? cc : b, hi_ = cc < b ? b : cc;
          const cplx y = row[kk * pv + pair_index(lo_, hi_, v)];
          r = cc < b ? y : cmake(-y.x, -y.y);
        }
        x[j] = r;
        if (++cc == v) { cc = 0; ++kk; }
      }
      return;
    }
    // mode 2: n = (vec, i), k = (kq, b)
    const int64_t vec = n / o, i = n - vec * o;
    int64_t kq = k0 / v, b = k0 - kq * v;
    const cplx *row = p + n1 + vec * N;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      cplx r = cmake(0.0, 0.0);
      if (k0 + j < K && kq != i) {
        const int64_t lo_ = i < kq ? i : kq, hi_ = i < kq ? kq : i;
        const cplx y = row[pair_index(lo_, hi_, o) * v + b];
        r = i < kq ? y : cmake(-y.x, -y.y);
      }
      x[j] = r;
      if (++b == v) { b = 0; ++kq; }
    }
  }
};

// An operand in the real embedding, split into BF16 planes of shape
// [rows][2*kp] (kp = K rounded up to 64): hi = bf16(x), lo = bf16(x - hi) and,
// for the six-product split, lo2 = bf16(x - hi - lo). For A, rows = M; for B,
// rows = 2N.
struct TcMat {
  DBuf hi, lo, lo2;
  int planes = 2;
  int64_t rows = 0, kp = 0, kreal = 0;
};

// rows [row0, row0 + rows) of a packed operand, without owning them
struct TcView {
  const void *hi = nullptr, *lo = nullptr, *lo2 = nullptr;
  int planes = 2;
  int64_t rows = 0, kp = 0, kreal = 0;
};
TcView tc_view(const TcMat &m, int64_t row0 = 0, int64_t rows = -1);

// A[m][k] = op(src[m*s_m + k*s_k]) (op = conj when conj is set); planes 2 or 3
void tc_pack_A(Exec &ex, TcMat &dst, const cplx *src, int64_t M, int64_t K, int64_t s_m, int64_t s_k, bool conj,
               int planes = 2);
// B[n][k] = op(src[(n / n_in)*s_nh + (n % n_in)*s_nl + k*s_k]), Nc complex rows
void tc_pack_B(Exec &ex, TcMat &dst, const cplx *src, int64_t Nc, int64_t K, int64_t s_nh, int64_t s_nl,
               int64_t n_in, int64_t s_k, bool conj, int planes = 2);
// B operand of the ring term, gathered from the packed satellite block of X
void tc_pack_B_ring(Exec &ex, TcMat &dst, const adc_ctx *c, const cplx *X, int64_t k, int planes = 2);
// out[m][n] (n = nh*n_in + nl at m*s_m + nh*s_nh + nl*s_nl) = alpha * A B^T + beta * out,
// with nseg = 3 products (hi hi, hi lo, lo hi) or 6 (plus hi lo2, lo lo, lo2 hi;
// both operands need three planes)
void tc_gemm(Exec &ex, const TcMat &A, const TcMat &B, int64_t M, int64_t N, cplx alpha, cplx beta, cplx *out,
             int64_t s_m, int64_t s_nh, int64_t s_nl, int64_t n_in, int *err, int nseg = 3);
// the same on views (row ranges of packed operands)
void tc_gemm(Exec &ex, const TcView &A, const TcView &B, int64_t M, int64_t N, cplx alpha, cplx beta, cplx *out,
             int64_t s_m, int64_t s_nh, int64_t s_nl, int64_t n_in, int *err, int nseg = 3);

// ---- grouped persistent launch (several problems and terms in one kernel)
constexpr int TC_BNMAX = 256;

// one job as the kernel reads it (device memory, 128-byte aligned tensor maps)
struct alignas(128) TcJob {
  CUtensorMap mAh, mAl, mBh, mBl;
  cplx *out;
  float *part;  // split-K partials [ksplit][M][N2] or null
  int64_t s_m, s_nh, s_nl, n_in;
  cplx alpha, beta;
  int M, N2, kps, bn, tiles_n, tiles_m, ksplit, kb_per_split, tile_begin, nseg;
  int l2keepB;  // 1: the B operand (re-read by every row block) loaded with an L2 evict-last
                // policy and A with evict-first, so that B stays in L2 while A streams
  int panel;    // column blocks per panel: tiles run panel by panel, row blocks inside a
                // panel, so that one panel of B is re-read from L2 (tiles_n: one panel)
};

// one job as the host describes it: out = alpha * A B^T + beta * out, same
// output addressing as tc_gemm; bn = tile width in real columns (0: autotuned)
struct TcJobDesc {
  const TcMat *A = nullptr, *B = nullptr;
  int64_t M = 0, N = 0;
  cplx alpha{1.0, 0.0}, beta{0.0, 0.0};
  cplx *out = nullptr;
  int64_t s_m = 0, s_nh = 0, s_nl = 0, n_in = 1;
  int bn = 0;
  // products per tile: 3 (hi hi, hi lo, lo hi) or 1 (hi hi: one plane of each
  // operand, e.g. one pair of slices of the sliced FP64 product)
  int nseg = 3;
  // raw mode: when set, the FP32 sums of each K split s are written to
  // out32[s][M][2N] (real columns) and out/alpha/beta are unused; every split
  // holds at most kb_split k-blocks of 64 (required in raw mode)
  float *out32 = nullptr;
  int kb_split = 0;
};

// device and pinned host state of a grouped launch. A captured graph copies
// the job table out of `host` at every replay, so a TcGroup captured into a
// graph belongs to that graph and is not reused for other launches.
struct TcGroup {
  DBuf jobs, counter, part;
  cudaEvent_t ev = nullptr;  // completion of the last copy out of `host`
  TcJob *host = nullptr;
  size_t host_cap = 0;
  size_t part_elems = 0;
  double flops = 0.0;  // algorithmic flops of the jobs (8 per complex MAC)
  TcGroup() = default;
  TcGroup(const TcGroup &) = delete;
  TcGroup &operator=(const TcGroup &) = delete;
  ~TcGroup();
};

// enqueue all jobs as one persistent launch (plus split-K reductions). With
// may_tune, jobs with bn == 0 get the autotuned tile width (timing runs need a
// stream that is not being captured); otherwise a size rule picks it.
void tc_gemm_grouped(Exec &ex, const std::vector<TcJobDesc> &jobs, TcGroup &grp, int *err, bool may_tune);
// tile width chosen by timing every candidate once per (M, N, K) shape; cached
int tc_autotune_bn(Exec &ex, const TcJobDesc &d, int *err);
// table of tuned shapes: (M, N2, kp, bn); returns the number of entries
int tc_autotune_table(int64_t *out, int cap);
// limit (ns) of the tensor-core kernels' pipeline waits on the current device;
// 0 restores the default of 2 s (the drains after an abort keep their own 2 s)
void tc_set_wait_ns(uint64_t ns);

struct TcCache {
  int planes = 2;            // BF16 planes of the copies (3 for the six-product split)
  TcMat Glad, W, Cpl, CplT;  // static operators (A side)
  TcMat LA, LB;              // B^Q_ac as both operands of the integral-direct ladder's J = L L^T
  TcMat Bx;                  // per-call B operand
  TcMat Bx1, Bx2, Bxl, Bxr;  // per-call B operands of the grouped product (X1, X2, ladder, ring)
  TcGroup grp;               // job table of the grouped product
  DBuf err;                  // device error word of the tensor-core kernels
  bool ready = false;
};

}  // namespace adc
