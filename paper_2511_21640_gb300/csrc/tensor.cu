// FP64 complex tensor toolkit (see tensor.cuh).
#include <algorithm>
#include <cstring>
#include <map>

#include <map>
#include <mutex>
#include <set>
#include <tuple>

#include "tensor.cuh"
#include "tc_slice.cuh"

namespace adc {

// ------------------------------------------------------------------ memory
void *Exec::alloc(size_t bytes) {
  if (bytes == 0) return nullptr;
  if (mem_limit > 0 && mem_used + (int64_t)bytes > mem_limit)
    throw Error(ADC_ERR_OOM, "context memory limit exceeded: need " + std::to_string(bytes) +
                                 " bytes, " + std::to_string(mem_used) + " in use of " +
                                 std::to_string(mem_limit));
  void *p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(e == cudaErrorMemoryAllocation ? ADC_ERR_OOM : ADC_ERR_CUDA,
                std::string("cudaMallocAsync(") + std::to_string(bytes) + "): " + cudaGetErrorString(e) +
                    " (" + std::to_string(mem_used) + " bytes held by the context" +
                    (stage.empty() ? std::string() : ", in " + stage) + (tag.empty() ? std::string() : "/" + tag) +
                    ")");
  }
  mem_used += (int64_t)bytes;
  mem_peak = std::max(mem_peak, mem_used);
  return p;
}

void Exec::release(void *p, size_t bytes) {
  if (!p) return;
  cudaFreeAsync(p, stream);
  mem_used -= (int64_t)bytes;
}

long long g_launches = 0;

cudaEvent_t Exec::event() {
  if (!event_pool.empty()) {
    cudaEvent_t e = event_pool.back();
    event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  ADC_CUDA(cudaEventCreate(&e));
  return e;
}

int Exec::prof_begin(const char *kernel, double flops, double bytes) {
  if (!prof) return -1;
  ProfRec r;
  r.name = std::string(kernel) + (tag.empty() ? "" : "/" + tag);
  r.a = event();
  r.b = event();
  r.flops = flops;
  r.bytes = bytes;
  ADC_CUDA(cudaEventRecord(r.a, stream));
  recs.push_back(r);
  return (int)recs.size() - 1;
}

void Exec::prof_end(int r) {
  if (r >= 0) ADC_CUDA(cudaEventRecord(recs[r].b, stream));
}

void Exec::prof_clear() {
  for (auto &r : recs) {
    event_pool.push_back(r.a);
    event_pool.push_back(r.b);
  }
  recs.clear();
}

void fill_zero(Exec &ex, void *p, size_t bytes) {
  if (bytes) ADC_CUDA(cudaMemsetAsync(p, 0, bytes, ex.stream));
}

// ------------------------------------------------------------------ GEMM
// 64x64 output tile per CTA, 256 threads (16x16), 4x4 complex outputs per
// thread, K staged 16 at a time through shared memory. FP64 FMA throughput
// bounds it on GB300, so the loads only need to be coalesced along whichever
// operand index has unit stride.
namespace {
constexpr int BM = 64, BN = 64, BKK = 16;
constexpr int ZG_SMEM = (2 * BKK * (BM + 1) + 2 * BKK * (BN + 1) + BKK * (BM + 1) + BKK * (BN + 1)) * 8;

__global__ void __launch_bounds__(256)
k_zgemm(int64_t M, int64_t N, int64_t K, const cplx *__restrict__ A, int64_t sAb, int64_t sAm,
        int64_t sAk, int conjA, int a_kfast, const cplx *__restrict__ B, int64_t sBb,
        int64_t sBk, int64_t sBn, int conjB, int b_nfast, cplx *C, int64_t sCb, int64_t sCm,
        int64_t sCn, cplx alpha, cplx beta, int64_t batch0, int ksplit, int64_t kchunk,
        cplx *part, int64_t nbatch, int mfast) {
  // 3M products: (ar + i ai)(br + i bi) = T1 - T2 + i (T3 - T1 - T2) with
  // T1 = ar br, T2 = ai bi, T3 = (ar + ai)(br + bi): three FP64 FMAs per
  // complex MAC instead of four. The sums are formed once per staged element.
  extern __shared__ double zsm[];
  cplx(*As)[BM + 1] = reinterpret_cast<cplx(*)[BM + 1]>(zsm);
  cplx(*Bs)[BN + 1] = reinterpret_cast<cplx(*)[BN + 1]>(zsm + 2 * BKK * (BM + 1));
  double(*Ass)[BM + 1] = reinterpret_cast<double(*)[BM + 1]>(zsm + 2 * BKK * (BM + 1) + 2 * BKK * (BN + 1));
  double(*Bss)[BN + 1] = reinterpret_cast<double(*)[BN + 1]>(zsm + 3 * BKK * (BM + 1) + 2 * BKK * (BN + 1));
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t zl = blockIdx.z;
  const int64_t split = zl % ksplit;
  const int64_t bl = zl / ksplit;
  const int64_t b = bl + batch0;
  // with mfast the row tiles vary fastest, so the CTAs that read one column
  // tile of B (the large operand of the skinny shapes) run together and share it in L2
  const int64_t m0 = (int64_t)(mfast ? blockIdx.x : blockIdx.y) * BM;
  const int64_t n0 = (int64_t)(mfast ? blockIdx.y : blockIdx.x) * BN;
  const int64_t kbeg = split * kchunk;
  const int64_t kend = (kbeg + kchunk < K) ? kbeg + kchunk : K;
  const cplx *Ab = A + b * sAb;
  const cplx *Bb = B + b * sBb;
  double t1[4][4], t2[4][4], t3[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) t1[i][j] = t2[i][j] = t3[i][j] = 0.0;
  const double sa = conjA ? -1.0 : 1.0, sb = conjB ? -1.0 : 1.0;
  for (int64_t k0 = kbeg; k0 < kend; k0 += BKK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int kk, mm;
      if (a_kfast) { kk = tid & 15; mm = (tid >> 4) + 16 * r; }
      else { mm = tid & 63; kk = (tid >> 6) + 4 * r; }
      int64_t gm = m0 + mm, gk = k0 + kk;
      cplx val = cmake(0.0, 0.0);
      if (gm < M && gk < kend) { val = Ab[gm * sAm + gk * sAk]; val.y *= sa; }
      As[kk][mm] = val;
      Ass[kk][mm] = val.x + val.y;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int kk, nn;
      if (b_nfast) { nn = tid & 63; kk = (tid >> 6) + 4 * r; }
      else { kk = tid & 15; nn = (tid >> 4) + 16 * r; }
      int64_t gn = n0 + nn, gk = k0 + kk;
      cplx val = cmake(0.0, 0.0);
      if (gn < N && gk < kend) { val = Bb[gk * sBk + gn * sBn]; val.y *= sb; }
      Bs[kk][nn] = val;
      Bss[kk][nn] = val.x + val.y;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BKK; ++kk) {
      cplx a[4], bv[4];
      double as[4], bs[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty + 16 * i]; as[i] = Ass[kk][ty + 16 * i]; }
#pragma unroll
      for (int j = 0; j < 4; ++j) { bv[j] = Bs[kk][tx + 16 * j]; bs[j] = Bss[kk][tx + 16 * j]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          t1[i][j] = fma(a[i].x, bv[j].x, t1[i][j]);
          t2[i][j] = fma(a[i].y, bv[j].y, t2[i][j]);
          t3[i][j] = fma(as[i], bs[j], t3[i][j]);
        }
    }
    __syncthreads();
  }
  cplx acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = cmake(t1[i][j] - t2[i][j], t3[i][j] - t1[i][j] - t2[i][j]);
  if (part) {
    // split-K partial tile, unscaled: part[split][bl][m][n]
    cplx *P = part + ((int64_t)split * nbatch + bl) * M * N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int64_t gm = m0 + ty + 16 * i;
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int64_t gn = n0 + tx + 16 * j;
        if (gn < N) P[gm * N + gn] = acc[i][j];
      }
    }
    return;
  }
  cplx *Cb = C + b * sCb;
  const bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      cplx *dst = Cb + gm * sCm + gn * sCn;
      cplx r = cmul(alpha, acc[i][j]);
      if (use_beta) r = cadd(r, cmul(beta, *dst));
      *dst = r;
    }
  }
}
__global__ void k_splitk_reduce(const cplx *__restrict__ part, int ksplit, int64_t nb, int64_t M,
                                int64_t N, cplx *C, int64_t sCb, int64_t sCm, int64_t sCn,
                                cplx alpha, cplx beta, int64_t batch0) {
  const int64_t total = nb * M * N;
  const bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t n = idx % N, r = idx / N;
    int64_t m = r % M, bl = r / M;
    cplx s = cmake(0.0, 0.0);
    for (int k = 0; k < ksplit; ++k) s = cadd(s, part[(int64_t)k * total + idx]);
    cplx *dst = C + (bl + batch0) * sCb + m * sCm + n * sCn;
    cplx res = cmul(alpha, s);
    if (use_beta) res = cadd(res, cmul(beta, *dst));
    *dst = res;
  }
}
}  // namespace

namespace {
std::mutex g_dev_mu;
std::map<int, int> g_dev_sms;
std::set<std::tuple<const void *, int, int>> g_smem_set;
}  // namespace

int device_sm_count() {
  int dev = 0;
  ADC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_dev_mu);
  auto it = g_dev_sms.find(dev);
  if (it != g_dev_sms.end()) return it->second;
  int s = 0;
  ADC_CUDA(cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev));
  if (s <= 0) s = 148;
  g_dev_sms[dev] = s;
  return s;
}

void set_smem_limit(const void *kernel, int bytes) {
  int dev = 0;
  ADC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_dev_mu);
  const auto key = std::make_tuple(kernel, dev, bytes);
  if (g_smem_set.count(key)) return;
  ADC_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  g_smem_set.insert(key);
}

static void zgemm_attr() { set_smem_limit((const void *)k_zgemm, ZG_SMEM); }
static int num_sms() { return device_sm_count(); }

void zgemm(Exec &ex, int64_t M, int64_t N, int64_t K, int64_t batch, cplx alpha, const cplx *A,
           int64_t sAb, int64_t sAm, int64_t sAk, bool conjA, const cplx *B, int64_t sBb,
           int64_t sBk, int64_t sBn, bool conjB, cplx beta, cplx *C, int64_t sCb, int64_t sCm,
           int64_t sCn) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K < 0) K = 0;  // the kernel then writes beta * C
  // (short inner sizes stay here: there the product is bound by memory, and the
  // sliced form reads and writes several times more)
  if (ex.sliced_bits > 0 && K >= 512 && 8.0 * (double)M * N * K * batch >= (double)(1 << 24)) {
    ex.n_sliced += 1;
    ex.flops_sliced += 8.0 * (double)M * N * K * batch;
    zgemm_sliced(ex, M, N, K, batch, alpha, A, sAb, sAm, sAk, conjA, B, sBb, sBk, sBn, conjB, beta, C, sCb, sCm,
                 sCn);
    return;
  }
  ex.n_fp64 += 1;
  ex.flops_fp64 += 8.0 * (double)M * N * K * batch;
  zgemm_attr();
  const int64_t mt_ = (M + BM - 1) / BM, nt_ = (N + BN - 1) / BN;
  const int mfast = (nt_ <= 65535) ? 1 : 0;
  ADC_REQUIRE(mfast || mt_ <= 65535, ADC_ERR_UNSUPPORTED, "zgemm: shape too large");
  int a_kfast = (sAk == 1) ? 1 : 0;
  int b_nfast = (sBn == 1) ? 1 : 0;
  dim3 block(256);
  const int64_t tiles = ((N + BN - 1) / BN) * ((M + BM - 1) / BM);
  // split K when the output tiles alone cannot fill the GPU (down to chunks of
  // 16: on GB300's FP64 units a few CTAs over a short K still take far longer
  // than the partial sums cost), the partial buffer within 2^26 elements
  int ksplit = 1;
  const int64_t want = 2 * (int64_t)num_sms();
  if (tiles * batch < want && K >= 32) {
    int64_t s = (want + tiles * batch - 1) / (tiles * batch);
    s = std::min<int64_t>(s, (K + BKK - 1) / BKK);
    s = std::min<int64_t>(s, 256);
    s = std::min<int64_t>(s, std::max<int64_t>(1, ((int64_t)1 << 26) / std::max<int64_t>(1, M * N * batch)));
    ksplit = (int)std::max<int64_t>(1, s);
  }
  const int64_t bmax = 65535 / ksplit;
  int pr = ex.prof_begin("zgemm_fp64", 8.0 * (double)M * N * K * batch,
                         16.0 * (double)batch * ((double)M * K + (double)K * N + (double)M * N));
  for (int64_t b0 = 0; b0 < batch; b0 += bmax) {
    int64_t nb = std::min<int64_t>(bmax, batch - b0);
    dim3 grid(mfast ? (unsigned)mt_ : (unsigned)nt_, mfast ? (unsigned)nt_ : (unsigned)mt_, (unsigned)(nb * ksplit));
    if (ksplit == 1) {
      k_zgemm<<<grid, block, ZG_SMEM, ex.stream>>>(M, N, K, A, sAb, sAm, sAk, conjA ? 1 : 0, a_kfast, B,
                                             sBb, sBk, sBn, conjB ? 1 : 0, b_nfast, C, sCb, sCm,
                                             sCn, alpha, beta, b0, 1, K, nullptr, nb, mfast);
      ADC_CHECK_LAUNCH();
    } else {
      int64_t kchunk = (K + ksplit - 1) / ksplit;
      kchunk = (kchunk + BKK - 1) / BKK * BKK;
      DBuf part = cbuf(ex, (int64_t)ksplit * nb * M * N);
      k_zgemm<<<grid, block, ZG_SMEM, ex.stream>>>(M, N, K, A, sAb, sAm, sAk, conjA ? 1 : 0, a_kfast, B,
                                             sBb, sBk, sBn, conjB ? 1 : 0, b_nfast, C, sCb, sCm,
                                             sCn, alpha, beta, b0, ksplit, kchunk, part.c(), nb, mfast);
      ADC_CHECK_LAUNCH();
      k_splitk_reduce<<<grid1d(nb * M * N, 256), 256, 0, ex.stream>>>(
          part.c(), ksplit, nb, M, N, C, sCb, sCm, sCn, alpha, beta, b0);
      ADC_CHECK_LAUNCH();
    }
  }
  ex.prof_end(pr);
}

void zgemm_ws(Exec &ex, int64_t M, int64_t N, int64_t K, int64_t batch, cplx alpha, const cplx *A,
              int64_t sAb, int64_t sAm, int64_t sAk, bool conjA, const cplx *B, int64_t sBb, int64_t sBk,
              int64_t sBn, bool conjB, cplx beta, cplx *C, int64_t sCb, int64_t sCm, int64_t sCn, cplx *ws,
              int64_t ws_elems) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K < 0) K = 0;
  zgemm_attr();
  const int64_t mt_ = (M + BM - 1) / BM, nt_ = (N + BN - 1) / BN;
  const int mfast = (nt_ <= 65535) ? 1 : 0;
  ADC_REQUIRE(mfast || mt_ <= 65535, ADC_ERR_UNSUPPORTED, "zgemm: shape too large");
  int a_kfast = (sAk == 1) ? 1 : 0;
  int b_nfast = (sBn == 1) ? 1 : 0;
  dim3 block(256);
  const int64_t tiles = ((N + BN - 1) / BN) * ((M + BM - 1) / BM);
  // same split-K choice as zgemm, capped by the workspace the caller provides
  int ksplit = 1;
  const int64_t want = 2 * (int64_t)num_sms();
  if (tiles * batch < want && K > 2048) {
    int64_t s = (want + tiles * batch - 1) / (tiles * batch);
    s = std::min<int64_t>(s, K / 1024);
    s = std::min<int64_t>(s, 256);
    ksplit = (int)std::max<int64_t>(1, s);
  }
  const int64_t bmax = 65535 / ksplit;
  for (int64_t b0 = 0; b0 < batch; b0 += bmax) {
    int64_t nb = std::min<int64_t>(bmax, batch - b0);
    int ks = ksplit;
    if (ks > 1 && ws) ks = (int)std::max<int64_t>(1, std::min<int64_t>(ks, ws_elems / std::max<int64_t>(1, nb * M * N)));
    if (!ws) ks = 1;
    dim3 grid(mfast ? (unsigned)mt_ : (unsigned)nt_, mfast ? (unsigned)nt_ : (unsigned)mt_, (unsigned)(nb * ks));
    if (ks == 1) {
      k_zgemm<<<grid, block, ZG_SMEM, ex.stream>>>(M, N, K, A, sAb, sAm, sAk, conjA ? 1 : 0, a_kfast, B, sBb, sBk, sBn,
                                             conjB ? 1 : 0, b_nfast, C, sCb, sCm, sCn, alpha, beta, b0, 1, K,
                                             nullptr, nb, mfast);
      ADC_CHECK_LAUNCH();
    } else {
      int64_t kchunk = (K + ks - 1) / ks;
      kchunk = (kchunk + BKK - 1) / BKK * BKK;
      k_zgemm<<<grid, block, ZG_SMEM, ex.stream>>>(M, N, K, A, sAb, sAm, sAk, conjA ? 1 : 0, a_kfast, B, sBb, sBk, sBn,
                                             conjB ? 1 : 0, b_nfast, C, sCb, sCm, sCn, alpha, beta, b0, ks, kchunk,
                                             ws, nb, mfast);
      ADC_CHECK_LAUNCH();
      k_splitk_reduce<<<grid1d(nb * M * N, 256), 256, 0, ex.stream>>>(ws, ks, nb, M, N, C, sCb, sCm, sCn, alpha,
                                                                      beta, b0);
      ADC_CHECK_LAUNCH();
    }
  }
}

// ------------------------------------------------------------------ permute
namespace {
constexpr int MAXD = 8;
struct PermArgs {
  int nd;
  int strided_dst;  // 0: dst contiguous in ext order; 1: dst at strides dstr
  int64_t ext[MAXD];
  int64_t sstr[MAXD];
  int64_t dstr[MAXD];
};

__global__ void k_permute(const cplx *__restrict__ src, PermArgs pa, int conj, cplx *dst,
                          cplx alpha, cplx beta, int use_beta, int64_t total) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = idx, off = 0, doff = 0;
    for (int d = pa.nd - 1; d >= 0; --d) {
      int64_t i = rem % pa.ext[d];
      rem /= pa.ext[d];
      off += i * pa.sstr[d];
      doff += i * pa.dstr[d];
    }
    if (!pa.strided_dst) doff = idx;
    cplx v = src[off];
    if (conj) v.y = -v.y;
    cplx r = cmul(alpha, v);
    if (use_beta) r = cadd(r, cmul(beta, dst[doff]));
    dst[doff] = r;
  }
}
}  // namespace

void permute(Exec &ex, const cplx *src, const std::vector<int64_t> &ext, const std::vector<int64_t> &sstr,
             bool conj, cplx *dst, const std::vector<int64_t> &dstr, cplx alpha, cplx beta) {
  PermArgs pa{};
  ADC_REQUIRE(ext.size() <= (size_t)MAXD && ext.size() == sstr.size() && ext.size() == dstr.size(), ADC_ERR_ARG,
              "permute: rank");
  pa.nd = (int)ext.size();
  pa.strided_dst = 1;
  int64_t total = 1;
  for (int d = 0; d < pa.nd; ++d) {
    pa.ext[d] = ext[d];
    pa.sstr[d] = sstr[d];
    pa.dstr[d] = dstr[d];
    total *= ext[d];
  }
  if (total == 0) return;
  const int use_beta = (beta.x != 0.0 || beta.y != 0.0) ? 1 : 0;
  k_permute<<<grid1d(total, 256), 256, 0, ex.stream>>>(src, pa, conj ? 1 : 0, dst, alpha, beta, use_beta, total);
  ADC_CHECK_LAUNCH();
}

void permute(Exec &ex, const cplx *src, const std::vector<int64_t> &ext,
             const std::vector<int64_t> &sstr, bool conj, cplx *dst, cplx alpha, cplx beta) {
  PermArgs pa{};
  ADC_REQUIRE(ext.size() <= (size_t)MAXD && ext.size() == sstr.size(), ADC_ERR_ARG, "permute: rank");
  pa.nd = (int)ext.size();
  int64_t total = 1;
  for (int d = 0; d < pa.nd; ++d) { pa.ext[d] = ext[d]; pa.sstr[d] = sstr[d]; total *= ext[d]; }
  if (pa.nd == 0) { pa.nd = 1; pa.ext[0] = 1; pa.sstr[0] = 0; }
  if (total == 0) return;
  int use_beta = (beta.x != 0.0 || beta.y != 0.0) ? 1 : 0;
  k_permute<<<grid1d(total, 256), 256, 0, ex.stream>>>(src, pa, conj ? 1 : 0, dst, alpha, beta,
                                                       use_beta, total);
  ADC_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ pairs
namespace {
__global__ void k_pair_unpack(const cplx *__restrict__ P, int64_t no1, int64_t no0, int64_t sP1,
                              int64_t sP0, int64_t n, int64_t inner, cplx *T, int64_t total) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t in = idx % inner;
    int64_t r = idx / inner;
    int64_t q = r % n; r /= n;
    int64_t p = r % n; r /= n;
    int64_t o0 = r % no0, o1 = r / no0;
    cplx v = cmake(0.0, 0.0);
    if (p < q) v = P[o1 * sP1 + o0 * sP0 + pair_index(p, q, n) * inner + in];
    else if (p > q) { v = P[o1 * sP1 + o0 * sP0 + pair_index(q, p, n) * inner + in]; v.x = -v.x; v.y = -v.y; }
    T[idx] = v;
  }
}

__global__ void k_pair_pack(const cplx *__restrict__ T, int64_t sTo1, int64_t sTo0, int64_t sTp,
                            int64_t sTq, int64_t sTin, double s, int64_t no1, int64_t no0,
                            int64_t n, int64_t inner, cplx *P, int64_t sP1, int64_t sP0,
                            cplx alpha, cplx beta, int use_beta, int64_t total) {
  // iterate over (o, p, q, in) with p < q encoded through the full square; half idle
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t in = idx % inner;
    int64_t r = idx / inner;
    int64_t q = r % n; r /= n;
    int64_t p = r % n; r /= n;
    if (p >= q) continue;
    int64_t o0 = r % no0, o1 = r / no0;
    const cplx *Tb = T + o1 * sTo1 + o0 * sTo0 + in * sTin;
    cplx v = Tb[p * sTp + q * sTq];
    if (s != 0.0) { cplx w = Tb[q * sTp + p * sTq]; v.x -= s * w.x; v.y -= s * w.y; }
    cplx *dst = P + o1 * sP1 + o0 * sP0 + pair_index(p, q, n) * inner + in;
    cplx res = cmul(alpha, v);
    if (use_beta) res = cadd(res, cmul(beta, *dst));
    *dst = res;
  }
}
}  // namespace

void pair_unpack(Exec &ex, const cplx *P, int64_t no1, int64_t no0, int64_t sP1, int64_t sP0,
                 int64_t n, int64_t inner, cplx *T) {
  int64_t total = no1 * no0 * n * n * inner;
  if (total == 0) return;
  k_pair_unpack<<<grid1d(total, 256), 256, 0, ex.stream>>>(P, no1, no0, sP1, sP0, n, inner, T, total);
  ADC_CHECK_LAUNCH();
}

void pair_pack(Exec &ex, const cplx *T, int64_t sTo1, int64_t sTo0, int64_t sTp, int64_t sTq,
               int64_t sTin, double s, int64_t no1, int64_t no0, int64_t n, int64_t inner,
               cplx *P, int64_t sP1, int64_t sP0, cplx alpha, cplx beta) {
  int64_t total = no1 * no0 * n * n * inner;
  if (total == 0 || n < 2) return;
  int use_beta = (beta.x != 0.0 || beta.y != 0.0) ? 1 : 0;
  k_pair_pack<<<grid1d(total, 256), 256, 0, ex.stream>>>(T, sTo1, sTo0, sTp, sTq, sTin, s, no1,
                                                         no0, n, inner, P, sP1, sP0, alpha, beta,
                                                         use_beta, total);
  ADC_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ elementwise
namespace {
__global__ void k_denom2(cplx *t, const double *eo, const double *ev, int64_t o, int64_t v,
                         int64_t total) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = idx % v, r = idx / v;
    int64_t a = r % v; r /= v;
    int64_t j = r % o, i = r / o;
    double D = eo[i] + eo[j] - ev[a] - ev[b];
    cplx x = t[idx];
    t[idx] = cmake(x.x / D, x.y / D);
  }
}
__global__ void k_denom1(cplx *t, const double *eo, const double *ev, int64_t o, int64_t v) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= o * v) return;
  int64_t a = idx % v, i = idx / v;
  double D = eo[i] - ev[a];
  cplx x = t[idx];
  t[idx] = cmake(x.x / D, x.y / D);
}
__global__ void k_oovv_from_t1(const cplx *t, const double *eo, const double *ev, int64_t o,
                               int64_t v, cplx *dst, int64_t total) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = idx % v, r = idx / v;
    int64_t a = r % v; r /= v;
    int64_t j = r % o, i = r / o;
    double D = eo[i] + eo[j] - ev[a] - ev[b];
    cplx x = t[idx];
    dst[idx] = cmake(D * x.x, -D * x.y);
  }
}
__global__ void k_eps_diff_T(cplx *M, const cplx *G, const double *e, int64_t n, double s) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  int64_t q = idx % n, p = idx / n;
  double f = s * (e[p] - e[q]);
  cplx g = G[q * n + p];
  M[idx].x += f * g.x;
  M[idx].y += f * g.y;
}
__global__ void k_add_diag(cplx *M, const double *e, int64_t n, double s) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < n) M[p * n + p].x += s * e[p];
}
__global__ void k_antisym_diag(const cplx *B, int64_t Q, int64_t nmo, double *g) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nmo * nmo) return;
  int64_t q = idx % nmo, p = idx / nmo;
  double acc = 0.0;
  for (int64_t Qi = 0; Qi < Q; ++Qi) {
    const cplx *Bq = B + Qi * nmo * nmo;
    cplx pp = Bq[p * nmo + p], qq = Bq[q * nmo + q], pq = Bq[p * nmo + q], qp = Bq[q * nmo + p];
    acc += (pp.x * qq.x - pp.y * qq.y) - (pq.x * qp.x - pq.y * qp.y);
  }
  g[idx] = acc;
}
__global__ void k_zaxpby(int64_t n, cplx a, const cplx *x, cplx b, cplx *y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = cadd(cmul(a, x[i]), cmul(b, y[i]));
}
__global__ void k_diag_mul_add(int64_t k, int64_t n, const double *d, const cplx *x, int64_t ldx,
                               cplx *y, int64_t ldy, double s) {
  int64_t total = k * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = idx % n, r = idx / n;
    double f = s * d[i];
    cplx xv = x[r * ldx + i];
    cplx &yv = y[r * ldy + i];
    yv.x += f * xv.x;
    yv.y += f * xv.y;
  }
}
}  // namespace

void denom2_div(Exec &ex, cplx *t, const double *eo, const double *ev, int64_t o, int64_t v) {
  int64_t total = o * o * v * v;
  if (!total) return;
  k_denom2<<<grid1d(total, 256), 256, 0, ex.stream>>>(t, eo, ev, o, v, total);
  ADC_CHECK_LAUNCH();
}
void denom1_div(Exec &ex, cplx *t, const double *eo, const double *ev, int64_t o, int64_t v) {
  if (!o || !v) return;
  k_denom1<<<grid1d(o * v, 256), 256, 0, ex.stream>>>(t, eo, ev, o, v);
  ADC_CHECK_LAUNCH();
}
void oovv_from_t1(Exec &ex, const cplx *t, const double *eo, const double *ev, int64_t o,
                  int64_t v, cplx *dst) {
  int64_t total = o * o * v * v;
  if (!total) return;
  k_oovv_from_t1<<<grid1d(total, 256), 256, 0, ex.stream>>>(t, eo, ev, o, v, dst, total);
  ADC_CHECK_LAUNCH();
}
void add_eps_diff_transpose(Exec &ex, cplx *M, const cplx *G, const double *e, int64_t n, double s) {
  if (!n) return;
  k_eps_diff_T<<<grid1d(n * n, 256), 256, 0, ex.stream>>>(M, G, e, n, s);
  ADC_CHECK_LAUNCH();
}
void add_diag(Exec &ex, cplx *M, const double *e, int64_t n, double s) {
  if (!n) return;
  k_add_diag<<<grid1d(n, 256), 256, 0, ex.stream>>>(M, e, n, s);
  ADC_CHECK_LAUNCH();
}
void antisym_diag(Exec &ex, const cplx *B, int64_t Q, int64_t nmo, double *g) {
  k_antisym_diag<<<grid1d(nmo * nmo, 256), 256, 0, ex.stream>>>(B, Q, nmo, g);
  ADC_CHECK_LAUNCH();
}
void zaxpby(Exec &ex, int64_t n, cplx a, const cplx *x, cplx b, cplx *y) {
  if (!n) return;
  k_zaxpby<<<grid1d(n, 256), 256, 0, ex.stream>>>(n, a, x, b, y);
  ADC_CHECK_LAUNCH();
}
void diag_mul_add(Exec &ex, int64_t k, int64_t n, const double *d, const cplx *x, int64_t ldx,
                  cplx *y, int64_t ldy, double s) {
  if (!k || !n) return;
  k_diag_mul_add<<<grid1d(k * n, 256), 256, 0, ex.stream>>>(k, n, d, x, ldx, y, ldy, s);
  ADC_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ einsum
namespace {
struct Group {
  std::vector<char> labels;
};

// can the labels (in order) of tensor t be merged into one index with a
// uniform stride? Returns the stride of the merged index (0 if empty).
bool mergeable(const TV &t, const std::string &lab, const std::vector<char> &grp, int64_t &stride,
               int64_t &extent) {
  std::vector<std::pair<int64_t, int64_t>> es;  // (ext, str) for ext > 1
  extent = 1;
  for (char c : grp) {
    size_t pos = lab.find(c);
    int64_t e = t.ext[pos];
    extent *= e;
    if (e > 1) es.push_back({e, t.str[pos]});
  }
  if (es.empty()) { stride = 0; return true; }
  for (size_t i = 0; i + 1 < es.size(); ++i)
    if (es[i].second != es[i + 1].second * es[i + 1].first) return false;
  stride = es.back().second;
  return true;
}

// dense copy of t arranged in the concatenated label order `order`
void to_dense(Exec &ex, const TV &t, const std::string &lab, const std::vector<char> &order,
              cplx *dst) {
  std::vector<int64_t> e, s;
  for (char c : order) {
    size_t pos = lab.find(c);
    e.push_back(t.ext[pos]);
    s.push_back(t.str[pos]);
  }
  permute(ex, t.p, e, s, false, dst, C1(), C0());
}
}  // namespace

void einsum(Exec &ex, cplx alpha, const TV &A, const char *la_, const TV &B, const char *lb_,
            cplx beta, const TV &C, const char *lc_) {
  std::string la(la_), lb(lb_), lc(lc_);
  ADC_REQUIRE(la.size() == A.ext.size() && lb.size() == B.ext.size() && lc.size() == C.ext.size(),
              ADC_ERR_ARG, "einsum: label/rank mismatch " + la + "," + lb + "->" + lc);
  std::map<char, int64_t> ext;
  auto reg = [&](const std::string &l, const TV &t) {
    for (size_t i = 0; i < l.size(); ++i) {
      auto it = ext.find(l[i]);
      if (it != ext.end())
        ADC_REQUIRE(it->second == t.ext[i], ADC_ERR_ARG, std::string("einsum: extent of ") + l[i]);
      else
        ext[l[i]] = t.ext[i];
    }
  };
  reg(la, A); reg(lb, B); reg(lc, C);
  std::vector<char> gb, gm, gn, gk;
  for (char c : lc) {
    bool inA = la.find(c) != std::string::npos, inB = lb.find(c) != std::string::npos;
    ADC_REQUIRE(inA || inB, ADC_ERR_ARG, "einsum: output label not in inputs");
    if (inA && inB) gb.push_back(c);
    else if (inA) gm.push_back(c);
    else gn.push_back(c);
  }
  for (char c : la) {
    bool inB = lb.find(c) != std::string::npos, inC = lc.find(c) != std::string::npos;
    if (!inC) {
      ADC_REQUIRE(inB, ADC_ERR_UNSUPPORTED, "einsum: trace index");
      gk.push_back(c);
    }
  }
  for (char c : lb)
    ADC_REQUIRE(la.find(c) != std::string::npos || lc.find(c) != std::string::npos,
                ADC_ERR_UNSUPPORTED, "einsum: trace index in B");
  int64_t nb = 1, nm = 1, nn = 1, nk = 1;
  for (char c : gb) nb *= ext[c];
  for (char c : gm) nm *= ext[c];
  for (char c : gn) nn *= ext[c];
  for (char c : gk) nk *= ext[c];
  if (nb == 0 || nm == 0 || nn == 0) return;

  // A as [b][m][k]
  int64_t sAb, sAm, sAk, e_;
  DBuf Abuf, Bbuf, Cbuf;
  const cplx *Ap = A.p;
  if (!(mergeable(A, la, gb, sAb, e_) && mergeable(A, la, gm, sAm, e_) && mergeable(A, la, gk, sAk, e_))) {
    std::vector<char> ord(gb);
    ord.insert(ord.end(), gm.begin(), gm.end());
    ord.insert(ord.end(), gk.begin(), gk.end());
    Abuf = cbuf(ex, nb * nm * nk);
    to_dense(ex, A, la, ord, Abuf.c());
    Ap = Abuf.c();
    sAb = nm * nk; sAm = nk; sAk = 1;
  }
  int64_t sBb, sBk, sBn;
  const cplx *Bp = B.p;
  if (!(mergeable(B, lb, gb, sBb, e_) && mergeable(B, lb, gk, sBk, e_) && mergeable(B, lb, gn, sBn, e_))) {
    std::vector<char> ord(gb);
    ord.insert(ord.end(), gk.begin(), gk.end());
    ord.insert(ord.end(), gn.begin(), gn.end());
    Bbuf = cbuf(ex, nb * nk * nn);
    to_dense(ex, B, lb, ord, Bbuf.c());
    Bp = Bbuf.c();
    sBb = nk * nn; sBk = nn; sBn = 1;
  }
  int64_t sCb, sCm, sCn;
  if (mergeable(C, lc, gb, sCb, e_) && mergeable(C, lc, gm, sCm, e_) && mergeable(C, lc, gn, sCn, e_)) {
    zgemm(ex, nm, nn, nk, nb, alpha, Ap, sAb, sAm, sAk, A.conj, Bp, sBb, sBk, sBn, B.conj, beta,
          C.p, sCb, sCm, sCn);
    return;
  }
  // compute into a dense [b][m][n] buffer, then scatter into C with beta
  Cbuf = cbuf(ex, nb * nm * nn);
  zgemm(ex, nm, nn, nk, nb, alpha, Ap, sAb, sAm, sAk, A.conj, Bp, sBb, sBk, sBn, B.conj, C0(),
        Cbuf.c(), nm * nn, nn, 1);
  // C[lc] = Cbuf[perm] + beta*C: iterate C in its own label order (contiguous target
  // required for the permute kernel), so build strides of Cbuf per C label.
  std::vector<char> ord(gb);
  ord.insert(ord.end(), gm.begin(), gm.end());
  ord.insert(ord.end(), gn.begin(), gn.end());
  std::vector<int64_t> bstr(ord.size());
  {
    int64_t acc = 1;
    for (int i = (int)ord.size() - 1; i >= 0; --i) { bstr[i] = acc; acc *= ext[ord[i]]; }
  }
  // C must be contiguous for the scatter; check
  TV Cd = TV::dense(C.p, C.ext);
  ADC_REQUIRE(Cd.str == C.str, ADC_ERR_UNSUPPORTED, "einsum: non-contiguous output needs a permute");
  std::vector<int64_t> e, s;
  for (char c : lc) {
    auto it = std::find(ord.begin(), ord.end(), c);
    e.push_back(ext[c]);
    s.push_back(bstr[it - ord.begin()]);
  }
  permute(ex, Cbuf.c(), e, s, false, C.p, C1(), beta);
}

}  // namespace adc
