// Split-precision complex GEMM on the Blackwell tensor cores (tcgen05).
//
// out[m][n] = alpha * sum_k A[m][k] * B[n][k] + beta * out[m][n]   (complex)
//
// Both operands are K-major. Each complex FP64 operand is stored once in the
// "real embedding" used by the MMA: an A row is [Re A | Im A] and a B row n
// becomes two rows, [Re B | -Im B] and [Im B | Re B], so one real GEMM of
// inner size 2K yields Re and Im of the complex product side by side (four
// real multiplications per complex one). Every embedded value x is split into
// two BF16 numbers, hi = bf16(x) and lo = bf16(x - hi), and the product is
// accumulated in FP32 as hi*hi + hi*lo + lo*hi (three K segments of one MMA
// chain). This keeps about 16 significant bits per operand.
//
// Kernel: one 128 x BN output tile per CTA (cta_group::1), BK = 64 BF16
// (one 128-byte swizzle atom). Warp 0 issues TMA loads (128B swizzle) into a
// ring of shared-memory stages guarded by mbarriers, warp 1 issues
// tcgen05.mma into a TMEM accumulator and commits each stage back to the
// producer, warps 2-5 read the accumulator with tcgen05.ld and write the
// complex128 result. Every wait is bounded (about two seconds of
// %globaltimer); a wait that gives up records an error code, the CTA drains
// its own copies in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "ctx.cuh"
#include "tc_gemm.cuh"

namespace adc {

namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;
constexpr uint64_t WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; false when it gave up or another role aborted
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int *abort_flag) {
  uint64_t t0 = gtimer();
  while (!mbar_try(a, parity)) {
    if (*abort_flag) return false;
    if (gtimer() - t0 > WAIT_NS) return false;
  }
  return true;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (SBO), descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}
// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      ::"r"(tmem_d), "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
      "[%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
        "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
        "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
        "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int BN, int ST>
struct TcLayout {
  static constexpr int A_BYTES = TC_BM * TC_BK * 2;
  static constexpr int B_BYTES = BN * TC_BK * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int BAR_OFF = ST * STAGE;
  static constexpr int SMEM = 1024 + BAR_OFF + 256;  // 1024 for the manual alignment
  static constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
};

template <int BN, int ST>
__global__ void __launch_bounds__(192, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
          const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, int M,
          int N2, int kps, int kb_per_split, cplx *out, int64_t s_m, int64_t s_nh, int64_t s_nl,
          int64_t n_in, cplx alpha, cplx beta, float *part, int *err) {
  using L = TcLayout<BN, ST>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(smem + L::BAR_OFF);
  uint64_t *empty = full + ST;
  uint64_t *accum = empty + ST;
  uint32_t *tmem_slot = (uint32_t *)(accum + 1);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * BN;
  const int split = blockIdx.z;
  const int total_kb = 3 * kps;
  const int kb_beg = split * kb_per_split;
  const int kb_end = min(total_kb, kb_beg + kb_per_split);
  const int nkb = kb_end - kb_beg;

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(accum), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(L::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- producer
    int issued = 0;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % ST, r = i / ST;
      if (r > 0 && !mbar_wait(smem_u32(&empty[s]), (r - 1) & 1, abort_flag)) {
        if (!*abort_flag) atomicExch(err, 1);
        *abort_flag = 1;
        break;
      }
      const int g = kb_beg + i;
      const int seg = g / kps;
      const int kx = (g - seg * kps) * TC_BK;
      const uint32_t fb = smem_u32(&full[s]);
      mbar_expect_tx(fb, L::STAGE);
      uint8_t *sa = smem + s * L::STAGE;
      tma_load_2d(smem_u32(sa), seg == 2 ? &mAl : &mAh, kx, m0, fb);
      tma_load_2d(smem_u32(sa + L::A_BYTES), seg == 1 ? &mBl : &mBh, kx, n0, fb);
      issued = i + 1;
    }
    if (*abort_flag) {
      // drain this CTA's copies in flight before shared memory is released
      for (int j = (issued > ST ? issued - ST : 0); j < issued; ++j) {
        const int s = j % ST, r = j / ST;
        uint64_t t0 = gtimer();
        while (!mbar_try(smem_u32(&full[s]), r & 1) && gtimer() - t0 < WAIT_NS) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = idesc_bf16(TC_BM, BN);
    for (int i = 0; i < nkb; ++i) {
      const int s = i % ST, r = i / ST;
      if (!mbar_wait(smem_u32(&full[s]), r & 1, abort_flag)) {
        if (!*abort_flag) atomicExch(err, 2);
        *abort_flag = 1;
        break;
      }
      fence_after();
      const uint32_t a0 = smem_u32(smem + s * L::STAGE);
      const uint32_t b0 = a0 + L::A_BYTES;
#pragma unroll
      for (int k = 0; k < TC_BK / 16; ++k)
        mma_bf16(tmem, sdesc(a0 + 32 * k), sdesc(b0 + 32 * k), idesc, (i > 0 || k > 0) ? 1u : 0u);
      mma_commit(smem_u32(&empty[s]));
    }
    mma_commit(smem_u32(accum));
  } else if (warp >= 2) {
    // ---------------- epilogue: TMEM -> registers -> complex128
    bool ok = mbar_wait(smem_u32(accum), 0, abort_flag);
    if (!ok && !*abort_flag) { atomicExch(err, 3); *abort_flag = 1; }
    fence_after();
    __syncwarp();
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const int64_t m = (int64_t)m0 + row;
    const bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
#pragma unroll 1
    for (int cch = 0; cch < BN / 32; ++cch) {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(cch * 32), v);
      if (!ok || *abort_flag || m >= M || nkb <= 0) continue;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int64_t n2 = (int64_t)n0 + cch * 32 + 2 * j;
        if (n2 >= N2) break;
        const float re = __uint_as_float(v[2 * j]), im = __uint_as_float(v[2 * j + 1]);
        if (part) {
          float *pp = part + ((int64_t)split * M + m) * N2 + n2;
          pp[0] = re;
          pp[1] = im;
        } else {
          const int64_t n = n2 >> 1;
          const int64_t nh = n / n_in, nl = n - nh * n_in;
          cplx *dst = out + m * s_m + nh * s_nh + nl * s_nl;
          cplx val = cmul(alpha, cmake((double)re, (double)im));
          if (use_beta) val = cadd(val, cmul(beta, *dst));
          *dst = val;
        }
      }
    }
    fence_before();
  }
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L::TMEM_COLS)
                 : "memory");
  }
}

__global__ void k_tc_reduce(const float *__restrict__ part, int ksplit, int64_t M, int64_t N2, cplx *out,
                            int64_t s_m, int64_t s_nh, int64_t s_nl, int64_t n_in, cplx alpha, cplx beta) {
  const int64_t total = M * (N2 / 2);
  const bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = idx % (N2 / 2), m = idx / (N2 / 2);
    double re = 0.0, im = 0.0;
    for (int s = 0; s < ksplit; ++s) {
      const float *pp = part + ((int64_t)s * M + m) * N2 + 2 * n;
      re += (double)pp[0];
      im += (double)pp[1];
    }
    const int64_t nh = n / n_in, nl = n - nh * n_in;
    cplx *dst = out + m * s_m + nh * s_nh + nl * s_nl;
    cplx val = cmul(alpha, cmake(re, im));
    if (use_beta) val = cadd(val, cmul(beta, *dst));
    *dst = val;
  }
}

// ---------------------------------------------------------------- operand packing
__device__ __forceinline__ void split_store(double x, __nv_bfloat16 *hi, __nv_bfloat16 *lo) {
  __nv_bfloat16 h = __double2bfloat16(x);
  *hi = h;
  *lo = __double2bfloat16(x - (double)__bfloat162float(h));
}

// A rows: [Re | Im] (conj negates Im); element (m, k) at src[m*s_m + k*s_k]
__global__ void k_emb_A(const cplx *__restrict__ src, int64_t M, int64_t K, int64_t s_m, int64_t s_k,
                        int conj, int64_t kp, __nv_bfloat16 *hi, __nv_bfloat16 *lo) {
  const int64_t total = M * kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = idx % kp, m = idx / kp;
    cplx x = cmake(0.0, 0.0);
    if (k < K) x = src[m * s_m + k * s_k];
    const double im = conj ? -x.y : x.y;
    const int64_t base = m * 2 * kp;
    split_store(x.x, hi + base + k, lo + base + k);
    split_store(im, hi + base + kp + k, lo + base + kp + k);
  }
}

// value of B[n][k] for the three gather patterns
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
};

// B rows: row 2n = [Re | -Im], row 2n+1 = [Im | Re] (conj negates Im first)
__global__ void k_emb_B(BSrc src, int64_t Nc, int64_t K, int conj, int64_t kp, __nv_bfloat16 *hi,
                        __nv_bfloat16 *lo) {
  const int64_t total = Nc * kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = idx % kp, n = idx / kp;
    cplx x = cmake(0.0, 0.0);
    if (k < K) x = src.get(n, k);
    const double im = conj ? -x.y : x.y;
    const int64_t r0 = (2 * n) * 2 * kp, r1 = (2 * n + 1) * 2 * kp;
    split_store(x.x, hi + r0 + k, lo + r0 + k);
    split_store(-im, hi + r0 + kp + k, lo + r0 + kp + k);
    split_store(im, hi + r1 + k, lo + r1 + k);
    split_store(x.x, hi + r1 + kp + k, lo + r1 + kp + k);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

void make_map(CUtensorMap *map, const void *base, int64_t rows, int64_t kp2, int box_rows) {
  if (!g_encode) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    ADC_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    ADC_REQUIRE(fn && q == cudaDriverEntryPointSuccess, ADC_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  ADC_REQUIRE(((uintptr_t)base & 15) == 0 && (kp2 * 2) % 16 == 0, ADC_ERR_ARG, "TMA alignment");
  cuuint64_t dims[2] = {(cuuint64_t)kp2, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(kp2 * 2)};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  ADC_REQUIRE(r == CUDA_SUCCESS, ADC_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
}

int g_sms = 0;

template <int BN, int ST>
void launch_tc(Exec &ex, const TcMat &A, const TcMat &B, int64_t M, int64_t N2, cplx alpha, cplx beta,
               cplx *out, int64_t s_m, int64_t s_nh, int64_t s_nl, int64_t n_in, int *err) {
  using L = TcLayout<BN, ST>;
  static bool attr = false;
  if (!attr) {
    ADC_CUDA(cudaFuncSetAttribute(k_tc_gemm<BN, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM));
    attr = true;
  }
  if (!g_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 148;
  }
  CUtensorMap mAh, mAl, mBh, mBl;
  const int64_t kp2 = 2 * A.kp;
  make_map(&mAh, A.hi.p, A.rows, kp2, TC_BM);
  make_map(&mAl, A.lo.p, A.rows, kp2, TC_BM);
  make_map(&mBh, B.hi.p, B.rows, kp2, BN);
  make_map(&mBl, B.lo.p, B.rows, kp2, BN);
  const int kps = (int)(kp2 / TC_BK);
  const int total_kb = 3 * kps;
  const int64_t tiles = ((N2 + BN - 1) / BN) * ((M + TC_BM - 1) / TC_BM);
  int ksplit = 1;
  if (tiles < g_sms) {
    int64_t s = (g_sms + tiles - 1) / tiles;
    s = std::min<int64_t>(s, std::max(1, total_kb / 8));
    ksplit = (int)std::max<int64_t>(1, s);
  }
  int kb_per_split = (total_kb + ksplit - 1) / ksplit;
  ksplit = (total_kb + kb_per_split - 1) / kb_per_split;
  ADC_REQUIRE((M + TC_BM - 1) / TC_BM <= 65535 && ksplit <= 65535, ADC_ERR_UNSUPPORTED, "tc_gemm grid");
  dim3 grid((unsigned)((N2 + BN - 1) / BN), (unsigned)((M + TC_BM - 1) / TC_BM), (unsigned)ksplit);
  DBuf part;
  if (ksplit > 1) part = DBuf(ex, (size_t)ksplit * M * N2 * sizeof(float));
  const int64_t Kc = A.kreal > 0 ? A.kreal : A.kp;
  int pr = ex.prof_begin("tc_gemm_bf16x3", 8.0 * (double)M * (double)(N2 / 2) * (double)Kc);
  k_tc_gemm<BN, ST><<<grid, 192, L::SMEM, ex.stream>>>(mAh, mAl, mBh, mBl, (int)M, (int)N2, kps, kb_per_split,
                                                      out, s_m, s_nh, s_nl, n_in, alpha, beta,
                                                      ksplit > 1 ? (float *)part.p : nullptr, err);
  ADC_CHECK_LAUNCH();
  if (ksplit > 1) {
    k_tc_reduce<<<grid1d(M * (N2 / 2), 256), 256, 0, ex.stream>>>((const float *)part.p, ksplit, M, N2, out, s_m,
                                                                  s_nh, s_nl, n_in, alpha, beta);
    ADC_CHECK_LAUNCH();
  }
  ex.prof_end(pr);
}

}  // namespace

void tc_pack_A(Exec &ex, TcMat &dst, const cplx *src, int64_t M, int64_t K, int64_t s_m, int64_t s_k, bool conj) {
  dst.rows = M;
  dst.kreal = K;
  dst.kp = (K + TC_BK - 1) / TC_BK * TC_BK;
  if (dst.kp == 0) dst.kp = TC_BK;
  const size_t bytes = (size_t)M * 2 * dst.kp * sizeof(__nv_bfloat16);
  if (dst.hi.bytes < bytes) {
    dst.hi.reset(); dst.lo.reset();
    dst.hi = DBuf(ex, bytes);
    dst.lo = DBuf(ex, bytes);
  }
  k_emb_A<<<grid1d(M * dst.kp, 256), 256, 0, ex.stream>>>(src, M, K, s_m, s_k, conj ? 1 : 0, dst.kp,
                                                          (__nv_bfloat16 *)dst.hi.p, (__nv_bfloat16 *)dst.lo.p);
  ADC_CHECK_LAUNCH();
}

static void pack_B_impl(Exec &ex, TcMat &dst, const BSrc &s, int64_t Nc, int64_t K, bool conj) {
  dst.rows = 2 * Nc;
  dst.kreal = K;
  dst.kp = (K + TC_BK - 1) / TC_BK * TC_BK;
  if (dst.kp == 0) dst.kp = TC_BK;
  const size_t bytes = (size_t)dst.rows * 2 * dst.kp * sizeof(__nv_bfloat16);
  if (dst.hi.bytes < bytes) {
    dst.hi.reset(); dst.lo.reset();
    dst.hi = DBuf(ex, bytes);
    dst.lo = DBuf(ex, bytes);
  }
  k_emb_B<<<grid1d(Nc * dst.kp, 256), 256, 0, ex.stream>>>(s, Nc, K, conj ? 1 : 0, dst.kp,
                                                           (__nv_bfloat16 *)dst.hi.p, (__nv_bfloat16 *)dst.lo.p);
  ADC_CHECK_LAUNCH();
}

void tc_pack_B(Exec &ex, TcMat &dst, const cplx *src, int64_t Nc, int64_t K, int64_t s_nh, int64_t s_nl,
               int64_t n_in, int64_t s_k, bool conj) {
  BSrc s{src, 0, s_nh, s_nl, n_in, s_k, 0, 0, 0, 0};
  pack_B_impl(ex, dst, s, Nc, K, conj);
}

void tc_pack_B_ring(Exec &ex, TcMat &dst, const adc_ctx *c, const cplx *X, int64_t k) {
  BSrc s{X, c->kind == ADC_EA ? 1 : 2, 0, 0, 1, 0, c->o, c->v, c->N, c->n1};
  const int64_t Nc = (c->kind == ADC_EA) ? k * c->v : k * c->o;
  pack_B_impl(ex, dst, s, Nc, c->o * c->v, false);
}

void tc_gemm(Exec &ex, const TcMat &A, const TcMat &B, int64_t M, int64_t N, cplx alpha, cplx beta, cplx *out,
             int64_t s_m, int64_t s_nh, int64_t s_nl, int64_t n_in, int *err) {
  ADC_REQUIRE(A.kp == B.kp, ADC_ERR_ARG, "tc_gemm: inner sizes differ");
  ADC_REQUIRE(A.rows >= M && B.rows >= 2 * N, ADC_ERR_ARG, "tc_gemm: operand rows");
  if (M <= 0 || N <= 0) return;
  ADC_REQUIRE(M < (1ll << 31) && 2 * N < (1ll << 31), ADC_ERR_UNSUPPORTED, "tc_gemm: size");
  if (n_in <= 0) n_in = 1;
  const int64_t N2 = 2 * N;
  if (N2 <= 32) launch_tc<32, 8>(ex, A, B, M, N2, alpha, beta, out, s_m, s_nh, s_nl, n_in, err);
  else if (N2 <= 64) launch_tc<64, 8>(ex, A, B, M, N2, alpha, beta, out, s_m, s_nh, s_nl, n_in, err);
  else if (N2 <= 128) launch_tc<128, 6>(ex, A, B, M, N2, alpha, beta, out, s_m, s_nh, s_nl, n_in, err);
  else launch_tc<256, 4>(ex, A, B, M, N2, alpha, beta, out, s_m, s_nh, s_nl, n_in, err);
}

}  // namespace adc
