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
constexpr uint64_t WAIT_NS = 2000000000ull;   // limit of every pipeline wait (default)
constexpr uint64_t DRAIN_NS = 2000000000ull;  // limit of the waits that drain work in flight after an abort
// limit of the pipeline waits in use; a diagnostic may lower it so that a
// wait gives up on purpose (the drains keep DRAIN_NS)
__device__ unsigned long long g_wait_ns = WAIT_NS;

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
  const uint64_t t0 = gtimer();
  const uint64_t lim = *(volatile unsigned long long *)&g_wait_ns;
  while (!mbar_try(a, parity)) {
    if (*abort_flag) return false;
    if (gtimer() - t0 > lim) return false;
  }
  return true;
}
// wait for work already in flight (copies, MMAs) after an abort: fixed limit
__device__ __forceinline__ void mbar_drain(uint32_t a, uint32_t parity) {
  const uint64_t t0 = gtimer();
  while (!mbar_try(a, parity) && gtimer() - t0 < DRAIN_NS) {
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
// the same with an L2 cache policy (createpolicy)
__device__ __forceinline__ void tma_load_2d_hint(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar,
                                                 uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;"
      ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(mbar), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
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
          const __grid_constant__ CUtensorMap mAl2, const __grid_constant__ CUtensorMap mBh,
          const __grid_constant__ CUtensorMap mBl, const __grid_constant__ CUtensorMap mBl2, int nseg, int M,
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
  const int total_kb = nseg * kps;
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
      // the products of one k-block back to back (second operand reads from L2)
      const int g = kb_beg + i;
      const int seg = g % nseg;
      const int kx = (g / nseg) * TC_BK;
      const uint32_t fb = smem_u32(&full[s]);
      mbar_expect_tx(fb, L::STAGE);
      uint8_t *sa = smem + s * L::STAGE;
      // segments: (hi,hi) (hi,lo) (lo,hi) (hi,lo2) (lo,lo) (lo2,hi)
      const CUtensorMap *am = (seg == 2 || seg == 4) ? &mAl : (seg == 5 ? &mAl2 : &mAh);
      const CUtensorMap *bm = (seg == 1 || seg == 4) ? &mBl : (seg == 3 ? &mBl2 : &mBh);
      tma_load_2d(smem_u32(sa), am, kx, m0, fb);
      tma_load_2d(smem_u32(sa + L::A_BYTES), bm, kx, n0, fb);
      issued = i + 1;
    }
    if (*abort_flag) {
      // drain this CTA's copies in flight before shared memory is released
      for (int j = (issued > ST ? issued - ST : 0); j < issued; ++j) {
        const int s = j % ST, r = j / ST;
        mbar_drain(smem_u32(&full[s]), r & 1);
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
    // after an abort the MMAs already issued finish before TMEM is freed
    if (*abort_flag) mbar_drain(smem_u32(accum), 0);
  } else if (warp >= 2) {
    // ---------------- epilogue: TMEM -> registers -> complex128
    bool ok = mbar_wait(smem_u32(accum), 0, abort_flag);
    if (!ok && !*abort_flag) { atomicExch(err, 3); *abort_flag = 1; }
    if (!ok) mbar_drain(smem_u32(accum), 0);
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
// hi = bf16(x), lo = bf16(x - hi), lo2 = bf16(x - hi - lo) (the differences are exact in FP64)
__device__ __forceinline__ void split_store(double x, __nv_bfloat16 *hi, __nv_bfloat16 *lo, __nv_bfloat16 *lo2) {
  __nv_bfloat16 h = __double2bfloat16(x);
  *hi = h;
  const double r = x - (double)__bfloat162float(h);
  __nv_bfloat16 l = __double2bfloat16(r);
  *lo = l;
  if (lo2) *lo2 = __double2bfloat16(r - (double)__bfloat162float(l));
}

// A rows: [Re | Im] (conj negates Im); element (m, k) at src[m*s_m + k*s_k]
__global__ void k_emb_A(const cplx *__restrict__ src, int64_t M, int64_t K, int64_t s_m, int64_t s_k,
                        int conj, int64_t kp, __nv_bfloat16 *hi, __nv_bfloat16 *lo, __nv_bfloat16 *lo2) {
  // one thread per 8 consecutive k of a row, 16-byte stores of every plane
  const int64_t kq = kp >> 3;
  const int64_t total = M * kq;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = idx / kq, k0 = (idx - m * kq) << 3;
    const cplx *row = src + m * s_m;
    __align__(16) __nv_bfloat16 rh[8], rl[8], rl2[8], ih[8], il[8], il2[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t k = k0 + j;
      cplx x = cmake(0.0, 0.0);
      if (k < K) x = row[k * s_k];
      split_store(x.x, &rh[j], &rl[j], &rl2[j]);
      split_store(conj ? -x.y : x.y, &ih[j], &il[j], &il2[j]);
    }
    const int64_t base = m * 2 * kp + k0;
    *(uint4 *)(hi + base) = *(const uint4 *)rh;
    *(uint4 *)(hi + base + kp) = *(const uint4 *)ih;
    *(uint4 *)(lo + base) = *(const uint4 *)rl;
    *(uint4 *)(lo + base + kp) = *(const uint4 *)il;
    if (lo2) {
      *(uint4 *)(lo2 + base) = *(const uint4 *)rl2;
      *(uint4 *)(lo2 + base + kp) = *(const uint4 *)il2;
    }
  }
}


// B rows: row 2n = [Re | -Im], row 2n+1 = [Im | Re] (conj negates Im first).
// One thread per 8 consecutive k of a row: one row index computation per
// thread, 16-byte stores of every plane (the splits of -Im are the negated
// splits of Im: round to nearest is symmetric)
__global__ void k_emb_B(BSrc src, int64_t Nc, int64_t K, int conj, int64_t kp, __nv_bfloat16 *hi,
                        __nv_bfloat16 *lo, __nv_bfloat16 *lo2) {
  const int64_t kq = kp >> 3;
  const int64_t total = Nc * kq;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = idx / kq, k0 = (idx - n * kq) << 3;
    cplx x[8];
    src.get8(n, k0, K, x);
    __align__(16) __nv_bfloat16 rh[8], rl[8], rl2[8], ih[8], il[8], il2[8], nh[8], nl[8], nl2[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const double im = conj ? -x[j].y : x[j].y;
      split_store(x[j].x, &rh[j], &rl[j], &rl2[j]);
      split_store(im, &ih[j], &il[j], &il2[j]);
      nh[j] = __hneg(ih[j]);
      nl[j] = __hneg(il[j]);
      nl2[j] = __hneg(il2[j]);
    }
    const int64_t r0 = (2 * n) * 2 * kp + k0, r1 = (2 * n + 1) * 2 * kp + k0;
    auto put = [&](__nv_bfloat16 *plane, const __nv_bfloat16 (&re)[8], const __nv_bfloat16 (&imv)[8],
                   const __nv_bfloat16 (&nim)[8]) {
      *(uint4 *)(plane + r0) = *(const uint4 *)re;
      *(uint4 *)(plane + r0 + kp) = *(const uint4 *)nim;
      *(uint4 *)(plane + r1) = *(const uint4 *)imv;
      *(uint4 *)(plane + r1 + kp) = *(const uint4 *)re;
    };
    put(hi, rh, ih, nh);
    put(lo, rl, il, nl);
    if (lo2) put(lo2, rl2, il2, nl2);
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


template <int BN, int ST>
void launch_tc(Exec &ex, const TcView &A, const TcView &B, int64_t M, int64_t N2, cplx alpha, cplx beta,
               cplx *out, int64_t s_m, int64_t s_nh, int64_t s_nl, int64_t n_in, int *err, int nseg) {
  using L = TcLayout<BN, ST>;
  set_smem_limit((const void *)k_tc_gemm<BN, ST>, L::SMEM);
  const int g_sms = device_sm_count();
  CUtensorMap mAh, mAl, mAl2, mBh, mBl, mBl2;
  const int64_t kp2 = 2 * A.kp;
  make_map(&mAh, A.hi, A.rows, kp2, TC_BM);
  make_map(&mAl, A.lo, A.rows, kp2, TC_BM);
  make_map(&mBh, B.hi, B.rows, kp2, BN);
  make_map(&mBl, B.lo, B.rows, kp2, BN);
  if (nseg == 6) {
    make_map(&mAl2, A.lo2, A.rows, kp2, TC_BM);
    make_map(&mBl2, B.lo2, B.rows, kp2, BN);
  } else {
    mAl2 = mAl;  // not read with three segments
    mBl2 = mBl;
  }
  const int kps = (int)(kp2 / TC_BK);
  const int total_kb = nseg * kps;
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
  int pr = ex.prof_begin(nseg == 6 ? "tc_gemm_bf16x6" : "tc_gemm_bf16x3",
                         8.0 * (double)M * (double)(N2 / 2) * (double)Kc);
  k_tc_gemm<BN, ST><<<grid, 192, L::SMEM, ex.stream>>>(mAh, mAl, mAl2, mBh, mBl, mBl2, nseg, (int)M, (int)N2, kps,
                                                      kb_per_split,
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

// ---------------------------------------------------------------- grouped persistent GEMM
// One launch for a list of independent GEMM jobs (several problems and terms).
// Every CTA stays resident and takes the next output tile from a global
// counter until none is left, so uneven jobs balance across the SMs. Tiles of a
// job are numbered (row block, column block, K split) with the K split fastest,
// so consecutive tiles reuse the same A rows from L2. Each job carries its own
// tensor maps, tile width (32..256 columns, runtime) and K split; the shared
// memory ring is sized for the widest tile.
// Roles run decoupled: warp 0 takes tile numbers from the counter into a small
// shared ring and issues the TMA loads, warp 1 issues the MMAs into one of two
// TMEM accumulators (2 x 256 columns), warps 2-5 drain the other accumulator,
// so the epilogue of one tile overlaps the main loop of the next.
constexpr int TG_ST = 4;  // shared-memory stages
constexpr int TG_TQ = 4;  // tile-number ring
struct TgLayout {
  static constexpr int A_BYTES = TC_BM * TC_BK * 2;
  static constexpr int B_BYTES = TC_BNMAX * TC_BK * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int BAR_OFF = TG_ST * STAGE;
  static constexpr int SMEM = 1024 + BAR_OFF + 256;
};

__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)m) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

struct TgTile {
  const TcJob *J;
  int m0, n0, bn, split, kb_beg, nkb;
};
__device__ __forceinline__ TgTile tg_decode(const TcJob *__restrict__ jobs, int njobs, int t) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].tile_begin <= t) lo = mid;
    else hi = mid - 1;
  }
  TgTile d;
  d.J = &jobs[lo];
  const TcJob &J = *d.J;
  const int lt = t - J.tile_begin;
  // panels of J.panel column blocks (the last one narrower), row blocks
  // inside a panel, column blocks inside a row block, K splits fastest
  const int pw = J.panel, np_full = J.tiles_n / pw;
  const int full = np_full * J.tiles_m * pw * J.ksplit;
  int P, r, w;
  if (lt < full) {
    P = lt / (J.tiles_m * pw * J.ksplit);
    r = lt - P * (J.tiles_m * pw * J.ksplit);
    w = pw;
  } else {
    P = np_full;
    r = lt - full;
    w = J.tiles_n - np_full * pw;
  }
  const int per_m = w * J.ksplit;
  const int tm = r / per_m, rem = r - tm * per_m;
  const int tn = P * pw + rem / J.ksplit;
  d.split = rem - (rem / J.ksplit) * J.ksplit;
  d.bn = J.bn;
  d.m0 = tm * TC_BM;
  d.n0 = tn * J.bn;
  d.kb_beg = d.split * J.kb_per_split;
  d.nkb = min(J.nseg * J.kps, d.kb_beg + J.kb_per_split) - d.kb_beg;
  return d;
}

__global__ void __launch_bounds__(192, 1)
k_tc_grouped(const TcJob *__restrict__ jobs, int njobs, int total_tiles, int *counter, int *err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = (uint64_t *)(smem + TgLayout::BAR_OFF);
  uint64_t *empty = full + TG_ST;
  uint64_t *accf = empty + TG_ST;   // accumulator b holds a finished tile (MMA -> epilogue)
  uint64_t *acce = accf + 2;        // accumulator b drained (epilogue -> MMA)
  uint64_t *tfull = acce + 2;       // tile number published (producer -> consumers)
  uint64_t *tempty = tfull + TG_TQ;  // tile number read by the MMA warp and the 4 epilogue warps
  uint32_t *tmem_slot = (uint32_t *)(tempty + TG_TQ);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
  volatile int *ring = (volatile int *)(tmem_slot + 2);
  uint64_t *fin = (uint64_t *)(tmem_slot + 2 + TG_TQ);  // every MMA of this CTA finished

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TG_ST; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&accf[b]), 1);
      mbar_init(smem_u32(&acce[b]), 4);
    }
    for (int q = 0; q < TG_TQ; ++q) {
      mbar_init(smem_u32(&tfull[q]), 1);
      mbar_init(smem_u32(&tempty[q]), 5);
    }
    mbar_init(smem_u32(fin), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)(2 * TC_BNMAX))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- tile scheduler and TMA producer
    uint32_t g = 0, g_issued = 0;
    const uint64_t pol_last = policy_evict_last(), pol_first = policy_evict_first();
    for (uint32_t q = 0;; ++q) {
      const int slot = (int)(q % TG_TQ);
      const uint32_t r = q / TG_TQ;
      if (r > 0 && !mbar_wait(smem_u32(&tempty[slot]), (r - 1) & 1, abort_flag)) {
        if (!*abort_flag) atomicExch(err, 14);
        *abort_flag = 1;
        break;
      }
      const int t = *abort_flag ? total_tiles : atomicAdd(counter, 1);
      ring[slot] = t;
      mbar_arrive(smem_u32(&tfull[slot]));
      if (t >= total_tiles) break;
      const TgTile d = tg_decode(jobs, njobs, t);
      const TcJob &J = *d.J;
      tensormap_acquire(&J.mAh);
      tensormap_acquire(&J.mAl);
      tensormap_acquire(&J.mBh);
      tensormap_acquire(&J.mBl);
      const uint32_t bytes = (uint32_t)(TgLayout::A_BYTES + d.bn * TC_BK * 2);
      bool stop = false;
      for (int i = 0; i < d.nkb; ++i) {
        const uint32_t gi = g + (uint32_t)i;
        const int s = (int)(gi % TG_ST);
        const uint32_t rr = gi / TG_ST;
        if (rr > 0 && !mbar_wait(smem_u32(&empty[s]), (rr - 1) & 1, abort_flag)) {
          if (!*abort_flag) atomicExch(err, 11);
          *abort_flag = 1;
          stop = true;
          break;
        }
        // the products of one k-block (hi hi, hi lo, lo hi) back to back, so
        // that the second read of an operand block comes from L2
        const int kg = d.kb_beg + i;
        const int seg = kg % J.nseg;
        const int kx = (kg / J.nseg) * TC_BK;
        const uint32_t fb = smem_u32(&full[s]);
        mbar_expect_tx(fb, bytes);
        uint8_t *sa = smem + s * TgLayout::STAGE;
        if (J.l2keepB) {
          tma_load_2d_hint(smem_u32(sa), seg == 2 ? &J.mAl : &J.mAh, kx, d.m0, fb, pol_first);
          tma_load_2d_hint(smem_u32(sa + TgLayout::A_BYTES), seg == 1 ? &J.mBl : &J.mBh, kx, d.n0, fb, pol_last);
        } else {
          tma_load_2d(smem_u32(sa), seg == 2 ? &J.mAl : &J.mAh, kx, d.m0, fb);
          tma_load_2d(smem_u32(sa + TgLayout::A_BYTES), seg == 1 ? &J.mBl : &J.mBh, kx, d.n0, fb);
        }
        g_issued = gi + 1;
      }
      if (stop) break;
      g += (uint32_t)d.nkb;
    }
    if (*abort_flag) {
      // drain this CTA's copies in flight before shared memory is released
      for (uint32_t gj = (g_issued > TG_ST ? g_issued - TG_ST : 0); gj < g_issued; ++gj) {
        const int s = (int)(gj % TG_ST);
        mbar_drain(smem_u32(&full[s]), (gj / TG_ST) & 1);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer, accumulators alternating
    uint32_t g = 0;
    for (uint32_t q = 0;; ++q) {
      const int slot = (int)(q % TG_TQ);
      if (!mbar_wait(smem_u32(&tfull[slot]), (q / TG_TQ) & 1, abort_flag)) {
        if (!*abort_flag) atomicExch(err, 15);
        *abort_flag = 1;
        break;
      }
      const int t = ring[slot];
      mbar_arrive(smem_u32(&tempty[slot]));
      if (t >= total_tiles) break;
      const TgTile d = tg_decode(jobs, njobs, t);
      const uint32_t b = q & 1u, use = q >> 1;
      if (use > 0 && !mbar_wait(smem_u32(&acce[b]), (use - 1) & 1, abort_flag)) {
        if (!*abort_flag) atomicExch(err, 16);
        *abort_flag = 1;
        break;
      }
      fence_after();
      const uint32_t dacc = tmem + b * (uint32_t)TC_BNMAX;
      const uint32_t idesc = idesc_bf16(TC_BM, d.bn);
      bool stop = false;
      for (int i = 0; i < d.nkb; ++i) {
        const uint32_t gi = g + (uint32_t)i;
        const int s = (int)(gi % TG_ST);
        if (!mbar_wait(smem_u32(&full[s]), (gi / TG_ST) & 1, abort_flag)) {
          if (!*abort_flag) atomicExch(err, 12);
          *abort_flag = 1;
          stop = true;
          break;
        }
        fence_after();
        const uint32_t a0 = smem_u32(smem + s * TgLayout::STAGE);
        const uint32_t b0 = a0 + TgLayout::A_BYTES;
#pragma unroll
        for (int k = 0; k < TC_BK / 16; ++k)
          mma_bf16(dacc, sdesc(a0 + 32 * k), sdesc(b0 + 32 * k), idesc, (i > 0 || k > 0) ? 1u : 0u);
        mma_commit(smem_u32(&empty[s]));
      }
      if (stop) break;
      mma_commit(smem_u32(&accf[b]));
      g += (uint32_t)d.nkb;
    }
    // every MMA this thread issued has finished before TMEM is freed (after an
    // abort the epilogue no longer waits for them)
    mma_commit(smem_u32(fin));
    mbar_drain(smem_u32(fin), 0);
  } else if (warp >= 2) {
    // ---------------- epilogue: TMEM -> registers -> complex128, one accumulator at a time
    const int qq = warp & 3;
    const int row = qq * 32 + lane;
    for (uint32_t q = 0;; ++q) {
      const int slot = (int)(q % TG_TQ);
      bool ok = mbar_wait(smem_u32(&tfull[slot]), (q / TG_TQ) & 1, abort_flag);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0 && !*abort_flag) { atomicExch(err, 17); *abort_flag = 1; }
        break;
      }
      const int t = ring[slot];
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty[slot]));
      if (t >= total_tiles) break;
      const TgTile d = tg_decode(jobs, njobs, t);
      const TcJob &J = *d.J;
      const uint32_t b = q & 1u, use = q >> 1;
      ok = mbar_wait(smem_u32(&accf[b]), use & 1, abort_flag);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0 && !*abort_flag) { atomicExch(err, 13); *abort_flag = 1; }
        break;
      }
      fence_after();
      __syncwarp();
      const int64_t m = (int64_t)d.m0 + row;
      const bool use_beta = (J.beta.x != 0.0 || J.beta.y != 0.0);
#pragma unroll 1
      for (int cch = 0; cch < d.bn / 32; ++cch) {
        uint32_t v[32];
        tmem_ld32(tmem + b * (uint32_t)TC_BNMAX + ((uint32_t)(qq * 32) << 16) + (uint32_t)(cch * 32), v);
        if (m >= J.M || d.nkb <= 0) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int64_t n2 = (int64_t)d.n0 + cch * 32 + 2 * j;
          if (n2 >= J.N2) break;
          const float re = __uint_as_float(v[2 * j]), im = __uint_as_float(v[2 * j + 1]);
          if (J.part) {
            float *pp = J.part + ((int64_t)d.split * J.M + m) * J.N2 + n2;
            pp[0] = re;
            pp[1] = im;
          } else {
            const int64_t n = n2 >> 1;
            const int64_t nh = n / J.n_in, nl = n - nh * J.n_in;
            cplx *dst = J.out + m * J.s_m + nh * J.s_nh + nl * J.s_nl;
            cplx val = cmul(J.alpha, cmake((double)re, (double)im));
            if (use_beta) val = cadd(val, cmul(J.beta, *dst));
            *dst = val;
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&acce[b]));
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * TC_BNMAX))
                 : "memory");
  }
}

}  // namespace

static void alloc_planes(Exec &ex, TcMat &dst, size_t bytes, int planes) {
  if (dst.hi.bytes < bytes || (planes == 3 && dst.lo2.bytes < bytes)) {
    dst.hi.reset(); dst.lo.reset(); dst.lo2.reset();
    dst.hi = DBuf(ex, bytes);
    dst.lo = DBuf(ex, bytes);
    if (planes == 3) dst.lo2 = DBuf(ex, bytes);
  }
  dst.planes = (planes == 3 && dst.lo2.p) ? 3 : 2;
}

void tc_pack_A(Exec &ex, TcMat &dst, const cplx *src, int64_t M, int64_t K, int64_t s_m, int64_t s_k, bool conj,
               int planes) {
  dst.rows = M;
  dst.kreal = K;
  dst.kp = (K + TC_BK - 1) / TC_BK * TC_BK;
  if (dst.kp == 0) dst.kp = TC_BK;
  const size_t bytes = (size_t)M * 2 * dst.kp * sizeof(__nv_bfloat16);
  alloc_planes(ex, dst, bytes, planes);
  k_emb_A<<<grid1d(M * (dst.kp / 8), 256), 256, 0, ex.stream>>>(src, M, K, s_m, s_k, conj ? 1 : 0, dst.kp,
                                                          (__nv_bfloat16 *)dst.hi.p, (__nv_bfloat16 *)dst.lo.p,
                                                          planes == 3 ? (__nv_bfloat16 *)dst.lo2.p : nullptr);
  ADC_CHECK_LAUNCH();
}

static void pack_B_impl(Exec &ex, TcMat &dst, const BSrc &s, int64_t Nc, int64_t K, bool conj, int planes) {
  dst.rows = 2 * Nc;
  dst.kreal = K;
  dst.kp = (K + TC_BK - 1) / TC_BK * TC_BK;
  if (dst.kp == 0) dst.kp = TC_BK;
  const size_t bytes = (size_t)dst.rows * 2 * dst.kp * sizeof(__nv_bfloat16);
  alloc_planes(ex, dst, bytes, planes);
  k_emb_B<<<grid1d(Nc * (dst.kp / 8), 256), 256, 0, ex.stream>>>(s, Nc, K, conj ? 1 : 0, dst.kp,
                                                           (__nv_bfloat16 *)dst.hi.p, (__nv_bfloat16 *)dst.lo.p,
                                                           planes == 3 ? (__nv_bfloat16 *)dst.lo2.p : nullptr);
  ADC_CHECK_LAUNCH();
}

void tc_pack_B(Exec &ex, TcMat &dst, const cplx *src, int64_t Nc, int64_t K, int64_t s_nh, int64_t s_nl,
               int64_t n_in, int64_t s_k, bool conj, int planes) {
  BSrc s{src, 0, s_nh, s_nl, n_in, s_k, 0, 0, 0, 0};
  pack_B_impl(ex, dst, s, Nc, K, conj, planes);
}

void tc_pack_B_ring(Exec &ex, TcMat &dst, const adc_ctx *c, const cplx *X, int64_t k, int planes) {
  BSrc s{X, c->kind == ADC_EA ? 1 : 2, 0, 0, 1, 0, c->o, c->v, c->N, c->n1};
  const int64_t Nc = (c->kind == ADC_EA) ? k * c->v : k * c->o;
  pack_B_impl(ex, dst, s, Nc, c->o * c->v, false, planes);
}

TcView tc_view(const TcMat &m, int64_t row0, int64_t rows) {
  TcView v;
  const int64_t off = row0 * 2 * m.kp;  // BF16 elements; rows are 4 kp bytes, a multiple of 256
  v.hi = m.hi.p ? (const __nv_bfloat16 *)m.hi.p + off : nullptr;
  v.lo = m.lo.p ? (const __nv_bfloat16 *)m.lo.p + off : nullptr;
  v.lo2 = m.lo2.p ? (const __nv_bfloat16 *)m.lo2.p + off : nullptr;
  v.planes = m.planes;
  v.rows = rows < 0 ? m.rows - row0 : rows;
  v.kp = m.kp;
  v.kreal = m.kreal;
  return v;
}

void tc_gemm(Exec &ex, const TcMat &A, const TcMat &B, int64_t M, int64_t N, cplx alpha, cplx beta, cplx *out,
             int64_t s_m, int64_t s_nh, int64_t s_nl, int64_t n_in, int *err, int nseg) {
  tc_gemm(ex, tc_view(A), tc_view(B), M, N, alpha, beta, out, s_m, s_nh, s_nl, n_in, err, nseg);
}

void tc_gemm(Exec &ex, const TcView &A, const TcView &B, int64_t M, int64_t N, cplx alpha, cplx beta, cplx *out,
             int64_t s_m, int64_t s_nh, int64_t s_nl, int64_t n_in, int *err, int nseg) {
  ADC_REQUIRE(A.kp == B.kp, ADC_ERR_ARG, "tc_gemm: inner sizes differ");
  ADC_REQUIRE(A.rows >= M && B.rows >= 2 * N, ADC_ERR_ARG, "tc_gemm: operand rows");
  ADC_REQUIRE(nseg == 3 || (nseg == 6 && A.planes == 3 && B.planes == 3), ADC_ERR_ARG,
              "tc_gemm: six products need three planes on both operands");
  if (M <= 0 || N <= 0) return;
  ADC_REQUIRE(M < (1ll << 31) && 2 * N < (1ll << 31), ADC_ERR_UNSUPPORTED, "tc_gemm: size");
  if (n_in <= 0) n_in = 1;
  const int64_t N2 = 2 * N;
  if (N2 <= 32) launch_tc<32, 8>(ex, A, B, M, N2, alpha, beta, out, s_m, s_nh, s_nl, n_in, err, nseg);
  else if (N2 <= 64) launch_tc<64, 8>(ex, A, B, M, N2, alpha, beta, out, s_m, s_nh, s_nl, n_in, err, nseg);
  else if (N2 <= 128) launch_tc<128, 6>(ex, A, B, M, N2, alpha, beta, out, s_m, s_nh, s_nl, n_in, err, nseg);
  else launch_tc<256, 4>(ex, A, B, M, N2, alpha, beta, out, s_m, s_nh, s_nl, n_in, err, nseg);
}

}  // namespace adc

// ---------------------------------------------------------------- grouped launch, host side
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

namespace adc {

namespace {

int sm_count() { return device_sm_count(); }

// smallest tile width (multiple of 32, at most 256) covering N2 real columns
// when it is narrow, else the widest tile
int bn_rule(int64_t N2) {
  if (N2 <= 32) return 32;
  if (N2 <= 64) return 64;
  if (N2 <= 128) return 128;
  return 256;
}

std::mutex g_tune_mu;
std::map<std::tuple<int64_t, int64_t, int64_t>, int> g_tuned;

}  // namespace

TcGroup::~TcGroup() {
  if (ev) {
    cudaEventSynchronize(ev);
    cudaEventDestroy(ev);
  }
  if (host) cudaFreeHost(host);
}

static int cached_bn(const TcJobDesc &d) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(std::make_tuple(d.M, 2 * d.N, d.A->kp));
  return it == g_tuned.end() ? 0 : it->second;
}

void tc_gemm_grouped(Exec &ex, const std::vector<TcJobDesc> &in, TcGroup &grp, int *err, bool may_tune) {
  const int nj = (int)in.size();
  if (nj == 0) return;
  set_smem_limit((const void *)k_tc_grouped, TgLayout::SMEM);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  ADC_CUDA(cudaStreamIsCapturing(ex.stream, &cs));
  const bool capturing = (cs != cudaStreamCaptureStatusNone);
  if (capturing) may_tune = false;
  struct Plan {
    int idx, bn, kps, tiles_m, tiles_n, ksplit, kbps, nseg;
    int64_t N2;
  };
  std::vector<Plan> pl;
  double work = 0.0;
  grp.flops = 0.0;
  for (int j = 0; j < nj; ++j) {
    const TcJobDesc &d = in[j];
    ADC_REQUIRE(d.A && d.B && (d.out || d.out32), ADC_ERR_ARG, "tc_gemm_grouped: job operands");
    ADC_REQUIRE(d.nseg == 3 || d.nseg == 1, ADC_ERR_ARG, "tc_gemm_grouped: products per tile");
    ADC_REQUIRE(!d.out32 || d.kb_split > 0, ADC_ERR_ARG, "tc_gemm_grouped: raw output needs kb_split");
    ADC_REQUIRE(d.A->kp == d.B->kp, ADC_ERR_ARG, "tc_gemm_grouped: inner sizes differ");
    ADC_REQUIRE(d.A->rows >= d.M && d.B->rows >= 2 * d.N, ADC_ERR_ARG, "tc_gemm_grouped: operand rows");
    ADC_REQUIRE(d.M < (1ll << 31) && 2 * d.N < (1ll << 31), ADC_ERR_UNSUPPORTED, "tc_gemm_grouped: size");
    if (d.M <= 0 || d.N <= 0) continue;
    Plan p{};
    p.idx = j;
    p.N2 = 2 * d.N;
    p.bn = d.bn;
    if (p.bn <= 0) p.bn = may_tune ? tc_autotune_bn(ex, d, err) : cached_bn(d);
    if (p.bn <= 0) p.bn = bn_rule(p.N2);
    ADC_REQUIRE(p.bn >= 32 && p.bn <= TC_BNMAX && p.bn % 32 == 0, ADC_ERR_ARG, "tc_gemm_grouped: tile width");
    p.kps = (int)(2 * d.A->kp / TC_BK);
    p.nseg = d.nseg;
    p.tiles_m = (int)((d.M + TC_BM - 1) / TC_BM);
    p.tiles_n = (int)((p.N2 + p.bn - 1) / p.bn);
    work += (double)p.tiles_m * p.tiles_n * (double)p.nseg * p.kps;
    const int64_t Kc = d.A->kreal > 0 ? d.A->kreal : d.A->kp;
    grp.flops += 8.0 * (double)d.M * (double)d.N * (double)Kc;
    pl.push_back(p);
  }
  if (pl.empty()) return;
  // split K of long, narrow jobs so that no tile is much longer than the
  // average per-SM share of four waves
  const int sms = sm_count();
  const double target = std::max(16.0, work / (4.0 * sms));
  size_t part_need = 0;
  for (auto &p : pl) {
    const int total_kb = p.nseg * p.kps;
    if (in[p.idx].out32) {
      // raw output: the caller fixes the split (exact FP32 sums need short splits)
      p.kbps = std::min(in[p.idx].kb_split, total_kb);
      p.ksplit = (total_kb + p.kbps - 1) / p.kbps;
      continue;
    }
    int ks = 1;
    if (total_kb > target) ks = (int)std::min<double>(128.0, std::ceil(total_kb / target));
    p.kbps = (total_kb + ks - 1) / ks;
    p.ksplit = (total_kb + p.kbps - 1) / p.kbps;
    if (p.ksplit > 1) part_need += (size_t)p.ksplit * in[p.idx].M * p.N2;
  }
  // longest tiles first (largest k-blocks per tile), whole jobs kept together
  std::stable_sort(pl.begin(), pl.end(), [](const Plan &a, const Plan &b) { return a.kbps > b.kbps; });
  if (grp.part_elems < part_need) {
    grp.part.reset();
    grp.part = DBuf(ex, part_need * sizeof(float));
    grp.part_elems = part_need;
  }
  const int np = (int)pl.size();
  // the previous copy out of the pinned table must have finished before it is rewritten
  if (grp.ev && !capturing) ADC_CUDA(cudaEventSynchronize(grp.ev));
  if (grp.host_cap < (size_t)np) {
    if (grp.host) cudaFreeHost(grp.host);
    grp.host = nullptr;
    ADC_CUDA(cudaMallocHost((void **)&grp.host, (size_t)np * sizeof(TcJob)));
    grp.host_cap = np;
    grp.jobs.reset();
    grp.jobs = DBuf(ex, (size_t)np * sizeof(TcJob));
  }
  if (!grp.counter.p) grp.counter = DBuf(ex, 256);
  int64_t tiles = 0;
  size_t poff = 0;
  for (int i = 0; i < np; ++i) {
    const Plan &p = pl[i];
    const TcJobDesc &d = in[p.idx];
    TcJob &J = grp.host[i];
    std::memset(&J, 0, sizeof(J));
    const int64_t kp2 = 2 * d.A->kp;
    // one-product jobs read only the hi planes (a single-plane operand has no lo)
    make_map(&J.mAh, d.A->hi.p, d.A->rows, kp2, TC_BM);
    make_map(&J.mAl, d.A->lo.p ? d.A->lo.p : d.A->hi.p, d.A->rows, kp2, TC_BM);
    make_map(&J.mBh, d.B->hi.p, d.B->rows, kp2, p.bn);
    make_map(&J.mBl, d.B->lo.p ? d.B->lo.p : d.B->hi.p, d.B->rows, kp2, p.bn);
    ADC_REQUIRE(p.nseg == 1 || (d.A->lo.p && d.B->lo.p), ADC_ERR_ARG, "tc_gemm_grouped: three products need lo planes");
    J.out = d.out;
    J.nseg = p.nseg;
    if (d.out32) {
      J.part = d.out32;
    } else {
      J.part = p.ksplit > 1 ? (float *)grp.part.p + poff : nullptr;
      if (p.ksplit > 1) poff += (size_t)p.ksplit * d.M * p.N2;
    }
    J.s_m = d.s_m;
    J.s_nh = d.s_nh;
    J.s_nl = d.s_nl;
    J.n_in = d.n_in > 0 ? d.n_in : 1;
    J.alpha = d.alpha;
    J.beta = d.beta;
    J.M = (int)d.M;
    J.N2 = (int)p.N2;
    J.kps = p.kps;
    J.bn = p.bn;
    J.tiles_n = p.tiles_n;
    J.tiles_m = p.tiles_m;
    J.ksplit = p.ksplit;
    J.kb_per_split = p.kbps;
    J.tile_begin = (int)tiles;
    {
      // B is re-read by every row block. When A is several times larger, the
      // tiles run in panels of B columns whose planes fit in about a third of
      // L2, loaded with an evict-last policy (A evict-first, streaming through)
      const double planes_used = (p.nseg == 1) ? 1.0 : 2.0;
      const double col_block = (double)p.bn * kp2 * 2.0 * planes_used;  // bytes of one column block of B
      const double bbytes = (double)std::min<int64_t>(d.B->rows, p.N2) * kp2 * 2.0 * planes_used;
      const double abytes = (double)std::min<int64_t>(d.A->rows, d.M) * kp2 * 2.0 * planes_used;
      J.panel = p.tiles_n;
      J.l2keepB = 0;
      if (p.tiles_m > 1 && abytes >= 4.0 * bbytes) {
        J.l2keepB = 1;
        J.panel = (int)std::max<double>(1.0, std::min<double>(p.tiles_n, std::floor(48e6 / col_block)));
      }
    }
    tiles += (int64_t)p.tiles_m * p.tiles_n * p.ksplit;
  }
  ADC_REQUIRE(tiles < (1ll << 31), ADC_ERR_UNSUPPORTED, "tc_gemm_grouped: too many tiles");
  ADC_CUDA(cudaMemcpyAsync(grp.jobs.p, grp.host, (size_t)np * sizeof(TcJob), cudaMemcpyHostToDevice, ex.stream));
  if (!capturing) {
    if (!grp.ev) ADC_CUDA(cudaEventCreateWithFlags(&grp.ev, cudaEventDisableTiming));
    ADC_CUDA(cudaEventRecord(grp.ev, ex.stream));
  }
  ADC_CUDA(cudaMemsetAsync(grp.counter.p, 0, sizeof(int), ex.stream));
  const int grid = (int)std::min<int64_t>(tiles, sms);
  // one-product raw jobs are the digit pairs of the sliced product (tc_slice.cu)
  bool raw = true;
  for (const auto &d : in) raw = raw && d.out32 && d.nseg == 1;
  int pr = ex.prof_begin(raw ? "tc_sliced_pairs" : "tc_grouped_bf16x3", grp.flops);
  k_tc_grouped<<<grid, 192, TgLayout::SMEM, ex.stream>>>((const TcJob *)grp.jobs.p, np, (int)tiles,
                                                         (int *)grp.counter.p, err);
  ADC_CHECK_LAUNCH();
  for (int i = 0; i < np; ++i) {
    const TcJob &J = grp.host[i];
    if (J.ksplit <= 1 || in[pl[i].idx].out32) continue;
    k_tc_reduce<<<grid1d((int64_t)J.M * (J.N2 / 2), 256), 256, 0, ex.stream>>>(
        J.part, J.ksplit, J.M, J.N2, J.out, J.s_m, J.s_nh, J.s_nl, J.n_in, J.alpha, J.beta);
    ADC_CHECK_LAUNCH();
  }
  ex.prof_end(pr);
}

void tc_set_wait_ns(uint64_t ns) {
  const unsigned long long v = ns ? (unsigned long long)ns : (unsigned long long)WAIT_NS;
  ADC_CUDA(cudaMemcpyToSymbol(g_wait_ns, &v, sizeof(v)));
}

int tc_autotune_bn(Exec &ex, const TcJobDesc &d, int *err) {
  const int64_t N2 = 2 * d.N;
  const auto key = std::make_tuple(d.M, N2, d.A->kp);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return it->second;
  }
  std::vector<int> cand;
  for (int bn = 32; bn <= TC_BNMAX; bn *= 2) {
    cand.push_back(bn);
    if (bn >= N2) break;
  }
  // also the narrowest width of the fewest tiles (no padded last tile where N2 allows)
  if (N2 > TC_BNMAX) {
    const int64_t nt = (N2 + TC_BNMAX - 1) / TC_BNMAX;
    const int even = (int)(((N2 + nt - 1) / nt + 31) / 32 * 32);
    if (even < TC_BNMAX) cand.push_back(even);
  }
  int best = bn_rule(N2);
  if (cand.size() > 1) {
    // time each candidate as a lone job writing a scratch output (beta = 0)
    DBuf scratch = cbuf(ex, d.M * d.N);
    TcGroup g;
    cudaEvent_t e0, e1;
    ADC_CUDA(cudaEventCreate(&e0));
    ADC_CUDA(cudaEventCreate(&e1));
    double tbest = 1e300;
    for (int bn : cand) {
      TcJobDesc t = d;
      t.bn = bn;
      t.out = scratch.c();
      t.s_m = d.N;
      t.s_nh = 1;
      t.s_nl = 0;
      t.n_in = 1;
      t.alpha = C1();
      t.beta = C0();
      std::vector<TcJobDesc> one{t};
      tc_gemm_grouped(ex, one, g, err, false);
      ADC_CUDA(cudaEventRecord(e0, ex.stream));
      for (int r = 0; r < 2; ++r) tc_gemm_grouped(ex, one, g, err, false);
      ADC_CUDA(cudaEventRecord(e1, ex.stream));
      ADC_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      ADC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < tbest) { tbest = ms; best = bn; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[key] = best;
  return best;
}

int tc_autotune_table(int64_t *out, int cap) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  int n = 0;
  for (auto &kv : g_tuned) {
    if (out && n < cap) {
      out[4 * n + 0] = std::get<0>(kv.first);
      out[4 * n + 1] = std::get<1>(kv.first);
      out[4 * n + 2] = std::get<2>(kv.first);
      out[4 * n + 3] = kv.second;
    }
    ++n;
  }
  return n;
}

}  // namespace adc
