// Diagnostics of the contraction kernels (see include/adc_gb300_diag.h).
#include <algorithm>
#include <cmath>
#include <vector>

#include "ctx.cuh"
#include "tc_gemm.cuh"
#include "tc_slice.cuh"
#include "blockops.cuh"
#include "eig.cuh"
#include "../../include/adc_gb300_diag.h"

using namespace adc;

namespace {
__global__ void k_fill_random(cplx *x, int64_t n, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    // splitmix64 of (seed, i)
    uint64_t z = seed * 0x9E3779B97F4A7C15ull + (uint64_t)i * 0xBF58476D1CE4E5B9ull + 0x94D049BB133111EBull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    double a = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    uint64_t w = z * 0xD1342543DE82EF95ull + 1;
    w ^= w >> 29;
    double b = (double)(w >> 11) * (1.0 / 9007199254740992.0);
    x[i] = cmake(2.0 * a - 1.0, 2.0 * b - 1.0);
  }
}
__global__ void k_diff(const cplx *a, const cplx *b, int64_t n, double *out) {
  double d = 0.0, r = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double dx = a[i].x - b[i].x, dy = a[i].y - b[i].y;
    d += dx * dx + dy * dy;
    r += b[i].x * b[i].x + b[i].y * b[i].y;
  }
  atomicAdd(out, d);
  atomicAdd(out + 1, r);
}

// three jobs of different shapes (ragged sizes, tile widths, one long narrow
// job that takes the split-K path) in one grouped launch; every output is
// checked against the FP64 GEMM, rel_err is the largest of the three
int diag_grouped(int64_t M, int64_t N, int64_t K, uint64_t seed, int reps, double *rel_err, double *ms) {
  Exec ex;
  try {
    ADC_CUDA(cudaStreamCreateWithFlags(&ex.stream, cudaStreamNonBlocking));
    {
      const int64_t Ms[3] = {M, M / 2 + 37, 129};
      const int64_t Ns[3] = {N, std::max<int64_t>(1, N / 3), 3};
      const int64_t Ks[3] = {K, K / 2 + 11, 2 * K + 5};
      DBuf A[3], B[3], C[3], R[3];
      TcMat Ta[3], Tb[3];
      DBuf acc(ex, 2 * sizeof(double)), err(ex, sizeof(int));
      fill_zero(ex, err.p, sizeof(int));
      std::vector<TcJobDesc> jobs;
      for (int j = 0; j < 3; ++j) {
        A[j] = cbuf(ex, Ms[j] * Ks[j]);
        B[j] = cbuf(ex, Ns[j] * Ks[j]);
        C[j] = cbuf(ex, Ms[j] * Ns[j]);
        R[j] = cbuf(ex, Ms[j] * Ns[j]);
        k_fill_random<<<grid1d(Ms[j] * Ks[j], 256), 256, 0, ex.stream>>>(A[j].c(), Ms[j] * Ks[j], seed + 13 * j);
        k_fill_random<<<grid1d(Ns[j] * Ks[j], 256), 256, 0, ex.stream>>>(B[j].c(), Ns[j] * Ks[j], seed + 13 * j + 7);
        ADC_CHECK_LAUNCH();
        zgemm(ex, Ms[j], Ns[j], Ks[j], 1, C1(), A[j].c(), 0, Ks[j], 1, false, B[j].c(), 0, 1, Ks[j], false, C0(),
              R[j].c(), 0, Ns[j], 1);
        tc_pack_A(ex, Ta[j], A[j].c(), Ms[j], Ks[j], Ks[j], 1, false);
        tc_pack_B(ex, Tb[j], B[j].c(), Ns[j], Ks[j], Ks[j], 0, 1, 1, false);
        TcJobDesc d;
        d.A = &Ta[j]; d.B = &Tb[j]; d.M = Ms[j]; d.N = Ns[j]; d.out = C[j].c();
        d.s_m = Ns[j]; d.s_nh = 1; d.n_in = 1;
        jobs.push_back(d);
      }
      TcGroup grp;
      tc_gemm_grouped(ex, jobs, grp, (int *)err.p, true);
      cudaEvent_t e0, e1;
      ADC_CUDA(cudaEventCreate(&e0));
      ADC_CUDA(cudaEventCreate(&e1));
      ADC_CUDA(cudaEventRecord(e0, ex.stream));
      for (int r = 0; r < reps; ++r) {
        ADC_CUDA(cudaStreamSynchronize(ex.stream));  // the pinned job table is rewritten by each call
        tc_gemm_grouped(ex, jobs, grp, (int *)err.p, true);
      }
      ADC_CUDA(cudaEventRecord(e1, ex.stream));
      ADC_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (ms) *ms = t / reps;
      double worst = 0.0;
      for (int j = 0; j < 3; ++j) {
        fill_zero(ex, acc.p, acc.bytes);
        k_diff<<<256, 256, 0, ex.stream>>>(C[j].c(), R[j].c(), Ms[j] * Ns[j], acc.d());
        ADC_CHECK_LAUNCH();
        double h[2];
        ADC_CUDA(cudaMemcpyAsync(h, acc.p, sizeof(h), cudaMemcpyDeviceToHost, ex.stream));
        ADC_CUDA(cudaStreamSynchronize(ex.stream));
        worst = std::max(worst, std::sqrt(h[0] / std::max(h[1], 1e-300)));
      }
      int he = 0;
      ADC_CUDA(cudaMemcpyAsync(&he, err.p, sizeof(int), cudaMemcpyDeviceToHost, ex.stream));
      ADC_CUDA(cudaStreamSynchronize(ex.stream));
      if (rel_err) *rel_err = worst;
      if (he) throw Error(ADC_ERR_TIMEOUT, "tensor-core GEMM wait gave up");
    }
    cudaStreamSynchronize(ex.stream);
    cudaStreamDestroy(ex.stream);
    return ADC_OK;
  } catch (const Error &e) {
    if (ex.stream) { cudaStreamSynchronize(ex.stream); cudaStreamDestroy(ex.stream); }
    fprintf(stderr, "adc_diag_gemm: %s\n", e.what());
    return e.code;
  }
}
}  // namespace

extern "C" int adc_diag_gemm(int which, int64_t M, int64_t N, int64_t K, uint64_t seed, int reps,
                             double *rel_err, double *ms) {
  if (M <= 0 || N <= 0 || K <= 0 || reps < 1 || which < 0 || which > 6) return ADC_ERR_ARG;
  if (which == 3) return diag_grouped(M, N, K, seed, reps, rel_err, ms);
  Exec ex;
  try {
    ADC_CUDA(cudaStreamCreateWithFlags(&ex.stream, cudaStreamNonBlocking));
    {
      DBuf A = cbuf(ex, M * K), B = cbuf(ex, N * K), C = cbuf(ex, M * N), R = cbuf(ex, M * N);
      DBuf acc(ex, 2 * sizeof(double)), err(ex, sizeof(int));
      fill_zero(ex, err.p, sizeof(int));
      k_fill_random<<<grid1d(M * K, 256), 256, 0, ex.stream>>>(A.c(), M * K, seed);
      k_fill_random<<<grid1d(N * K, 256), 256, 0, ex.stream>>>(B.c(), N * K, seed + 7);
      ADC_CHECK_LAUNCH();
      zgemm(ex, M, N, K, 1, C1(), A.c(), 0, K, 1, false, B.c(), 0, 1, K, false, C0(), R.c(), 0, N, 1);
      TcMat Ta, Tb;
      TcGroup grp;
      SlMat Sa, Sb;
      SlWork sw;
      auto run = [&]() {
        if (which == 5) {
          sl_gemm(ex, Sa, Sb, M, N, C1(), C0(), C.c(), N, 1, 0, 1, (int *)err.p, sw);
        } else if (which == 6) {
          // the setup's route: zgemm as the sliced product with 48 bits (operand chunks, inner splits)
          ex.sliced_bits = 48;
          zgemm(ex, M, N, K, 1, C1(), A.c(), 0, K, 1, false, B.c(), 0, 1, K, false, C0(), C.c(), 0, N, 1);
          ex.sliced_bits = 0;
        } else if (which == 0) {
          zgemm(ex, M, N, K, 1, C1(), A.c(), 0, K, 1, false, B.c(), 0, 1, K, false, C0(), C.c(), 0, N, 1);
        } else if (which == 1 || which == 4) {
          tc_gemm(ex, Ta, Tb, M, N, C1(), C0(), C.c(), N, 1, 0, 1, (int *)err.p, which == 4 ? 6 : 3);
        } else {
          TcJobDesc d;
          d.A = &Ta; d.B = &Tb; d.M = M; d.N = N; d.out = C.c(); d.s_m = N; d.s_nh = 1; d.n_in = 1;
          tc_gemm_grouped(ex, std::vector<TcJobDesc>{d}, grp, (int *)err.p, true);
        }
      };
      if (which == 5) {
        sl_pack_A(ex, Sa, A.c(), M, K, K, 1, false, 40);
        sl_pack_B(ex, Sb, B.c(), N, K, K, 0, 1, 1, false, Sa);
      } else if (which >= 1 && which != 6) {
        const int planes = which == 4 ? 3 : 2;
        tc_pack_A(ex, Ta, A.c(), M, K, K, 1, false, planes);
        tc_pack_B(ex, Tb, B.c(), N, K, K, 0, 1, 1, false, planes);
      }
      run();
      cudaEvent_t e0, e1;
      ADC_CUDA(cudaEventCreate(&e0));
      ADC_CUDA(cudaEventCreate(&e1));
      ADC_CUDA(cudaEventRecord(e0, ex.stream));
      for (int r = 0; r < reps; ++r) run();
      ADC_CUDA(cudaEventRecord(e1, ex.stream));
      ADC_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (ms) *ms = t / reps;
      fill_zero(ex, acc.p, acc.bytes);
      k_diff<<<256, 256, 0, ex.stream>>>(C.c(), R.c(), M * N, acc.d());
      ADC_CHECK_LAUNCH();
      double h[2];
      int he = 0;
      ADC_CUDA(cudaMemcpyAsync(h, acc.p, sizeof(h), cudaMemcpyDeviceToHost, ex.stream));
      ADC_CUDA(cudaMemcpyAsync(&he, err.p, sizeof(int), cudaMemcpyDeviceToHost, ex.stream));
      ADC_CUDA(cudaStreamSynchronize(ex.stream));
      if (rel_err) *rel_err = std::sqrt(h[0] / std::max(h[1], 1e-300));
      if (he) throw Error(ADC_ERR_TIMEOUT, "tensor-core GEMM wait gave up");
    }
    cudaStreamSynchronize(ex.stream);
    cudaStreamDestroy(ex.stream);
    return ADC_OK;
  } catch (const Error &e) {
    if (ex.stream) { cudaStreamSynchronize(ex.stream); cudaStreamDestroy(ex.stream); }
    fprintf(stderr, "adc_diag_gemm: %s\n", e.what());
    return e.code;
  }
}

extern "C" int adc_profile_enable(adc_ctx *c, int on) {
  if (!c) return ADC_ERR_STATE;
  try {
    cudaStreamSynchronize(c->ex.stream);
    c->ex.prof_clear();
    c->ex.prof = (on != 0);
    return ADC_OK;
  } catch (const Error &e) {
    return e.code;
  }
}

extern "C" int adc_diag_set_sliced_cap(int64_t bytes) {
  set_sliced_cap_bytes(bytes > 0 ? (size_t)bytes : 0);
  return ADC_OK;
}

extern "C" int adc_diag_set_setup_chunk(int64_t elems) {
  set_setup_chunk_elems(elems);
  return ADC_OK;
}

extern "C" int adc_diag_set_wait_ns(uint64_t ns) {
  try {
    tc_set_wait_ns(ns);
    return ADC_OK;
  } catch (const Error &e) {
    return e.code;
  }
}

extern "C" int adc_ladder_mode(const adc_ctx *c, int *direct) {
  if (!c) return ADC_ERR_STATE;
  if (!direct) return ADC_ERR_ARG;
  *direct = c->direct_ladder ? 1 : 0;  // setup (both kinds) and, for EA, every product
  return ADC_OK;
}

extern "C" int adc_setup_routes(const adc_ctx *c, int64_t *n_sliced, int64_t *n_fp64, double *flops_sliced,
                                double *flops_fp64) {
  if (!c) return ADC_ERR_STATE;
  if (!n_sliced || !n_fp64 || !flops_sliced || !flops_fp64) return ADC_ERR_ARG;
  *n_sliced = c->setup_n[0];
  *n_fp64 = c->setup_n[1];
  *flops_sliced = c->setup_flops[0];
  *flops_fp64 = c->setup_flops[1];
  return ADC_OK;
}

extern "C" int adc_memory(const adc_ctx *c, int64_t *in_use, int64_t *peak) {
  if (!c) return ADC_ERR_STATE;
  if (!in_use || !peak) return ADC_ERR_ARG;
  *in_use = c->ex.mem_used;
  *peak = c->ex.mem_peak;
  return ADC_OK;
}

extern "C" int adc_profile_read(adc_ctx *c, adc_kernel_stat *out, int max, int *n) {
  if (!c || !n) return c ? ADC_ERR_ARG : ADC_ERR_STATE;
  try {
    ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
    std::vector<adc_kernel_stat> agg;
    for (auto &r : c->ex.recs) {
      float ms = 0.f;
      ADC_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
      adc_kernel_stat *s = nullptr;
      for (auto &a : agg)
        if (r.name == a.name) s = &a;
      if (!s) {
        adc_kernel_stat z{};
        snprintf(z.name, sizeof(z.name), "%s", r.name.c_str());
        agg.push_back(z);
        s = &agg.back();
      }
      s->launches += 1;
      s->total_ms += ms;
      s->flops += r.flops;
      s->bytes += r.bytes;
    }
    *n = (int)std::min<size_t>(agg.size(), (size_t)std::max(max, 0));
    for (int i = 0; i < *n; ++i) out[i] = agg[i];
    return ADC_OK;
  } catch (const Error &e) {
    return e.code;
  }
}

extern "C" int64_t adc_launch_count(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

namespace {
// 16 independent FMA chains per thread; the result feeds an output so that
// nothing is removed by the compiler
__global__ void __launch_bounds__(256) k_fp64_fma(double *out, int64_t iters, double m, double c) {
  double a[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) a[j] = (double)(threadIdx.x + j) * 1e-3;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = fma(a[j], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 16; ++j) s += a[j];
  if (s == 12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace

extern "C" int adc_diag_fp64_peak(int blocks, int64_t iters, double *tflops, double *ms) {
  if (blocks < 1 || iters < 1 || !tflops || !ms) return ADC_ERR_ARG;
  Exec ex;
  try {
    ADC_CUDA(cudaStreamCreateWithFlags(&ex.stream, cudaStreamNonBlocking));
    {
      DBuf out(ex, (size_t)blocks * 256 * sizeof(double));
      k_fp64_fma<<<blocks, 256, 0, ex.stream>>>(out.d(), std::min<int64_t>(iters, 64), 0.999999, 1e-7);
      ADC_CHECK_LAUNCH();
      cudaEvent_t e0, e1;
      ADC_CUDA(cudaEventCreate(&e0));
      ADC_CUDA(cudaEventCreate(&e1));
      ADC_CUDA(cudaEventRecord(e0, ex.stream));
      k_fp64_fma<<<blocks, 256, 0, ex.stream>>>(out.d(), iters, 0.999999, 1e-7);
      ADC_CHECK_LAUNCH();
      ADC_CUDA(cudaEventRecord(e1, ex.stream));
      ADC_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      *ms = t;
      *tflops = 2.0 * 16.0 * (double)iters * blocks * 256.0 / (t * 1e-3) / 1e12;
    }
    cudaStreamSynchronize(ex.stream);
    cudaStreamDestroy(ex.stream);
    return ADC_OK;
  } catch (const Error &e) {
    if (ex.stream) { cudaStreamSynchronize(ex.stream); cudaStreamDestroy(ex.stream); }
    fprintf(stderr, "adc_diag_fp64_peak: %s\n", e.what());
    return e.code;
  }
}

extern "C" int adc_diag_blockops(int which, int64_t m, int64_t nb, int64_t n, uint64_t seed, int reps,
                                 double *rel_err, double *ms) {
  if (which < 0 || which > 1 || m < 1 || nb < 1 || n < 1 || reps < 1 || m > 1024 || nb > 1024) return ADC_ERR_ARG;
  Exec ex;
  try {
    ADC_CUDA(cudaStreamCreateWithFlags(&ex.stream, cudaStreamNonBlocking));
    {
      // gram: A [m][n], B [nb][n], out [m][nb]; combine: C [m][nb], V [m][n], out [nb][n]
      const int64_t na = (which == 0) ? m * n : m * nb;
      const int64_t nbb = (which == 0) ? nb * n : m * n;
      const int64_t no = (which == 0) ? m * nb : nb * n;
      DBuf A = cbuf(ex, na), B = cbuf(ex, nbb), C = cbuf(ex, no), R = cbuf(ex, no);
      DBuf acc(ex, 2 * sizeof(double));
      k_fill_random<<<grid1d(na, 256), 256, 0, ex.stream>>>(A.c(), na, seed);
      k_fill_random<<<grid1d(nbb, 256), 256, 0, ex.stream>>>(B.c(), nbb, seed + 7);
      ADC_CHECK_LAUNCH();
      if (which == 0)
        zgemm(ex, m, nb, n, 1, C1(), A.c(), 0, n, 1, true, B.c(), 0, 1, n, false, C0(), R.c(), 0, nb, 1);
      else
        zgemm(ex, nb, n, m, 1, C1(), A.c(), 0, 1, nb, false, B.c(), 0, n, 1, false, C0(), R.c(), 0, n, 1);
      auto run = [&]() {
        if (which == 0) gram(ex, A.c(), n, (int)m, B.c(), n, (int)nb, n, C1(), C.c(), nb);
        else combine(ex, A.c(), nb, (int)m, (int)nb, B.c(), n, n, C1(), C0(), C.c(), n);
      };
      run();
      cudaEvent_t e0, e1;
      ADC_CUDA(cudaEventCreate(&e0));
      ADC_CUDA(cudaEventCreate(&e1));
      ADC_CUDA(cudaEventRecord(e0, ex.stream));
      for (int r = 0; r < reps; ++r) run();
      ADC_CUDA(cudaEventRecord(e1, ex.stream));
      ADC_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (ms) *ms = t / reps;
      fill_zero(ex, acc.p, acc.bytes);
      k_diff<<<256, 256, 0, ex.stream>>>(C.c(), R.c(), no, acc.d());
      ADC_CHECK_LAUNCH();
      double h[2];
      ADC_CUDA(cudaMemcpyAsync(h, acc.p, sizeof(h), cudaMemcpyDeviceToHost, ex.stream));
      ADC_CUDA(cudaStreamSynchronize(ex.stream));
      if (rel_err) *rel_err = std::sqrt(h[0] / std::max(h[1], 1e-300));
    }
    cudaStreamSynchronize(ex.stream);
    cudaStreamDestroy(ex.stream);
    return ADC_OK;
  } catch (const Error &e) {
    if (ex.stream) { cudaStreamSynchronize(ex.stream); cudaStreamDestroy(ex.stream); }
    fprintf(stderr, "adc_diag_blockops: %s\n", e.what());
    return e.code;
  }
}

extern "C" int adc_diag_eigh(int which, const adc_c128 *A, int n, double *w, adc_c128 *V, double *ms, int *steps) {
  if (which < 0 || which > 1 || n < 1 || !A || !w || !V) return ADC_ERR_ARG;
  if (which == 1 && !eigh_refined_fits(n)) return ADC_ERR_UNSUPPORTED;
  Exec ex;
  try {
    ADC_CUDA(cudaStreamCreateWithFlags(&ex.stream, cudaStreamNonBlocking));
    {
      const int64_t nn = (int64_t)n * n;
      DBuf Ad = cbuf(ex, nn), Aw = cbuf(ex, nn), Vd = cbuf(ex, nn), wd(ex, n * sizeof(double)), info(ex, 16);
      ADC_CUDA(cudaMemcpyAsync(Ad.p, A, nn * sizeof(cplx), cudaMemcpyHostToDevice, ex.stream));
      auto run = [&]() {
        ADC_CUDA(cudaMemcpyAsync(Aw.p, Ad.p, nn * sizeof(cplx), cudaMemcpyDeviceToDevice, ex.stream));
        if (which == 0) jacobi_eigh(ex, Aw.c(), n, n, wd.d(), Vd.c(), n, (int *)info.p);
        else eigh_refined(ex, Aw.c(), n, n, wd.d(), Vd.c(), n);
      };
      run();
      cudaEvent_t e0, e1;
      ADC_CUDA(cudaEventCreate(&e0));
      ADC_CUDA(cudaEventCreate(&e1));
      ADC_CUDA(cudaEventRecord(e0, ex.stream));
      run();
      ADC_CUDA(cudaEventRecord(e1, ex.stream));
      ADC_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (ms) *ms = t;
      if (steps) *steps = (which == 1) ? eigh_refined_last_steps() : 0;
      ADC_CUDA(cudaMemcpyAsync(w, wd.p, n * sizeof(double), cudaMemcpyDeviceToHost, ex.stream));
      ADC_CUDA(cudaMemcpyAsync(V, Vd.p, nn * sizeof(cplx), cudaMemcpyDeviceToHost, ex.stream));
      ADC_CUDA(cudaStreamSynchronize(ex.stream));
    }
    cudaStreamDestroy(ex.stream);
    return ADC_OK;
  } catch (const Error &e) {
    if (ex.stream) { cudaStreamSynchronize(ex.stream); cudaStreamDestroy(ex.stream); }
    fprintf(stderr, "adc_diag_eigh: %s\n", e.what());
    return e.code;
  }
}
