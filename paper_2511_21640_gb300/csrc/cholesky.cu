// One-step pivoted Cholesky decomposition of the two-electron integrals and
// the transformation of the vectors to molecular spinors (Sec. 2.5, Eqs. 41-42).
//
// Eq. 41 from the positive semidefinite V[(mu nu)][(kappa lambda)]: at every
// step the largest remaining diagonal d_max is the pivot (the decomposition
// stops when d_max < tau or d_max <= 0), the new vector is
//   L^P = (V[piv][:] - sum_{P' < P} L^P'[piv] L^P') / sqrt(d_max)
// (V is symmetric, so its row is the pivot column), and the remaining
// diagonal loses (L^P)^2. Eq. 42: B^P = C^H L^P C.
#include <cmath>

#include "ctx.cuh"

namespace adc {

namespace {

__global__ void k_diag_of(const double *__restrict__ V, int64_t n, double *d) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x)
    d[m] = V[m * n + m];
}

// largest element of d (the lowest index among equal ones), one block of 1024 threads
__global__ void __launch_bounds__(1024) k_argmax(const double *__restrict__ d, int64_t n, double *val, int64_t *idx) {
  __shared__ double sv[1024];
  __shared__ int64_t si[1024];
  const int t = threadIdx.x;
  double bv = -INFINITY;
  int64_t bi = 0;
  for (int64_t m = t; m < n; m += blockDim.x) {
    const double x = d[m];
    if (x > bv) { bv = x; bi = m; }
  }
  sv[t] = bv;
  si[t] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) {
      const double ov = sv[t + s];
      const int64_t oi = si[t + s];
      if (ov > sv[t] || (ov == sv[t] && oi < si[t])) { sv[t] = ov; si[t] = oi; }
    }
    __syncthreads();
  }
  if (t == 0) { *val = sv[0]; *idx = si[0]; }
}

// new vector P and the diagonal update
__global__ void k_chol_vector(const double *__restrict__ V, int64_t n, const double *L, int64_t P, int64_t piv,
                              double inv_sqrt, double *Lp, double *d) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x) {
    double s = V[piv * n + m];
    for (int64_t q = 0; q < P; ++q) s -= L[q * n + m] * L[q * n + piv];
    const double l = s * inv_sqrt;
    Lp[m] = l;
    d[m] = (m == piv) ? 0.0 : d[m] - l * l;
  }
}

__global__ void k_real_to_complex(const double *__restrict__ x, int64_t n, cplx *y) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x)
    y[m] = cmake(x[m], 0.0);
}

}  // namespace

int64_t cholesky_run(Exec &ex, const double *V, int64_t n, double tau, int64_t max_rank, double *L,
                     int64_t *pivots) {
  DBuf d(ex, n * sizeof(double)), mv(ex, sizeof(double) + sizeof(int64_t));
  double *dval = (double *)mv.p;
  int64_t *didx = (int64_t *)((char *)mv.p + sizeof(double));
  k_diag_of<<<grid1d(n, 256), 256, 0, ex.stream>>>(V, n, d.d());
  ADC_CHECK_LAUNCH();
  int64_t P = 0;
  for (; P < max_rank; ++P) {
    k_argmax<<<1, 1024, 0, ex.stream>>>(d.d(), n, dval, didx);
    ADC_CHECK_LAUNCH();
    double h_val = 0.0;
    int64_t h_idx = 0;
    ADC_CUDA(cudaMemcpyAsync(&h_val, dval, sizeof(double), cudaMemcpyDeviceToHost, ex.stream));
    ADC_CUDA(cudaMemcpyAsync(&h_idx, didx, sizeof(int64_t), cudaMemcpyDeviceToHost, ex.stream));
    ADC_CUDA(cudaStreamSynchronize(ex.stream));
    if (!(h_val >= tau) || h_val <= 0.0) break;
    ADC_REQUIRE(h_idx >= 0 && h_idx < n, ADC_ERR_NUMERIC, "cholesky: pivot index");
    k_chol_vector<<<grid1d(n, 256), 256, 0, ex.stream>>>(V, n, L, P, h_idx, 1.0 / std::sqrt(h_val), L + P * n,
                                                         d.d());
    ADC_CHECK_LAUNCH();
    if (pivots) pivots[P] = h_idx;
  }
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
  return P;
}

void cholesky_mo(Exec &ex, const double *L, int64_t rank, int64_t nao, const cplx *C, int64_t nmo, cplx *B) {
  if (rank <= 0) return;
  DBuf Lc = cbuf(ex, rank * nao * nao), T = cbuf(ex, rank * nao * nmo);
  k_real_to_complex<<<grid1d(rank * nao * nao, 256), 256, 0, ex.stream>>>(L, rank * nao * nao, Lc.c());
  ADC_CHECK_LAUNCH();
  // T[P] = L^P C, then B[P] = C^H T[P]
  zgemm(ex, nao, nmo, nao, rank, C1(), Lc.c(), nao * nao, nao, 1, false, C, 0, nmo, 1, false, C0(), T.c(),
        nao * nmo, nmo, 1);
  zgemm(ex, nmo, nmo, nao, rank, C1(), C, 0, 1, nmo, true, T.c(), nao * nmo, nmo, 1, false, C0(), B, nmo * nmo,
        nmo, 1);
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
}

}  // namespace adc
