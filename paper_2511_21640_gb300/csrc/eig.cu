// Small dense Hermitian eigensolver on the device: cyclic Jacobi with the
// round-robin ordering (disjoint pairs rotated in parallel), FP64, one CTA.
// Used for the Rayleigh-Ritz step of Davidson (Eq. 10 projected onto the
// subspace) and for the natural-spinor and semicanonical diagonalisations
// (Eqs. 26 and 29).
#include "eig.cuh"

namespace adc {

namespace {

__device__ inline double block_sum(double v, double *red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

// A (n x n, leading dimension lda) is overwritten; eigenvalues ascending into
// w, eigenvectors as columns of Vout (leading dimension ldv). Vwork n x n.
// info[0] = sweeps used, or -1 when the sweep limit was reached.
// With in_smem the matrix and the eigenvector work array live in shared
// memory for the whole iteration (n up to about 80), else in global memory.
__global__ void __launch_bounds__(1024)
k_jacobi(cplx *Ag, int n, int ldag, cplx *Vg, double *w, cplx *Vout, int ldv, int *info,
         int max_sweeps, double rel_tol, int in_smem) {
  extern __shared__ double sm[];
  const int np = n + (n & 1);       // even number of players
  const int npairs = np / 2;
  double *rc = sm;                  // cos per pair
  double *rs = rc + npairs;         // sin per pair
  double *rpr = rs + npairs;        // phase re
  double *rpi = rpr + npairs;       // phase im
  int *pp = (int *)(rpi + npairs);
  int *pq = pp + npairs;
  double *red = (double *)(pq + npairs);
  const int tid = threadIdx.x, nt = blockDim.x;
  cplx *A = Ag, *Vwork = Vg;
  int lda = ldag;
  if (in_smem) {
    // after the 64 reduction slots, 16-byte aligned
    uintptr_t base = ((uintptr_t)(red + 64) + 15) & ~(uintptr_t)15;
    A = (cplx *)base;
    Vwork = A + (int64_t)n * n;
    lda = n;
    for (int idx = tid; idx < n * n; idx += nt) A[idx] = Ag[(int64_t)(idx / n) * ldag + idx % n];
    __syncthreads();
  }

  for (int idx = tid; idx < n * n; idx += nt) {
    int r = idx / n, cI = idx % n;
    Vwork[(int64_t)r * n + cI] = cmake(r == cI ? 1.0 : 0.0, 0.0);
  }
  // Frobenius norm for the stopping test
  double loc = 0.0;
  for (int idx = tid; idx < n * n; idx += nt) {
    cplx a = A[(int64_t)(idx / n) * lda + idx % n];
    loc += a.x * a.x + a.y * a.y;
  }
  const double fro2 = block_sum(loc, red);
  int sweeps = 0;
  bool done = (n <= 1);
  while (!done && sweeps < max_sweeps) {
    for (int step = 0; step < np - 1; ++step) {
      // pairs of this round
      for (int k = tid; k < npairs; k += nt) {
        int a = (k == 0) ? 0 : ((k - 1 + step) % (np - 1)) + 1;
        int kb = np - 1 - k;
        int b = ((kb - 1 + step) % (np - 1)) + 1;
        int p = min(a, b), q = max(a, b);
        pp[k] = p;
        pq[k] = q;
        double cs = 1.0, sn = 0.0, er = 1.0, ei = 0.0;
        if (q < n) {
          double app = A[(int64_t)p * lda + p].x, aqq = A[(int64_t)q * lda + q].x;
          cplx apq = A[(int64_t)p * lda + q];
          double mag = sqrt(apq.x * apq.x + apq.y * apq.y);
          if (mag > 1e-300) {
            er = apq.x / mag;
            ei = apq.y / mag;
            double tau = (aqq - app) / (2.0 * mag);
            double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            cs = 1.0 / sqrt(1.0 + t * t);
            sn = t * cs;
          }
        }
        rc[k] = cs; rs[k] = sn; rpr[k] = er; rpi[k] = ei;
      }
      __syncthreads();
      // rows: new row p = cs A[p,:] - sn e^{i phi} A[q,:]; row q = sn A[p,:] + cs e^{i phi} A[q,:]
      for (int idx = tid; idx < npairs * n; idx += nt) {
        int k = idx / n, col = idx % n;
        int p = pp[k], q = pq[k];
        if (q >= n) continue;
        double cs = rc[k], sn = rs[k];
        cplx e = cmake(rpr[k], rpi[k]);
        cplx ap = A[(int64_t)p * lda + col], aq = A[(int64_t)q * lda + col];
        cplx eaq = cmul(e, aq);
        A[(int64_t)p * lda + col] = cmake(cs * ap.x - sn * eaq.x, cs * ap.y - sn * eaq.y);
        A[(int64_t)q * lda + col] = cmake(sn * ap.x + cs * eaq.x, sn * ap.y + cs * eaq.y);
      }
      __syncthreads();
      // columns (A and V): new col p = cs X[:,p] - sn e^{-i phi} X[:,q]; col q = sn X[:,p] + cs e^{-i phi} X[:,q]
      for (int idx = tid; idx < npairs * n * 2; idx += nt) {
        int which = idx / (npairs * n);
        int rem = idx % (npairs * n);
        int k = rem / n, row = rem % n;
        int p = pp[k], q = pq[k];
        if (q >= n) continue;
        double cs = rc[k], sn = rs[k];
        cplx ec = cmake(rpr[k], -rpi[k]);
        cplx *X = which ? Vwork : A;
        int64_t ld = which ? n : lda;
        cplx xp = X[(int64_t)row * ld + p], xq = X[(int64_t)row * ld + q];
        cplx exq = cmul(ec, xq);
        X[(int64_t)row * ld + p] = cmake(cs * xp.x - sn * exq.x, cs * xp.y - sn * exq.y);
        X[(int64_t)row * ld + q] = cmake(sn * xp.x + cs * exq.x, sn * xp.y + cs * exq.y);
      }
      __syncthreads();
    }
    ++sweeps;
    double off = 0.0;
    for (int idx = tid; idx < n * n; idx += nt) {
      int r = idx / n, cI = idx % n;
      if (r != cI) {
        cplx a = A[(int64_t)r * lda + cI];
        off += a.x * a.x + a.y * a.y;
      }
    }
    off = block_sum(off, red);
    done = (off <= rel_tol * rel_tol * fro2) || (off == 0.0);
  }
  // sort ascending by rank counting (ties broken by index)
  for (int i = tid; i < n; i += nt) {
    double di = A[(int64_t)i * lda + i].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double dj = A[(int64_t)j * lda + j].x;
      if (dj < di || (dj == di && j < i)) ++rank;
    }
    w[rank] = di;
    for (int r = 0; r < n; ++r) Vout[(int64_t)r * ldv + rank] = Vwork[(int64_t)r * n + i];
  }
  if (in_smem) {
    __syncthreads();
    // the diagonalised matrix back to the caller's array (its diagonal holds the eigenvalues)
    for (int idx = tid; idx < n * n; idx += nt) Ag[(int64_t)(idx / n) * ldag + idx % n] = A[idx];
  }
  if (tid == 0) info[0] = done ? sweeps : -1;
}

}  // namespace

void jacobi_eigh(Exec &ex, cplx *A, int n, int lda, double *w, cplx *V, int ldv, int *info_dev) {
  if (n <= 0) return;
  ADC_REQUIRE(n <= 2048, ADC_ERR_UNSUPPORTED, "jacobi_eigh: matrix larger than 2048");
  DBuf work = cbuf(ex, (int64_t)n * n);
  int np = n + (n & 1), npairs = np / 2;
  size_t smem = (size_t)npairs * 4 * sizeof(double) + (size_t)(2 * npairs + 2) * sizeof(int) +
                64 * sizeof(double);
  constexpr size_t kMaxSmem = 200 * 1024;
  const size_t mats = 16 + 2 * (size_t)n * n * sizeof(cplx);
  const int in_smem = (smem + mats <= kMaxSmem) ? 1 : 0;
  if (in_smem) smem += mats;
  static bool attr_set = false;
  if (!attr_set) {
    ADC_CUDA(cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem));
    attr_set = true;
  }
  k_jacobi<<<1, 1024, smem, ex.stream>>>(A, n, lda, work.c(), w, V, ldv, info_dev, 40, 1e-14, in_smem);
  ADC_CHECK_LAUNCH();
}

}  // namespace adc
