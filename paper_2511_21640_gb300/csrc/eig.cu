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

// ---------------------------------------------------------------- FP32 start + FP64 refinement
// For the Rayleigh-Ritz steps of the Davidson solver (n up to 128) one SM's
// FP64 units (two FMAs per clock) make an FP64 Jacobi take milliseconds.
// Instead: (1) cyclic Jacobi in FP32 on A - sigma I (sigma the mean diagonal),
// one CTA, to about 1e-7 of the spectrum's spread; (2) FP64 iterative
// refinement of the whole eigendecomposition after Ogita and Aishima (2018):
// with X the current eigenvectors, H = X^H X and S = X^H (A - sigma) X (both
// made exactly Hermitian), R = I - H,
//   lambda_i = S_ii / H_ii,
//   F_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i)   for separated i, j,
//          R_ij / 2                                         within a cluster and for i = j,
//   X <- X (I + F),
// which converges quadratically for separated eigenvalues. Hermitian S and H
// make F_ij + conj(F_ji) = R_ij exactly, so the update keeps X orthonormal to
// second order whatever the gap. Columns are coupled when their gap is below
// delta = 2 (||S - diag S||_F + max|lambda| ||R||_F) (the bound of the method),
// below 1e-8 max|lambda| (gaps the FP64 products resolve too coarsely), or when the
// first-order correction would exceed 1e-3 (its second-order error would not
// be small); clusters are the connected components of the coupling. Each
// cluster of at most CL_MAX columns is diagonalised exactly: the FP64 Jacobi
// eigenvectors U of P^H S_c P (P = I + R_c / 2, the first-order Loewdin
// factor of its non-orthonormal basis) rotate its columns of I + F, and their
// eigenvalues replace its lambda. The host repeats steps until the
// corrections between clusters are below 1e-8 of the gaps (beyond the
// rounding noise of S) and the updated X is orthonormal to 1e-13, at least
// nsteps and at most nsteps + 3; otherwise (a cluster wider than CL_MAX, no
// convergence) the FP64 Jacobi solves the matrix instead. The n^3 products
// run as small FP64 GEMMs over many SMs.

constexpr int EIG_NMAX = 128;
constexpr int CL_MAX = 8;
constexpr double OA_ETA = 1e-3;   // largest first-order correction between separate clusters
// gaps below this fraction of max|lambda| always couple: beyond it the rounding
// of S (about eps |lambda|) gives first-order corrections below 1e-8, whose
// squares stay below the rounding of an orthonormal basis
constexpr double OA_TAU = 1e-8;
constexpr double OA_ORTH = 1e-13;  // largest |X^H X - I| of an accepted decomposition

__device__ inline float2 f2mul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

__device__ inline float block_sum_f(float v, float *red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.f;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  float r = red[0];
  __syncthreads();
  return r;
}

__device__ inline double block_max(double v, double *red) {
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

// shared memory of k_jacobi32 before the matrices (rotation tables, pair lists, reduction)
__host__ __device__ inline size_t jacobi32_head_bytes(int n) {
  const int np = n + (n & 1);
  return (size_t)np / 2 * 4 * sizeof(float) + (size_t)np * sizeof(int) + 64 * sizeof(float) + 16;
}

// A (FP64, lda) -> FP32 A - sigma I in shared memory; cyclic Jacobi (round robin);
// eigenvectors sorted by ascending eigenvalue into X (FP64, n x n, columns), sigma
// into *shift. The eigenvector work array lives in shared memory, or in Vg
// (n x n FP32 complex in global memory) when Vg is given.
__global__ void __launch_bounds__(1024)
k_jacobi32(const cplx *__restrict__ Ag, int n, int lda, cplx *X, double *shift, int max_sweeps, float2 *Vg) {
  extern __shared__ float smf[];
  const int np = n + (n & 1), npairs = np / 2;
  float *rc = smf, *rs = rc + npairs, *rpr = rs + npairs, *rpi = rpr + npairs;
  int *pp = (int *)(rpi + npairs), *pq = pp + npairs;
  float *red = (float *)(pq + npairs);
  // rows padded to n + 1 elements: the column rotations walk down a column
  // with consecutive lanes on consecutive rows, free of bank conflicts
  const int ld = n + 1;
  float2 *A = (float2 *)(((uintptr_t)(red + 64) + 15) & ~(uintptr_t)15);
  float2 *V = Vg ? Vg : A + n * ld;
  __shared__ double dred[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  // shift by the mean diagonal (FP64), then round
  double ds = 0.0;
  for (int i = tid; i < n; i += nt) ds += Ag[(int64_t)i * lda + i].x;
  for (int off = 16; off > 0; off >>= 1) ds += __shfl_down_sync(0xffffffffu, ds, off);
  if ((tid & 31) == 0) dred[tid >> 5] = ds;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < (nt >> 5); ++w) t += dred[w];
    dred[0] = t / n;
  }
  __syncthreads();
  const double sigma = dred[0];
  for (int idx = tid; idx < n * n; idx += nt) {
    const int r = idx / n, c = idx % n;
    const cplx a = Ag[(int64_t)r * lda + c];
    A[r * ld + c] = make_float2((float)(a.x - (r == c ? sigma : 0.0)), (float)a.y);
    V[r * ld + c] = make_float2(r == c ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  float loc = 0.f;
  for (int idx = tid; idx < n * n; idx += nt) {
    const float2 a = A[(idx / n) * ld + idx % n];
    loc += a.x * a.x + a.y * a.y;
  }
  const float fro2 = block_sum_f(loc, red);
  bool done = (n <= 1);
  float prev = 3.0e38f;
  for (int sweep = 0; !done && sweep < max_sweeps; ++sweep) {
    for (int step = 0; step < np - 1; ++step) {
      for (int k = tid; k < npairs; k += nt) {
        const int a = (k == 0) ? 0 : ((k - 1 + step) % (np - 1)) + 1;
        const int kb = np - 1 - k;
        const int b = ((kb - 1 + step) % (np - 1)) + 1;
        const int p = min(a, b), q = max(a, b);
        pp[k] = p;
        pq[k] = q;
        float cs = 1.f, sn = 0.f, er = 1.f, ei = 0.f;
        if (q < n) {
          const float app = A[p * ld + p].x, aqq = A[q * ld + q].x;
          const float2 apq = A[p * ld + q];
          const float mag = sqrtf(apq.x * apq.x + apq.y * apq.y);
          if (mag > 1e-30f) {
            er = apq.x / mag;
            ei = apq.y / mag;
            const float tau = (aqq - app) / (2.f * mag);
            const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            cs = 1.f / sqrtf(1.f + t * t);
            sn = t * cs;
          }
        }
        rc[k] = cs; rs[k] = sn; rpr[k] = er; rpi[k] = ei;
      }
      __syncthreads();
      for (int idx = tid; idx < npairs * n; idx += nt) {
        const int k = idx / n, col = idx % n;
        const int p = pp[k], q = pq[k];
        if (q >= n) continue;
        const float cs = rc[k], sn = rs[k];
        const float2 ap = A[p * ld + col], eaq = f2mul(make_float2(rpr[k], rpi[k]), A[q * ld + col]);
        A[p * ld + col] = make_float2(cs * ap.x - sn * eaq.x, cs * ap.y - sn * eaq.y);
        A[q * ld + col] = make_float2(sn * ap.x + cs * eaq.x, sn * ap.y + cs * eaq.y);
      }
      __syncthreads();
      for (int idx = tid; idx < npairs * n * 2; idx += nt) {
        const int which = idx / (npairs * n), rem = idx % (npairs * n);
        const int k = rem / n, row = rem % n;
        const int p = pp[k], q = pq[k];
        if (q >= n) continue;
        const float cs = rc[k], sn = rs[k];
        float2 *M = which ? V : A;
        const float2 xp = M[row * ld + p], exq = f2mul(make_float2(rpr[k], -rpi[k]), M[row * ld + q]);
        M[row * ld + p] = make_float2(cs * xp.x - sn * exq.x, cs * xp.y - sn * exq.y);
        M[row * ld + q] = make_float2(sn * xp.x + cs * exq.x, sn * xp.y + cs * exq.y);
      }
      __syncthreads();
    }
    float off = 0.f;
    for (int idx = tid; idx < n * n; idx += nt) {
      const int r = idx / n, c = idx % n;
      if (r != c) off += A[r * ld + c].x * A[r * ld + c].x + A[r * ld + c].y * A[r * ld + c].y;
    }
    off = block_sum_f(off, red);
    // converged, or at the FP32 rounding floor (the off-diagonal norm no longer drops)
    done = (off <= 1e-13f * fro2) || (off == 0.f) || (off <= 1e-9f * fro2 && sweep >= 1 && off > 0.25f * prev);
    prev = off;
  }
  // columns sorted by ascending eigenvalue, promoted to FP64
  for (int i = tid; i < n; i += nt) {
    const float di = A[i * ld + i].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const float dj = A[j * ld + j].x;
      if (dj < di || (dj == di && j < i)) ++rank;
    }
    for (int r = 0; r < n; ++r) X[(int64_t)r * n + rank] = cmake((double)V[r * ld + i].x, (double)V[r * ld + i].y);
  }
  if (tid == 0) *shift = sigma;
}

// C = op(A) op(B) (n x n, FP64): 8 x 8 output tile per CTA, A rows and B
// columns of the tile staged in shared memory; opA: 0 = A, 1 = A^H; B as is;
// with shift, A - shift I is used for A (opA = 0). beta_one adds C0 (C = C0 + AB).
constexpr int SG_T = 8;
__global__ void __launch_bounds__(SG_T * SG_T)
k_small_gemm(const cplx *__restrict__ A, int lda, int opA, const double *shift, const cplx *__restrict__ B, int ldb,
             int n, const cplx *C0, cplx *C, int ldc) {
  extern __shared__ double smg[];
  cplx *sa = (cplx *)smg;            // [SG_T][n] rows i of op(A)
  cplx *sb = sa + SG_T * n;          // [n][SG_T] columns j of B
  const int i0 = blockIdx.y * SG_T, j0 = blockIdx.x * SG_T;
  const double sh = shift ? *shift : 0.0;
  for (int e = threadIdx.x; e < SG_T * n; e += blockDim.x) {
    const int ii = e / n, k = e % n, i = i0 + ii;
    cplx a = cmake(0.0, 0.0);
    if (i < n) {
      if (opA) { a = A[(int64_t)k * lda + i]; a.y = -a.y; }
      else { a = A[(int64_t)i * lda + k]; if (k == i) a.x -= sh; }
    }
    sa[ii * n + k] = a;
    const int k2 = e / SG_T, jj = e % SG_T, j = j0 + jj;
    sb[k2 * SG_T + jj] = (j < n) ? B[(int64_t)k2 * ldb + j] : cmake(0.0, 0.0);
  }
  __syncthreads();
  const int ii = threadIdx.x / SG_T, jj = threadIdx.x % SG_T;
  const int i = i0 + ii, j = j0 + jj;
  double re = 0.0, im = 0.0;
  for (int k = 0; k < n; ++k) {
    const cplx a = sa[ii * n + k], b = sb[k * SG_T + jj];
    re = fma(a.x, b.x, re);
    re = fma(-a.y, b.y, re);
    im = fma(a.x, b.y, im);
    im = fma(a.y, b.x, im);
  }
  if (i < n && j < n) {
    cplx r = cmake(re, im);
    if (C0) r = cadd(r, C0[(int64_t)i * ldc + j]);
    C[(int64_t)i * ldc + j] = r;
  }
}

// Hermitian part of M (n x n) at (i, j)
__device__ inline cplx herm_at(const cplx *__restrict__ M, int n, int i, int j) {
  const cplx a = M[(int64_t)i * n + j], b = M[(int64_t)j * n + i];
  return cmake(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
}

// One refinement step: from H = X^H X and S = X^H (A - shift) X the estimates
// lam, the clusters (label[i] = smallest column of i's cluster) and
// F = I + correction. stat[0]: largest (|num_ij| - 1e-14 max|lam|) / |gap_ij|
// over pairs in different clusters; stat[1]: clusters wider than CL_MAX.
__global__ void __launch_bounds__(1024)
k_oa_step(const cplx *__restrict__ H, const cplx *__restrict__ S, int n, double *lam, int *label, cplx *F,
          double *stat) {
  __shared__ double red[32];
  __shared__ unsigned int cmask[EIG_NMAX * (EIG_NMAX / 32)];
  __shared__ int lab[EIG_NMAX];
  __shared__ double sl[EIG_NMAX];
  __shared__ int changed;
  constexpr int W = EIG_NMAX / 32;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < n; i += nt) {
    sl[i] = S[(int64_t)i * n + i].x / H[(int64_t)i * n + i].x;
    lab[i] = i;
  }
  for (int w = tid; w < n * W; w += nt) cmask[w] = 0u;
  __syncthreads();
  double so = 0.0, rr = 0.0, lm = 0.0;
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx % n;
    const cplx h = herm_at(H, n, i, j);
    const double rx = (i == j ? 1.0 : 0.0) - h.x, ry = -h.y;
    rr += rx * rx + ry * ry;
    if (i != j) {
      const cplx sv = herm_at(S, n, i, j);
      so += sv.x * sv.x + sv.y * sv.y;
    }
  }
  for (int i = tid; i < n; i += nt) lm = fmax(lm, fabs(sl[i]));
  so = block_sum(so, red);
  rr = block_sum(rr, red);
  lm = block_max(lm, red);
  const double thr = fmax(2.0 * (sqrt(so) + lm * sqrt(rr)), OA_TAU * lm);
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx % n;
    if (j <= i) continue;
    const cplx h = herm_at(H, n, i, j), sv = herm_at(S, n, i, j);
    const double gap = sl[j] - sl[i];
    const double nx = sv.x - sl[j] * h.x, ny = sv.y - sl[j] * h.y;   // S_ij + lam_j R_ij
    if (fabs(gap) <= thr || OA_ETA * fabs(gap) <= sqrt(nx * nx + ny * ny)) {
      atomicOr(&cmask[i * W + (j >> 5)], 1u << (j & 31));
      atomicOr(&cmask[j * W + (i >> 5)], 1u << (i & 31));
    }
  }
  __syncthreads();
  // connected components: every column takes the smallest label among its
  // neighbours until nothing changes (labels only decrease)
  for (int iter = 0; iter <= n; ++iter) {
    if (tid == 0) changed = 0;
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
      int best = lab[i];
      for (int w = 0; w < W; ++w) {
        unsigned int m = cmask[i * W + w];
        while (m) {
          const int b = __ffs(m) - 1;
          m &= m - 1u;
          best = min(best, lab[w * 32 + b]);
        }
      }
      if (best < lab[i]) { lab[i] = best; changed = 1; }
    }
    __syncthreads();
    const int again = changed;
    __syncthreads();
    if (!again) break;
  }
  double fr = 0.0;
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx % n;
    const cplx h = herm_at(H, n, i, j);
    const double rx = (i == j ? 1.0 : 0.0) - h.x, ry = -h.y;
    cplx f;
    if (i == j) {
      f = cmake(1.0 + 0.5 * rx, 0.0);
    } else if (lab[i] == lab[j]) {
      f = cmake(0.5 * rx, 0.5 * ry);
    } else {
      const cplx sv = herm_at(S, n, i, j);
      const double gap = sl[j] - sl[i];
      const double nx = sv.x + sl[j] * rx, ny = sv.y + sl[j] * ry;
      f = cmake(nx / gap, ny / gap);
      fr = fmax(fr, (sqrt(nx * nx + ny * ny) - 1e-14 * lm) / fabs(gap));
    }
    F[idx] = f;
  }
  fr = block_max(fr, red);
  int big = 0;
  for (int i = tid; i < n; i += nt) {
    lam[i] = sl[i];
    label[i] = lab[i];
    if (lab[i] == i) {
      int cnt = 0;
      for (int j = i; j < n; ++j) cnt += (lab[j] == i);
      big += (cnt > CL_MAX);
    }
  }
  const double bigd = block_sum((double)big, red);
  if (tid == 0) {
    stat[0] = fr;
    stat[1] = bigd;
  }
}

// Each cluster of 2..CL_MAX columns (label from k_oa_step) is diagonalised
// exactly: U, w = eig(P^H S_c P), P = I + R_c / 2; its columns of F become
// F[:, c] U and its lam the eigenvalues w. Other columns of F are copied.
__global__ void __launch_bounds__(1024)
k_cluster_rotate(const cplx *__restrict__ F, const cplx *__restrict__ H, const cplx *__restrict__ S,
                 const int *__restrict__ label, int n, double *lam, cplx *Fout) {
  __shared__ cplx U[EIG_NMAX * CL_MAX];    // row j: j's row of its cluster's U
  __shared__ int mem[EIG_NMAX * CL_MAX];   // members of the cluster rooted at i, ascending
  __shared__ int csize[EIG_NMAX], pos[EIG_NMAX], lab[EIG_NMAX];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int j = tid; j < n; j += nt) lab[j] = label[j];
  __syncthreads();
  for (int j = tid; j < n; j += nt) {
    const int root = lab[j];
    int before = 0, total = 0;
    for (int k = 0; k < n; ++k) {
      const int in = (lab[k] == root);
      total += in;
      before += in && k < j;
    }
    pos[j] = before;
    csize[j] = total;
    if (before < CL_MAX) mem[root * CL_MAX + before] = j;
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    if (lab[i] != i) continue;
    const int sc = csize[i];
    if (sc < 2 || sc > CL_MAX) continue;
    const int *mi = mem + i * CL_MAX;
    cplx a[CL_MAX][CL_MAX], u[CL_MAX][CL_MAX], t[CL_MAX][CL_MAX];
    // t = S_c P, a = P^H t with P = I + R_c / 2 (R = I - H)
    for (int r = 0; r < sc; ++r)
      for (int c = 0; c < sc; ++c) {
        cplx acc = cmake(0.0, 0.0);
        for (int l = 0; l < sc; ++l) {
          const cplx hl = herm_at(H, n, mi[l], mi[c]);
          const cplx p = cmake((l == c ? 1.5 : 0.0) - 0.5 * hl.x, -0.5 * hl.y);
          acc = cadd(acc, cmul(herm_at(S, n, mi[r], mi[l]), p));
        }
        t[r][c] = acc;
      }
    for (int r = 0; r < sc; ++r)
      for (int c = 0; c < sc; ++c) {
        cplx acc = cmake(0.0, 0.0);
        for (int l = 0; l < sc; ++l) {
          const cplx hl = herm_at(H, n, mi[l], mi[r]);
          const cplx pc = cmake((l == r ? 1.5 : 0.0) - 0.5 * hl.x, 0.5 * hl.y);   // conj(P[l][r])
          acc = cadd(acc, cmul(pc, t[l][c]));
        }
        a[r][c] = acc;
        u[r][c] = cmake(r == c ? 1.0 : 0.0, 0.0);
      }
    for (int r = 0; r < sc; ++r)
      for (int c = r + 1; c < sc; ++c) {   // exact Hermitian symmetry for the Jacobi sweeps
        const cplx m = cmake(0.5 * (a[r][c].x + a[c][r].x), 0.5 * (a[r][c].y - a[c][r].y));
        a[r][c] = m;
        a[c][r] = cconj(m);
      }
    for (int sweep = 0; sweep < 12; ++sweep) {
      double off = 0.0, dia = 0.0;
      for (int r = 0; r < sc; ++r)
        for (int c = 0; c < sc; ++c) {
          const double m2 = a[r][c].x * a[r][c].x + a[r][c].y * a[r][c].y;
          if (r == c) dia += m2; else off += m2;
        }
      if (off <= 1e-32 * dia || off == 0.0) break;
      for (int p = 0; p < sc - 1; ++p)
        for (int q = p + 1; q < sc; ++q) {
          const cplx apq = a[p][q];
          const double mag = sqrt(apq.x * apq.x + apq.y * apq.y);
          if (mag <= 1e-300) continue;
          const cplx e = cmake(apq.x / mag, apq.y / mag), ec = cconj(e);
          const double tau = (a[q][q].x - a[p][p].x) / (2.0 * mag);
          const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = tt * cs;
          for (int c = 0; c < sc; ++c) {   // rows p, q
            const cplx ap = a[p][c], eaq = cmul(e, a[q][c]);
            a[p][c] = cmake(cs * ap.x - sn * eaq.x, cs * ap.y - sn * eaq.y);
            a[q][c] = cmake(sn * ap.x + cs * eaq.x, sn * ap.y + cs * eaq.y);
          }
          for (int r = 0; r < sc; ++r) {   // columns p, q of a and u
            const cplx xp = a[r][p], exq = cmul(ec, a[r][q]);
            a[r][p] = cmake(cs * xp.x - sn * exq.x, cs * xp.y - sn * exq.y);
            a[r][q] = cmake(sn * xp.x + cs * exq.x, sn * xp.y + cs * exq.y);
            const cplx up = u[r][p], euq = cmul(ec, u[r][q]);
            u[r][p] = cmake(cs * up.x - sn * euq.x, cs * up.y - sn * euq.y);
            u[r][q] = cmake(sn * up.x + cs * euq.x, sn * up.y + cs * euq.y);
          }
        }
    }
    for (int r = 0; r < sc; ++r)
      for (int c = 0; c < sc; ++c) U[mi[r] * CL_MAX + c] = u[r][c];
    for (int c = 0; c < sc; ++c) lam[mi[c]] = a[c][c].x;
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += nt) {
    const int r = idx / n, j = idx % n;
    const int sc = csize[j];
    if (sc < 2 || sc > CL_MAX) {
      Fout[idx] = F[idx];
      continue;
    }
    const int *mj = mem + lab[j] * CL_MAX, jj = pos[j];
    cplx acc = cmake(0.0, 0.0);
    for (int l = 0; l < sc; ++l) acc = cadd(acc, cmul(F[(int64_t)r * n + mj[l]], U[mj[l] * CL_MAX + jj]));
    Fout[idx] = acc;
  }
}

// eigenvalues lam + shift sorted ascending into w, the columns of X likewise into V (ldv)
__global__ void k_sort_out(const double *lam, const double *shift, const cplx *X, int n, double *w, cplx *V,
                           int ldv) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double di = lam[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double dj = lam[j];
      if (dj < di || (dj == di && j < i)) ++rank;
    }
    w[rank] = di + *shift;
    for (int r = 0; r < n; ++r) V[(int64_t)r * ldv + rank] = X[(int64_t)r * n + i];
  }
}

// *out = max |H - I| (H n x n)
__global__ void k_orth_err(const cplx *__restrict__ H, int n, double *out) {
  __shared__ double red[32];
  double m = 0.0;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    const cplx h = H[idx];
    m = fmax(m, fmax(fabs(h.x - (i == j ? 1.0 : 0.0)), fabs(h.y)));
  }
  m = block_max(m, red);
  if (threadIdx.x == 0) *out = m;
}

__global__ void k_copy_square(const cplx *__restrict__ A, int n, int lda, cplx *B) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)n * n;
       idx += (int64_t)gridDim.x * blockDim.x)
    B[idx] = A[(idx / n) * lda + idx % n];
}

constexpr size_t kJacobi32Smem = 200 * 1024;

}  // namespace

namespace {
thread_local int last_steps_ = 0;
}

int eigh_refined_last_steps() { return last_steps_; }

bool eigh_refined_fits(int n) { return n >= 1 && n <= EIG_NMAX; }

void eigh_refined(Exec &ex, const cplx *A, int n, int lda, double *w, cplx *V, int ldv, int nsteps) {
  if (n <= 0) return;
  ADC_REQUIRE(eigh_refined_fits(n), ADC_ERR_UNSUPPORTED, "eigh_refined: matrix too large");
  const int64_t nn = (int64_t)n * n;
  // the FP32 eigenvector work array in shared memory when both (padded) matrices fit
  const size_t mat = (size_t)n * (n + 1) * sizeof(float2);
  size_t smem = jacobi32_head_bytes(n) + mat;
  DBuf vg;
  if (smem + mat <= kJacobi32Smem) smem += mat;
  else vg = DBuf(ex, mat);
  set_smem_limit((const void *)k_jacobi32, (int)kJacobi32Smem);
  set_smem_limit((const void *)k_small_gemm, 64 * 1024);
  DBuf X0 = cbuf(ex, nn), X1 = cbuf(ex, nn), T = cbuf(ex, nn), H = cbuf(ex, nn), S = cbuf(ex, nn), F = cbuf(ex, nn);
  DBuf lam(ex, n * sizeof(double)), sc(ex, 4 * sizeof(double)), lab(ex, n * sizeof(int));
  k_jacobi32<<<1, 1024, smem, ex.stream>>>(A, n, lda, X0.c(), sc.d(), 30, (float2 *)vg.p);
  ADC_CHECK_LAUNCH();
  const dim3 g((n + SG_T - 1) / SG_T, (n + SG_T - 1) / SG_T);
  const size_t gs = 2 * (size_t)SG_T * n * sizeof(cplx);
  cplx *X = X0.c(), *Xn = X1.c();
  bool ok = false;
  for (int it = 0; it < nsteps + 3; ++it) {
    // T = (A - shift) X, S = X^H T, H = X^H X
    k_small_gemm<<<g, SG_T * SG_T, gs, ex.stream>>>(A, lda, 0, sc.d(), X, n, n, nullptr, T.c(), n);
    ADC_CHECK_LAUNCH();
    k_small_gemm<<<g, SG_T * SG_T, gs, ex.stream>>>(X, n, 1, nullptr, T.c(), n, n, nullptr, S.c(), n);
    ADC_CHECK_LAUNCH();
    k_small_gemm<<<g, SG_T * SG_T, gs, ex.stream>>>(X, n, 1, nullptr, X, n, n, nullptr, H.c(), n);
    ADC_CHECK_LAUNCH();
    k_oa_step<<<1, 1024, 0, ex.stream>>>(H.c(), S.c(), n, lam.d(), (int *)lab.p, F.c(), sc.d() + 1);
    ADC_CHECK_LAUNCH();
    k_cluster_rotate<<<1, 1024, 0, ex.stream>>>(F.c(), H.c(), S.c(), (const int *)lab.p, n, lam.d(), T.c());
    ADC_CHECK_LAUNCH();
    // X <- X (I + F) blockdiag(U)
    k_small_gemm<<<g, SG_T * SG_T, gs, ex.stream>>>(X, n, 0, nullptr, T.c(), n, n, nullptr, Xn, n);
    ADC_CHECK_LAUNCH();
    std::swap(X, Xn);
    if (it + 1 >= nsteps) {
      // orthonormality of the updated vectors
      k_small_gemm<<<g, SG_T * SG_T, gs, ex.stream>>>(X, n, 1, nullptr, X, n, n, nullptr, H.c(), n);
      ADC_CHECK_LAUNCH();
      k_orth_err<<<1, 1024, 0, ex.stream>>>(H.c(), n, sc.d() + 3);
      ADC_CHECK_LAUNCH();
      double st[3];
      ADC_CUDA(cudaMemcpyAsync(st, sc.d() + 1, sizeof(st), cudaMemcpyDeviceToHost, ex.stream));
      ADC_CUDA(cudaStreamSynchronize(ex.stream));
      last_steps_ = it + 1;
      if (st[0] <= 1e-8 && st[1] == 0.0 && st[2] <= OA_ORTH) { ok = true; break; }
    }
  }
  if (ok) {
    // eigenvalues: Rayleigh quotients of the vectors before the last update
    // (exact to the square of their error), exact ones within clusters
    k_sort_out<<<1, 256, 0, ex.stream>>>(lam.d(), sc.d(), X, n, w, V, ldv);
    ADC_CHECK_LAUNCH();
    return;
  }
  last_steps_ = -1;
  // a cluster too wide for the exact step, or no convergence: FP64 Jacobi
  k_copy_square<<<(int)std::min<int64_t>((nn + 255) / 256, 1024), 256, 0, ex.stream>>>(A, n, lda, T.c());
  ADC_CHECK_LAUNCH();
  jacobi_eigh(ex, T.c(), n, n, w, V, ldv, (int *)lab.p);
}

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
  set_smem_limit((const void *)k_jacobi, (int)kMaxSmem);
  k_jacobi<<<1, 1024, smem, ex.stream>>>(A, n, lda, work.c(), w, V, ldv, info_dev, 40, 1e-14, in_smem);
  ADC_CHECK_LAUNCH();
}

}  // namespace adc
