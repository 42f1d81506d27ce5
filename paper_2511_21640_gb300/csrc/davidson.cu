// Block Davidson for the lowest roots of M (Eq. 10: M X = X Omega, X^H X = 1).
//
// Subspace matrices, Rayleigh-Ritz (device Jacobi), residual norms, Gram-Schmidt
// and the diagonal preconditioner are FP64 throughout. With the split-precision
// sigma the method runs in two phases:
//   1. plain Davidson with tensor-core sigma products until the residual norms
//      stop decreasing (the split-precision floor);
//   2. refinement: the subspace is collapsed onto the current Ritz vectors and
//      their sigma is recomputed in FP64, so that sigma(y + delta) =
//      sigma64(y) + sigma_mixed(delta); new correction vectors keep using the
//      tensor-core product. The projected couplings between an FP64 base
//      vector b and a correction t are taken as <sigma64(b)|t> (M is
//      Hermitian), so split-precision noise enters only the correction-
//      correction block, whose weight shrinks with the residual. Every
//      collapse (subspace full, stall, or apparent convergence) recomputes
//      sigma64 of the Ritz vectors, and convergence is only accepted on FP64
//      residuals ||sigma64(y) - omega y|| <= tol.
//   3. when the refinement itself stalls twice, the correction vectors take
//      the next precision: with the sliced refinement first the sliced product
//      with about 24 bits (an intermediate step at about a third of the digit
//      products), after a further stall the refinement precision itself.
// The refinement products (sigma64) are FP64, or with opts.refine the sliced
// tensor-core product of tc_slice.cu, exact digit products combined in FP64.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>

#include "ctx.cuh"
#include "blockops.cuh"
#include "eig.cuh"

namespace adc {

namespace {

__global__ void k_hermitize(const cplx *G, int ldg, int m, cplx *H, int ldh) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * m) return;
  int i = idx / m, j = idx % m;
  cplx a = G[(int64_t)i * ldg + j], b = G[(int64_t)j * ldg + i];
  H[(int64_t)i * ldh + j] = cmake(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
}

// G[m0 + i][j] = conj(G[j][m0 + i]) for j < m0
__global__ void k_fill_lower(cplx *G, int ldg, int m0, int na) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= na * m0) return;
  int i = idx / m0, j = idx % m0;
  cplx a = G[(int64_t)j * ldg + m0 + i];
  G[(int64_t)(m0 + i) * ldg + j] = cmake(a.x, -a.y);
}

// swap column 0 and column r of C (rows 0..m-1, leading dimension ldc) and w[0], w[r]
__global__ void k_swap_first(cplx *C, int ldc, int m, double *w, int r) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const cplx t = C[(int64_t)i * ldc];
    C[(int64_t)i * ldc] = C[(int64_t)i * ldc + r];
    C[(int64_t)i * ldc + r] = t;
  }
  if (threadIdx.x == 0) {
    const double t = w[0];
    w[0] = w[r];
    w[r] = t;
  }
}

// R[r] = SY[r] - w[r] Y[r]
__global__ void k_residual(const cplx *SY, const cplx *Y, const double *w, int64_t k, int64_t n,
                           cplx *R) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < k * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = idx / n;
    cplx s = SY[idx], y = Y[idx];
    R[idx] = cmake(s.x - w[r] * y.x, s.y - w[r] * y.y);
  }
}

// part[r][b] = sum of |X[r][i]|^2 over segment b of row r (gridDim.x segments per row)
__global__ void k_row_norms_part(const cplx *X, int64_t n, int64_t ld, double *part) {
  __shared__ double red[32];
  const cplx *x = X + blockIdx.y * ld;
  const int64_t seg = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * seg, i1 = min(n, i0 + seg);
  double s = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) s += x[i].x * x[i].x + x[i].y * x[i].y;
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// out[r] = sqrt(sum_b part[r][b]), the segments in order (deterministic)
__global__ void k_row_norms_fin(const double *part, int nseg, int k, double *out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= k) return;
  double s = 0.0;
  for (int b = 0; b < nseg; ++b) s += part[(int64_t)r * nseg + b];
  out[r] = sqrt(s);
}

// T[r] = R[r] / (w[r] - diag), |denominator| floored at 1e-4
__global__ void k_precondition(const cplx *R, const double *w, const int *rows, const double *diag,
                               int64_t nt, int64_t n, cplx *T) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nt * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = idx / n, i = idx % n;
    int r = rows[t];
    double den = w[r] - diag[i];
    if (fabs(den) < 1e-4) den = (den < 0.0) ? -1e-4 : 1e-4;
    cplx v = R[(int64_t)r * n + i];
    T[idx] = cmake(v.x / den, v.y / den);
  }
}

// Olsen's correction: for each correction t (root rows[t]), over segment b of
// the vector, part[t][b] = (sum conj(y) r / den, sum |y|^2 / den) with the
// preconditioner's denominators den = w - diag (|den| floored as above)
__global__ void k_olsen_part(const cplx *R, const cplx *Y, const double *w, const int *rows, const double *diag,
                             int64_t n, double *part) {
  __shared__ double red[3][32];
  const int t = blockIdx.y, r = rows[t];
  const int64_t seg = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * seg, i1 = min(n, i0 + seg);
  double ar = 0.0, ai = 0.0, b = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    double den = w[r] - diag[i];
    if (fabs(den) < 1e-4) den = (den < 0.0) ? -1e-4 : 1e-4;
    const cplx y = Y[(int64_t)r * n + i], v = R[(int64_t)r * n + i];
    ar += (y.x * v.x + y.y * v.y) / den;
    ai += (y.x * v.y - y.y * v.x) / den;
    b += (y.x * y.x + y.y * y.y) / den;
  }
  for (int off = 16; off > 0; off >>= 1) {
    ar += __shfl_down_sync(0xffffffffu, ar, off);
    ai += __shfl_down_sync(0xffffffffu, ai, off);
    b += __shfl_down_sync(0xffffffffu, b, off);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { red[0][wid] = ar; red[1][wid] = ai; red[2][wid] = b; }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[threadIdx.x][k];
    part[((int64_t)t * gridDim.x + blockIdx.x) * 3 + threadIdx.x] = s;
  }
}

// e_t = (y^H den^-1 r) / (y^H den^-1 y), the segment sums in order
__global__ void k_olsen_fin(const double *part, int nseg, int nt, cplx *e) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double ar = 0.0, ai = 0.0, b = 0.0;
  for (int s = 0; s < nseg; ++s) {
    const double *p = part + ((int64_t)t * nseg + s) * 3;
    ar += p[0];
    ai += p[1];
    b += p[2];
  }
  e[t] = (b != 0.0) ? cmake(ar / b, ai / b) : cmake(0.0, 0.0);
}

// T[t] = (R[r] - e_t Y[r]) / den: the correction is orthogonal to its Ritz vector
__global__ void k_olsen_apply(const cplx *R, const cplx *Y, const double *w, const int *rows, const double *diag,
                              const cplx *ev, int64_t nt, int64_t n, cplx *T) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nt * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = idx / n, i = idx % n;
    const int r = rows[t];
    const cplx e = ev[t];
    double den = w[r] - diag[i];
    if (fabs(den) < 1e-4) den = (den < 0.0) ? -1e-4 : 1e-4;
    const cplx v = R[(int64_t)r * n + i], y = Y[(int64_t)r * n + i];
    const cplx u = csub(v, cmul(e, y));
    T[idx] = cmake(u.x / den, u.y / den);
  }
}

// T[t] = R[rows[t]]
__global__ void k_gather_rows(const cplx *R, const int *rows, int64_t nt, int64_t n, cplx *T) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nt * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = idx / n, i = idx - t * n;
    T[idx] = R[(int64_t)rows[t] * n + i];
  }
}

__global__ void k_unit_vectors(cplx *V, int64_t n, const int64_t *idx, int k) {
  int r = blockIdx.x;
  if (r >= k) return;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) V[(int64_t)r * n + i] = cmake(0.0, 0.0);
  __syncthreads();
  if (threadIdx.x == 0) V[(int64_t)r * n + idx[r]] = cmake(1.0, 0.0);
}

// W[:, c] = Z[:, keep[c]] / sqrt(lam[keep[c]])  (nt x nk, row-major, ld nk)
__global__ void k_lowdin(const cplx *Z, int nt, const double *lam, const int *keep, int nk, cplx *W) {
  for (int idx = threadIdx.x; idx < nt * nk; idx += blockDim.x) {
    int i = idx / nk, cI = idx % nk;
    int j = keep[cI];
    double s = 1.0 / sqrt(lam[j]);
    cplx z = Z[(int64_t)i * nt + j];
    W[(int64_t)i * nk + cI] = cmake(z.x * s, z.y * s);
  }
}

struct Timer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double s() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

}  // namespace

struct Davidson {
  adc_ctx *c;
  Exec &ex;
  int64_t N;
  int nroots, mmax, krmax;
  DBuf V, AV, G, H, Cv, w, T, Tn, Y, SY, R, nrm, rowsb, info, tmp, Gs, Zs, Ws, w2;
  adc_stats st{};
  double tsig = 0.0;
  int m = 0;
  int nb = 0;  // leading subspace vectors whose sigma is FP64
  bool follow = false;  // root-specific: track the Ritz vector closest to gfol
  DBuf gfol, ovl;
  int prec64 = ADC_PREC_FP64;  // precision of the refinement products (FP64 or the sliced FP64-accurate product)

  Davidson(adc_ctx *c_, int nr, int mmax_, int krmax_)
      : c(c_), ex(c_->ex), N(c_->N), nroots(nr), mmax(mmax_), krmax(krmax_) {
    V = cbuf(ex, (int64_t)mmax * N);
    AV = cbuf(ex, (int64_t)mmax * N);
    G = cbuf(ex, (int64_t)mmax * mmax);
    H = cbuf(ex, (int64_t)mmax * mmax);
    Cv = cbuf(ex, (int64_t)mmax * mmax);
    w = DBuf(ex, mmax * sizeof(double));
    T = cbuf(ex, (int64_t)nr * N);
    Tn = cbuf(ex, (int64_t)nr * N);
    fill_zero(ex, T.p, T.bytes);
    Gs = cbuf(ex, (int64_t)nr * nr);
    Zs = cbuf(ex, (int64_t)nr * nr);
    Ws = cbuf(ex, (int64_t)nr * nr);
    w2 = DBuf(ex, nr * sizeof(double));
    Y = cbuf(ex, (int64_t)krmax * N);
    SY = cbuf(ex, (int64_t)krmax * N);
    R = cbuf(ex, (int64_t)nr * N);
    nrm = DBuf(ex, mmax * sizeof(double));
    rowsb = DBuf(ex, mmax * sizeof(int));
    info = DBuf(ex, 16);
    tmp = cbuf(ex, (int64_t)mmax * std::max(mmax, nr));
  }

  void apply_sigma(const cplx *X, cplx *S, int64_t k, int prec) {
    Timer t;
    // inside a batch the other problems go on without this one meanwhile
    if (c->batch) batch_leave(c);
    try {
      sigma(c, X, S, k, prec);
      ADC_CUDA(cudaStreamSynchronize(ex.stream));
    } catch (...) {
      if (c->batch) batch_rejoin(c);
      throw;
    }
    if (c->batch) batch_rejoin(c);
    tsig += t.s();
    st.sigma_calls += (int)k;
    if (prec == ADC_PREC_FP64 || prec == ADC_PREC_SLICED) st.sigma_calls_fp64 += (int)k;
    if (prec == ADC_PREC_SLICED24) st.sigma_calls_mid += (int)k;
  }

  // sigma of the na new vectors (in T and in V[m:m+na]) into AV[m:m+na]. In a
  // batch the split-precision product of the whole T block (nroots rows, the
  // rows past na are ignored) joins the other problems' blocks; T and Tn keep
  // their addresses, so a repeated batch replays a captured graph.
  void apply_sigma_new(int na, int prec) {
    if (c->batch && prec == ADC_PREC_BF16X3 && na <= nroots) {
      Timer t;
      batch_submit(c, T.c(), Tn.c(), nroots);
      ADC_CUDA(cudaMemcpyAsync(AV.c() + (int64_t)m * N, Tn.c(), (int64_t)na * N * sizeof(cplx),
                               cudaMemcpyDeviceToDevice, ex.stream));
      tsig += t.s();
      st.sigma_calls += na;
      return;
    }
    apply_sigma(V.c() + (int64_t)m * N, AV.c() + (int64_t)m * N, na, prec);
  }

  // G[0:m+na][m:m+na] = V^H AV[m:m+na], lower part by Hermiticity
  void extend_projection(int m0, int na) {
    int mt = m0 + na;
    gram(ex, V.c(), N, mt, AV.c() + (int64_t)m0 * N, N, na, N, C1(), G.c() + m0, mmax);
    if (nb > 0 && m0 >= nb) {
      // rows of the FP64 base: <b|M|t> = <sigma64(b)|t>
      gram(ex, AV.c(), N, nb, V.c() + (int64_t)m0 * N, N, na, N, C1(), G.c() + m0, mmax);
    }
    if (m0 > 0) {
      k_fill_lower<<<(na * m0 + 255) / 256, 256, 0, ex.stream>>>(G.c(), mmax, m0, na);
      ADC_CHECK_LAUNCH();
    }
  }

  std::vector<double> row_norms(const cplx *X, int k) {
    std::vector<double> h(k);
    if (!k) return h;
    // about four CTAs per SM in all, segments of at least 4096 elements
    const int nseg = (int)std::max<int64_t>(1, std::min<int64_t>((608 + k - 1) / k, (N + 4095) / 4096));
    DBuf part(ex, (size_t)k * nseg * sizeof(double));
    k_row_norms_part<<<dim3(nseg, k), 256, 0, ex.stream>>>(X, N, N, part.d());
    ADC_CHECK_LAUNCH();
    k_row_norms_fin<<<(k + 127) / 128, 128, 0, ex.stream>>>(part.d(), nseg, k, nrm.d());
    ADC_CHECK_LAUNCH();
    ADC_CUDA(cudaMemcpyAsync(h.data(), nrm.d(), k * sizeof(double), cudaMemcpyDeviceToHost, ex.stream));
    ADC_CUDA(cudaStreamSynchronize(ex.stream));
    return h;
  }

  // project out span(V[0:m]) from T[0:nt] by block classical Gram-Schmidt,
  // a second pass only when the first removed more than 1 - 1/sqrt(2) of some
  // vector's norm (the criterion of Daniel, Gragg, Kaufman and Stewart: past
  // it one pass leaves T orthogonal to V to the rounding of the products),
  // then orthonormalise the block symmetrically (Loewdin, as in Eq. 6): with
  // <t_a|t_b> = Z diag(l) Z^H, the kept directions are T' = (Z l^-1/2)^T T for
  // eigenvalues l above the rank threshold. Returns the number of vectors kept,
  // stored at the front of T.
  int cgs_passes = 0;
  int orthonormalise(int nt) {
    if (nt <= 0) return 0;
    std::vector<double> n0 = row_norms(T.c(), nt);
    double nmax = *std::max_element(n0.begin(), n0.end());
    if (!(nmax > 1e-300) || !std::isfinite(nmax)) return 0;
    for (int pass = 0; pass < 2 && m > 0; ++pass) {
      gram(ex, V.c(), N, m, T.c(), N, nt, N, C1(), tmp.c(), nt);
      combine(ex, tmp.c(), nt, m, nt, V.c(), N, N, CR(-1.0), C1(), T.c(), N);
      ++cgs_passes;
      if (pass == 0) {
        const std::vector<double> n1 = row_norms(T.c(), nt);
        bool enough = true;
        for (int j = 0; j < nt; ++j)
          if (!(n1[j] >= 0.70710678118654752 * n0[j])) enough = false;
        if (enough) break;
      }
    }
    gram(ex, T.c(), N, nt, T.c(), N, nt, N, C1(), Gs.c(), nt);
    // FP64 Jacobi: its small eigenvalues (which decide the directions kept)
    // carry relative accuracy; the block is at most a few vectors wide
    jacobi_eigh(ex, Gs.c(), nt, nt, w2.d(), Zs.c(), nt, (int *)info.p);
    std::vector<double> lam(nt);
    ADC_CUDA(cudaMemcpyAsync(lam.data(), w2.d(), nt * sizeof(double), cudaMemcpyDeviceToHost, ex.stream));
    ADC_CUDA(cudaStreamSynchronize(ex.stream));
    const double thr = std::max(1e-28, (1e-8 * nmax) * (1e-8 * nmax));
    std::vector<int> keep;
    for (int j = nt - 1; j >= 0; --j)
      if (lam[j] > thr && std::isfinite(lam[j])) keep.push_back(j);
    const int nk = (int)keep.size();
    if (nk == 0) return 0;
    ADC_CUDA(cudaMemcpyAsync(rowsb.p, keep.data(), nk * sizeof(int), cudaMemcpyHostToDevice, ex.stream));
    k_lowdin<<<1, 256, 0, ex.stream>>>(Zs.c(), nt, w2.d(), (const int *)rowsb.p, nk, Ws.c());
    ADC_CHECK_LAUNCH();
    combine(ex, Ws.c(), nk, nt, nk, T.c(), N, N, C1(), C0(), Tn.c(), N);
    ADC_CUDA(cudaMemcpyAsync(T.c(), Tn.c(), (int64_t)nk * N * sizeof(cplx), cudaMemcpyDeviceToDevice, ex.stream));
    return nk;
  }

  // Rayleigh-Ritz on V[0:m]: w (host copy), Y and SY for the nroots lowest
  // (more columns only when a collapse asks for them: ritz_vectors), R for nroots
  int ycols = 0;  // columns of Y and SY formed from the current eigenvectors Cv
  void ritz_vectors(int nr) {
    nr = std::min(nr, std::min(m, krmax));
    if (nr <= ycols) return;
    // Y[r][n] = sum_i Cv[i][r] V[i][n], SY likewise from AV (columns ycols .. nr)
    combine(ex, Cv.c() + ycols, mmax, m, nr - ycols, V.c(), N, N, C1(), C0(), Y.c() + (int64_t)ycols * N, N);
    combine(ex, Cv.c() + ycols, mmax, m, nr - ycols, AV.c(), N, N, C1(), C0(), SY.c() + (int64_t)ycols * N, N);
    ycols = nr;
  }
  // root-specific step: the Ritz vector with the largest |<g|y_r>| (y_r = sum_i Cv[i][r] v_i)
  // becomes column 0 of Cv and w
  void pick_followed() {
    gram(ex, gfol.c(), N, 1, V.c(), N, m, N, C1(), ovl.c(), m);
    std::vector<cplx> s(m), cv((size_t)m * m);
    ADC_CUDA(cudaMemcpyAsync(s.data(), ovl.p, m * sizeof(cplx), cudaMemcpyDeviceToHost, ex.stream));
    ADC_CUDA(cudaMemcpy2DAsync(cv.data(), m * sizeof(cplx), Cv.p, mmax * sizeof(cplx), m * sizeof(cplx), m,
                               cudaMemcpyDeviceToHost, ex.stream));
    ADC_CUDA(cudaStreamSynchronize(ex.stream));
    int best = 0;
    double bo = -1.0;
    for (int r = 0; r < m; ++r) {
      double re = 0.0, im = 0.0;
      for (int i = 0; i < m; ++i) {
        const cplx a = cv[(size_t)i * m + r], b = s[i];
        re += a.x * b.x - a.y * b.y;
        im += a.x * b.y + a.y * b.x;
      }
      const double o2 = re * re + im * im;
      if (o2 > bo) { bo = o2; best = r; }
    }
    if (best != 0) {
      k_swap_first<<<1, 256, 0, ex.stream>>>(Cv.c(), mmax, m, w.d(), best);
      ADC_CHECK_LAUNCH();
    }
  }

  std::vector<double> ritz(int nr) {
    nr = std::min(std::max(nr, nroots), std::min(m, krmax));
    k_hermitize<<<(m * m + 255) / 256, 256, 0, ex.stream>>>(G.c(), mmax, m, H.c(), mmax);
    ADC_CHECK_LAUNCH();
    // the projected matrix: FP32 Jacobi start refined in FP64 (absolute accuracy
    // about n eps |omega|, which is what the Ritz pairs need)
    if (eigh_refined_fits(m)) eigh_refined(ex, H.c(), m, mmax, w.d(), Cv.c(), mmax);
    else jacobi_eigh(ex, H.c(), m, mmax, w.d(), Cv.c(), mmax, (int *)info.p);
    if (follow) pick_followed();
    ycols = 0;
    ritz_vectors(std::min(nr, nroots));
    k_residual<<<grid1d((int64_t)nroots * N, 256), 256, 0, ex.stream>>>(SY.c(), Y.c(), w.d(), nroots, N, R.c());
    ADC_CHECK_LAUNCH();
    std::vector<double> wh(m);
    ADC_CUDA(cudaMemcpyAsync(wh.data(), w.d(), m * sizeof(double), cudaMemcpyDeviceToHost, ex.stream));
    ADC_CUDA(cudaStreamSynchronize(ex.stream));
    return wh;
  }

  // V <- Y (orthonormal Ritz vectors), AV <- sigma64(Y) or SY, G <- Y^H AV
  void collapse(int nr, bool fp64_sigma) {
    ritz_vectors(nr);
    ADC_CUDA(cudaMemcpyAsync(V.c(), Y.c(), (int64_t)nr * N * sizeof(cplx), cudaMemcpyDeviceToDevice, ex.stream));
    if (fp64_sigma) apply_sigma(V.c(), AV.c(), nr, prec64);
    else
      ADC_CUDA(cudaMemcpyAsync(AV.c(), SY.c(), (int64_t)nr * N * sizeof(cplx), cudaMemcpyDeviceToDevice, ex.stream));
    m = 0;
    nb = 0;
    extend_projection(0, nr);
    m = nr;
    nb = fp64_sigma ? nr : 0;
  }
};

int davidson_run(adc_ctx *c, int nroots, double tol, int max_iter, int precision, const cplx *guess,
                 int64_t nguess, double *omega, cplx *Yout, double *err64, adc_stats *st_out, bool follow) {
  Timer total;
  const int64_t N = c->N;
  ADC_REQUIRE(nroots >= 1 && nroots <= N, ADC_ERR_ARG, "nroots out of range");
  ADC_REQUIRE(tol > 0.0, ADC_ERR_ARG, "tol must be positive");
  ADC_REQUIRE(precision == ADC_PREC_FP64 || precision == ADC_PREC_BF16X3 || precision == ADC_PREC_BF16X6,
              ADC_ERR_ARG, "precision");
  const int mixed = (precision == ADC_PREC_FP64) ? ADC_PREC_BF16X3 : precision;
  const int kb = std::max(nroots, c->opts.block);
  int mmax = c->opts.max_subspace > 0 ? c->opts.max_subspace : std::max(8 * kb, 40);
  mmax = (int)std::min<int64_t>(std::min<int64_t>(mmax, N), 1024);
  mmax = std::max(mmax, std::min<int>((int)N, nroots + 1));
  int krmax = std::max(2 * nroots, kb);
  if (c->opts.max_subspace <= 0) {
    // the operators of the products first (their transient buffers never meet
    // the subspace); then V and AV take what is left after the Davidson's
    // other vectors (T, Tn, R: nroots each; Y, SY: krmax each), an estimate of
    // the largest scratch of one product, and a margin of 8%
    if (c->kind == ADC_EE && c->ee)
      ee_prepare(c, precision == ADC_PREC_FP64 ? 0 : (mixed == ADC_PREC_BF16X6 ? 3 : 2),
                 c->opts.refine == ADC_PREC_SLICED);
    ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
    size_t fr = 0, tot = 0;
    ADC_CUDA(cudaMemGetInfo(&fr, &tot));
    double avail = (double)fr;
    if (c->ex.mem_limit > 0) avail = std::min(avail, (double)(c->ex.mem_limit - c->ex.mem_used));
    const double vec = (double)N * sizeof(cplx);
    const double scratch = sigma_scratch_bytes(c, kb);
    auto fit_of = [&](int kr) {
      return (int64_t)((0.92 * std::max(avail, 0.0) - (3.0 * nroots + 2.0 * kr) * vec - scratch) / (2.0 * vec));
    };
    int lo = (int)std::min<int64_t>(N, std::max(2 * nroots, kb) + kb);
    int64_t fit = fit_of(krmax);
    // short of memory: keep only the wanted roots at a collapse (thick restart
    // of nroots) and allow a subspace of nroots plus one block
    if (fit < lo) {
      krmax = nroots;
      lo = (int)std::min<int64_t>(N, nroots + kb);
      fit = fit_of(krmax);
    }
    if (fit < mmax) mmax = (int)std::max<int64_t>(fit, std::max(lo, std::min<int>((int)N, nroots + 1)));
  }
  krmax = std::min(mmax, krmax);
  ADC_REQUIRE(!follow || (nroots == 1 && guess && nguess >= 1), ADC_ERR_ARG,
              "root-specific Davidson: one root and a guess vector");
  Davidson d(c, nroots, mmax, krmax);
  if (follow) {
    d.follow = true;
    d.gfol = cbuf(c->ex, N);
    d.ovl = cbuf(c->ex, mmax);
    ADC_CUDA(cudaMemcpyAsync(d.gfol.p, guess, N * sizeof(cplx), cudaMemcpyDeviceToDevice, c->ex.stream));
  }
  // refinement products: FP64, or the sliced FP64-accurate tensor-core product
  if (precision != ADC_PREC_FP64 && c->opts.refine == ADC_PREC_SLICED) d.prec64 = ADC_PREC_SLICED;
  Exec &ex = c->ex;

  // ---- starting space
  int m0;
  ADC_REQUIRE(!(guess && nguess > 0) || nguess >= nroots, ADC_ERR_ARG, "need at least nroots guess vectors");
  if (guess && nguess > 0) {
    m0 = (int)std::min<int64_t>(nguess, mmax);
    ADC_CUDA(cudaMemcpyAsync(d.T.c(), guess, (int64_t)std::min<int64_t>(m0, nroots) * N * sizeof(cplx),
                             cudaMemcpyDeviceToDevice, ex.stream));
    m0 = std::min(m0, nroots);
  } else {
    m0 = (int)std::min<int64_t>(N, std::min(mmax - nroots, std::max(2 * nroots, kb)));
    m0 = std::max(m0, std::min<int>((int)N, nroots));
    std::vector<double> dh(N);
    ADC_CUDA(cudaMemcpyAsync(dh.data(), c->diag.d(), N * sizeof(double), cudaMemcpyDeviceToHost, ex.stream));
    ADC_CUDA(cudaStreamSynchronize(ex.stream));
    std::vector<int64_t> idx(N);
    std::iota(idx.begin(), idx.end(), 0);
    std::partial_sort(idx.begin(), idx.begin() + m0, idx.end(),
                      [&](int64_t a, int64_t b) { return dh[a] < dh[b] || (dh[a] == dh[b] && a < b); });
    DBuf ib(ex, m0 * sizeof(int64_t));
    ADC_CUDA(cudaMemcpyAsync(ib.p, idx.data(), m0 * sizeof(int64_t), cudaMemcpyHostToDevice, ex.stream));
    k_unit_vectors<<<m0, 256, 0, ex.stream>>>(d.V.c(), N, (const int64_t *)ib.p, m0);
    ADC_CHECK_LAUNCH();
    ADC_CUDA(cudaStreamSynchronize(ex.stream));
  }
  if (guess && nguess > 0) {
    // guesses go through the orthonormalisation into V
    d.m = 0;
    int acc = d.orthonormalise(m0);
    ADC_REQUIRE(acc > 0, ADC_ERR_ARG, "guess vectors are linearly dependent");
    ADC_CUDA(cudaMemcpyAsync(d.V.c(), d.T.c(), (int64_t)acc * N * sizeof(cplx), cudaMemcpyDeviceToDevice,
                             ex.stream));
    m0 = acc;
  }
  // phases: 0 mixed products; 1 FP64 base (the current Ritz vectors' products
  // in prec64, taken at each collapse) and mixed corrections; 2 the same with
  // the corrections in the intermediate sliced precision (only when the
  // refinement is sliced); 3 every product in prec64, the final phase
  const int prec_mid = (precision != ADC_PREC_FP64 && d.prec64 == ADC_PREC_SLICED) ? ADC_PREC_SLICED24 : -1;
  auto prec_of = [&](int ph) { return ph <= 1 ? mixed : (ph == 2 ? prec_mid : d.prec64); };
  auto next_phase = [&](int ph) { return ph == 0 ? 1 : (ph == 1 && prec_mid >= 0 ? 2 : 3); };
  int phase = (precision == ADC_PREC_FP64) ? 3 : 0;
  int prec_new = (phase == 3) ? ADC_PREC_FP64 : mixed;
  d.apply_sigma(d.V.c(), d.AV.c(), m0, prec_new);
  d.m = 0;
  d.nb = 0;
  d.extend_projection(0, m0);
  d.m = m0;

  std::vector<double> wh, rn(nroots, 0.0);
  bool converged = false;
  double best = 1e300;
  int since = 0;
  const int stall_window = 5;
  int refine_stalls = 0;
  int it = 0;
  for (it = 1; it <= max_iter; ++it) {
    const int kr = std::min(d.m, krmax);
    wh = d.ritz(kr);
    rn = d.row_norms(d.R.c(), nroots);
    double mx = *std::max_element(rn.begin(), rn.end());
    ADC_REQUIRE(std::isfinite(mx), ADC_ERR_NUMERIC, "non-finite residual norm in Davidson");
    if (c->opts.verbose)
      fprintf(stderr, "[davidson] it %d phase %d m %d nb %d max|r| %.3e w0 %.12f\n", it, phase, d.m, d.nb, mx, wh[0]);
    d.st.iterations = it;
    if (phase != 0) d.st.iterations_fp64++;
    if (mx < 0.7 * best) { best = mx; since = 0; }
    else ++since;
    if (mx <= tol) {
      if (phase == 3) { converged = true; break; }
      // accept only on FP64 residuals: collapse onto the wanted roots with sigma64 and re-check
      d.collapse(nroots, true);
      phase = std::max(phase, 1);
      wh = d.ritz(nroots);
      rn = d.row_norms(d.R.c(), nroots);
      mx = *std::max_element(rn.begin(), rn.end());
      if (c->opts.verbose) fprintf(stderr, "[davidson] fp64 check max|r| %.3e\n", mx);
      if (mx <= tol) { converged = true; break; }
      best = mx;
      since = 0;
    } else if (phase != 3 && since >= stall_window) {
      // stalled at the floor of the corrections' precision: FP64 base for the
      // current Ritz vectors; when the refinement itself keeps stalling, the
      // corrections go to the next precision (intermediate, then prec64)
      d.collapse(nroots, true);
      if (phase == 1) ++refine_stalls;
      if (phase == 0 || (phase == 1 && refine_stalls >= 2) || phase == 2) phase = next_phase(phase);
      best = 1e300;
      since = 0;
      continue;
    }
    // new correction vectors for the unconverged roots
    std::vector<int> rows;
    for (int r = 0; r < nroots; ++r)
      if (rn[r] > tol) rows.push_back(r);
    if (d.m + (int)rows.size() > d.mmax) {
      // with products of two precisions in the subspace, prec64 for the wanted roots
      const bool base = (phase == 1 || phase == 2);
      const int kc = base ? nroots : kr;
      d.collapse(kc, base);
      wh = d.ritz(kc);
    }
    ADC_CUDA(cudaMemcpyAsync(d.rowsb.p, rows.data(), rows.size() * sizeof(int), cudaMemcpyHostToDevice, ex.stream));
    if (c->opts.correction == 1) {
      const int nt = (int)rows.size();
      const int nseg = (int)std::max<int64_t>(1, std::min<int64_t>((608 + nt - 1) / nt, (N + 4095) / 4096));
      DBuf part(ex, (size_t)nt * nseg * 3 * sizeof(double));
      k_olsen_part<<<dim3(nseg, nt), 256, 0, ex.stream>>>(d.R.c(), d.Y.c(), d.w.d(), (const int *)d.rowsb.p,
                                                           c->diag.d(), N, part.d());
      ADC_CHECK_LAUNCH();
      DBuf ev = cbuf(ex, nt);
      k_olsen_fin<<<(nt + 31) / 32, 32, 0, ex.stream>>>(part.d(), nseg, nt, ev.c());
      ADC_CHECK_LAUNCH();
      k_olsen_apply<<<grid1d((int64_t)nt * N, 256), 256, 0, ex.stream>>>(
          d.R.c(), d.Y.c(), d.w.d(), (const int *)d.rowsb.p, c->diag.d(), ev.c(), nt, N, d.T.c());
      ADC_CHECK_LAUNCH();
    } else {
      k_precondition<<<grid1d((int64_t)rows.size() * N, 256), 256, 0, ex.stream>>>(
          d.R.c(), d.w.d(), (const int *)d.rowsb.p, c->diag.d(), (int64_t)rows.size(), N, d.T.c());
      ADC_CHECK_LAUNCH();
    }
    int na = d.orthonormalise((int)rows.size());
    if (na == 0) {
      // the preconditioned corrections lie in the subspace (an eigenvalue next
      // to a diagonal element of M): take the residuals themselves
      k_gather_rows<<<grid1d((int64_t)rows.size() * N, 256), 256, 0, ex.stream>>>(
          d.R.c(), (const int *)d.rowsb.p, (int64_t)rows.size(), N, d.T.c());
      ADC_CHECK_LAUNCH();
      na = d.orthonormalise((int)rows.size());
    }
    if (na == 0) {
      if (phase == 3) break;
      // no new direction at this precision: continue from an FP64 base, with
      // the corrections in the next precision
      d.collapse(nroots, true);
      phase = next_phase(phase);
      best = 1e300;
      since = 0;
      continue;
    }
    ADC_CUDA(cudaMemcpyAsync(d.V.c() + (int64_t)d.m * N, d.T.c(), (int64_t)na * N * sizeof(cplx),
                             cudaMemcpyDeviceToDevice, ex.stream));
    prec_new = prec_of(phase);
    d.apply_sigma_new(na, prec_new);
    d.extend_projection(d.m, na);
    d.m += na;
  }
  if (it > max_iter) it = max_iter;
  if (!converged && phase != 3) {
    // report FP64 residuals of the best vectors
    d.collapse(nroots, true);
    wh = d.ritz(nroots);
    rn = d.row_norms(d.R.c(), nroots);
  }
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
  for (int r = 0; r < nroots; ++r) {
    omega[r] = wh[r];
    if (err64) err64[r] = rn[r];
  }
  if (Yout)
    ADC_CUDA(cudaMemcpyAsync(Yout, d.Y.c(), (int64_t)nroots * N * sizeof(cplx), cudaMemcpyDeviceToDevice,
                             ex.stream));
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
  d.st.time_total_s = total.s();
  d.st.time_sigma_s = d.tsig;
  d.st.max_residual = *std::max_element(rn.begin(), rn.end());
  if (st_out) *st_out = d.st;
  return converged ? ADC_OK : ADC_ERR_NOCONV;
}

}  // namespace adc
