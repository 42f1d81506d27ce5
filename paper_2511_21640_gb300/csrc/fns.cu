// Frozen natural spinors from the MP2 virtual density (Sec. 2.4, Eqs. 25-30),
// optionally plus a state density (Eq. 31, state-specific natural spinors).
//   Eq. 25: D_ab = 1/2 sum_cij <ac||ij><ij||bc> / (eps_ij^ac eps_ij^bc)
//               = 1/2 sum_ijc t_ij^ac conj(t_ij^bc)
//   Eq. 26: D V = V eta (eta descending);  Eq. 27: keep eta_i >= eta_crit
//   Eq. 28-29: F~ = V~^H diag(eps_vir) V~,  F~ Z~ = Z~ eps~
//   Eq. 30: U = V~ Z~
#include "ctx.cuh"
#include "eig.cuh"

namespace adc {

namespace {
// reverse the column order (ascending -> descending) of V and w
__global__ void k_reverse(const double *w, const cplx *V, int n, double *wo, cplx *Vo) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n) wo[idx] = w[n - 1 - idx];
  if (idx < n * n) {
    int r = idx / n, col = idx % n;
    Vo[r * n + col] = V[r * n + (n - 1 - col)];
  }
}
}  // namespace

// Dadd (device, v x v, or null) is added to the MP2 density before Eq. 26: the
// state density of a root for the state-specific natural spinors (Eq. 31)
void fns_run(adc_ctx *c, cplx *D, double *eta, cplx *Vout, double eta_crit, int64_t *n_keep, cplx *U,
             double *eps_new, const cplx *Dadd) {
  Exec &ex = c->ex;
  const int64_t o = c->o, v = c->v;
  TV t1 = TV::dense(c->t1.c(), {o, o, v, v});
  DBuf Db = cbuf(ex, v * v);
  einsum(ex, CR(0.5), t1, "ijac", t1.cj(), "ijbc", C0(), TV::dense(Db.c(), {v, v}), "ab");
  if (Dadd) zaxpby(ex, v * v, C1(), Dadd, C1(), Db.c());
  if (D) ADC_CUDA(cudaMemcpyAsync(D, Db.c(), v * v * sizeof(cplx), cudaMemcpyDeviceToDevice, ex.stream));
  DBuf A = cbuf(ex, v * v), Vasc = cbuf(ex, v * v), Vd = cbuf(ex, v * v);
  DBuf wasc(ex, v * sizeof(double)), wd(ex, v * sizeof(double)), info(ex, 16);
  ADC_CUDA(cudaMemcpyAsync(A.c(), Db.c(), v * v * sizeof(cplx), cudaMemcpyDeviceToDevice, ex.stream));
  jacobi_eigh(ex, A.c(), (int)v, (int)v, wasc.d(), Vasc.c(), (int)v, (int *)info.p);
  k_reverse<<<grid1d(v * v, 256), 256, 0, ex.stream>>>(wasc.d(), Vasc.c(), (int)v, wd.d(), Vd.c());
  ADC_CHECK_LAUNCH();
  std::vector<double> wh(v);
  ADC_CUDA(cudaMemcpyAsync(wh.data(), wd.d(), v * sizeof(double), cudaMemcpyDeviceToHost, ex.stream));
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
  int64_t nk = 0;
  while (nk < v && wh[nk] >= eta_crit) ++nk;
  *n_keep = nk;
  if (eta) ADC_CUDA(cudaMemcpyAsync(eta, wd.d(), v * sizeof(double), cudaMemcpyDeviceToDevice, ex.stream));
  if (Vout) ADC_CUDA(cudaMemcpyAsync(Vout, Vd.c(), v * v * sizeof(cplx), cudaMemcpyDeviceToDevice, ex.stream));
  if (nk > 0 && (U || eps_new)) {
    // F~ = V~^H diag(eps) V~ : scale rows of V~ by eps, then V~^H (eps V~)
    DBuf EV = cbuf(ex, v * nk), F = cbuf(ex, nk * nk), Z = cbuf(ex, nk * nk);
    DBuf ew(ex, nk * sizeof(double));
    {
      // EV[a][k] = eps_a V~[a][k], as diag(eps) times V~
      DBuf Dg = cbuf(ex, v * v);
      fill_zero(ex, Dg.p, Dg.bytes);
      add_diag(ex, Dg.c(), c->ev.d(), v, 1.0);
      zgemm(ex, v, nk, v, 1, C1(), Dg.c(), 0, v, 1, false, Vd.c(), 0, v, 1, false, C0(), EV.c(), 0, nk, 1);
    }
    // F[k][l] = sum_a conj(V~[a][k]) EV[a][l]
    zgemm(ex, nk, nk, v, 1, C1(), Vd.c(), 0, 1, v, true, EV.c(), 0, nk, 1, false, C0(), F.c(), 0, nk, 1);
    jacobi_eigh(ex, F.c(), (int)nk, (int)nk, ew.d(), Z.c(), (int)nk, (int *)info.p);
    if (eps_new) ADC_CUDA(cudaMemcpyAsync(eps_new, ew.d(), nk * sizeof(double), cudaMemcpyDeviceToDevice, ex.stream));
    if (U) {
      // U[a][l] = sum_k V~[a][k] Z[k][l], written with leading dimension v
      zgemm(ex, v, nk, nk, 1, C1(), Vd.c(), 0, v, 1, false, Z.c(), 0, nk, 1, false, C0(), U, 0, v, 1);
    }
  }
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
}

// B' in the truncated basis: oo copied, ov = B_ov U, vo = U^H B_vo, vv = U^H B_vv U
void fns_transform(adc_ctx *c, const cplx *U, int64_t ldu, int64_t nk, cplx *Bout) {
  Exec &ex = c->ex;
  const int64_t o = c->o, v = c->v, Q = c->Q, nmo = c->nmo, n2 = o + nk;
  const cplx *B = c->B.c();
  const int64_t sQ = nmo * nmo, sQo = n2 * n2;
  // oo block: one strided 2-D copy per Cholesky vector
  for (int64_t q = 0; q < Q; ++q)
    ADC_CUDA(cudaMemcpy2DAsync(Bout + q * sQo, n2 * sizeof(cplx), B + q * sQ, nmo * sizeof(cplx), o * sizeof(cplx),
                               o, cudaMemcpyDeviceToDevice, ex.stream));
  if (nk == 0) return;
  // ov: Bout[Q][i][o+l] = sum_a B[Q][i][o+a] U[a][l]
  zgemm(ex, o, nk, v, Q, C1(), B + o, sQ, nmo, 1, false, U, 0, ldu, 1, false, C0(), Bout + o, sQo, n2, 1);
  // vo: Bout[Q][o+l][i] = sum_a conj(U[a][l]) B[Q][o+a][i]
  zgemm(ex, nk, o, v, Q, C1(), U, 0, 1, ldu, true, B + o * nmo, sQ, nmo, 1, false, C0(), Bout + o * n2, sQo, n2, 1);
  // vv: T[Q][a][m] = sum_b B[Q][o+a][o+b] U[b][m]; Bout[Q][o+l][o+m] = sum_a conj(U[a][l]) T[Q][a][m]
  DBuf T = cbuf(ex, Q * v * nk);
  zgemm(ex, v, nk, v, Q, C1(), B + o * nmo + o, sQ, nmo, 1, false, U, 0, ldu, 1, false, C0(), T.c(), v * nk, nk, 1);
  zgemm(ex, nk, nk, v, Q, C1(), U, 0, 1, ldu, true, T.c(), v * nk, nk, 1, false, C0(), Bout + o * n2 + o, sQo, n2, 1);
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
}

}  // namespace adc
