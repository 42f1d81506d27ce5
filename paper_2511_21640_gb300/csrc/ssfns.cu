// State-specific frozen natural spinors for EA and EE (Sec. 2.4, Eqs. 31-32).
//
// For root k of the canonical ADC(2) problem with eigenvector y, the state's
// virtual density is that of the excited configurations weighted by y (the
// zeroth-order intermediate states), D_ab = <Psi| a+_b a_a |Psi>, the index
// order of the MP2 density of Eq. 25:
//   EA  D_ab = y_a conj(y_b) + sum_{j,c} Y_jac conj(Y_jbc)
//   EE  D_ab = sum_i y_ia conj(y_ib) + 1/2 sum_{ijc} Y_ijac conj(Y_ijbc)
// (Y: the doubles as full antisymmetric arrays). Eq. 31 adds it to the MP2
// density; Eqs. 26-30 then give U = V~ Z~ and the semicanonical energies, and
// the Cholesky vectors are rotated into the truncated basis. The canonical
// eigenvector is carried over through the virtual creation operators,
// y'_a' = sum_a conj(U_aa') y_a on every virtual index, and is the guess of
// the root-specific solves (davidson_run with follow) of ADC(2) and of the
// target order in the new basis. Eq. 32: omega_corrected = omega_fns +
// omega2_canonical - omega2_fns.
#include <vector>

#include "ctx.cuh"

namespace adc {

void state_density(adc_ctx *c, const cplx *y, cplx *D) {
  Exec &ex = c->ex;
  const int64_t o = c->o, v = c->v, n1 = c->n1;
  ADC_REQUIRE(c->kind == ADC_EA || c->kind == ADC_EE, ADC_ERR_UNSUPPORTED, "state density: EA or EE");
  TV Dv = TV::dense(D, {v, v});
  if (c->kind == ADC_EA) {
    // D[a][b] = y_a conj(y_b): a product over an inner size of one
    zgemm(ex, v, v, 1, 1, C1(), y, 0, 1, 1, false, y, 0, 1, 1, true, C0(), D, 0, v, 1);
    const int64_t pv = npairs(v);
    if (pv > 0) {
      DBuf Yf = cbuf(ex, o * v * v);
      pair_unpack(ex, y + n1, 1, o, 0, pv, v, 1, Yf.c());
      TV Y = TV::dense(Yf.c(), {o, v, v});
      einsum(ex, C1(), Y, "jac", Y.cj(), "jbc", C1(), Dv, "ab");
    }
  } else {
    TV y1(const_cast<cplx *>(y), {o, v}, {v, 1});
    einsum(ex, C1(), y1, "ia", y1.cj(), "ib", C0(), Dv, "ab");
    const int64_t po = npairs(o), pv = npairs(v);
    if (po > 0 && pv > 0) {
      DBuf half = cbuf(ex, po * v * v), Yf = cbuf(ex, o * o * v * v);
      pair_unpack(ex, y + n1, 1, po, 0, pv, v, 1, half.c());
      pair_unpack(ex, half.c(), 1, 1, po * v * v, 0, o, v * v, Yf.c());
      TV Y = TV::dense(Yf.c(), {o, o, v, v});
      einsum(ex, CR(0.5), Y, "ijac", Y.cj(), "ijbc", C1(), Dv, "ab");
    }
  }
}

int64_t fns_dim(int kind, int64_t o, int64_t nk) {
  return kind == ADC_EA ? nk + o * npairs(nk) : o * nk + npairs(o) * npairs(nk);
}

void to_fns_basis(adc_ctx *c, const cplx *y, const cplx *U, int64_t ldu, int64_t nk, cplx *g) {
  Exec &ex = c->ex;
  const int64_t o = c->o, v = c->v, n1 = c->n1, pnk = npairs(nk);
  ADC_REQUIRE(c->kind == ADC_EA || c->kind == ADC_EE, ADC_ERR_UNSUPPORTED, "basis transformation: EA or EE");
  ADC_REQUIRE(nk >= 1 && nk <= v && ldu >= nk, ADC_ERR_ARG, "basis transformation: n_keep");
  TV Uc(const_cast<cplx *>(U), {v, nk}, {ldu, 1}, true);
  if (c->kind == ADC_EA) {
    // g[A] = sum_a conj(U[a][A]) y[a]
    zgemm(ex, nk, 1, v, 1, C1(), U, 0, 1, ldu, true, y, 0, 1, 1, false, C0(), g, 0, 1, 1);
    const int64_t pv = npairs(v);
    if (pnk > 0) {
      DBuf Yf = cbuf(ex, o * v * v), G1 = cbuf(ex, o * nk * v), G = cbuf(ex, o * nk * nk);
      if (pv > 0) pair_unpack(ex, y + n1, 1, o, 0, pv, v, 1, Yf.c());
      else fill_zero(ex, Yf.p, Yf.bytes);
      einsum(ex, C1(), Uc, "aA", TV::dense(Yf.c(), {o, v, v}), "jab", C0(), TV::dense(G1.c(), {o, nk, v}), "jAb");
      einsum(ex, C1(), Uc, "bB", TV::dense(G1.c(), {o, nk, v}), "jAb", C0(), TV::dense(G.c(), {o, nk, nk}), "jAB");
      pair_pack(ex, G.c(), 0, nk * nk, nk, 1, 0, 0.0, 1, o, nk, 1, g + nk, 0, pnk, C1(), C0());
    }
  } else {
    // g[i][A] = sum_a y[i][a] conj(U[a][A])
    zgemm(ex, o, nk, v, 1, C1(), y, 0, v, 1, false, U, 0, ldu, 1, true, C0(), g, 0, nk, 1);
    const int64_t po = npairs(o), pv = npairs(v);
    if (po > 0 && pnk > 0) {
      DBuf half = cbuf(ex, po * v * v), Yf = cbuf(ex, o * o * v * v);
      if (pv > 0) {
        pair_unpack(ex, y + n1, 1, po, 0, pv, v, 1, half.c());
        pair_unpack(ex, half.c(), 1, 1, po * v * v, 0, o, v * v, Yf.c());
      } else {
        fill_zero(ex, Yf.p, Yf.bytes);
      }
      half.reset();
      DBuf G1 = cbuf(ex, o * o * nk * v), G = cbuf(ex, o * o * nk * nk), P1 = cbuf(ex, o * o * pnk);
      einsum(ex, C1(), Uc, "aA", TV::dense(Yf.c(), {o, o, v, v}), "ijab", C0(),
             TV::dense(G1.c(), {o, o, nk, v}), "ijAb");
      einsum(ex, C1(), Uc, "bB", TV::dense(G1.c(), {o, o, nk, v}), "ijAb", C0(),
             TV::dense(G.c(), {o, o, nk, nk}), "ijAB");
      pair_pack(ex, G.c(), 0, nk * nk, nk, 1, 0, 0.0, 1, o * o, nk, 1, P1.c(), 0, pnk, C1(), C0());
      pair_pack(ex, P1.c(), 0, 0, o * pnk, pnk, 1, 0.0, 1, 1, o, pnk, g + o * nk, 0, 0, C1(), C0());
    }
  }
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
}

namespace {
struct CtxGuard {
  adc_ctx *c = nullptr;
  ~CtxGuard() { adc_free(c); }
};
}  // namespace

int ssfns_run(const adc_c128 *B, int64_t naux, const double *eps_occ, int64_t nocc, const double *eps_vir,
              int64_t nvir, int kind, int order, double x, int nroots, double eta_crit, double tol, int max_iter,
              int precision, const adc_opts *opts, adc_ssfns_root *out) {
  ADC_REQUIRE(kind == ADC_EA || kind == ADC_EE, ADC_ERR_UNSUPPORTED, "state-specific natural spinors: EA or EE");
  CtxGuard can;
  int rc = adc_init(&can.c, B, naux, eps_occ, nocc, eps_vir, nvir, kind, 2, 0.0, opts);
  if (rc != ADC_OK) return rc;
  adc_ctx *c = can.c;
  Exec &ex = c->ex;
  const int64_t N = c->N, o = c->o, v = c->v;
  ADC_REQUIRE(nroots >= 1 && nroots <= N, ADC_ERR_ARG, "nroots out of range");
  // canonical ADC(2) roots and vectors
  DBuf Yc = cbuf(ex, (int64_t)nroots * N);
  std::vector<double> w2(nroots), e2(nroots);
  adc_stats st{};
  rc = davidson_run(c, nroots, tol, max_iter, precision, nullptr, 0, w2.data(), Yc.c(), e2.data(), &st);
  if (rc != ADC_OK && rc != ADC_ERR_NOCONV) return rc;
  const int rc_can = rc;
  DBuf Dst = cbuf(ex, v * v), U = cbuf(ex, v * v), eta(ex, v * sizeof(double)), epsn(ex, v * sizeof(double));
  for (int k = 0; k < nroots; ++k) {
    adc_ssfns_root &r = out[k];
    r = adc_ssfns_root{};
    r.omega2_canonical = w2[k];
    r.status = rc_can;
    // Eq. 31 and Eqs. 26-30
    state_density(c, Yc.c() + (int64_t)k * N, Dst.c());
    fill_zero(ex, U.p, U.bytes);
    int64_t nk = 0;
    fns_run(c, nullptr, eta.d(), nullptr, eta_crit, &nk, U.c(), epsn.d(), Dst.c());
    r.n_keep = nk;
    if (nk < (kind == ADC_EA ? 2 : 1)) {
      r.status = ADC_ERR_ARG;  // too few natural spinors kept for this kind
      continue;
    }
    const int64_t n2 = o + nk;
    DBuf Bk = cbuf(ex, naux * n2 * n2);
    fns_transform(c, U.c(), v, nk, Bk.c());
    DBuf g = cbuf(ex, fns_dim(kind, o, nk));
    to_fns_basis(c, Yc.c() + (int64_t)k * N, U.c(), v, nk, g.c());
    // root-specific solves in the truncated basis: ADC(2), then the target order
    for (int pass = 0; pass < 2; ++pass) {
      CtxGuard t;
      const int ord = pass == 0 ? 2 : order;
      rc = adc_init(&t.c, (const adc_c128 *)Bk.c(), naux, c->eo.d(), o, epsn.d(), nk, kind, ord,
                    pass == 0 ? 0.0 : x, opts);
      if (rc != ADC_OK) return rc;
      double w = 0.0, e = 0.0;
      adc_stats s2{};
      rc = davidson_run(t.c, 1, tol, max_iter, precision, g.c(), 1, &w, nullptr, &e, &s2, true);
      if (rc != ADC_OK && rc != ADC_ERR_NOCONV) return rc;
      if (rc != ADC_OK) r.status = rc;
      if (pass == 0) {
        r.omega2_fns = w;
      } else {
        r.omega_fns = w;
        r.err64 = e;
      }
    }
    r.omega_corrected = r.omega_fns + r.omega2_canonical - r.omega2_fns;  // Eq. 32
  }
  return ADC_OK;
}

}  // namespace adc
