// C ABI of the library (declared in include/adc_gb300.h). Every entry point
// converts internal errors into negative return codes; nothing aborts.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ctx.cuh"
#include "tc_gemm.cuh"
#include "tc_slice.cuh"
#include "ee.cuh"

namespace adc {
void adjoint_ee(adc_ctx *c, const cplx *Y, const double *g_host, int64_t k, cplx *gB, double *geo, double *gev,
                double *gx);
void adjoint_ipea(adc_ctx *c, const cplx *Y, const double *g_host, int64_t k, cplx *gB, double *geo, double *gev,
                  double *gx);
}  // namespace adc

using namespace adc;

namespace {

thread_local std::string g_last_error;

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// device view of a caller input (copied when it lives on the host)
struct DevIn {
  DBuf buf;
  const void *p = nullptr;
  DevIn(Exec &ex, const void *src, size_t bytes) {
    if (!src || !bytes) return;
    if (is_device_ptr(src)) { p = src; return; }
    buf = DBuf(ex, bytes);
    ADC_CUDA(cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, ex.stream));
    p = buf.p;
  }
};

// device target for a caller output (copied back at finish() when on the host)
struct DevOut {
  DBuf buf;
  void *user = nullptr, *p = nullptr;
  size_t bytes = 0;
  bool host = false;
  DevOut(Exec &ex, void *dst, size_t b) : user(dst), bytes(b) {
    if (!dst || !b) return;
    if (is_device_ptr(dst)) { p = dst; return; }
    host = true;
    buf = DBuf(ex, b);
    p = buf.p;
  }
  void finish(Exec &ex) {
    if (host && user) ADC_CUDA(cudaMemcpyAsync(user, p, bytes, cudaMemcpyDeviceToHost, ex.stream));
  }
};

__device__ inline void atomic_max_nonneg(double *addr, double v) {
  atomicMax((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}

__global__ void k_herm_check(const cplx *B, int64_t Q, int64_t n, double *out) {
  const int64_t total = Q * n * n;
  double dev = 0.0, mag = 0.0;
  bool bad = false;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = idx % n, r = idx / n;
    int64_t p = r % n, Qi = r / n;
    cplx a = B[idx], b = B[(Qi * n + q) * n + p];
    if (!isfinite(a.x) || !isfinite(a.y)) bad = true;
    dev = fmax(dev, fmax(fabs(a.x - b.x), fabs(a.y + b.y)));
    mag = fmax(mag, fmax(fabs(a.x), fabs(a.y)));
  }
  if (bad) dev = 1e300;
  atomic_max_nonneg(out, dev);
  atomic_max_nonneg(out + 1, mag);
}

int fail(adc_ctx *c, const std::exception &e, int code) {
  if (c) c->err = e.what();
  g_last_error = e.what();
  return code;
}

#define ADC_API_TRY try {
#define ADC_API_CATCH(ctxp)                                           \
  }                                                                   \
  catch (const adc::Error &e) { return fail((ctxp), e, e.code); }     \
  catch (const std::bad_alloc &e) { return fail((ctxp), e, ADC_ERR_OOM); } \
  catch (const std::exception &e) { return fail((ctxp), e, ADC_ERR_CUDA); }

}  // namespace

adc_ctx::~adc_ctx() {
  release_tc(this);
  ee.reset();
  scratch.reset();
  t1.reset(); W.reset(); Glad.reset(); Lvv.reset(); diag.reset(); d2.reset(); Cpl.reset(); M11.reset();
  B.reset(); eo.reset(); ev.reset();
  if (ex.stream) cudaStreamSynchronize(ex.stream);
  if (own_stream && ex.stream) cudaStreamDestroy(ex.stream);
}

extern "C" {

int adc_opts_default(adc_opts *o) {
  if (!o) return ADC_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  o->precision = ADC_PREC_FP64;
  o->herm_tol = 1e-12;
  o->dd_order = 1;
  return ADC_OK;
}

int adc_init(adc_ctx **out, const adc_c128 *B, int64_t naux, const double *eps_occ, int64_t nocc,
             const double *eps_vir, int64_t nvir, int kind, int order, double x,
             const adc_opts *opts) {
  if (!out) return ADC_ERR_ARG;
  *out = nullptr;
  adc_ctx *c = nullptr;
  try {
    if (kind != ADC_IP && kind != ADC_EA && kind != ADC_EE) throw Error(ADC_ERR_ARG, "kind must be ADC_IP, ADC_EA or ADC_EE");
    if (order != 2 && order != 3) throw Error(ADC_ERR_ARG, "order must be 2 or 3");
    if (!B || !eps_occ || !eps_vir) throw Error(ADC_ERR_ARG, "NULL input");
    if (naux < 1 || nocc < 1 || nvir < 1) throw Error(ADC_ERR_ARG, "sizes must be positive");
    if (!std::isfinite(x)) throw Error(ADC_ERR_ARG, "x must be finite");
    if (kind == ADC_IP && nocc < 2) throw Error(ADC_ERR_ARG, "IP needs nocc >= 2");
    if (kind == ADC_EA && nvir < 2) throw Error(ADC_ERR_ARG, "EA needs nvir >= 2");
    c = new adc_ctx();
    if (opts) c->opts = *opts;
    else adc_opts_default(&c->opts);
    if (c->opts.herm_tol <= 0.0) c->opts.herm_tol = 1e-12;
    ADC_REQUIRE(c->opts.refine == ADC_PREC_FP64 || c->opts.refine == ADC_PREC_SLICED, ADC_ERR_ARG,
                "opts.refine: ADC_PREC_FP64 or ADC_PREC_SLICED");
    ADC_REQUIRE(c->opts.setup == ADC_PREC_FP64 || c->opts.setup == ADC_PREC_SLICED, ADC_ERR_ARG,
                "opts.setup: ADC_PREC_FP64 or ADC_PREC_SLICED");
    ADC_REQUIRE(c->opts.ee_vvvv >= -1 && c->opts.ee_vvvv <= 1, ADC_ERR_ARG, "opts.ee_vvvv: -1, 0 or 1");
    ADC_REQUIRE(c->opts.correction == 0 || c->opts.correction == 1, ADC_ERR_ARG, "opts.correction: 0 or 1");
    ADC_REQUIRE(c->opts.ladder >= -1 && c->opts.ladder <= 1, ADC_ERR_ARG, "opts.ladder: -1, 0 or 1");
    ADC_REQUIRE(c->opts.grouped_sigma == 0 || c->opts.grouped_sigma == -1, ADC_ERR_ARG,
                "opts.grouped_sigma: 0 or -1");
    c->kind = kind;
    c->order = order;
    c->x = (order == 3) ? x : 0.0;
    c->o = nocc; c->v = nvir; c->Q = naux; c->nmo = nocc + nvir;
    if (kind == ADC_IP) { c->n1 = nocc; c->n2 = npairs(nocc) * nvir; }
    else if (kind == ADC_EA) { c->n1 = nvir; c->n2 = nocc * npairs(nvir); }
    else { c->n1 = nocc * nvir; c->n2 = npairs(nocc) * npairs(nvir); }
    c->dd_order = (c->opts.dd_order == 0) ? 0 : 1;
    c->N = c->n1 + c->n2;
    c->ex.mem_limit = c->opts.mem_limit;
    ADC_CUDA(cudaGetDevice(&c->dev));
    if (c->opts.stream) {
      c->ex.stream = (cudaStream_t)c->opts.stream;
    } else {
      ADC_CUDA(cudaStreamCreateWithFlags(&c->ex.stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    Exec &ex = c->ex;
    ex.prof = (c->opts.profile != 0);
    // orbital energies
    std::vector<double> eo(nocc), ev(nvir);
    if (is_device_ptr(eps_occ)) ADC_CUDA(cudaMemcpy(eo.data(), eps_occ, nocc * 8, cudaMemcpyDeviceToHost));
    else std::memcpy(eo.data(), eps_occ, nocc * 8);
    if (is_device_ptr(eps_vir)) ADC_CUDA(cudaMemcpy(ev.data(), eps_vir, nvir * 8, cudaMemcpyDeviceToHost));
    else std::memcpy(ev.data(), eps_vir, nvir * 8);
    for (double e : eo) if (!std::isfinite(e)) throw Error(ADC_ERR_ARG, "non-finite eps_occ");
    for (double e : ev) if (!std::isfinite(e)) throw Error(ADC_ERR_ARG, "non-finite eps_vir");
    if (*std::max_element(eo.begin(), eo.end()) >= *std::min_element(ev.begin(), ev.end()))
      throw Error(ADC_ERR_ARG, "every occupied energy must lie below every virtual energy");
    c->eo = DBuf(ex, nocc * sizeof(double));
    c->ev = DBuf(ex, nvir * sizeof(double));
    ADC_CUDA(cudaMemcpyAsync(c->eo.p, eo.data(), nocc * 8, cudaMemcpyHostToDevice, ex.stream));
    ADC_CUDA(cudaMemcpyAsync(c->ev.p, ev.data(), nvir * 8, cudaMemcpyHostToDevice, ex.stream));
    // Cholesky vectors
    const int64_t nb = naux * c->nmo * c->nmo;
    c->B = cbuf(ex, nb);
    ADC_CUDA(cudaMemcpyAsync(c->B.p, B, nb * sizeof(cplx),
                             is_device_ptr(B) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ex.stream));
    {
      DBuf chk(ex, 2 * sizeof(double));
      fill_zero(ex, chk.p, chk.bytes);
      k_herm_check<<<grid1d(nb, 256) > 4096 ? 4096 : grid1d(nb, 256), 256, 0, ex.stream>>>(c->B.c(), naux,
                                                                                         c->nmo, chk.d());
      ADC_CHECK_LAUNCH();
      double h[2];
      ADC_CUDA(cudaMemcpyAsync(h, chk.p, sizeof(h), cudaMemcpyDeviceToHost, ex.stream));
      ADC_CUDA(cudaStreamSynchronize(ex.stream));
      if (!(h[0] <= c->opts.herm_tol * std::max(h[1], 1e-300)))
        throw Error(ADC_ERR_ARG, "B is not Hermitian in (p,q) (max deviation " + std::to_string(h[0]) +
                                     ", max |B| " + std::to_string(h[1]) + ")");
    }
    // the setup's large contractions as the sliced tensor-core product when asked for
    c->ex.sliced_bits = (c->opts.setup == ADC_PREC_SLICED) ? 48 : 0;
    c->ex.n_sliced = c->ex.n_fp64 = 0;
    c->ex.flops_sliced = c->ex.flops_fp64 = 0.0;
    {
      StageScope st(ex, "setup");
      if (kind == ADC_EE) setup_ee(c);
      else setup_operators(c);
    }
    c->ex.sliced_bits = 0;
    c->setup_n[0] = c->ex.n_sliced;
    c->setup_n[1] = c->ex.n_fp64;
    c->setup_flops[0] = c->ex.flops_sliced;
    c->setup_flops[1] = c->ex.flops_fp64;
    *out = c;
    return ADC_OK;
  } catch (const adc::Error &e) {
    g_last_error = e.what();
    delete c;
    return e.code;
  } catch (const std::bad_alloc &e) {
    g_last_error = e.what();
    delete c;
    return ADC_ERR_OOM;
  } catch (const std::exception &e) {
    g_last_error = e.what();
    delete c;
    return ADC_ERR_CUDA;
  }
}

int adc_dims(const adc_ctx *c, int64_t *n1, int64_t *n2) {
  if (!c) return ADC_ERR_STATE;
  if (n1) *n1 = c->n1;
  if (n2) *n2 = c->n2;
  return ADC_OK;
}

int adc_sigma(adc_ctx *c, const adc_c128 *X, adc_c128 *S, int64_t k, int precision) {
  if (!c) return ADC_ERR_STATE;
  if (k < 0 || (k > 0 && (!X || !S))) return ADC_ERR_ARG;
  if (precision != ADC_PREC_FP64 && precision != ADC_PREC_BF16X3 && precision != ADC_PREC_BF16X6 &&
      precision != ADC_PREC_SLICED && precision != ADC_PREC_SLICED24)
    return ADC_ERR_ARG;
  if (k == 0) return ADC_OK;
  ADC_API_TRY
  const size_t bytes = (size_t)k * c->N * sizeof(cplx);
  DevIn xin(c->ex, X, bytes);
  DevOut sout(c->ex, S, bytes);
  sigma(c, (const cplx *)xin.p, (cplx *)sout.p, k, precision);
  sout.finish(c->ex);
  if (sout.host || xin.buf.p) ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
  return ADC_OK;
  ADC_API_CATCH(c)
}

int adc_sigma_share(adc_ctx *c, const adc_c128 *X, adc_c128 *S, int64_t k, int64_t i0, int64_t i1,
                    int with_main) {
  if (!c) return ADC_ERR_STATE;
  if (k < 0 || (k > 0 && (!X || !S))) return ADC_ERR_ARG;
  ADC_API_TRY
  if (c->kind != ADC_EA) throw Error(ADC_ERR_UNSUPPORTED, "adc_sigma_share covers EA");
  if (i0 < 0 || i1 < i0 || i1 > c->o)
    throw Error(ADC_ERR_ARG, "adc_sigma_share: occupied range [" + std::to_string(i0) + ", " + std::to_string(i1) +
                                 ") outside [0, " + std::to_string(c->o) + ")");
  if (k == 0) return ADC_OK;
  const int64_t ls = c->n1 + (i1 - i0) * npairs(c->v);
  DevIn xin(c->ex, X, (size_t)k * c->N * sizeof(cplx));
  DevOut sout(c->ex, S, (size_t)k * ls * sizeof(cplx));
  sigma_fp64_share(c, (const cplx *)xin.p, (cplx *)sout.p, k, i0, i1, with_main != 0);
  sout.finish(c->ex);
  if (sout.host || xin.buf.p) ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
  return ADC_OK;
  ADC_API_CATCH(c)
}

int adc_diagonal(adc_ctx *c, double *diag) {
  if (!c) return ADC_ERR_STATE;
  if (!diag) return ADC_ERR_ARG;
  ADC_API_TRY
  ADC_CUDA(cudaMemcpyAsync(diag, c->diag.p, c->N * sizeof(double), cudaMemcpyDefault, c->ex.stream));
  ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
  return ADC_OK;
  ADC_API_CATCH(c)
}

int adc_main_block(adc_ctx *c, adc_c128 *M11) {
  if (!c) return ADC_ERR_STATE;
  if (!M11) return ADC_ERR_ARG;
  ADC_API_TRY
  ADC_CUDA(cudaMemcpyAsync(M11, c->M11.p, c->n1 * c->n1 * sizeof(cplx), cudaMemcpyDefault, c->ex.stream));
  ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
  return ADC_OK;
  ADC_API_CATCH(c)
}

int adc_davidson(adc_ctx *c, int nroots, double tol, int max_iter, int precision, const adc_c128 *guess,
                 int64_t nguess, double *omega, adc_c128 *Y, double *err64, adc_stats *st) {
  if (!c) return ADC_ERR_STATE;
  if (!omega || nroots < 1 || max_iter < 1) return ADC_ERR_ARG;
  ADC_API_TRY
  const size_t vb = (size_t)nroots * c->N * sizeof(cplx);
  DevIn gin(c->ex, guess, guess ? (size_t)nguess * c->N * sizeof(cplx) : 0);
  DevOut yout(c->ex, Y, Y ? vb : 0);
  std::vector<double> om(nroots), er(nroots);
  int rc = davidson_run(c, nroots, tol, max_iter, precision, (const cplx *)gin.p, guess ? nguess : 0,
                        om.data(), (cplx *)yout.p, er.data(), st);
  yout.finish(c->ex);
  ADC_CUDA(cudaMemcpyAsync(omega, om.data(), nroots * sizeof(double), cudaMemcpyDefault, c->ex.stream));
  if (err64) ADC_CUDA(cudaMemcpyAsync(err64, er.data(), nroots * sizeof(double), cudaMemcpyDefault, c->ex.stream));
  ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
  if (rc == ADC_ERR_NOCONV) c->err = "Davidson did not converge within max_iter";
  return rc;
  ADC_API_CATCH(c)
}

int adc_fns_density(adc_ctx *c, adc_c128 *D, double *eta, adc_c128 *V, double eta_crit, int64_t *n_keep,
                    adc_c128 *U, double *eps_new) {
  if (!c) return ADC_ERR_STATE;
  if (!n_keep) return ADC_ERR_ARG;
  ADC_API_TRY
  const int64_t v = c->v;
  DevOut dD(c->ex, D, D ? v * v * sizeof(cplx) : 0);
  DevOut dE(c->ex, eta, eta ? v * sizeof(double) : 0);
  DevOut dV(c->ex, V, V ? v * v * sizeof(cplx) : 0);
  DevOut dU(c->ex, U, U ? v * v * sizeof(cplx) : 0);
  DevOut dN(c->ex, eps_new, eps_new ? v * sizeof(double) : 0);
  if (dU.p) fill_zero(c->ex, dU.p, dU.bytes);
  if (dN.p) fill_zero(c->ex, dN.p, dN.bytes);
  int64_t nk = 0;
  fns_run(c, (cplx *)dD.p, (double *)dE.p, (cplx *)dV.p, eta_crit, &nk, (cplx *)dU.p, (double *)dN.p);
  dD.finish(c->ex); dE.finish(c->ex); dV.finish(c->ex); dU.finish(c->ex); dN.finish(c->ex);
  ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
  *n_keep = nk;
  return ADC_OK;
  ADC_API_CATCH(c)
}

int adc_fns_transform(adc_ctx *c, const adc_c128 *U, int64_t ldu, int64_t n_keep, adc_c128 *Bout) {
  if (!c) return ADC_ERR_STATE;
  if (!Bout || n_keep < 0 || n_keep > c->v || (n_keep > 0 && (!U || ldu < n_keep))) return ADC_ERR_ARG;
  ADC_API_TRY
  const int64_t n2 = c->o + n_keep;
  DevIn uin(c->ex, U, n_keep > 0 ? (size_t)c->v * ldu * sizeof(cplx) : 0);
  DevOut bout(c->ex, Bout, (size_t)c->Q * n2 * n2 * sizeof(cplx));
  fns_transform(c, (const cplx *)uin.p, ldu, n_keep, (cplx *)bout.p);
  bout.finish(c->ex);
  ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
  return ADC_OK;
  ADC_API_CATCH(c)
}

int adc_state_density(adc_ctx *c, const adc_c128 *y, adc_c128 *D) {
  if (!c) return ADC_ERR_STATE;
  if (!y || !D) return ADC_ERR_ARG;
  if (c->kind != ADC_EA && c->kind != ADC_EE) return ADC_ERR_UNSUPPORTED;
  ADC_API_TRY
  const int64_t v = c->v;
  DevIn yin(c->ex, y, (size_t)c->N * sizeof(cplx));
  DevOut dD(c->ex, D, (size_t)v * v * sizeof(cplx));
  state_density(c, (const cplx *)yin.p, (cplx *)dD.p);
  dD.finish(c->ex);
  ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
  return ADC_OK;
  ADC_API_CATCH(c)
}

int adc_ssfns_density(adc_ctx *c, const adc_c128 *y, double eta_crit, adc_c128 *D, double *eta, int64_t *n_keep,
                      adc_c128 *U, double *eps_new) {
  if (!c) return ADC_ERR_STATE;
  if (!y || !n_keep) return ADC_ERR_ARG;
  if (c->kind != ADC_EA && c->kind != ADC_EE) return ADC_ERR_UNSUPPORTED;
  ADC_API_TRY
  const int64_t v = c->v;
  DevIn yin(c->ex, y, (size_t)c->N * sizeof(cplx));
  DBuf Dst = cbuf(c->ex, v * v);
  state_density(c, (const cplx *)yin.p, Dst.c());
  DevOut dD(c->ex, D, D ? v * v * sizeof(cplx) : 0);
  DevOut dE(c->ex, eta, eta ? v * sizeof(double) : 0);
  DevOut dU(c->ex, U, U ? v * v * sizeof(cplx) : 0);
  DevOut dN(c->ex, eps_new, eps_new ? v * sizeof(double) : 0);
  if (dU.p) fill_zero(c->ex, dU.p, dU.bytes);
  if (dN.p) fill_zero(c->ex, dN.p, dN.bytes);
  int64_t nk = 0;
  fns_run(c, (cplx *)dD.p, (double *)dE.p, nullptr, eta_crit, &nk, (cplx *)dU.p, (double *)dN.p, Dst.c());
  dD.finish(c->ex); dE.finish(c->ex); dU.finish(c->ex); dN.finish(c->ex);
  ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
  *n_keep = nk;
  return ADC_OK;
  ADC_API_CATCH(c)
}

int adc_fns_vector(adc_ctx *c, const adc_c128 *y, const adc_c128 *U, int64_t ldu, int64_t n_keep, adc_c128 *g) {
  if (!c) return ADC_ERR_STATE;
  if (!y || !U || !g || n_keep < 1 || n_keep > c->v || ldu < n_keep) return ADC_ERR_ARG;
  if (c->kind != ADC_EA && c->kind != ADC_EE) return ADC_ERR_UNSUPPORTED;
  ADC_API_TRY
  DevIn yin(c->ex, y, (size_t)c->N * sizeof(cplx));
  DevIn uin(c->ex, U, (size_t)c->v * ldu * sizeof(cplx));
  DevOut gout(c->ex, g, (size_t)fns_dim(c->kind, c->o, n_keep) * sizeof(cplx));
  to_fns_basis(c, (const cplx *)yin.p, (const cplx *)uin.p, ldu, n_keep, (cplx *)gout.p);
  gout.finish(c->ex);
  ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
  return ADC_OK;
  ADC_API_CATCH(c)
}

int adc_davidson_follow(adc_ctx *c, const adc_c128 *guess, double tol, int max_iter, int precision, double *omega,
                        adc_c128 *Y, double *err64, adc_stats *st) {
  if (!c) return ADC_ERR_STATE;
  if (!guess || !omega || max_iter < 1) return ADC_ERR_ARG;
  ADC_API_TRY
  const int64_t N = c->N;
  DevIn gin(c->ex, guess, (size_t)N * sizeof(cplx));
  DevOut yout(c->ex, Y, Y ? (size_t)N * sizeof(cplx) : 0);
  double e = 0.0;
  int rc = davidson_run(c, 1, tol, max_iter, precision, (const cplx *)gin.p, 1, omega, (cplx *)yout.p, &e, st,
                        true);
  yout.finish(c->ex);
  ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
  if (err64) *err64 = e;
  if (rc == ADC_ERR_NOCONV) {
    c->err = "davidson: not converged within max_iter";
    g_last_error = c->err;
  }
  return rc;
  ADC_API_CATCH(c)
}

int adc_ssfns(const adc_c128 *B, int64_t naux, const double *eps_occ, int64_t nocc, const double *eps_vir,
              int64_t nvir, int kind, int order, double x, int nroots, double eta_crit, double tol, int max_iter,
              int precision, const adc_opts *opts, adc_ssfns_root *out) {
  if (!B || !eps_occ || !eps_vir || !out || nroots < 1 || max_iter < 1 || !(tol > 0.0)) return ADC_ERR_ARG;
  if (kind != ADC_EA && kind != ADC_EE) return ADC_ERR_UNSUPPORTED;
  if (order != 2 && order != 3) return ADC_ERR_ARG;
  try {
    return ssfns_run(B, naux, eps_occ, nocc, eps_vir, nvir, kind, order, x, nroots, eta_crit, tol, max_iter,
                     precision, opts, out);
  } catch (const adc::Error &e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc &e) {
    g_last_error = e.what();
    return ADC_ERR_OOM;
  } catch (const std::exception &e) {
    g_last_error = e.what();
    return ADC_ERR_CUDA;
  }
}

int adc_transition_density(adc_ctx *c, const adc_c128 *Y, int64_t k, adc_c128 *rho) {
  if (!c) return ADC_ERR_STATE;
  if (!Y || !rho || k < 1) return ADC_ERR_ARG;
  if (c->kind != ADC_EE) return ADC_ERR_UNSUPPORTED;
  ADC_API_TRY
  DevIn yin(c->ex, Y, (size_t)k * c->N * sizeof(cplx));
  DevOut rout(c->ex, rho, (size_t)k * c->nmo * c->nmo * sizeof(cplx));
  transition_density(c, (const cplx *)yin.p, k, (cplx *)rout.p);
  rout.finish(c->ex);
  ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
  return ADC_OK;
  ADC_API_CATCH(c)
}

int adc_state_pair_density(adc_ctx *c, const adc_c128 *YK, const adc_c128 *YL, int64_t k, adc_c128 *rho) {
  if (!c) return ADC_ERR_STATE;
  if (!YK || !YL || !rho || k < 1) return ADC_ERR_ARG;
  ADC_API_TRY
  DevIn kin(c->ex, YK, (size_t)k * c->N * sizeof(cplx));
  DevIn lin(c->ex, YL, (size_t)k * c->N * sizeof(cplx));
  DevOut rout(c->ex, rho, (size_t)k * c->nmo * c->nmo * sizeof(cplx));
  state_pair_density(c, (const cplx *)kin.p, (const cplx *)lin.p, k, (cplx *)rout.p);
  rout.finish(c->ex);
  ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
  return ADC_OK;
  ADC_API_CATCH(c)
}

int adc_spectroscopic_amplitudes(adc_ctx *c, const adc_c128 *Y, int64_t k, adc_c128 *x) {
  if (!c) return ADC_ERR_STATE;
  if (!Y || !x || k < 1) return ADC_ERR_ARG;
  if (c->kind != ADC_IP && c->kind != ADC_EA) return ADC_ERR_UNSUPPORTED;
  ADC_API_TRY
  DevIn yin(c->ex, Y, (size_t)k * c->N * sizeof(cplx));
  DevOut xout(c->ex, x, (size_t)k * c->nmo * sizeof(cplx));
  spectroscopic_amplitudes(c, (const cplx *)yin.p, k, (cplx *)xout.p);
  xout.finish(c->ex);
  ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
  return ADC_OK;
  ADC_API_CATCH(c)
}

int adc_excited_density(adc_ctx *c, const adc_c128 *Y, int64_t k, adc_c128 *rho) {
  if (!c) return ADC_ERR_STATE;
  if (!Y || !rho || k < 1) return ADC_ERR_ARG;
  ADC_API_TRY
  DevIn yin(c->ex, Y, (size_t)k * c->N * sizeof(cplx));
  DevOut rout(c->ex, rho, (size_t)k * c->nmo * c->nmo * sizeof(cplx));
  excited_density(c, (const cplx *)yin.p, k, (cplx *)rout.p);
  rout.finish(c->ex);
  ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
  return ADC_OK;
  ADC_API_CATCH(c)
}

int adc_cholesky(const double *V, int64_t n, double tau, int64_t max_rank, double *L, int64_t *pivots,
                 int64_t *rank) {
  if (!V || !L || !rank || n < 1 || max_rank < 1 || !(tau >= 0.0)) return ADC_ERR_ARG;
  Exec ex;
  try {
    ADC_CUDA(cudaStreamCreateWithFlags(&ex.stream, cudaStreamNonBlocking));
    int64_t r = 0;
    {
      DevIn vin(ex, V, (size_t)n * n * sizeof(double));
      DevOut lout(ex, L, (size_t)max_rank * n * sizeof(double));
      fill_zero(ex, lout.p, lout.bytes);
      r = cholesky_run(ex, (const double *)vin.p, n, tau, max_rank, (double *)lout.p, pivots);
      lout.finish(ex);
      ADC_CUDA(cudaStreamSynchronize(ex.stream));
    }
    cudaStreamDestroy(ex.stream);
    *rank = r;
    return ADC_OK;
  } catch (const adc::Error &e) {
    if (ex.stream) { cudaStreamSynchronize(ex.stream); cudaStreamDestroy(ex.stream); }
    g_last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc &e) {
    if (ex.stream) { cudaStreamSynchronize(ex.stream); cudaStreamDestroy(ex.stream); }
    g_last_error = e.what();
    return ADC_ERR_OOM;
  }
}

int adc_cholesky_mo(const double *L, int64_t rank, int64_t nao, const adc_c128 *C, int64_t nmo, adc_c128 *B) {
  if (!L || !C || !B || rank < 1 || nao < 1 || nmo < 1) return ADC_ERR_ARG;
  Exec ex;
  try {
    ADC_CUDA(cudaStreamCreateWithFlags(&ex.stream, cudaStreamNonBlocking));
    {
      DevIn lin(ex, L, (size_t)rank * nao * nao * sizeof(double));
      DevIn cin(ex, C, (size_t)nao * nmo * sizeof(cplx));
      DevOut bout(ex, B, (size_t)rank * nmo * nmo * sizeof(cplx));
      cholesky_mo(ex, (const double *)lin.p, rank, nao, (const cplx *)cin.p, nmo, (cplx *)bout.p);
      bout.finish(ex);
      ADC_CUDA(cudaStreamSynchronize(ex.stream));
    }
    cudaStreamDestroy(ex.stream);
    return ADC_OK;
  } catch (const adc::Error &e) {
    if (ex.stream) { cudaStreamSynchronize(ex.stream); cudaStreamDestroy(ex.stream); }
    g_last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc &e) {
    if (ex.stream) { cudaStreamSynchronize(ex.stream); cudaStreamDestroy(ex.stream); }
    g_last_error = e.what();
    return ADC_ERR_OOM;
  }
}

int adc_sigma_adjoint(adc_ctx *c, const adc_c128 *Y, const double *gomega, int64_t nroots, adc_c128 *gB,
                      double *geps_occ, double *geps_vir, double *gx) {
  if (!c) return ADC_ERR_STATE;
  if (!Y || !gomega || nroots < 1 || !gB || !geps_occ || !geps_vir || !gx) return ADC_ERR_ARG;
  ADC_API_TRY
  for (int64_t r = 0; r < nroots; ++r)
    ADC_REQUIRE(std::isfinite(gomega[r]), ADC_ERR_ARG, "adc_sigma_adjoint: non-finite gomega");
  const int64_t nb = c->Q * c->nmo * c->nmo;
  DevIn yin(c->ex, Y, (size_t)nroots * c->N * sizeof(cplx));
  DevOut gbo(c->ex, gB, (size_t)nb * sizeof(cplx));
  DevOut geo(c->ex, geps_occ, (size_t)c->o * sizeof(double));
  DevOut gev(c->ex, geps_vir, (size_t)c->v * sizeof(double));
  fill_zero(c->ex, gbo.p, nb * sizeof(cplx));
  fill_zero(c->ex, geo.p, c->o * sizeof(double));
  fill_zero(c->ex, gev.p, c->v * sizeof(double));
  double gxh = 0.0;
  if (c->kind == ADC_EE)
    adjoint_ee(c, (const cplx *)yin.p, gomega, nroots, (cplx *)gbo.p, (double *)geo.p, (double *)gev.p, &gxh);
  else
    adjoint_ipea(c, (const cplx *)yin.p, gomega, nroots, (cplx *)gbo.p, (double *)geo.p, (double *)gev.p, &gxh);
  gbo.finish(c->ex);
  geo.finish(c->ex);
  gev.finish(c->ex);
  ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
  *gx = gxh;
  return ADC_OK;
  ADC_API_CATCH(c)
}

int adc_sync(adc_ctx *c) {
  if (!c) return ADC_ERR_STATE;
  cudaError_t e = cudaStreamSynchronize(c->ex.stream);
  if (e != cudaSuccess) {
    c->err = cudaGetErrorString(e);
    return ADC_ERR_CUDA;
  }
  return ADC_OK;
}

void adc_free(adc_ctx *c) { delete c; }

const char *adc_strerror(int code) {
  switch (code) {
    case ADC_OK: return "ADC_OK";
    case ADC_ERR_ARG: return "ADC_ERR_ARG: invalid argument";
    case ADC_ERR_OOM: return "ADC_ERR_OOM: out of device memory";
    case ADC_ERR_CUDA: return "ADC_ERR_CUDA: CUDA runtime error";
    case ADC_ERR_NOCONV: return "ADC_ERR_NOCONV: Davidson did not converge";
    case ADC_ERR_TIMEOUT: return "ADC_ERR_TIMEOUT: bounded device wait gave up";
    case ADC_ERR_UNSUPPORTED: return "ADC_ERR_UNSUPPORTED: combination not built";
    case ADC_ERR_STATE: return "ADC_ERR_STATE: context not usable";
    case ADC_ERR_NUMERIC: return "ADC_ERR_NUMERIC: NaN or Inf encountered";
    default: return "unknown ADC error code";
  }
}

const char *adc_last_error(const adc_ctx *c) {
  if (c && !c->err.empty()) return c->err.c_str();
  return g_last_error.c_str();
}

}  // extern "C"
