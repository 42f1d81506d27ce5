// Adjoint of the EE-ADC secular matrix: gradients of sum_r g_r y_r^H M y_r
// with respect to the Cholesky vectors B, the orbital energies and x. For
// normalised eigenvectors y_r (Eq. 10) this is sum_r g_r d omega_r (the
// Hellmann-Feynman theorem), i.e. the backward pass of the roots.
//
// With C = sum_r g_r y_r^H M y_r written as the sum of the term tables of
// ee.cu (singles block through the density rho = sum_r g_r conj(y1_r) y1_r^T,
// coupling and doubles block through the vectors themselves), every tensor T
// of the tables receives G_T = dC/d conj(T) + conj(dC/dT) (ee.cu's
// eval_terms_grad), the gradient in the convention d/dRe + i d/dIm. The
// coupling enters M twice (M_SD and M_DS = M_SD^H), so its share is doubled.
// The amplitudes are then differentiated back through their definitions
// (t1 = <ab||ij>/D, the second-order doubles and singles as tables over
// <pq||rs> and t1, divided by their denominators), and every integral block
// <pq||rs> = sum_Q (B_pr B_qs - B_ps B_qr) (Eq. 43) is contracted back onto B.
// Intermediates of the setup (K1, S2, S3, Y3) are recomputed, not stored.
#include <map>

#include "ctx.cuh"
#include "ee.cuh"
#include "terms.cuh"

namespace adc {

namespace {

__device__ __forceinline__ double vdot_re(cplx a, cplx b) { return a.x * b.x - a.y * b.y; }  // Re(a b)

// out[z][p] = g[z] conj(Y[z][p]) for p < n, rows of Y at pitch ld
__global__ void k_scale_conj_rows(const cplx *Y, int64_t ld, int64_t k, int64_t n, const double *g, cplx *out) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < k * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t z = idx / n, p = idx - z * n;
    const cplx y = Y[z * ld + p];
    out[idx] = cmake(g[z] * y.x, -g[z] * y.y);
  }
}

// acc[P] for P = (i, a): Re rho[P][P] + (col[P] - row[P]) / 2, with
// row[P] = sum_Q Re(rho S)[P][Q], col[P] = sum_Q Re(rho S)[Q][P]
// (S = S2 + x S3): the derivative of sum rho o (diag(eps_a - eps_i) + W o S)
// with respect to eps_a (and minus it with respect to eps_i).
__global__ void k_rowsum_re(const cplx *A, const cplx *Bm, int64_t n, double *row) {
  __shared__ double red[32];
  const int64_t r = blockIdx.x;
  double s = 0.0;
  for (int64_t q = threadIdx.x; q < n; q += blockDim.x) s += vdot_re(A[r * n + q], Bm[r * n + q]);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) row[r] = s;
  }
}
__global__ void k_colsum_re(const cplx *A, const cplx *Bm, int64_t n, double *col) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t p = 0; p < n; ++p) s += vdot_re(A[p * n + q], Bm[p * n + q]);
    col[q] = s;
  }
}
// geo[i] -= sum_a acc[ia], gev[a] += sum_i acc[ia], acc = Re rho_PP + (col - row)/2
__global__ void k_eps_from_singles(const cplx *rho, const double *row, const double *col, int64_t o, int64_t v,
                                   double *geo, double *gev) {
  const int64_t n1 = o * v;
  for (int64_t t = threadIdx.x; t < o + v; t += blockDim.x) {
    double s = 0.0;
    if (t < o) {
      for (int64_t a = 0; a < v; ++a) {
        const int64_t P = t * v + a;
        s -= rho[P * n1 + P].x + 0.5 * (col[P] - row[P]);
      }
      geo[t] += s;
    } else {
      const int64_t a = t - o;
      for (int64_t i = 0; i < o; ++i) {
        const int64_t P = i * v + a;
        s += rho[P * n1 + P].x + 0.5 * (col[P] - row[P]);
      }
      gev[a] += s;
    }
  }
}

// out[P][Q] = s * W[P][Q] * R[P][Q] (+ out if accumulate), W_ia,jb = ((eps_b - eps_j) - (eps_a - eps_i)) / 2
__global__ void k_wmul(const cplx *R, const double *eo, const double *ev, int64_t o, int64_t v, double s,
                       int accumulate, cplx *out) {
  const int64_t n1 = o * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n1 * n1;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = idx % n1, row = idx / n1;
    const int64_t i = row / v, a = row % v, j = col / v, b = col % v;
    const double w = s * 0.5 * ((ev[b] - eo[j]) - (ev[a] - eo[i]));
    cplx r = cmake(w * R[idx].x, w * R[idx].y);
    if (accumulate) r = cadd(r, out[idx]);
    out[idx] = r;
  }
}

// *out += s Re sum_i a[i] b[i]
__global__ void k_dot_re(const cplx *a, const cplx *b, int64_t n, double s, double *out) {
  __shared__ double red[32];
  double t = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    t += vdot_re(a[i], b[i]);
  for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x < 32) {
    t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    if (threadIdx.x == 0) atomicAdd(out, s * t);
  }
}

// dst[z][k][l][c][d] = src * (eps_c + eps_d - eps_k - eps_l)
__global__ void k_dk(const cplx *src, const double *eo, const double *ev, int64_t k, int64_t o, int64_t v,
                     cplx *dst) {
  const int64_t total = k * o * o * v * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t d = idx % v, r = idx / v;
    const int64_t c = r % v;
    r /= v;
    const int64_t l = r % o;
    r /= o;
    const int64_t kk = r % o;
    const double f = ev[c] + ev[d] - eo[kk] - eo[l];
    dst[idx] = cmake(src[idx].x * f, src[idx].y * f);
  }
}

// dst[z][i][a] = src * (eps_a - eps_i)
__global__ void k_ds(const cplx *src, const double *eo, const double *ev, int64_t k, int64_t o, int64_t v,
                     cplx *dst) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < k * o * v;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = idx % v, i = (idx / v) % o;
    const double f = ev[a] - eo[i];
    dst[idx] = cmake(src[idx].x * f, src[idx].y * f);
  }
}

// u[k][l][c][d] = s Re sum_z A[z] B[z] over a [k][o][o][v][v] pair of arrays,
// added as d/d eps: gev[c] += u, gev[d] += u, geo[k] -= u, geo[l] -= u
__global__ void k_eps_from_doubles(const cplx *A, const cplx *Bm, int64_t nz, int64_t o, int64_t v, double s,
                                   double *geo, double *gev) {
  extern __shared__ double acc[];  // o + v
  for (int t = threadIdx.x; t < o + v; t += blockDim.x) acc[t] = 0.0;
  __syncthreads();
  const int64_t n = o * o * v * v;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double u = 0.0;
    for (int64_t z = 0; z < nz; ++z) u += vdot_re(A[z * n + e], Bm[z * n + e]);
    u *= s;
    if (u == 0.0) continue;
    const int64_t d = e % v, c = (e / v) % v, l = (e / (v * v)) % o, kk = e / (v * v * o);
    atomicAdd(&acc[o + c], u);
    atomicAdd(&acc[o + d], u);
    atomicAdd(&acc[kk], -u);
    atomicAdd(&acc[l], -u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < o + v; t += blockDim.x) {
    if (acc[t] == 0.0) continue;
    if (t < o) atomicAdd(&geo[t], acc[t]);
    else atomicAdd(&gev[t - o], acc[t]);
  }
}

// the same for singles arrays [z][i][a]: gev[a] += u, geo[i] -= u
__global__ void k_eps_from_singles_vec(const cplx *A, const cplx *Bm, int64_t nz, int64_t o, int64_t v, double s,
                                       double *geo, double *gev) {
  for (int64_t P = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; P < o * v; P += (int64_t)gridDim.x * blockDim.x) {
    double u = 0.0;
    for (int64_t z = 0; z < nz; ++z) u += vdot_re(A[z * o * v + P], Bm[z * o * v + P]);
    u *= s;
    atomicAdd(&gev[P % v], u);
    atomicAdd(&geo[P / v], -u);
  }
}

// reverse of N = num / D for N[i][j][a][b] (doubles, D = eo_i + eo_j - ev_a - ev_b):
// rho[i][j][a][b] = conj(G / D) (the density for the numerator's table),
// eps gets -Re(conj(G) N) / D times dD/d eps
__global__ void k_rev_denom2(const cplx *G, const cplx *Nv, const double *eo, const double *ev, int64_t o,
                             int64_t v, cplx *rho, double *geo, double *gev) {
  extern __shared__ double acc[];
  for (int t = threadIdx.x; t < o + v; t += blockDim.x) acc[t] = 0.0;
  __syncthreads();
  const int64_t n = o * o * v * v;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e % v, a = (e / v) % v, j = (e / (v * v)) % o, i = e / (v * v * o);
    const double D = eo[i] + eo[j] - ev[a] - ev[b];
    const cplx g = G[e];
    if (rho) rho[e] = cmake(g.x / D, -g.y / D);
    const double q = -(g.x * Nv[e].x + g.y * Nv[e].y) / D;
    if (q == 0.0) continue;
    atomicAdd(&acc[i], q);
    atomicAdd(&acc[j], q);
    atomicAdd(&acc[o + a], -q);
    atomicAdd(&acc[o + b], -q);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < o + v; t += blockDim.x) {
    if (acc[t] == 0.0) continue;
    if (t < o) atomicAdd(&geo[t], acc[t]);
    else atomicAdd(&gev[t - o], acc[t]);
  }
}

// singles: N[i][a] = num / (eo_i - ev_a)
__global__ void k_rev_denom1(const cplx *G, const cplx *Nv, const double *eo, const double *ev, int64_t o,
                             int64_t v, cplx *rho, double *geo, double *gev) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < o * v; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e % v, i = e / v;
    const double D = eo[i] - ev[a];
    const cplx g = G[e];
    rho[e] = cmake(g.x / D, -g.y / D);
    const double q = -(g.x * Nv[e].x + g.y * Nv[e].y) / D;
    atomicAdd(&geo[i], q);
    atomicAdd(&gev[a], -q);
  }
}

// Gv[a][b][i][j] += Gt1[i][j][a][b] / D (t1 = <ab||ij> / D)
__global__ void k_t1_to_vvoo(const cplx *Gt, const double *eo, const double *ev, int64_t o, int64_t v, cplx *Gv) {
  const int64_t n = o * o * v * v;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e % v, a = (e / v) % v, j = (e / (v * v)) % o, i = e / (v * v * o);
    const double D = eo[i] + eo[j] - ev[a] - ev[b];
    const int64_t t = ((a * v + b) * o + i) * o + j;
    Gv[t] = cadd(Gv[t], cmake(Gt[e].x / D, Gt[e].y / D));
  }
}

// gB[Q][p0 + p][q0 + q] += s T[Q][p][q]
__global__ void k_add_block(const cplx *T, int64_t Q, int64_t np, int64_t nq, int64_t p0, int64_t q0, int64_t nmo,
                            double s, cplx *gB) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < Q * np * nq;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = idx % nq, p = (idx / nq) % np, z = idx / (nq * np);
    cplx *d = gB + (z * nmo + p0 + p) * nmo + q0 + q;
    *d = cmake(d->x + s * T[idx].x, d->y + s * T[idx].y);
  }
}

bool is_occ_label(char ch) { return std::string("ijklMNOPRSTW").find(ch) != std::string::npos; }

// gradient buffers of the tensors of a term table: t1, t2 [i][j][a][b] and
// s2 [i][a] as stored, integral blocks dense by o/v spec (created on first use)
struct GradBufs {
  DBuf Gt1, Gt2, Gs2;
  std::map<std::string, DBuf> Gv;
};

TermSource grad_source(Exec &ex, int64_t o, int64_t v, bool third, GradBufs &G) {
  G.Gt1 = cbuf(ex, o * o * v * v);
  fill_zero(ex, G.Gt1.p, G.Gt1.bytes);
  if (third) {
    G.Gt2 = cbuf(ex, o * o * v * v);
    G.Gs2 = cbuf(ex, o * v);
    fill_zero(ex, G.Gt2.p, G.Gt2.bytes);
    fill_zero(ex, G.Gs2.p, G.Gs2.bytes);
  }
  TermSource gsrc;
  gsrc.o = o;
  gsrc.v = v;
  gsrc.get = [&ex, &G, o, v, third](const std::string &name, const std::string &lab) -> TV {
    if (name == "v") {
      std::string spec;
      for (char ch : lab) spec.push_back(is_occ_label(ch) ? 'o' : 'v');
      std::vector<int64_t> e;
      int64_t n = 1;
      for (char ch : spec) { e.push_back(ch == 'o' ? o : v); n *= e.back(); }
      if (!G.Gv.count(spec)) {
        G.Gv[spec] = cbuf(ex, n);
        fill_zero(ex, G.Gv[spec].p, G.Gv[spec].bytes);
      }
      return TV::dense(G.Gv[spec].c(), e);
    }
    if (name == "t1" || name == "t1c" || ((name == "t2" || name == "t2c") && third)) {
      cplx *p = (name[1] == '1') ? G.Gt1.c() : G.Gt2.c();
      TV t(p, {v, v, o, o}, {v, 1, o * v * v, v * v});
      t.conj = (name.back() == 'c');
      return t;
    }
    if ((name == "s2" || name == "s2c") && third) {
      TV t(G.Gs2.c(), {v, o}, {1, v});
      t.conj = (name == "s2c");
      return t;
    }
    return TV();
  };
  return gsrc;
}

// The amplitudes back through their definitions (t1 = <ab||ij> / D, the
// second-order doubles and singles as numerator tables over <pq||rs> and t1,
// divided by their denominators), then every integral block
// <pq||rs> = sum_Q (B_pr B_qs - B_ps B_qr) (Eq. 43) back onto B.
void amplitudes_and_integrals_back(adc_ctx *c, const TermSource &src, const TermSource &gsrc, GradBufs &G,
                                   bool third, const DBuf &t2d, const DBuf &t2s, cplx *gB, double *geo,
                                   double *gev) {
  Exec &ex = c->ex;
  const int64_t o = c->o, v = c->v, Q = c->Q, nmo = c->nmo;
  const double *eo = c->eo.d(), *ev = c->ev.d();
  if (third) {
    std::vector<Term> T2N, S2N;
    amplitude_tables(T2N, S2N);
    DBuf rs = cbuf(ex, o * v);
    k_rev_denom1<<<grid1d(o * v, 256), 256, 0, ex.stream>>>(G.Gs2.c(), t2s.c(), eo, ev, o, v, rs.c(), geo, gev);
    ADC_CHECK_LAUNCH();
    eval_terms_grad(ex, S2N, src, gsrc, {{"ai", TV(rs.c(), {v, o}, {1, v})}}, false, C1());
    DBuf rt = cbuf(ex, o * o * v * v);
    k_rev_denom2<<<1024, 256, (o + v) * sizeof(double), ex.stream>>>(G.Gt2.c(), t2d.c(), eo, ev, o, v, rt.c(),
                                                                     geo, gev);
    ADC_CHECK_LAUNCH();
    eval_terms_grad(ex, T2N, src, gsrc, {{"abij", TV(rt.c(), {v, v, o, o}, {v, 1, o * v * v, v * v})}}, false,
                    C1());
  }
  k_rev_denom2<<<1024, 256, (o + v) * sizeof(double), ex.stream>>>(G.Gt1.c(), c->t1.c(), eo, ev, o, v, nullptr,
                                                                   geo, gev);
  ADC_CHECK_LAUNCH();
  {
    TV gvv = gsrc.get("v", "abij");
    k_t1_to_vvoo<<<grid1d(o * o * v * v, 256), 256, 0, ex.stream>>>(G.Gt1.c(), eo, ev, o, v, gvv.p);
    ADC_CHECK_LAUNCH();
  }
  G.Gt1.reset(); G.Gt2.reset(); G.Gs2.reset();

  for (auto &kv : G.Gv) {
    const std::string &sp = kv.first;
    std::vector<int64_t> e;
    for (char ch : sp) e.push_back(ch == 'o' ? o : v);
    TV Gb = TV::dense(kv.second.c(), e);
    auto off = [&](char ch) { return ch == 'o' ? (int64_t)0 : o; };
    auto dim = [&](char ch) { return ch == 'o' ? o : v; };
    struct Part { char p, q; const char *gl, *bl, *tl; double s; };
    // (output block rows p, cols q; labels of G, of the conjugated B factor, of the result)
    const Part parts[4] = {{sp[0], sp[2], "pqrs", "Qqs", "Qpr", 1.0},
                           {sp[1], sp[3], "pqrs", "Qpr", "Qqs", 1.0},
                           {sp[0], sp[3], "pqrs", "Qqr", "Qps", -1.0},
                           {sp[1], sp[2], "pqrs", "Qps", "Qqr", -1.0}};
    for (const Part &pt : parts) {
      // the conjugated B factor's block classes follow its labels
      const char b0 = sp[std::string("pqrs").find(pt.bl[1])], b1 = sp[std::string("pqrs").find(pt.bl[2])];
      const int64_t np = dim(pt.p), nq = dim(pt.q);
      DBuf T = cbuf(ex, Q * np * nq);
      einsum(ex, C1(), Gb, pt.gl, Bview(c, b0, b1).cj(), pt.bl, C0(), TV::dense(T.c(), {Q, np, nq}), pt.tl);
      k_add_block<<<grid1d(Q * np * nq, 256), 256, 0, ex.stream>>>(T.c(), Q, np, nq, off(pt.p), off(pt.q), nmo,
                                                                 pt.s, gB);
      ADC_CHECK_LAUNCH();
    }
  }
  G.Gv.clear();
}


}  // namespace

// gB (device [Q][nmo][nmo]), geo, gev (device), gx (host): accumulated
void adjoint_ee(adc_ctx *c, const cplx *Y, const double *g_host, int64_t k, cplx *gB, double *geo, double *gev,
                double *gx) {
  Exec &ex = c->ex;
  EEOps &E = *c->ee;
  const int64_t o = c->o, v = c->v, n1 = c->n1, N = c->N;
  const int64_t po = npairs(o), pv = npairs(v);
  const bool third = (c->order == 3);  // x-dependent pieces exist (gradient of x even at x = 0)
  const double x = third ? c->x : 0.0;
  const double xdd = (third && c->dd_order == 1) ? x : 0.0;
  const double *eo = c->eo.d(), *ev = c->ev.d();
  TermSource src = ee_source(c);
  TagScope tg(ex, "adjoint");
  StageScope stage(ex, "adjoint_vectors");

  DBuf gdev(ex, k * sizeof(double));
  ADC_CUDA(cudaMemcpyAsync(gdev.p, g_host, k * sizeof(double), cudaMemcpyHostToDevice, ex.stream));
  DBuf gxd(ex, sizeof(double));
  fill_zero(ex, gxd.p, sizeof(double));
  double *gxp = gxd.d();

  // ---- gradient buffers of the table tensors
  GradBufs G;
  TermSource gsrc = grad_source(ex, o, v, third, G);

  // ---- left/right vectors
  DBuf Y1c = cbuf(ex, k * n1);
  k_scale_conj_rows<<<grid1d(k * n1, 256), 256, 0, ex.stream>>>(Y, N, k, n1, gdev.d(), Y1c.c());
  ADC_CHECK_LAUNCH();
  const int64_t nf = k * o * o * v * v;
  DBuf Y2f = cbuf(ex, nf), Y2c = cbuf(ex, nf);
  {
    DBuf half = cbuf(ex, k * po * v * v);
    pair_unpack(ex, Y + n1, k, po, N, pv, v, 1, half.c());
    pair_unpack(ex, half.c(), k, 1, po * v * v, 0, o, v * v, Y2f.c());
  }
  k_scale_conj_rows<<<grid1d(nf, 256), 256, 0, ex.stream>>>(Y2f.c(), o * o * v * v, k, o * o * v * v, gdev.d(),
                                                           Y2c.c());
  ADC_CHECK_LAUNCH();
  TV tY1c = TV::dense(Y1c.c(), {k, o, v});
  TV tY1(const_cast<cplx *>(Y), {k, o, v}, {N, v, 1});
  TV tY2f = TV::dense(Y2f.c(), {k, o, o, v, v});
  TV tY2c = TV::dense(Y2c.c(), {k, o, o, v, v});

  // ---- singles block: rho[P][Q] = sum_z g_z conj(y1[z][P]) y1[z][Q]
  stage.next("adjoint_singles");
  DBuf rho = cbuf(ex, n1 * n1);
  zgemm(ex, n1, n1, k, 1, C1(), Y1c.c(), 0, 1, n1, false, Y, 0, N, 1, false, C0(), rho.c(), 0, n1, 1);
  const std::vector<int64_t> e4 = {o, v, o, v};
  const std::string L = "iajb";
  DBuf K1 = cbuf(ex, n1 * n1), S2 = cbuf(ex, n1 * n1);
  fill_zero(ex, K1.p, K1.bytes);
  fill_zero(ex, S2.p, S2.bytes);
  eval_terms(ex, E.K1, src, {}, false, C1(), TV::dense(K1.c(), e4), L);
  eval_terms(ex, E.S2, src, {}, false, C1(), TV::dense(S2.c(), e4), L);
  DBuf S3;
  if (third) {
    S3 = cbuf(ex, n1 * n1);
    fill_zero(ex, S3.p, S3.bytes);
    eval_terms(ex, E.S3, src, {}, false, C1(), TV::dense(S3.c(), e4), L);
  }
  {
    // orbital energies through diag(eps_a - eps_i) and W o (S2 + x S3)
    DBuf Sx = cbuf(ex, n1 * n1);
    ADC_CUDA(cudaMemcpyAsync(Sx.p, S2.p, Sx.bytes, cudaMemcpyDeviceToDevice, ex.stream));
    if (third && x != 0.0) zaxpby(ex, n1 * n1, CR(x), S3.c(), C1(), Sx.c());
    DBuf row(ex, n1 * sizeof(double)), col(ex, n1 * sizeof(double));
    k_rowsum_re<<<(unsigned)n1, 256, 0, ex.stream>>>(rho.c(), Sx.c(), n1, row.d());
    k_colsum_re<<<grid1d(n1, 128), 128, 0, ex.stream>>>(rho.c(), Sx.c(), n1, col.d());
    k_eps_from_singles<<<1, 256, 0, ex.stream>>>(rho.c(), row.d(), col.d(), o, v, geo, gev);
    ADC_CHECK_LAUNCH();
  }
  {
    // densities of the tables: d/dK1 and d/dS2 include the -x/2 (S2 K1 + K1 S2) products
    DBuf rK = cbuf(ex, n1 * n1), rS = cbuf(ex, n1 * n1);
    ADC_CUDA(cudaMemcpyAsync(rK.p, rho.p, rK.bytes, cudaMemcpyDeviceToDevice, ex.stream));
    k_wmul<<<grid1d(n1 * n1, 256), 256, 0, ex.stream>>>(rho.c(), eo, ev, o, v, 1.0, 0, rS.c());
    ADC_CHECK_LAUNCH();
    if (third && x != 0.0) {
      // rK -= x/2 (S2^T rho + rho S2^T), rS -= x/2 (rho K1^T + K1^T rho)
      zgemm(ex, n1, n1, n1, 1, CR(-0.5 * x), S2.c(), 0, 1, n1, false, rho.c(), 0, n1, 1, false, C1(), rK.c(), 0,
            n1, 1);
      zgemm(ex, n1, n1, n1, 1, CR(-0.5 * x), rho.c(), 0, n1, 1, false, S2.c(), 0, 1, n1, false, C1(), rK.c(), 0,
            n1, 1);
      zgemm(ex, n1, n1, n1, 1, CR(-0.5 * x), rho.c(), 0, n1, 1, false, K1.c(), 0, 1, n1, false, C1(), rS.c(), 0,
            n1, 1);
      zgemm(ex, n1, n1, n1, 1, CR(-0.5 * x), K1.c(), 0, 1, n1, false, rho.c(), 0, n1, 1, false, C1(), rS.c(), 0,
            n1, 1);
    }
    eval_terms_grad(ex, E.K1, src, gsrc, {{L, TV::dense(rK.c(), e4)}}, false, C1());
    eval_terms_grad(ex, E.S2, src, gsrc, {{L, TV::dense(rS.c(), e4)}}, false, C1());
    eval_terms_grad(ex, E.Y2, src, gsrc, {{L, TV::dense(rho.c(), e4)}}, false, C1());
    if (third) {
      if (x != 0.0) {
        DBuf rW = cbuf(ex, n1 * n1);
        k_wmul<<<grid1d(n1 * n1, 256), 256, 0, ex.stream>>>(rho.c(), eo, ev, o, v, x, 0, rW.c());
        ADC_CHECK_LAUNCH();
        eval_terms_grad(ex, E.S3, src, gsrc, {{L, TV::dense(rW.c(), e4)}}, false, C1());
        eval_terms_grad(ex, E.Y3, src, gsrc, {{L, TV::dense(rho.c(), e4)}}, false, CR(x));
      }
      // d/dx of the singles block: W o S3 + Y3 - 1/2 (S2 K1 + K1 S2)
      DBuf Mx = cbuf(ex, n1 * n1);
      k_wmul<<<grid1d(n1 * n1, 256), 256, 0, ex.stream>>>(S3.c(), eo, ev, o, v, 1.0, 0, Mx.c());
      ADC_CHECK_LAUNCH();
      eval_terms(ex, E.Y3, src, {}, false, C1(), TV::dense(Mx.c(), e4), L);
      zgemm(ex, n1, n1, n1, 1, CR(-0.5), S2.c(), 0, n1, 1, false, K1.c(), 0, n1, 1, false, C1(), Mx.c(), 0, n1, 1);
      zgemm(ex, n1, n1, n1, 1, CR(-0.5), K1.c(), 0, n1, 1, false, S2.c(), 0, n1, 1, false, C1(), Mx.c(), 0, n1, 1);
      k_dot_re<<<256, 256, 0, ex.stream>>>(rho.c(), Mx.c(), n1 * n1, 1.0, gxp);
      ADC_CHECK_LAUNCH();
    }
  }
  rho.reset(); K1.reset(); S2.reset(); S3.reset();

  // ---- coupling (twice: M_SD and its Hermitian partner M_DS)
  stage.next("adjoint_coupling");
  eval_terms_grad(ex, E.SD1, src, gsrc, {{"zia", tY1c}, {"zklcd", tY2f}}, false, CR(0.5));
  if (third) {
    DBuf Y2k = cbuf(ex, nf), Y1s = cbuf(ex, k * n1);
    k_dk<<<grid1d(nf, 256), 256, 0, ex.stream>>>(Y2f.c(), eo, ev, k, o, v, Y2k.c());
    k_ds<<<grid1d(k * n1, 256), 256, 0, ex.stream>>>(Y1c.c(), eo, ev, k, o, v, Y1s.c());
    ADC_CHECK_LAUNCH();
    TV tY2k = TV::dense(Y2k.c(), {k, o, o, v, v});
    TV tY1s = TV::dense(Y1s.c(), {k, o, v});
    if (x != 0.0) {
      eval_terms_grad(ex, E.O2, src, gsrc, {{"zia", tY1c}, {"zklcd", tY2k}}, false, CR(0.5 * x));
      eval_terms_grad(ex, E.O2, src, gsrc, {{"zia", tY1s}, {"zklcd", tY2f}}, false, CR(-0.5 * x));
      eval_terms_grad(ex, E.Z1, src, gsrc, {{"zia", tY1c}, {"zklcd", tY2f}}, false, CR(0.5 * x));
    }
    // orbital energies through Delta_K and Delta_S
    DBuf A = cbuf(ex, nf);
    fill_zero(ex, A.p, A.bytes);
    eval_terms(ex, E.O2, src, {{"zia", tY1c}}, false, C1(), TV::dense(A.c(), {k, o, o, v, v}), "zklcd");
    k_eps_from_doubles<<<1024, 256, (o + v) * sizeof(double), ex.stream>>>(A.c(), Y2f.c(), k, o, v, 0.5 * x, geo,
                                                                         gev);
    ADC_CHECK_LAUNCH();
    A.reset();
    DBuf T0 = cbuf(ex, k * n1), TK = cbuf(ex, k * n1), TZ = cbuf(ex, k * n1);
    fill_zero(ex, T0.p, T0.bytes);
    fill_zero(ex, TK.p, TK.bytes);
    fill_zero(ex, TZ.p, TZ.bytes);
    eval_terms(ex, E.O2, src, {{"zklcd", tY2f}}, false, C1(), TV::dense(T0.c(), {k, o, v}), "zia");
    eval_terms(ex, E.O2, src, {{"zklcd", tY2k}}, false, C1(), TV::dense(TK.c(), {k, o, v}), "zia");
    eval_terms(ex, E.Z1, src, {{"zklcd", tY2f}}, false, C1(), TV::dense(TZ.c(), {k, o, v}), "zia");
    k_eps_from_singles_vec<<<grid1d(n1, 256), 256, 0, ex.stream>>>(Y1c.c(), T0.c(), k, o, v, -0.5 * x, geo, gev);
    ADC_CHECK_LAUNCH();
    // d/dx: 2 Re 1/4 sum Y1c (TK - Delta_S T0 + TZ)
    k_dot_re<<<64, 256, 0, ex.stream>>>(Y1c.c(), TK.c(), k * n1, 0.5, gxp);
    k_dot_re<<<64, 256, 0, ex.stream>>>(Y1s.c(), T0.c(), k * n1, -0.5, gxp);
    k_dot_re<<<64, 256, 0, ex.stream>>>(Y1c.c(), TZ.c(), k * n1, 0.5, gxp);
    ADC_CHECK_LAUNCH();
  }

  // ---- doubles block: zeroth order (packed = full / 4) and, at third order, M_DD^(1)
  stage.next("adjoint_doubles");
  k_eps_from_doubles<<<1024, 256, (o + v) * sizeof(double), ex.stream>>>(Y2c.c(), Y2f.c(), k, o, v, 0.25, geo, gev);
  ADC_CHECK_LAUNCH();
  if (third && c->dd_order == 1) {
    if (xdd != 0.0)
      eval_terms_grad(ex, E.DD1, src, gsrc, {{"zijab", tY2c}, {"zklcd", tY2f}}, false, CR(xdd / 16.0));
    DBuf T = cbuf(ex, nf);
    fill_zero(ex, T.p, T.bytes);
    eval_terms(ex, E.DD1, src, {{"zklcd", tY2f}}, false, C1(), TV::dense(T.c(), {k, o, o, v, v}), "zijab");
    k_dot_re<<<256, 256, 0, ex.stream>>>(Y2c.c(), T.c(), nf, 1.0 / 16.0, gxp);
    ADC_CHECK_LAUNCH();
  }
  Y1c.reset(); Y2f.reset(); Y2c.reset();

  stage.next("adjoint_amplitudes_integrals");
  amplitudes_and_integrals_back(c, src, gsrc, G, third, E.t2d, E.t2s, gB, geo, gev);
  double h = 0.0;
  ADC_CUDA(cudaMemcpyAsync(&h, gxp, sizeof(double), cudaMemcpyDeviceToHost, ex.stream));
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
  *gx += h;
}

namespace {

using Rows = std::vector<std::pair<const char *, const char *>>;

// IP/EA-ADC term tables: the matrix elements that setup.cu builds (Sec. 2.1,
// Eqs. 5-7, 11-12). Main block [p][q] (EA p,q = a,b; IP p,q = i,j):
//   M2 + s/2 (e_p - e_q) P2 + x [Y3 + s/2 (e_p - e_q) P3],  s = +1 (EA), -1 (IP),
// P2 and P3 being the transposed second- and third-order one-particle
// densities of the class (EA g_ba, IP h_ji). Coupling C[p][satellite], first
// order plus x times second order; satellite block first order (x-scaled)
// over full antisymmetric indices.
const Rows kEA_M2 = {{"-1/2", "t1(aA,MN) v(MN,bA)"}};
const Rows kEA_P2 = {{"1/2", "t1c(bA,MN) t1(aA,MN)"}};
const Rows kEA_Y3 = {{"-1/2", "t2(aA,MN) v(MN,bA)"},
                     {"-1", "v(Ma,bA) s2(A,M)"},
                     {"1", "v(aA,bM) s2c(A,M)"},
                     {"1/2", "v(aA,bB) t1c(AC,MN) t1(BC,MN)"},
                     {"1/4", "v(AB,bC) t1c(AB,MN) t1(Ca,MN)"},
                     {"1/2", "v(Ma,bN) t1c(AB,NO) t1(AB,MO)"},
                     {"-1", "v(MA,bN) t1c(AB,NO) t1(aB,MO)"}};
const Rows kEA_P3 = {{"1/2", "t1c(bA,MN) t2(aA,MN)"}, {"1/2", "t2c(bA,MN) t1(aA,MN)"}};
const Rows kEA_C1 = {{"1", "v(ck,de)"}};
const Rows kEA_C2 = {{"1/2", "v(ck,MN) t1c(de,MN)"}, {"1", "v(cA,eM) t1c(Ad,kM)"}, {"-1", "v(cA,dM) t1c(Ae,kM)"}};
const Rows kEA_S1 = {{"1", "v(ab,cd) d(jk)"}, {"-1", "v(ak,cj) d(bd)"}, {"1", "v(bk,cj) d(ad)"},
                     {"1", "v(ak,dj) d(bc)"}, {"-1", "v(bk,dj) d(ac)"}};
const Rows kIP_M2 = {{"1/2", "v(Mj,AB) t1(AB,iM)"}};
const Rows kIP_P2 = {{"1/2", "t1c(AB,jM) t1(AB,iM)"}};
const Rows kIP_Y3 = {{"1/2", "v(Mj,AB) t2(AB,iM)"},
                     {"-1", "v(Mj,Ai) s2(A,M)"},
                     {"1", "v(Aj,iM) s2c(A,M)"},
                     {"1/2", "v(Mj,Ni) t1c(AB,NO) t1(AB,MO)"},
                     {"1/4", "v(Mj,NO) t1c(AB,NO) t1(AB,iM)"},
                     {"-1/2", "v(Aj,Bi) t1c(AC,MN) t1(BC,MN)"},
                     {"1", "v(Aj,BM) t1c(AC,MN) t1(BC,iN)"}};
const Rows kIP_P3 = {{"1/2", "t1c(AB,jM) t2(AB,iM)"}, {"1/2", "t2c(AB,jM) t1(AB,iM)"}};
const Rows kIP_C1 = {{"1", "v(ji,ak)"}};
const Rows kIP_C2 = {{"1/2", "v(AB,ak) t1c(AB,ji)"}, {"-1", "v(Ai,Mk) t1c(Aa,jM)"}, {"1", "v(Aj,Mk) t1c(Aa,iM)"}};
const Rows kIP_S1 = {{"1", "v(kl,ij) d(ab)"}, {"-1", "v(ak,bi) d(jl)"}, {"1", "v(ak,bj) d(il)"},
                     {"1", "v(al,bi) d(jk)"}, {"-1", "v(al,bj) d(ik)"}};

// out[p][q] = s (e_p - e_q) / 2 * R[p][q] (+ out if accumulate)
__global__ void k_wmain(const cplx *R, const double *e, int64_t n, double s, int accumulate, cplx *out) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const double w = s * 0.5 * (e[idx / n] - e[idx % n]);
    cplx r = cmake(w * R[idx].x, w * R[idx].y);
    if (accumulate) r = cadd(r, out[idx]);
    out[idx] = r;
  }
}

// out[p] += sign (Re rho[p][p] + (row[p] - col[p]) / 2): the main block's
// orbital energies, on its diagonal and in s/2 (e_p - e_q) (P2 + x P3)
__global__ void k_eps_main(const cplx *rho, const double *row, const double *col, int64_t n, double sign,
                           double *out) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    out[p] += sign * (rho[p * n + p].x + 0.5 * (row[p] - col[p]));
}

// row r of the strict upper triangle of an n x n pair table holding pair index pr
__device__ __forceinline__ void pair_rc(int64_t pr, int64_t n, int64_t &r, int64_t &cidx) {
  r = 0;
  while ((r + 1) * n - (r + 1) * (r + 2) / 2 <= pr) ++r;
  cidx = pr - (r * n - r * (r + 1) / 2) + r + 1;
}

// zeroth-order satellite diagonal: u = sum_z g_z |y2[z][P]|^2 per packed index
// P enters the orbital energies of EA (j, a<b): eps_a + eps_b - eps_j, or of
// IP (i<j, a): eps_a - eps_i - eps_j
__global__ void k_eps_sat0(const cplx *Y, int64_t ld, int64_t n1, int64_t k, const double *g, int64_t o, int64_t v,
                           int ea, double *geo, double *gev) {
  extern __shared__ double acc[];  // o + v
  for (int t = threadIdx.x; t < o + v; t += blockDim.x) acc[t] = 0.0;
  __syncthreads();
  const int64_t po = o * (o - 1) / 2, pv = v * (v - 1) / 2, n2 = ea ? o * pv : po * v;
  for (int64_t P = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; P < n2; P += (int64_t)gridDim.x * blockDim.x) {
    double u = 0.0;
    for (int64_t z = 0; z < k; ++z) {
      const cplx y = Y[z * ld + n1 + P];
      u += g[z] * (y.x * y.x + y.y * y.y);
    }
    if (u == 0.0) continue;
    int64_t p, q;
    if (ea) {
      pair_rc(P % pv, v, p, q);
      atomicAdd(&acc[o + p], u);
      atomicAdd(&acc[o + q], u);
      atomicAdd(&acc[P / pv], -u);
    } else {
      pair_rc(P / v, o, p, q);
      atomicAdd(&acc[o + P % v], u);
      atomicAdd(&acc[p], -u);
      atomicAdd(&acc[q], -u);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < o + v; t += blockDim.x) {
    if (acc[t] == 0.0) continue;
    if (t < o) atomicAdd(&geo[t], acc[t]);
    else atomicAdd(&gev[t - o], acc[t]);
  }
}

}  // namespace

// IP/EA: the same adjoint as adjoint_ee over the tables above. With packed
// satellite vectors expanded to full antisymmetric arrays Y2 (packed = full / 2
// over the one packed pair), sum_r g_r y_r^H M y_r is
//   sum rho o M11 + Re sum Y1c C Y2 + sum g |y2|^2 d0 + x/4 sum Y2c S1 Y2,
// rho = sum_r g_r conj(y1_r) y1_r^T, Y1c = g conj(y1), Y2c = g conj(Y2); the
// coupling term already counts both M12 and M21 = M12^H.
void adjoint_ipea(adc_ctx *c, const cplx *Y, const double *g_host, int64_t k, cplx *gB, double *geo, double *gev,
                  double *gx) {
  Exec &ex = c->ex;
  const bool ea = (c->kind == ADC_EA);
  const int64_t o = c->o, v = c->v, n1 = c->n1, N = c->N;
  const int64_t pv = npairs(v);
  const bool third = (c->order == 3);  // x-dependent pieces exist (gradient of x even at x = 0)
  const double x = third ? c->x : 0.0;
  const double *eo = c->eo.d(), *ev = c->ev.d();
  TagScope tg(ex, "adjoint");

  // second-order amplitudes (the setup does not keep them) and the table tensors
  DBuf t2d, t2s;
  if (third) {
    DBuf Gvv, Lad;
    second_order_amplitudes(c, Gvv, Lad, t2d, t2s);
  }
  std::map<std::string, DBuf> eri;
  TermSource src;
  src.o = o;
  src.v = v;
  src.get = [c, &eri, &t2d, &t2s, o, v](const std::string &name, const std::string &lab) -> TV {
    if (name == "v") {
      std::string spec;
      for (char ch : lab) spec.push_back(is_occ_label(ch) ? 'o' : 'v');
      if (!eri.count(spec)) eri[spec] = eri_block(c, spec.c_str());
      std::vector<int64_t> e;
      for (char ch : spec) e.push_back(ch == 'o' ? o : v);
      return TV::dense(eri[spec].c(), e);
    }
    if (name == "t1" || name == "t1c" || name == "t2" || name == "t2c") {
      cplx *p = (name[1] == '1') ? c->t1.c() : t2d.c();
      ADC_REQUIRE(p != nullptr, ADC_ERR_STATE, "IP/EA terms: second-order amplitudes missing");
      TV t(p, {v, v, o, o}, {v, 1, o * v * v, v * v});
      t.conj = (name.back() == 'c');
      return t;
    }
    if (name == "s2" || name == "s2c") {
      ADC_REQUIRE(t2s.p != nullptr, ADC_ERR_STATE, "IP/EA terms: second-order singles missing");
      TV t(t2s.c(), {v, o}, {1, v});
      t.conj = (name == "s2c");
      return t;
    }
    throw Error(ADC_ERR_ARG, "IP/EA terms: unknown tensor " + name);
  };
  const std::vector<Term> M2 = parse_terms(ea ? kEA_M2 : kIP_M2), P2 = parse_terms(ea ? kEA_P2 : kIP_P2),
                          Y3 = parse_terms(ea ? kEA_Y3 : kIP_Y3), P3 = parse_terms(ea ? kEA_P3 : kIP_P3),
                          Cp1 = parse_terms(ea ? kEA_C1 : kIP_C1), Cp2 = parse_terms(ea ? kEA_C2 : kIP_C2),
                          S1 = parse_terms(ea ? kEA_S1 : kIP_S1);
  const double sgn = ea ? 1.0 : -1.0;
  const double *e1 = ea ? ev : eo;  // orbital energies of the main class
  double *g1 = ea ? gev : geo;
  const std::string L = ea ? "ab" : "ij";
  const std::vector<int64_t> e2 = {n1, n1};

  DBuf gdev(ex, k * sizeof(double));
  ADC_CUDA(cudaMemcpyAsync(gdev.p, g_host, k * sizeof(double), cudaMemcpyHostToDevice, ex.stream));
  DBuf gxd(ex, sizeof(double));
  fill_zero(ex, gxd.p, sizeof(double));
  double *gxp = gxd.d();

  GradBufs G;
  TermSource gsrc = grad_source(ex, o, v, third, G);

  // ---- left/right vectors
  DBuf Y1c = cbuf(ex, k * n1);
  k_scale_conj_rows<<<grid1d(k * n1, 256), 256, 0, ex.stream>>>(Y, N, k, n1, gdev.d(), Y1c.c());
  ADC_CHECK_LAUNCH();
  const std::vector<int64_t> ef = ea ? std::vector<int64_t>{k, o, v, v} : std::vector<int64_t>{k, o, o, v};
  const int64_t per = ef[1] * ef[2] * ef[3], nf = k * per;
  DBuf Y2f = cbuf(ex, nf), Y2c = cbuf(ex, nf);
  if (ea) pair_unpack(ex, Y + n1, k, o, N, pv, v, 1, Y2f.c());
  else pair_unpack(ex, Y + n1, k, 1, N, 0, o, v, Y2f.c());
  k_scale_conj_rows<<<grid1d(nf, 256), 256, 0, ex.stream>>>(Y2f.c(), per, k, per, gdev.d(), Y2c.c());
  ADC_CHECK_LAUNCH();
  TV tY1c = TV::dense(Y1c.c(), {k, n1});
  TV tY2f = TV::dense(Y2f.c(), ef), tY2c = TV::dense(Y2c.c(), ef);

  // ---- main block: rho[p][q] = sum_z g_z conj(y1[z][p]) y1[z][q]
  DBuf rho = cbuf(ex, n1 * n1);
  zgemm(ex, n1, n1, k, 1, C1(), Y1c.c(), 0, 1, n1, false, Y, 0, N, 1, false, C0(), rho.c(), 0, n1, 1);
  TV trho = TV::dense(rho.c(), e2);
  {
    DBuf Sx = cbuf(ex, n1 * n1), P3m;
    fill_zero(ex, Sx.p, Sx.bytes);
    eval_terms(ex, P2, src, {}, false, C1(), TV::dense(Sx.c(), e2), L);
    if (third) {
      P3m = cbuf(ex, n1 * n1);
      fill_zero(ex, P3m.p, P3m.bytes);
      eval_terms(ex, P3, src, {}, false, C1(), TV::dense(P3m.c(), e2), L);
      if (x != 0.0) zaxpby(ex, n1 * n1, CR(x), P3m.c(), C1(), Sx.c());
    }
    DBuf row(ex, n1 * sizeof(double)), col(ex, n1 * sizeof(double));
    k_rowsum_re<<<(unsigned)n1, 256, 0, ex.stream>>>(rho.c(), Sx.c(), n1, row.d());
    k_colsum_re<<<grid1d(n1, 128), 128, 0, ex.stream>>>(rho.c(), Sx.c(), n1, col.d());
    k_eps_main<<<grid1d(n1, 128), 128, 0, ex.stream>>>(rho.c(), row.d(), col.d(), n1, sgn, g1);
    ADC_CHECK_LAUNCH();
    DBuf rW = cbuf(ex, n1 * n1);
    k_wmain<<<grid1d(n1 * n1, 256), 256, 0, ex.stream>>>(rho.c(), e1, n1, sgn, 0, rW.c());
    ADC_CHECK_LAUNCH();
    eval_terms_grad(ex, M2, src, gsrc, {{L, trho}}, false, C1());
    eval_terms_grad(ex, P2, src, gsrc, {{L, TV::dense(rW.c(), e2)}}, false, C1());
    if (third) {
      if (x != 0.0) {
        eval_terms_grad(ex, Y3, src, gsrc, {{L, trho}}, false, CR(x));
        eval_terms_grad(ex, P3, src, gsrc, {{L, TV::dense(rW.c(), e2)}}, false, CR(x));
      }
      // d/dx of the main block: Y3 + s/2 (e_p - e_q) P3
      DBuf Mx = cbuf(ex, n1 * n1);
      fill_zero(ex, Mx.p, Mx.bytes);
      eval_terms(ex, Y3, src, {}, false, C1(), TV::dense(Mx.c(), e2), L);
      k_wmain<<<grid1d(n1 * n1, 256), 256, 0, ex.stream>>>(P3m.c(), e1, n1, sgn, 1, Mx.c());
      k_dot_re<<<256, 256, 0, ex.stream>>>(rho.c(), Mx.c(), n1 * n1, 1.0, gxp);
      ADC_CHECK_LAUNCH();
    }
  }
  rho.reset();

  // ---- coupling
  const std::string l1 = ea ? "zc" : "zk", l2 = ea ? "zkde" : "zija";
  eval_terms_grad(ex, Cp1, src, gsrc, {{l1, tY1c}, {l2, tY2f}}, false, C1());
  if (third) {
    if (x != 0.0) eval_terms_grad(ex, Cp2, src, gsrc, {{l1, tY1c}, {l2, tY2f}}, false, CR(x));
    DBuf T = cbuf(ex, k * n1);
    fill_zero(ex, T.p, T.bytes);
    eval_terms(ex, Cp2, src, {{l2, tY2f}}, false, C1(), TV::dense(T.c(), {k, n1}), l1);
    k_dot_re<<<64, 256, 0, ex.stream>>>(Y1c.c(), T.c(), k * n1, 1.0, gxp);
    ADC_CHECK_LAUNCH();
  }

  // ---- satellite block: zeroth-order diagonal and x times first order
  k_eps_sat0<<<1024, 256, (o + v) * sizeof(double), ex.stream>>>(Y, N, n1, k, gdev.d(), o, v, ea ? 1 : 0, geo, gev);
  ADC_CHECK_LAUNCH();
  if (third) {
    const std::string la = ea ? "zjab" : "zija", lb = ea ? "zkcd" : "zklb";
    if (x != 0.0) eval_terms_grad(ex, S1, src, gsrc, {{la, tY2c}, {lb, tY2f}}, false, CR(0.25 * x));
    DBuf T = cbuf(ex, nf);
    fill_zero(ex, T.p, T.bytes);
    eval_terms(ex, S1, src, {{lb, tY2f}}, false, C1(), TV::dense(T.c(), ef), la);
    k_dot_re<<<256, 256, 0, ex.stream>>>(Y2c.c(), T.c(), nf, 0.25, gxp);
    ADC_CHECK_LAUNCH();
  }
  Y1c.reset(); Y2f.reset(); Y2c.reset();

  amplitudes_and_integrals_back(c, src, gsrc, G, third, t2d, t2s, gB, geo, gev);
  double h = 0.0;
  ADC_CUDA(cudaMemcpyAsync(&h, gxp, sizeof(double), cudaMemcpyDeviceToHost, ex.stream));
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
  *gx += h;
}

}  // namespace adc
