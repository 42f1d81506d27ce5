// EE-ADC sigma: the expensive pieces as packed GEMMs.
//
// With the doubles X(ij,ab) antisymmetric in both pairs and stored for i<j,
// a<b, the term tables of ee.cu reduce to
//
//   singles <- doubles (first order):
//     S1(ia) = sum_{l, c<d} <al||cd> X(il,cd) + sum_{k<l, d} <kl||di> X(kl,ad)
//   doubles <- singles (its Hermitian partner):
//     S2(il,cd) += A_il [ sum_a conj<al||cd> X1(ia) ],
//     S2(kl,ad) += A_ad [ sum_i conj<kl||di> X1(ia) ]      (A: antisymmetriser)
//   second order (scaled by x): the terms with two Kronecker deltas cancel
//     against the energy-weighted overlap term, and the rest folds into the
//     two operators above plus two separable pieces,
//     <al||cd> -> <al||cd> + x KA(l,cd,a),  <kl||di> -> <kl||di> + x KB(kl,d,i),
//     KA = sum_AM conj(t_lM^dA) <aA||cM> - (c<->d) + 1/2 sum_MN conj(t_MN^cd) <al||MN>,
//     KB = sum_AM conj(t_kM^dA) <lA||iM> - (k<->l) + 1/2 sum_AB conj(t_kl^AB) <AB||di>,
//     S1(ia) += x sum_kM <ak||iM> Y1(k,M),  Y1(k,M) = sum_{l,c<d} conj(t_lM^cd) X(kl,cd),
//     S1(ia) += x sum_Ac <aA||ci> Y2(c,A),  Y2(c,A) = sum_{k<l,d} conj(t_kl^dA) X(kl,cd),
//     and their Hermitian partners for S2;
//   doubles <- doubles (first order, scaled by x at third order):
//     S2(ij,ab) += sum_{c<d} <ab||cd> X(ij,cd) + sum_{k<l} <kl||ij> X(kl,ab)
//                + P(ij) P(ab) T(ia,jb),   T(ia,jb) = sum_kc <ak||cj> X(ki,cb)
//
// (Eq. 43 integrals; checked element by element against the tables.) Each
// line is one GEMM over packed or gathered operands; nothing of size
// o^2 v^2 per vector is formed except the ring operand. Vectors are processed
// in chunks whose scratch stays below a fixed budget.
#include "ctx.cuh"
#include "ee.cuh"

namespace adc {

namespace {

__device__ __forceinline__ cplx neg(cplx a) { return cmake(-a.x, -a.y); }

// Va[(l, (c<d))][a] = <al||cd>  from vovv[a][l][c][d]
__global__ void k_pack_va(const cplx *vovv, const int *pc, const int *pd, int64_t o, int64_t v, int64_t pv,
                          cplx *Va) {
  const int64_t total = o * pv * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = idx % v, r = idx / v;
    const int64_t pcd = r % pv, l = r / pv;
    Va[idx] = vovv[((a * o + l) * v + pc[pcd]) * v + pd[pcd]];
  }
}
// Vb[i][((k<l), d)] = <kl||di>  from oovo[k][l][d][i]
__global__ void k_pack_vb(const cplx *oovo, const int *pk, const int *pl, int64_t o, int64_t v, int64_t po,
                          cplx *Vb) {
  const int64_t total = o * po * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = idx % v, r = idx / v;
    const int64_t pkl = r % po, i = r / po;
    Vb[idx] = oovo[((pk[pkl] * o + pl[pkl]) * v + d) * o + i];
  }
}
// Goo[(i<j)][(k<l)] = <kl||ij>  from oooo[k][l][i][j]
__global__ void k_pack_goo(const cplx *oooo, const int *pi, const int *pj, int64_t o, int64_t po, cplx *G) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < po * po;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pkl = idx % po, pij = idx / po;
    G[idx] = oooo[((pi[pkl] * o + pj[pkl]) * o + pi[pij]) * o + pj[pij]];
  }
}

// signed element X(p q, r s) of the packed doubles block (pairs of o and of v)
__device__ __forceinline__ cplx xel(const cplx *X2, int64_t p, int64_t q, int64_t r, int64_t s, int64_t o,
                                   int64_t v, int64_t pv) {
  if (p == q || r == s) return cmake(0.0, 0.0);
  const bool sw1 = p > q, sw2 = r > s;
  const int64_t a = sw1 ? q : p, b = sw1 ? p : q, c = sw2 ? s : r, d = sw2 ? r : s;
  const cplx x = X2[pair_index(a, b, o) * pv + pair_index(c, d, v)];
  return (sw1 != sw2) ? neg(x) : x;
}

// Xa[z][i][l][(c<d)] = X_z(il, cd)
__global__ void k_gather_xa(const cplx *X, int64_t ldx, int64_t kc, const int *pc, const int *pd, int64_t o,
                            int64_t v, int64_t pv, cplx *Xa) {
  const int64_t total = kc * o * o * pv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pcd = idx % pv, r = idx / pv;
    const int64_t l = r % o, r2 = r / o;
    const int64_t i = r2 % o, z = r2 / o;
    Xa[idx] = xel(X + z * ldx, i, l, pc[pcd], pd[pcd], o, v, pv);
  }
}
// Xb[z][(k<l)][d][a] = X_z(kl, ad)
__global__ void k_gather_xb(const cplx *X, int64_t ldx, int64_t kc, const int *pk, const int *pl, int64_t o,
                            int64_t v, int64_t po, int64_t pv, cplx *Xb) {
  const int64_t total = kc * po * v * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = idx % v, r = idx / v;
    const int64_t d = r % v, r2 = r / v;
    const int64_t pkl = r2 % po, z = r2 / po;
    Xb[idx] = xel(X + z * ldx, pk[pkl], pl[pkl], a, d, o, v, pv);
  }
}
// Xt[(k, c)][(z, i, b)] = X_z(ki, cb)
__global__ void k_gather_xt(const cplx *X, int64_t ldx, int64_t kc, int64_t o, int64_t v, int64_t pv, cplx *Xt) {
  const int64_t ncol = kc * o * v, total = o * v * ncol;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = idx % ncol, row = idx / ncol;
    const int64_t b = col % v, i = (col / v) % o, z = col / (v * o);
    const int64_t kk = row / v, c = row % v;
    Xt[idx] = xel(X + z * ldx, kk, i, c, b, o, v, pv);
  }
}

// XbT[z][a][((k<l), d)] = X_z(kl, ad)
__global__ void k_gather_xbt(const cplx *X, int64_t ldx, int64_t kc, const int *pk, const int *pl, int64_t o,
                             int64_t v, int64_t po, int64_t pv, cplx *Xb) {
  const int64_t total = kc * v * po * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = idx % v, r = idx / v;
    const int64_t pkl = r % po, r2 = r / po;
    const int64_t a = r2 % v, z = r2 / v;
    Xb[idx] = xel(X + z * ldx, pk[pkl], pl[pkl], a, d, o, v, pv);
  }
}
// XtT[(z, i, b)][(k, c)] = X_z(ki, cb)
__global__ void k_gather_xtt(const cplx *X, int64_t ldx, int64_t kc, int64_t o, int64_t v, int64_t pv, cplx *Xt) {
  const int64_t ov = o * v, total = kc * ov * ov;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t kcol = idx % ov, row = idx / ov;
    const int64_t c = kcol % v, kk = kcol / v;
    const int64_t b = row % v, i = (row / v) % o, z = row / ov;
    Xt[idx] = xel(X + z * ldx, kk, i, c, b, o, v, pv);
  }
}

// S2_z[(i<l)][(cd)] += F_z[i][l][(cd)] - F_z[l][i][(cd)]
__global__ void k_scatter_f(const cplx *F, int64_t kc, const int *pi, const int *pj, int64_t o, int64_t po,
                            int64_t pv, cplx *S2, int64_t lds) {
  const int64_t total = kc * po * pv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pcd = idx % pv, r = idx / pv;
    const int64_t pil = r % po, z = r / po;
    const int64_t i = pi[pil], l = pj[pil];
    const cplx *Fz = F + z * o * o * pv;
    const cplx d = csub(Fz[(i * o + l) * pv + pcd], Fz[(l * o + i) * pv + pcd]);
    cplx *t = S2 + z * lds + pil * pv + pcd;
    *t = cadd(*t, d);
  }
}
// S2_z[(kl)][(a<d)] += G_z[(kl)][d][a] - G_z[(kl)][a][d]
__global__ void k_scatter_g(const cplx *G, int64_t kc, const int *pa, const int *pd, int64_t v, int64_t po,
                            int64_t pv, cplx *S2, int64_t lds) {
  const int64_t total = kc * po * pv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pad = idx % pv, r = idx / pv;
    const int64_t pkl = r % po, z = r / po;
    const int64_t a = pa[pad], d = pd[pad];
    const cplx *Gz = G + (z * po + pkl) * v * v;
    const cplx s = csub(Gz[d * v + a], Gz[a * v + d]);
    cplx *t = S2 + z * lds + pkl * pv + pad;
    *t = cadd(*t, s);
  }
}
// S2_z[(i<j)][(a<b)] += s [T(ia,jb) - T(ja,ib) - T(ib,ja) + T(jb,ia)], T(ia,jb) = R[(j,a)][(z,i,b)]
__global__ void k_scatter_ring(const cplx *R, int64_t kc, const int *pi, const int *pj, const int *pa,
                               const int *pb, int64_t o, int64_t v, int64_t po, int64_t pv, double s, cplx *S2,
                               int64_t lds) {
  const int64_t ncol = kc * o * v, total = kc * po * pv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pab = idx % pv, r = idx / pv;
    const int64_t pij = r % po, z = r / po;
    const int64_t i = pi[pij], j = pj[pij], a = pa[pab], b = pb[pab];
    auto T = [&](int64_t p, int64_t q, int64_t rr, int64_t t) {  // T(p q, rr t) = R[(rr,q)][(z,p,t)]
      return R[(rr * v + q) * ncol + (z * o + p) * v + t];
    };
    cplx val = csub(T(i, a, j, b), T(j, a, i, b));
    val = csub(val, T(i, b, j, a));
    val = cadd(val, T(j, b, i, a));
    cplx *t = S2 + z * lds + pij * pv + pab;
    *t = cadd(*t, cmake(s * val.x, s * val.y));
  }
}

// T1p[(l, (c<d))][M] = conj(t_lM^cd)   (t1 stored [i][j][a][b])
__global__ void k_pack_t1p(const cplx *t1, const int *pc, const int *pd, int64_t o, int64_t v, int64_t pv,
                           cplx *T) {
  const int64_t total = o * pv * o;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t M = idx % o, r = idx / o;
    const int64_t pcd = r % pv, l = r / pv;
    const cplx t = t1[((l * o + M) * v + pc[pcd]) * v + pd[pcd]];
    T[idx] = cmake(t.x, -t.y);
  }
}
// T2p[((k<l), d)][A] = conj(t_kl^dA)
__global__ void k_pack_t2p(const cplx *t1, const int *pk, const int *pl, int64_t o, int64_t v, int64_t po,
                           cplx *T) {
  const int64_t total = po * v * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t A = idx % v, r = idx / v;
    const int64_t d = r % v, pkl = r / v;
    const cplx t = t1[((pk[pkl] * o + pl[pkl]) * v + d) * v + A];
    T[idx] = cmake(t.x, -t.y);
  }
}
// V1[(i,a)][(k,M)] = <ak||iM> from vooo[a][k][i][M];  V2[(i,a)][(c,A)] = <aA||ci> from vvvo[a][A][c][i]
__global__ void k_pack_v1(const cplx *vooo, int64_t o, int64_t v, cplx *V1) {
  const int64_t total = o * v * o * o;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t M = idx % o, k = (idx / o) % o, a = (idx / (o * o)) % v, i = idx / (o * o * v);
    V1[idx] = vooo[((a * o + k) * o + i) * o + M];
  }
}
__global__ void k_pack_v2(const cplx *vvvo, int64_t o, int64_t v, cplx *V2) {
  const int64_t total = o * v * v * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t A = idx % v, c = (idx / v) % v, a = (idx / (v * v)) % v, i = idx / (v * v * v);
    V2[idx] = vvvo[((a * v + A) * v + c) * o + i];
  }
}
// Va[(l,(c<d))][a] += x (P[l][c][d][a] - P[l][d][c][a])
__global__ void k_fold_a(const cplx *P, const int *pc, const int *pd, int64_t o, int64_t v, int64_t pv, double x,
                         cplx *Va) {
  const int64_t total = o * pv * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = idx % v, r = idx / v;
    const int64_t pcd = r % pv, l = r / pv;
    const int64_t c = pc[pcd], d = pd[pcd];
    const cplx k = csub(P[((l * v + c) * v + d) * v + a], P[((l * v + d) * v + c) * v + a]);
    Va[idx] = cadd(Va[idx], cmake(x * k.x, x * k.y));
  }
}
// Vb[i][((k<l), d)] += x (P[k][l][d][i] - P[l][k][d][i])
__global__ void k_fold_b(const cplx *P, const int *pk, const int *pl, int64_t o, int64_t v, int64_t po, double x,
                         cplx *Vb) {
  const int64_t total = o * po * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = idx % v, r = idx / v;
    const int64_t pkl = r % po, i = r / po;
    const int64_t k = pk[pkl], l = pl[pkl];
    const cplx q = csub(P[((k * o + l) * v + d) * o + i], P[((l * o + k) * v + d) * o + i]);
    Vb[idx] = cadd(Vb[idx], cmake(x * q.x, x * q.y));
  }
}

__global__ void k_pair_table(int64_t n, int *p, int *q) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t j = i + 1; j < n; ++j) {
      const int64_t t = pair_index(i, j, n);
      p[t] = (int)i;
      q[t] = (int)j;
    }
  }
}

}  // namespace

void ee_struct_build(adc_ctx *c, bool dd) {
  Exec &ex = c->ex;
  EEOps &E = *c->ee;
  const int64_t o = c->o, v = c->v, po = npairs(o), pv = npairs(v);
  if (!E.pair_o.p) {
    E.pair_o = DBuf(ex, 2 * std::max<int64_t>(po, 1) * sizeof(int));
    E.pair_v = DBuf(ex, 2 * std::max<int64_t>(pv, 1) * sizeof(int));
    int *po_p = (int *)E.pair_o.p, *pv_p = (int *)E.pair_v.p;
    k_pair_table<<<grid1d(o, 128), 128, 0, ex.stream>>>(o, po_p, po_p + std::max<int64_t>(po, 1));
    k_pair_table<<<grid1d(v, 128), 128, 0, ex.stream>>>(v, pv_p, pv_p + std::max<int64_t>(pv, 1));
    ADC_CHECK_LAUNCH();
  }
  const int *pio = (const int *)E.pair_o.p, *pjo = pio + std::max<int64_t>(po, 1);
  const int *pav = (const int *)E.pair_v.p, *pbv = pav + std::max<int64_t>(pv, 1);
  if (!E.Va.p) {
    DBuf vovv = eri_block(c, "vovv");
    E.Va = cbuf(ex, o * pv * v);
    k_pack_va<<<grid1d(o * pv * v, 256), 256, 0, ex.stream>>>(vovv.c(), pav, pbv, o, v, pv, E.Va.c());
    ADC_CHECK_LAUNCH();
    DBuf oovo = eri_block(c, "oovo");
    E.Vb = cbuf(ex, o * po * v);
    k_pack_vb<<<grid1d(o * po * v, 256), 256, 0, ex.stream>>>(oovo.c(), pio, pjo, o, v, po, E.Vb.c());
    ADC_CHECK_LAUNCH();
  }
  const bool second = (c->order == 3 && c->x != 0.0);
  if (second && !E.T1p.p) {
    const double x = c->x;
    TV t1c = TV::dense(c->t1.c(), {o, o, v, v}).cj();
    {
      // KA folded into Va
      DBuf vvvo = eri_block(c, "vvvo"), vooo = eri_block(c, "vooo");
      DBuf P = cbuf(ex, o * v * v * v);
      TV Pt = TV::dense(P.c(), {o, v, v, v});
      einsum(ex, C1(), t1c, "lMdA", TV::dense(vvvo.c(), {v, v, v, o}), "aAcM", C0(), Pt, "lcda");
      einsum(ex, CR(0.25), t1c, "MNcd", TV::dense(vooo.c(), {v, o, o, o}), "alMN", C1(), Pt, "lcda");
      k_fold_a<<<grid1d(o * pv * v, 256), 256, 0, ex.stream>>>(P.c(), pav, pbv, o, v, pv, x, E.Va.c());
      ADC_CHECK_LAUNCH();
      P.reset();
      E.V1 = cbuf(ex, o * v * o * o);
      k_pack_v1<<<grid1d(o * v * o * o, 256), 256, 0, ex.stream>>>(vooo.c(), o, v, E.V1.c());
      E.V2 = cbuf(ex, o * v * v * v);
      k_pack_v2<<<grid1d(o * v * v * v, 256), 256, 0, ex.stream>>>(vvvo.c(), o, v, E.V2.c());
      ADC_CHECK_LAUNCH();
      // KB folded into Vb
      DBuf ovoo = eri_block(c, "ovoo");
      DBuf R = cbuf(ex, o * o * v * o);
      TV Rt = TV::dense(R.c(), {o, o, v, o});
      einsum(ex, C1(), t1c, "kMdA", TV::dense(ovoo.c(), {o, v, o, o}), "lAiM", C0(), Rt, "kldi");
      einsum(ex, CR(0.25), t1c, "klAB", TV::dense(vvvo.c(), {v, v, v, o}), "ABdi", C1(), Rt, "kldi");
      k_fold_b<<<grid1d(o * po * v, 256), 256, 0, ex.stream>>>(R.c(), pio, pjo, o, v, po, x, E.Vb.c());
      ADC_CHECK_LAUNCH();
    }
    E.T1p = cbuf(ex, o * pv * o);
    k_pack_t1p<<<grid1d(o * pv * o, 256), 256, 0, ex.stream>>>(c->t1.c(), pav, pbv, o, v, pv, E.T1p.c());
    E.T2p = cbuf(ex, po * v * v);
    k_pack_t2p<<<grid1d(po * v * v, 256), 256, 0, ex.stream>>>(c->t1.c(), pio, pjo, o, v, po, E.T2p.c());
    ADC_CHECK_LAUNCH();
  }
  if (dd && !E.Goo.p) {
    DBuf oooo = eri_block(c, "oooo");
    E.Goo = cbuf(ex, po * po);
    k_pack_goo<<<grid1d(po * po, 256), 256, 0, ex.stream>>>(oooo.c(), pio, pjo, o, po, E.Goo.c());
    ADC_CHECK_LAUNCH();
  }
  // (rebuilt here when a solve released it, see ee_prepare)
  if (dd && !E.Gvv.p) E.Gvv = build_vvvv_packed(c);
}

// the structured pieces for vectors [X | ...] of one chunk: S1 += SD X2,
// S2 += SD^H X1 and, with sdd != 0, S2 += sdd * M_DD^(1) X2
void ee_struct_apply(adc_ctx *c, const cplx *X, cplx *S, int64_t kc, double sdd) {
  Exec &ex = c->ex;
  EEOps &E = *c->ee;
  const int64_t o = c->o, v = c->v, n1 = c->n1, N = c->N, po = npairs(o), pv = npairs(v);
  if (po == 0 || pv == 0 || kc <= 0) return;
  const int *pio = (const int *)E.pair_o.p, *pjo = pio + std::max<int64_t>(po, 1);
  const int *pav = (const int *)E.pair_v.p, *pbv = pav + std::max<int64_t>(pv, 1);
  const bool second = (c->order == 3 && c->x != 0.0);
  const double x = second ? c->x : 0.0;
  TagScope tg(ex, "ee_coupling");
  {
    // S1 += sum_{l,(cd)} X(il,cd) <al||cd>, one GEMM per vector
    DBuf Xa = cbuf(ex, kc * o * o * pv);
    k_gather_xa<<<grid1d(kc * o * o * pv, 256), 256, 0, ex.stream>>>(X + n1, N, kc, pav, pbv, o, v, pv, Xa.c());
    ADC_CHECK_LAUNCH();
    zgemm(ex, o, v, o * pv, kc, C1(), Xa.c(), o * o * pv, o * pv, 1, false, E.Va.c(), 0, v, 1, false, C1(), S, N,
          v, 1);
    DBuf Y1, U;
    if (second) {
      // S1 += x sum_kM <ak||iM> Y1(k,M),  Y1[z][k][M] = sum_(l,cd) Xa[z][k][(l,cd)] T1p[(l,cd)][M]
      Y1 = cbuf(ex, kc * o * o);
      zgemm(ex, o, o, o * pv, kc, C1(), Xa.c(), o * o * pv, o * pv, 1, false, E.T1p.c(), 0, o, 1, false, C0(),
            Y1.c(), o * o, o, 1);
      zgemm(ex, kc, n1, o * o, 1, CR(x), Y1.c(), 0, o * o, 1, false, E.V1.c(), 0, 1, o * o, false, C1(), S, 0, N, 1);
      // Hermitian partner: U[z][(k,M)] = sum_(ia) conj(<ak||iM>) X1(ia)
      U = cbuf(ex, kc * o * o);
      zgemm(ex, kc, o * o, n1, 1, C1(), X, 0, N, 1, false, E.V1.c(), 0, o * o, 1, true, C0(), U.c(), 0, o * o, 1);
    }
    // S2 += A_il sum_a conj<al||cd> X1(ia)   (+ x sum_M t_lM^cd U(i,M))
    zgemm(ex, o, o * pv, v, kc, C1(), X, N, v, 1, false, E.Va.c(), 0, 1, v, true, C0(), Xa.c(), o * o * pv,
          o * pv, 1);
    if (second)
      zgemm(ex, o, o * pv, o, kc, CR(x), U.c(), o * o, o, 1, false, E.T1p.c(), 0, 1, o, true, C1(), Xa.c(),
            o * o * pv, o * pv, 1);
    k_scatter_f<<<grid1d(kc * po * pv, 256), 256, 0, ex.stream>>>(Xa.c(), kc, pio, pjo, o, po, pv, S + n1, N);
    ADC_CHECK_LAUNCH();
  }
  {
    // S1 += sum_{(kl),d} <kl||di> X(kl,ad)
    DBuf Xb = cbuf(ex, kc * po * v * v);
    k_gather_xb<<<grid1d(kc * po * v * v, 256), 256, 0, ex.stream>>>(X + n1, N, kc, pio, pjo, o, v, po, pv,
                                                                    Xb.c());
    ADC_CHECK_LAUNCH();
    zgemm(ex, o, v, po * v, kc, C1(), E.Vb.c(), 0, po * v, 1, false, Xb.c(), po * v * v, v, 1, false, C1(), S, N,
          v, 1);
    DBuf Y2, U2;
    if (second) {
      // S1 += x sum_(c,A) <aA||ci> Y2(c,A),  Y2[z][c][A] = sum_((kl),d) Xb[z][((kl),d)][c] T2p[((kl),d)][A]
      Y2 = cbuf(ex, kc * v * v);
      zgemm(ex, v, v, po * v, kc, C1(), Xb.c(), po * v * v, 1, v, false, E.T2p.c(), 0, v, 1, false, C0(), Y2.c(),
            v * v, v, 1);
      zgemm(ex, kc, n1, v * v, 1, CR(x), Y2.c(), 0, v * v, 1, false, E.V2.c(), 0, 1, v * v, false, C1(), S, 0, N, 1);
      // Hermitian partner: U2[z][(c,A)] = sum_(ia) conj(<aA||ci>) X1(ia)
      U2 = cbuf(ex, kc * v * v);
      zgemm(ex, kc, v * v, n1, 1, C1(), X, 0, N, 1, false, E.V2.c(), 0, v * v, 1, true, C0(), U2.c(), 0, v * v, 1);
    }
    // S2 += A_ad sum_i conj<kl||di> X1(ia)   (+ x sum_A t_kl^dA U2(a,A))
    zgemm(ex, po * v, v, o, kc, C1(), E.Vb.c(), 0, 1, po * v, true, X, N, v, 1, false, C0(), Xb.c(),
          po * v * v, v, 1);
    if (second)
      zgemm(ex, po * v, v, v, kc, CR(x), E.T2p.c(), 0, v, 1, true, U2.c(), v * v, 1, v, false, C1(), Xb.c(),
            po * v * v, v, 1);
    k_scatter_g<<<grid1d(kc * po * pv, 256), 256, 0, ex.stream>>>(Xb.c(), kc, pav, pbv, v, po, pv, S + n1, N);
    ADC_CHECK_LAUNCH();
  }
  if (sdd == 0.0) return;
  ex.tag = "ee_ladder";
  zgemm(ex, po, pv, pv, kc, CR(sdd), X + n1, N, pv, 1, false, E.Gvv.c(), 0, 1, pv, false, C1(), S + n1, N, pv, 1);
  zgemm(ex, po, pv, po, kc, CR(sdd), E.Goo.c(), 0, po, 1, false, X + n1, N, pv, 1, false, C1(), S + n1, N, pv, 1);
  ex.tag = "ee_ring";
  const int64_t ncol = kc * o * v;
  DBuf Xt = cbuf(ex, o * v * ncol), R = cbuf(ex, o * v * ncol);
  k_gather_xt<<<grid1d(o * v * ncol, 256), 256, 0, ex.stream>>>(X + n1, N, kc, o, v, pv, Xt.c());
  ADC_CHECK_LAUNCH();
  zgemm(ex, o * v, ncol, o * v, 1, C1(), c->W.c(), 0, o * v, 1, false, Xt.c(), 0, ncol, 1, false, C0(), R.c(), 0,
        ncol, 1);
  k_scatter_ring<<<grid1d(kc * po * pv, 256), 256, 0, ex.stream>>>(R.c(), kc, pio, pjo, pav, pbv, o, v, po, pv, sdd,
                                                                   S + n1, N);
  ADC_CHECK_LAUNCH();
}

// split-precision copies of the static operators (after ee_struct_build)
static void ee_tc_build(adc_ctx *c, bool dd, int planes) {
  Exec &ex = c->ex;
  EEOps &E = *c->ee;
  const int64_t o = c->o, v = c->v, po = npairs(o), pv = npairs(v), ov = o * v;
  tc_pack_A(ex, E.tVaT, E.Va.c(), v, o * pv, 1, v, false, planes);
  tc_pack_A(ex, E.tVaC, E.Va.c(), o * pv, v, v, 1, true, planes);
  tc_pack_A(ex, E.tVb, E.Vb.c(), o, po * v, po * v, 1, false, planes);
  tc_pack_A(ex, E.tVbC, E.Vb.c(), po * v, o, 1, po * v, true, planes);
  if (dd) {
    tc_pack_A(ex, E.tGvv, E.Gvv.c(), pv, pv, pv, 1, false, planes);
    tc_pack_A(ex, E.tGoo, E.Goo.c(), po, po, po, 1, false, planes);
    tc_pack_A(ex, E.tW, c->W.c(), ov, ov, ov, 1, false, planes);
  }
  if (c->order == 3 && c->x != 0.0) {
    // T1p [(l,cd)][M] and T2p [((kl),d)][A] as the A side of the separable pieces
    tc_pack_A(ex, E.tT1T, E.T1p.c(), o, o * pv, 1, o, false, planes);
    tc_pack_A(ex, E.tT1C, E.T1p.c(), o * pv, o, o, 1, true, planes);
    tc_pack_A(ex, E.tT2T, E.T2p.c(), v, po * v, 1, v, false, planes);
    tc_pack_A(ex, E.tT2C, E.T2p.c(), po * v, v, v, 1, true, planes);
  }
  E.tc_planes = planes;
  E.tcerr = DBuf(ex, sizeof(int));
  fill_zero(ex, E.tcerr.p, sizeof(int));
  E.tc_ready = true;
}

// sliced copies of the same operators (FP64-accurate tensor-core products);
// products with fewer bits use their leading slices
static void ee_sl_build(adc_ctx *c, bool dd) {
  Exec &ex = c->ex;
  EEOps &E = *c->ee;
  const int64_t o = c->o, v = c->v, po = npairs(o), pv = npairs(v), ov = o * v;
  constexpr int bits = kSlicedBits;
  SlMat *op = E.sop;
  sl_pack_A(ex, op[EE_VAT], E.Va.c(), v, o * pv, 1, v, false, bits);
  sl_pack_A(ex, op[EE_VAC], E.Va.c(), o * pv, v, v, 1, true, bits);
  sl_pack_A(ex, op[EE_VB], E.Vb.c(), o, po * v, po * v, 1, false, bits);
  sl_pack_A(ex, op[EE_VBC], E.Vb.c(), po * v, o, 1, po * v, true, bits);
  if (dd) {
    sl_pack_A(ex, op[EE_GVV], E.Gvv.c(), pv, pv, pv, 1, false, bits);
    sl_pack_A(ex, op[EE_GOO], E.Goo.c(), po, po, po, 1, false, bits);
    sl_pack_A(ex, op[EE_W], c->W.c(), ov, ov, ov, 1, false, bits);
  }
  if (!E.tcerr.p) {
    E.tcerr = DBuf(ex, sizeof(int));
    fill_zero(ex, E.tcerr.p, sizeof(int));
  }
  E.sl_dd = dd;
  E.sl_ready = true;
}

// ee_struct_apply with the GEMMs over the doubles on the tensor cores, as the
// BF16x3/BF16x6 split (nseg 3 or 6) or as the sliced FP64-accurate product
// (nseg 0). The separable second-order pieces (o x o and v x v intermediates):
// with the split, their contractions over the long (l, c<d) and ((k<l), d)
// indices and their updates of the gathered doubles run on the tensor cores
// as well (the small products against V1, V2 stay FP64); with the sliced
// product they go through zgemm, which the caller switches to the sliced route
static void ee_struct_apply_tc(adc_ctx *c, const cplx *X, cplx *S, int64_t kc, double sdd, int nseg, int bits) {
  Exec &ex = c->ex;
  EEOps &E = *c->ee;
  const int64_t o = c->o, v = c->v, n1 = c->n1, N = c->N, po = npairs(o), pv = npairs(v), ov = o * v;
  if (po == 0 || pv == 0 || kc <= 0) return;
  const int *pio = (const int *)E.pair_o.p, *pjo = pio + std::max<int64_t>(po, 1);
  const int *pav = (const int *)E.pair_v.p, *pbv = pav + std::max<int64_t>(pv, 1);
  const bool second = (c->order == 3 && c->x != 0.0);
  const double x = second ? c->x : 0.0;
  int *err = (int *)E.tcerr.p;
  const bool sliced = (nseg == 0);
  const int planes = (nseg == 6) ? 3 : 2;
  const TcMat *tops[EE_NOPS] = {&E.tVaT, &E.tVaC, &E.tVb, &E.tVbC, &E.tGvv, &E.tGoo, &E.tW};
  // out = alpha op B^T + beta out, B[n][k] = src[(n / b_in) b_nh + (n % b_in) b_nl + k b_k]
  auto mul = [&](int op, const cplx *src, int64_t Nc, int64_t K, int64_t b_nh, int64_t b_nl, int64_t b_in,
                 int64_t b_k, int64_t M, cplx alpha, cplx beta, cplx *out, int64_t s_m, int64_t s_nh, int64_t s_nl,
                 int64_t n_in) {
    if (sliced) {
      const SlMat &A = E.sop[op];
      sl_pack_B(ex, E.sbx, src, Nc, K, b_nh, b_nl, b_in, b_k, false, A, bits);
      sl_gemm(ex, A, E.sbx, M, Nc, alpha, beta, out, s_m, s_nh, s_nl, n_in, err, E.slw);
    } else {
      tc_pack_B(ex, E.bx, src, Nc, K, b_nh, b_nl, b_in, b_k, false, planes);
      tc_gemm(ex, *tops[op], E.bx, M, Nc, alpha, beta, out, s_m, s_nh, s_nl, n_in, err, nseg);
    }
  };
  TagScope tg(ex, "ee_coupling");
  {
    DBuf Xa = cbuf(ex, kc * o * o * pv);
    k_gather_xa<<<grid1d(kc * o * o * pv, 256), 256, 0, ex.stream>>>(X + n1, N, kc, pav, pbv, o, v, pv, Xa.c());
    ADC_CHECK_LAUNCH();
    // S1[z][i][a] += sum_(l,cd) Va[(l,cd)][a] Xa[z][i][(l,cd)]
    mul(EE_VAT, Xa.c(), kc * o, o * pv, o * pv, 0, 1, 1, v, C1(), C1(), S, 1, N, v, o);
    DBuf U;
    if (second) {
      DBuf Y1 = cbuf(ex, kc * o * o);
      if (sliced) {
        zgemm(ex, o, o, o * pv, kc, C1(), Xa.c(), o * o * pv, o * pv, 1, false, E.T1p.c(), 0, o, 1, false, C0(),
              Y1.c(), o * o, o, 1);
      } else {
        // Y1[z][i][M] = sum_(l,cd) T1p[(l,cd)][M] Xa[z][i][(l,cd)]
        tc_pack_B(ex, E.bx, Xa.c(), kc * o, o * pv, o * pv, 0, 1, 1, false, planes);
        tc_gemm(ex, E.tT1T, E.bx, o, kc * o, C1(), C0(), Y1.c(), 1, o, 0, 1, err, nseg);
      }
      zgemm(ex, kc, n1, o * o, 1, CR(x), Y1.c(), 0, o * o, 1, false, E.V1.c(), 0, 1, o * o, false, C1(), S, 0, N, 1);
      U = cbuf(ex, kc * o * o);
      zgemm(ex, kc, o * o, n1, 1, C1(), X, 0, N, 1, false, E.V1.c(), 0, o * o, 1, true, C0(), U.c(), 0, o * o, 1);
    }
    // F[z][i][(l,cd)] = sum_a conj(Va[(l,cd)][a]) X1[z][i][a]
    mul(EE_VAC, X, kc * o, v, N, v, o, 1, o * pv, C1(), C0(), Xa.c(), 1, o * o * pv, o * pv, o);
    if (second) {
      if (sliced) {
        zgemm(ex, o, o * pv, o, kc, CR(x), U.c(), o * o, o, 1, false, E.T1p.c(), 0, 1, o, true, C1(), Xa.c(),
              o * o * pv, o * pv, 1);
      } else {
        // Xa[z][i][(l,cd)] += x sum_M conj(T1p[(l,cd)][M]) U[z][i][M]
        tc_pack_B(ex, E.bx, U.c(), kc * o, o, o, 0, 1, 1, false, planes);
        tc_gemm(ex, E.tT1C, E.bx, o * pv, kc * o, CR(x), C1(), Xa.c(), 1, o * pv, 0, 1, err, nseg);
      }
    }
    k_scatter_f<<<grid1d(kc * po * pv, 256), 256, 0, ex.stream>>>(Xa.c(), kc, pio, pjo, o, po, pv, S + n1, N);
    ADC_CHECK_LAUNCH();
  }
  {
    DBuf Xb = cbuf(ex, kc * v * po * v);
    k_gather_xbt<<<grid1d(kc * v * po * v, 256), 256, 0, ex.stream>>>(X + n1, N, kc, pio, pjo, o, v, po, pv,
                                                                     Xb.c());
    ADC_CHECK_LAUNCH();
    // S1[z][i][a] += sum_((kl),d) Vb[i][((kl),d)] XbT[z][a][((kl),d)]
    mul(EE_VB, Xb.c(), kc * v, po * v, po * v, 0, 1, 1, o, C1(), C1(), S, v, N, 1, v);
    DBuf U2;
    if (second) {
      DBuf Y2 = cbuf(ex, kc * v * v);
      if (sliced) {
        zgemm(ex, v, v, po * v, kc, C1(), Xb.c(), v * po * v, po * v, 1, false, E.T2p.c(), 0, v, 1, false, C0(),
              Y2.c(), v * v, v, 1);
      } else {
        // Y2[z][c][A] = sum_((kl),d) T2p[((kl),d)][A] XbT[z][c][((kl),d)]
        tc_pack_B(ex, E.bx, Xb.c(), kc * v, po * v, po * v, 0, 1, 1, false, planes);
        tc_gemm(ex, E.tT2T, E.bx, v, kc * v, C1(), C0(), Y2.c(), 1, v, 0, 1, err, nseg);
      }
      zgemm(ex, kc, n1, v * v, 1, CR(x), Y2.c(), 0, v * v, 1, false, E.V2.c(), 0, 1, v * v, false, C1(), S, 0, N, 1);
      U2 = cbuf(ex, kc * v * v);
      zgemm(ex, kc, v * v, n1, 1, C1(), X, 0, N, 1, false, E.V2.c(), 0, v * v, 1, true, C0(), U2.c(), 0, v * v, 1);
    }
    // G[z][((kl),d)][a] = sum_i conj(Vb[i][((kl),d)]) X1[z][i][a]  (reusing the buffer)
    mul(EE_VBC, X, kc * v, o, N, 1, v, v, po * v, C1(), C0(), Xb.c(), v, po * v * v, 1, v);
    if (second) {
      if (sliced) {
        zgemm(ex, po * v, v, v, kc, CR(x), E.T2p.c(), 0, v, 1, true, U2.c(), v * v, 1, v, false, C1(), Xb.c(),
              po * v * v, v, 1);
      } else {
        // G[z][((kl),d)][a] += x sum_A conj(T2p[((kl),d)][A]) U2[z][a][A]
        tc_pack_B(ex, E.bx, U2.c(), kc * v, v, v, 0, 1, 1, false, planes);
        tc_gemm(ex, E.tT2C, E.bx, po * v, kc * v, CR(x), C1(), Xb.c(), v, po * v * v, 1, v, err, nseg);
      }
    }
    k_scatter_g<<<grid1d(kc * po * pv, 256), 256, 0, ex.stream>>>(Xb.c(), kc, pav, pbv, v, po, pv, S + n1, N);
    ADC_CHECK_LAUNCH();
  }
  if (sdd == 0.0) return;
  ex.tag = "ee_ladder";
  mul(EE_GVV, X + n1, kc * po, pv, N, pv, po, 1, pv, CR(sdd), C1(), S + n1, 1, N, pv, po);
  mul(EE_GOO, X + n1, kc * pv, po, N, 1, pv, pv, po, CR(sdd), C1(), S + n1, pv, N, 1, pv);
  ex.tag = "ee_ring";
  const int64_t ncol = kc * ov;
  DBuf Xt = cbuf(ex, ncol * ov), R = cbuf(ex, ov * ncol);
  k_gather_xtt<<<grid1d(ncol * ov, 256), 256, 0, ex.stream>>>(X + n1, N, kc, o, v, pv, Xt.c());
  ADC_CHECK_LAUNCH();
  mul(EE_W, Xt.c(), ncol, ov, ov, 0, 1, 1, ov, C1(), C0(), R.c(), ncol, 1, 0, 1);
  Xt.reset();
  k_scatter_ring<<<grid1d(kc * po * pv, 256), 256, 0, ex.stream>>>(R.c(), kc, pio, pjo, pav, pbv, o, v, po, pv, sdd,
                                                                   S + n1, N);
  ADC_CHECK_LAUNCH();
}

void sigma_ee_split(adc_ctx *c, const cplx *X, cplx *S, int64_t k, int nseg, int bits) {
  Exec &ex = c->ex;
  EEOps &E = *c->ee;
  const int64_t o = c->o, v = c->v, n1 = c->n1, n2 = c->n2, N = c->N;
  const int64_t po = npairs(o), pv = npairs(v);
  const bool third = (c->order == 3) && (c->x != 0.0);
  const double sdd = (third && c->dd_order == 1) ? c->x : 0.0;
  const int planes = (nseg == 6) ? 3 : 2;
  ee_struct_build(c, sdd != 0.0);
  if (nseg == 0) {
    if (!E.sl_ready) ee_sl_build(c, sdd != 0.0);
  } else if (!E.tc_ready || E.tc_planes < planes) {
    ee_tc_build(c, sdd != 0.0, planes);
  }
  TagScope tg(ex, "ee");
  zgemm(ex, k, n1, n1, 1, C1(), X, 0, N, 1, false, E.MSS.c(), 0, 1, n1, false, C0(), S, 0, N, 1);
  ADC_CUDA(cudaMemset2DAsync(S + n1, N * sizeof(cplx), 0, n2 * sizeof(cplx), k, ex.stream));
  diag_mul_add(ex, k, n2, c->d2.d(), X + n1, N, S + n1, N, 1.0);
  int64_t per = std::max<int64_t>(o * o * pv, po * v * v);
  if (sdd != 0.0) per = std::max<int64_t>(per, 3 * o * v * o * v);
  per *= (int64_t)sizeof(cplx);
  const int64_t kc = std::max<int64_t>(1, std::min<int64_t>(k, (4ll << 30) / std::max<int64_t>(per, 1)));
  // with the sliced products, the separable second-order pieces (zgemm over
  // the long (l, c<d) and ((k<l), d) indices) run as sliced products too; next
  // to the BF16 split they stay FP64 (measured: faster there)
  const int old_bits = ex.sliced_bits;
  if (nseg == 0) ex.sliced_bits = bits;
  try {
    for (int64_t z0 = 0; z0 < k; z0 += kc) {
      const int64_t kk = std::min(kc, k - z0);
      ee_struct_apply_tc(c, X + z0 * N, S + z0 * N, kk, sdd, nseg, bits);
    }
  } catch (...) {
    ex.sliced_bits = old_bits;
    throw;
  }
  ex.sliced_bits = old_bits;
  int h = 0;
  ADC_CUDA(cudaMemcpyAsync(&h, E.tcerr.p, sizeof(int), cudaMemcpyDeviceToHost, ex.stream));
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
  if (h != 0) {
    fill_zero(ex, E.tcerr.p, sizeof(int));
    throw Error(ADC_ERR_TIMEOUT, "tensor-core GEMM wait gave up (code " + std::to_string(h) + ")");
  }
}

// the operands of the EE products a solve will use, built ahead of its subspace
// (planes: 0 = no split-precision copies, 2 or 3 = BF16x3 or BF16x6)
void ee_prepare(adc_ctx *c, int planes, bool sliced) {
  EEOps &E = *c->ee;
  const bool third = (c->order == 3) && (c->x != 0.0);
  const bool dd = third && c->dd_order == 1;
  ee_struct_build(c, dd);
  if (planes > 0 && (!E.tc_ready || E.tc_planes < planes)) ee_tc_build(c, dd, planes);
  if (sliced && !E.sl_ready) ee_sl_build(c, dd);
  // a mixed solve with sliced refinement reads only the split and sliced
  // copies of the packed <ab||cd>; above 4 GiB its FP64 copy makes room for
  // the subspace and is assembled again by the next FP64 product
  if (dd && planes > 0 && sliced && E.Gvv.bytes > (4ull << 30)) E.Gvv.reset();
}

}  // namespace adc
