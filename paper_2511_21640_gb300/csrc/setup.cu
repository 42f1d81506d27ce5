// One-time construction of the IP/EA-ADC operators on the device (FP64).
//
// Everything that does not depend on the trial vectors is built here from the
// Cholesky vectors and orbital energies: first- and second-order MP
// amplitudes, ground-state densities, the static main block (1h or 1p, up to
// third order), the coupling block (first + x * second order), the packed
// ladder integrals, the ring integrals and the exact diagonal.
//
// Matrix elements follow the ISR construction of Sec. 2.1 (Eqs. 5-7, 11-12):
//   lowest class (IP 1h / EA 1p), orthonormalised within itself:
//     EA  M_ab = eps_a d_ab - 1/2 sum_klc t_kl^ac <kl||bc> + 1/2 (eps_a - eps_b) g_ba
//              + x [Y3_ab + 1/2 (eps_a - eps_b) g3_ba]
//     IP  M_ij = -eps_i d_ij + 1/2 sum_kcd <kj||cd> t_ik^cd - 1/2 (eps_i - eps_j) h_ji
//              + x [Y3_ij - 1/2 (eps_i - eps_j) h3_ji]
//   coupling (2p1h: a+_a a+_b a_j, 2h1p: a+_a a_i a_j):
//     EA  M_c,kde = <ck||de> + x [1/2 sum_mn <ck||mn> t*_mn^de + P(de) sum_gm <cg||em> t*_km^gd]
//     IP  M_k,ija = <ji||ak> + x [1/2 sum_ef <ef||ak> t*_ji^ef - P(ij) sum_fm <fi||mk> t*_jm^fa]
//   satellite: zeroth-order diagonal + x * first-order ladder and ring terms.
// <pq||rs> = sum_Q (B_pr B_qs - B_ps B_qr) (Sec. 2.5, Eq. 43); ladder (4- and
// 3-external) classes are assembled from B on the device, never read from host.
#include "ctx.cuh"

namespace adc {

TV Bview(adc_ctx *c, char p, char q) {
  int64_t p0 = (p == 'o') ? 0 : c->o, q0 = (q == 'o') ? 0 : c->o;
  int64_t np = (p == 'o') ? c->o : c->v, nq = (q == 'o') ? c->o : c->v;
  return TV(c->B.c() + p0 * c->nmo + q0, {c->Q, np, nq}, {c->nmo * c->nmo, c->nmo, 1});
}

int64_t dim_of(adc_ctx *c, char x) { return x == 'o' ? c->o : c->v; }

// dense <pq||rs> block [p][q][r][s]
DBuf eri_block(adc_ctx *c, const char *spec) {
  std::vector<int64_t> e = {dim_of(c, spec[0]), dim_of(c, spec[1]), dim_of(c, spec[2]),
                            dim_of(c, spec[3])};
  DBuf out = cbuf(c->ex, e[0] * e[1] * e[2] * e[3]);
  TV O = TV::dense(out.c(), e);
  einsum(c->ex, C1(), Bview(c, spec[0], spec[2]), "Qpr", Bview(c, spec[1], spec[3]), "Qqs", C0(), O,
         "pqrs");
  einsum(c->ex, CR(-1.0), Bview(c, spec[0], spec[3]), "Qps", Bview(c, spec[1], spec[2]), "Qqr", C1(),
         O, "pqrs");
  return out;
}

namespace {

DBuf eri(adc_ctx *c, const char *spec) { return eri_block(c, spec); }

TV dense(const DBuf &b, std::vector<int64_t> e) { return TV::dense(b.c(), e); }

// packed <ab||cd>, a<b, c<d, rows [(ab) - p0][Pv], from J_(ac),(bd) = sum_Q B_ac B_bd
// computed one block of a at a time (only b >= a0 is formed).
__global__ void k_assemble_ladder(const cplx *__restrict__ J, int64_t a0, int64_t ca, int64_t v,
                                  cplx *G, int64_t total, int64_t p0) {
  // J layout: [a - a0][c][b - a0][d], b range v - a0
  const int64_t nb = v - a0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t d = idx % v, r = idx / v;
    int64_t cc = r % v; r /= v;
    int64_t bb = r % nb; r /= nb;
    int64_t aa = r;  // < ca
    int64_t a = a0 + aa, b = a0 + bb;
    if (!(a < b) || !(cc < d)) continue;
    cplx j1 = J[((aa * v + cc) * nb + bb) * v + d];
    cplx j2 = J[((aa * v + d) * nb + bb) * v + cc];
    G[(pair_index(a, b, v) - p0) * (v * (v - 1) / 2) + pair_index(cc, d, v)] = csub(j1, j2);
  }
}

__global__ void k_diag_ea(const cplx *M11, const double *g, const double *eo, const double *ev,
                          int64_t o, int64_t v, double x, double *diag, double *d2) {
  const int64_t nmo = o + v, pv = v * (v - 1) / 2, n2 = o * pv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < v + n2;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (idx < v) { diag[idx] = M11[idx * v + idx].x; continue; }
    int64_t r = idx - v;
    int64_t j = r / pv, pr = r % pv;
    // invert the pair index: a is the largest row with start <= pr
    int64_t a = 0;
    while ((a + 1) * v - (a + 1) * (a + 2) / 2 <= pr) ++a;
    int64_t b = pr - (a * v - a * (a + 1) / 2) + a + 1;
    double z = ev[a] + ev[b] - eo[j];
    double f = g[(o + a) * nmo + (o + b)] - g[(o + a) * nmo + j] - g[(o + b) * nmo + j];
    d2[r] = z;
    diag[idx] = z + x * f;
  }
}

__global__ void k_diag_ip(const cplx *M11, const double *g, const double *eo, const double *ev,
                          int64_t o, int64_t v, double x, double *diag, double *d2) {
  const int64_t nmo = o + v, po = o * (o - 1) / 2, n2 = po * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < o + n2;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (idx < o) { diag[idx] = M11[idx * o + idx].x; continue; }
    int64_t r = idx - o;
    int64_t a = r % v, pr = r / v;
    int64_t i = 0;
    while ((i + 1) * o - (i + 1) * (i + 2) / 2 <= pr) ++i;
    int64_t j = pr - (i * o - i * (i + 1) / 2) + i + 1;
    double z = ev[a] - eo[i] - eo[j];
    double f = g[i * nmo + j] - g[(o + a) * nmo + i] - g[(o + a) * nmo + j];
    d2[r] = z;
    diag[idx] = z + x * f;
  }
}

}  // namespace

// packed ladder integrals <ab||cd> (a<b, c<d) of the virtual block
DBuf build_vvvv_packed(adc_ctx *c) {
  const int64_t v = c->v, Q = c->Q, pv = npairs(v);
  DBuf G = cbuf(c->ex, pv * pv);
  if (pv == 0) return G;
  // L[(a,c)][Q] = B^Q_ac
  DBuf L = cbuf(c->ex, v * v * Q);
  permute(c->ex, c->B.c() + c->o * c->nmo + c->o, {v, v, Q}, {c->nmo, 1, c->nmo * c->nmo}, false,
          L.c(), C1(), C0());
  // a blocks sized so that J stays below ~1 GiB
  int64_t ca = std::max<int64_t>(1, (int64_t)(1ll << 26) / (v * v * v));
  ca = std::min(ca, v);
  DBuf J = cbuf(c->ex, ca * v * v * v);
  for (int64_t a0 = 0; a0 < v - 1; a0 += ca) {
    int64_t na = std::min(ca, v - a0);
    int64_t nb = v - a0;
    // J[(a,c)][(b,d)] = sum_Q L[(a,c)][Q] L[(b,d)][Q]
    zgemm(c->ex, na * v, nb * v, Q, 1, C1(), L.c() + a0 * v * Q, 0, Q, 1, false,
          L.c() + a0 * v * Q, 0, 1, Q, false, C0(), J.c(), 0, nb * v, 1);
    int64_t total = na * v * nb * v;
    k_assemble_ladder<<<grid1d(total, 256), 256, 0, c->ex.stream>>>(J.c(), a0, na, v, G.c(), total, 0);
    ADC_CHECK_LAUNCH();
  }
  return G;
}

DBuf vvvv_L(adc_ctx *c) {
  const int64_t v = c->v, Q = c->Q;
  DBuf L = cbuf(c->ex, v * v * Q);
  permute(c->ex, c->B.c() + c->o * c->nmo + c->o, {v, v, Q}, {c->nmo, 1, c->nmo * c->nmo}, false, L.c(), C1(), C0());
  return L;
}

// complex elements of one chunk of the setup's chunked intermediates (the
// IP coupling's (ea|fk) block); a test hook lowers it to force several chunks
static int64_t g_setup_chunk_elems = (int64_t)1 << 28;
void set_setup_chunk_elems(int64_t n) { g_setup_chunk_elems = n > 0 ? n : ((int64_t)1 << 28); }

int64_t vvvv_chunk(adc_ctx *c) {
  const int64_t v = c->v;
  return std::min<int64_t>(v, std::max<int64_t>(1, ((int64_t)1 << 26) / (v * v * v)));
}

void vvvv_assemble_rows(adc_ctx *c, const cplx *J, int64_t a0, int64_t a1, cplx *Gc) {
  const int64_t v = c->v, na = a1 - a0, nb = v - a0;
  const int64_t total = na * v * nb * v;
  k_assemble_ladder<<<grid1d(total, 256), 256, 0, c->ex.stream>>>(J, a0, na, v, Gc, total, ladder_row0(a0, v));
  ADC_CHECK_LAUNCH();
}

void vvvv_rows(adc_ctx *c, const cplx *L, int64_t a0, int64_t a1, cplx *J, cplx *Gc) {
  const int64_t v = c->v, Q = c->Q, na = a1 - a0, nb = v - a0;
  // J[(a,c)][(b,d)] = sum_Q L[(a,c)][Q] L[(b,d)][Q], a in [a0, a1), b >= a0
  zgemm(c->ex, na * v, nb * v, Q, 1, C1(), L + a0 * v * Q, 0, Q, 1, false, L + a0 * v * Q, 0, 1, Q, false, C0(), J,
        0, nb * v, 1);
  vvvv_assemble_rows(c, J, a0, a1, Gc);
}

void first_order_amplitudes(adc_ctx *c) {
  Exec &ex = c->ex;
  const int64_t o = c->o, v = c->v;
  TV Boo = Bview(c, 'o', 'o'), Bov = Bview(c, 'o', 'v'), Bvo = Bview(c, 'v', 'o'), Bvv = Bview(c, 'v', 'v');
  const double *eo = c->eo.d(), *ev = c->ev.d();
  // t_ij^ab = <ab||ij> / D_ij^ab
  c->t1 = cbuf(ex, o * o * v * v);
  TV t1 = dense(c->t1, {o, o, v, v});
  einsum(ex, C1(), Bvo, "Qai", Bvo, "Qbj", C0(), t1, "ijab");
  einsum(ex, CR(-1.0), Bvo, "Qaj", Bvo, "Qbi", C1(), t1, "ijab");
  denom2_div(ex, c->t1.c(), eo, ev, o, v);
  // ring integrals W[j][a][k][c] = <ak||cj>
  c->W = cbuf(ex, o * v * o * v);
  TV W = dense(c->W, {o, v, o, v});
  einsum(ex, C1(), Bvv, "Qac", Boo, "Qkj", C0(), W, "jakc");
  einsum(ex, CR(-1.0), Bvo, "Qaj", Bov, "Qkc", C1(), W, "jakc");
}

void second_order_amplitudes(adc_ctx *c, DBuf &G_vv, DBuf &Lad_b, DBuf &t2d_b, DBuf &t2s_b) {
  Exec &ex = c->ex;
  const int64_t o = c->o, v = c->v, Q = c->Q;
  const int64_t po = npairs(o), pv = npairs(v);
  TV Bov = Bview(c, 'o', 'v'), Bvv = Bview(c, 'v', 'v');
  const double *eo = c->eo.d(), *ev = c->ev.d();
  TV t1 = dense(c->t1, {o, o, v, v});
  TV W = dense(c->W, {o, v, o, v});
    // Lad_ij^ab = 1/2 sum_cd <ab||cd> t_ij^cd = sum_{c<d} G[(ab),(cd)] t_ij^cd
    DBuf tp1 = cbuf(ex, o * o * pv), tp2 = cbuf(ex, po * pv);
    pair_pack(ex, c->t1.c(), 0, v * v, v, 1, 0, 0.0, 1, o * o, v, 1, tp1.c(), 0, pv, C1(), C0());
    pair_pack(ex, tp1.c(), 0, 0, o * pv, pv, 1, 0.0, 1, 1, o, pv, tp2.c(), 0, 0, C1(), C0());
    DBuf lp = cbuf(ex, po * pv);
    if (c->direct_ladder) {
      // integral-direct: chunks of rows (a<b) of <ab||cd>, each contracted at once
      DBuf L = vvvv_L(c);
      const int64_t ca = vvvv_chunk(c);
      DBuf J = cbuf(ex, ca * v * v * v), Gc = cbuf(ex, std::min<int64_t>(ca * v, pv) * pv);
      for (int64_t a0 = 0; a0 < v - 1; a0 += ca) {
        const int64_t a1 = std::min(v - 1, a0 + ca), r0 = ladder_row0(a0, v), r1 = ladder_row0(a1, v);
        vvvv_rows(c, L.c(), a0, a1, J.c(), Gc.c());
        zgemm(ex, po, r1 - r0, pv, 1, C1(), tp2.c(), 0, pv, 1, false, Gc.c(), 0, 1, pv, false, C0(), lp.c() + r0, 0,
              pv, 1);
      }
    } else {
      G_vv = build_vvvv_packed(c);
      zgemm(ex, po, pv, pv, 1, C1(), tp2.c(), 0, pv, 1, false, G_vv.c(), 0, 1, pv, false, C0(), lp.c(),
            0, pv, 1);
    }
    DBuf l1 = cbuf(ex, po * v * v);
    pair_unpack(ex, lp.c(), 1, po, 0, pv, v, 1, l1.c());
    Lad_b = cbuf(ex, o * o * v * v);
    pair_unpack(ex, l1.c(), 1, 1, 0, 0, o, v * v, Lad_b.c());
    tp1.reset(); tp2.reset(); lp.reset(); l1.reset();
    TV Lad = dense(Lad_b, {o, o, v, v});

    // t2_ij^ab D = Lad + 1/2 sum_kl <kl||ij> t_kl^ab + P(ij)P(ab) sum_kc <kb||cj> t_ik^ac
    t2d_b = cbuf(ex, o * o * v * v);
    ADC_CUDA(cudaMemcpyAsync(t2d_b.c(), Lad_b.c(), o * o * v * v * sizeof(cplx),
                             cudaMemcpyDeviceToDevice, ex.stream));
    TV t2d = dense(t2d_b, {o, o, v, v});
    {
      DBuf oooo = eri(c, "oooo");
      einsum(ex, CR(0.5), dense(oooo, {o, o, o, o}), "klij", t1, "klab", C1(), t2d, "ijab");
    }
    {
      // Rg[i][a][j][b] = sum_kc <kb||cj> t_ik^ac = -sum_kc W[j][b][k][c] t[i][k][a][c]
      DBuf Rg = cbuf(ex, o * v * o * v);
      einsum(ex, CR(-1.0), W, "jbkc", t1, "ikac", C0(), dense(Rg, {o, v, o, v}), "iajb");
      const int64_t sRi = v * o * v, sRa = o * v, sRj = v, sRb = 1;
      std::vector<int64_t> e = {o, o, v, v};
      permute(ex, Rg.c(), e, {sRi, sRj, sRa, sRb}, false, t2d_b.c(), C1(), C1());
      permute(ex, Rg.c(), e, {sRj, sRi, sRa, sRb}, false, t2d_b.c(), CR(-1.0), C1());
      permute(ex, Rg.c(), e, {sRi, sRj, sRb, sRa}, false, t2d_b.c(), CR(-1.0), C1());
      permute(ex, Rg.c(), e, {sRj, sRi, sRb, sRa}, false, t2d_b.c(), C1(), C1());
    }
    denom2_div(ex, t2d_b.c(), eo, ev, o, v);

    t2s_b = second_order_singles(c);
}

DBuf second_order_singles(adc_ctx *c) {
  Exec &ex = c->ex;
  const int64_t o = c->o, v = c->v, Q = c->Q;
  TV Bov = Bview(c, 'o', 'v'), Bvv = Bview(c, 'v', 'v');
  TV t1 = dense(c->t1, {o, o, v, v});
  // t2_i^a (eps_i - eps_a) = 1/2 sum_jcd <aj||cd> t_ij^cd - 1/2 sum_jkc <jk||ic> t_jk^ac
  DBuf t2s_b = cbuf(ex, o * v);
  TV t2s = dense(t2s_b, {o, v});
  {
    DBuf Y = cbuf(ex, Q * o * v);
    einsum(ex, C1(), Bov, "Qjd", t1, "ijcd", C0(), dense(Y, {Q, o, v}), "Qic");
    einsum(ex, C1(), Bvv, "Qac", dense(Y, {Q, o, v}), "Qic", C0(), t2s, "ia");
    DBuf ooov = eri(c, "ooov");
    einsum(ex, CR(-0.5), dense(ooov, {o, o, o, v}), "jkic", t1, "jkac", C1(), t2s, "ia");
  }
  denom1_div(ex, t2s_b.c(), c->eo.d(), c->ev.d(), o, v);
  return t2s_b;
}

void setup_operators(adc_ctx *c) {
  Exec &ex = c->ex;
  const int64_t o = c->o, v = c->v, Q = c->Q;
  const bool third = (c->order == 3) && (c->x != 0.0);
  const double x = c->x;
  const int64_t po = npairs(o), pv = npairs(v);
  TV Boo = Bview(c, 'o', 'o'), Bov = Bview(c, 'o', 'v'), Bvo = Bview(c, 'v', 'o'),
     Bvv = Bview(c, 'v', 'v');
  const double *eo = c->eo.d(), *ev = c->ev.d();

  // packed <ab||cd> (EA satellite ladder, and the ladder intermediate of the
  // second-order amplitudes of both kinds): stored, or integral-direct when it
  // would take more than a quarter of the free device memory (opts.ladder)
  c->direct_ladder = false;
  if (third) {
    if (c->opts.ladder == 1) {
      c->direct_ladder = true;
    } else if (c->opts.ladder == 0) {
      size_t fr = 0, tot = 0;
      ADC_CUDA(cudaMemGetInfo(&fr, &tot));
      c->direct_ladder = (double)pv * (double)pv * sizeof(cplx) > 0.25 * (double)fr;
    }
  }
  StageScope stage(ex, "first_order_amplitudes");
  first_order_amplitudes(c);
  TV t1 = dense(c->t1, {o, o, v, v});
  DBuf oovv = cbuf(ex, o * o * v * v);
  oovv_from_t1(ex, c->t1.c(), eo, ev, o, v, oovv.c());
  TV Toovv = dense(oovv, {o, o, v, v});
  TV W = dense(c->W, {o, v, o, v});

  // ---- second-order densities of Psi1
  stage.next("densities");
  DBuf gvv_b = cbuf(ex, v * v), hoo_b = cbuf(ex, o * o);
  TV gvv = dense(gvv_b, {v, v}), hoo = dense(hoo_b, {o, o});
  einsum(ex, CR(0.5), t1.cj(), "ijdf", t1, "ijef", C0(), gvv, "de");
  einsum(ex, CR(0.5), t1.cj(), "njef", t1, "mjef", C0(), hoo, "nm");

  // ---- second-order amplitudes, ladder intermediate, R (third order only)
  stage.next("second_order_amplitudes");
  DBuf t2d_b, t2s_b, R_b, Lad_b, G_vv;
  if (third) {
    second_order_amplitudes(c, G_vv, Lad_b, t2d_b, t2s_b);
    // R[c][a][n][m] = sum_jf conj(t_nj^cf) t_mj^af
    R_b = cbuf(ex, v * v * o * o);
    einsum(ex, C1(), t1.cj(), "njcf", t1, "mjaf", C0(), dense(R_b, {v, v, o, o}), "canm");
  }

  // ---- main block
  stage.next("main_block");
  c->M11 = cbuf(ex, c->n1 * c->n1);
  fill_zero(ex, c->M11.p, c->M11.bytes);
  if (c->kind == ADC_EA) {
    TV M = dense(c->M11, {v, v});
    add_diag(ex, c->M11.c(), ev, v, 1.0);
    einsum(ex, CR(-0.5), t1, "klac", Toovv, "klbc", C1(), M, "ab");
    add_eps_diff_transpose(ex, c->M11.c(), gvv_b.c(), ev, v, 0.5);
    if (third && x != 0.0) {
      DBuf M3b = cbuf(ex, v * v);
      TV M3 = dense(M3b, {v, v});
      TV t2d = dense(t2d_b, {o, o, v, v}), t2s = dense(t2s_b, {o, v});
      einsum(ex, CR(-0.5), t2d, "klac", Toovv, "klbc", C0(), M3, "ab");
      {  // - sum_md <ma||bd> t2_m^d,  <ma||bd> = sum_Q (B_mb B_ad - B_md B_ab)
        DBuf Z = cbuf(ex, Q * v * v), u = cbuf(ex, Q);
        einsum(ex, C1(), Bov, "Qmb", t2s, "md", C0(), dense(Z, {Q, v, v}), "Qdb");
        einsum(ex, CR(-1.0), Bvv, "Qad", dense(Z, {Q, v, v}), "Qdb", C1(), M3, "ab");
        einsum(ex, C1(), Bov, "Qmd", t2s, "md", C0(), dense(u, {Q}), "Q");
        einsum(ex, C1(), Bvv, "Qab", dense(u, {Q}), "Q", C1(), M3, "ab");
      }
      {  // + sum_dk <ad||bk> conj(t2_k^d),  <ad||bk> = sum_Q (B_ab B_dk - B_ak B_db)
        DBuf Z = cbuf(ex, Q * o * v), u = cbuf(ex, Q);
        einsum(ex, C1(), Bvo, "Qdk", t2s.cj(), "kd", C0(), dense(u, {Q}), "Q");
        einsum(ex, C1(), Bvv, "Qab", dense(u, {Q}), "Q", C1(), M3, "ab");
        einsum(ex, C1(), Bvv, "Qdb", t2s.cj(), "kd", C0(), dense(Z, {Q, o, v}), "Qkb");
        einsum(ex, CR(-1.0), Bvo, "Qak", dense(Z, {Q, o, v}), "Qkb", C1(), M3, "ab");
      }
      {  // + sum_de <ad||be> g_de,  <ad||be> = sum_Q (B_ab B_de - B_ae B_db)
        DBuf Z = cbuf(ex, Q * v * v), u = cbuf(ex, Q);
        einsum(ex, C1(), Bvv, "Qde", gvv, "de", C0(), dense(u, {Q}), "Q");
        einsum(ex, C1(), Bvv, "Qab", dense(u, {Q}), "Q", C1(), M3, "ab");
        einsum(ex, C1(), Bvv, "Qae", gvv, "de", C0(), dense(Z, {Q, v, v}), "Qad");
        einsum(ex, CR(-1.0), dense(Z, {Q, v, v}), "Qad", Bvv, "Qdb", C1(), M3, "ab");
      }
      // + 1/4 sum <cd||be> conj(t_ij^cd) t_ij^ea = 1/2 sum conj(Lad_ij^be) t_ij^ea
      einsum(ex, CR(0.5), dense(Lad_b, {o, o, v, v}).cj(), "ijbe", t1, "ijea", C1(), M3, "ab");
      // + sum_mn <ma||bn> h_nm = - sum W[n][a][m][b] h_nm
      einsum(ex, CR(-1.0), W, "namb", hoo, "nm", C1(), M3, "ab");
      // - sum_mcn <mc||bn> R_ca,nm = + sum W[n][c][m][b] R[c][a][n][m]
      einsum(ex, C1(), W, "ncmb", dense(R_b, {v, v, o, o}), "canm", C1(), M3, "ab");
      // + 1/2 (eps_a - eps_b) g3_ba
      DBuf g3 = cbuf(ex, v * v);
      einsum(ex, CR(0.5), t1.cj(), "ijdf", t2d, "ijef", C0(), dense(g3, {v, v}), "de");
      einsum(ex, CR(0.5), t2d.cj(), "ijdf", t1, "ijef", C1(), dense(g3, {v, v}), "de");
      add_eps_diff_transpose(ex, M3b.c(), g3.c(), ev, v, 0.5);
      zaxpby(ex, v * v, CR(x), M3b.c(), C1(), c->M11.c());
    }
  } else {
    TV M = dense(c->M11, {o, o});
    add_diag(ex, c->M11.c(), eo, o, -1.0);
    einsum(ex, CR(0.5), Toovv, "kjcd", t1, "ikcd", C1(), M, "ij");
    add_eps_diff_transpose(ex, c->M11.c(), hoo_b.c(), eo, o, -0.5);
    if (third && x != 0.0) {
      DBuf M3b = cbuf(ex, o * o);
      TV M3 = dense(M3b, {o, o});
      TV t2d = dense(t2d_b, {o, o, v, v}), t2s = dense(t2s_b, {o, v});
      einsum(ex, CR(0.5), Toovv, "kjcd", t2d, "ikcd", C0(), M3, "ij");
      {
        DBuf oovo = eri(c, "oovo");
        einsum(ex, CR(-1.0), dense(oovo, {o, o, v, o}), "kjei", t2s, "ke", C1(), M3, "ij");
        DBuf vooo = eri(c, "vooo");
        einsum(ex, C1(), dense(vooo, {v, o, o, o}), "cjik", t2s.cj(), "kc", C1(), M3, "ij");
      }
      {
        DBuf oooo = eri(c, "oooo");
        TV O4 = dense(oooo, {o, o, o, o});
        einsum(ex, C1(), O4, "kjli", hoo, "lk", C1(), M3, "ij");
        DBuf Zo = cbuf(ex, o * o * o * o);
        einsum(ex, C1(), t1.cj(), "lmef", t1, "ikef", C0(), dense(Zo, {o, o, o, o}), "lmik");
        einsum(ex, CR(0.25), O4, "kjlm", dense(Zo, {o, o, o, o}), "lmik", C1(), M3, "ij");
      }
      // - sum_cd <cj||di> g_cd = - sum W[i][c][j][d] g_cd
      einsum(ex, CR(-1.0), W, "icjd", gvv, "cd", C1(), M3, "ij");
      // + sum <cj||dk> R[c][d][k][i] = sum W[k][c][j][d] R[c][d][k][i]
      einsum(ex, C1(), W, "kcjd", dense(R_b, {v, v, o, o}), "cdki", C1(), M3, "ij");
      DBuf h3 = cbuf(ex, o * o);
      einsum(ex, CR(0.5), t1.cj(), "jkcd", t2d, "ikcd", C0(), dense(h3, {o, o}), "ji");
      einsum(ex, CR(0.5), t2d.cj(), "jkcd", t1, "ikcd", C1(), dense(h3, {o, o}), "ji");
      add_eps_diff_transpose(ex, M3b.c(), h3.c(), eo, o, -0.5);
      zaxpby(ex, o * o, CR(x), M3b.c(), C1(), c->M11.c());
    }
  }
  Lad_b.reset(); R_b.reset(); t2d_b.reset(); t2s_b.reset();

  // ---- coupling block
  stage.next("coupling");
  c->Cpl = cbuf(ex, c->n1 * c->n2);
  if (c->kind == ADC_EA) {
    // <ck||de> = J(c,k,d,e) - J(c,k,e,d), J = sum_Q B_cd B_ke
    {
      DBuf J = cbuf(ex, v * o * v * v);
      einsum(ex, C1(), Bvv, "Qcd", Bov, "Qke", C0(), dense(J, {v, o, v, v}), "ckde");
      pair_pack(ex, J.c(), 0, v * v, v, 1, 0, 1.0, 1, v * o, v, 1, c->Cpl.c(), 0, pv, C1(), C0());
    }
    if (third && x != 0.0) {
      {
        DBuf vooo = eri(c, "vooo");
        DBuf TA = cbuf(ex, v * o * v * v);
        einsum(ex, CR(0.5), dense(vooo, {v, o, o, o}), "ckmn", t1.cj(), "mnde", C0(),
               dense(TA, {v, o, v, v}), "ckde");
        pair_pack(ex, TA.c(), 0, v * v, v, 1, 0, 0.0, 1, v * o, v, 1, c->Cpl.c(), 0, pv, CR(x), C1());
      }
      {
        // U[c][k][e][d] = sum_gm <cg||em> conj(t_km^gd), <cg||em> = sum_Q (B_ce B_gm - B_cm B_ge)
        DBuf U = cbuf(ex, v * o * v * v);
        TV Ut = dense(U, {v, o, v, v});
        DBuf Y = cbuf(ex, Q * o * v);
        einsum(ex, C1(), Bvo, "Qgm", t1.cj(), "kmgd", C0(), dense(Y, {Q, o, v}), "Qkd");
        einsum(ex, C1(), Bvv, "Qce", dense(Y, {Q, o, v}), "Qkd", C0(), Ut, "cked");
        Y.reset();
        DBuf X = cbuf(ex, v * v * v * o);  // X[c][e][g][m] = sum_Q B_cm B_ge
        einsum(ex, C1(), Bvo, "Qcm", Bvv, "Qge", C0(), dense(X, {v, v, v, o}), "cegm");
        einsum(ex, CR(-1.0), dense(X, {v, v, v, o}), "cegm", t1.cj(), "kmgd", C1(), Ut, "cked");
        X.reset();
        pair_pack(ex, U.c(), 0, v * v, v, 1, 0, 1.0, 1, v * o, v, 1, c->Cpl.c(), 0, pv, CR(-x), C1());
      }
    }
  } else {
    // T[k][i][j][a] = <ji||ak>, antisymmetric in (i, j)
    DBuf T = cbuf(ex, o * o * o * v);
    TV Tt = dense(T, {o, o, o, v});
    {
      DBuf oovo = eri(c, "oovo");
      permute(ex, oovo.c(), {o, o, o, v}, {1, o * v, o * o * v, o}, false, T.c(), C1(), C0());
    }
    if (third && x != 0.0) {
      // + x/2 sum_ef <ef||ak> conj(t_ji^ef) = x sum_ef (ea|fk) conj(t_ji^ef), in chunks of the
      // virtual index a whose (ea|fk) block stays within about 4 GiB:
      // J[a][e][k][f] = sum_Q B_ea B_fk, Tc[a][k][j][i] = sum_ef J[a][e][k][f] conj(t_ji^ef)
      const int64_t ca = std::max<int64_t>(1, std::min<int64_t>(v, g_setup_chunk_elems / (o * v * v)));
      DBuf J = cbuf(ex, ca * v * o * v), Tc = cbuf(ex, ca * o * o * o);
      for (int64_t a0 = 0; a0 < v; a0 += ca) {
        const int64_t na = std::min(ca, v - a0);
        TV Bea(Bvv.p + a0, {Q, v, na}, {Bvv.str[0], Bvv.str[1], 1});
        einsum(ex, C1(), Bea, "Qea", Bvo, "Qfk", C0(), dense(J, {na, v, o, v}), "aekf");
        einsum(ex, C1(), dense(J, {na, v, o, v}), "aekf", t1.cj(), "jief", C0(), dense(Tc, {na, o, o, o}), "akji");
        // T[k][i][j][a0 + a] += x Tc[a][k][j][i]
        permute(ex, Tc.c(), {o, o, o, na}, {o * o, 1, o, o * o * o}, false, T.c() + a0,
                {o * o * v, o * v, v, 1}, CR(x), C1());
      }
    }
    pair_pack(ex, T.c(), 0, o * o * v, o * v, v, 1, 0.0, 1, o, o, v, c->Cpl.c(), 0, po * v, C1(), C0());
    if (third && x != 0.0) {
      // - x P(ij) sum_fm <fi||mk> conj(t_jm^fa)
      DBuf vooo = eri(c, "vooo");
      einsum(ex, C1(), dense(vooo, {v, o, o, o}), "fimk", t1.cj(), "jmfa", C0(), Tt, "kija");
      pair_pack(ex, T.c(), 0, o * o * v, o * v, v, 1, 1.0, 1, o, o, v, c->Cpl.c(), 0, po * v, CR(-x), C1());
    }
  }

  // ---- ladder integrals of the satellite block (first order, x-scaled)
  stage.next("satellite_ladder");
  if (third && x != 0.0) {
    if (c->kind == ADC_EA) {
      if (!c->direct_ladder) c->Glad = std::move(G_vv);
    } else {
      // Glad[(ij)][(kl)] = <kl||ij>
      DBuf oooo = eri(c, "oooo");
      DBuf F = cbuf(ex, o * o * o * o);
      permute(ex, oooo.c(), {o, o, o, o}, {o, 1, o * o * o, o * o}, false, F.c(), C1(), C0());
      DBuf F1 = cbuf(ex, o * o * po);
      pair_pack(ex, F.c(), 0, o * o, o, 1, 0, 0.0, 1, o * o, o, 1, F1.c(), 0, po, C1(), C0());
      c->Glad = cbuf(ex, po * po);
      pair_pack(ex, F1.c(), 0, 0, o * po, po, 1, 0.0, 1, 1, o, po, c->Glad.c(), 0, 0, C1(), C0());
    }
  }
  G_vv.reset();

  // ---- diagonal
  stage.next("diagonal");
  c->diag = DBuf(ex, c->N * sizeof(double));
  c->d2 = DBuf(ex, c->n2 * sizeof(double));
  {
    DBuf g(ex, c->nmo * c->nmo * sizeof(double));
    antisym_diag(ex, c->B.c(), Q, c->nmo, g.d());
    double xe = third ? x : 0.0;
    if (c->kind == ADC_EA)
      k_diag_ea<<<grid1d(c->N, 256), 256, 0, ex.stream>>>(c->M11.c(), g.d(), eo, ev, o, v, xe,
                                                          c->diag.d(), c->d2.d());
    else
      k_diag_ip<<<grid1d(c->N, 256), 256, 0, ex.stream>>>(c->M11.c(), g.d(), eo, ev, o, v, xe,
                                                          c->diag.d(), c->d2.d());
    ADC_CHECK_LAUNCH();
  }
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
}

}  // namespace adc
