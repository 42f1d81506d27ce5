// EE-ADC(2), ADC(2)+x(3) and ADC(3): operators and FP64 sigma product.
//
// Manifold (Sec. 2.1, Eq. 2): singles a+_a a_i |Psi0>, doubles
// a+_a a_i a+_b a_j |Psi0> (i<j, a<b); vector layout [X_(i,a) | X_(i<j),(a<b)],
// the virtual pair fastest. The singles are orthogonalised against Psi0
// (Eq. 5), so M_SS = S^-1/2 K S^-1/2 with S_ia,jb = <E_ai^+ E_bj> - <E_ai^+><E_bj>
// and K_ia,jb = <E_ai^+ [H, E_bj]> (Eqs. 6-7). With W_ia,jb =
// ((eps_b - eps_j) - (eps_a - eps_i))/2 and the connected parts of the
// expectation values (Wick's theorem on the MP ground state):
//
//   M_SS = diag(eps_a - eps_i) + K1 + W o S2 + Y2
//          + x [ W o S3 + Y3 - 1/2 (S2 K1 + K1 S2) ]
//   M_SD = M1_SD + x [ (Delta_K - Delta_S) O2 + Z1 ]
//   M_DD = diag(eps_a + eps_b - eps_i - eps_j) + x dd M1_DD
//
// The tables below list every connected term (disconnected pieces cancel
// against the normalisation of Psi0). The static singles block is assembled
// once; the coupling and the doubles block are applied matrix-free.
#include "ctx.cuh"
#include "ee.cuh"

namespace adc {

namespace {

using Rows = std::vector<std::pair<const char *, const char *>>;

// singles-singles, first order: K1_ia,jb = -<aj||bi>
const Rows kK1 = {{"-1", "v(aj,bi)"}};
// connected second-order overlap <E_ai^+ E_bj>
const Rows kS2 = {{"1", "t1(aA,iM) t1c(bA,jM)"},
                  {"-1/2", "t1(aA,MN) t1c(bA,MN) d(ij)"},
                  {"-1/2", "t1(AB,iM) t1c(AB,jM) d(ab)"}};
// first-order expectation of E_ai^+ [V_N, E_bj]
const Rows kY2 = {{"1", "t1(aA,iM) v(jM,bA)"},
                  {"-1/2", "t1(aA,MN) v(MN,bA) d(ij)"},
                  {"-1/2", "t1(AB,iM) v(jM,AB) d(ab)"}};
// connected third-order overlap (t1 with the second-order doubles t2)
const Rows kS3 = {{"1", "t1(aA,iM) t2c(bA,jM)"},
                  {"1", "t1c(bA,jM) t2(aA,iM)"},
                  {"-1/2", "t1(aA,MN) t2c(bA,MN) d(ij)"},
                  {"-1/2", "t1(AB,iM) t2c(AB,jM) d(ab)"},
                  {"-1/2", "t1c(bA,MN) t2(aA,MN) d(ij)"},
                  {"-1/2", "t1c(AB,jM) t2(AB,iM) d(ab)"}};
// connected second-order expectation of E_ai^+ [V_N, E_bj]: Psi1 x Psi1 ...
const Rows kY3 = {{"1", "t1(aA,iM) t1c(AB,jN) v(BM,bN)"},
                  {"1", "t1(aA,iM) t1c(AB,MN) v(jB,bN)"},
                  {"1/2", "t1(aA,iM) t1c(bA,NO) v(jM,NO)"},
                  {"1/2", "t1(aA,MN) t1c(AB,MN) v(jB,bi)"},
                  {"1/2", "t1(AB,iM) t1c(AB,jN) v(aM,bN)"},
                  {"1/2", "t1(AB,MN) t1c(bA,MN) v(aj,iB)"},
                  {"-1", "t1(aA,iM) t1c(bB,MN) v(jB,AN)"},
                  {"-1", "t1(aA,MN) t1c(bA,MO) v(jN,iO)"},
                  {"-1", "t1(aA,MN) t1c(AB,jM) v(BN,bi)"},
                  {"-1", "t1(AB,iM) t1c(bA,MN) v(aj,BN)"},
                  {"-1/2", "t1(AB,iM) t1c(AB,MN) v(aj,bN)"},
                  {"-1/2", "t1(AB,MN) t1c(AB,jM) v(aN,bi)"},
                  {"1", "t1(AB,iM) t1c(AC,MN) v(jC,BN) d(ab)"},
                  {"1/2", "t1(AB,MN) t1c(AB,MO) v(jN,iO) d(ab)"},
                  {"-1", "t1(aA,MN) t1c(AB,MO) v(BN,bO) d(ij)"},
                  {"-1/2", "t1(AB,MN) t1c(AB,MO) v(aN,bO) d(ij)"},
                  {"-1/2", "t1(AB,MN) t1c(AC,MN) v(jC,iB) d(ab)"},
                  {"-1/4", "t1(AB,iM) t1c(AB,NO) v(jM,NO) d(ab)"},
                  // ... and Psi2 (doubles t2, singles s2) with Phi
                  {"1", "t2(aA,iM) v(jM,bA)"},
                  {"-1", "s2(a,M) v(jM,bi)"},
                  {"-1", "s2(A,i) v(aj,bA)"},
                  {"-1", "s2c(b,M) v(aj,iM)"},
                  {"-1", "s2c(A,j) v(aA,bi)"},
                  {"1", "s2(A,M) v(aM,bA) d(ij)"},
                  {"1", "s2c(A,M) v(aA,bM) d(ij)"},
                  {"-1", "s2(A,M) v(jM,iA) d(ab)"},
                  {"-1", "s2c(A,M) v(jA,iM) d(ab)"},
                  {"-1/2", "t2(aA,MN) v(MN,bA) d(ij)"},
                  {"-1/2", "t2(AB,iM) v(jM,AB) d(ab)"}};
// the rows of Y3 with four virtual indices: <ab||cd>, or (first row) the
// product of two amplitudes over four virtual indices; evaluated from these rows
// with the dense integrals, or in chunks (y3_vvvv_chunked) for large v
const Rows kY3V = {{"1/2", "t1(aA,iM) t1c(BC,jM) v(BC,bA)"},
                   {"1/2", "t1(aA,MN) t1c(bB,MN) v(jB,iA)"},
                   {"-1", "t1(AB,iM) t1c(AC,jM) v(aC,bB)"},
                   {"1/2", "t1(AB,MN) t1c(AC,MN) v(aC,bB) d(ij)"},
                   {"-1/4", "t1(aA,MN) t1c(BC,MN) v(BC,bA) d(ij)"}};
// singles-doubles, first order <Phi| E_ia^+ [V_N, C_klcd] |Phi>
const Rows kSD1 = {{"1", "v(al,cd) d(ik)"}, {"1", "v(kl,di) d(ac)"},
                   {"-1", "v(ak,cd) d(il)"}, {"-1", "v(kl,ci) d(ad)"}};
// second-order overlap <E_ia^+ C_klcd> (second-order singles)
const Rows kO2 = {{"1", "s2c(c,k) d(ad) d(il)"}, {"1", "s2c(d,l) d(ac) d(ik)"},
                  {"-1", "s2c(c,l) d(ad) d(ik)"}, {"-1", "s2c(d,k) d(ac) d(il)"}};
// first-order expectation of E_ia^+ [V_N, C_klcd]
const Rows kZ1 = {{"1", "t1c(cd,lM) v(ak,iM)"},
                  {"1", "t1c(dA,kl) v(aA,ci)"},
                  {"-1", "t1c(cd,kM) v(al,iM)"},
                  {"-1", "t1c(cA,kl) v(aA,di)"},
                  {"1", "t1c(cA,kM) v(aA,dM) d(il)"},
                  {"1", "t1c(cA,lM) v(kA,iM) d(ad)"},
                  {"1", "t1c(dA,kM) v(lA,iM) d(ac)"},
                  {"1", "t1c(dA,lM) v(aA,cM) d(ik)"},
                  {"1/2", "t1c(cd,MN) v(al,MN) d(ik)"},
                  {"1/2", "t1c(AB,kl) v(AB,di) d(ac)"},
                  {"-1", "t1c(cA,kM) v(lA,iM) d(ad)"},
                  {"-1", "t1c(cA,lM) v(aA,dM) d(ik)"},
                  {"-1", "t1c(dA,kM) v(aA,cM) d(il)"},
                  {"-1", "t1c(dA,lM) v(kA,iM) d(ac)"},
                  {"-1/2", "t1c(cd,MN) v(ak,MN) d(il)"},
                  {"-1/2", "t1c(AB,kl) v(AB,ci) d(ad)"},
                  {"1/2", "t1c(cA,MN) v(lA,MN) d(ad) d(ik)"},
                  {"1/2", "t1c(dA,MN) v(kA,MN) d(ac) d(il)"},
                  {"1/2", "t1c(AB,kM) v(AB,cM) d(ad) d(il)"},
                  {"1/2", "t1c(AB,lM) v(AB,dM) d(ac) d(ik)"},
                  {"-1/2", "t1c(cA,MN) v(kA,MN) d(ad) d(il)"},
                  {"-1/2", "t1c(dA,MN) v(lA,MN) d(ac) d(ik)"},
                  {"-1/2", "t1c(AB,kM) v(AB,dM) d(ac) d(il)"},
                  {"-1/2", "t1c(AB,lM) v(AB,cM) d(ad) d(ik)"}};
// doubles-doubles, first order <Phi_ijab| V_N |Phi_klcd>
const Rows kDD1 = {{"1", "v(ab,cd) d(ik) d(jl)"}, {"1", "v(kl,ij) d(ac) d(bd)"},
                   {"-1", "v(ab,cd) d(il) d(jk)"}, {"-1", "v(kl,ij) d(ad) d(bc)"},
                   {"1", "v(ak,cj) d(bd) d(il)"},  {"1", "v(ak,di) d(bc) d(jl)"},
                   {"1", "v(al,ci) d(bd) d(jk)"},  {"1", "v(al,dj) d(bc) d(ik)"},
                   {"1", "v(bk,ci) d(ad) d(jl)"},  {"1", "v(bk,dj) d(ac) d(il)"},
                   {"1", "v(bl,cj) d(ad) d(ik)"},  {"1", "v(bl,di) d(ac) d(jk)"},
                   {"-1", "v(ak,ci) d(bd) d(jl)"}, {"-1", "v(ak,dj) d(bc) d(il)"},
                   {"-1", "v(al,cj) d(bd) d(ik)"}, {"-1", "v(al,di) d(bc) d(jk)"},
                   {"-1", "v(bk,cj) d(ad) d(il)"}, {"-1", "v(bk,di) d(ac) d(jl)"},
                   {"-1", "v(bl,ci) d(ad) d(jk)"}, {"-1", "v(bl,dj) d(ac) d(ik)"}};

// numerators of the second-order amplitudes (second_order_amplitudes in
// setup.cu), as tables for the adjoint:
//   t2_ij^ab D_ij^ab = 1/2 <ab||CD> t_ij^CD + 1/2 <MN||ij> t_MN^ab + P(ij)P(ab) <Mb||Cj> t_iM^aC
//   t2_i^a (eps_i - eps_a) = 1/2 <aM||CD> t_iM^CD - 1/2 <MN||iC> t_MN^aC
const Rows kT2N = {{"1/2", "v(ab,CD) t1(CD,ij)"},   {"1/2", "v(MN,ij) t1(ab,MN)"},
                   {"1", "v(Mb,Cj) t1(aC,iM)"},     {"-1", "v(Mb,Ci) t1(aC,jM)"},
                   {"-1", "v(Ma,Cj) t1(bC,iM)"},    {"1", "v(Ma,Ci) t1(bC,jM)"}};
const Rows kS2N = {{"1/2", "v(aM,CD) t1(CD,iM)"}, {"-1/2", "v(MN,iC) t1(aC,MN)"}};

// M[ia][jb] += s ((eps_b - eps_j) - (eps_a - eps_i)) / 2 * S[ia][jb]
__global__ void k_wmul_add(cplx *M, const cplx *S, const double *eo, const double *ev, int64_t o, int64_t v,
                           double s) {
  const int64_t n1 = o * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n1 * n1;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = idx % n1, row = idx / n1;
    const int64_t i = row / v, a = row % v, j = col / v, b = col % v;
    const double w = s * 0.5 * ((ev[b] - eo[j]) - (ev[a] - eo[i]));
    M[idx].x += w * S[idx].x;
    M[idx].y += w * S[idx].y;
  }
}

// dst[z][k][l][c][d] = src[z][k][l][c][d] * (eps_c + eps_d - eps_k - eps_l)
__global__ void k_dk_mul(const cplx *src, const double *eo, const double *ev, int64_t k, int64_t o, int64_t v,
                         cplx *dst) {
  const int64_t total = k * o * o * v * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t d = idx % v, r = idx / v;
    int64_t c = r % v; r /= v;
    int64_t l = r % o; r /= o;
    int64_t kk = r % o;
    const double f = ev[c] + ev[d] - eo[kk] - eo[l];
    dst[idx] = cmake(src[idx].x * f, src[idx].y * f);
  }
}

__global__ void k_ee_diag(const cplx *MSS, const double *g, const double *eo, const double *ev, int64_t o,
                          int64_t v, double xd, double *diag, double *d2) {
  const int64_t nmo = o + v, n1 = o * v, po = o * (o - 1) / 2, pv = v * (v - 1) / 2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n1 + po * pv;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (idx < n1) { diag[idx] = MSS[idx * n1 + idx].x; continue; }
    const int64_t r = idx - n1;
    const int64_t pij = r / pv, pab = r % pv;
    int64_t i = 0;
    while ((i + 1) * o - (i + 1) * (i + 2) / 2 <= pij) ++i;
    const int64_t j = pij - (i * o - i * (i + 1) / 2) + i + 1;
    int64_t a = 0;
    while ((a + 1) * v - (a + 1) * (a + 2) / 2 <= pab) ++a;
    const int64_t b = pab - (a * v - a * (a + 1) / 2) + a + 1;
    const double z = ev[a] + ev[b] - eo[i] - eo[j];
    const int64_t A = o + a, Bv = o + b;
    const double f = g[A * nmo + Bv] + g[i * nmo + j] - g[A * nmo + i] - g[A * nmo + j] - g[Bv * nmo + i] -
                     g[Bv * nmo + j];
    d2[r] = z;
    diag[idx] = z + xd * f;
  }
}

}  // namespace


void amplitude_tables(std::vector<Term> &t2n, std::vector<Term> &s2n) {
  t2n = parse_terms(kT2N);
  s2n = parse_terms(kS2N);
}

TermSource ee_source(adc_ctx *c) {
  TermSource s;
  s.o = c->o;
  s.v = c->v;
  s.get = [c](const std::string &name, const std::string &lab) -> TV {
    const int64_t o = c->o, v = c->v;
    auto type = [](char ch) { return std::string("ijklMNOPRSTW").find(ch) != std::string::npos ? 'o' : 'v'; };
    if (name == "v") {
      std::string spec;
      for (char ch : lab) spec.push_back(type(ch));
      auto &m = c->ee->eri;
      if (!m.count(spec)) m[spec] = eri_block(c, spec.c_str());
      std::vector<int64_t> e;
      for (char ch : spec) e.push_back(ch == 'o' ? o : v);
      return TV::dense(m[spec].c(), e);
    }
    if (name == "t1" || name == "t1c" || name == "t2" || name == "t2c") {
      cplx *p = (name[1] == '1') ? c->t1.c() : c->ee->t2d.c();
      // stored [i][j][a][b]; labels are (a, b, i, j)
      TV t(p, {v, v, o, o}, {v, 1, o * v * v, v * v});
      t.conj = (name.back() == 'c');
      return t;
    }
    if (name == "s2" || name == "s2c") {
      TV t(c->ee->t2s.c(), {v, o}, {1, v});
      t.conj = (name == "s2c");
      return t;
    }
    throw Error(ADC_ERR_ARG, "EE terms: unknown tensor " + name);
  };
  return s;
}

bool ee_vvvv_chunked(adc_ctx *c) {
  if (c->opts.ee_vvvv == 1) return true;
  if (c->opts.ee_vvvv == -1) return false;
  const double v = (double)c->v;
  return v * v * v * v * (double)sizeof(cplx) > 32.0 * (double)(1ll << 30);
}

namespace {
// M[i][a][i][b] += s G[a][b] for every i (M is [o][v][o][v])
__global__ void k_add_ij_diag(cplx *M, const cplx *__restrict__ G, int64_t o, int64_t v, double s) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < o * v * v;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / (v * v), r = idx - i * v * v, a = r / v, b = r - a * v;
    cplx &m = M[((i * v + a) * o + i) * v + b];
    m = cmake(m.x + s * G[r].x, m.y + s * G[r].y);
  }
}

// M[i][a0 + a][j][b] += s T[i][j][a][b], a < na
__global__ void k_add_chunk(const cplx *__restrict__ T, int64_t o, int64_t na, int64_t v, int64_t a0, double s,
                            cplx *M) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < o * o * na * v;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = idx % v;
    int64_t r = idx / v;
    const int64_t a = r % na;
    r /= na;
    const int64_t j = r % o, i = r / o;
    cplx &m = M[((i * v + a0 + a) * o + j) * v + b];
    m = cmake(m.x + s * T[idx].x, m.y + s * T[idx].y);
  }
}
}  // namespace

// The rows of kY3V times x, added to the singles block M [o][v][o][v], without
// the dense <ab||cd> (t: first-order doubles, Lad_ij^ab = 1/2 sum_cd <ab||cd>
// t_ij^cd, <pq||rs>* = <rs||pq>, <pq||rs> = sum_Q (B_pr B_qs - B_ps B_qr)):
//   1/2 t(aA,iM) t*(BC,jM) <BC||bA>        = sum_AM t_iM^aA conj(Lad_jM^bA)
//   -1/4 t(aA,MN) t*(BC,MN) <BC||bA> d_ij  = -1/2 d_ij sum_AMN t_MN^aA conj(Lad_MN^bA)
//   1/2 t(AB,MN) t*(AC,MN) <aC||bB> d_ij   = 1/2 d_ij sum_BC P_BC <aC||bB>,
//        P_BC = sum_AMN t_MN^AB conj(t_MN^AC), contracted through B
//   1/2 t(aA,MN) t*(bB,MN) <jB||iA>        = 1/2 sum_AB D[a][A][b][B] <jB||iA>
//   -t(AB,iM) t*(AC,jM) <aC||bB>           = -sum_BC R[i][j][B][C] <aC||bB>,
//        R = sum_AM t_iM^AB conj(t_jM^AC)
// The last two run over chunks of a: D[a][A][b][B] = sum_MN t_MN^aA conj(t_MN^bB)
// and <aC||bB> (assembled from B) exist for one chunk at a time.
void y3_vvvv_chunked(adc_ctx *c, const DBuf &Lad, double x, cplx *Mp) {
  Exec &ex = c->ex;
  const int64_t o = c->o, v = c->v, Q = c->Q;
  TagScope tg(ex, "ee_y3_chunked");
  ADC_REQUIRE(Lad.p != nullptr, ADC_ERR_STATE, "EE setup: ladder intermediate missing");
  const TV t = TV::dense(c->t1.c(), {o, o, v, v}), tc = t.cj();
  const TV Ladc = TV::dense(Lad.c(), {o, o, v, v}).cj();
  const TV M = TV::dense(Mp, {o, v, o, v});
  einsum(ex, CR(x), t, "iMaA", Ladc, "jMbA", C1(), M, "iajb");
  // the d_ij rows as one [v][v] matrix
  {
    DBuf G = cbuf(ex, v * v), P = cbuf(ex, v * v), pQ = cbuf(ex, Q), H = cbuf(ex, Q * v * v);
    const TV Gv = TV::dense(G.c(), {v, v}), Pv = TV::dense(P.c(), {v, v}), pv = TV::dense(pQ.c(), {Q}),
             Hv = TV::dense(H.c(), {Q, v, v});
    const TV Bvv = Bview(c, 'v', 'v');
    einsum(ex, CR(-0.5), t, "MNaA", Ladc, "MNbA", C0(), Gv, "ab");
    einsum(ex, C1(), t, "MNAB", tc, "MNAC", C0(), Pv, "BC");
    einsum(ex, C1(), Pv, "BC", Bvv, "QCB", C0(), pv, "Q");
    einsum(ex, CR(0.5), pv, "Q", Bvv, "Qab", C1(), Gv, "ab");
    einsum(ex, C1(), Bvv, "QaB", Pv, "BC", C0(), Hv, "QaC");
    einsum(ex, CR(-0.5), Hv, "QaC", Bvv, "QCb", C1(), Gv, "ab");
    k_add_ij_diag<<<grid1d(o * v * v, 256), 256, 0, ex.stream>>>(Mp, G.c(), o, v, x);
    ADC_CHECK_LAUNCH();
  }
  // R[i][j][B][C], W[i][j][A][B] = <jB||iA>, Bt[Q][B][C] = B^Q_CB
  DBuf R = cbuf(ex, o * o * v * v), W = cbuf(ex, o * o * v * v), Bt = cbuf(ex, Q * v * v);
  einsum(ex, C1(), t, "iMAB", tc, "jMAC", C0(), TV::dense(R.c(), {o, o, v, v}), "ijBC");
  {
    DBuf ovov = eri_block(c, "ovov");  // [j][B][i][A]
    permute(ex, ovov.c(), {o, o, v, v}, {v, v * o * v, 1, o * v}, false, W.c(), C1(), C0());
  }
  {
    const TV Bvv = Bview(c, 'v', 'v');
    permute(ex, Bvv.p, {Q, v, v}, {Bvv.str[0], 1, Bvv.str[1]}, false, Bt.c(), C1(), C0());
  }
  const TV Rv = TV::dense(R.c(), {o, o, v, v}), Wv = TV::dense(W.c(), {o, o, v, v});
  // chunk of a: each of the four chunk buffers within about 2 GiB, and at
  // least four chunks (ceil(v/4) wide) so that every size runs the chunk loop
  const int64_t per_a = v * v * v * (int64_t)sizeof(cplx);
  const int64_t na = std::max<int64_t>(
      1, std::min<int64_t>((v + 3) / 4, (2ll << 30) / std::max<int64_t>(per_a, 1)));
  DBuf D = cbuf(ex, na * v * v * v), Vc = cbuf(ex, na * v * v * v), T = cbuf(ex, o * o * na * v);
  for (int64_t a0 = 0; a0 < v; a0 += na) {
    const int64_t n = std::min(na, v - a0);
    const TV Dv = TV::dense(D.c(), {n, v, v, v}), Vv = TV::dense(Vc.c(), {v, v, n, v}),
             Tv = TV::dense(T.c(), {o, o, n, v});
    // D[a][A][b][B] = sum_MN t_MN^aA conj(t_MN^bB), a in the chunk
    const TV ta(c->t1.c() + a0 * v, {o, o, n, v}, {o * v * v, v * v, v, 1});
    einsum(ex, C1(), ta, "MNaA", tc, "MNbB", C0(), Dv, "aAbB");
    // Vc[B][C][a][b] = <aC||bB> = sum_Q (B_ab B_CB - B_aB B_Cb), a in the chunk
    const TV Bvv = Bview(c, 'v', 'v');
    const TV Ba(Bvv.p + a0 * Bvv.str[1], {Q, n, v}, Bvv.str);
    const TV BtCB(Bt.c(), {Q, v, v}, {v * v, 1, v});  // labels Q, C, B
    einsum(ex, C1(), Ba, "Qab", BtCB, "QCB", C0(), Vv, "BCab");
    einsum(ex, CR(-1.0), Ba, "QaB", Bvv, "QCb", C1(), Vv, "BCab");
    // T[i][j][a][b] = 1/2 sum_AB W[i][j][A][B] D[a][A][b][B] - sum_BC R[i][j][B][C] Vc[B][C][a][b]
    einsum(ex, CR(0.5), Wv, "ijAB", Dv, "aAbB", C0(), Tv, "ijab");
    einsum(ex, CR(-1.0), Rv, "ijBC", Vv, "BCab", C1(), Tv, "ijab");
    k_add_chunk<<<grid1d(o * o * n * v, 256), 256, 0, ex.stream>>>(T.c(), o, n, v, a0, x, Mp);
    ADC_CHECK_LAUNCH();
  }
}

void setup_ee(adc_ctx *c) {
  Exec &ex = c->ex;
  const int64_t o = c->o, v = c->v, n1 = c->n1;
  const bool third = (c->order == 3) && (c->x != 0.0);
  const double x = c->x;
  c->ee.reset(new EEOps());
  EEOps &E = *c->ee;
  E.K1 = parse_terms(kK1); E.S2 = parse_terms(kS2); E.Y2 = parse_terms(kY2);
  E.S3 = parse_terms(kS3);
  E.Y3L = parse_terms(kY3);
  E.Y3 = E.Y3L;
  {
    const std::vector<Term> y3v = parse_terms(kY3V);
    E.Y3.insert(E.Y3.end(), y3v.begin(), y3v.end());
  }
  E.SD1 = parse_terms(kSD1); E.O2 = parse_terms(kO2); E.Z1 = parse_terms(kZ1); E.DD1 = parse_terms(kDD1);
  amplitude_tables(E.T2N, E.S2N);
  StageScope stage(ex, "first_order_amplitudes");
  first_order_amplitudes(c);
  const bool chunked = ee_vvvv_chunked(c);
  DBuf Lad_keep;  // the ladder intermediate, for the chunked four-virtual terms
  if (c->order == 3) {
    // also at x = 0: the derivative with respect to x needs them
    DBuf G_vv, Lad;
    stage.next("second_order_amplitudes");
    second_order_amplitudes(c, G_vv, Lad, E.t2d, E.t2s);
    if (chunked && third) Lad_keep = std::move(Lad);
  }
  stage.next("singles_second_order");
  TermSource src = ee_source(c);
  const std::string L = "iajb";
  std::vector<int64_t> e4 = {o, v, o, v};
  E.MSS = cbuf(ex, n1 * n1);
  TV M = TV::dense(E.MSS.c(), e4);
  fill_zero(ex, E.MSS.p, E.MSS.bytes);
  DBuf K1 = cbuf(ex, n1 * n1), S2 = cbuf(ex, n1 * n1);
  fill_zero(ex, K1.p, K1.bytes);
  fill_zero(ex, S2.p, S2.bytes);
  eval_terms(ex, E.K1, src, {}, false, C1(), TV::dense(K1.c(), e4), L);
  eval_terms(ex, E.S2, src, {}, false, C1(), TV::dense(S2.c(), e4), L);
  // zeroth order on the diagonal
  E.dS = DBuf(ex, n1 * sizeof(double));
  {
    std::vector<double> eo(o), ev(v), d(n1);
    ADC_CUDA(cudaMemcpyAsync(eo.data(), c->eo.p, o * 8, cudaMemcpyDeviceToHost, ex.stream));
    ADC_CUDA(cudaMemcpyAsync(ev.data(), c->ev.p, v * 8, cudaMemcpyDeviceToHost, ex.stream));
    ADC_CUDA(cudaStreamSynchronize(ex.stream));
    for (int64_t i = 0; i < o; ++i)
      for (int64_t a = 0; a < v; ++a) d[i * v + a] = ev[a] - eo[i];
    ADC_CUDA(cudaMemcpyAsync(E.dS.p, d.data(), n1 * 8, cudaMemcpyHostToDevice, ex.stream));
    ADC_CUDA(cudaStreamSynchronize(ex.stream));
  }
  add_diag(ex, E.MSS.c(), E.dS.d(), n1, 1.0);
  zaxpby(ex, n1 * n1, C1(), K1.c(), C1(), E.MSS.c());
  k_wmul_add<<<grid1d(n1 * n1, 256), 256, 0, ex.stream>>>(E.MSS.c(), S2.c(), c->eo.d(), c->ev.d(), o, v, 1.0);
  ADC_CHECK_LAUNCH();
  eval_terms(ex, E.Y2, src, {}, false, C1(), M, L);
  if (third) {
    stage.next("singles_third_order");
    DBuf S3 = cbuf(ex, n1 * n1);
    fill_zero(ex, S3.p, S3.bytes);
    eval_terms(ex, E.S3, src, {}, false, C1(), TV::dense(S3.c(), e4), L);
    k_wmul_add<<<grid1d(n1 * n1, 256), 256, 0, ex.stream>>>(E.MSS.c(), S3.c(), c->eo.d(), c->ev.d(), o, v, x);
    ADC_CHECK_LAUNCH();
    if (chunked) {
      eval_terms(ex, E.Y3L, src, {}, false, CR(x), M, L);
      y3_vvvv_chunked(c, Lad_keep, x, E.MSS.c());
      Lad_keep.reset();
    } else {
      eval_terms(ex, E.Y3, src, {}, false, CR(x), M, L);
    }
    // - x/2 (S2 K1 + K1 S2)
    zgemm(ex, n1, n1, n1, 1, CR(-0.5 * x), S2.c(), 0, n1, 1, false, K1.c(), 0, n1, 1, false, C1(), E.MSS.c(), 0,
          n1, 1);
    zgemm(ex, n1, n1, n1, 1, CR(-0.5 * x), K1.c(), 0, n1, 1, false, S2.c(), 0, n1, 1, false, C1(), E.MSS.c(), 0,
          n1, 1);
  }
  // a copy as the generic main block
  stage.next("diagonal");
  c->M11 = cbuf(ex, n1 * n1);
  ADC_CUDA(cudaMemcpyAsync(c->M11.p, E.MSS.p, n1 * n1 * sizeof(cplx), cudaMemcpyDeviceToDevice, ex.stream));
  // diagonal
  c->diag = DBuf(ex, c->N * sizeof(double));
  c->d2 = DBuf(ex, c->n2 * sizeof(double));
  {
    DBuf g(ex, c->nmo * c->nmo * sizeof(double));
    antisym_diag(ex, c->B.c(), c->Q, c->nmo, g.d());
    const double xd = (third && c->dd_order == 1) ? x : 0.0;
    k_ee_diag<<<grid1d(c->N, 256), 256, 0, ex.stream>>>(E.MSS.c(), g.d(), c->eo.d(), c->ev.d(), o, v, xd,
                                                        c->diag.d(), c->d2.d());
    ADC_CHECK_LAUNCH();
  }
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
  // at sizes where the four-virtual terms are chunked, the dense integral
  // blocks of the tables are dropped (they are rebuilt on demand)
  if (chunked) E.eri.clear();
}

void ee_struct_build(adc_ctx *c, bool dd);
void ee_struct_apply(adc_ctx *c, const cplx *X, cplx *S, int64_t kc, double sdd);

void sigma_ee_fp64(adc_ctx *c, const cplx *X, cplx *S, int64_t k) {
  Exec &ex = c->ex;
  EEOps &E = *c->ee;
  const int64_t o = c->o, v = c->v, n1 = c->n1, n2 = c->n2, N = c->N;
  const int64_t po = npairs(o), pv = npairs(v);
  const bool third = (c->order == 3) && (c->x != 0.0);
  const double x = third ? c->x : 0.0;
  const double sdd = (third && c->dd_order == 1) ? x : 0.0;
  ee_struct_build(c, sdd != 0.0);
  TagScope tg(ex, "ee");
  // singles <- singles: static block; doubles: zeroth order
  zgemm(ex, k, n1, n1, 1, C1(), X, 0, N, 1, false, E.MSS.c(), 0, 1, n1, false, C0(), S, 0, N, 1);
  ADC_CUDA(cudaMemset2DAsync(S + n1, N * sizeof(cplx), 0, n2 * sizeof(cplx), k, ex.stream));
  diag_mul_add(ex, k, n2, c->d2.d(), X + n1, N, S + n1, N, 1.0);
  // chunks of vectors whose scratch stays within about 4 GiB
  int64_t per = std::max<int64_t>(o * o * pv, po * v * v);
  if (sdd != 0.0) per = std::max<int64_t>(per, 2 * o * v * o * v);
  per *= (int64_t)sizeof(cplx);
  const int64_t kc = std::max<int64_t>(1, std::min<int64_t>(k, (4ll << 30) / std::max<int64_t>(per, 1)));
  for (int64_t z0 = 0; z0 < k; z0 += kc) {
    const int64_t kk = std::min(kc, k - z0);
    ee_struct_apply(c, X + z0 * N, S + z0 * N, kk, sdd);
  }
}

}  // namespace adc
