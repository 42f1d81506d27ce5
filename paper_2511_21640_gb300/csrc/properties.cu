// One-particle properties of ADC states from the intermediate-state
// representation (Sec. 2.2): EE transition densities, state and
// state-to-state densities of every kind, IP/EA spectroscopic amplitudes.
//
// EE transition densities rho_pq = <Psi_K| a+_p a_q |Psi0> = sum_I conj(Y_I) f_I(pq) with the ISR
// transition moments f_I(pq) = <Psi~_I| a+_p a_q |Psi0>, singles to second
// and doubles to first order (t / t2: first- / second-order doubles, s2:
// second-order singles, S2: second-order overlap of the orthogonalised
// singles precursors, Y the doubles as a full antisymmetric array):
//   rho_bj = conj(y_jb) + 1/2 sum_ia conj(y_ia) S2_{ia,jb}
//   rho_jb = sum_ia conj(y_ia) (t_ij^ab + t2_ij^ab)
//   rho_kl = -sum_a conj(y_la) s2_k^a - 1/2 sum_jab conj(Y_ljab) t_kj^ab
//   rho_ef = sum_i conj(y_ie) s2_i^f + 1/2 sum_ijb conj(Y_ijeb) t_ij^fb
// A transition moment of a one-particle operator d is sum_pq d_pq rho_pq.
//
// State and state-to-state densities rho^KL_pq = <Psi_K| a+_p a_q |Psi_L> of
// all three kinds at the level stated for ADC(2) states: the ground-state
// density through second order times y_K^H y_L plus the configurations
// weighted by the eigenvectors (zeroth-order intermediate states) for D - D0:
//   rho0_ij = d_ij - 1/2 sum_kab conj(t_jk^ab) t_ik^ab,  rho0_ab = 1/2 sum_ijc conj(t_ij^ac) t_ij^bc,
//   rho0_jb = s2_j^b,  rho0_bj = conj(s2_j^b);
// EE  kl: -sum_a conj(yK_la) yL_ka - 1/2 sum_jab conj(YK_ljab) YL_kjab
//     ef:  sum_i conj(yK_ie) yL_if + 1/2 sum_ijc conj(YK_ijec) YL_ijfc
//     jb:  sum_ia conj(yK_ia) YL_ijab,   bj: sum_ia conj(YK_ijab) yL_ia
// IP  kl: -conj(yK_l) yL_k - sum_ja conj(YK_lja) YL_kja,  ab: 1/2 sum_ij conj(YK_ija) YL_ijb
//     jb: -sum_i conj(yK_i) YL_ijb,      bj: -sum_i conj(YK_ijb) yL_i
// EA  kl: -1/2 sum_ab conj(YK_lab) YL_kab,  ab: conj(yK_a) yL_b + sum_jc conj(YK_jac) YL_jbc
//     jb:  sum_a conj(yK_a) YL_jab,      bj: sum_a conj(YK_jab) yL_a
//
// Spectroscopic amplitudes of IP/EA states, x_p = <Psi_n| a_p |Psi0> (IP) or
// <Psi_n| a+_p |Psi0> (EA) = sum_I conj(Y_I) f_I(p), main class through
// second and satellites through first order (Y the satellites as a full
// antisymmetric array, H the second-order hole / particle density pieces):
//   IP  x_k = conj(y_k) - 1/4 sum_i conj(y_i) H_ik,  H_ik = sum_jab t_ij^ab conj(t_kj^ab)
//       x_b = sum_i conj(y_i) s2_i^b + 1/2 sum_ija conj(Y_ija) t_ij^ab
//   EA  x_b = conj(y_b) - 1/4 sum_a conj(y_a) H_ab,  H_ab = sum_ijc t_ij^ac conj(t_ij^bc)
//       x_k = -sum_a conj(y_a) s2_k^a + 1/2 sum_jab conj(Y_jab) t_jk^ab
#include <vector>

#include "ctx.cuh"
#include "blockops.cuh"
#include "ee.cuh"

namespace adc {

namespace {
// dst[(r0 + r) * ld + c0 + c] = src[r * cols + c]
__global__ void k_put_block(const cplx *__restrict__ src, int64_t rows, int64_t cols, cplx *dst, int64_t ld,
                            int64_t r0, int64_t c0) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < rows * cols;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / cols, cc = idx - r * cols;
    dst[(r0 + r) * ld + c0 + cc] = src[idx];
  }
}

// dst[r * ld + c0 + c] = conj(src[r * lds + c]), r < rows, c < cols
__global__ void k_put_conj(const cplx *__restrict__ src, int64_t lds, int64_t rows, int64_t cols, cplx *dst,
                           int64_t ld, int64_t c0) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < rows * cols;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / cols, cc = idx - r * cols;
    const cplx a = src[r * lds + cc];
    dst[r * ld + c0 + cc] = cmake(a.x, -a.y);
  }
}
}  // namespace

void transition_density(adc_ctx *c, const cplx *Y, int64_t k, cplx *rho) {
  ADC_REQUIRE(c->kind == ADC_EE && c->ee, ADC_ERR_UNSUPPORTED, "transition densities: EE-ADC");
  Exec &ex = c->ex;
  EEOps &E = *c->ee;
  const int64_t o = c->o, v = c->v, n1 = c->n1, N = c->N, nmo = c->nmo;
  const int64_t po = npairs(o), pv = npairs(v);
  TagScope tg(ex, "properties");
  // second-order amplitudes (the setup keeps them at third order only)
  if (!E.t2d.p || !E.t2s.p) {
    DBuf Gvv, Lad;
    second_order_amplitudes(c, Gvv, Lad, E.t2d, E.t2s);
  }
  DBuf S2 = cbuf(ex, n1 * n1);
  fill_zero(ex, S2.p, S2.bytes);
  eval_terms(ex, E.S2, ee_source(c), {}, false, C1(), TV::dense(S2.c(), {o, v, o, v}), "iajb");
  DBuf tt = cbuf(ex, o * o * v * v);
  ADC_CUDA(cudaMemcpyAsync(tt.p, c->t1.p, tt.bytes, cudaMemcpyDeviceToDevice, ex.stream));
  zaxpby(ex, o * o * v * v, C1(), E.t2d.c(), C1(), tt.c());
  const TV t1 = TV::dense(c->t1.c(), {o, o, v, v}), T12 = TV::dense(tt.c(), {o, o, v, v});
  const TV s2 = TV::dense(E.t2s.c(), {o, v}), S2v = TV::dense(S2.c(), {o, v, o, v});
  DBuf Yf = cbuf(ex, o * o * v * v), half = cbuf(ex, std::max<int64_t>(po, 1) * v * v);
  DBuf Bvo = cbuf(ex, v * o), Bov = cbuf(ex, o * v), Boo = cbuf(ex, o * o), Bvv = cbuf(ex, v * v);
  for (int64_t z = 0; z < k; ++z) {
    const cplx *y = Y + z * N;
    cplx *R = rho + z * nmo * nmo;
    const TV y1c(const_cast<cplx *>(y), {o, v}, {v, 1}, true);
    if (po > 0 && pv > 0) {
      pair_unpack(ex, y + n1, 1, po, 0, pv, v, 1, half.c());
      pair_unpack(ex, half.c(), 1, 1, po * v * v, 0, o, v * v, Yf.c());
    } else {
      fill_zero(ex, Yf.p, Yf.bytes);
    }
    const TV Yc = TV::dense(Yf.c(), {o, o, v, v}).cj();
    // excitation block rho[o+b][j]
    permute(ex, y, {v, o}, {1, v}, true, Bvo.c(), C1(), C0());
    einsum(ex, CR(0.5), y1c, "ia", S2v, "iajb", C1(), TV::dense(Bvo.c(), {v, o}), "bj");
    // de-excitation block rho[j][o+b]
    einsum(ex, C1(), y1c, "ia", T12, "ijab", C0(), TV::dense(Bov.c(), {o, v}), "jb");
    // occupied block rho[k][l]
    einsum(ex, CR(-1.0), y1c, "la", s2, "ka", C0(), TV::dense(Boo.c(), {o, o}), "kl");
    einsum(ex, CR(-0.5), Yc, "ljab", t1, "kjab", C1(), TV::dense(Boo.c(), {o, o}), "kl");
    // virtual block rho[o+e][o+f]
    einsum(ex, C1(), y1c, "ie", s2, "if", C0(), TV::dense(Bvv.c(), {v, v}), "ef");
    einsum(ex, CR(0.5), Yc, "ijeb", t1, "ijfb", C1(), TV::dense(Bvv.c(), {v, v}), "ef");
    k_put_block<<<grid1d(v * o, 256), 256, 0, ex.stream>>>(Bvo.c(), v, o, R, nmo, o, 0);
    k_put_block<<<grid1d(o * v, 256), 256, 0, ex.stream>>>(Bov.c(), o, v, R, nmo, 0, o);
    k_put_block<<<grid1d(o * o, 256), 256, 0, ex.stream>>>(Boo.c(), o, o, R, nmo, 0, 0);
    k_put_block<<<grid1d(v * v, 256), 256, 0, ex.stream>>>(Bvv.c(), v, v, R, nmo, o, o);
    ADC_CHECK_LAUNCH();
  }
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
}

namespace {
// dst = s * src, s read on the device
__global__ void k_scaled_copy(const cplx *__restrict__ src, const cplx *__restrict__ s, int64_t n, cplx *dst) {
  const cplx a = *s;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const cplx x = src[idx];
    dst[idx] = cmake(a.x * x.x - a.y * x.y, a.x * x.y + a.y * x.x);
  }
}

// dst[(r0 + r) * ld + c0 + c] += src[r * cols + c]
__global__ void k_add_block(const cplx *__restrict__ src, int64_t rows, int64_t cols, cplx *dst, int64_t ld,
                            int64_t r0, int64_t c0) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < rows * cols;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / cols, cc = idx - r * cols;
    cplx &d = dst[(r0 + r) * ld + c0 + cc];
    d = cmake(d.x + src[idx].x, d.y + src[idx].y);
  }
}

__global__ void k_add_identity(cplx *R, int64_t n, int64_t ld) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    R[i * ld + i].x += 1.0;
}

// class-2 amplitudes of one vector as the full antisymmetric array: EE [o][o][v][v],
// IP [o][o][v], EA [o][v][v]; half is EE scratch of [max(Po,1)][v][v]
void unpack_class2(adc_ctx *c, const cplx *y, cplx *full, size_t full_bytes, cplx *half) {
  Exec &ex = c->ex;
  const int64_t o = c->o, v = c->v, n1 = c->n1, po = npairs(o), pv = npairs(v);
  if (c->n2 == 0) {
    fill_zero(ex, full, full_bytes);
  } else if (c->kind == ADC_EE) {
    pair_unpack(ex, y + n1, 1, po, 0, pv, v, 1, half);
    pair_unpack(ex, half, 1, 1, po * v * v, 0, o, v * v, full);
  } else if (c->kind == ADC_EA) {
    pair_unpack(ex, y + n1, 1, o, 0, pv, v, 1, full);
  } else {
    pair_unpack(ex, y + n1, 1, 1, 0, 0, o, v, full);
  }
}
}  // namespace

void state_pair_density(adc_ctx *c, const cplx *YK, const cplx *YL, int64_t k, cplx *rho) {
  Exec &ex = c->ex;
  const int kind = c->kind;
  const int64_t o = c->o, v = c->v, N = c->N, nmo = c->nmo;
  const int64_t po = npairs(o);
  TagScope tg(ex, "properties");
  // ground-state density through second order
  DBuf s2b = second_order_singles(c);
  const TV t1 = TV::dense(c->t1.c(), {o, o, v, v});
  DBuf R0 = cbuf(ex, nmo * nmo), s2t = cbuf(ex, v * o);
  cplx *r0 = R0.c();
  einsum(ex, CR(-0.5), t1.cj(), "jkab", t1, "ikab", C0(), TV(r0, {o, o}, {nmo, 1}), "ij");
  k_add_identity<<<grid1d(o, 256), 256, 0, ex.stream>>>(r0, o, nmo);
  einsum(ex, CR(0.5), t1.cj(), "ijac", t1, "ijbc", C0(), TV(r0 + o * nmo + o, {v, v}, {nmo, 1}), "ab");
  k_put_block<<<grid1d(o * v, 256), 256, 0, ex.stream>>>(s2b.c(), o, v, r0, nmo, 0, o);
  permute(ex, s2b.c(), {v, o}, {1, v}, true, s2t.c(), C1(), C0());
  k_put_block<<<grid1d(v * o, 256), 256, 0, ex.stream>>>(s2t.c(), v, o, r0, nmo, o, 0);
  ADC_CHECK_LAUNCH();
  // overlaps y_K^H y_L
  DBuf sd = cbuf(ex, k);
  for (int64_t z = 0; z < k; ++z) gram(ex, YK + z * N, N, 1, YL + z * N, N, 1, N, C1(), sd.c() + z, 1);
  // class-2 amplitudes as full arrays
  std::vector<int64_t> ef;
  if (kind == ADC_EE) ef = {o, o, v, v};
  else if (kind == ADC_IP) ef = {o, o, v};
  else ef = {o, v, v};
  int64_t nf = 1;
  for (int64_t e : ef) nf *= e;
  DBuf YKf = cbuf(ex, nf), YLf = cbuf(ex, nf);
  DBuf half = cbuf(ex, kind == ADC_EE ? std::max<int64_t>(po, 1) * v * v : 1);
  // the configuration blocks of one pair, dense
  DBuf Boo = cbuf(ex, o * o), Bvv = cbuf(ex, v * v), Bov = cbuf(ex, o * v), Bvo = cbuf(ex, v * o);
  const TV Roo = TV::dense(Boo.c(), {o, o}), Rvv = TV::dense(Bvv.c(), {v, v}), Rov = TV::dense(Bov.c(), {o, v}),
           Rvo = TV::dense(Bvo.c(), {v, o});
  for (int64_t z = 0; z < k; ++z) {
    const cplx *yk = YK + z * N, *yl = YL + z * N;
    cplx *R = rho + z * nmo * nmo;
    k_scaled_copy<<<grid1d(nmo * nmo, 256), 256, 0, ex.stream>>>(r0, sd.c() + z, nmo * nmo, R);
    ADC_CHECK_LAUNCH();
    unpack_class2(c, yk, YKf.c(), YKf.bytes, half.c());
    unpack_class2(c, yl, YLf.c(), YLf.bytes, half.c());
    const TV YKc = TV::dense(YKf.c(), ef).cj(), YLv = TV::dense(YLf.c(), ef);
    if (kind == ADC_EE) {
      const TV aKc(const_cast<cplx *>(yk), {o, v}, {v, 1}, true), aL(const_cast<cplx *>(yl), {o, v}, {v, 1});
      einsum(ex, CR(-1.0), aKc, "la", aL, "ka", C0(), Roo, "kl");
      einsum(ex, CR(-0.5), YKc, "ljab", YLv, "kjab", C1(), Roo, "kl");
      einsum(ex, C1(), aKc, "ie", aL, "if", C0(), Rvv, "ef");
      einsum(ex, CR(0.5), YKc, "ijec", YLv, "ijfc", C1(), Rvv, "ef");
      einsum(ex, C1(), aKc, "ia", YLv, "ijab", C0(), Rov, "jb");
      einsum(ex, C1(), YKc, "ijab", aL, "ia", C0(), Rvo, "bj");
    } else if (kind == ADC_IP) {
      const TV aKc(const_cast<cplx *>(yk), {o}, {1}, true), aL(const_cast<cplx *>(yl), {o}, {1});
      einsum(ex, CR(-1.0), aKc, "l", aL, "k", C0(), Roo, "kl");
      einsum(ex, CR(-1.0), YKc, "lja", YLv, "kja", C1(), Roo, "kl");
      einsum(ex, CR(0.5), YKc, "ija", YLv, "ijb", C0(), Rvv, "ab");
      einsum(ex, CR(-1.0), aKc, "i", YLv, "ijb", C0(), Rov, "jb");
      einsum(ex, CR(-1.0), YKc, "ijb", aL, "i", C0(), Rvo, "bj");
    } else {
      const TV aKc(const_cast<cplx *>(yk), {v}, {1}, true), aL(const_cast<cplx *>(yl), {v}, {1});
      einsum(ex, CR(-0.5), YKc, "lab", YLv, "kab", C0(), Roo, "kl");
      einsum(ex, C1(), aKc, "a", aL, "b", C0(), Rvv, "ab");
      einsum(ex, C1(), YKc, "jac", YLv, "jbc", C1(), Rvv, "ab");
      einsum(ex, C1(), aKc, "a", YLv, "jab", C0(), Rov, "jb");
      einsum(ex, C1(), YKc, "jab", aL, "a", C0(), Rvo, "bj");
    }
    k_add_block<<<grid1d(o * o, 256), 256, 0, ex.stream>>>(Boo.c(), o, o, R, nmo, 0, 0);
    k_add_block<<<grid1d(v * v, 256), 256, 0, ex.stream>>>(Bvv.c(), v, v, R, nmo, o, o);
    k_add_block<<<grid1d(o * v, 256), 256, 0, ex.stream>>>(Bov.c(), o, v, R, nmo, 0, o);
    k_add_block<<<grid1d(v * o, 256), 256, 0, ex.stream>>>(Bvo.c(), v, o, R, nmo, o, 0);
    ADC_CHECK_LAUNCH();
  }
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
}

void excited_density(adc_ctx *c, const cplx *Y, int64_t k, cplx *rho) { state_pair_density(c, Y, Y, k, rho); }

void spectroscopic_amplitudes(adc_ctx *c, const cplx *Y, int64_t k, cplx *x) {
  ADC_REQUIRE(c->kind == ADC_IP || c->kind == ADC_EA, ADC_ERR_UNSUPPORTED, "spectroscopic amplitudes: IP/EA-ADC");
  Exec &ex = c->ex;
  const bool ea = (c->kind == ADC_EA);
  const int64_t o = c->o, v = c->v, n1 = c->n1, n2 = c->n2, N = c->N, nmo = c->nmo;
  const int64_t pv = npairs(v);
  TagScope tg(ex, "properties");
  DBuf s2b = second_order_singles(c);
  const TV t1 = TV::dense(c->t1.c(), {o, o, v, v}), s2 = TV::dense(s2b.c(), {o, v});
  const TV y1c(const_cast<cplx *>(Y), {k, n1}, {N, 1}, true);
  const TV xo(x, {k, o}, {nmo, 1}), xv(x + o, {k, v}, {nmo, 1});
  const std::vector<int64_t> ef = ea ? std::vector<int64_t>{k, o, v, v} : std::vector<int64_t>{k, o, o, v};
  DBuf Y2f = cbuf(ex, ef[0] * ef[1] * ef[2] * ef[3]);
  if (n2 == 0) fill_zero(ex, Y2f.p, Y2f.bytes);
  else if (ea) pair_unpack(ex, Y + n1, k, o, N, pv, v, 1, Y2f.c());
  else pair_unpack(ex, Y + n1, k, 1, N, 0, o, v, Y2f.c());
  const TV Y2c = TV::dense(Y2f.c(), ef).cj();
  // the main orbitals: conj(y) at zeroth order
  k_put_conj<<<grid1d(k * n1, 256), 256, 0, ex.stream>>>(Y, N, k, n1, x, nmo, ea ? o : 0);
  ADC_CHECK_LAUNCH();
  if (!ea) {
    DBuf H = cbuf(ex, o * o);
    einsum(ex, C1(), t1, "ijab", t1.cj(), "kjab", C0(), TV::dense(H.c(), {o, o}), "ik");
    einsum(ex, CR(-0.25), y1c, "zi", TV::dense(H.c(), {o, o}), "ik", C1(), xo, "zk");
    einsum(ex, C1(), y1c, "zi", s2, "ib", C0(), xv, "zb");
    einsum(ex, CR(0.5), Y2c, "zija", t1, "ijab", C1(), xv, "zb");
  } else {
    DBuf H = cbuf(ex, v * v);
    einsum(ex, C1(), t1, "ijac", t1.cj(), "ijbc", C0(), TV::dense(H.c(), {v, v}), "ab");
    einsum(ex, CR(-0.25), y1c, "za", TV::dense(H.c(), {v, v}), "ab", C1(), xv, "zb");
    einsum(ex, CR(-1.0), y1c, "za", s2, "ka", C0(), xo, "zk");
    einsum(ex, CR(0.5), Y2c, "zjab", t1, "jkab", C1(), xo, "zk");
  }
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
}

}  // namespace adc
