// Matrix-free sigma product S = M X in FP64 with the cached operators.
//
// EA, X = [X_a | X_j,(a<b)]:
//   S1 = M11 X1 + Cpl X2
//   S2 = Cpl^H X1 + d2 * X2
//        + x [ sum_{c<d} <ab||cd> X_j,cd  -  P(ab) sum_kc <ak||cj> X_k,cb ]
// IP, X = [X_i | X_(i<j),a]:
//   S1 = M11 X1 + Cpl X2
//   S2 = Cpl^H X1 + d2 * X2
//        + x [ sum_{k<l} <kl||ij> X_(kl),a  +  P(ij) sum_kb <ak||bj> X_k,i,b ]
// (Sec. 2.1 Eqs. 10-12; integrals from Eq. 43.) The satellite terms of
// first order are the ladder (packed GEMM) and the ring (GEMM over (k,c)).
#include "ctx.cuh"

namespace adc {

namespace {
// dst rows (pitch ldd) += alpha * src rows (pitch lds), k rows of length n
__global__ void k_rows_axpy(int64_t k, int64_t n, cplx alpha, const cplx *src, int64_t lds, cplx *dst,
                            int64_t ldd) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < k * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / n, i = idx % n;
    dst[r * ldd + i] = cadd(dst[r * ldd + i], cmul(alpha, src[r * lds + i]));
  }
}
}  // namespace

cplx *scratch(adc_ctx *c, int64_t ncplx) {
  size_t need = (size_t)ncplx * sizeof(cplx);
  if (c->scratch.bytes < need) {
    c->scratch.reset();
    c->scratch = DBuf(c->ex, need);
  }
  return c->scratch.c();
}

void sigma_fp64(adc_ctx *c, const cplx *X, cplx *S, int64_t k) {
  Exec &ex = c->ex;
  const int64_t o = c->o, v = c->v, n1 = c->n1, n2 = c->n2, N = c->N;
  const bool sat = (c->order == 3 && c->x != 0.0);
  const double x = sat ? c->x : 0.0;
  // S1 = X1 M11^T  (S1[r][p] = sum_q M11[p][q] X1[r][q])
  TagScope tg(ex, "main");
  zgemm(ex, k, n1, n1, 1, C1(), X, 0, N, 1, false, c->M11.c(), 0, 1, n1, false, C0(), S, 0, N, 1);
  // S1 += X2 Cpl^T
  ex.tag = "coupling";
  zgemm(ex, k, n1, n2, 1, C1(), X + n1, 0, N, 1, false, c->Cpl.c(), 0, 1, n2, false, C1(), S, 0, N, 1);
  // S2 = X1 conj(Cpl)
  zgemm(ex, k, n2, n1, 1, C1(), X, 0, N, 1, false, c->Cpl.c(), 0, n2, 1, true, C0(), S + n1, 0, N, 1);
  // S2 += d2 * X2
  diag_mul_add(ex, k, n2, c->d2.d(), X + n1, N, S + n1, N, 1.0);
  if (!sat) return;
  if (c->kind == ADC_EA) {
    const int64_t pv = npairs(v);
    // ladder: S2[r][j][(ab)] += x sum_(cd) X2[r][j][(cd)] Glad[(ab)][(cd)], one GEMM over all (r, j)
    ex.tag = "ladder";
    cplx *Xf = scratch(c, 2 * k * o * v * v + 2 * k * o * pv);
    cplx *T = Xf + k * o * v * v;
    cplx *Xg = T + k * o * v * v, *Og = Xg + k * o * pv;
    if (c->direct_ladder) {
      ladder_direct(c, X + n1, N, o, S + n1, N, k, x, ADC_LADDER_FP64, nullptr);
    } else {
      ADC_CUDA(cudaMemcpy2DAsync(Xg, o * pv * sizeof(cplx), X + n1, N * sizeof(cplx), o * pv * sizeof(cplx), k,
                                 cudaMemcpyDeviceToDevice, ex.stream));
      zgemm(ex, k * o, pv, pv, 1, C1(), Xg, 0, pv, 1, false, c->Glad.c(), 0, 1, pv, false, C0(), Og, 0, pv, 1);
      k_rows_axpy<<<grid1d(k * o * pv, 256), 256, 0, ex.stream>>>(k, o * pv, CR(x), Og, o * pv, S + n1, N);
      ADC_CHECK_LAUNCH();
    }
    // ring: Xf[r][k][c][b] (antisymmetric in c,b); T[(j,a)][(r,b)] = sum_(kc) W[(j,a)][(kc)] Xt[(kc)][(r,b)]
    ex.tag = "ring";
    pair_unpack(ex, X + n1, k, o, N, pv, v, 1, Xf);
    // Xt[(kc)][r][b] = Xf[r][(kc)][b]
    permute(ex, Xf, {o * v, k, v}, {v, o * v * v, 1}, false, T, C1(), C0());
    zgemm(ex, o * v, k * v, o * v, 1, C1(), c->W.c(), 0, o * v, 1, false, T, 0, k * v, 1, false, C0(), Xf, 0, k * v,
          1);
    // Xf now holds R[(j,a)][r][b]; S2[r][j][(a<b)] -= x (R[j,a][r][b] - R[j,b][r][a])
    pair_pack(ex, Xf, v, v * k * v, k * v, 1, 0, 1.0, k, o, v, 1, S + n1, N, pv, CR(-x), C1());
  } else {
    const int64_t po = npairs(o);
    // ladder: S2[r][(ij)][a] += x sum_(kl) Glad[(ij)][(kl)] X2[r][(kl)][a]
    ex.tag = "ladder";
    zgemm(ex, po, v, po, k, CR(x), c->Glad.c(), 0, po, 1, false, X + n1, N, v, 1, false, C1(),
          S + n1, N, v, 1);
    // ring: Xf[r][i][k][b]; T[r][(j,a)][i] = -sum_(kb) W[(j,a)][(kb)] Xf[r][i][(kb)]
    ex.tag = "ring";
    cplx *Xf = scratch(c, 2 * k * o * o * v);
    cplx *T = Xf + k * o * o * v;
    pair_unpack(ex, X + n1, k, 1, N, 0, o, v, Xf);
    zgemm(ex, o * v, o, o * v, k, CR(-1.0), c->W.c(), 0, o * v, 1, false, Xf, o * o * v, 1, o * v,
          false, C0(), T, o * v * o, o, 1);
    // S2[r][(i<j)][a] += x (T[r][j][a][i] - T[r][i][a][j]); view T'(p=i, q=j, in=a) = T[q][in][p]
    pair_pack(ex, T, o * v * o, 0, 1, v * o, o, 1.0, k, 1, o, v, S + n1, N, 0, CR(x), C1());
  }
}

// One rank's share of the FP64 EA sigma when the satellite space is split by
// its occupied index j into [i0, i1) (nb = i1 - i0). X is the whole [k][N]
// block (every rank holds it after an all-gather); S is [k][n1 + nb Pv]:
//   S[:, :n1]  the partial main rows X2[j in share] Cpl[:, j in share]^T
//              (plus X1 M11^T when with_main): summed over the ranks they give S1;
//   S[:, n1:]  the satellite rows of the share, complete: coupling
//              conj(Cpl[:, j in share])^T X1, zeroth-order diagonal, the ladder
//              (diagonal in j: only the share's own X2 rows) and the ring (all of
//              X2, through the all-gathered block).
// The same terms and kernels as sigma_fp64 (Sec. 2.1 Eqs. 10-12), restricted.
void sigma_fp64_share(adc_ctx *c, const cplx *X, cplx *S, int64_t k, int64_t i0, int64_t i1, bool with_main) {
  Exec &ex = c->ex;
  ADC_REQUIRE(c->kind == ADC_EA, ADC_ERR_UNSUPPORTED, "sigma share: EA only");
  ADC_REQUIRE(0 <= i0 && i0 <= i1 && i1 <= c->o, ADC_ERR_ARG, "sigma share: occupied range");
  const int64_t o = c->o, v = c->v, n1 = c->n1, N = c->N;
  const int64_t pv = npairs(v), nb = i1 - i0, ns = nb * pv, ldS = n1 + ns;
  const bool sat = (c->order == 3 && c->x != 0.0);
  const double x = sat ? c->x : 0.0;
  TagScope tg(ex, "main");
  if (with_main)
    zgemm(ex, k, n1, n1, 1, C1(), X, 0, N, 1, false, c->M11.c(), 0, 1, n1, false, C0(), S, 0, ldS, 1);
  ex.tag = "coupling";
  if (ns > 0)
    zgemm(ex, k, n1, ns, 1, C1(), X + n1 + i0 * pv, 0, N, 1, false, c->Cpl.c() + i0 * pv, 0, 1, c->n2, false,
          with_main ? C1() : C0(), S, 0, ldS, 1);
  else if (!with_main)
    for (int64_t r = 0; r < k; ++r) ADC_CUDA(cudaMemsetAsync(S + r * ldS, 0, n1 * sizeof(cplx), ex.stream));
  if (ns == 0) return;
  zgemm(ex, k, ns, n1, 1, C1(), X, 0, N, 1, false, c->Cpl.c() + i0 * pv, 0, c->n2, 1, true, C0(), S + n1, 0, ldS,
        1);
  diag_mul_add(ex, k, ns, c->d2.d() + i0 * pv, X + n1 + i0 * pv, N, S + n1, ldS, 1.0);
  if (!sat) return;
  // ladder on the share's rows: Og[r][j][(ab)] = sum_(cd) X2[r][j][(cd)] Glad[(ab)][(cd)]
  ex.tag = "ladder";
  cplx *Xf = scratch(c, 2 * k * o * v * v + 2 * k * ns);
  cplx *T = Xf + k * o * v * v;
  cplx *Xg = T + k * o * v * v, *Og = Xg + k * ns;
  if (c->direct_ladder) {
    ladder_direct(c, X + n1 + i0 * pv, N, nb, S + n1, ldS, k, x, ADC_LADDER_FP64, nullptr);
  } else {
    ADC_CUDA(cudaMemcpy2DAsync(Xg, ns * sizeof(cplx), X + n1 + i0 * pv, N * sizeof(cplx), ns * sizeof(cplx), k,
                               cudaMemcpyDeviceToDevice, ex.stream));
    zgemm(ex, k * nb, pv, pv, 1, C1(), Xg, 0, pv, 1, false, c->Glad.c(), 0, 1, pv, false, C0(), Og, 0, pv, 1);
    k_rows_axpy<<<grid1d(k * ns, 256), 256, 0, ex.stream>>>(k, ns, CR(x), Og, ns, S + n1, ldS);
    ADC_CHECK_LAUNCH();
  }
  // ring rows (j, a) of the share: R[(j,a)][r][b] = sum_(kc) W[(j,a)][(kc)] Xt[(kc)][r][b], all k
  ex.tag = "ring";
  pair_unpack(ex, X + n1, k, o, N, pv, v, 1, Xf);
  permute(ex, Xf, {o * v, k, v}, {v, o * v * v, 1}, false, T, C1(), C0());
  zgemm(ex, nb * v, k * v, o * v, 1, C1(), c->W.c() + i0 * v * (o * v), 0, o * v, 1, false, T, 0, k * v, 1, false,
        C0(), Xf, 0, k * v, 1);
  pair_pack(ex, Xf, v, v * k * v, k * v, 1, 0, 1.0, k, nb, v, 1, S + n1, ldS, pv, CR(-x), C1());
}

double sigma_scratch_bytes(const adc_ctx *c, int64_t k) {
  const double cs = (double)sizeof(cplx);
  const double o = (double)c->o, v = (double)c->v, po = (double)npairs(c->o), pv = (double)npairs(c->v);
  if (c->kind == ADC_EE) {
    // one vector of the structured product: the gathered doubles of both
    // coupling GEMMs, their BF16 planes and the sliced digit planes of one of them
    double b = 8.0 * cs * std::max(o * o * pv, po * v * v);
    if (c->order == 3 && c->x != 0.0 && c->dd_order == 1) b += 3.0 * cs * (o * v) * (o * v);
    return b;
  }
  // IP/EA: the ring block, the packed B operands (BF16 planes or digit slices) of the block
  const double ring = (c->kind == ADC_EA) ? (double)k * o * v * v : (double)k * o * v * o;
  return cs * (2.0 * ring + 8.0 * (double)k * (double)c->N);
}

void sigma(adc_ctx *c, const cplx *X, cplx *S, int64_t k, int precision) {
  if (k <= 0) return;
  if (precision != ADC_PREC_FP64 && precision != ADC_PREC_BF16X3 && precision != ADC_PREC_BF16X6 &&
      precision != ADC_PREC_SLICED && precision != ADC_PREC_SLICED24)
    throw Error(ADC_ERR_ARG, "unknown precision");
  const int nseg = (precision == ADC_PREC_BF16X6) ? 6 : 3;
  if (precision == ADC_PREC_SLICED || precision == ADC_PREC_SLICED24) {
    const int bits = (precision == ADC_PREC_SLICED) ? kSlicedBits : kSliced24Bits;
    if (c->kind == ADC_EE) sigma_ee_split(c, X, S, k, 0, bits);  // nseg 0: sliced products
    else sigma_sliced(c, X, S, k, bits);
  } else if (c->kind == ADC_EE) {
    if (precision == ADC_PREC_FP64) sigma_ee_fp64(c, X, S, k);
    else sigma_ee_split(c, X, S, k, nseg);
  } else if (precision == ADC_PREC_FP64) {
    sigma_fp64(c, X, S, k);
  } else {
    sigma_split(c, X, S, k, nseg);
  }
}

}  // namespace adc
