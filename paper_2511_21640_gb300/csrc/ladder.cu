// Integral-direct ladder of the EA satellite block (Sec. 2.1; Sec. 2.5, Eq. 43
// and the paragraph after it: the four-external integrals are formed on the
// fly, never stored). For a trial block X the term
//   S2[r][j][(a<b)] += x sum_(c<d) <ab||cd> X2[r][j][(c<d)]
// is evaluated one chunk of rows (a<b), a in [a0, a1), at a time:
//   J[(a,c)][(b,d)] = sum_Q B^Q_ac B^Q_bd   (b >= a0: a GEMM over the Cholesky index)
//   G[(ab)][(cd)]   = J[(a,c)][(b,d)] - J[(a,d)][(b,c)]
//   S2[.][.][(ab)] += x G X2[.][.]^T       (a GEMM over the packed pairs)
// so that device memory holds one chunk instead of the Pv x Pv block. Both
// GEMMs run in the product's precision: FP64 CUDA cores, the BF16 split on the
// tensor cores (the Cholesky operand packed once per context), or the sliced
// FP64-accurate product (48 bits for the integrals, 40 for the contraction).
#include <algorithm>

#include "ctx.cuh"
#include "tc_gemm.cuh"

namespace adc {

void ladder_direct(adc_ctx *c, const cplx *X2, int64_t ldX, int64_t nj, cplx *S2, int64_t ldS, int64_t k,
                   double x, int mode, int *err) {
  ADC_REQUIRE(c->kind == ADC_EA && c->direct_ladder, ADC_ERR_ARG, "ladder_direct: EA context without stored ladder");
  if (k <= 0 || nj <= 0) return;
  Exec &ex = c->ex;
  const int64_t v = c->v, Q = c->Q, pv = npairs(v);
  if (pv == 0) return;
  TagScope tg(ex, "ladder_direct");
  if (!c->Lvv.p) c->Lvv = vvvv_L(c);
  const int64_t ca = vvvv_chunk(c);
  DBuf J = cbuf(ex, ca * v * v * v), Gc = cbuf(ex, std::min<int64_t>(ca * v, pv) * pv);
  if (mode == ADC_LADDER_FP64 || mode == ADC_LADDER_SLICED) {
    const int saved = ex.sliced_bits;
    try {
      for (int64_t a0 = 0; a0 < v - 1; a0 += ca) {
        const int64_t a1 = std::min(v - 1, a0 + ca), r0 = ladder_row0(a0, v), r1 = ladder_row0(a1, v);
        ex.sliced_bits = (mode == ADC_LADDER_SLICED) ? 48 : 0;
        vvvv_rows(c, c->Lvv.c(), a0, a1, J.c(), Gc.c());
        ex.sliced_bits = (mode == ADC_LADDER_SLICED) ? 40 : 0;
        // S2[r][j][(ab)] += x sum_(cd) Gc[(ab)][(cd)] X2[r][j][(cd)], batched over r
        zgemm(ex, r1 - r0, nj, pv, k, CR(x), Gc.c(), 0, pv, 1, false, X2, ldX, 1, pv, false, C1(), S2 + r0, ldS, 1,
              pv);
      }
    } catch (...) {
      ex.sliced_bits = saved;
      throw;
    }
    ex.sliced_bits = saved;
    return;
  }
  // BF16 split (nseg 3 or 6)
  const int nseg = mode;
  const int planes = (nseg == 6) ? 3 : 2;
  tc_ensure(c, planes);
  TcCache &tc = *c->tc;
  if (tc.LA.rows == 0 || tc.LA.planes < planes) {
    tc_pack_A(ex, tc.LA, c->Lvv.c(), v * v, Q, Q, 1, false, planes);
    tc_pack_B(ex, tc.LB, c->Lvv.c(), v * v, Q, Q, 0, 1, 1, false, planes);
  }
  tc_pack_B(ex, tc.Bx, X2, k * nj, pv, ldX, pv, nj, 1, false, planes);
  TcMat Gt;
  for (int64_t a0 = 0; a0 < v - 1; a0 += ca) {
    const int64_t a1 = std::min(v - 1, a0 + ca), r0 = ladder_row0(a0, v), r1 = ladder_row0(a1, v);
    const int64_t na = a1 - a0, nb = v - a0;
    tc_gemm(ex, tc_view(tc.LA, a0 * v, na * v), tc_view(tc.LB, 2 * a0 * v, 2 * nb * v), na * v, nb * v, C1(), C0(),
            J.c(), nb * v, 1, 0, 1, err, nseg);
    vvvv_assemble_rows(c, J.c(), a0, a1, Gc.c());
    tc_pack_A(ex, Gt, Gc.c(), r1 - r0, pv, pv, 1, false, planes);
    tc_gemm(ex, tc_view(Gt), tc_view(tc.Bx), r1 - r0, k * nj, CR(x), C1(), S2 + r0, 1, ldS, pv, nj, err, nseg);
  }
}

}  // namespace adc
