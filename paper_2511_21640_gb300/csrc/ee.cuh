// EE-ADC operators held by a context (built by setup_ee in ee.cu).
#pragma once

#include <map>

#include "ctx.cuh"
#include "tc_slice.cuh"
#include "terms.cuh"

namespace adc {
// operators of the structured EE sigma that run as tensor-core products
enum { EE_VAT = 0, EE_VAC, EE_VB, EE_VBC, EE_GVV, EE_GOO, EE_W, EE_NOPS };

struct EEOps {
  std::vector<Term> K1, S2, Y2, S3, Y3, SD1, O2, Z1, DD1;
  std::vector<Term> Y3L;            // Y3 without its four-virtual rows (chunked evaluation)
  std::vector<Term> T2N, S2N;  // numerators of the second-order doubles and singles (adjoint only)
  DBuf t2d, t2s;
  std::map<std::string, DBuf> eri;  // dense integral blocks by o/v spec
  DBuf MSS;                         // [n1][n1] static singles block
  DBuf dS;                          // [n1] eps_a - eps_i
  // packed operands of the structured sigma (ee_struct.cu)
  DBuf pair_o, pair_v;              // pair tables (p, q) of the occupied and virtual pairs
  DBuf Va, Vb, Goo, Gvv;            // <al||cd> [(l,cd)][a], <kl||di> [i][(kl,d)], <kl||ij>, <ab||cd> packed
                                    // (Va, Vb with the folded second-order coupling at third order)
  DBuf T1p, T2p, V1, V2;            // conj(t_lM^cd) [(l,cd)][M], conj(t_kl^dA) [(kl,d)][A],
                                    // <ak||iM> [(i,a)][(k,M)], <aA||ci> [(i,a)][(c,A)]
  // split-precision copies for the tensor-core sigma (A operands) and the per-call B operand
  TcMat tVaT, tVaC, tVb, tVbC, tGvv, tGoo, tW, bx;
  // the second-order amplitude operands of the separable pieces: T1p^T, conj(T1p), T2p^T, conj(T2p)
  TcMat tT1T, tT1C, tT2T, tT2C;
  DBuf tcerr;
  bool tc_ready = false;
  int tc_planes = 0;
  // sliced copies (FP64-accurate products), indexed by EE_VAT .. EE_W, and the per-call B operand
  SlMat sop[EE_NOPS];
  SlMat sbx;
  SlWork slw;
  bool sl_ready = false, sl_dd = false;
};
// numerators of the second-order doubles and singles (second_order_amplitudes in
// setup.cu) as term tables: t2_ij^ab D_ij^ab and t2_i^a (eps_i - eps_a)
void amplitude_tables(std::vector<Term> &t2n, std::vector<Term> &s2n);
// tensors of the EE term tables (v blocks cached in EEOps::eri)
TermSource ee_source(adc_ctx *c);
}  // namespace adc
