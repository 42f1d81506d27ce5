// EE-ADC operators held by a context (built by setup_ee in ee.cu).
#pragma once

#include <map>

#include "ctx.cuh"
#include "terms.cuh"

namespace adc {
struct EEOps {
  std::vector<Term> K1, S2, Y2, S3, Y3, SD1, O2, Z1, DD1;
  std::vector<Term> T2N, S2N;  // numerators of the second-order doubles and singles (adjoint only)
  DBuf t2d, t2s;
  std::map<std::string, DBuf> eri;  // dense integral blocks by o/v spec
  DBuf MSS;                         // [n1][n1] static singles block
  DBuf dS;                          // [n1] eps_a - eps_i
};
// tensors of the EE term tables (v blocks cached in EEOps::eri)
TermSource ee_source(adc_ctx *c);
}  // namespace adc
