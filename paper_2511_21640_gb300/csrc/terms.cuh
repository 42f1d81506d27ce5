// Term tables of the EE-ADC blocks and their evaluation on the device.
//
// A term is a rational coefficient times a product of tensors written with
// index labels, e.g. "t1(aA,iM) t1c(bA,NO) v(jM,NO)": lower-case labels are
// free (i j k l occupied, a b c d virtual), upper-case labels are summed
// (M N O P R S T W occupied, A..H virtual). Tensors: v(pq,rs) = <pq||rs>
// (Eq. 43), t1(ab,ij) = t_ij^ab, t1c its conjugate, t2/t2c the second-order
// doubles, s2(a,i) = t2_i^a, s2c, d(xy) a Kronecker delta.
#pragma once

#include <functional>
#include <map>
#include <string>
#include <vector>

#include "tensor.cuh"

namespace adc {

struct Factor {
  std::string name, labels;
};

struct Term {
  double coef = 1.0;
  std::vector<Factor> f;
};

std::vector<Term> parse_terms(const std::vector<std::pair<const char *, const char *>> &rows);

// Provides the device tensors of a term table (views in label order).
struct TermSource {
  int64_t o = 0, v = 0;
  std::function<TV(const std::string &name, const std::string &labels)> get;
  int64_t extent(char c) const;  // o for occupied labels, v for virtual ones
};

// out[out_labels] += alpha * sum over rows of coef * product * (extra operands)
// (conj: complex conjugate of the table's product). Deltas between two output
// labels are written on the corresponding diagonal of out; deltas between an
// output label and an extra operand's label are substituted into the operand.
// Each product of two or three operands is contracted pairwise in the cheaper
// order with the contraction engine.
void eval_terms(Exec &ex, const std::vector<Term> &terms, const TermSource &src,
                const std::vector<std::pair<std::string, TV>> &extra, bool conj, cplx alpha,
                const TV &out, const std::string &out_labels);

// Adjoint of eval_terms for a real target f = Re C, where C is what
// eval_terms would sum over every label (the extras carry the output side,
// e.g. a density or the conjugated left vectors). For every factor whose
// tensor has a gradient buffer (grad.get returns a view in the same label
// convention as src, with conj set for the conjugated names, or a null view),
// G_T += dC/d conj(T) where the factor enters as conj(T) and conj(dC/dT)
// where it enters as T: the gradient in the convention d/dRe + i d/dIm. Each
// derivative is the same contraction with the factor left out and its labels
// as the output.
void eval_terms_grad(Exec &ex, const std::vector<Term> &terms, const TermSource &src, const TermSource &grad,
                     const std::vector<std::pair<std::string, TV>> &extra, bool conj, cplx alpha);

}  // namespace adc
