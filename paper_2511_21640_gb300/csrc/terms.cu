// Evaluation of EE-ADC term tables with the device contraction engine.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "terms.cuh"

namespace adc {

namespace {

bool is_occ_label(char c) { return std::strchr("ijklMNOPRSTW", c) != nullptr; }

double parse_coef(const char *s) {
  // "p", "-p", "p/q", "-p/q"
  double num = std::atof(s);
  const char *slash = std::strchr(s, '/');
  if (slash) num /= std::atof(slash + 1);
  return num;
}

// merge repeated labels of an operand into one axis (a diagonal view)
void merge_duplicates(TV &t, std::string &lab) {
  for (size_t p = 0; p < lab.size(); ++p) {
    for (size_t q = p + 1; q < lab.size();) {
      if (lab[q] == lab[p]) {
        ADC_REQUIRE(t.ext[p] == t.ext[q], ADC_ERR_ARG, "terms: diagonal of unequal extents");
        t.str[p] += t.str[q];
        t.ext.erase(t.ext.begin() + q);
        t.str.erase(t.str.begin() + q);
        lab.erase(lab.begin() + q);
      } else {
        ++q;
      }
    }
  }
}

constexpr int SA_MAXD = 10;
struct SAArgs {
  int nd;
  int64_t ext[SA_MAXD], sstr[SA_MAXD], dstr[SA_MAXD];
};

__global__ void k_strided_add(const cplx *__restrict__ src, SAArgs a, cplx alpha, cplx *dst, int64_t total) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = idx, so = 0, dof = 0;
    for (int d = a.nd - 1; d >= 0; --d) {
      int64_t i = rem % a.ext[d];
      rem /= a.ext[d];
      so += i * a.sstr[d];
      dof += i * a.dstr[d];
    }
    dst[dof] = cadd(dst[dof], cmul(alpha, src[so]));
  }
}

// dst (strided view, extents ext) += alpha * src (strided, stride 0 broadcasts)
void strided_add(Exec &ex, const cplx *src, const std::vector<int64_t> &sstr, const TV &dst, cplx alpha) {
  SAArgs a;
  a.nd = (int)dst.ext.size();
  ADC_REQUIRE(a.nd <= SA_MAXD, ADC_ERR_UNSUPPORTED, "terms: rank");
  int64_t total = 1;
  for (int d = 0; d < a.nd; ++d) {
    a.ext[d] = dst.ext[d];
    a.sstr[d] = sstr[d];
    a.dstr[d] = dst.str[d];
    total *= dst.ext[d];
  }
  if (!total) return;
  k_strided_add<<<grid1d(total, 256), 256, 0, ex.stream>>>(src, a, alpha, dst.p, total);
  ADC_CHECK_LAUNCH();
}

struct Operand {
  TV t;
  std::string lab;
};

constexpr int RD_MAXD = 10;
struct RDArgs {
  int nk, ns;                                    // kept and summed axes
  int64_t kext[RD_MAXD], kstr[RD_MAXD];
  int64_t sext[RD_MAXD], sstr[RD_MAXD];
  int64_t nsum;
};

// out[kept] = sum over the summed axes of (conj) src
__global__ void k_reduce_axes(const cplx *__restrict__ src, RDArgs a, int conj, cplx *out, int64_t total) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = idx, base = 0;
    for (int d = a.nk - 1; d >= 0; --d) {
      base += (rem % a.kext[d]) * a.kstr[d];
      rem /= a.kext[d];
    }
    cplx s = cmake(0.0, 0.0);
    for (int64_t t = 0; t < a.nsum; ++t) {
      int64_t r2 = t, off = 0;
      for (int d = a.ns - 1; d >= 0; --d) {
        off += (r2 % a.sext[d]) * a.sstr[d];
        r2 /= a.sext[d];
      }
      s = cadd(s, src[base + off]);
    }
    out[idx] = conj ? cmake(s.x, -s.y) : s;
  }
}

// sums out the labels of op that no other operand and not the output carry
// (a contraction of one tensor with itself along an index it alone holds)
void reduce_private_labels(Exec &ex, std::vector<Operand> &ops, const std::string &out_labels,
                           std::vector<DBuf> &keep_alive) {
  for (size_t i = 0; i < ops.size(); ++i) {
    std::string kept, summed;
    for (char ch : ops[i].lab) {
      bool elsewhere = out_labels.find(ch) != std::string::npos;
      for (size_t j = 0; j < ops.size() && !elsewhere; ++j)
        if (j != i && ops[j].lab.find(ch) != std::string::npos) elsewhere = true;
      (elsewhere ? kept : summed).push_back(ch);
    }
    if (summed.empty()) continue;
    ADC_REQUIRE(!kept.empty() || ops.size() == 1, ADC_ERR_UNSUPPORTED, "terms: operand reduces to a scalar");
    RDArgs a{};
    a.nk = (int)kept.size();
    a.ns = (int)summed.size();
    ADC_REQUIRE(a.nk <= RD_MAXD && a.ns <= RD_MAXD, ADC_ERR_UNSUPPORTED, "terms: rank");
    std::vector<int64_t> kext;
    int64_t total = 1;
    a.nsum = 1;
    int nk = 0, ns = 0;
    for (size_t d = 0; d < ops[i].lab.size(); ++d) {
      const char ch = ops[i].lab[d];
      if (kept.find(ch) != std::string::npos) {
        a.kext[nk] = ops[i].t.ext[d];
        a.kstr[nk] = ops[i].t.str[d];
        kext.push_back(ops[i].t.ext[d]);
        total *= ops[i].t.ext[d];
        ++nk;
      } else {
        a.sext[ns] = ops[i].t.ext[d];
        a.sstr[ns] = ops[i].t.str[d];
        a.nsum *= ops[i].t.ext[d];
        ++ns;
      }
    }
    keep_alive.push_back(cbuf(ex, std::max<int64_t>(total, 1)));
    cplx *dst = keep_alive.back().c();
    k_reduce_axes<<<grid1d(total, 256), 256, 0, ex.stream>>>(ops[i].t.p, a, ops[i].t.conj ? 1 : 0, dst, total);
    ADC_CHECK_LAUNCH();
    ops[i].t = TV::dense(dst, kext);
    ops[i].lab = kept;
  }
}

double prod_ext(const std::string &labs, const std::map<char, int64_t> &ext) {
  double p = 1.0;
  for (char c : labs) p *= (double)ext.at(c);
  return p;
}

std::string label_union(const std::string &a, const std::string &b) {
  std::string u = a;
  for (char c : b)
    if (u.find(c) == std::string::npos) u.push_back(c);
  return u;
}

// labels of (P, Q) still needed by `rest` or by the output
std::string kept(const std::string &pq, const std::string &rest, const std::string &out) {
  std::string k;
  for (char c : pq)
    if (rest.find(c) != std::string::npos || out.find(c) != std::string::npos) k.push_back(c);
  return k;
}

}  // namespace

int64_t TermSource::extent(char c) const { return is_occ_label(c) ? o : v; }

std::vector<Term> parse_terms(const std::vector<std::pair<const char *, const char *>> &rows) {
  std::vector<Term> out;
  for (auto &r : rows) {
    Term t;
    t.coef = parse_coef(r.first);
    std::string s(r.second);
    size_t pos = 0;
    while (pos < s.size()) {
      while (pos < s.size() && s[pos] == ' ') ++pos;
      if (pos >= s.size()) break;
      size_t lp = s.find('(', pos), rp = s.find(')', pos);
      ADC_REQUIRE(lp != std::string::npos && rp != std::string::npos, ADC_ERR_ARG, "terms: parse " + s);
      Factor f;
      f.name = s.substr(pos, lp - pos);
      for (size_t q = lp + 1; q < rp; ++q)
        if (s[q] != ',') f.labels.push_back(s[q]);
      t.f.push_back(f);
      pos = rp + 1;
    }
    out.push_back(t);
  }
  return out;
}

void eval_terms(Exec &ex, const std::vector<Term> &terms, const TermSource &src,
                const std::vector<std::pair<std::string, TV>> &extra, bool conj, cplx alpha, const TV &out,
                const std::string &out_labels) {
  for (const Term &term : terms) {
    std::vector<Operand> ops;
    std::vector<std::pair<char, char>> deltas;
    for (const Factor &f : term.f) {
      if (f.name == "d") {
        deltas.push_back({f.labels[0], f.labels[1]});
        continue;
      }
      Operand op{src.get(f.name, f.labels), f.labels};
      if (conj) op.t.conj = !op.t.conj;
      ops.push_back(op);
    }
    for (auto &e : extra) ops.push_back(Operand{e.second, e.first});
    // output view (diagonals for deltas between output labels)
    TV ov = out;
    std::string olab = out_labels;
    for (auto &d : deltas) {
      char x = d.first, y = d.second;
      bool xo = olab.find(x) != std::string::npos, yo = olab.find(y) != std::string::npos;
      if (xo && yo) {
        size_t px = olab.find(x), py = olab.find(y);
        ov.str[px] += ov.str[py];
        ov.ext.erase(ov.ext.begin() + py);
        ov.str.erase(ov.str.begin() + py);
        olab.erase(olab.begin() + py);
        for (auto &op : ops) std::replace(op.lab.begin(), op.lab.end(), y, x);
      } else {
        char from = xo ? y : x, to = xo ? x : y;
        for (auto &op : ops) std::replace(op.lab.begin(), op.lab.end(), from, to);
      }
    }
    for (auto &op : ops) merge_duplicates(op.t, op.lab);
    std::vector<DBuf> reduced;
    reduce_private_labels(ex, ops, olab, reduced);
    std::map<char, int64_t> ext;
    for (auto &op : ops)
      for (size_t i = 0; i < op.lab.size(); ++i) ext[op.lab[i]] = op.t.ext[i];
    for (size_t i = 0; i < olab.size(); ++i) ext[olab[i]] = ov.ext[i];
    const cplx coef = cmul(alpha, cmake(term.coef, 0.0));
    // output labels the product depends on (the others are broadcast)
    std::string all;
    for (auto &op : ops) all += op.lab;
    std::string full_olab = olab;
    olab.clear();
    std::vector<int64_t> rext;
    for (char c : full_olab)
      if (all.find(c) != std::string::npos) { olab.push_back(c); rext.push_back(ext[c]); }
    int64_t nout = 1;
    for (auto e : rext) nout *= e;
    DBuf res = cbuf(ex, nout);
    TV R = TV::dense(res.c(), rext);
    if (ops.size() == 1) {
      std::vector<int64_t> e, s;
      for (char c : olab) {
        size_t p = ops[0].lab.find(c);
        ADC_REQUIRE(p != std::string::npos && ops[0].lab.size() == olab.size(), ADC_ERR_UNSUPPORTED,
                    "terms: single operand must carry the output labels");
        e.push_back(ops[0].t.ext[p]);
        s.push_back(ops[0].t.str[p]);
      }
      permute(ex, ops[0].t.p, e, s, ops[0].t.conj, res.c(), C1(), C0());
    } else if (ops.size() == 2) {
      einsum(ex, C1(), ops[0].t, ops[0].lab.c_str(), ops[1].t, ops[1].lab.c_str(), C0(), R, olab.c_str());
    } else if (ops.size() == 3) {
      int best[3] = {0, 1, 2};
      double bestc = 1e300;
      const int pairs[3][3] = {{0, 1, 2}, {0, 2, 1}, {1, 2, 0}};
      for (auto &pp : pairs) {
        std::string u = label_union(ops[pp[0]].lab, ops[pp[1]].lab);
        std::string I = kept(u, ops[pp[2]].lab, olab);
        double c = prod_ext(u, ext) + prod_ext(label_union(I, ops[pp[2]].lab), ext);
        if (c < bestc) { bestc = c; best[0] = pp[0]; best[1] = pp[1]; best[2] = pp[2]; }
      }
      std::string u = label_union(ops[best[0]].lab, ops[best[1]].lab);
      std::string I = kept(u, ops[best[2]].lab, olab);
      std::vector<int64_t> ie;
      int64_t ni = 1;
      for (char c : I) { ie.push_back(ext[c]); ni *= ext[c]; }
      DBuf ib = cbuf(ex, ni);
      TV IT = TV::dense(ib.c(), ie);
      einsum(ex, C1(), ops[best[0]].t, ops[best[0]].lab.c_str(), ops[best[1]].t, ops[best[1]].lab.c_str(), C0(), IT,
             I.c_str());
      einsum(ex, C1(), IT, I.c_str(), ops[best[2]].t, ops[best[2]].lab.c_str(), C0(), R, olab.c_str());
    } else {
      throw Error(ADC_ERR_UNSUPPORTED, "terms: more than three operands");
    }
    std::vector<int64_t> sstr(full_olab.size(), 0);
    for (size_t q = 0; q < full_olab.size(); ++q) {
      size_t p = olab.find(full_olab[q]);
      if (p != std::string::npos) sstr[q] = R.str[p];
    }
    strided_add(ex, res.c(), sstr, ov, coef);
  }
}

void eval_terms_grad(Exec &ex, const std::vector<Term> &terms, const TermSource &src, const TermSource &grad,
                     const std::vector<std::pair<std::string, TV>> &extra, bool conj, cplx alpha) {
  for (const Term &term : terms) {
    for (size_t j = 0; j < term.f.size(); ++j) {
      const Factor &f = term.f[j];
      if (f.name == "d") continue;
      TV G = grad.get(f.name, f.labels);
      if (!G.p) continue;  // no gradient wanted for this tensor
      const bool appears_conj = (G.conj != conj);
      G.conj = false;
      Term rest;
      rest.coef = term.coef;
      for (size_t i = 0; i < term.f.size(); ++i)
        if (i != j) rest.f.push_back(term.f[i]);
      const std::vector<Term> one{rest};
      if (appears_conj) {
        // the factor enters as conj(T): G_T += dC/d conj(T)
        eval_terms(ex, one, src, extra, conj, alpha, G, f.labels);
      } else {
        // the factor enters as T: G_T += conj(dC/dT), i.e. every operand conjugated
        std::vector<std::pair<std::string, TV>> ex2 = extra;
        for (auto &e : ex2) e.second.conj = !e.second.conj;
        eval_terms(ex, one, src, ex2, !conj, cmake(alpha.x, -alpha.y), G, f.labels);
      }
    }
  }
}

}  // namespace adc
