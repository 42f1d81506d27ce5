// FP64 complex tensor toolkit: strided permutes, batched GEMM, pair packing
// and a small contraction engine (permute + batched GEMM) for the one-time
// setup of the ADC operators.
#pragma once

#include "common.cuh"

namespace adc {

// Execution environment of one context: its stream and a byte budget for
// every device allocation the context makes.
struct ProfRec {
  std::string name;
  cudaEvent_t a = nullptr, b = nullptr;
  double flops = 0.0;  // algorithmic flops of the launch (8 per complex multiply-add)
  double bytes = 0.0;  // algorithmic device-memory bytes (operands read once, result written once)
};

struct Exec {
  cudaStream_t stream = nullptr;
  // > 0: zgemm runs large products (at least 2^24 flops, inner size at least
  // 512) as the sliced tensor-core product with about this many significant
  // bits (tc_slice.cu)
  int sliced_bits = 0;
  // complex GEMMs issued through zgemm since the counters were cleared: how
  // many took the sliced tensor-core route and how many the FP64 kernel, with
  // their algorithmic flops (host-side counts)
  int64_t n_sliced = 0, n_fp64 = 0;
  double flops_sliced = 0.0, flops_fp64 = 0.0;
  int64_t mem_limit = 0;  // 0 = unlimited
  int64_t mem_used = 0;
  int64_t mem_peak = 0;
  // per-kernel timing with CUDA events on this stream (off unless enabled)
  bool prof = false;
  std::string tag;
  std::string stage;  // step of a longer procedure in progress (StageScope), for error messages
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> event_pool;
  cudaEvent_t event();
  int prof_begin(const char *kernel, double flops, double bytes = 0.0);  // record index, -1 when off
  void prof_end(int r);
  void prof_clear();

  void *alloc(size_t bytes);           // cudaMallocAsync on the stream, counted
  void release(void *p, size_t bytes);  // cudaFreeAsync on the stream
};

// RAII device buffer counted against the context budget.
struct DBuf {
  Exec *ex = nullptr;
  void *p = nullptr;
  size_t bytes = 0;
  DBuf() {}
  DBuf(Exec &e, size_t b) : ex(&e), p(b ? e.alloc(b) : nullptr), bytes(b) {}
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  DBuf(DBuf &&o) noexcept : ex(o.ex), p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
  DBuf &operator=(DBuf &&o) noexcept {
    reset();
    ex = o.ex; p = o.p; bytes = o.bytes;
    o.p = nullptr; o.bytes = 0;
    return *this;
  }
  ~DBuf() { reset(); }
  void reset() {
    if (p && ex) ex->release(p, bytes);
    p = nullptr;
    bytes = 0;
  }
  cplx *c() const { return (cplx *)p; }
  double *d() const { return (double *)p; }
};

// device time of one step of a longer procedure ("stage:<name>" in the profile)
// (next() ends the current step and starts the following one)
struct StageScope {
  Exec &ex;
  int rec = -1;
  StageScope(Exec &e, const char *name) : ex(e) { begin(name); }
  ~StageScope() { end(); }
  void next(const char *name) {
    end();
    begin(name);
  }

 private:
  void begin(const char *name) {
    ex.stage = name;
    rec = ex.prof ? ex.prof_begin((std::string("stage:") + name).c_str(), 0.0) : -1;
  }
  void end() {
    if (rec >= 0 && rec < (int)ex.recs.size()) cudaEventRecord(ex.recs[rec].b, ex.stream);
    rec = -1;
    ex.stage.clear();
  }
};

// names the sigma term whose kernels are being launched (for the profile)
struct TagScope {
  Exec &ex;
  std::string old;
  TagScope(Exec &e, const char *t) : ex(e), old(e.tag) { ex.tag = t; }
  ~TagScope() { ex.tag = old; }
};

inline DBuf cbuf(Exec &e, int64_t n) { return DBuf(e, (size_t)n * sizeof(cplx)); }

// A strided view of a complex tensor; extents and strides in label order.
struct TV {
  cplx *p = nullptr;
  std::vector<int64_t> ext, str;
  bool conj = false;
  TV() {}
  TV(cplx *p_, std::vector<int64_t> e, std::vector<int64_t> s, bool c = false)
      : p(p_), ext(e), str(s), conj(c) {}
  // contiguous row-major view
  static TV dense(cplx *p_, std::vector<int64_t> e) {
    std::vector<int64_t> s(e.size());
    int64_t acc = 1;
    for (int i = (int)e.size() - 1; i >= 0; --i) { s[i] = acc; acc *= e[i]; }
    return TV(p_, e, s);
  }
  TV cj() const { TV t = *this; t.conj = !t.conj; return t; }
  int64_t size() const { int64_t n = 1; for (auto e : ext) n *= e; return n; }
};

// ---------------------------------------------------------------- kernels' host wrappers
// C[b] = alpha * opA(A[b]) opB(B[b]) + beta * C[b]; element strides.
void zgemm(Exec &ex, int64_t M, int64_t N, int64_t K, int64_t batch, cplx alpha,
           const cplx *A, int64_t sAb, int64_t sAm, int64_t sAk, bool conjA,
           const cplx *B, int64_t sBb, int64_t sBk, int64_t sBn, bool conjB, cplx beta,
           cplx *C, int64_t sCb, int64_t sCm, int64_t sCn);

// zgemm without any allocation: split-K partial sums go to ws (ws_elems complex
// elements; fewer splits when it is small, none when ws is NULL)
void zgemm_ws(Exec &ex, int64_t M, int64_t N, int64_t K, int64_t batch, cplx alpha,
              const cplx *A, int64_t sAb, int64_t sAm, int64_t sAk, bool conjA,
              const cplx *B, int64_t sBb, int64_t sBk, int64_t sBn, bool conjB, cplx beta,
              cplx *C, int64_t sCb, int64_t sCm, int64_t sCn, cplx *ws, int64_t ws_elems);

// dst (contiguous, extents ext) = alpha * op(src at strides sstr) + beta * dst
void permute(Exec &ex, const cplx *src, const std::vector<int64_t> &ext,
             const std::vector<int64_t> &sstr, bool conj, cplx *dst, cplx alpha, cplx beta);
// the same with dst at strides dstr
void permute(Exec &ex, const cplx *src, const std::vector<int64_t> &ext, const std::vector<int64_t> &sstr,
             bool conj, cplx *dst, const std::vector<int64_t> &dstr, cplx alpha, cplx beta);

// T[o][p][q][in] (contiguous) from packed P: P addr = o1*sP1 + o0*sP0 + pair*inner + in,
// o = o1*no0 + o0. Antisymmetric fill, zero diagonal.
void pair_unpack(Exec &ex, const cplx *P, int64_t no1, int64_t no0, int64_t sP1, int64_t sP0,
                 int64_t n, int64_t inner, cplx *T);

// P[o][pair(p<q)][in] = alpha*(T(o,p,q,in) - s*T(o,q,p,in)) + beta*P, T with general strides.
void pair_pack(Exec &ex, const cplx *T, int64_t sTo1, int64_t sTo0, int64_t sTp, int64_t sTq,
               int64_t sTin, double s, int64_t no1, int64_t no0, int64_t n, int64_t inner,
               cplx *P, int64_t sP1, int64_t sP0, cplx alpha, cplx beta);

// t[i][j][a][b] /= (eo_i + eo_j - ev_a - ev_b)
void denom2_div(Exec &ex, cplx *t, const double *eo, const double *ev, int64_t o, int64_t v);
// t[i][a] /= (eo_i - ev_a)
void denom1_div(Exec &ex, cplx *t, const double *eo, const double *ev, int64_t o, int64_t v);
// dst[i][j][a][b] = conj(D_ij^ab * t[i][j][a][b])  (= <ij||ab> from the amplitudes)
void oovv_from_t1(Exec &ex, const cplx *t, const double *eo, const double *ev, int64_t o,
                  int64_t v, cplx *dst);
// M[p][q] += s * (e_p - e_q) * G[q][p]   (the orthonormalisation term of the main block)
void add_eps_diff_transpose(Exec &ex, cplx *M, const cplx *G, const double *e, int64_t n, double s);
// M[p][p] += e[p] * s
void add_diag(Exec &ex, cplx *M, const double *e, int64_t n, double s);
// g[p][q] = Re sum_Q (B_pp B_qq - B_pq B_qp)
void antisym_diag(Exec &ex, const cplx *B, int64_t Q, int64_t nmo, double *g);
// y = a*x + b*y (complex, n elements)
void zaxpby(Exec &ex, int64_t n, cplx a, const cplx *x, cplx b, cplx *y);
// y[r][i] += d[i] * x[r][i] for r < k (strided rows)
void diag_mul_add(Exec &ex, int64_t k, int64_t n, const double *d, const cplx *x, int64_t ldx,
                  cplx *y, int64_t ldy, double s);
void fill_zero(Exec &ex, void *p, size_t bytes);
// number of SMs of the current device (looked up once per device)
int device_sm_count();
// raise a kernel's dynamic shared-memory limit on the current device, once per
// (kernel, device): the attribute belongs to the device, so a process that
// drives several GPUs sets it on each
void set_smem_limit(const void *kernel, int bytes);

// ---------------------------------------------------------------- contraction engine
// C[lc] = alpha * sum A[la] B[lb] + beta * C[lc] with Einstein labels (one char
// each). Indices in A and B but not C are summed; indices in all three are
// batched. Operands are permuted into GEMM order when their strides do not
// allow a direct batched GEMM.
void einsum(Exec &ex, cplx alpha, const TV &A, const char *la, const TV &B, const char *lb,
            cplx beta, const TV &C, const char *lc);

inline cplx C1() { return cmake(1.0, 0.0); }
inline cplx C0() { return cmake(0.0, 0.0); }
inline cplx CR(double r) { return cmake(r, 0.0); }

}  // namespace adc
