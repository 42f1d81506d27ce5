// Context of one ADC problem: sizes, device operators, caches.
#pragma once

#include <memory>

#include "tensor.cuh"

namespace adc {
struct TcCache;  // split-precision operator copies (tc_gemm.cu)
struct SlCache;  // sliced (FP64-accurate) operator copies (tc_slice.cu)
struct EEOps;    // EE-ADC operators (ee.cu)
struct BatchCoord;  // cross-problem sigma batching (batch.cu)
}

struct adc_ctx {
  adc::Exec ex;
  bool own_stream = false;
  int dev = -1;  // CUDA device that was current at adc_init (holds every buffer)
  // zgemm routes taken by adc_init: products (sliced, FP64) and their algorithmic flops
  int64_t setup_n[2] = {0, 0};
  double setup_flops[2] = {0.0, 0.0};
  int kind = 0, order = 2;
  double x = 0.0;   // the x of ADC(2)+x(3); 0 for order 2
  int64_t o = 0, v = 0, Q = 0, nmo = 0, n1 = 0, n2 = 0, N = 0;
  adc_opts opts;
  std::string err;

  // inputs on the device
  adc::DBuf B;    // [Q][nmo][nmo]
  adc::DBuf eo, ev;

  // operators of the sigma product (FP64)
  adc::DBuf M11;   // [n1][n1] static main block (all orders, x applied)
  adc::DBuf Cpl;   // [n1][n2] coupling block, first order + x * second order
  adc::DBuf d2;    // [n2] zeroth-order satellite diagonal (real)
  adc::DBuf diag;  // [N] exact diagonal of M (real)
  adc::DBuf Glad;  // ladder integrals, packed: EA [Pv][Pv] <ab||cd>; IP [Po][Po] <kl||ij>
  adc::DBuf W;     // ring integrals [o][v][o][v]: W[j][a][k][c] = <ak||cj>
  adc::DBuf t1;    // first-order doubles [o][o][v][v]
  // third order: the packed <ab||cd> is never stored; the setup's ladder
  // intermediate and, for EA, the satellite ladder of every product form it
  // chunk by chunk (integral-direct); IP keeps its <kl||ij> ladder in Glad
  bool direct_ladder = false;
  adc::DBuf Lvv;   // [(a,c)][Q] = B^Q_ac of the integral-direct ladder

  // split-precision copies for the tensor-core sigma
  std::unique_ptr<adc::TcCache> tc;
  // integer-digit slices for the FP64-accurate tensor-core sigma
  std::unique_ptr<adc::SlCache> sl;

  // EE-ADC operators (kind == ADC_EE)
  std::unique_ptr<adc::EEOps> ee;
  int dd_order = 1;

  // per-call scratch, grown on demand
  adc::DBuf scratch;

  // set while the context's Davidson runs inside a batch: its split-precision
  // sigma products are then gathered with the other problems' into one launch
  adc::BatchCoord *batch = nullptr;
  int batch_slot = -1;

  ~adc_ctx();
};

namespace adc {
TV Bview(adc_ctx *c, char p, char q);               // B^Q block view [Q][p][q]
DBuf eri_block(adc_ctx *c, const char *spec);       // dense <pq||rs> of a 4-letter o/v spec
DBuf build_vvvv_packed(adc_ctx *c);                 // [Pv][Pv] <ab||cd>, a<b, c<d
// integral-direct ladder pieces (setup.cu): L[(a,c)][Q] = B^Q_ac; the number of
// virtual indices a per chunk; rows (a<b) of the packed <ab||cd> for a in
// [a0, a1) into Gc [rows][Pv] from J = L L^T (J [(a,c)][(b,d)], b >= a0); the
// first packed row of a given a
DBuf vvvv_L(adc_ctx *c);
int64_t vvvv_chunk(adc_ctx *c);
void vvvv_rows(adc_ctx *c, const cplx *L, int64_t a0, int64_t a1, cplx *J, cplx *Gc);
void vvvv_assemble_rows(adc_ctx *c, const cplx *J, int64_t a0, int64_t a1, cplx *Gc);
inline int64_t ladder_row0(int64_t a, int64_t v) { return a * v - a * (a + 1) / 2; }
// the EA ladder term, integral-direct (ladder.cu): for r < k, j < nj,
// S2[r*ldS + j*Pv + (ab)] += x sum_(cd) <ab||cd> X2[r*ldX + j*Pv + (cd)], in the precision
// mode (ADC_LADDER_FP64, ADC_LADDER_SLICED, or 3 / 6 for the BF16 split; err: the
// tensor-core error word)
enum { ADC_LADDER_SLICED = 0, ADC_LADDER_FP64 = 1 };
void ladder_direct(adc_ctx *c, const cplx *X2, int64_t ldX, int64_t nj, cplx *S2, int64_t ldS, int64_t k,
                   double x, int mode, int *err);
void setup_operators(adc_ctx *c);
// t1 (c->t1) and ring integrals (c->W) from B
void first_order_amplitudes(adc_ctx *c);
// second-order doubles and singles, packed <ab||cd> and the ladder intermediate
// Lad_ij^ab = 1/2 sum_cd <ab||cd> t_ij^cd (needs c->t1 and c->W)
void second_order_amplitudes(adc_ctx *c, DBuf &G_vv, DBuf &Lad, DBuf &t2d, DBuf &t2s);
// the second-order singles t2_i^a alone (needs c->t1)
DBuf second_order_singles(adc_ctx *c);
void setup_ee(adc_ctx *c);
// EE: the four-virtual rows of the third-order singles block in chunks (opts.ee_vvvv, size)
bool ee_vvvv_chunked(adc_ctx *c);
// EE: build the product operands (structured, split-precision planes 0/2/3, sliced) ahead of a solve
void ee_prepare(adc_ctx *c, int planes, bool sliced);
// block Davidson for the lowest nroots roots (davidson.cu); with follow, one
// root: the Ritz vector with the largest overlap with the (single) guess at
// every iteration, instead of the lowest (root-specific solve)
int davidson_run(adc_ctx *c, int nroots, double tol, int max_iter, int precision, const cplx *guess,
                 int64_t nguess, double *omega, cplx *Yout, double *err64, adc_stats *st_out, bool follow = false);
// natural spinors (Eqs. 25-30): D^MP2 (+ Dadd, device v x v, Eq. 31), eta descending, V, U = V~ Z~
// ([v][v], leading dimension v), eps~; all outputs device pointers or null
void fns_run(adc_ctx *c, cplx *D, double *eta, cplx *Vout, double eta_crit, int64_t *n_keep, cplx *U,
             double *eps_new, const cplx *Dadd = nullptr);
// Cholesky vectors in the occupied + truncated-virtual basis (U [v][ldu], first nk columns)
void fns_transform(adc_ctx *c, const cplx *U, int64_t ldu, int64_t nk, cplx *Bout);
// state-specific natural spinors (ssfns.cu): state density (device y [N], D [v][v]),
// a vector in the truncated basis (g packed for o, nk), its length, the whole procedure
void state_density(adc_ctx *c, const cplx *y, cplx *D);
void to_fns_basis(adc_ctx *c, const cplx *y, const cplx *U, int64_t ldu, int64_t nk, cplx *g);
int64_t fns_dim(int kind, int64_t o, int64_t nk);
// EE ground-to-excited transition densities rho [k][nmo][nmo] of the vectors Y [k][N] (properties.cu)
void transition_density(adc_ctx *c, const cplx *Y, int64_t k, cplx *rho);
// pivoted Cholesky of the PSD V [n][n] (device) into L [max_rank][n] (device); pivots (host) or null;
// returns the rank (cholesky.cu)
int64_t cholesky_run(Exec &ex, const double *V, int64_t n, double tau, int64_t max_rank, double *L, int64_t *pivots);
// B[P] = C^H L^P C for real L [rank][nao][nao] and C [nao][nmo] (all device)
void cholesky_mo(Exec &ex, const double *L, int64_t rank, int64_t nao, const cplx *C, int64_t nmo, cplx *B);
// state densities rho [k][nmo][nmo] of any kind: ground state to second order + zeroth-order ISR
// difference (properties.cu); state_pair_density gives <Psi_K|a+_p a_q|Psi_L> for the pairs (YK[z], YL[z])
void excited_density(adc_ctx *c, const cplx *Y, int64_t k, cplx *rho);
void state_pair_density(adc_ctx *c, const cplx *YK, const cplx *YL, int64_t k, cplx *rho);
// IP/EA spectroscopic amplitudes x [k][nmo] of the vectors Y [k][N] (properties.cu)
void spectroscopic_amplitudes(adc_ctx *c, const cplx *Y, int64_t k, cplx *x);
int ssfns_run(const adc_c128 *B, int64_t naux, const double *eps_occ, int64_t nocc, const double *eps_vir,
              int64_t nvir, int kind, int order, double x, int nroots, double eta_crit, double tol, int max_iter,
              int precision, const adc_opts *opts, adc_ssfns_root *out);
void sigma_ee_fp64(adc_ctx *c, const cplx *X, cplx *S, int64_t k);
// chunk size (complex elements) of the setup's chunked intermediates; <= 0 restores the default
void set_setup_chunk_elems(int64_t n);
// significant bits of the sliced sigma products (ADC_PREC_SLICED, ADC_PREC_SLICED24)
constexpr int kSlicedBits = 40, kSliced24Bits = 24;
void sigma_ee_split(adc_ctx *c, const cplx *X, cplx *S, int64_t k, int nseg, int bits = kSlicedBits);
void sigma_fp64(adc_ctx *c, const cplx *X, cplx *S, int64_t k);
// one rank's share of the EA sigma with the satellites split by occupied index [i0, i1) (sigma.cu)
void sigma_fp64_share(adc_ctx *c, const cplx *X, cplx *S, int64_t k, int64_t i0, int64_t i1, bool with_main);
// split-precision sigma on the tensor cores: nseg = 3 (BF16x3) or 6 (BF16x6) products
void sigma_split(adc_ctx *c, const cplx *X, cplx *S, int64_t k, int nseg);
// FP64-accurate sigma with the dense contractions as sliced tensor-core products (IP/EA)
void sigma_sliced(adc_ctx *c, const cplx *X, cplx *S, int64_t k, int bits = kSlicedBits);
// estimate of the largest device scratch one sigma call of k vectors allocates (bytes)
double sigma_scratch_bytes(const adc_ctx *c, int64_t k);
void sigma(adc_ctx *c, const cplx *X, cplx *S, int64_t k, int precision);
void release_tc(adc_ctx *c);
void tc_ensure(adc_ctx *c, int planes = 2);  // split-precision operator copies, built on first use
cplx *scratch(adc_ctx *c, int64_t ncplx);
// inside a batch (c->batch set): S = M X (split precision) of this problem's
// block, executed together with the other problems' blocks; blocks until done
void batch_submit(adc_ctx *c, const cplx *X, cplx *S, int64_t k);
// the problem stops / resumes taking part in the batched products (FP64 work)
void batch_leave(adc_ctx *c);
void batch_rejoin(adc_ctx *c);
}  // namespace adc
