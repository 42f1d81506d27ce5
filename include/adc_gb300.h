/*
 * adc_gb300.h -- C ABI of the GB300 relativistic CD-ADC sigma library.
 *
 * The library computes the matrix-free product S = M X of the ISR secular
 * matrix M of IP-ADC (1h + 2h1p), EA-ADC (1p + 2p1h) and EE-ADC (1h1p +
 * 2h2p) at second order, third order, or the scaled ADC(2)+x(3) mixture
 * (Sec. 2.1, Eqs. 10-12 of arXiv:2511.21640), solves M X = X Omega for the lowest roots by a block
 * Davidson method, and builds the MP2 virtual density and frozen natural
 * spinors (Sec. 2.4, Eqs. 25-30). Antisymmetrised integrals are assembled on
 * the device from Cholesky vectors, <pq||rs> = sum_Q (B_pr B_qs - B_ps B_qr)
 * (Sec. 2.5, Eq. 43).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Complex numbers are interleaved (re, im) doubles: adc_c128.
 * Spinors are numbered occupied first: 0..nocc-1 occupied, nocc..nmo-1 virtual,
 * nmo = nocc + nvir. The reference is canonical Hartree-Fock: the Fock matrix
 * is diag(eps_occ, eps_vir).
 * Pointer arguments may be host or device (CUDA unified addressing decides).
 * Host pointers make the call synchronous; device pointers make it
 * asynchronous on the context's stream, except where stated.
 * The library copies every input it keeps; the caller keeps ownership of all
 * buffers it passes. Every call returns ADC_OK (0) or a negative ADC_ERR_*
 * code; no call aborts, traps or exits the process. adc_strerror() names
 * the code and adc_last_error() gives the context's last message.
 *
 * Vector layout (dimension N = n1 + n2, basis-state phases of Eqs. 2-4):
 *   IP: [ X_i (n1 = nocc) | X_(i<j),a (n2 = nocc(nocc-1)/2 * nvir) ]
 *       state a+_a a_i a_j |Psi0>, a fastest, pairs row-major over i<j.
 *   EA: [ X_a (n1 = nvir) | X_j,(a<b) (n2 = nocc * nvir(nvir-1)/2) ]
 *       state a+_a a+_b a_j |Psi0>, pair fastest, pairs row-major over a<b.
 *   EE: [ X_(i,a) (n1 = nocc*nvir) | X_(i<j),(a<b) (n2 = npairs_o * npairs_v) ]
 *       states a+_a a_i |Psi0> and a+_a a_i a+_b a_j |Psi0>, a and the virtual
 *       pair fastest.
 * Blocks of k vectors are row-major [k][N].
 */
#ifndef ADC_GB300_H
#define ADC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double re, im;
} adc_c128;

typedef struct adc_ctx adc_ctx;

enum { ADC_IP = 0, ADC_EA = 1, ADC_EE = 2 };

/* Arithmetic of a sigma product.
 * ADC_PREC_FP64:   every operation in FP64 (CUDA cores).
 * ADC_PREC_BF16X3: the dense contractions on the tensor cores (tcgen05) with
 *   each FP64 operand split into two BF16 parts (hi + lo) and the three
 *   products hi*hi + hi*lo + lo*hi accumulated in FP32; complex arithmetic by
 *   the real 2x2 embedding. Diagonal terms stay FP64.
 * ADC_PREC_BF16X6: as BF16X3 with three BF16 parts (hi, lo = bf16(x - hi),
 *   lo2 = bf16(x - hi - lo)) and the six products of combined order up to
 *   2^-16 (hh, hl, lh, hl2, ll, l2h): about 2^-24 per operand at twice the
 *   tensor-core work of BF16X3. The tensor cores' FP32 accumulation, not the
 *   split, limits both (1e-6 to 1e-5 relative measured), so BF16X6 is rarely
 *   more accurate. Batches (adc_batch_*) use BF16X3.
 * ADC_PREC_SLICED: FP64-accurate products on the tensor cores.
 *   Each operand row is scaled by a power of two and written as a sum of
 *   integer BF16 digits of 4 to 7 bits; every digit product is summed exactly
 *   in the FP32 accumulator (the inner size is split so that the sums stay
 *   below 2^24) and the pair products are combined in FP64, for about 40
 *   significant bits relative to the row and column maxima (about 1e-11
 *   relative to the largest output). Used for the refinement products of the
 *   mixed Davidson when opts.refine selects it.
 * ADC_PREC_SLICED24: the same sliced product with digits for about 24
 *   significant bits (about 1e-7 relative to the largest output): the trial
 *   vectors' leading digits against the same leading digit slices of the
 *   operators, about 40% of the digit products. The intermediate step of that
 *   refinement, for the correction vectors once the BF16x3 products stall. */
enum { ADC_PREC_FP64 = 0, ADC_PREC_BF16X3 = 1, ADC_PREC_BF16X6 = 2, ADC_PREC_SLICED = 3, ADC_PREC_SLICED24 = 4 };

enum {
  ADC_OK = 0,
  ADC_ERR_ARG = -1,         /* invalid argument (sizes, kind, order, non-Hermitian B) */
  ADC_ERR_OOM = -2,         /* device memory exhausted (or above opts.mem_limit) */
  ADC_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  ADC_ERR_NOCONV = -4,      /* Davidson did not converge; best results returned */
  ADC_ERR_TIMEOUT = -5,     /* a bounded device wait gave up */
  ADC_ERR_UNSUPPORTED = -6, /* combination not built (e.g. adc_sigma_noalloc on an EE context) */
  ADC_ERR_STATE = -7,       /* context not initialised / unusable */
  ADC_ERR_NUMERIC = -8      /* NaN or Inf met in a residual or input */
};

typedef struct {
  int precision;        /* default precision of adc_davidson's mixed phase */
  void *stream;         /* cudaStream_t to run on; NULL = the context's own */
  int block;            /* Davidson block size kb, 0 = nroots: the starting
                           space holds max(2 nroots, kb) unit vectors, the
                           default subspace 8 kb; every iteration adds the
                           corrections of the unconverged wanted roots (at
                           most nroots vectors), also when kb > nroots */
  int max_subspace;     /* Davidson subspace limit, 0 = automatic: 8 x the
                           block (at least 40), lowered to what the device
                           memory left once the operators are built holds
                           after the Davidson's other vectors, an estimate of
                           one product's scratch and an 8% margin (short of
                           memory: nroots plus one block, keeping nroots Ritz
                           vectors at a collapse) */
  double herm_tol;      /* relative tolerance of the Hermiticity check of B */
  int64_t mem_limit;    /* bytes the context may allocate, 0 = no limit */
  int verbose;          /* 1 = per-iteration lines on stderr */
  int dd_order;         /* EE only: order of the doubles-doubles block at third
                           order, 1 (full ADC(3), default) or 0 (kept at the
                           ADC(2) level, zeroth order) */
  int refine;           /* products of adc_davidson's refinement (the FP64 base
                           of the Ritz vectors and the final residual check):
                           ADC_PREC_FP64 (default) or ADC_PREC_SLICED */
  int setup;            /* dense contractions of adc_init: ADC_PREC_FP64
                           (default) or ADC_PREC_SLICED (those of at least 2^24
                           flops and inner size 512 as the sliced product with about 48
                           significant bits; the operators then differ from
                           the FP64 ones by about 1e-13 relative) */
  int ee_vvvv;          /* EE third order: the terms of the singles block
                           with four virtual indices (<ab||cd>, or a product
                           of two amplitudes over four virtual indices).
                           0 = automatic: formed in chunks of the first
                           virtual index, never whole, when the dense
                           <ab||cd> would take more than 32 GiB; 1 = always
                           in chunks; -1 = always from the dense block */
  int correction;       /* Davidson correction vectors: 0 = the residuals
                           preconditioned by (omega - diag M)^-1 (default);
                           1 = Olsen's: (omega - diag M)^-1 (r - e y) with e
                           chosen so that the correction is orthogonal to its
                           Ritz vector y */
  int ladder;           /* third order, the four-virtual integrals <ab||cd>
                           (Sec. 2.5: four-external integrals formed on the
                           fly), used by the ladder intermediate of the
                           second-order amplitudes and, for EA, by the 2p1h
                           ladder of every product: 0 = automatic
                           (integral-direct when the packed block would take
                           more than a quarter of the free device memory),
                           1 = integral-direct (formed from B in chunks where
                           needed), -1 = stored once (the packed Pv x Pv block) */
  int profile;          /* 1 = per-kernel timing from the start of adc_init, so
                           that adc_profile_read also reports the setup's GEMMs
                           and its stages ("stage:<name>" entries, each the
                           device time of one step of the setup); 0 = off
                           (default; adc_profile_enable switches it later) */
  int grouped_sigma;    /* IP/EA BF16x3 products with the stored operators:
                           0 = every tensor-core term (both coupling
                           directions, ladder, ring) as jobs of one grouped
                           persistent launch (default); -1 = one launch per term */
} adc_opts;

typedef struct {
  int iterations;       /* Davidson iterations (mixed + FP64 phases) */
  int iterations_fp64;  /* iterations of the FP64 refinement phase */
  int sigma_calls;      /* vectors multiplied by M (all precisions) */
  int sigma_calls_fp64; /* of those, in FP64 or the FP64-accurate sliced product */
  double time_total_s;  /* wall time of the call */
  double time_sigma_s;  /* time inside sigma products */
  double max_residual;  /* largest final FP64 residual norm over the roots */
  int sigma_calls_mid;  /* vectors multiplied with ADC_PREC_SLICED24 (the
                           intermediate refinement step) */
} adc_stats;

/* Fills *opts with the defaults (precision FP64, own stream, herm_tol 1e-12). */
int adc_opts_default(adc_opts *opts);

/* Creates a context for one ADC problem and precomputes on the device
 * everything that does not depend on the trial vectors: the first- and
 * second-order MP amplitudes, the ground-state densities, the static main
 * block (1h or 1p), the coupling block, the packed antisymmetrised ladder
 * integrals (<ab||cd> for EA, <ij||kl> for IP), the ring integrals and the
 * exact diagonal of M (Sec. 2.1 Eqs. 10-12, Sec. 2.5 Eq. 43).
 *   B        [naux][nmo][nmo] Cholesky vectors, B[Q][p][q] = conj(B[Q][q][p]);
 *            checked to opts->herm_tol * max|B|, else ADC_ERR_ARG.
 *   eps_occ  [nocc], eps_vir [nvir]: orbital energies (Hartree); every
 *            eps_occ must lie below every eps_vir, else ADC_ERR_ARG.
 *   kind     ADC_IP, ADC_EA or ADC_EE.
 *   order    2 (ADC(2)) or 3 (ADC(2)+x(3); x = 1 is ADC(3), x = 0 is ADC(2)).
 *   x        scale of every term ADC(3) adds to ADC(2) (used when order == 3).
 *   opts     NULL for the defaults.
 * On success *ctx owns device memory until adc_free(). Synchronous. */
int adc_init(adc_ctx **ctx, const adc_c128 *B, int64_t naux,
             const double *eps_occ, int64_t nocc, const double *eps_vir,
             int64_t nvir, int kind, int order, double x,
             const adc_opts *opts);

/* n1, n2 of the vector layout above. */
int adc_dims(const adc_ctx *ctx, int64_t *n1, int64_t *n2);

/* S[r] = M X[r] for r < k (Eqs. 10-12). X, S: [k][N], host or device, not
 * overlapping. precision: ADC_PREC_FP64, ADC_PREC_BF16X3, ADC_PREC_BF16X6,
 * ADC_PREC_SLICED (the FP64-accurate product from exact BF16 digit products
 * on the tensor cores) or ADC_PREC_SLICED24 (its 24-bit form). Uses scratch
 * device memory owned by the context (grown on demand). */
int adc_sigma(adc_ctx *ctx, const adc_c128 *X, adc_c128 *S, int64_t k,
              int precision);

/* The FP64 product of adc_sigma for callers that cannot allocate GPU memory
 * during the call (device memory owned by another allocator, regions where
 * cudaMalloc is forbidden or would synchronise the device, code that must not
 * fail with out-of-memory halfway). No counterpart in the paper: it is a
 * variant of adc_sigma's FP64 path. It calls no cudaMalloc, cudaFree or
 * allocating library routine; every per-call intermediate lives in one
 * file-scope __device__ array of 64 MiB that each GPU loading the library
 * holds until the process exits.
 *   X, S   [k][N] device pointers on the context's device, which must be
 *          the current device (host pointers, or memory or a current device
 *          other than the one adc_init ran on, give ADC_ERR_ARG).
 *   Sizes whose intermediates exceed the array (2 k o v^2 complex elements
 *   for EA, 2 k o^2 v for IP, order 3) give ADC_ERR_ARG with the required
 *   size; call again with fewer vectors.
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress); make that first call before any
 * stream capture. Every call shares the array and overwrites what it needs
 * (nothing is assumed to start at zero), so calls whose work overlaps on the
 * GPU (other streams, other contexts, other threads) race: serialise them.
 * Asynchronous on the context's stream. */
int adc_sigma_noalloc(adc_ctx *ctx, const adc_c128 *X, adc_c128 *S, int64_t k);

/* One rank's share of the FP64 sigma product (Sec. 2.1, Eqs. 10-12) when an
 * EA problem is split across ranks by the occupied index j of its satellite
 * amplitudes X_j,(a<b): the rank owning j in [i0, i1) holds the satellite
 * rows of those j and a copy of the 1p rows. The ladder term is diagonal in
 * j; the ring and the coupling reach every j, so every rank first gathers the
 * whole trial block.
 *   X          [k][N] the whole trial block (host or device).
 *   S          [k][n1 + (i1 - i0) Pv] output (host or device), Pv = nvir
 *              (nvir - 1) / 2:
 *              S[:, :n1]  partial 1p rows: the coupling of the share's
 *                         satellites, plus M11 X1 when with_main != 0; the
 *                         sum over the ranks (one of them with_main) is S1;
 *              S[:, n1:]  the share's satellite rows of S = M X, complete.
 *   i0, i1     occupied range of the share, 0 <= i0 <= i1 <= nocc.
 * EA contexts only (ADC_ERR_UNSUPPORTED otherwise); ADC_ERR_ARG for a range
 * outside [0, nocc]. Asynchronous on the context's stream unless a pointer
 * is on the host. */
int adc_sigma_share(adc_ctx *ctx, const adc_c128 *X, adc_c128 *S, int64_t k,
                    int64_t i0, int64_t i1, int with_main);

/* Exact diagonal of M as real numbers, [N] (host or device). */
int adc_diagonal(adc_ctx *ctx, double *diag);

/* Static main block (IP: [nocc][nocc], EA: [nvir][nvir], row-major). */
int adc_main_block(adc_ctx *ctx, adc_c128 *M11);

/* Lowest nroots eigenpairs of M (Eq. 10: M X = X Omega, X^H X = 1) by a
 * block Davidson method. Subspace matrices, Rayleigh-Ritz (device Jacobi),
 * residual norms, Gram-Schmidt and the diagonal preconditioner are always
 * FP64. With precision = ADC_PREC_BF16X3 the trial-vector sigma products run
 * on the tensor cores; when the residuals stop decreasing the subspace is
 * collapsed onto the Ritz vectors and their sigma is recomputed in FP64
 * (sigma(y + d) = sigma64(y) + sigma_bf16x3(d)); couplings between those FP64
 * base vectors and later corrections come from the FP64 products. A result
 * is accepted only when every FP64 residual norm ||M y - omega y|| <= tol.
 * With opts.refine = ADC_PREC_SLICED those FP64 products (base, check) are
 * the sliced FP64-accurate tensor-core products instead, and once the
 * refinement stalls twice the corrections take ADC_PREC_SLICED24 before the
 * 40-bit product (st->sigma_calls_mid counts them).
 *   guess   NULL, or [nguess][N] starting vectors (nguess >= nroots).
 *   omega   [nroots] eigenvalues, ascending (host or device).
 *   Y       NULL or [nroots][N] eigenvectors.
 *   err64   NULL or [nroots] residual norms ||M y - omega y|| of the
 *           returned vectors, from the refinement product: FP64 CUDA cores,
 *           or with opts.refine = ADC_PREC_SLICED the sliced product (about
 *           40 significant bits, well below any tolerance above 1e-10 of the
 *           norm of M y); an FP64 check is adc_sigma(ADC_PREC_FP64) of Y.
 *   st      NULL or statistics.
 * Returns ADC_ERR_NOCONV (with the best results written) if max_iter is hit. */
int adc_davidson(adc_ctx *ctx, int nroots, double tol, int max_iter,
                 int precision, const adc_c128 *guess, int64_t nguess,
                 double *omega, adc_c128 *Y, double *err64, adc_stats *st);

/* MP2 virtual-virtual density and frozen natural spinors (Eqs. 25-30):
 *   D_ab = 1/2 sum_cij <ac||ij><ij||bc> / (eps_ij^ac eps_ij^bc)      [nvir][nvir]
 *   D V = V eta, eta descending; keep eta_i >= eta_crit (n_keep of them);
 *   F~ = V~^H diag(eps_vir) V~, F~ Z~ = Z~ eps~ (eps~ ascending);
 *   U = V~ Z~                                                   [nvir][n_keep].
 * Outputs (host or device): D, eta [nvir], V (NULL or [nvir][nvir], column i =
 * natural spinor i), n_keep (host), U (NULL or [nvir][nvir] with the first
 * n_keep columns used, row-major, leading dimension nvir), eps_new (NULL or
 * [nvir], first n_keep used). Eigenvector phases are arbitrary. */
int adc_fns_density(adc_ctx *ctx, adc_c128 *D, double *eta, adc_c128 *V,
                    double eta_crit, int64_t *n_keep, adc_c128 *U,
                    double *eps_new);

/* Cholesky vectors in the truncated natural-spinor basis (Eq. 30 applied as
 * the MO transformation of Eq. 42 to the virtual block):
 *   B'_oo = B_oo,  B'_ov = B_ov U,  B'_vo = U^H B_vo,  B'_vv = U^H B_vv U.
 *   U     [nvir][ldu], its first n_keep columns used (as written by
 *         adc_fns_density with ldu = nvir); host or device.
 *   Bout  [naux][nocc + n_keep][nocc + n_keep]; host or device, caller-owned.
 * With the eps_new of adc_fns_density, (Bout, eps_occ, eps_new) define the
 * ADC problem in the FNS basis (a new context). */
int adc_fns_transform(adc_ctx *ctx, const adc_c128 *U, int64_t ldu,
                      int64_t n_keep, adc_c128 *Bout);

/* Ground-to-excited transition densities of EE-ADC (Sec. 2.2):
 * rho_pq = <Psi_K| a+_p a_q |Psi0> = sum_I conj(Y_I) <Psi~_I| a+_p a_q |Psi0>
 * for each of the k vectors Y [k][N] (normally eigenvectors), with the ISR
 * transition moments through second order for the singles and first order
 * for the doubles:
 *   rho_bj = conj(y_jb) + 1/2 sum_ia conj(y_ia) S2_{ia,jb}   (b virtual, j occupied)
 *   rho_jb = sum_ia conj(y_ia) (t_ij^ab + t2_ij^ab)
 *   rho_kl = -sum_a conj(y_la) s2_k^a - 1/2 sum_jab conj(Y_ljab) t_kj^ab
 *   rho_ef = sum_i conj(y_ie) s2_i^f + 1/2 sum_ijb conj(Y_ijeb) t_ij^fb
 * (t, t2: first- and second-order doubles, s2: second-order singles, S2: the
 * second-order overlap of the orthogonalised singles precursors, Y the
 * doubles as a full antisymmetric array). rho [k][nmo][nmo], orbitals in
 * the order of B (occupied first); host or device. A transition moment of a
 * one-particle operator d is sum_pq d_pq rho_pq. EE contexts only
 * (ADC_ERR_UNSUPPORTED otherwise). Synchronous. */
int adc_transition_density(adc_ctx *ctx, const adc_c128 *Y, int64_t k, adc_c128 *rho);

/* One-particle densities of ADC states of any kind (Sec. 2.2), at the level
 * stated for ADC(2) states: rho^KL_pq = <Psi_K| a+_p a_q |Psi_L> =
 * (y_K^H y_L) rho0_pq + y_K^H G y_L, with rho0 the MP ground-state density
 * through second order (rho0_ij = d_ij - 1/2 sum_kab conj(t_jk^ab) t_ik^ab,
 * rho0_ab = 1/2 sum_ijc conj(t_ij^ac) t_ij^bc, rho0_jb = s2_j^b, rho0_bj =
 * conj(s2_j^b)) and G the zeroth-order intermediate-state representation of
 * a+_p a_q - rho0 (the configurations; Y the class-2 amplitudes as a full
 * antisymmetric array):
 *   EE  kl: -sum_a conj(yK_la) yL_ka - 1/2 sum_jab conj(YK_ljab) YL_kjab
 *       ef:  sum_i conj(yK_ie) yL_if + 1/2 sum_ijc conj(YK_ijec) YL_ijfc
 *       jb:  sum_ia conj(yK_ia) YL_ijab,   bj: sum_ia conj(YK_ijab) yL_ia
 *   IP  kl: -conj(yK_l) yL_k - sum_ja conj(YK_lja) YL_kja
 *       ab:  1/2 sum_ij conj(YK_ija) YL_ijb
 *       jb: -sum_i conj(yK_i) YL_ijb,      bj: -sum_i conj(YK_ijb) yL_i
 *   EA  kl: -1/2 sum_ab conj(YK_lab) YL_kab
 *       ab:  conj(yK_a) yL_b + sum_jc conj(YK_jac) YL_jbc
 *       jb:  sum_a conj(yK_a) YL_jab,      bj: sum_a conj(YK_jab) yL_a
 * adc_excited_density: the state densities rho^KK of the vectors Y [k][N]
 * (trace = electrons of the state for normalised y). adc_state_pair_density:
 * the state-to-state densities of the pairs (YK[z], YL[z]), z < k, YK and YL
 * [k][N]. rho [k][nmo][nmo]; all host or device. Expectation values and
 * state-to-state transition moments are sum_pq d_pq rho_pq. Synchronous. */
int adc_excited_density(adc_ctx *ctx, const adc_c128 *Y, int64_t k, adc_c128 *rho);
int adc_state_pair_density(adc_ctx *ctx, const adc_c128 *YK, const adc_c128 *YL, int64_t k, adc_c128 *rho);

/* Spectroscopic amplitudes of IP/EA-ADC states (Sec. 2.2, the ISR transition
 * moments of a_p and a+_p): x_p = <Psi_n| a_p |Psi0> (IP) or
 * <Psi_n| a+_p |Psi0> (EA) = sum_I conj(Y_I) f_I(p), main class through
 * second and satellites through first order (t: first-order doubles, s2:
 * second-order singles, Y the satellites as a full antisymmetric array):
 *   IP  x_k = conj(y_k) - 1/4 sum_ijab conj(y_i) conj(t_kj^ab) t_ij^ab,
 *       x_b = sum_i conj(y_i) s2_i^b + 1/2 sum_ija conj(Y_ija) t_ij^ab
 *   EA  x_b = conj(y_b) - 1/4 sum_aijc conj(y_a) conj(t_ij^bc) t_ij^ac,
 *       x_k = -sum_a conj(y_a) s2_k^a + 1/2 sum_jab conj(Y_jab) t_jk^ab
 * Pole strengths are |x_p|^2. Y [k][N], x [k][nmo] (orbitals in the order of
 * B, occupied first); host or device. IP and EA contexts only
 * (ADC_ERR_UNSUPPORTED otherwise). Synchronous. */
int adc_spectroscopic_amplitudes(adc_ctx *ctx, const adc_c128 *Y, int64_t k, adc_c128 *x);

/* ------------------------------------------------------------------------
 * Cholesky vectors from two-electron integrals (Sec. 2.5, Eqs. 41-42).
 * ---------------------------------------------------------------------- */

/* One-step pivoted Cholesky decomposition (Eq. 41) of the symmetric positive
 * semidefinite V [n][n] (n = nao^2, V[(mu nu)][(kappa lambda)] = (mu nu|kappa
 * lambda), real): at each step the largest remaining diagonal element is the
 * pivot; the decomposition stops when it is below tau (or not positive) or
 * after max_rank vectors. Every residual element is then below tau.
 *   L      [max_rank][n] (host or device): the vectors, rows beyond the rank zero.
 *   pivots NULL or [max_rank] (host): pivot of each vector.
 *   rank   (host): number of vectors.
 * Synchronous; runs on a stream of its own. */
int adc_cholesky(const double *V, int64_t n, double tau, int64_t max_rank, double *L, int64_t *pivots,
                 int64_t *rank);

/* Eq. 42: B[P] = C^H L^P C, the Cholesky vectors in the molecular spinor
 * basis (the B of adc_init; Hermitian per P when each L^P is symmetric).
 * L [rank][nao][nao] real, C [nao][nmo] complex (columns: spinors), B
 * [rank][nmo][nmo]; host or device. Synchronous. */
int adc_cholesky_mo(const double *L, int64_t rank, int64_t nao, const adc_c128 *C, int64_t nmo, adc_c128 *B);

/* ------------------------------------------------------------------------
 * State-specific frozen natural spinors (Sec. 2.4, Eqs. 31-32), EA and EE.
 * ---------------------------------------------------------------------- */

/* Virtual density of one state, D_ab = <Psi| a+_b a_a |Psi>, with |Psi> the
 * excited configurations weighted by y (the zeroth-order intermediate states
 * of Eq. 31): EA D_ab = y_a conj(y_b) + sum_jc Y_jac conj(Y_jbc), EE D_ab =
 * sum_i y_ia conj(y_ib) + 1/2 sum_ijc Y_ijac conj(Y_ijbc), Y the doubles as
 * full antisymmetric arrays. y [N] (packed layout of adc_dims), D [nvir][nvir];
 * host or device. EA and EE contexts (else ADC_ERR_UNSUPPORTED). Synchronous. */
int adc_state_density(adc_ctx *ctx, const adc_c128 *y, adc_c128 *D);

/* adc_fns_density with the state density of y added to the MP2 density
 * before Eq. 26 (Eq. 31): the state-specific natural spinors of that state.
 * Arguments as adc_fns_density; y [N] host or device. */
int adc_ssfns_density(adc_ctx *ctx, const adc_c128 *y, double eta_crit, adc_c128 *D, double *eta,
                      int64_t *n_keep, adc_c128 *U, double *eps_new);

/* A vector of this context carried into the truncated basis of U ([nvir][ldu],
 * its first n_keep columns): y'_a' = sum_a conj(U_aa') y_a on every virtual
 * index, written packed for nocc occupied and n_keep virtual spinors into
 * g (EA: n_keep + nocc n_keep (n_keep - 1)/2 entries; EE: nocc n_keep +
 * nocc (nocc - 1)/2 n_keep (n_keep - 1)/2). Host or device. Synchronous. */
int adc_fns_vector(adc_ctx *ctx, const adc_c128 *y, const adc_c128 *U, int64_t ldu, int64_t n_keep,
                   adc_c128 *g);

/* Root-specific Davidson: the eigenpair whose vector overlaps `guess` [N]
 * most, followed through the iterations (at every Rayleigh-Ritz step the Ritz
 * vector with the largest |<guess|y>| is the one refined). Precision and
 * refinement as adc_davidson; Y [N] or NULL. ADC_ERR_NOCONV with the best
 * result when max_iter is reached. */
int adc_davidson_follow(adc_ctx *ctx, const adc_c128 *guess, double tol, int max_iter, int precision,
                        double *omega, adc_c128 *Y, double *err64, adc_stats *st);

/* One root of adc_ssfns. */
typedef struct {
  double omega_corrected;  /* Eq. 32: omega_fns + omega2_canonical - omega2_fns */
  double omega_fns;        /* ADC(order) root in the state-specific basis (root-specific solve) */
  double omega2_canonical; /* ADC(2) root k in the canonical basis */
  double omega2_fns;       /* ADC(2) root in the state-specific basis (root-specific solve) */
  double err64;            /* residual norm of the ADC(order) solve */
  int64_t n_keep;          /* natural spinors kept */
  int status;              /* ADC_OK, ADC_ERR_NOCONV (a solve did not converge) or ADC_ERR_ARG
                              (too few natural spinors kept: EA needs 2, EE 1) */
  int pad_;
} adc_ssfns_root;

/* The state-specific natural-spinor procedure for the nroots lowest roots of
 * EA- or EE-ADC: canonical ADC(2) roots and vectors; per root the density of
 * Eq. 31, natural spinors with occupation >= eta_crit and their
 * semicanonical energies (Eqs. 26-30), the Cholesky vectors in that basis,
 * root-specific ADC(2) and ADC(order) (x as in adc_init) solves from the
 * carried-over canonical vector, and the corrected energy of Eq. 32. Inputs
 * as adc_init (host or device); out [nroots] (host). Every solve uses
 * `precision` and `tol`; opts (or NULL) applies to every context. Returns
 * ADC_OK when every root has a result (see status), else an error code. */
int adc_ssfns(const adc_c128 *B, int64_t naux, const double *eps_occ, int64_t nocc, const double *eps_vir,
              int64_t nvir, int kind, int order, double x, int nroots, double eta_crit, double tol, int max_iter,
              int precision, const adc_opts *opts, adc_ssfns_root *out);

/* Backward pass of the roots (Hellmann-Feynman, Eq. 10): with Y the
 * normalised eigenvectors of nroots non-degenerate roots ([nroots][N], host
 * or device) and weights gomega[r] (host), writes the gradients of
 * L = sum_r gomega[r] y_r^H M y_r = sum_r gomega[r] omega_r with respect to
 * the inputs of adc_init: gB [naux][nmo][nmo] complex in the convention
 * dL/dRe + i dL/dIm per element (the Hermitian structure of B is not
 * imposed, so a Hermitian change dB changes L by sum Re(conj(gB) dB)),
 * geps_occ [nocc], geps_vir [nvir] and *gx (host). gB and the energy
 * gradients may be host or device arrays. The integral and amplitude
 * intermediates are recomputed from the context's cached blocks (the
 * second-order amplitudes of IP/EA-ADC(3) anew). All kinds (IP, EA, EE) and
 * orders; at order 3 *gx is dL/dx even for x = 0. Memory: the dense integral
 * blocks the term tables name and their gradients, up to two v^4 arrays for
 * EA and EE at third order. Synchronous. */
int adc_sigma_adjoint(adc_ctx *ctx, const adc_c128 *Y, const double *gomega, int64_t nroots, adc_c128 *gB,
                      double *geps_occ, double *geps_vir, double *gx);

/* Blocks until all work the context has queued on its stream is done. Needed
 * after an asynchronous call with device pointers before another stream (or
 * the host) reads the outputs. */
int adc_sync(adc_ctx *ctx);

/* Releases every resource of the context (NULL is accepted). */
void adc_free(adc_ctx *ctx);

/* Static string naming an ADC_ERR_* code. */
const char *adc_strerror(int code);

/* Last error message recorded by the context (or by the library when ctx is
 * NULL); valid until the next call on the same context. */
const char *adc_last_error(const adc_ctx *ctx);

/* ------------------------------------------------------------------------
 * Batches of independent problems (IP/EA; EE contexts take part in FP64
 * only). The paper solves one problem at a time; batching is this library's
 * addition for many small problems on one GPU.
 * ---------------------------------------------------------------------- */
typedef struct adc_batch adc_batch;

/* Counters of a batch (all since adc_batch_create, or of one adc_batch_solve). */
typedef struct {
  int64_t batches;          /* batched split-precision sigma products executed */
  int64_t graph_launches;   /* of those, replays of a captured CUDA graph */
  int64_t graphs_captured;  /* graphs captured (a batch is captured at its second occurrence) */
  int64_t direct_launches;  /* batches enqueued without a graph */
  int64_t sigma_vectors;    /* vectors multiplied in batched products (padding included) */
  double batch_ms;          /* device time of the batched products (CUDA events) */
  double tc_flops;          /* algorithmic flops of their tensor-core jobs (8 per complex MAC) */
  int64_t tuned_shapes;     /* GEMM shapes whose tile width the autotuner has timed (process-wide) */
  int64_t waves;            /* adc_batch_solve: groups of problems resident together */
  double init_s;            /* adc_batch_solve: wall time of the adc_init calls */
  double solve_s;           /* adc_batch_solve: wall time of the batched Davidson runs */
  int64_t grouped_launches; /* batches run without a graph, whose grouped kernel was timed alone */
  double grouped_ms;        /* device time of those grouped tensor-core launches (CUDA events) */
  double grouped_flops;     /* their algorithmic flops */
} adc_batch_info;

/* Groups n existing contexts (distinct, each in no other batch; the caller
 * keeps ownership and frees the batch before the contexts). */
int adc_batch_create(adc_batch **batch, adc_ctx *const *ctxs, int n);

/* S[i] = M_i X[i] for every context i with k[i] > 0 vectors (X[i], S[i]:
 * [k[i]][N_i] device arrays, same layout as adc_sigma). With
 * ADC_PREC_BF16X3 all coupling, ladder and ring products of all problems are
 * the jobs of one grouped persistent tensor-core launch (tile widths chosen
 * by an autotuner that times each new GEMM shape once); a call that repeats
 * with the same contexts, block sizes and pointers is captured as a CUDA
 * graph at its second occurrence and replayed from then on. ADC_PREC_FP64
 * runs the problems' FP64 products one after the other. Synchronous. EE
 * contexts with ADC_PREC_BF16X3: ADC_ERR_UNSUPPORTED. */
int adc_batch_sigma(adc_batch *batch, const adc_c128 *const *X, adc_c128 *const *S, const int64_t *k,
                    int precision);

/* The lowest nroots roots of every problem (adc_davidson semantics per
 * problem, FP64 residual tolerance tol): each problem runs on its own host
 * thread and stream, and the split-precision sigma products of the new
 * blocks of all running problems are executed together as one batched
 * product (nroots vectors per problem; rows beyond a problem's new block are
 * computed and ignored). omega, err64: [n][nroots] host arrays; status[i] =
 * the problem's return code; st: NULL or [n]. Returns ADC_OK, ADC_ERR_NOCONV
 * if a problem did not converge, or the last other error. */
int adc_batch_davidson(adc_batch *batch, int nroots, double tol, int max_iter, int precision, double *omega,
                       double *err64, int *status, adc_stats *st);

/* Switches graph capture of repeated batches on (default) or off. */
int adc_batch_use_graphs(adc_batch *batch, int on);
int adc_batch_info_get(const adc_batch *batch, adc_batch_info *info);
void adc_batch_free(adc_batch *batch);
const char *adc_batch_last_error(const adc_batch *batch);

/* One problem given as raw inputs (the arguments of adc_init). */
typedef struct {
  const adc_c128 *B;
  int64_t naux;
  const double *eps_occ;
  int64_t nocc;
  const double *eps_vir;
  int64_t nvir;
  int kind, order;
  double x;
} adc_problem;

typedef struct {
  int64_t mem_budget;  /* device bytes for resident problems, 0 = 85% of the free memory */
  int init_lanes;      /* concurrent adc_init calls, 0 = 4 */
  int verbose;
  int setup;           /* adc_opts.setup of every problem's adc_init (ADC_PREC_FP64 or ADC_PREC_SLICED) */
  int refine;          /* adc_opts.refine of every problem (ADC_PREC_FP64 or ADC_PREC_SLICED;
                          the waves then leave room for the sliced operator copies) */
} adc_batch_opts;

/* Host-only planner (no GPU needed): estimated device bytes mem_est[i] and
 * work cost_est[i] (complex MACs) of every problem, the order of decreasing
 * cost (order[0..n)), and the wave wave[i] of every problem: problems are
 * taken in that order and each joins the first wave whose estimated memory
 * stays within mem_budget (a problem larger than the budget gets a wave of
 * its own). Returns the number of waves or a negative error code. Only the
 * sizes, kind, order and x of the problems are read. */
int adc_batch_plan(int n, const adc_problem *problems, int nroots, int64_t mem_budget, int *order, int *wave,
                   int64_t *mem_est, double *cost_est);

/* Solves n problems wave by wave: each wave's contexts are initialised on
 * opts->init_lanes concurrent lanes, solved with adc_batch_davidson and
 * freed. omega, err64: [n][nroots]; status: [n]; info: NULL or totals. */
int adc_batch_solve(int n, const adc_problem *problems, int nroots, double tol, int max_iter, int precision,
                    const adc_batch_opts *opts, double *omega, double *err64, int *status, adc_batch_info *info);

#ifdef __cplusplus
}
#endif

#endif /* ADC_GB300_H */
