// Sigma product with the dense contractions on the tensor cores: the BF16x3
// (BF16x6) split (sigma_split) or the sliced FP64-accurate product
// (sigma_sliced, tc_slice.cu). Same terms as sigma.cu (Sec. 2.1 Eqs. 10-12);
// the coupling, ladder and ring contractions run on the tensor cores, the main
// block (n1 x n1) and the zeroth-order diagonal stay FP64.
#include "ctx.cuh"
#include "tc_gemm.cuh"
#include "tc_slice.cuh"

namespace adc {

static void build_cache(adc_ctx *c, int planes) {
  Exec &ex = c->ex;
  auto &tc = *c->tc;
  const int64_t o = c->o, v = c->v, n1 = c->n1, n2 = c->n2;
  tc.planes = planes;
  tc_pack_A(ex, tc.Cpl, c->Cpl.c(), n1, n2, n2, 1, false, planes);
  tc_pack_A(ex, tc.CplT, c->Cpl.c(), n2, n1, 1, n2, true, planes);
  if (c->order == 3 && c->x != 0.0) {
    const int64_t P = (c->kind == ADC_EA) ? npairs(v) : npairs(o);
    if (!(c->kind == ADC_EA && c->direct_ladder)) tc_pack_A(ex, tc.Glad, c->Glad.c(), P, P, P, 1, false, planes);
    tc_pack_A(ex, tc.W, c->W.c(), o * v, o * v, o * v, 1, false, planes);
  }
  tc.err = DBuf(ex, sizeof(int));
  fill_zero(ex, tc.err.p, sizeof(int));
  tc.ready = true;
}

void release_tc(adc_ctx *c) {
  c->tc.reset();
  c->sl.reset();
}

void tc_ensure(adc_ctx *c, int planes) {
  if (c->tc && c->tc->ready && c->tc->planes < planes) c->tc.reset();  // rebuild with more planes
  if (!c->tc) c->tc.reset(new TcCache());
  if (!c->tc->ready) build_cache(c, planes);
}

namespace {
// S2[r][i] += T2[r][i] + d2[i] X2[r][i] (rows r of pitch N in S and X, n2 in T2)
__global__ void k_sat_finish(int64_t k, int64_t n2, const double *__restrict__ d2, const cplx *__restrict__ X2,
                             const cplx *__restrict__ T2, int64_t N, cplx *S2) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < k * n2;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / n2, i = idx - r * n2;
    const cplx x = X2[r * N + i], t = T2[idx];
    cplx *s = S2 + r * N + i;
    *s = cmake(s->x + t.x + d2[i] * x.x, s->y + t.y + d2[i] * x.y);
  }
}
}  // namespace

// The BF16x3 product with every tensor-core contraction (both coupling
// directions, the satellite ladder and ring) as jobs of one persistent grouped
// launch: tiles of all terms share the SMs, so no term leaves a partly idle
// last wave, and the long-K coupling into the 1p rows is split over the SMs.
// Jobs never accumulate into the same output: the ladder writes the satellite
// rows, the coupling into them goes to a scratch block added afterwards.
static void sigma_split_grouped(adc_ctx *c, const cplx *X, cplx *S, int64_t k) {
  Exec &ex = c->ex;
  auto &tc = *c->tc;
  int *err = (int *)tc.err.p;
  const int64_t o = c->o, v = c->v, n1 = c->n1, n2 = c->n2, N = c->N;
  const bool sat = (c->order == 3 && c->x != 0.0);
  const double x = sat ? c->x : 0.0;
  const bool ea = (c->kind == ADC_EA);
  TagScope tg(ex, "main");
  zgemm(ex, k, n1, n1, 1, C1(), X, 0, N, 1, false, c->M11.c(), 0, 1, n1, false, C0(), S, 0, N, 1);
  ex.tag = "grouped";
  const int64_t nring = sat ? (ea ? k * o * v * v : k * o * v * o) : 0;
  cplx *T = scratch(c, nring + k * n2);  // ring block, then the coupling into the satellites
  cplx *T2 = T + nring;
  std::vector<TcJobDesc> jobs;
  // S1 += Cpl X2 : out[c][r] = sum_K Cpl[c][K] X2[r][K]
  tc_pack_B(ex, tc.Bx2, X + n1, k, n2, N, 0, 1, 1, false, 2);
  {
    TcJobDesc d;
    d.A = &tc.Cpl; d.B = &tc.Bx2; d.M = n1; d.N = k;
    d.alpha = C1(); d.beta = C1(); d.out = S; d.s_m = 1; d.s_nh = N; d.s_nl = 0; d.n_in = 1;
    jobs.push_back(d);
  }
  // T2 = Cpl^H X1 : out[K][r] = sum_c conj(Cpl[c][K]) X1[r][c]
  tc_pack_B(ex, tc.Bx1, X, k, n1, N, 0, 1, 1, false, 2);
  {
    TcJobDesc d;
    d.A = &tc.CplT; d.B = &tc.Bx1; d.M = n2; d.N = k;
    d.alpha = C1(); d.beta = C0(); d.out = T2; d.s_m = 1; d.s_nh = n2; d.s_nl = 0; d.n_in = 1;
    jobs.push_back(d);
  }
  if (sat) {
    if (ea) {
      const int64_t pv = npairs(v);
      // ladder: out[(ab)][(r,j)] = x sum_(cd) Glad[(ab)][(cd)] X2[r][j][(cd)], the satellite rows set
      tc_pack_B(ex, tc.Bxl, X + n1, k * o, pv, N, pv, o, 1, false, 2);
      TcJobDesc d;
      d.A = &tc.Glad; d.B = &tc.Bxl; d.M = pv; d.N = k * o;
      d.alpha = CR(x); d.beta = C0(); d.out = S + n1; d.s_m = 1; d.s_nh = N; d.s_nl = pv; d.n_in = o;
      jobs.push_back(d);
      // ring: T[r][j][a][b] = sum_(kc) W[(j,a)][(kc)] Xf[r][k][c][b]
      tc_pack_B_ring(ex, tc.Bxr, c, X, k, 2);
      TcJobDesc e;
      e.A = &tc.W; e.B = &tc.Bxr; e.M = o * v; e.N = k * v;
      e.alpha = C1(); e.beta = C0(); e.out = T; e.s_m = v; e.s_nh = o * v * v; e.s_nl = 1; e.n_in = v;
      jobs.push_back(e);
    } else {
      const int64_t po = npairs(o);
      // ladder: out[(ij)][(r,a)] = x sum_(kl) Glad[(ij)][(kl)] X2[r][(kl)][a], the satellite rows set
      tc_pack_B(ex, tc.Bxl, X + n1, k * v, po, N, 1, v, v, false, 2);
      TcJobDesc d;
      d.A = &tc.Glad; d.B = &tc.Bxl; d.M = po; d.N = k * v;
      d.alpha = CR(x); d.beta = C0(); d.out = S + n1; d.s_m = v; d.s_nh = N; d.s_nl = 1; d.n_in = v;
      jobs.push_back(d);
      // ring: T[r][j][a][i] = -sum_(kb) W[(j,a)][(kb)] Xf[r][i][k][b]
      tc_pack_B_ring(ex, tc.Bxr, c, X, k, 2);
      TcJobDesc e;
      e.A = &tc.W; e.B = &tc.Bxr; e.M = o * v; e.N = k * o;
      e.alpha = CR(-1.0); e.beta = C0(); e.out = T; e.s_m = o; e.s_nh = o * v * o; e.s_nl = 1; e.n_in = o;
      jobs.push_back(e);
    }
  } else {
    ADC_CUDA(cudaMemset2DAsync(S + n1, N * sizeof(cplx), 0, n2 * sizeof(cplx), k, ex.stream));
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  ADC_CUDA(cudaStreamIsCapturing(ex.stream, &cs));
  tc_gemm_grouped(ex, jobs, tc.grp, err, cs == cudaStreamCaptureStatusNone);
  ex.tag = "satellites";
  k_sat_finish<<<grid1d(k * n2, 256), 256, 0, ex.stream>>>(k, n2, c->d2.d(), X + n1, T2, N, S + n1);
  ADC_CHECK_LAUNCH();
  if (sat) {
    if (ea)
      pair_pack(ex, T, o * v * v, v * v, v, 1, 0, 1.0, k, o, v, 1, S + n1, N, npairs(v), CR(-x), C1());
    else
      pair_pack(ex, T, o * v * o, 0, 1, v * o, o, 1.0, k, 1, o, v, S + n1, N, 0, CR(x), C1());
  }
  int h = 0;
  ADC_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, ex.stream));
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
  if (h != 0) {
    fill_zero(ex, err, sizeof(int));
    throw Error(ADC_ERR_TIMEOUT, "tensor-core GEMM wait gave up (code " + std::to_string(h) + ")");
  }
}

void sigma_split(adc_ctx *c, const cplx *X, cplx *S, int64_t k, int nseg) {
  Exec &ex = c->ex;
  const int planes = (nseg == 6) ? 3 : 2;
  tc_ensure(c, planes);
  // the three-product split of the stored operators: one grouped launch
  if (nseg == 3 && !(c->kind == ADC_EA && c->direct_ladder) && c->opts.grouped_sigma != -1) {
    sigma_split_grouped(c, X, S, k);
    return;
  }
  auto &tc = *c->tc;
  int *err = (int *)tc.err.p;
  const int64_t o = c->o, v = c->v, n1 = c->n1, n2 = c->n2, N = c->N;
  const bool sat = (c->order == 3 && c->x != 0.0);
  const double x = sat ? c->x : 0.0;
  // S1 = X1 M11^T (FP64, n1 x n1)
  TagScope tg(ex, "main");
  zgemm(ex, k, n1, n1, 1, C1(), X, 0, N, 1, false, c->M11.c(), 0, 1, n1, false, C0(), S, 0, N, 1);
  // S1 += Cpl X2  : out[c][r] = sum_K Cpl[c][K] X2[r][K]
  ex.tag = "coupling";
  tc_pack_B(ex, tc.Bx, X + n1, k, n2, N, 0, 1, 1, false, planes);
  tc_gemm(ex, tc.Cpl, tc.Bx, n1, k, C1(), C1(), S, 1, N, 0, 1, err, nseg);
  // S2 = Cpl^H X1 : out[K][r] = sum_c conj(Cpl[c][K]) X1[r][c]
  tc_pack_B(ex, tc.Bx, X, k, n1, N, 0, 1, 1, false, planes);
  tc_gemm(ex, tc.CplT, tc.Bx, n2, k, C1(), C0(), S + n1, 1, N, 0, 1, err, nseg);
  diag_mul_add(ex, k, n2, c->d2.d(), X + n1, N, S + n1, N, 1.0);
  if (sat) {
    if (c->kind == ADC_EA) {
      const int64_t pv = npairs(v);
      // ladder: out[(ab)][(r,j)] = sum_(cd) Glad[(ab)][(cd)] X2[r][j][(cd)]
      ex.tag = "ladder";
      if (c->direct_ladder) {
        ladder_direct(c, X + n1, N, o, S + n1, N, k, x, nseg, err);
      } else {
        tc_pack_B(ex, tc.Bx, X + n1, k * o, pv, N, pv, o, 1, false, planes);
        tc_gemm(ex, tc.Glad, tc.Bx, pv, k * o, CR(x), C1(), S + n1, 1, N, pv, o, err, nseg);
      }
      // ring: T[r][j][a][b] = sum_(kc) W[(j,a)][(kc)] Xf[r][k][c][b]
      ex.tag = "ring";
      cplx *T = scratch(c, k * o * v * v);
      tc_pack_B_ring(ex, tc.Bx, c, X, k, planes);
      tc_gemm(ex, tc.W, tc.Bx, o * v, k * v, C1(), C0(), T, v, o * v * v, 1, v, err, nseg);
      pair_pack(ex, T, o * v * v, v * v, v, 1, 0, 1.0, k, o, v, 1, S + n1, N, pv, CR(-x), C1());
    } else {
      const int64_t po = npairs(o);
      // ladder: out[(ij)][(r,a)] = sum_(kl) Glad[(ij)][(kl)] X2[r][(kl)][a]
      ex.tag = "ladder";
      tc_pack_B(ex, tc.Bx, X + n1, k * v, po, N, 1, v, v, false, planes);
      tc_gemm(ex, tc.Glad, tc.Bx, po, k * v, CR(x), C1(), S + n1, v, N, 1, v, err, nseg);
      // ring: T[r][j][a][i] = -sum_(kb) W[(j,a)][(kb)] Xf[r][i][k][b]
      ex.tag = "ring";
      cplx *T = scratch(c, k * o * v * o);
      tc_pack_B_ring(ex, tc.Bx, c, X, k, planes);
      tc_gemm(ex, tc.W, tc.Bx, o * v, k * o, CR(-1.0), C0(), T, o, o * v * o, 1, o, err, nseg);
      pair_pack(ex, T, o * v * o, 0, 1, v * o, o, 1.0, k, 1, o, v, S + n1, N, 0, CR(x), C1());
    }
  }
  int h = 0;
  ADC_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, ex.stream));
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
  if (h != 0) {
    fill_zero(ex, err, sizeof(int));
    throw Error(ADC_ERR_TIMEOUT, "tensor-core GEMM wait gave up (code " + std::to_string(h) + ")");
  }
}

// ---- FP64-accurate sigma: the same contractions as sliced tensor-core products.
// The operators are sliced once for kSlicedBits; a product with fewer bits
// (the intermediate refinement step) slices only the leading digits of the
// trial vectors and pairs them with the same leading slices of the operators.
static void build_sl(adc_ctx *c) {
  Exec &ex = c->ex;
  c->sl.reset(new SlCache());
  SlCache &sl = *c->sl;
  const int64_t o = c->o, v = c->v, n1 = c->n1, n2 = c->n2;
  sl.bits = kSlicedBits;
  sl_pack_A(ex, sl.Cpl, c->Cpl.c(), n1, n2, n2, 1, false, sl.bits);
  sl_pack_A(ex, sl.CplT, c->Cpl.c(), n2, n1, 1, n2, true, sl.bits);
  if (c->order == 3 && c->x != 0.0) {
    const int64_t P = (c->kind == ADC_EA) ? npairs(v) : npairs(o);
    if (!(c->kind == ADC_EA && c->direct_ladder)) sl_pack_A(ex, sl.Glad, c->Glad.c(), P, P, P, 1, false, sl.bits);
    sl_pack_A(ex, sl.W, c->W.c(), o * v, o * v, o * v, 1, false, sl.bits);
  }
  sl.err = DBuf(ex, sizeof(int));
  fill_zero(ex, sl.err.p, sizeof(int));
  sl.ready = true;
}

void sigma_sliced(adc_ctx *c, const cplx *X, cplx *S, int64_t k, int bits) {
  ADC_REQUIRE(c->kind != ADC_EE, ADC_ERR_ARG, "sigma_sliced: IP and EA (EE goes through sigma_ee_split)");
  Exec &ex = c->ex;
  if (!c->sl || !c->sl->ready) build_sl(c);
  SlCache &sl = *c->sl;
  int *err = (int *)sl.err.p;
  const int64_t o = c->o, v = c->v, n1 = c->n1, n2 = c->n2, N = c->N;
  const bool sat = (c->order == 3 && c->x != 0.0);
  const double x = sat ? c->x : 0.0;
  // S1 = X1 M11^T (FP64, n1 x n1)
  TagScope tg(ex, "main");
  zgemm(ex, k, n1, n1, 1, C1(), X, 0, N, 1, false, c->M11.c(), 0, 1, n1, false, C0(), S, 0, N, 1);
  // S1 += Cpl X2, S2 = Cpl^H X1
  ex.tag = "coupling";
  sl_pack_B(ex, sl.Bx, X + n1, k, n2, N, 0, 1, 1, false, sl.Cpl, bits);
  sl_gemm(ex, sl.Cpl, sl.Bx, n1, k, C1(), C1(), S, 1, N, 0, 1, err, sl.w);
  sl_pack_B(ex, sl.Bx, X, k, n1, N, 0, 1, 1, false, sl.CplT, bits);
  sl_gemm(ex, sl.CplT, sl.Bx, n2, k, C1(), C0(), S + n1, 1, N, 0, 1, err, sl.w);
  diag_mul_add(ex, k, n2, c->d2.d(), X + n1, N, S + n1, N, 1.0);
  if (sat) {
    if (c->kind == ADC_EA) {
      const int64_t pv = npairs(v);
      ex.tag = "ladder";
      if (c->direct_ladder) {
        ladder_direct(c, X + n1, N, o, S + n1, N, k, x, ADC_LADDER_SLICED, err);
      } else {
        sl_pack_B(ex, sl.Bx, X + n1, k * o, pv, N, pv, o, 1, false, sl.Glad, bits);
        sl_gemm(ex, sl.Glad, sl.Bx, pv, k * o, CR(x), C1(), S + n1, 1, N, pv, o, err, sl.w);
      }
      ex.tag = "ring";
      cplx *T = scratch(c, k * o * v * v);
      sl_pack_B_ring(ex, sl.Bx, c, X, k, sl.W, bits);
      sl_gemm(ex, sl.W, sl.Bx, o * v, k * v, C1(), C0(), T, v, o * v * v, 1, v, err, sl.w);
      pair_pack(ex, T, o * v * v, v * v, v, 1, 0, 1.0, k, o, v, 1, S + n1, N, pv, CR(-x), C1());
    } else {
      const int64_t po = npairs(o);
      ex.tag = "ladder";
      sl_pack_B(ex, sl.Bx, X + n1, k * v, po, N, 1, v, v, false, sl.Glad, bits);
      sl_gemm(ex, sl.Glad, sl.Bx, po, k * v, CR(x), C1(), S + n1, v, N, 1, v, err, sl.w);
      ex.tag = "ring";
      cplx *T = scratch(c, k * o * v * o);
      sl_pack_B_ring(ex, sl.Bx, c, X, k, sl.W, bits);
      sl_gemm(ex, sl.W, sl.Bx, o * v, k * o, CR(-1.0), C0(), T, o, o * v * o, 1, o, err, sl.w);
      pair_pack(ex, T, o * v * o, 0, 1, v * o, o, 1.0, k, 1, o, v, S + n1, N, 0, CR(x), C1());
    }
  }
  int h = 0;
  ADC_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, ex.stream));
  ADC_CUDA(cudaStreamSynchronize(ex.stream));
  if (h != 0) {
    fill_zero(ex, err, sizeof(int));
    throw Error(ADC_ERR_TIMEOUT, "tensor-core GEMM wait gave up (code " + std::to_string(h) + ")");
  }
}

}  // namespace adc
