// Batches of independent ADC problems on one GPU.
//
// * Batched sigma: the split-precision sigma products of many IP/EA problems
//   (each with its own block of trial vectors) go through one grouped
//   persistent tensor-core launch (coupling, ladder and ring of every problem
//   are jobs of the same launch), framed by per-problem packing and epilogue
//   kernels. A batch that repeats (same problems, block sizes and vectors) is
//   captured once as a CUDA graph and replayed.
// * Batched Davidson: every problem runs its own Davidson (Eq. 10) on its own
//   host thread and stream; whenever all running problems ask for a
//   split-precision sigma of their new block, one thread executes the whole
//   set as one batched sigma. FP64 sigma products (refinement) stay per
//   problem.
// * Scheduler: for problems given as raw inputs, a host-only planner orders
//   them by estimated cost (longest first) and packs them into waves whose
//   estimated device memory fits the budget; each wave is initialised on a
//   few concurrent lanes and solved as one batch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "ctx.cuh"
#include "tc_gemm.cuh"
#include "../../include/adc_gb300.h"

namespace adc {

namespace {
// dst rows (pitch ldd) += src rows (pitch lds), k rows of n elements
__global__ void k_rows_add(int64_t k, int64_t n, const cplx *src, int64_t lds, cplx *dst, int64_t ldd) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < k * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / n, i = idx - r * n;
    dst[r * ldd + i] = cadd(dst[r * ldd + i], src[r * lds + i]);
  }
}

struct BatchReq {
  int slot;
  const cplx *X;
  cplx *S;
  int64_t k;
  bool done = false;
  int rc = 0;
  std::string msg;
};

// per-problem operands of the batched launch (sized for the largest block seen)
struct Scratch {
  TcMat BxC, BxT, BxL, BxR;
  DBuf P2, T;
};

struct Plan {
  TcGroup grp;     // owned by the captured graph once there is one
  TcGroup direct;  // for launches without the graph after capture
  cudaGraphExec_t exec = nullptr;
  int uses = 0;
  ~Plan() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
}  // namespace

struct BatchCoord {
  std::vector<adc_ctx *> ctx;
  std::vector<Scratch> scr;
  Exec bex;
  DBuf err;
  int dev = 0;
  bool use_graphs = true;
  std::mutex mu;
  std::condition_variable cv;
  int active = 0;
  std::vector<BatchReq *> pending;
  std::map<std::vector<int64_t>, std::unique_ptr<Plan>> plans;
  cudaEvent_t e0 = nullptr, e1 = nullptr, g0 = nullptr, g1 = nullptr;
  bool grouped_timed = false;
  adc_batch_info info{};

  ~BatchCoord() {
    if (bex.stream) cudaStreamSynchronize(bex.stream);
    plans.clear();
    scr.clear();
    err.reset();
    if (bex.stream) cudaStreamSynchronize(bex.stream);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (g0) cudaEventDestroy(g0);
    if (g1) cudaEventDestroy(g1);
    if (bex.stream) cudaStreamDestroy(bex.stream);
  }

  // all work of one batched split-precision sigma, enqueued on the batch stream
  void enqueue(const std::vector<BatchReq *> &reqs, TcGroup &grp, bool may_tune) {
    std::vector<TcJobDesc> jobs;
    int *errw = (int *)err.p;
    for (BatchReq *r : reqs) {
      adc_ctx *c = ctx[r->slot];
      Scratch &sc = scr[r->slot];
      const int64_t k = r->k, o = c->o, v = c->v, n1 = c->n1, n2 = c->n2, N = c->N;
      const bool sat = (c->order == 3 && c->x != 0.0);
      const double x = sat ? c->x : 0.0;
      const cplx *X = r->X;
      cplx *S = r->S;
      auto &tc = *c->tc;
      // S1 = X1 M11^T (FP64); the coupling job then accumulates into it
      zgemm(bex, k, n1, n1, 1, C1(), X, 0, N, 1, false, c->M11.c(), 0, 1, n1, false, C0(), S, 0, N, 1);
      tc_pack_B(bex, sc.BxC, X + n1, k, n2, N, 0, 1, 1, false);
      tc_pack_B(bex, sc.BxT, X, k, n1, N, 0, 1, 1, false);
      TcJobDesc jc;
      jc.A = &tc.Cpl; jc.B = &sc.BxC; jc.M = n1; jc.N = k; jc.beta = C1();
      jc.out = S; jc.s_m = 1; jc.s_nh = N;
      jobs.push_back(jc);
      TcJobDesc jt;
      jt.A = &tc.CplT; jt.B = &sc.BxT; jt.M = n2; jt.N = k;
      if (sat) {
        const int64_t p2 = k * n2;
        if (sc.P2.bytes < (size_t)p2 * sizeof(cplx)) { sc.P2.reset(); sc.P2 = cbuf(bex, p2); }
        jt.out = sc.P2.c(); jt.s_m = 1; jt.s_nh = n2;
      } else {
        jt.out = S + n1; jt.s_m = 1; jt.s_nh = N;
      }
      jobs.push_back(jt);
      if (sat) {
        TcJobDesc jl, jr;
        jl.A = &tc.Glad; jl.B = &sc.BxL; jl.alpha = CR(x);
        jr.A = &tc.W; jr.B = &sc.BxR;
        const int64_t tsz = (c->kind == ADC_EA) ? k * o * v * v : k * o * v * o;
        if (sc.T.bytes < (size_t)tsz * sizeof(cplx)) { sc.T.reset(); sc.T = cbuf(bex, tsz); }
        if (c->kind == ADC_EA) {
          const int64_t pv = npairs(v);
          tc_pack_B(bex, sc.BxL, X + n1, k * o, pv, N, pv, o, 1, false);
          jl.M = pv; jl.N = k * o; jl.out = S + n1; jl.s_m = 1; jl.s_nh = N; jl.s_nl = pv; jl.n_in = o;
          tc_pack_B_ring(bex, sc.BxR, c, X, k);
          jr.M = o * v; jr.N = k * v; jr.out = sc.T.c(); jr.s_m = v; jr.s_nh = o * v * v; jr.s_nl = 1; jr.n_in = v;
        } else {
          const int64_t po = npairs(o);
          tc_pack_B(bex, sc.BxL, X + n1, k * v, po, N, 1, v, v, false);
          jl.M = po; jl.N = k * v; jl.out = S + n1; jl.s_m = v; jl.s_nh = N; jl.s_nl = 1; jl.n_in = v;
          tc_pack_B_ring(bex, sc.BxR, c, X, k);
          jr.M = o * v; jr.N = k * o; jr.alpha = CR(-1.0); jr.out = sc.T.c(); jr.s_m = o; jr.s_nh = o * v * o;
          jr.s_nl = 1; jr.n_in = o;
        }
        jobs.push_back(jl);
        jobs.push_back(jr);
      }
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    ADC_CUDA(cudaStreamIsCapturing(bex.stream, &cs));
    const bool timed = (cs == cudaStreamCaptureStatusNone);
    if (may_tune) {
      // tile widths are timed before the launch that is measured
      for (auto &j : jobs)
        if (j.bn <= 0 && j.M > 0 && j.N > 0) j.bn = tc_autotune_bn(bex, j, errw);
    }
    if (timed) ADC_CUDA(cudaEventRecord(g0, bex.stream));
    tc_gemm_grouped(bex, jobs, grp, errw, may_tune);
    if (timed) {
      ADC_CUDA(cudaEventRecord(g1, bex.stream));
      grouped_timed = true;
    }
    for (BatchReq *r : reqs) {
      adc_ctx *c = ctx[r->slot];
      Scratch &sc = scr[r->slot];
      const int64_t k = r->k, o = c->o, v = c->v, n1 = c->n1, n2 = c->n2, N = c->N;
      const bool sat = (c->order == 3 && c->x != 0.0);
      cplx *S = r->S;
      if (sat) {
        k_rows_add<<<grid1d(k * n2, 256), 256, 0, bex.stream>>>(k, n2, sc.P2.c(), n2, S + n1, N);
        ADC_CHECK_LAUNCH();
        if (c->kind == ADC_EA)
          pair_pack(bex, sc.T.c(), o * v * v, v * v, v, 1, 0, 1.0, k, o, v, 1, S + n1, N, npairs(v), CR(-c->x), C1());
        else
          pair_pack(bex, sc.T.c(), o * v * o, 0, 1, v * o, o, 1.0, k, 1, o, v, S + n1, N, 0, CR(c->x), C1());
      }
      diag_mul_add(bex, k, n2, c->d2.d(), r->X + n1, N, S + n1, N, 1.0);
    }
  }

  // execute one batch (leader thread, no lock held); rethrows on failure
  void run(const std::vector<BatchReq *> &reqs) {
    std::vector<int64_t> key;
    for (BatchReq *r : reqs) {
      key.push_back(r->slot);
      key.push_back(r->k);
      key.push_back((int64_t)(uintptr_t)r->X);
      key.push_back((int64_t)(uintptr_t)r->S);
    }
    for (BatchReq *r : reqs) {
      adc_ctx *c = ctx[r->slot];
      if (!c->tc || !c->tc->ready) {
        // built on the problem's own stream, whose thread waits for this batch
        tc_ensure(c);
        ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
      }
    }
    auto &pp = plans[key];
    if (!pp) pp.reset(new Plan());
    Plan &pl = *pp;
    ADC_CUDA(cudaEventRecord(e0, bex.stream));
    if (use_graphs && pl.uses >= 1 && !pl.exec) {
      // second occurrence: capture what the first one enqueued (all sizes are known now)
      cudaGraph_t g = nullptr;
      ADC_CUDA(cudaStreamBeginCapture(bex.stream, cudaStreamCaptureModeThreadLocal));
      try {
        enqueue(reqs, pl.grp, false);
      } catch (...) {
        cudaStreamEndCapture(bex.stream, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      ADC_CUDA(cudaStreamEndCapture(bex.stream, &g));
      cudaError_t e = cudaGraphInstantiate(&pl.exec, g, 0);
      cudaGraphDestroy(g);
      ADC_CUDA(e);
      info.graphs_captured++;
    }
    if (pl.exec && use_graphs) {
      ADC_CUDA(cudaGraphLaunch(pl.exec, bex.stream));
      info.graph_launches++;
    } else {
      enqueue(reqs, pl.exec ? pl.direct : pl.grp, true);
      info.direct_launches++;
    }
    pl.uses++;
    ADC_CUDA(cudaEventRecord(e1, bex.stream));
    int h = 0;
    ADC_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, bex.stream));
    ADC_CUDA(cudaStreamSynchronize(bex.stream));
    float ms = 0.f;
    ADC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (grouped_timed) {
      float gm = 0.f;
      ADC_CUDA(cudaEventElapsedTime(&gm, g0, g1));
      info.grouped_ms += gm;
      info.grouped_flops += pl.grp.flops;
      info.grouped_launches++;
      grouped_timed = false;
    }
    info.batches++;
    for (BatchReq *r : reqs) info.sigma_vectors += r->k;
    info.batch_ms += ms;
    info.tc_flops += pl.grp.flops;
    if (plans.size() > 256) plans.clear();  // many distinct batches: start over
    if (h != 0) {
      fill_zero(bex, err.p, sizeof(int));
      throw Error(ADC_ERR_TIMEOUT, "tensor-core GEMM wait gave up (code " + std::to_string(h) + ")");
    }
  }

  // leader loop: run the pending batch while every running problem waits in it
  void lead(std::unique_lock<std::mutex> &lk) {
    while (!pending.empty() && (int)pending.size() >= active) {
      std::vector<BatchReq *> reqs;
      reqs.swap(pending);
      lk.unlock();
      int rc = 0;
      std::string msg;
      try {
        run(reqs);
      } catch (const Error &e) {
        rc = e.code;
        msg = e.what();
      } catch (const std::exception &e) {
        rc = ADC_ERR_CUDA;
        msg = e.what();
      }
      lk.lock();
      for (BatchReq *r : reqs) {
        r->rc = rc;
        r->msg = msg;
        r->done = true;
      }
      cv.notify_all();
    }
  }

  // a problem's thread: sigma of its block through the next batch
  void submit(BatchReq &r) {
    std::unique_lock<std::mutex> lk(mu);
    pending.push_back(&r);
    lead(lk);
    cv.wait(lk, [&] { return r.done; });
    if (r.rc != 0) throw Error(r.rc, r.msg);
  }
  // a problem leaves the batch for a while (FP64 work) or for good
  void leave() {
    std::unique_lock<std::mutex> lk(mu);
    --active;
    lead(lk);
  }
  void rejoin() {
    std::lock_guard<std::mutex> lk(mu);
    ++active;
  }
};

void batch_submit(adc_ctx *c, const cplx *X, cplx *S, int64_t k) {
  ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
  BatchReq r;
  r.slot = c->batch_slot;
  r.X = X;
  r.S = S;
  r.k = k;
  c->batch->submit(r);
}
void batch_leave(adc_ctx *c) { c->batch->leave(); }
void batch_rejoin(adc_ctx *c) { c->batch->rejoin(); }

}  // namespace adc

using namespace adc;

struct adc_batch {
  std::unique_ptr<BatchCoord> co;
  std::string err;
};

namespace {

thread_local std::string g_batch_error;

int bfail(adc_batch *b, const std::string &m, int code) {
  if (b) b->err = m;
  g_batch_error = m;
  return code;
}

bool is_dev(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// device bytes a context of this problem holds after adc_init, plus its
// split-precision copies (and, with the sliced refinement, the digit slices
// of the same operators: about five times the split copies), a Davidson run
// with nroots (subspace max(8 nroots, 40)) and the batched-sigma scratch
int64_t mem_estimate(const adc_problem &p, int nroots, bool sliced = false) {
  const int64_t o = p.nocc, v = p.nvir, Q = p.naux, nmo = o + v;
  const int64_t pv = v * (v - 1) / 2, po = o * (o - 1) / 2;
  int64_t n1, n2;
  if (p.kind == ADC_IP) { n1 = o; n2 = po * v; }
  else if (p.kind == ADC_EA) { n1 = v; n2 = o * pv; }
  else { n1 = o * v; n2 = po * pv; }
  const int64_t N = n1 + n2;
  const bool sat = (p.order == 3 && p.x != 0.0);
  int64_t b = 16 * Q * nmo * nmo;               // B
  b += 16 * (o * o * v * v) * 2;                // t1, ring W
  b += 16 * n1 * n2 + 16 * n1 * n1 + 24 * N;    // coupling, main block, diagonals
  const int64_t P = (p.kind == ADC_EA) ? pv : po;
  if (p.kind != ADC_EE) {
    if (sat) b += 16 * P * P;                   // packed ladder integrals
    int64_t split = 4 * (n1 * 2 * ((n2 + 63) / 64 * 64) + n2 * 2 * ((n1 + 63) / 64 * 64));  // Cpl, CplT
    if (sat) split += 4 * (P * 2 * ((P + 63) / 64 * 64) + o * v * 2 * ((o * v + 63) / 64 * 64));
    b += split + (sliced ? 5 * split : 0);
  }
  const int64_t m = std::max<int64_t>(8 * nroots, 40);
  b += 32 * m * N + 16 * 6 * nroots * N;        // V, AV, Davidson work vectors
  b += 16 * nroots * N * 3;                     // batched-sigma scratch
  b += 16 * (o * v) * (o * v) * 2;              // setup intermediates (peak)
  return b;
}

// setup and sigma work in complex MACs (the dominant terms)
double cost_estimate(const adc_problem &p, int nroots) {
  const double o = (double)p.nocc, v = (double)p.nvir, Q = (double)p.naux;
  const double pv = v * (v - 1) / 2, po = o * (o - 1) / 2;
  double c = 0.0;
  if (p.order == 3) c += 2 * Q * pv * pv + po * pv * pv;
  if (p.kind == ADC_EA) c += v * v * v * v * o * o + Q * v * v * v * o;
  else if (p.kind == ADC_IP) c += Q * o * o * o * v + o * o * o * o * v * v;
  else c += o * o * v * v * v * v;
  const double n2 = p.kind == ADC_IP ? po * v : (p.kind == ADC_EA ? o * pv : po * pv);
  c += 50.0 * nroots * n2 * (p.kind == ADC_EA ? pv : o * v) / 64.0;  // mixed sigma share
  return c;
}

}  // namespace

extern "C" {

int adc_batch_create(adc_batch **out, adc_ctx *const *ctxs, int n) {
  if (!out) return ADC_ERR_ARG;
  *out = nullptr;
  if (!ctxs || n < 1) return bfail(nullptr, "adc_batch_create: need at least one context", ADC_ERR_ARG);
  adc_batch *b = new adc_batch();
  try {
    b->co.reset(new BatchCoord());
    BatchCoord &co = *b->co;
    ADC_CUDA(cudaGetDevice(&co.dev));
    for (int i = 0; i < n; ++i) {
      ADC_REQUIRE(ctxs[i] != nullptr, ADC_ERR_ARG, "adc_batch_create: NULL context");
      ADC_REQUIRE(ctxs[i]->batch == nullptr, ADC_ERR_STATE, "adc_batch_create: context already in a batch");
      for (int j = 0; j < i; ++j) ADC_REQUIRE(ctxs[j] != ctxs[i], ADC_ERR_ARG, "adc_batch_create: repeated context");
      ADC_REQUIRE(!(ctxs[i]->kind == ADC_EA && ctxs[i]->direct_ladder), ADC_ERR_UNSUPPORTED,
                  "adc_batch_create: contexts with the integral-direct ladder are solved one at a time");
      co.ctx.push_back(ctxs[i]);
    }
    co.scr.resize(n);
    ADC_CUDA(cudaStreamCreateWithFlags(&co.bex.stream, cudaStreamNonBlocking));
    ADC_CUDA(cudaEventCreate(&co.e0));
    ADC_CUDA(cudaEventCreate(&co.e1));
    ADC_CUDA(cudaEventCreate(&co.g0));
    ADC_CUDA(cudaEventCreate(&co.g1));
    co.err = DBuf(co.bex, sizeof(int));
    fill_zero(co.bex, co.err.p, sizeof(int));
    ADC_CUDA(cudaStreamSynchronize(co.bex.stream));
    *out = b;
    return ADC_OK;
  } catch (const Error &e) {
    delete b;
    return bfail(nullptr, e.what(), e.code);
  } catch (const std::exception &e) {
    delete b;
    return bfail(nullptr, e.what(), ADC_ERR_CUDA);
  }
}

int adc_batch_sigma(adc_batch *b, const adc_c128 *const *X, adc_c128 *const *S, const int64_t *k, int precision) {
  if (!b || !b->co) return ADC_ERR_STATE;
  BatchCoord &co = *b->co;
  const int n = (int)co.ctx.size();
  if (!X || !S || !k) return bfail(b, "adc_batch_sigma: NULL argument", ADC_ERR_ARG);
  try {
    std::vector<BatchReq> reqs(n);
    std::vector<BatchReq *> rp;
    for (int i = 0; i < n; ++i) {
      ADC_REQUIRE(k[i] >= 0, ADC_ERR_ARG, "adc_batch_sigma: negative block size");
      if (k[i] == 0) continue;
      ADC_REQUIRE(is_dev(X[i]) && is_dev(S[i]), ADC_ERR_ARG, "adc_batch_sigma: X and S must be device pointers");
      reqs[i].slot = i;
      reqs[i].X = (const cplx *)X[i];
      reqs[i].S = (cplx *)S[i];
      reqs[i].k = k[i];
      rp.push_back(&reqs[i]);
    }
    // the inputs may come from any stream of the caller
    ADC_CUDA(cudaDeviceSynchronize());
    if (precision == ADC_PREC_FP64) {
      for (BatchReq *r : rp) {
        adc_ctx *c = co.ctx[r->slot];
        sigma(c, r->X, r->S, r->k, ADC_PREC_FP64);
        ADC_CUDA(cudaStreamSynchronize(c->ex.stream));
      }
      return ADC_OK;
    }
    ADC_REQUIRE(precision == ADC_PREC_BF16X3, ADC_ERR_ARG, "adc_batch_sigma: unknown precision");
    for (BatchReq *r : rp)
      ADC_REQUIRE(co.ctx[r->slot]->kind != ADC_EE, ADC_ERR_UNSUPPORTED,
                  "adc_batch_sigma: EE-ADC runs FP64 sigma products only");
    if (rp.empty()) return ADC_OK;
    std::lock_guard<std::mutex> lk(co.mu);
    co.run(rp);
    return ADC_OK;
  } catch (const Error &e) {
    return bfail(b, e.what(), e.code);
  } catch (const std::exception &e) {
    return bfail(b, e.what(), ADC_ERR_CUDA);
  }
}

int adc_batch_davidson(adc_batch *b, int nroots, double tol, int max_iter, int precision, double *omega,
                       double *err64, int *status, adc_stats *st) {
  if (!b || !b->co) return ADC_ERR_STATE;
  BatchCoord &co = *b->co;
  const int n = (int)co.ctx.size();
  if (!omega || !err64 || !status || nroots < 1) return bfail(b, "adc_batch_davidson: bad arguments", ADC_ERR_ARG);
  for (int i = 0; i < n; ++i) {
    if (co.ctx[i]->kind == ADC_EE && precision != ADC_PREC_FP64)
      return bfail(b, "adc_batch_davidson: EE-ADC runs FP64 sigma products only", ADC_ERR_UNSUPPORTED);
    if (nroots > co.ctx[i]->N) return bfail(b, "adc_batch_davidson: nroots larger than a problem", ADC_ERR_ARG);
  }
  {
    std::lock_guard<std::mutex> lk(co.mu);
    co.active = n;
    co.pending.clear();
  }
  for (int i = 0; i < n; ++i) {
    co.ctx[i]->batch = (precision == ADC_PREC_FP64) ? nullptr : &co;
    co.ctx[i]->batch_slot = i;
  }
  std::vector<std::thread> th;
  std::vector<std::string> msgs(n);
  for (int i = 0; i < n; ++i) {
    th.emplace_back([&, i]() {
      int rc = ADC_OK;
      cudaSetDevice(co.dev);
      adc_ctx *c = co.ctx[i];
      try {
        rc = davidson_run(c, nroots, tol, max_iter, precision, nullptr, 0, omega + (int64_t)i * nroots, nullptr,
                          err64 + (int64_t)i * nroots, st ? st + i : nullptr);
      } catch (const Error &e) {
        rc = e.code;
        msgs[i] = e.what();
      } catch (const std::exception &e) {
        rc = ADC_ERR_CUDA;
        msgs[i] = e.what();
      }
      status[i] = rc;
      co.leave();
    });
  }
  for (auto &t : th) t.join();
  for (int i = 0; i < n; ++i) {
    co.ctx[i]->batch = nullptr;
    co.ctx[i]->batch_slot = -1;
  }
  int worst = ADC_OK;
  for (int i = 0; i < n; ++i)
    if (status[i] != ADC_OK && status[i] != ADC_ERR_NOCONV) {
      worst = status[i];
      b->err = "problem " + std::to_string(i) + ": " + msgs[i];
    }
  if (worst == ADC_OK)
    for (int i = 0; i < n; ++i)
      if (status[i] == ADC_ERR_NOCONV) worst = ADC_ERR_NOCONV;
  return worst;
}

int adc_batch_use_graphs(adc_batch *b, int on) {
  if (!b || !b->co) return ADC_ERR_STATE;
  std::lock_guard<std::mutex> lk(b->co->mu);
  b->co->use_graphs = (on != 0);
  return ADC_OK;
}

int adc_batch_info_get(const adc_batch *b, adc_batch_info *info) {
  if (!b || !b->co || !info) return ADC_ERR_ARG;
  *info = b->co->info;
  info->tuned_shapes = tc_autotune_table(nullptr, 0);
  return ADC_OK;
}

void adc_batch_free(adc_batch *b) {
  if (!b) return;
  if (b->co)
    for (adc_ctx *c : b->co->ctx)
      if (c->batch == b->co.get()) c->batch = nullptr;
  delete b;
}

const char *adc_batch_last_error(const adc_batch *b) {
  if (b && !b->err.empty()) return b->err.c_str();
  return g_batch_error.c_str();
}

static int plan_waves(int n, const adc_problem *p, int nroots, int64_t mem_budget, int *order, int *wave,
                      int64_t *mem_est, double *cost_est, bool sliced);

int adc_batch_plan(int n, const adc_problem *p, int nroots, int64_t mem_budget, int *order, int *wave,
                   int64_t *mem_est, double *cost_est) {
  return plan_waves(n, p, nroots, mem_budget, order, wave, mem_est, cost_est, false);
}

static int plan_waves(int n, const adc_problem *p, int nroots, int64_t mem_budget, int *order, int *wave,
                      int64_t *mem_est, double *cost_est, bool sliced) {
  if (n < 0 || (n > 0 && (!p || !order || !wave)) || nroots < 1 || mem_budget <= 0) return ADC_ERR_ARG;
  std::vector<int64_t> mem(n);
  std::vector<double> cost(n);
  for (int i = 0; i < n; ++i) {
    if (p[i].nocc < 1 || p[i].nvir < 1 || p[i].naux < 1) return ADC_ERR_ARG;
    if (p[i].kind != ADC_IP && p[i].kind != ADC_EA && p[i].kind != ADC_EE) return ADC_ERR_ARG;
    mem[i] = mem_estimate(p[i], nroots, sliced);
    cost[i] = cost_estimate(p[i], nroots);
    if (mem_est) mem_est[i] = mem[i];
    if (cost_est) cost_est[i] = cost[i];
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  // first fit in cost order: each problem joins the earliest wave with room
  std::vector<int64_t> used;
  for (int t = 0; t < n; ++t) {
    const int i = idx[t];
    order[t] = i;
    int w = 0;
    while (w < (int)used.size() && used[w] + mem[i] > mem_budget) ++w;
    if (w == (int)used.size()) used.push_back(0);
    used[w] += mem[i];
    wave[i] = w;
  }
  return (int)used.size();
}

int adc_batch_solve(int n, const adc_problem *p, int nroots, double tol, int max_iter, int precision,
                    const adc_batch_opts *bo, double *omega, double *err64, int *status, adc_batch_info *info) {
  if (n < 1 || !p || !omega || !err64 || !status) return bfail(nullptr, "adc_batch_solve: bad arguments", ADC_ERR_ARG);
  adc_batch_opts o{};
  if (bo) o = *bo;
  const int lanes = o.init_lanes > 0 ? o.init_lanes : 4;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return bfail(nullptr, "adc_batch_solve: no device", ADC_ERR_CUDA);
  int64_t budget = o.mem_budget;
  if (budget <= 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return bfail(nullptr, "adc_batch_solve: cudaMemGetInfo", ADC_ERR_CUDA);
    budget = (int64_t)(0.85 * (double)fr);
  }
  std::vector<int> order(n), wave(n);
  int nw = plan_waves(n, p, nroots, budget, order.data(), wave.data(), nullptr, nullptr, o.refine == ADC_PREC_SLICED);
  if (nw < 0) return bfail(nullptr, "adc_batch_solve: invalid problem sizes", nw);
  adc_batch_info acc{};
  int worst = ADC_OK;
  for (int i = 0; i < n; ++i) status[i] = ADC_ERR_STATE;
  for (int w = 0; w < nw; ++w) {
    std::vector<int> ids;
    for (int t = 0; t < n; ++t)
      if (wave[order[t]] == w) ids.push_back(order[t]);
    std::vector<adc_ctx *> ctxs(ids.size(), nullptr);
    std::vector<int> irc(ids.size(), ADC_OK);
    // initialise the wave on a few lanes, largest problems first
    const double t0 = now_s();
    std::atomic<int> next{0};
    std::vector<std::thread> th;
    for (int l = 0; l < std::min<int>(lanes, (int)ids.size()); ++l) {
      th.emplace_back([&]() {
        cudaSetDevice(dev);
        for (;;) {
          const int j = next.fetch_add(1);
          if (j >= (int)ids.size()) break;
          const adc_problem &q = p[ids[j]];
          adc_opts op;
          adc_opts_default(&op);
          op.setup = o.setup;
          op.refine = o.refine;
          irc[j] = adc_init(&ctxs[j], q.B, q.naux, q.eps_occ, q.nocc, q.eps_vir, q.nvir, q.kind, q.order, q.x, &op);
          if (irc[j] == ADC_OK) irc[j] = adc_sync(ctxs[j]);
        }
      });
    }
    for (auto &t : th) t.join();
    acc.init_s += now_s() - t0;
    std::vector<adc_ctx *> ok;
    std::vector<int> okid;
    for (size_t j = 0; j < ids.size(); ++j) {
      if (irc[j] == ADC_OK) { ok.push_back(ctxs[j]); okid.push_back(ids[j]); }
      else { status[ids[j]] = irc[j]; worst = irc[j]; }
    }
    if (!ok.empty()) {
      adc_batch *b = nullptr;
      int rc = adc_batch_create(&b, ok.data(), (int)ok.size());
      if (rc == ADC_OK) {
        std::vector<double> om(ok.size() * nroots), e6(ok.size() * nroots);
        std::vector<int> sts(ok.size());
        const double t1 = now_s();
        rc = adc_batch_davidson(b, nroots, tol, max_iter, precision, om.data(), e6.data(), sts.data(), nullptr);
        acc.solve_s += now_s() - t1;
        for (size_t j = 0; j < ok.size(); ++j) {
          status[okid[j]] = sts[j];
          for (int r = 0; r < nroots; ++r) {
            omega[(int64_t)okid[j] * nroots + r] = om[j * nroots + r];
            err64[(int64_t)okid[j] * nroots + r] = e6[j * nroots + r];
          }
        }
        adc_batch_info bi{};
        adc_batch_info_get(b, &bi);
        acc.batches += bi.batches;
        acc.graph_launches += bi.graph_launches;
        acc.graphs_captured += bi.graphs_captured;
        acc.direct_launches += bi.direct_launches;
        acc.sigma_vectors += bi.sigma_vectors;
        acc.batch_ms += bi.batch_ms;
        acc.tc_flops += bi.tc_flops;
        acc.tuned_shapes = bi.tuned_shapes;
        acc.grouped_launches += bi.grouped_launches;
        acc.grouped_ms += bi.grouped_ms;
        acc.grouped_flops += bi.grouped_flops;
        adc_batch_free(b);
      } else {
        for (int id : okid) status[id] = rc;
      }
      if (rc != ADC_OK && worst == ADC_OK) worst = rc;
    }
    for (adc_ctx *c : ctxs)
      if (c) adc_free(c);
    acc.waves++;
  }
  if (info) *info = acc;
  return worst;
}

}  // extern "C"
