// FP64 sigma product that allocates no device memory (adc_sigma_noalloc).
//
// Some callers cannot allocate GPU memory while they run: a caller whose
// device memory is entirely owned by another allocator (a framework's caching
// allocator, a serving process with a fixed budget), a caller inside a region
// where cudaMalloc is forbidden or would synchronise the device (a real-time
// loop, a plugin that must not stall its host application), or a caller that
// must not fail halfway with out-of-memory. For them this entry point runs the
// same FP64 sigma product as adc_sigma, with every per-call intermediate (the
// unpacked satellite block, the ring contraction result, split-K partial sums)
// placed in one file-scope __device__ array of fixed size, SCRATCH_BYTES.
// Every GPU that loads the library holds that array until the process exits.
#include "ctx.cuh"

namespace adc {

namespace {
constexpr int64_t SCRATCH_ELEMS = (int64_t)1 << 22;  // complex128 elements = 64 MiB
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double2 g_noalloc_scratch[SCRATCH_ELEMS];

// device address of the array, looked up once per device with that device
// current (in host code the symbol itself is only a host-side stand-in)
cplx *g_scratch_addr[MAX_DEVICES] = {nullptr};

cplx *scratch_address() {
  int dev = 0;
  ADC_CUDA(cudaGetDevice(&dev));
  ADC_REQUIRE(dev >= 0 && dev < MAX_DEVICES, ADC_ERR_UNSUPPORTED, "device ordinal too large");
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      throw Error(ADC_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                                    cudaGetErrorString(e));
    }
    g_scratch_addr[dev] = (cplx *)p;
  }
  return g_scratch_addr[dev];
}

// device that holds p (device or managed memory), -1 for host memory or an unknown pointer
int pointer_device(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? a.device : -1;
}

// profiling (per-kernel CUDA events) stays off for the call and is put back on
// every exit, thrown errors included
struct ProfOff {
  Exec &ex;
  bool prev;
  explicit ProfOff(Exec &e) : ex(e), prev(e.prof) { e.prof = false; }
  ~ProfOff() { ex.prof = prev; }
};
}  // namespace

// Same terms and order as sigma_fp64 (Sec. 2.1 Eqs. 10-12), scratch from the static array.
static void sigma_fp64_noalloc(adc_ctx *c, const cplx *X, cplx *S, int64_t k) {
  Exec &ex = c->ex;
  const int64_t o = c->o, v = c->v, n1 = c->n1, n2 = c->n2, N = c->N;
  const bool sat = (c->order == 3 && c->x != 0.0);
  const double x = sat ? c->x : 0.0;
  const int64_t ring = sat ? (c->kind == ADC_EA ? k * o * v * v : k * o * o * v) : 0;
  const int64_t need = 2 * ring;
  if (need > SCRATCH_ELEMS)
    throw Error(ADC_ERR_ARG, "adc_sigma_noalloc needs " + std::to_string(need * 16) +
                                 " bytes of scratch for this call; the static array holds " +
                                 std::to_string(SCRATCH_ELEMS * 16) + " (use fewer vectors per call)");
  cplx *base = scratch_address();
  cplx *Xf = base, *T = base + ring;
  cplx *ws = base + need;
  const int64_t ws_elems = SCRATCH_ELEMS - need;
  zgemm_ws(ex, k, n1, n1, 1, C1(), X, 0, N, 1, false, c->M11.c(), 0, 1, n1, false, C0(), S, 0, N, 1, ws, ws_elems);
  zgemm_ws(ex, k, n1, n2, 1, C1(), X + n1, 0, N, 1, false, c->Cpl.c(), 0, 1, n2, false, C1(), S, 0, N, 1, ws,
           ws_elems);
  zgemm_ws(ex, k, n2, n1, 1, C1(), X, 0, N, 1, false, c->Cpl.c(), 0, n2, 1, true, C0(), S + n1, 0, N, 1, ws,
           ws_elems);
  diag_mul_add(ex, k, n2, c->d2.d(), X + n1, N, S + n1, N, 1.0);
  if (!sat) return;
  if (c->kind == ADC_EA) {
    const int64_t pv = npairs(v);
    zgemm_ws(ex, o, pv, pv, k, CR(x), X + n1, N, pv, 1, false, c->Glad.c(), 0, 1, pv, false, C1(), S + n1, N, pv, 1,
             ws, ws_elems);
    pair_unpack(ex, X + n1, k, o, N, pv, v, 1, Xf);
    zgemm_ws(ex, o * v, v, o * v, k, C1(), c->W.c(), 0, o * v, 1, false, Xf, o * v * v, v, 1, false, C0(), T,
             o * v * v, v, 1, ws, ws_elems);
    pair_pack(ex, T, o * v * v, v * v, v, 1, 0, 1.0, k, o, v, 1, S + n1, N, pv, CR(-x), C1());
  } else {
    const int64_t po = npairs(o);
    zgemm_ws(ex, po, v, po, k, CR(x), c->Glad.c(), 0, po, 1, false, X + n1, N, v, 1, false, C1(), S + n1, N, v, 1,
             ws, ws_elems);
    pair_unpack(ex, X + n1, k, 1, N, 0, o, v, Xf);
    zgemm_ws(ex, o * v, o, o * v, k, CR(-1.0), c->W.c(), 0, o * v, 1, false, Xf, o * o * v, 1, o * v, false, C0(),
             T, o * v * o, o, 1, ws, ws_elems);
    pair_pack(ex, T, o * v * o, 0, 1, v * o, o, 1.0, k, 1, o, v, S + n1, N, 0, CR(x), C1());
  }
}

}  // namespace adc

using namespace adc;

extern "C" int adc_sigma_noalloc(adc_ctx *c, const adc_c128 *X, adc_c128 *S, int64_t k) {
  if (!c) return ADC_ERR_STATE;
  if (k < 0 || (k > 0 && (!X || !S))) return ADC_ERR_ARG;
  if (k == 0) return ADC_OK;
  try {
    if (c->kind == ADC_EE) throw Error(ADC_ERR_UNSUPPORTED, "adc_sigma_noalloc covers IP and EA");
    if (c->kind == ADC_EA && c->direct_ladder)
      throw Error(ADC_ERR_UNSUPPORTED, "adc_sigma_noalloc needs the stored ladder integrals (opts.ladder)");
    int cur = -1;
    ADC_CUDA(cudaGetDevice(&cur));
    if (cur != c->dev)
      throw Error(ADC_ERR_ARG, "adc_sigma_noalloc: device " + std::to_string(cur) +
                                   " is current, the context lives on device " + std::to_string(c->dev));
    const int dx = pointer_device(X), ds = pointer_device(S);
    if (dx < 0 || ds < 0)
      throw Error(ADC_ERR_ARG, "adc_sigma_noalloc takes device pointers only (a host copy would allocate)");
    if (dx != c->dev || ds != c->dev)
      throw Error(ADC_ERR_ARG, "adc_sigma_noalloc: X is on device " + std::to_string(dx) + ", S on device " +
                                   std::to_string(ds) + ", the context on device " + std::to_string(c->dev));
    ProfOff off(c->ex);  // no event bookkeeping on this path
    sigma_fp64_noalloc(c, (const cplx *)X, (cplx *)S, k);
    return ADC_OK;
  } catch (const Error &e) {
    c->err = e.what();
    return e.code;
  } catch (const std::bad_alloc &e) {
    c->err = e.what();
    return ADC_ERR_OOM;
  } catch (const std::exception &e) {
    c->err = e.what();
    return ADC_ERR_CUDA;
  }
}
