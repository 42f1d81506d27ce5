// Shared definitions of the GB300 ADC library (host and device).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/adc_gb300.h"

namespace adc {

typedef double2 cplx;  // interleaved (re, im), the layout of adc_c128

// Error carried from deep inside the setup code to the ABI boundary, where it
// becomes a negative return code. Nothing below the boundary aborts.
struct Error : public std::runtime_error {
  int code;
  Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define ADC_CUDA(call)                                                           \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess)                                                       \
      throw ::adc::Error(ADC_ERR_CUDA, std::string(#call) + ": " +              \
                                           cudaGetErrorString(e_) + " at " +     \
                                           __FILE__ + ":" + std::to_string(__LINE__)); \
  } while (0)

// every kernel launch site calls ADC_CHECK_LAUNCH(), which also counts it
extern long long g_launches;
#define ADC_CHECK_LAUNCH()                               \
  do {                                                   \
    __atomic_add_fetch(&::adc::g_launches, 1, __ATOMIC_RELAXED); \
    ADC_CUDA(cudaGetLastError());                        \
  } while (0)

#define ADC_REQUIRE(cond, code, msg)                 \
  do {                                               \
    if (!(cond)) throw ::adc::Error((code), (msg));  \
  } while (0)

__host__ __device__ inline cplx cmake(double r, double i) { return make_double2(r, i); }
__host__ __device__ inline cplx cadd(cplx a, cplx b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline cplx csub(cplx a, cplx b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline cplx cmul(cplx a, cplx b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline cplx cconj(cplx a) { return make_double2(a.x, -a.y); }
__host__ __device__ inline cplx cscale(cplx a, double s) { return make_double2(a.x * s, a.y * s); }
// acc += a * b
__host__ __device__ inline void cfma(cplx &acc, cplx a, cplx b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// index of the pair (p < q) among the n(n-1)/2 pairs, row-major upper triangle
__host__ __device__ inline int64_t pair_index(int64_t p, int64_t q, int64_t n) {
  return p * n - p * (p + 1) / 2 + (q - p - 1);
}

inline int64_t npairs(int64_t n) { return n * (n - 1) / 2; }

inline unsigned grid1d(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > (int64_t)1 << 30) b = (int64_t)1 << 30;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace adc
