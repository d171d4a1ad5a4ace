// Arithmetic peak probe: the FP32 (FFMA) and FP64 (DFMA) issue rates of this
// GPU, measured rather than derived from unit counts, as the denominators of
// the MAP-LM kernel's "fraction of FP32 peak" and of the float64 cost the
// 4x4 solve would have.  Every thread advances CH independent multiply-add
// chains x <- x a + b, so no instruction waits on the previous one's result;
// the grid fills every SM several times over.  The caller times the launch
// with CUDA events on its stream.

#include "kcs_internal.cuh"

namespace kcs {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_CHAINS = 16;

template <class T>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_peak(int iters, T a, T b, T* sink) {
  T x[PEAK_CHAINS];
#pragma unroll
  for (int i = 0; i < PEAK_CHAINS; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; ++i) x[i] = fma(x[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < PEAK_CHAINS; ++i) s += x[i];
  // a store the compiler cannot prove dead; never taken for the caller's a, b
  if (s == (T)-1) sink[blockIdx.x] = s;
}

}  // namespace kcs

using namespace kcs;

extern "C" int kcs_fma_peak_launch(int precision, int blocks, int iters, double* flops,
                                   void* sink, void* stream) {
  clear_error();
  KCS_REQUIRE(precision == 32 || precision == 64, "precision %d must be 32 or 64", precision);
  KCS_REQUIRE(blocks > 0 && iters > 0, "blocks and iters must be positive");
  KCS_REQUIRE(flops && sink, "NULL argument");
  cudaStream_t s = as_stream(stream);
  // x <- x a + b with |a| < 1 converges to b / (1 - a) ~ 1: no overflow, no subnormals
  if (precision == 32)
    k_fma_peak<float><<<blocks, PEAK_THREADS, 0, s>>>(iters, 0.9999999f, 1e-7f,
                                                      static_cast<float*>(sink));
  else
    k_fma_peak<double><<<blocks, PEAK_THREADS, 0, s>>>(iters, 0.999999999, 1e-9,
                                                       static_cast<double*>(sink));
  KCS_LAUNCHED();
  *flops = 2.0 * PEAK_CHAINS * (double)iters * (double)blocks * PEAK_THREADS;
  return KCS_OK;
}
