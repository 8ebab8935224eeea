// Arithmetic-peak microbenchmark: the denominator of the fused kernels'
// roofline fraction.  The fused imaging kernel is bound by FP32 arithmetic
// (its FFT is not a dense contraction), and the device's FP32 (and FP64)
// fused multiply-add rates are not among the figures measured for the
// memory copy and the BF16 tensor GEMM, so the library measures them
// itself: a grid of independent FMA chains with enough chains per thread
// to cover the pipe latency, timed by the caller with CUDA events.
// The paper has no counterpart (measurement aid of this implementation).
#include "../../include/epic.h"

#include <cuda_runtime.h>

#include "epic_internal.h"

namespace {

constexpr int kChains = 8;       // independent FMA chains per thread
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_peak_kernel(long long iters, T b, T c, T* sink) {
  T x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = static_cast<T>(threadIdx.x + i);
  for (long long k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], b, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  // never true for the arguments the host passes (b < 1, c > 0): keeps the
  // chains alive without a store per thread
  if (s == static_cast<T>(-1.0)) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" epic_status epic_measure_fma_peak(int fp64, int blocks, long long iters, void* d_sink,
                                             void* cuda_stream, double* flops) {
  if (blocks < 1 || iters < 1 || !d_sink || !flops)
    return static_cast<epic_status>(epic::set_error(EPIC_ERR_INVALID_ARG, "bad peak arguments"));
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (fp64)
    fma_peak_kernel<double><<<blocks, kThreads, 0, s>>>(iters, 0.999999, 1e-7, static_cast<double*>(d_sink));
  else
    fma_peak_kernel<float><<<blocks, kThreads, 0, s>>>(iters, 0.999999f, 1e-7f, static_cast<float*>(d_sink));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return static_cast<epic_status>(epic::set_error(EPIC_ERR_CUDA, cudaGetErrorString(e)));
  *flops = 2.0 * static_cast<double>(blocks) * kThreads * static_cast<double>(iters) * 16.0 * kChains;
  return EPIC_OK;
}
