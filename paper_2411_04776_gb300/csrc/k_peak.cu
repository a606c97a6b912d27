// Arithmetic peak of the device's plain (non-tensor) FMA pipes, measured: the denominators of the
// FP64 / FP32 roofline fractions of the solver kernels.  Every thread runs four independent FMA
// chains (enough independent work to cover the pipe latency), with enough warps on every SM to
// keep each sub-partition's pipe busy; the launch is timed with CUDA events on the caller's
// stream.  On GB300 this form gives the highest FP64 rate of those tried, about 1.19 TFLOP/s near
// 2 GHz (2 FP64 FMAs per clock and SM); twelve chains per thread measured about 1.01.
#include <cuda_runtime.h>

#include "tx_gel.h"
#include "txgel_common.cuh"

namespace txg {

constexpr int PEAK_T = 256;
constexpr int PEAK_CHAINS = 4;

static __device__ double g_peak_sink;  // a result the compiler cannot drop (written only if s < 0)

// x <- a x + b with a = 1 - 100 b formed in the kernel: with both a and b passed as launch
// parameters the same loop measured about 16 % slower in FP64 on GB300 (1.01 against 1.19
// TFLOP/s); the rate of the FMA pipe is the faster one
template <typename T>
__global__ void __launch_bounds__(PEAK_T) k_fma_peak(int iters, T b) {
  T x[PEAK_CHAINS];
#pragma unroll
  for (int k = 0; k < PEAK_CHAINS; ++k) x[k] = T(1e-3) * T(threadIdx.x + k);
  const T a = T(1) - b * T(100);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) x[k] = fma(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < PEAK_CHAINS; ++k) s += x[k];
  if (s < T(0)) g_peak_sink = (double)s;  // never true (positive start, a and b): keeps the chains live
}

}  // namespace txg

using namespace txg;

extern "C" tx_status tx_peak_fma(int32_t bits, int32_t iters, double* flops, double* ms, void* stream) {
  if (iters < 1 || (bits != 64 && bits != 32) || !flops || !ms) return TX_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TX_ERR_CUDA;
  const bool f64 = bits == 64;
  if (f64)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma_peak<double>, PEAK_T, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma_peak<float>, PEAK_T, 0);
  if (occ < 1) occ = 1;
  const int grid = nsm * occ;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return TX_ERR_CUDA;
  }
  cudaEventRecord(e0, st);
  if (f64)
    k_fma_peak<double><<<grid, PEAK_T, 0, st>>>(iters, 1e-9);  // a = 0.9999999
  else
    k_fma_peak<float><<<grid, PEAK_T, 0, st>>>(iters, 1e-6f);  // a = 0.9999
  count_launch(1);
  cudaEventRecord(e1, st);
  float t = 0.f;
  const cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return TX_ERR_CUDA;
  *flops = 2.0 * PEAK_CHAINS * (double)iters * (double)grid * PEAK_T;
  *ms = t;
  return TX_OK;
}
