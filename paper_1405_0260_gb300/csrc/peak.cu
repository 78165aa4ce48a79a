// Arithmetic-peak microbenchmark: the float32 and float64 fused multiply-add
// rates of the SIMT pipes (no tensor cores).  The paper has no counterpart;
// the library's float-float and float64 kernels are bound by these pipes, and
// their roofline denominators come from here.  Each thread runs 8 independent
// FMA chains (enough to cover the pipe latency) for `iters` steps; every chain
// ends in a store, so nothing is folded away.
#include <cuda_runtime.h>

#include "../../include/paro.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T a, T b, T* out) {
  T x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < 8; ++c) x[c] = x[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int paro_peak_fma(int dtype, int iters, void* out, double* tflops, void* cuda_stream) {
  if ((dtype != PARO_F64 && dtype != PARO_F32) || iters < 1 || !out || !tflops) return PARO_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PARO_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int threads = 256, blocks = sms * 8;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PARO_ERR_CUDA;
  float ms = 0.f;
  bool ok = true;
  for (int rep = 0; rep < 2 && ok; ++rep) {  // the second run is timed
    ok = cudaEventRecord(e0, st) == cudaSuccess;
    if (dtype == PARO_F32)
      k_fma_chains<float><<<blocks, threads, 0, st>>>(iters, 0.999f, 1e-4f, static_cast<float*>(out));
    else
      k_fma_chains<double><<<blocks, threads, 0, st>>>(iters, 0.999, 1e-4, static_cast<double*>(out));
    ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, st) == cudaSuccess &&
         cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok || ms <= 0.f) return PARO_ERR_CUDA;
  const double flops = 2.0 * 8.0 * 16.0 * (double)iters * threads * blocks;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return PARO_OK;
}
