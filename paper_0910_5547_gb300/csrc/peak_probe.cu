// peak_probe.cu -- arithmetic ceilings of the GPU the library runs on, for the
// rooflines of the stage kernels: the FP32 and FP64 fused multiply-add rates of
// the CUDA cores (no tensor cores).  Each thread runs eight independent FMA
// chains, so the pipe, not the dependency latency, limits the rate; the grid
// fills every SM with eight CTAs of 256 threads.  Not part of the method.
#include <cuda_runtime.h>

#include "../../include/amr.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chains(T* sink, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-1.2345) sink[blockIdx.x] = s;   // keeps the chains live; never true for these inputs
}

template <typename T>
double rate(int sms, int iters) {
  T* sink = nullptr;
  const int grid = sms * 8;
  if (cudaMalloc(&sink, grid * sizeof(T)) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // a = 1 - 2^-20 keeps the values bounded and away from denormals
  const T a = (T)(1.0 - 1.0 / 1048576.0), b = (T)0.5;
  fma_chains<T><<<grid, kThreads>>>(sink, iters / 8, a, b);   // warm-up
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0);
    fma_chains<T><<<grid, kThreads>>>(sink, iters, a, b);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (cudaGetLastError() != cudaSuccess) return -1.0;
  const double flops = 2.0 * kChains * (double)iters * grid * kThreads;
  return flops / (best * 1e-3);
}

}  // namespace

extern "C" amr_status amr_peak_fma_rates(double* out) {
  if (!out) return AMR_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return AMR_ERR_CUDA;
  out[0] = rate<float>(sms, 1 << 14);
  out[1] = rate<double>(sms, 1 << 11);
  return (out[0] > 0 && out[1] > 0) ? AMR_OK : AMR_ERR_CUDA;
}
