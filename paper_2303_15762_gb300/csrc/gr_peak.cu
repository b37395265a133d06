// FP32 FMA throughput of the device: the denominator of the traversal
// kernels' ALU roofline.  Not part of the rendering method.
//
// Every thread runs 16 independent fmaf chains (enough instruction-level
// parallelism to cover the FMA latency at any occupancy), the grid holds 64
// warps on every SM, and the launch is timed with CUDA events on the caller's
// stream.  Work = 2 FLOP per fmaf.
#include <cuda_runtime.h>

#include <algorithm>

#include "gr_build.h"

namespace gr {

namespace {

constexpr int kChains = 16;
constexpr int kUnroll = 4;

__global__ void __launch_bounds__(256) k_fma_chains(float* sink, float a, float b, int iters) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // never true for the arguments used; keeps the chains live
  if (s == -1.0f) sink[blockIdx.x] = s;
}

}  // namespace

cudaError_t fma_peak_impl(cudaStream_t st, double* tflops, double* best_ms) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = sms * 8, threads = 256, iters = 16384;
  float* sink = nullptr;
  e = cudaMallocAsync(&sink, sizeof(float) * blocks, st);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.0f;
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {  // one warm-up launch, best of three
    cudaEventRecord(e0, st);
    k_fma_chains<<<blocks, threads, 0, st>>>(sink, 1.0000001f, 1e-7f, iters);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(sink, st);
  if (e != cudaSuccess) return e;
  const double flop = 2.0 * (double)blocks * threads * (double)iters * kUnroll * kChains;
  *tflops = flop / ((double)best * 1e-3) / 1e12;
  *best_ms = best;
  return cudaSuccess;
}

}  // namespace gr
