// Measured FP64 rate of the CUDA cores (the pipe the FP64 chi0 kernel runs on): a plain loop of
// independent fused multiply-adds, timed with CUDA events.  Instrumentation for the roofline of
// the FP64 form; no part of the response path.
#include "lrt_internal.h"

namespace lrt {
namespace {

constexpr int kChains = 8;   // independent FMA chains per thread (hides the FMA latency)

__global__ void __launch_bounds__(256) dfma_loop(double seed, int iters, double* __restrict__ sink) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x * 1e-9 + c;
  const double x = 0.999999999, y = 1e-12;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.678) sink[blockIdx.x] = s;   // never true; keeps the loop alive
}

}  // namespace
}  // namespace lrt

using namespace lrt;

// FP64 FMA throughput of `device` in TFLOP/s (2 flops per FMA), best of 5 timed launches.
extern "C" lrt_status lrtddft_measure_fp64(int device, double* tflops) {
  if (!tflops) {
    set_error("NULL argument");
    return LRT_EINVAL;
  }
  LRT_CUDA(cudaSetDevice(device));
  int nsm = 0;
  LRT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device));
  double* sink = nullptr;
  LRT_CUDA(cudaMalloc(&sink, 64 * (size_t)nsm * sizeof(double)));
  cudaEvent_t e0, e1;
  LRT_CUDA(cudaEventCreate(&e0));
  LRT_CUDA(cudaEventCreate(&e1));
  const int blocks = 8 * nsm, threads = 256, iters = 4096;
  dfma_loop<<<blocks, threads>>>(1.0, iters, sink);   // warm-up
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    dfma_loop<<<blocks, threads>>>(1.0 + r, iters, sink);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess) {
    set_error(std::string("FP64 rate probe: ") + cudaGetErrorString(err));
    return LRT_ECUDA;
  }
  const double flops = 2.0 * kChains * (double)iters * blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return LRT_OK;
}
