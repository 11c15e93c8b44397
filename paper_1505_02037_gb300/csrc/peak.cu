// Measured FP64 arithmetic rate of the current device. The FP64 lattice
// Boltzmann step is bound by the FP64 pipe rather than by HBM, so its
// roofline needs the rate that pipe actually sustains: this file times a
// kernel of independent fused multiply-add chains held in registers, at
// full occupancy, with CUDA events.
#include <cuda_runtime.h>

#include "../../include/lbnr.h"
#include "dispatch.h"

namespace {

constexpr int kChains = 8;    // independent chains per thread
constexpr int kBlock = 256;
constexpr int kIters = 4096;  // multiply-adds per chain

__global__ void __launch_bounds__(kBlock) k_fma64(double* sink, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-9 * threadIdx.x + c;
#pragma unroll 4
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  double s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0) sink[blockIdx.x] = s;  // never true; keeps the chains live
}

}  // namespace

extern "C" int lbnr_fp64_fma_rate(void* cuda_stream, double* tflops) {
  using namespace lbnr;
  if (!tflops) {
    set_thread_error("null output");
    return LBNR_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma64, kBlock, 0);
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  float best = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) {
      k_fma64<<<grid, kBlock, 0, st>>>(nullptr, 0.9999999, 1e-7);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;  // first: warm-up
  }
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  if (e != cudaSuccess) {
    set_thread_error(cudaGetErrorString(e));
    return LBNR_ECUDA;
  }
  const double flops = 2.0 * kChains * (double)kIters * (double)grid * kBlock;
  *tflops = flops / (best * 1e-3) / 1e12;
  return LBNR_OK;
}
