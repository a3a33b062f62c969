// FP64 fused multiply-add throughput of the device, the denominator of the
// FP64 path's arithmetic roofline (the FP64 units of this GPU are few, so
// the plain FP64 path is bounded by them rather than by HBM).
//
// Every thread runs kChains independent FMA chains a <- a * b + c for
// `iters` iterations (b, c are kernel arguments, so nothing folds at compile
// time) and stores the sum of its chains, so no chain is dead code.  The grid
// is a multiple of the SM count with enough warps per SM to cover the FMA
// latency.  FLOPs per launch = 2 x threads x iters x kChains.
#include <cuda_runtime.h>

#include "llg.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma64_kernel(double b, double c, int iters, double* out) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * (size_t)kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" llg_status llg_fp64_fma_rate(int iters, double* tflops, double* ms, void* cuda_stream) {
  if (!tflops || iters < 1) return LLG_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LLG_ECUDA;
  const int blocks = sms * 8;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * (size_t)blocks * kThreads) != cudaSuccess) return LLG_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  llg_status rc = LLG_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = LLG_ECUDA;
  float best = 0.f;
  // b slightly below 1 keeps every chain bounded: a -> c / (1 - b)
  for (int rep = 0; rc == LLG_OK && rep < 6; ++rep) {
    cudaEventRecord(e0, st);
    fma64_kernel<<<blocks, kThreads, 0, st>>>(0.999999, 1e-7, iters, out);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      rc = LLG_ECUDA;
      break;
    }
    float f = 0.f;
    cudaEventElapsedTime(&f, e0, e1);
    if (rep >= 2 && (best == 0.f || f < best)) best = f;   // first two launches warm up
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc != LLG_OK) return rc;
  const double flops = 2.0 * (double)blocks * kThreads * (double)iters * kChains;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms) *ms = best;
  return LLG_OK;
}
