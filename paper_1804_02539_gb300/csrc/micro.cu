// FP64 throughput probes of this GPU, the denominators of the FP64 roofline fractions:
// dependent chains of FP64 FMAs on the FP64 pipe (kind 0) and FP64 tensor-core MMAs
// mma.sync m8n8k4 (kind 1), each thread running 8 independent chains so that the pipes, not
// the latencies, bound the rate.  Not a step of the method.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/igamg.h"

namespace {

constexpr int kChains = 8;

__global__ void k_dfma_rate(int64_t iters, double seed, double* out) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3 * c + 1e-6 * threadIdx.x;
  const double m = 0.999999, d = 1e-7;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, d);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.678) out[blockIdx.x] = s;  // keeps the chains live; never true in practice
}

__global__ void k_dmma_rate(int64_t iters, double seed, double* out) {
  // per warp: kChains independent 8x8x4 FP64 accumulations D += A B (A, B fixed)
  double acc[kChains][2];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c][0] = acc[c][1] = seed * (c + 1);
  const double a = 1e-3 * (threadIdx.x & 31), b = 1e-3;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(acc[c][0]), "+d"(acc[c][1]) : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c][0] + acc[c][1];
  if (s == 12345.678) out[blockIdx.x] = s;
}

}  // namespace

extern "C" igamg_status igamg_micro_fp64(int kind, int64_t iters, double* tflops, int* sm_count) {
  if (kind < 0 || kind > 1 || iters < 1 || !tflops) return IGAMG_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return IGAMG_ERR_CUDA;
  const int blocks = sms * 4, threads = 256;
  double* out = nullptr;
  if (cudaMalloc(&out, blocks * sizeof(double)) != cudaSuccess) return IGAMG_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto run = [&](int64_t n) {
    if (kind == 0) k_dfma_rate<<<blocks, threads>>>(n, 0.5, out);
    else k_dmma_rate<<<blocks, threads>>>(n, 0.5, out);
  };
  run(iters / 10 + 1);  // warm-up
  cudaEventRecord(e0);
  run(iters);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return IGAMG_ERR_CUDA;
  // FLOPs: an FMA is 2; an m8n8k4 MMA is 2 * 8 * 8 * 4 per warp
  const double per_iter = kind == 0 ? 2.0 * kChains * double(blocks) * threads
                                    : 2.0 * 8 * 8 * 4 * kChains * double(blocks) * threads / 32;
  *tflops = per_iter * double(iters) / (ms * 1e-3) / 1e12;
  if (sm_count) *sm_count = sms;
  return IGAMG_OK;
}
