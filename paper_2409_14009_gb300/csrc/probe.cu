// probe.cu -- measured FP64 throughput of this GPU, the denominator the
// binary64 factorization is compared with (its dense updates are DFMA-bound).
//
// DFMA: every thread runs ACC independent chains of fused multiply-adds (one
// dependent FMA per chain per iteration). DMMA: every warp issues mma.sync
// m8n8k4 f64 (512 flops each) on ACC independent accumulator tiles. Both are
// tried with 8 and 16 chains and 2, 4 and 6 CTAs of 256 threads per SM; the
// best shape is the measured peak. Flops = 2 per FMA (the convention of the
// factorization's flop count).
#include <cuda_runtime.h>

#include "device.h"

namespace {

constexpr int kIters = 4096;

template <int kAcc>
__global__ void __launch_bounds__(256) k_probe_dfma(double* out, double seed) {
  double a[kAcc];
#pragma unroll
  for (int i = 0; i < kAcc; ++i) a[i] = seed + i + threadIdx.x;
  const double m = 1.0 - 1e-12, c = 1e-9;
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int i = 0; i < kAcc; ++i) a[i] = fma(a[i], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kAcc; ++i) s += a[i];
  if (s == 12345.678) out[0] = s;   // keeps the chains alive; never true for these inputs
}

template <int kAcc>
__global__ void __launch_bounds__(256) k_probe_dmma(double* out, double seed) {
  double acc[kAcc][2];
#pragma unroll
  for (int i = 0; i < kAcc; ++i) acc[i][0] = acc[i][1] = 0.0;
  const double a = seed + threadIdx.x * 1e-3, b = 1.0 - 1e-12;
  for (int it = 0; it < kIters / 4; ++it) {
#pragma unroll
    for (int i = 0; i < kAcc; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(acc[i][0]), "+d"(acc[i][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kAcc; ++i) s += acc[i][0] + acc[i][1];
  if (s == 12345.678) out[0] = s;
}

}  // namespace

extern "C" int chol_probe_fp64(int32_t kind, int32_t reps, double* gflops, void* stream) {
  if (kind != 0 && kind != 1) return -1;
  if (reps < 1) return -2;
  if (!gflops) return -3;
  int dev = 0, sms = 0;
  CHOL_CUDA_TRY(cudaGetDevice(&dev));
  CHOL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = (cudaStream_t)stream;
  double* out = nullptr;
  CHOL_CUDA_TRY(cudaMalloc(&out, sizeof(double)));
  cudaEvent_t e0, e1;
  CHOL_CUDA_TRY(cudaEventCreate(&e0));
  CHOL_CUDA_TRY(cudaEventCreate(&e1));
  double best_rate = 0.0;
  int rc = CHOL_OK;
  for (int acc : {8, 16}) {
    for (int per_sm : {2, 4, 6}) {
      const int grid = per_sm * sms;
      float best = 1e30f;
      for (int r = 0; r < reps + 1 && rc == CHOL_OK; ++r) {   // the first run is a warm-up
        cudaEventRecord(e0, st);
        if (kind == 0 && acc == 8) k_probe_dfma<8><<<grid, 256, 0, st>>>(out, 1.0 + r);
        if (kind == 0 && acc == 16) k_probe_dfma<16><<<grid, 256, 0, st>>>(out, 1.0 + r);
        if (kind == 1 && acc == 8) k_probe_dmma<8><<<grid, 256, 0, st>>>(out, 1.0 + r);
        if (kind == 1 && acc == 16) k_probe_dmma<16><<<grid, 256, 0, st>>>(out, 1.0 + r);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = CHOL_ECUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) best = ms < best ? ms : best;
      }
      if (rc != CHOL_OK) break;
      if (cudaGetLastError() != cudaSuccess) { rc = CHOL_ECUDA; break; }
      const double threads = (double)grid * 256.0;
      const double flops = kind == 0 ? threads * kIters * acc * 2.0
                                     : (threads / 32.0) * (kIters / 4) * acc * 512.0;
      const double rate = flops / (best * 1e-3) / 1e9;
      best_rate = rate > best_rate ? rate : best_rate;
    }
  }
  *gflops = rc == CHOL_OK ? best_rate : 0.0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}
