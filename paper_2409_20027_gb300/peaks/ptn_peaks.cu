// ptn_peaks.cu -- FMA throughput of the FP32 and FP64 pipes (declared in
// include/ptn_peaks.h): the measured peaks that the benchmark's "alu" roofline divides by.
#include <cuda_runtime.h>

#include "../../include/ptn_peaks.h"

namespace {

constexpr int kChains = 8;    // independent FMA chains per thread (hide the pipe latency)
constexpr int kThreads = 256;

template <class S>
__global__ void __launch_bounds__(kThreads) k_fma(S* out, int iters, S b, S c) {
  S a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) a[k] = S(threadIdx.x + k) * S(1e-3);
#pragma unroll 4
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = fma(a[k], b, c);
  }
  S s = S(0);
#pragma unroll
  for (int k = 0; k < kChains; k++) s += a[k];
  // a store that depends on every chain keeps them live; it never happens for these b, c
  if (s == S(-1)) out[0] = s;
}

template <class S>
int run(int blocks_per_sm, int iters, double* tflops, double* ms_out) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return -(int)e;
  const int grid = sms * blocks_per_sm;
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  S* out = nullptr;  // one element; never written for these b, c (see k_fma)
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(S));
  float ms = 0.0f;
  if (e == cudaSuccess) {
    k_fma<S><<<grid, kThreads>>>(out, iters, S(0.999999), S(1e-6));  // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(a);
  if (e == cudaSuccess) {
    k_fma<S><<<grid, kThreads>>>(out, iters, S(0.999999), S(1e-6));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return -(int)e;
  const double flops = 2.0 * kChains * (double)iters * (double)grid * kThreads;
  if (tflops) *tflops = flops / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return 0;
}

}  // namespace

extern "C" int ptn_peak_fma(int fp64, int blocks_per_sm, int iters, double* tflops, double* ms) {
  if ((fp64 != 0 && fp64 != 1) || blocks_per_sm < 1 || iters < 1) return -1;
  return fp64 ? run<double>(blocks_per_sm, iters, tflops, ms) : run<float>(blocks_per_sm, iters, tflops, ms);
}
