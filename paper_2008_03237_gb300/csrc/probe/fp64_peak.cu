// FP64 FMA-pipe throughput probe: the denominator of the fused pair kernels'
// roofline, measured on the device the benchmark runs on.  Every thread runs
// kChains independent FMA chains (enough independent work to keep the FP64
// pipe busy at any occupancy), the grid fills every SM several times over,
// and the device time comes from CUDA events around the launch.  Algorithmic
// flops: 2 per FMA.  Built into its own small library (libpf12probe.so); it
// is a measurement tool, not part of the pair-F12 path.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) dfma_chains(double* out, int iters, double x, double y) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  out[blockIdx.x * kThreads + threadIdx.x] = s;   // keeps every chain live
}

}  // namespace

// Measures the sustained FP64 FMA rate of the current device.
//   iters: FMA iterations per chain (the launch runs ~iters * 8 us at 1.2 TFLOP/s)
//   tflops (host, out): 2 * FMAs / device time, in TFLOP/s
//   ms (host, out): device time of the timed launch
// A warm-up launch precedes the timed one.  Returns 0, or a CUDA error code.
extern "C" int pf12probe_fp64_fma(int iters, double* tflops, double* ms) {
  int dev = 0, n_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  const int blocks = n_sm * 8;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&out, sizeof(double) * blocks * kThreads);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    dfma_chains<<<blocks, kThreads>>>(out, iters / 8 + 1, 0.999999, 1e-7);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0);
  if (e == cudaSuccess) {
    dfma_chains<<<blocks, kThreads>>>(out, iters, 0.999999, 1e-7);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e == cudaSuccess) {
    *ms = t;
    *tflops = 2.0 * kChains * (double)iters * blocks * kThreads / (t * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  return (int)e;
}
