// Test harness: runs the product's tcgen05 split-TF32 GEMM (pf12_tc.cuh) on one
// CTA so that tests can compare it with an FP64 product.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../paper_2008_03237_gb300/csrc/pf12_tc.cuh"

using namespace pf12;

__global__ void __launch_bounds__(256) tc_harness_kernel(int M, int N, int K, const double* A,
                                                         int64_t lda, const double* B, int64_t ldb,
                                                         double* Out, int64_t ldo, int ta, int tb,
                                                         double alpha, int accumulate, int* flag) {
  extern __shared__ __align__(1024) unsigned char smem[];
  tc::Stage& st = *reinterpret_cast<tc::Stage*>(smem);
  tc::Ctrl& c = *reinterpret_cast<tc::Ctrl*>(smem + sizeof(tc::Stage));
  int* s_flag = reinterpret_cast<int*>(smem + sizeof(tc::Stage) + sizeof(tc::Ctrl));
  if (threadIdx.x == 0) *s_flag = 0;
  tc::setup(c);
  bool ok;
  if (ta && tb)
    ok = tc::gemm<true, true>(M, N, K, A, lda, B, ldb, Out, ldo, alpha, accumulate, st, c, s_flag);
  else if (ta)
    ok = tc::gemm<true, false>(M, N, K, A, lda, B, ldb, Out, ldo, alpha, accumulate, st, c, s_flag);
  else if (tb)
    ok = tc::gemm<false, true>(M, N, K, A, lda, B, ldb, Out, ldo, alpha, accumulate, st, c, s_flag);
  else
    ok = tc::gemm<false, false>(M, N, K, A, lda, B, ldb, Out, ldo, alpha, accumulate, st, c, s_flag);
  tc::teardown(c);
  if (threadIdx.x == 0) *flag = ok ? 0 : 1;
}

extern "C" int tc_harness(int M, int N, int K, const double* A, int64_t lda, const double* B,
                          int64_t ldb, double* Out, int64_t ldo, int ta, int tb, double alpha,
                          int accumulate, int* flag_dev) {
  const size_t bytes = sizeof(tc::Stage) + sizeof(tc::Ctrl) + 16;
  cudaError_t e = cudaFuncSetAttribute(tc_harness_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return (int)e;
  tc_harness_kernel<<<1, 256, bytes>>>(M, N, K, A, lda, B, ldb, Out, ldo, ta, tb, alpha, accumulate,
                                       flag_dev);
  e = cudaDeviceSynchronize();
  return (int)e;
}
