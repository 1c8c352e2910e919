// Complete pair-energy kernel, FP64 products, 3 CTAs per SM.
// One kernel variant per translation unit, so that the variants compile in
// parallel.
#include "../pf12_full.cuh"

namespace pf12 {

cudaError_t launch_full_f64_3(const FullParams& prm, int n_ctas, cudaStream_t s) {
  pair_full_kernel<double, 3><<<n_ctas, kThreads, 0, s>>>(prm);
  return cudaGetLastError();
}

int occupancy_full_f64_3() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_full_kernel<double, 3>, kThreads, 0);
  return n;
}

}  // namespace pf12
