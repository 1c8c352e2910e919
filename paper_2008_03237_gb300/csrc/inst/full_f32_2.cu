// Complete pair-energy kernel, FP32-class products, 2 CTAs per SM.
// One kernel variant per translation unit, so that the variants compile in
// parallel.
#include "../pf12_full.cuh"

namespace pf12 {

cudaError_t launch_full_f32_2(const FullParams& prm, int n_ctas, cudaStream_t s) {
  pair_full_kernel<float, 2><<<n_ctas, kThreads, 0, s>>>(prm);
  return cudaGetLastError();
}

int occupancy_full_f32_2() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_full_kernel<float, 2>, kThreads, 0);
  return n;
}

}  // namespace pf12
