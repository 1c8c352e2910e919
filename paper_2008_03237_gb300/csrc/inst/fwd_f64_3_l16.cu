// Forward pair kernel, FP64 products, 3 CTAs per SM, Cholesky look-ahead
// groups of 16 panels (one deep trailing update per 512 columns).
// One kernel variant per translation unit, so that the variants compile in
// parallel.
#include "../pf12_forward.cuh"

namespace pf12 {

cudaError_t launch_fwd_f64_3_l16(const FwdParams& prm, int n_ctas, cudaStream_t s) {
  pair_forward_kernel<double, 3, 16><<<n_ctas, kThreads, 0, s>>>(prm);
  return cudaGetLastError();
}

int occupancy_fwd_f64_3_l16() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_forward_kernel<double, 3, 16>, kThreads, 0);
  return n;
}

}  // namespace pf12
