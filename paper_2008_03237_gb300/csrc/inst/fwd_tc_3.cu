// Forward pair kernel with the tcgen05 split-TF32 contractions, 3 CTAs per SM.
// One kernel variant per translation unit, so that the variants compile in
// parallel.
#include <algorithm>

#define PF12_FORWARD_TC
#include "../pf12_forward.cuh"

namespace pf12 {

static cudaError_t tc_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(pair_forward_tc_kernel<3>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  // prefer the largest shared-memory carveout so that three 66 KB CTAs fit per SM
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pair_forward_tc_kernel<3>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess) done = true;
  return e;
}

cudaError_t launch_fwd_tc_3(const FwdParams& prm, int n_ctas, cudaStream_t s) {
  cudaError_t e = tc_attr();
  if (e != cudaSuccess) return e;
  pair_forward_tc_kernel<3><<<n_ctas, kThreads, kTcSmem, s>>>(prm);
  return cudaGetLastError();
}

int occupancy_fwd_tc_3() {
  if (tc_attr() != cudaSuccess) return 0;
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_forward_tc_kernel<3>, kThreads, kTcSmem);
  // resource model (registers, shared memory with the per-CTA reserve,
  // threads); the runtime's answer for this dynamic-smem kernel can be lower
  cudaFuncAttributes fa{};
  int dev = 0, smem_sm = 0, regs_sm = 0, thr_sm = 0, reserve = 0;
  if (cudaFuncGetAttributes(&fa, pair_forward_tc_kernel<3>) == cudaSuccess &&
      cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&reserve, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess) {
    const int by_regs = regs_sm / std::max(1, fa.numRegs * kThreads);
    const int by_smem = smem_sm / (int)(fa.sharedSizeBytes + kTcSmem + reserve);
    const int by_thr = thr_sm / kThreads;
    n = std::max(n, std::min(by_regs, std::min(by_smem, by_thr)));
  }
  return std::min(n, 4);  // 4 x 128 TMEM columns per SM at most
}

}  // namespace pf12
