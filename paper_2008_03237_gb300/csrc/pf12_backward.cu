// Host side of the adjoint: variant dispatch (device code: pf12_backward.cuh,
// one translation unit per variant under csrc/inst/) and the deterministic
// gather-mode scatter of per-pair gradients into the per-orbital blocks.
#include <cuda_runtime.h>

#include "pf12_internal.h"

namespace pf12 {

// Adjoint variants: 0 / 1 = MINB 2 / 3 CTAs per SM (chosen by the tuner at the
// first pf12_backward).
cudaError_t launch_backward(const BwdParams& prm, int precision, int variant, int n_ctas,
                            cudaStream_t s) {
  if (precision == 0) return variant == 1 ? launch_bwd_f64_3(prm, n_ctas, s) : launch_bwd_f64_2(prm, n_ctas, s);
  return variant == 1 ? launch_bwd_f32_3(prm, n_ctas, s) : launch_bwd_f32_2(prm, n_ctas, s);
}

int backward_blocks_per_sm(int precision, int variant) {
  if (precision == 0) return variant == 1 ? occupancy_bwd_f64_3() : occupancy_bwd_f64_2();
  return variant == 1 ? occupancy_bwd_f32_3() : occupancy_bwd_f32_2();
}

// Deterministic scatter of per-pair factor gradients into the per-orbital
// blocks: CTA o walks its (pair, side) list in pair order; within one entry the
// row and column maps are strictly increasing, so no two threads touch the
// same element, and a barrier separates consecutive entries.
__global__ void __launch_bounds__(kThreads) scatter_kernel(
    const double* dAgi, const double* dAgj, const double* dAfi, const double* dAfj,
    const PairDesc* desc_by_pair, const GatherDesc* gdesc, const int32_t* map_pao,
    const int32_t* map_aux, const int64_t* orb_ptr, const int32_t* orb_list, const int64_t* off_orb,
    const int32_t* ld_orb, double* dBg, double* dBf) {
  const int o = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ld = ld_orb[o];
  double* bg = dBg + off_orb[o];
  double* bf = dBf + off_orb[o];
  for (int64_t q = orb_ptr[o]; q < orb_ptr[o + 1]; ++q) {
    const int32_t entry = orb_list[q];
    const int32_t P = entry >> 1, side = entry & 1;
    const PairDesc pd = desc_by_pair[P];
    const GatherDesc g = gdesc[P];
    const int p = pd.p, m = pd.m;
    const int32_t* rows = map_pao + g.map_pao + (int64_t)side * p;
    const int32_t* cols = map_aux + g.map_aux + (int64_t)side * m;
    const double* sg = (side ? dAgj : dAgi) + pd.off_pm;
    const double* sf = (side ? dAfj : dAfi) + pd.off_pm;
    for (int r = warp; r < p; r += kThreads / 32) {
      const int64_t rb = (int64_t)rows[r] * ld;
      for (int c = lane; c < m; c += 32) {
        bg[rb + cols[c]] += sg[(int64_t)r * m + c];
        bf[rb + cols[c]] += sf[(int64_t)r * m + c];
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_scatter(const double* dAgi, const double* dAgj, const double* dAfi,
                           const double* dAfj, const PairDesc* desc_by_pair, const GatherDesc* gdesc,
                           const int32_t* map_pao, const int32_t* map_aux, const int64_t* orb_ptr,
                           const int32_t* orb_list, const int64_t* off_orb, const int32_t* ld_orb,
                           int32_t n_orb, double* dBg, double* dBf, cudaStream_t s) {
  if (n_orb <= 0) return cudaSuccess;
  scatter_kernel<<<n_orb, kThreads, 0, s>>>(dAgi, dAgj, dAfi, dAfj, desc_by_pair, gdesc, map_pao,
                                            map_aux, orb_ptr, orb_list, off_orb, ld_orb, dBg, dBf);
  return cudaGetLastError();
}

}  // namespace pf12
