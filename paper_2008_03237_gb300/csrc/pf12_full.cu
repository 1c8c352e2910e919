// Host side of the complete pair-energy kernel (device code: pf12_full.cuh):
// variant dispatch.
#include <cuda_runtime.h>

#include "pf12_internal.h"

namespace pf12 {

// Variants: 0 / 1 = 2 / 3 CTAs per SM (chosen by the autotuner at the first fit).
cudaError_t launch_full(const FullParams& prm, int precision, int variant, int n_ctas,
                        cudaStream_t s) {
  if (precision == 0) return variant == 1 ? launch_full_f64_3(prm, n_ctas, s) : launch_full_f64_2(prm, n_ctas, s);
  return variant == 1 ? launch_full_f32_3(prm, n_ctas, s) : launch_full_f32_2(prm, n_ctas, s);
}

int full_blocks_per_sm(int precision, int variant) {
  if (precision == 0) return variant == 1 ? occupancy_full_f64_3() : occupancy_full_f64_2();
  return variant == 1 ? occupancy_full_f32_3() : occupancy_full_f32_2();
}

}  // namespace pf12
