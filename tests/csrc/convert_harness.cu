// Test harness: the product's integer FP64 <-> FP32 conversions
// (pf12_device.cuh) next to the hardware conversions, element by element.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../paper_2008_03237_gb300/csrc/pf12_device.cuh"

using namespace pf12;

__global__ void convert_kernel(const double* x, int64_t n, float* f_int, float* f_hw,
                               const float* y, double* d_int, double* d_hw) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    f_int[i] = f64_to_f32_rne(x[i]);
    f_hw[i] = __double2float_rn(x[i]);
    d_int[i] = f32_to_f64(y[i]);
    d_hw[i] = static_cast<double>(y[i]);
  }
}

extern "C" int convert_harness(const double* x, int64_t n, float* f_int, float* f_hw,
                               const float* y, double* d_int, double* d_hw) {
  if (n <= 0) return 0;
  convert_kernel<<<152, 256>>>(x, n, f_int, f_hw, y, d_int, d_hw);
  cudaError_t e = cudaDeviceSynchronize();
  return (int)e;
}
