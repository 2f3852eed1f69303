// co_tensor.cu -- FP32 and FP64 instantiations of the colour-ordered
// recursion in the tensor form (auxiliary tensor field, Eqs. 2.23-2.26).
#include "co_recursion.cuh"

namespace bg {
cudaError_t launch_co_tensor_f32(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel,
                                 const double* q, float* amps, int* status, cudaStream_t s) {
  return launch_co_tensor_t<float>(n, B, sqrt_s, p, hel, q, amps, status, s);
}
cudaError_t launch_co_tensor_f64(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel,
                                 const double* q, double* amps, int* status, cudaStream_t s) {
  return launch_co_tensor_t<double>(n, B, sqrt_s, p, hel, q, amps, status, s);
}
}  // namespace bg
