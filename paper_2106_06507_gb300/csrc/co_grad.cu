// co_grad.cu -- FP32 and FP64 instantiations of the reverse-mode recursion.
#include "co_grad.cuh"

namespace bg {
cudaError_t launch_co_grad_f32(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                               const float* Y, double* kbar, double* ebar, int* status, cudaStream_t s) {
  return launch_co_grad_t<float>(n, B, sqrt_s, p, hel, q, Y, kbar, ebar, status, s);
}
cudaError_t launch_co_grad_f64(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                               const double* Y, double* kbar, double* ebar, int* status, cudaStream_t s) {
  return launch_co_grad_t<double>(n, B, sqrt_s, p, hel, q, Y, kbar, ebar, status, s);
}
}  // namespace bg
