// co_f32.cu -- FP32 instantiations of the colour-ordered recursion.
#include "co_recursion.cuh"

namespace bg {
cudaError_t launch_co_f32(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                          float* amps, int* status, cudaStream_t s, const int64_t* dB) {
  return launch_co_t<float>(n, B, sqrt_s, p, hel, q, amps, status, s, dB);
}
}  // namespace bg
