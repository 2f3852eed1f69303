// co_f64.cu -- FP64 instantiations of the colour-ordered recursion.
#include "co_recursion.cuh"

namespace bg {
cudaError_t launch_co_f64(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                          double* amps, int* status, cudaStream_t s, const int64_t* dB, int variant) {
  if (variant < 0) variant = tune_variant(kTuneCO, n, BG_F64);
  return launch_co_t<double>(n, B, sqrt_s, p, hel, q, amps, status, s, dB, variant);
}
}  // namespace bg
