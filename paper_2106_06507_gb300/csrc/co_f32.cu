// co_f32.cu -- FP32 instantiations of the colour-ordered recursion.
#include "co_recursion.cuh"

namespace bg {
cudaError_t launch_co_f32(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                          float* amps, int* status, cudaStream_t s, const int64_t* dB, int variant) {
  if (variant < 0) variant = tune_variant(kTuneCO, n, BG_F32);
  return launch_co_t<float>(n, B, sqrt_s, p, hel, q, amps, status, s, dB, variant);
}
int co_variants(int n, bool helicity_sum) { return (n >= 4 && n <= 9) ? co_num_variants(n, helicity_sum) : 0; }
}  // namespace bg
