// comc_f32.cu -- FP32 instantiations of the colour-flow kernel with
// colour-ordered amplitudes.
#include "comc.cuh"

namespace bg {
cudaError_t launch_comc_f32(int n, const ComcParams& prm, const double* p, const int8_t* hel, const int8_t* col,
                            const uint8_t* accept, const double* q, double* me2, void* workspace, int sms, int* status,
                            cudaStream_t s) {
  return launch_comc_t<float>(n, prm, p, hel, col, accept, q, me2, workspace, sms, status, s);
}
}  // namespace bg
