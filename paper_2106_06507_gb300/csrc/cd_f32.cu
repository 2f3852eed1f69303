// cd_f32.cu -- FP32 instantiations of the colour-dressed recursion.
#include "cd_recursion.cuh"

namespace bg {
size_t cd_workspace_bytes_f32(int n, int sms) { return cd_workspace_bytes_t<float>(n, sms); }
int cd_variants(int n) { return (n >= 4 && n <= 12) ? cd_num_variants(n) : 0; }
cudaError_t launch_cd_f32(int n, const CdParams& prm, const double* p, const int8_t* hel, const int8_t* col,
                          const uint8_t* accept, double* me2, void* workspace, int* status, int sms, cudaStream_t s,
                          int variant) {
  if (variant < 0) variant = tune_variant(kTuneCD, n, BG_F32);
  return launch_cd_t<float>(n, prm, p, hel, col, accept, me2, workspace, status, sms, s, variant);
}
}  // namespace bg
