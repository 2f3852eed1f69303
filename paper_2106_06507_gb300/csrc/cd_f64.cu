// cd_f64.cu -- FP64 instantiations of the colour-dressed recursion.
#include "cd_recursion.cuh"

namespace bg {
size_t cd_workspace_bytes_f64(int n, int sms) { return cd_workspace_bytes_t<double>(n, sms); }
cudaError_t launch_cd_f64(int n, const CdParams& prm, const double* p, const int8_t* hel, const int8_t* col,
                          const uint8_t* accept, double* me2, void* workspace, int* status, int sms, cudaStream_t s,
                          int variant) {
  if (variant < 0) variant = tune_variant(kTuneCD, n, BG_F64);
  return launch_cd_t<double>(n, prm, p, hel, col, accept, me2, workspace, status, sms, s, variant);
}
}  // namespace bg
