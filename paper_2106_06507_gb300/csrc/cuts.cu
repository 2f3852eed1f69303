// cuts.cu -- the paper's kinematic constraints on the final-state gluons
// (Sec. 5): pT > pt_min, |eta| < eta_max and Delta R > dr_min for every pair,
// with the pseudorapidity eta = asinh(p_z / p_T), the azimuth phi =
// atan2(p_y, p_x) and Delta R^2 = (Delta eta)^2 + (Delta phi)^2, Delta phi
// taken in [0, pi].  One thread per event, FP64, on the momenta written by
// the Rambo kernel.
#include <cmath>

#include "bg_internal.h"

namespace bg {
namespace {

template <int N>
__global__ void __launch_bounds__(128) cuts_kernel(int64_t B, const double* __restrict__ p, double pt_min,
                                                   double eta_max, double dr_min, uint8_t* __restrict__ accept) {
  constexpr int NOUT = N - 2;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B) return;
  double eta[NOUT], phi[NOUT];
  bool ok = true;
#pragma unroll
  for (int i = 0; i < NOUT; ++i) {
    const double px = p[((int64_t)1 * N + 2 + i) * B + e];
    const double py = p[((int64_t)2 * N + 2 + i) * B + e];
    const double pz = p[((int64_t)3 * N + 2 + i) * B + e];
    const double pt = sqrt(px * px + py * py);
    ok = ok && pt > pt_min;
    eta[i] = asinh(pz / pt);
    phi[i] = atan2(py, px);
    if (eta_max > 0.0) ok = ok && fabs(eta[i]) < eta_max;
  }
  if (dr_min > 0.0) {
    const double dr2 = dr_min * dr_min;
#pragma unroll
    for (int i = 0; i < NOUT; ++i)
#pragma unroll
      for (int j = i + 1; j < NOUT; ++j) {
        double dphi = fabs(phi[i] - phi[j]);
        if (dphi > M_PI) dphi = 2.0 * M_PI - dphi;
        const double deta = eta[i] - eta[j];
        ok = ok && (deta * deta + dphi * dphi > dr2);
      }
  }
  accept[e] = ok ? 1 : 0;
}

template <int N>
cudaError_t launch(int64_t B, const double* p, double pt_min, double eta_max, double dr_min, uint8_t* accept,
                   cudaStream_t s) {
  const int64_t blocks = (B + 127) / 128;
  cuts_kernel<N><<<(unsigned)blocks, 128, 0, s>>>(B, p, pt_min, eta_max, dr_min, accept);
  return cudaGetLastError();
}

}  // namespace
}  // namespace bg

using namespace bg;

extern "C" bg_status bg_apply_cuts(int n, int64_t B, const double* p, double pt_min, double eta_max,
                                   double dr_min, uint8_t* accept, void* stream) {
  if (n < 4 || n > kMaxN) return fail(BG_EINVAL, "bg_apply_cuts: n must be in 4..12");
  if (B < 0) return fail(BG_EINVAL, "bg_apply_cuts: B < 0");
  if (B == 0) return BG_OK;
  if (!p || !accept) return fail(BG_EINVAL, "bg_apply_cuts: NULL p or accept");
  if (reinterpret_cast<uintptr_t>(p) & 7) return fail(BG_EINVAL, "bg_apply_cuts: p must be 8-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  switch (n) {
    case 4: e = launch<4>(B, p, pt_min, eta_max, dr_min, accept, s); break;
    case 5: e = launch<5>(B, p, pt_min, eta_max, dr_min, accept, s); break;
    case 6: e = launch<6>(B, p, pt_min, eta_max, dr_min, accept, s); break;
    case 7: e = launch<7>(B, p, pt_min, eta_max, dr_min, accept, s); break;
    case 8: e = launch<8>(B, p, pt_min, eta_max, dr_min, accept, s); break;
    case 9: e = launch<9>(B, p, pt_min, eta_max, dr_min, accept, s); break;
    case 10: e = launch<10>(B, p, pt_min, eta_max, dr_min, accept, s); break;
    case 11: e = launch<11>(B, p, pt_min, eta_max, dr_min, accept, s); break;
    default: e = launch<12>(B, p, pt_min, eta_max, dr_min, accept, s); break;
  }
  return cuda_check(e, "bg_apply_cuts");
}
