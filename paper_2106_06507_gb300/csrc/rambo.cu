// rambo.cu -- Rambo flat massless phase space (Kleiss, Stirling, Ellis), the
// generator the paper uses (Sec. 3), plus the final-state pT cut of Sec. 5.
// One thread per event, FP64 throughout.
#include "bg_internal.h"
#include "device_common.cuh"

namespace bg {
namespace {

template <int N>
__global__ void __launch_bounds__(128) rambo_kernel(int64_t S, const int64_t* __restrict__ dB, double sqrt_s,
                                                    const double* __restrict__ u, double* __restrict__ p,
                                                    double pt_min, uint8_t* __restrict__ accept) {
  // S: capacity (row stride of p); dB: device-side event count (NULL: S)
  constexpr int NOUT = N - 2;
  constexpr int D = 4 * NOUT;
  const int64_t B = dB ? (*dB < S ? *dB : S) : S;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B) return;
  const double* ue = u + e * D;
  double q[NOUT][4];
  double Q[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < NOUT; ++i) {
    const double c = 2.0 * ue[4 * i + 0] - 1.0;
    const double q0 = -log(ue[4 * i + 2] * ue[4 * i + 3]);
    const double st = sqrt(1.0 - c * c);
    double sphi, cphi;
    sincospi(2.0 * ue[4 * i + 1], &sphi, &cphi);
    q[i][0] = q0;
    q[i][1] = q0 * st * cphi;
    q[i][2] = q0 * st * sphi;
    q[i][3] = q0 * c;
#pragma unroll
    for (int m = 0; m < 4; ++m) Q[m] += q[i][m];
  }
  const double M = sqrt(Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3]);
  const double invM = 1.0 / M;
  const double b[3] = {-Q[1] * invM, -Q[2] * invM, -Q[3] * invM};
  const double x = sqrt_s * invM;
  const double gamma = Q[0] * invM;
  const double a = 1.0 / (1.0 + gamma);
  const double E = 0.5 * sqrt_s;
  // p layout [4][N][B]
  p[(0 * N + 0) * S + e] = E;
  p[(1 * N + 0) * S + e] = 0.0;
  p[(2 * N + 0) * S + e] = 0.0;
  p[(3 * N + 0) * S + e] = E;
  p[(0 * N + 1) * S + e] = E;
  p[(1 * N + 1) * S + e] = 0.0;
  p[(2 * N + 1) * S + e] = 0.0;
  p[(3 * N + 1) * S + e] = -E;
  bool ok = true;
#pragma unroll
  for (int i = 0; i < NOUT; ++i) {
    const double bq = b[0] * q[i][1] + b[1] * q[i][2] + b[2] * q[i][3];
    const double p0 = x * (gamma * q[i][0] + bq);
    const double p1 = x * (q[i][1] + b[0] * q[i][0] + a * bq * b[0]);
    const double p2 = x * (q[i][2] + b[1] * q[i][0] + a * bq * b[1]);
    const double p3 = x * (q[i][3] + b[2] * q[i][0] + a * bq * b[2]);
    p[(0 * N + 2 + i) * S + e] = p0;
    p[(1 * N + 2 + i) * S + e] = p1;
    p[(2 * N + 2 + i) * S + e] = p2;
    p[(3 * N + 2 + i) * S + e] = p3;
    ok = ok && (sqrt(p1 * p1 + p2 * p2) > pt_min);
  }
  if (accept) accept[e] = ok ? 1 : 0;
}

template <int N>
cudaError_t launch(int64_t B, double sqrt_s, const double* u, double* p, double pt_min, uint8_t* accept,
                   cudaStream_t s, const int64_t* dB) {
  const int threads = 128;
  const int64_t blocks = (B + threads - 1) / threads;
  rambo_kernel<N><<<(unsigned)blocks, threads, 0, s>>>(B, dB, sqrt_s, u, p, pt_min, accept);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rambo(int n, int64_t B, double sqrt_s, const double* u, double* p, double pt_min,
                         uint8_t* accept, cudaStream_t s, const int64_t* dB) {
  switch (n) {
    case 4: return launch<4>(B, sqrt_s, u, p, pt_min, accept, s, dB);
    case 5: return launch<5>(B, sqrt_s, u, p, pt_min, accept, s, dB);
    case 6: return launch<6>(B, sqrt_s, u, p, pt_min, accept, s, dB);
    case 7: return launch<7>(B, sqrt_s, u, p, pt_min, accept, s, dB);
    case 8: return launch<8>(B, sqrt_s, u, p, pt_min, accept, s, dB);
    case 9: return launch<9>(B, sqrt_s, u, p, pt_min, accept, s, dB);
    case 10: return launch<10>(B, sqrt_s, u, p, pt_min, accept, s, dB);
    case 11: return launch<11>(B, sqrt_s, u, p, pt_min, accept, s, dB);
    case 12: return launch<12>(B, sqrt_s, u, p, pt_min, accept, s, dB);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bg
