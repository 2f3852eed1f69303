// grad_rambo.cu -- last stage of the gradient of |M|^2 with respect to the
// Rambo uniforms: from the adjoints of the scaled momenta and polarisation
// vectors (co_grad.cuh) through the light-cone polarisations (Eq. 2.7) and
// through Rambo (Sec. 3) to the 4(n-2) uniforms of each event.  One thread
// per event, FP64.  The Rambo Jacobian is applied in forward mode, one
// uniform at a time (4(n-2) tangent sweeps of the momentum construction);
// the incoming momenta do not depend on the uniforms.
#include "bg_internal.h"
#include "device_common.cuh"

namespace bg {
namespace {

// value + derivative along one direction
struct D1 {
  double v, d;
};
__device__ __forceinline__ D1 mk(double v, double d = 0.0) { return D1{v, d}; }
__device__ __forceinline__ D1 operator+(D1 a, D1 b) { return D1{a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ D1 operator-(D1 a, D1 b) { return D1{a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ D1 operator*(D1 a, D1 b) { return D1{a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ D1 operator/(D1 a, D1 b) {
  const double iv = 1.0 / b.v;
  return D1{a.v * iv, (a.d - a.v * iv * b.d) * iv};
}
__device__ __forceinline__ D1 dsqrt(D1 a) {
  const double s = sqrt(a.v);
  return D1{s, a.d * 0.5 / s};
}
__device__ __forceinline__ D1 dlog(D1 a) { return D1{log(a.v), a.d / a.v}; }

// Rambo final-state momenta and their derivative along uniform `dir`.
template <int N>
__device__ void rambo_tangent(const double* u, double sqrt_s, int dir, D1 (&p)[N - 2][4]) {
  constexpr int NOUT = N - 2;
  D1 q[NOUT][4];
  D1 Q[4] = {mk(0), mk(0), mk(0), mk(0)};
  for (int i = 0; i < NOUT; ++i) {
    const D1 u1 = mk(u[4 * i + 0], dir == 4 * i + 0 ? 1.0 : 0.0);
    const D1 u2 = mk(u[4 * i + 1], dir == 4 * i + 1 ? 1.0 : 0.0);
    const D1 u3 = mk(u[4 * i + 2], dir == 4 * i + 2 ? 1.0 : 0.0);
    const D1 u4 = mk(u[4 * i + 3], dir == 4 * i + 3 ? 1.0 : 0.0);
    const D1 c = mk(2.0) * u1 - mk(1.0);
    double sphi, cphi;
    sincospi(2.0 * u2.v, &sphi, &cphi);
    const double tp = 6.283185307179586477;
    const D1 sp = mk(sphi, tp * cphi * u2.d), cp = mk(cphi, -tp * sphi * u2.d);
    const D1 q0 = mk(0.0) - dlog(u3 * u4);
    const D1 st = dsqrt(mk(1.0) - c * c);
    q[i][0] = q0;
    q[i][1] = q0 * st * cp;
    q[i][2] = q0 * st * sp;
    q[i][3] = q0 * c;
    for (int m = 0; m < 4; ++m) Q[m] = Q[m] + q[i][m];
  }
  const D1 M = dsqrt(Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3]);
  const D1 b[3] = {mk(0.0) - Q[1] / M, mk(0.0) - Q[2] / M, mk(0.0) - Q[3] / M};
  const D1 x = mk(sqrt_s) / M;
  const D1 gamma = Q[0] / M;
  const D1 a = mk(1.0) / (mk(1.0) + gamma);
  for (int i = 0; i < NOUT; ++i) {
    const D1 bq = b[0] * q[i][1] + b[1] * q[i][2] + b[2] * q[i][3];
    p[i][0] = x * (gamma * q[i][0] + bq);
    for (int j = 0; j < 3; ++j) p[i][1 + j] = x * (q[i][1 + j] + b[j] * q[i][0] + a * bq * b[j]);
  }
}

template <int N>
__global__ void __launch_bounds__(128) rambo_grad_kernel(int64_t B, double sqrt_s, const double* __restrict__ u,
                                                         const double* __restrict__ p, const int8_t* __restrict__ hel,
                                                         Q4 qin, const double* __restrict__ kbar,
                                                         const double* __restrict__ ebar, double scale,
                                                         const double* __restrict__ upstream,
                                                         const uint8_t* __restrict__ accept,
                                                         double* __restrict__ grad_u) {
  constexpr int NOUT = N - 2;
  constexpr int DIM = 4 * NOUT;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B) return;
  double* gout = grad_u + e * DIM;
  const bool ok = (accept == nullptr) || (accept[e] != 0);
  const double w = ok ? scale * (upstream ? upstream[e] : 1.0) : 0.0;
  if (w == 0.0) {
    for (int j = 0; j < DIM; ++j) gout[j] = 0.0;
    return;
  }
  const double inv_s = 1.0 / sqrt_s;
  // adjoints of the final-state lab momenta (k_hat = p / sqrt_s for g >= 2)
  double pbar[NOUT][4];
  for (int i = 0; i < NOUT; ++i) {
    const int g = 2 + i;
    double k[4], kb[4], eb[4];
    for (int m = 0; m < 4; ++m) {
      k[m] = p[((int64_t)m * N + g) * B + e] * inv_s;
      kb[m] = kbar[(e * N + g) * 4 + m];
      eb[m] = ebar[(e * N + g) * 4 + m];
    }
    // polarisation e = A - c q, c = (A.k)/(q.k), with the gauge frame and
    // tie-break of the forward construction
    double q[4] = {qin.v[0], qin.v[1], qin.v[2], qin.v[3]};
    double kq = k[0] * q[0] - k[1] * q[1] - k[2] * q[2] - k[3] * q[3];
    if (fabs(kq) <= 1e-9 * fabs(k[0]) * q[0]) {
      q[1] = -q[1];
      q[2] = -q[2];
      q[3] = -q[3];
      kq = k[0] * q[0] - k[1] * q[1] - k[2] * q[2] - k[3] * q[3];
    }
    const double inv_qn = 1.0 / sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double nx = q[1] * inv_qn, ny = q[2] * inv_qn, nz = q[3] * inv_qn, sb = 1.0;
    if (nz < 0.0) {
      nx = -nx;
      ny = -ny;
      nz = -nz;
      sb = -1.0;
    }
    const double h = 1.0 / (1.0 + nz);
    double A[4];
    if (hel[(int64_t)g * B + e] > 0) {
      A[0] = 0.0; A[1] = 1.0 - nx * nx * h; A[2] = -nx * ny * h; A[3] = -nx;
    } else {
      A[0] = 0.0; A[1] = sb * (-nx * ny * h); A[2] = sb * (1.0 - ny * ny * h); A[3] = sb * (-ny);
    }
    const double Ak = -(A[1] * k[1] + A[2] * k[2] + A[3] * k[3]);
    double ebq = 0.0;
    for (int m = 0; m < 4; ++m) ebq += eb[m] * q[m];
    const double g_[4] = {1.0, -1.0, -1.0, -1.0};
    for (int m = 0; m < 4; ++m) {
      const double dc = (g_[m] * A[m] * kq - Ak * g_[m] * q[m]) / (kq * kq);
      kb[m] += -ebq * dc;
      pbar[i][m] = kb[m] * inv_s;
    }
  }
  const double* ue = u + e * DIM;
  for (int dir = 0; dir < DIM; ++dir) {
    D1 pt[NOUT][4];
    rambo_tangent<N>(ue, sqrt_s, dir, pt);
    double s = 0.0;
    for (int i = 0; i < NOUT; ++i)
      for (int m = 0; m < 4; ++m) s += pbar[i][m] * pt[i][m].d;
    gout[dir] = w * s;
  }
}

template <int N>
cudaError_t launch_n(int64_t B, double sqrt_s, const double* u, const double* p, const int8_t* hel, const double* q,
                     const double* kbar, const double* ebar, double scale, const double* upstream,
                     const uint8_t* accept, double* grad_u, cudaStream_t s) {
  Q4 qq;
  for (int m = 0; m < 4; ++m) qq.v[m] = q[m];
  const int threads = 128;
  const int64_t blocks = (B + threads - 1) / threads;
  rambo_grad_kernel<N><<<(unsigned)blocks, threads, 0, s>>>(B, sqrt_s, u, p, hel, qq, kbar, ebar, scale, upstream,
                                                            accept, grad_u);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rambo_grad(int n, int64_t B, double sqrt_s, const double* u, const double* p, const int8_t* hel,
                              const double* q, const double* kbar, const double* ebar, double scale,
                              const double* upstream, const uint8_t* accept, double* grad_u, cudaStream_t s) {
  switch (n) {
    case 4: return launch_n<4>(B, sqrt_s, u, p, hel, q, kbar, ebar, scale, upstream, accept, grad_u, s);
    case 5: return launch_n<5>(B, sqrt_s, u, p, hel, q, kbar, ebar, scale, upstream, accept, grad_u, s);
    case 6: return launch_n<6>(B, sqrt_s, u, p, hel, q, kbar, ebar, scale, upstream, accept, grad_u, s);
    case 7: return launch_n<7>(B, sqrt_s, u, p, hel, q, kbar, ebar, scale, upstream, accept, grad_u, s);
    case 8: return launch_n<8>(B, sqrt_s, u, p, hel, q, kbar, ebar, scale, upstream, accept, grad_u, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bg
