// grad_rambo.cu -- last stage of the gradient of |M|^2 with respect to the
// Rambo uniforms: from the adjoints of the scaled momenta and polarisation
// vectors (co_grad.cuh) through the light-cone polarisations (Eq. 2.7) and
// through Rambo (Sec. 3) to the 4(n-2) uniforms of each event.  One thread
// per event, FP64, one reverse sweep through the Rambo construction; the
// incoming momenta do not depend on the uniforms.
#include "bg_internal.h"
#include "device_common.cuh"

namespace bg {
namespace {

// Reverse mode through Rambo: given the adjoints pbar of the final-state lab
// momenta, accumulate the adjoints of the 4(n-2) uniforms.  Forward:
//   q_i = q0_i (1, st_i cos phi_i, st_i sin phi_i, c_i),  c_i = 2u1 - 1,
//   phi_i = 2 pi u2, q0_i = -log(u3 u4), st_i = sqrt(1 - c_i^2);
//   Q = sum_i q_i, M = sqrt(Q^2), b = -Q_vec/M, x = sqrt_s/M, gamma = Q0/M,
//   a = 1/(1 + gamma);  p_i = x y_i with y0 = gamma q0 + b.q, y_vec = q_vec
//   + b q0 + a (b.q) b.
template <int N>
__device__ void rambo_reverse(const double* u, double sqrt_s, const double (&pbar)[N - 2][4], double* ubar) {
  constexpr int NOUT = N - 2;
  double q[NOUT][4], st[NOUT], cphi[NOUT], sphi[NOUT];
  double Q[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = 0; i < NOUT; ++i) {
    const double c = 2.0 * u[4 * i + 0] - 1.0;
    sincospi(2.0 * u[4 * i + 1], &sphi[i], &cphi[i]);
    const double q0 = -log(u[4 * i + 2] * u[4 * i + 3]);
    st[i] = sqrt(1.0 - c * c);
    q[i][0] = q0;
    q[i][1] = q0 * st[i] * cphi[i];
    q[i][2] = q0 * st[i] * sphi[i];
    q[i][3] = q0 * c;
    for (int m = 0; m < 4; ++m) Q[m] += q[i][m];
  }
  const double M = sqrt(Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3]);
  const double b[3] = {-Q[1] / M, -Q[2] / M, -Q[3] / M};
  const double x = sqrt_s / M;
  const double gamma = Q[0] / M;
  const double a = 1.0 / (1.0 + gamma);
  // adjoints of x, gamma, a, b and of the q_i (direct terms)
  double xbar = 0.0, gbar = 0.0, abar = 0.0, bbar[3] = {0.0, 0.0, 0.0};
  double qbar[NOUT][4];
  for (int i = 0; i < NOUT; ++i) {
    const double bq = b[0] * q[i][1] + b[1] * q[i][2] + b[2] * q[i][3];
    const double y0 = gamma * q[i][0] + bq;
    double yb[4];
    for (int m = 0; m < 4; ++m) yb[m] = x * pbar[i][m];
    xbar += pbar[i][0] * y0;
    double ybb = 0.0;  // sum_k ybar_k b_k
    for (int k = 0; k < 3; ++k) {
      const double yk = q[i][1 + k] + b[k] * q[i][0] + a * bq * b[k];
      xbar += pbar[i][1 + k] * yk;
      ybb += yb[1 + k] * b[k];
    }
    gbar += yb[0] * q[i][0];
    abar += bq * ybb;
    const double bqbar = yb[0] + a * ybb;
    qbar[i][0] = yb[0] * gamma + ybb;
    for (int k = 0; k < 3; ++k) {
      bbar[k] += yb[1 + k] * (q[i][0] + a * bq) + bqbar * q[i][1 + k];
      qbar[i][1 + k] = yb[1 + k] + bqbar * b[k];
    }
  }
  // a = 1/(1+gamma), x = sqrt_s/M, gamma = Q0/M, b = -Q_vec/M, M = sqrt(Q^2)
  gbar += -a * a * abar;
  double Mbar = -xbar * x / M - gbar * gamma / M;
  double Qbar[4] = {gbar / M, 0.0, 0.0, 0.0};
  for (int k = 0; k < 3; ++k) {
    Qbar[1 + k] = -bbar[k] / M;
    Mbar += -bbar[k] * b[k] / M;
  }
  Qbar[0] += Mbar * Q[0] / M;
  for (int k = 0; k < 3; ++k) Qbar[1 + k] += -Mbar * Q[1 + k] / M;
  // Q = sum q_i; then q_i(u)
  const double twopi = 6.283185307179586477;
  for (int i = 0; i < NOUT; ++i) {
    double qb[4];
    for (int m = 0; m < 4; ++m) qb[m] = qbar[i][m] + Qbar[m];
    const double q0 = q[i][0];
    const double c = 2.0 * u[4 * i + 0] - 1.0;
    const double q0bar = qb[0] + qb[1] * st[i] * cphi[i] + qb[2] * st[i] * sphi[i] + qb[3] * c;
    const double stbar = q0 * (qb[1] * cphi[i] + qb[2] * sphi[i]);
    const double cbar = q0 * qb[3] - stbar * c / st[i];
    const double phibar = q0 * st[i] * (-qb[1] * sphi[i] + qb[2] * cphi[i]);
    ubar[4 * i + 0] = 2.0 * cbar;
    ubar[4 * i + 1] = twopi * phibar;
    ubar[4 * i + 2] = -q0bar / u[4 * i + 2];
    ubar[4 * i + 3] = -q0bar / u[4 * i + 3];
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
  double ub[DIM];
  rambo_reverse<N>(u + e * DIM, sqrt_s, pbar, ub);
  for (int j = 0; j < DIM; ++j) gout[j] = w * ub[j];
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
