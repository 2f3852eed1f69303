// device_common.cuh -- small device helpers shared by the kernels of libbg.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bg {

// A light-like reference vector passed to kernels by value.
struct Q4 {
  double v[4];
};

// Minkowski product, metric (+,-,-,-), written as a chain of fused
// multiply-adds: x0 y0 - x1 y1 - x2 y2 - x3 y3.
template <typename T>
__device__ __forceinline__ T mdot(const T* x, const T* y) {
  T r = x[0] * y[0];
  r = fma(-x[1], y[1], r);
  r = fma(-x[2], y[2], r);
  r = fma(-x[3], y[3], r);
  return r;
}

template <typename T>
__device__ __forceinline__ T recip(T x) {
  return T(1) / x;
}

// Status codes written to the device status word by kernels that meet an
// invalid label (the first code wins).
__device__ __forceinline__ void flag_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Light-cone-gauge polarisation pair for one gluon, FP64 (Eq. 2.7 with the
// projector of Eq. 2.2).  k: outgoing momentum (any overall scale);
// q: reference vector (q0 > 0, light-like).  Gauge frame a, b: x^ and y^
// rotated by the rotation taking z^ to q_vec/|q_vec| (for a negative z
// component: a(-n), -b(-n)); if k is parallel to q, q -> (q0, -q_vec).
__device__ __forceinline__ void lc_polarisations(const double k[4], const double qin[4], double e1[4],
                                                 double e2[4]) {
  double q[4] = {qin[0], qin[1], qin[2], qin[3]};
  double kq = k[0] * q[0] - k[1] * q[1] - k[2] * q[2] - k[3] * q[3];
  if (fabs(kq) <= 1e-9 * fabs(k[0]) * q[0]) {
    q[1] = -q[1];
    q[2] = -q[2];
    q[3] = -q[3];
    kq = k[0] * q[0] - k[1] * q[1] - k[2] * q[2] - k[3] * q[3];
  }
  const double inv_qn = 1.0 / sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double nx = q[1] * inv_qn, ny = q[2] * inv_qn, nz = q[3] * inv_qn;
  double sb = 1.0;
  if (nz < 0.0) {
    nx = -nx;
    ny = -ny;
    nz = -nz;
    sb = -1.0;
  }
  const double h = 1.0 / (1.0 + nz);
  const double a1 = 1.0 - nx * nx * h, a2 = -nx * ny * h, a3 = -nx;
  const double b1 = sb * (-nx * ny * h), b2 = sb * (1.0 - ny * ny * h), b3 = sb * (-ny);
  // A.k and B.k with A = (0, a): A.k = -(a . k_vec)
  const double inv_kq = 1.0 / kq;
  const double ca = -(a1 * k[1] + a2 * k[2] + a3 * k[3]) * inv_kq;
  const double cb = -(b1 * k[1] + b2 * k[2] + b3 * k[3]) * inv_kq;
  e1[0] = -ca * q[0];
  e1[1] = a1 - ca * q[1];
  e1[2] = a2 - ca * q[2];
  e1[3] = a3 - ca * q[3];
  e2[0] = -cb * q[0];
  e2[1] = b1 - cb * q[1];
  e2[2] = b2 - cb * q[2];
  e2[3] = b3 - cb * q[3];
}

}  // namespace bg
