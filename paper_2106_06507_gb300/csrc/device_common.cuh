// device_common.cuh -- small device helpers shared by the kernels of libbg.so.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
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

// (T X)^nu = T^{nu b} X_b and (Y T)^nu = Y_a T^{a nu} for an antisymmetric
// tensor stored as its 6 upper components t01 t02 t03 t12 t13 t23.
template <typename T>
__device__ __forceinline__ void ten_vec_acc(const T* t, const T* X, T* acc) {
  // X_b = g_bb X^b: X_0 = X0, X_i = -Xi
  acc[0] += -t[0] * X[1] - t[1] * X[2] - t[2] * X[3];
  acc[1] += -t[0] * X[0] - t[3] * X[2] - t[4] * X[3];
  acc[2] += -t[1] * X[0] + t[3] * X[1] - t[5] * X[3];
  acc[3] += -t[2] * X[0] + t[4] * X[1] + t[5] * X[2];
}
template <typename T>
__device__ __forceinline__ void vec_ten_acc(const T* Y, const T* t, T* acc) {
  // (Y T)^nu = Y_a T^{a nu} = -(T Y)^nu for antisymmetric T
  acc[0] -= -t[0] * Y[1] - t[1] * Y[2] - t[2] * Y[3];
  acc[1] -= -t[0] * Y[0] - t[3] * Y[2] - t[4] * Y[3];
  acc[2] -= -t[1] * Y[0] + t[3] * Y[1] - t[5] * Y[3];
  acc[3] -= -t[2] * Y[0] + t[4] * Y[1] + t[5] * Y[2];
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

// The gauge frame of lc_polarisations depends only on q: PolFrame holds it,
// computed once on the host, for q (index 0) and for its tie-break partner
// (q0, -q_vec) (index 1), so that each gluon needs two dot products and one
// division.  Same construction as lc_polarisations.
struct PolFrame {
  double q[2][4];
  double a[2][3];
  double b[2][3];
};

inline PolFrame make_pol_frame(const double* qin) {
  PolFrame F;
  for (int f = 0; f < 2; ++f) {
    const double sg = f ? -1.0 : 1.0;
    const double q[4] = {qin[0], sg * qin[1], sg * qin[2], sg * qin[3]};
    for (int m = 0; m < 4; ++m) F.q[f][m] = q[m];
    const double inv_qn = 1.0 / std::sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double nx = q[1] * inv_qn, ny = q[2] * inv_qn, nz = q[3] * inv_qn, sb = 1.0;
    if (nz < 0.0) {
      nx = -nx;
      ny = -ny;
      nz = -nz;
      sb = -1.0;
    }
    const double h = 1.0 / (1.0 + nz);
    F.a[f][0] = 1.0 - nx * nx * h;
    F.a[f][1] = -nx * ny * h;
    F.a[f][2] = -nx;
    F.b[f][0] = sb * (-nx * ny * h);
    F.b[f][1] = sb * (1.0 - ny * ny * h);
    F.b[f][2] = sb * (-ny);
  }
  return F;
}

// e = A - (A.k / q.k) q for A = (0, a) (label +1) or (0, b) (label -1); the
// ratio in the arithmetic of T (the vector is rounded to T anyway).
template <typename T>
__device__ __forceinline__ void lc_polarisation_frame(const double k[4], const PolFrame& F, bool plus, T (&e)[4]) {
  int f = 0;
  double kq = k[0] * F.q[0][0] - k[1] * F.q[0][1] - k[2] * F.q[0][2] - k[3] * F.q[0][3];
  if (fabs(kq) <= 1e-9 * fabs(k[0]) * F.q[0][0]) {
    f = 1;
    kq = k[0] * F.q[1][0] - k[1] * F.q[1][1] - k[2] * F.q[1][2] - k[3] * F.q[1][3];
  }
  const double* A = plus ? F.a[f] : F.b[f];
  const double Ak = -(A[0] * k[1] + A[1] * k[2] + A[2] * k[3]);
  const T c = T(Ak) / T(kq);
  e[0] = -c * T(F.q[f][0]);
#pragma unroll
  for (int i = 0; i < 3; ++i) e[1 + i] = T(A[i]) - c * T(F.q[f][1 + i]);
}

}  // namespace bg
