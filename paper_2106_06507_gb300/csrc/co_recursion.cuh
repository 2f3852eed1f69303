// co_recursion.cuh -- colour-ordered Berends-Giele currents on the GPU,
// Eqs. (2.20)-(2.22) of the paper, for every ordering sigma in S_{n-2} of
// the adjoint basis, Eq. (2.15).
//
// Work decomposition: one thread per (event, polarisation configuration,
// ordering).  A block takes a tile of EB events chosen so that the
// EB * H * (n-2)! tasks fill whole rounds of the 256 threads.  Per event the
// block first builds, in FP64, the scaled momenta, the polarisation vectors
// (Eq. 2.7) and a table of inverse propagators 1/P(S)^2 for every subset S of
// the first n-1 gluons (from the pair invariants 2 k_a.k_b, so that nearly
// collinear subsets keep full precision), and stores them in shared memory
// in the recursion's arithmetic type T.  Each thread then runs the whole
// recursion of its ordering in registers: the current table J(i..j) is fully
// unrolled at compile time for the given n.
//
// Arithmetic per segment (i..j) of the ordering, with X_s = J(i..s),
// Y_s = J(s+1..j), P = P(i..j) and unit vertex factors (the couplings
// 1/sqrt2 per three-vertex and 1/2 per four-vertex combine to
// (1/sqrt2)^(n-2) per amplitude, applied once at the end):
//   V3 terms (Eq. 2.21): with current conservation P_s.X_s = 0 and
//   Q_s.Y_s = 0 the vertex becomes
//     (X_s.Y_s)(P_s - Q_s) + 2 (P.X_s) Y_s - 2 (P.Y_s) X_s,
//   and sum_s (X_s.Y_s)(P_s - Q_s) = 2 sum_s (X_s.Y_s) S_{s+1}
//                                   - (sum_s X_s.Y_s)(S_i + S_{j+1})
//   with prefix sums S of the ordered momenta.
//   V4 terms (Eq. 2.21): 2(X.Z)Y - (X.Y)Z - (Y.Z)X with X = J(i..s),
//   Y = J(s+1..t), Z = J(t+1..j); the X and Z parts are collected as scalar
//   coefficients of J(i..s) and J(t+1..j) and applied once per split.
//   Propagator: J(i..j) = bracket / P(i..j)^2; the full segment is put on
//   shell and contracted with the last gluon's polarisation (Eq. 2.22).
#pragma once

#include "bg_internal.h"
#include "device_common.cuh"

namespace bg {

__host__ __device__ constexpr int ct_fact(int m) { return m <= 1 ? 1 : m * ct_fact(m - 1); }
__host__ __device__ constexpr int ct_gcd(int a, int b) { return b == 0 ? a : ct_gcd(b, a % b); }

template <int N, bool SUMHEL>
struct CoShape {
  static constexpr int NT = 256;                    // threads per block
  static constexpr int M = N - 1;                   // legs of the off-shell current
  static constexpr int K = ct_fact(N - 2);          // orderings
  static constexpr int H = SUMHEL ? (1 << N) : 1;   // polarisation configurations
  static constexpr int TPE = K * H;                 // tasks per event
  static constexpr int EB0 = NT / ct_gcd(NT, TPE);  // events per block: EB*TPE % NT == 0
  static constexpr int EB = EB0 > 128 ? 128 : EB0;
  static constexpr int NPOL = SUMHEL ? 2 : 1;
  static constexpr int NMASK = 1 << M;
  static constexpr int NPAIR = M * (M - 1) / 2;
};

template <int N, typename T, bool SUMHEL>
struct CoSmem {
  using S = CoShape<N, SUMHEL>;
  static constexpr size_t off_pair = 0;                                                   // double [EB][NPAIR]
  static constexpr size_t off_inv = off_pair + sizeof(double) * S::EB * S::NPAIR;          // T [EB][NMASK]
  static constexpr size_t off_k = off_inv + sizeof(T) * S::EB * S::NMASK;                  // T [EB][N][4]
  static constexpr size_t off_e = off_k + sizeof(T) * S::EB * N * 4;                       // T [EB][NPOL][N][4]
  static constexpr size_t off_ord = off_e + sizeof(T) * S::EB * S::NPOL * N * 4;           // int [K]
  static constexpr size_t off_p2 = (off_ord + sizeof(int) * S::K + 7) & ~size_t(7);       // double [EB][NMASK]
  static constexpr size_t bytes = off_p2 + sizeof(double) * S::EB * S::NMASK;
};

// Inverse propagators 1/P(S)^2 for every subset S of the first M gluons of
// each of the block's EB events, from the FP64 pair invariants 2 k_a.k_b
// (s_pair [EB][M(M-1)/2], a < b lexicographic).  P(S)^2 is built by the
// highest member h of S: P(S)^2 = P(S - h)^2 + sum_{a in S-h} 2 k_a.k_h, in M
// rounds separated by barriers (s_p2 [EB][2^M] FP64).  The full set and the
// single gluons get 0.  Called by all threads of the block.
template <int M, int EB, int NT, typename T>
__device__ __forceinline__ void co_inverse_table(const double* __restrict__ s_pair, double* __restrict__ s_p2,
                                                 T* __restrict__ s_inv, int64_t e0, int64_t B) {
  constexpr int NMASK = 1 << M, NPAIR = M * (M - 1) / 2;
  const int tid = threadIdx.x;
#pragma unroll 1
  for (int h = 0; h < M; ++h) {
    for (int it = tid; it < (EB << h); it += NT) {
      const int el = it >> h, low = it & ((1 << h) - 1);
      if (e0 + el >= B) continue;
      double v = low ? s_p2[el * NMASK + low] : 0.0;
      for (int r = low; r; r &= r - 1) {
        const int a = __ffs(r) - 1;
        v += s_pair[el * NPAIR + a * M - a * (a + 1) / 2 + (h - a - 1)];
      }
      s_p2[el * NMASK + (low | (1 << h))] = v;
    }
    __syncthreads();
  }
  for (int it = tid; it < EB * NMASK; it += NT) {
    const int el = it / NMASK, mask = it % NMASK;
    if (e0 + el >= B) continue;
    s_inv[el * NMASK + mask] =
        (__popc(mask) >= 2 && mask != NMASK - 1) ? T(1) / T(s_p2[el * NMASK + mask]) : T(0);
  }
  __syncthreads();
}

// y[m] = fma(a, x[m], y[m]) for the four components; in FP32 as two packed
// f32x2 FMAs (same per-component arithmetic, half the instructions).
template <typename T>
__device__ __forceinline__ void axpy4(T a, const T (&x)[4], T (&y)[4]) {
#pragma unroll
  for (int m = 0; m < 4; ++m) y[m] = fma(a, x[m], y[m]);
}
template <>
__device__ __forceinline__ void axpy4<float>(float a, const float (&x)[4], float (&y)[4]) {
  unsigned long long aa, x01, x23, y01, y23;
  asm("mov.b64 %0, {%1, %1};" : "=l"(aa) : "f"(a));
  asm("mov.b64 %0, {%1, %2};" : "=l"(x01) : "f"(x[0]), "f"(x[1]));
  asm("mov.b64 %0, {%1, %2};" : "=l"(x23) : "f"(x[2]), "f"(x[3]));
  asm("mov.b64 %0, {%1, %2};" : "=l"(y01) : "f"(y[0]), "f"(y[1]));
  asm("mov.b64 %0, {%1, %2};" : "=l"(y23) : "f"(y[2]), "f"(y[3]));
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(y01) : "l"(aa), "l"(x01));
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(y23) : "l"(aa), "l"(x23));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(y[0]), "=f"(y[1]) : "l"(y01));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(y[2]), "=f"(y[3]) : "l"(y23));
}

// Component-wise helpers of the same shape: z = x + y, z = x - y, z = a x.
template <typename T>
__device__ __forceinline__ void add4(const T (&x)[4], const T (&y)[4], T (&z)[4]) {
#pragma unroll
  for (int m = 0; m < 4; ++m) z[m] = x[m] + y[m];
}
template <typename T>
__device__ __forceinline__ void sub4(const T (&x)[4], const T (&y)[4], T (&z)[4]) {
#pragma unroll
  for (int m = 0; m < 4; ++m) z[m] = x[m] - y[m];
}
template <typename T>
__device__ __forceinline__ void scale4(T a, const T (&x)[4], T (&z)[4]) {
#pragma unroll
  for (int m = 0; m < 4; ++m) z[m] = a * x[m];
}
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk2(unsigned long long r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
template <>
__device__ __forceinline__ void add4<float>(const float (&x)[4], const float (&y)[4], float (&z)[4]) {
  unsigned long long a = pk2(x[0], x[1]), b = pk2(x[2], x[3]);
  asm("add.rn.f32x2 %0, %0, %1;" : "+l"(a) : "l"(pk2(y[0], y[1])));
  asm("add.rn.f32x2 %0, %0, %1;" : "+l"(b) : "l"(pk2(y[2], y[3])));
  upk2(a, z[0], z[1]);
  upk2(b, z[2], z[3]);
}
template <>
__device__ __forceinline__ void sub4<float>(const float (&x)[4], const float (&y)[4], float (&z)[4]) {
  unsigned long long a = pk2(x[0], x[1]), b = pk2(x[2], x[3]);
  asm("sub.rn.f32x2 %0, %0, %1;" : "+l"(a) : "l"(pk2(y[0], y[1])));
  asm("sub.rn.f32x2 %0, %0, %1;" : "+l"(b) : "l"(pk2(y[2], y[3])));
  upk2(a, z[0], z[1]);
  upk2(b, z[2], z[3]);
}
template <>
__device__ __forceinline__ void scale4<float>(float s, const float (&x)[4], float (&z)[4]) {
  unsigned long long a = pk2(x[0], x[1]), b = pk2(x[2], x[3]);
  const unsigned long long ss = pk2(s, s);
  asm("mul.rn.f32x2 %0, %0, %1;" : "+l"(a) : "l"(ss));
  asm("mul.rn.f32x2 %0, %0, %1;" : "+l"(b) : "l"(ss));
  upk2(a, z[0], z[1]);
  upk2(b, z[2], z[3]);
}

// Bracket of segment (i..j) of one ordering (the V3 and V4 sums before the
// propagator); i and j are compile-time after unrolling.  J[a][b] hold the
// currents of the shorter segments, Sp[p] the prefix sums of the ordered
// momenta.  Unit vertex factors.
template <int N, typename T>
__device__ __forceinline__ void co_bracket(const T (&J)[N - 1][N - 1][4], const T (&Sp)[N][4], const int i,
                                           const int j, T (&br)[4]) {
  constexpr int M = N - 1;
  T P2[4];
  sub4(Sp[j + 1], Sp[i], P2);
  scale4(T(2), P2, P2);
  T by[4], W[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) { br[m] = T(0); by[m] = T(0); W[m] = T(0); }
  T sxy = T(0);
  T cX[M], cR[M];
#pragma unroll
  for (int s = i; s < j; ++s) {
    const T xy = mdot(J[i][s], J[s + 1][j]);
    const T px = mdot(P2, J[i][s]);
    const T py = mdot(P2, J[s + 1][j]);
    sxy += xy;
    axpy4(xy, Sp[s + 1], W);
    cX[s] = -py;
    cR[s] = px;
  }
#pragma unroll
  for (int s = i; s < j; ++s) {
#pragma unroll
    for (int t = s + 1; t < j; ++t) {
      const T xz = mdot(J[i][s], J[t + 1][j]);
      const T xy = mdot(J[i][s], J[s + 1][t]);
      const T yz = mdot(J[s + 1][t], J[t + 1][j]);
      cX[s] -= yz;
      cR[t] -= xy;
      axpy4(xz, J[s + 1][t], by);
    }
  }
#pragma unroll
  for (int s = i; s < j; ++s) {
    axpy4(cR[s], J[s + 1][j], br);
    axpy4(cX[s], J[i][s], br);
  }
  // br += 2 (W + by) - sxy (S_i + S_{j+1})
  T t[4], u[4];
  add4(W, by, t);
  add4(Sp[i], Sp[j + 1], u);
  add4(t, t, t);
  axpy4(-sxy, u, t);
  add4(br, t, br);
}

// co_bracket with a cache of the V3 dot products.  D[a][s][t] holds
// J(a..s).J(s+1..t), the dot of segment (a..t) at split s; this call writes
// D[i][s][j] for its splits and reads two of the three dot products of each
// V4 term from earlier segments: J(i..s).J(s+1..t) = D[i][s][t] (segment
// (i..t), shorter) and J(s+1..t).J(t+1..j) = D[s+1][t][j] (segment (s+1..j),
// the same column, evaluated before (i..j) because both the by-length and
// the column-wise orders evaluate it first).  The cached values are the same
// products of the same operands, so the result equals co_bracket's bit for
// bit, with 8 of the 16 multiply-adds of a V4 term removed.
template <int N, typename T>
__device__ __forceinline__ void co_bracket_dc(const T (&J)[N - 1][N - 1][4], const T (&Sp)[N][4],
                                              T (&D)[N - 1][N - 1][N - 1], const int i, const int j, T (&br)[4]) {
  constexpr int M = N - 1;
  T P2[4];
  sub4(Sp[j + 1], Sp[i], P2);
  scale4(T(2), P2, P2);
  T by[4], W[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) { br[m] = T(0); by[m] = T(0); W[m] = T(0); }
  T sxy = T(0);
  T cX[M], cR[M];
#pragma unroll
  for (int s = i; s < j; ++s) {
    const T xy = mdot(J[i][s], J[s + 1][j]);
    D[i][s][j] = xy;
    const T px = mdot(P2, J[i][s]);
    const T py = mdot(P2, J[s + 1][j]);
    sxy += xy;
    axpy4(xy, Sp[s + 1], W);
    cX[s] = -py;
    cR[s] = px;
  }
#pragma unroll
  for (int s = i; s < j; ++s) {
#pragma unroll
    for (int t = s + 1; t < j; ++t) {
      const T xz = mdot(J[i][s], J[t + 1][j]);
      cX[s] -= D[s + 1][t][j];
      cR[t] -= D[i][s][t];
      axpy4(xz, J[s + 1][t], by);
    }
  }
#pragma unroll
  for (int s = i; s < j; ++s) {
    axpy4(cR[s], J[s + 1][j], br);
    axpy4(cX[s], J[i][s], br);
  }
  T t[4], u[4];
  add4(W, by, t);
  add4(Sp[i], Sp[j + 1], u);
  add4(t, t, t);
  axpy4(-sxy, u, t);
  add4(br, t, br);
}

// Recursion for one ordering; J[i][i] hold the external currents in colour
// order, Sp[p] the prefix sums of the ordered momenta, msk[p] the prefix
// subset masks, inv the event's inverse-propagator table, en the last
// gluon's polarisation.  Returns the amplitude with unit vertex factors.
template <int N, typename T>
__device__ __forceinline__ T co_recursion(T (&J)[N - 1][N - 1][4], const T (&Sp)[N][4], const int (&msk)[N],
                                          const T* __restrict__ inv, const T (&en)[4]) {
  constexpr int M = N - 1;
  T amp = T(0);
  T D[M][M][M];
#pragma unroll
  for (int len = 2; len <= M; ++len) {
#pragma unroll
    for (int i = 0; i + len - 1 < M; ++i) {
      const int j = i + len - 1;
      T br[4];
      co_bracket_dc<N, T>(J, Sp, D, i, j, br);
      if (len < M) {
        const T ip = inv[msk[j + 1] ^ msk[i]];
        scale4(ip, br, J[i][j]);
      } else {
        amp = mdot(en, br);
      }
    }
  }
  return amp;
}

// Tensor form of the bracket (Eqs. 2.23-2.26): the four-gluon vertex is
// replaced by the auxiliary antisymmetric tensor field.  With unit vertex
// factors (the paper's 1/sqrt2 at the creation and at the absorption of the
// tensor combine to the 1/2 of the four-vertex, collected with the other
// couplings at the end):
//   T(i..j)  = sum_s J(i..s) ^ J(s+1..j),
//   br(i..j) = sum_s [ V3 terms + T(s+1..j) J(i..s) + J(s+1..j) T(i..s) ],
// with (T X)^nu = T^{nu b} X_b and (Y T)^nu = Y_a T^{a nu}; single gluons
// carry no tensor.  The V3 terms are those of co_bracket.  TT holds the
// tensors of the shorter segments (6 upper components each); the tensor of
// (i..j) is formed only if `need_t` (not for the full current).
template <int N, typename T>
__device__ __forceinline__ void co_bracket_tf(const T (&J)[N - 1][N - 1][4], const T (&TT)[N - 1][N - 1][6],
                                              const T (&Sp)[N][4], const int i, const int j, const bool need_t,
                                              T (&br)[4], T (&tt)[6]) {
  constexpr int M = N - 1;
  T P2[4];
  sub4(Sp[j + 1], Sp[i], P2);
  scale4(T(2), P2, P2);
  T W[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) { br[m] = T(0); W[m] = T(0); }
#pragma unroll
  for (int m = 0; m < 6; ++m) tt[m] = T(0);
  T sxy = T(0);
  T cX[M], cR[M];
#pragma unroll
  for (int s = i; s < j; ++s) {
    const T xy = mdot(J[i][s], J[s + 1][j]);
    const T px = mdot(P2, J[i][s]);
    const T py = mdot(P2, J[s + 1][j]);
    sxy += xy;
    axpy4(xy, Sp[s + 1], W);
    cX[s] = -py;
    cR[s] = px;
  }
#pragma unroll
  for (int s = i; s < j; ++s) {
    axpy4(cR[s], J[s + 1][j], br);
    axpy4(cX[s], J[i][s], br);
    if (s + 1 < j) ten_vec_acc(TT[s + 1][j], J[i][s], br);
    if (s > i) vec_ten_acc(J[s + 1][j], TT[i][s], br);
    if (need_t) {
      const T* X = J[i][s];
      const T* Y = J[s + 1][j];
      tt[0] += X[0] * Y[1] - X[1] * Y[0];
      tt[1] += X[0] * Y[2] - X[2] * Y[0];
      tt[2] += X[0] * Y[3] - X[3] * Y[0];
      tt[3] += X[1] * Y[2] - X[2] * Y[1];
      tt[4] += X[1] * Y[3] - X[3] * Y[1];
      tt[5] += X[2] * Y[3] - X[3] * Y[2];
    }
  }
  T t[4], u[4];
  add4(W, W, t);
  add4(Sp[i], Sp[j + 1], u);
  axpy4(-sxy, u, t);
  add4(br, t, br);
}

// co_recursion with the tensor form of the bracket.
template <int N, typename T>
__device__ __forceinline__ T co_recursion_tf(T (&J)[N - 1][N - 1][4], const T (&Sp)[N][4], const int (&msk)[N],
                                             const T* __restrict__ inv, const T (&en)[4]) {
  constexpr int M = N - 1;
  T TT[M][M][6];
  T amp = T(0);
#pragma unroll
  for (int len = 2; len <= M; ++len) {
#pragma unroll
    for (int i = 0; i + len - 1 < M; ++i) {
      const int j = i + len - 1;
      T br[4], tt[6];
      co_bracket_tf<N, T>(J, TT, Sp, i, j, len < M, br, tt);
      if (len < M) {
        const T ip = inv[msk[j + 1] ^ msk[i]];
        scale4(ip, br, J[i][j]);
#pragma unroll
        for (int m = 0; m < 6; ++m) TT[i][j][m] = tt[m];
      } else {
        amp = mdot(en, br);
      }
    }
  }
  return amp;
}

template <int N, typename T, bool SUMHEL, bool TF = false>
__global__ void __launch_bounds__(256) co_kernel(int64_t S_, const int64_t* __restrict__ dB, double inv_sqrt_s,
                                                 const double* __restrict__ p, const int8_t* __restrict__ hel,
                                                 PolFrame F, T* __restrict__ amps, int* __restrict__ status) {
  // S_: capacity (row stride of p and hel); dB: device-side event count (NULL: S_)
  const int64_t B = dB ? (*dB < S_ ? *dB : S_) : S_;
  using S = CoShape<N, SUMHEL>;
  using L = CoSmem<N, T, SUMHEL>;
  constexpr int M = S::M, K = S::K, H = S::H, EB = S::EB, NPOL = S::NPOL;
  extern __shared__ __align__(16) unsigned char smem[];
  double* s_pair = reinterpret_cast<double*>(smem + L::off_pair);
  T* s_inv = reinterpret_cast<T*>(smem + L::off_inv);
  T* s_k = reinterpret_cast<T*>(smem + L::off_k);
  T* s_e = reinterpret_cast<T*>(smem + L::off_e);
  int* s_ord = reinterpret_cast<int*>(smem + L::off_ord);

  const int64_t e0 = (int64_t)blockIdx.x * EB;
  const int tid = threadIdx.x;
  if (e0 >= B) return;

  // ---- phase 1a: ordering table (packed 4-bit labels), momenta, polarisations
  for (int r = tid; r < K; r += S::NT) {
    int avail = (1 << (N - 2)) - 1;
    int rr = r, packed = 0;
#pragma unroll
    for (int pos = 0; pos < N - 2; ++pos) {
      const int f = ct_fact(N - 3 - pos);
      const int d = rr / f;
      rr -= d * f;
      int lab = 0, cnt = -1;
#pragma unroll
      for (int b = 0; b < N - 2; ++b) {
        const bool on = (avail >> b) & 1;
        cnt += on ? 1 : 0;
        if (on && cnt == d) lab = b;
      }
      avail &= ~(1 << lab);
      packed |= (lab + 1) << (4 * pos);  // gluon index 1..N-2
    }
    s_ord[r] = packed;
  }
  for (int it = tid; it < EB * N; it += S::NT) {
    const int el = it / N, g = it % N;
    const int64_t e = e0 + el;
    if (e >= B) continue;
    double k[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) k[m] = p[((int64_t)m * N + g) * S_ + e] * inv_sqrt_s;
    if (g < 2) {
#pragma unroll
      for (int m = 0; m < 4; ++m) k[m] = -k[m];
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) s_k[(el * N + g) * 4 + m] = T(k[m]);
    if (SUMHEL) {
      T e1[4], e2[4];
      lc_polarisation_frame<T>(k, F, true, e1);
      lc_polarisation_frame<T>(k, F, false, e2);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        s_e[((el * 2 + 0) * N + g) * 4 + m] = e1[m];
        s_e[((el * 2 + 1) * N + g) * 4 + m] = e2[m];
      }
    } else {
      const int h = hel[(int64_t)g * S_ + e];
      if (h != 1 && h != -1) flag_status(status, BG_EINVAL);
      T ev[4];
      lc_polarisation_frame<T>(k, F, h >= 0, ev);
#pragma unroll
      for (int m = 0; m < 4; ++m) s_e[(el * N + g) * 4 + m] = ev[m];
    }
  }
  // pair invariants 2 k_a.k_b (FP64) among the first M gluons
  for (int it = tid; it < EB * S::NPAIR; it += S::NT) {
    const int el = it / S::NPAIR;
    int pr = it % S::NPAIR;
    const int64_t e = e0 + el;
    if (e >= B) continue;
    int a = 0;
    while (pr >= M - 1 - a) { pr -= M - 1 - a; ++a; }
    const int b = a + 1 + pr;
    double ka[4], kb[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      ka[m] = p[((int64_t)m * N + a) * S_ + e];
      kb[m] = p[((int64_t)m * N + b) * S_ + e];
    }
    // both beams or neither flipped -> +, one flipped -> - (k = -p for gluons 1, 2)
    const double sgn = ((a < 2) != (b < 2)) ? -1.0 : 1.0;
    s_pair[el * S::NPAIR + it % S::NPAIR] =
        sgn * 2.0 * (ka[0] * kb[0] - ka[1] * kb[1] - ka[2] * kb[2] - ka[3] * kb[3]) * inv_sqrt_s * inv_sqrt_s;
  }
  __syncthreads();
  // ---- phase 1b: inverse propagators for every subset of the first M gluons
  co_inverse_table<M, EB, S::NT, T>(s_pair, reinterpret_cast<double*>(smem + L::off_p2), s_inv, e0, B);

  // ---- phase 2: one ordering (and polarisation configuration) per thread
  constexpr int TOTAL = EB * S::TPE;
  const T vfac = T(1.0 / double(1 << ((N - 2) / 2)) * (((N - 2) & 1) ? 0.70710678118654752440 : 1.0));
  for (int t = tid; t < TOTAL; t += S::NT) {
    const int el = t / S::TPE;
    const int rem = t - el * S::TPE;
    const int h = rem / K;
    const int r = rem - h * K;
    const int64_t e = e0 + el;
    if (e >= B) continue;
    const int packed = s_ord[r];
    int gl[N];
    gl[0] = 0;
#pragma unroll
    for (int pos = 1; pos < N - 1; ++pos) gl[pos] = (packed >> (4 * (pos - 1))) & 15;
    gl[N - 1] = N - 1;
    const T* ke = s_k + el * N * 4;
    T J[M][M][4];
    T Sp[N][4];
    int msk[N];
#pragma unroll
    for (int m = 0; m < 4; ++m) Sp[0][m] = T(0);
    msk[0] = 0;
#pragma unroll
    for (int pos = 0; pos < M; ++pos) {
      const int g = gl[pos];
      const int pol = SUMHEL ? ((h >> g) & 1) : 0;
      const T* ev = s_e + ((el * NPOL + pol) * N + g) * 4;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        J[pos][pos][m] = ev[m];
        Sp[pos + 1][m] = Sp[pos][m] + ke[g * 4 + m];
      }
      msk[pos + 1] = msk[pos] | (1 << g);
    }
    T en[4];
    {
      const int pol = SUMHEL ? ((h >> (N - 1)) & 1) : 0;
      const T* ev = s_e + ((el * NPOL + pol) * N + (N - 1)) * 4;
#pragma unroll
      for (int m = 0; m < 4; ++m) en[m] = ev[m];
    }
    T a;
    if constexpr (TF)
      a = co_recursion_tf<N, T>(J, Sp, msk, s_inv + el * S::NMASK, en);
    else
      a = co_recursion<N, T>(J, Sp, msk, s_inv + el * S::NMASK, en);
    amps[(e * H + h) * (int64_t)K + r] = a * vfac;
  }
}

template <int N, typename T, bool SUMHEL, bool TF = false>
cudaError_t launch_co_n(int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q, T* amps,
                        int* status, cudaStream_t s, const int64_t* dB) {
  using S = CoShape<N, SUMHEL>;
  using L = CoSmem<N, T, SUMHEL>;
  auto kern = co_kernel<N, T, SUMHEL, TF>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
  if (err != cudaSuccess) return err;
  const PolFrame F = make_pol_frame(q);
  const int64_t blocks = (B + S::EB - 1) / S::EB;
  kern<<<(unsigned)blocks, S::NT, L::bytes, s>>>(B, dB, 1.0 / sqrt_s, p, hel, F, amps, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Variant for n >= 5 that shares work between orderings: a thread takes the
// six orderings that differ only in the gluons at the last three positions of
// the off-shell current (consecutive in lexicographic order).  The columns of
// the common prefix are computed once, the column of the third-to-last
// position once per choice of its gluon (3), and the last two columns once per
// ordering (6).  At n = 8 this removes ~21 % of the arithmetic.
// ---------------------------------------------------------------------------
template <int N, int NT_ = 256>
struct CoDfsShape {
  static constexpr int NT = NT_;
  static constexpr int M = N - 1;
  static constexpr int K = ct_fact(N - 2);
  static constexpr int G = K / 6;                  // groups of six orderings
  static constexpr int EB0 = NT / ct_gcd(NT, G);   // events per block: EB*G % NT == 0
  static constexpr int EB = EB0 > 128 ? 128 : EB0;
  static constexpr int NMASK = 1 << M;
  static constexpr int NPAIR = M * (M - 1) / 2;
};

template <int N, typename T, int NT_ = 256>
struct CoDfsSmem {
  using S = CoDfsShape<N, NT_>;
  static constexpr size_t off_pair = 0;                                                // double [EB][NPAIR]
  static constexpr size_t off_inv = off_pair + sizeof(double) * S::EB * S::NPAIR;      // T [EB][NMASK]
  static constexpr size_t off_k = off_inv + sizeof(T) * S::EB * S::NMASK;              // T [EB][N][4]
  static constexpr size_t off_e = off_k + sizeof(T) * S::EB * N * 4;                   // T [EB][N][4]
  static constexpr size_t off_ord = off_e + sizeof(T) * S::EB * N * 4;                 // int [G]
  static constexpr size_t off_p2 = (off_ord + sizeof(int) * S::G + 7) & ~size_t(7);     // double [EB][NMASK]
  static constexpr size_t bytes = off_p2 + sizeof(double) * S::EB * S::NMASK;
};

template <int N, typename T, int NT_>
__device__ __forceinline__ void co_dfs_body(int64_t S_, const int64_t* __restrict__ dB, double inv_sqrt_s,
                                            const double* __restrict__ p, const int8_t* __restrict__ hel,
                                            const PolFrame& F, T* __restrict__ amps, int* __restrict__ status) {
  // S_: capacity (row stride of p and hel); dB: device-side event count (NULL: S_)
  const int64_t B = dB ? (*dB < S_ ? *dB : S_) : S_;
  using S = CoDfsShape<N, NT_>;
  using L = CoDfsSmem<N, T, NT_>;
  constexpr int M = S::M, K = S::K, G = S::G, EB = S::EB, NT = S::NT;
  extern __shared__ __align__(16) unsigned char smem[];
  double* s_pair = reinterpret_cast<double*>(smem + L::off_pair);
  T* s_inv = reinterpret_cast<T*>(smem + L::off_inv);
  T* s_k = reinterpret_cast<T*>(smem + L::off_k);
  T* s_e = reinterpret_cast<T*>(smem + L::off_e);
  int* s_ord = reinterpret_cast<int*>(smem + L::off_ord);

  const int64_t e0 = (int64_t)blockIdx.x * EB;
  const int tid = threadIdx.x;
  if (e0 >= B) return;

  // ---- phase 1: ordering of the first member of each group, momenta,
  //      polarisations, pair invariants, inverse propagators (FP64 -> T)
  for (int gi = tid; gi < G; gi += NT) {
    int avail = (1 << (N - 2)) - 1;
    int rr = 6 * gi, packed = 0;
#pragma unroll
    for (int pos = 0; pos < N - 2; ++pos) {
      const int f = ct_fact(N - 3 - pos);
      const int d = rr / f;
      rr -= d * f;
      int lab = 0, cnt = -1;
#pragma unroll
      for (int b = 0; b < N - 2; ++b) {
        const bool on = (avail >> b) & 1;
        cnt += on ? 1 : 0;
        if (on && cnt == d) lab = b;
      }
      avail &= ~(1 << lab);
      packed |= (lab + 1) << (4 * pos);
    }
    s_ord[gi] = packed;
  }
  for (int it = tid; it < EB * N; it += NT) {
    const int el = it / N, g = it % N;
    const int64_t e = e0 + el;
    if (e >= B) continue;
    double k[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) k[m] = p[((int64_t)m * N + g) * S_ + e] * inv_sqrt_s;
    if (g < 2) {
#pragma unroll
      for (int m = 0; m < 4; ++m) k[m] = -k[m];
    }
    const int h = hel[(int64_t)g * S_ + e];
    if (h != 1 && h != -1) flag_status(status, BG_EINVAL);
    T ev[4];
    lc_polarisation_frame<T>(k, F, h >= 0, ev);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      s_k[(el * N + g) * 4 + m] = T(k[m]);
      s_e[(el * N + g) * 4 + m] = ev[m];
    }
  }
  for (int it = tid; it < EB * S::NPAIR; it += NT) {
    const int el = it / S::NPAIR;
    int pr = it % S::NPAIR;
    const int64_t e = e0 + el;
    if (e >= B) continue;
    int a = 0;
    while (pr >= M - 1 - a) { pr -= M - 1 - a; ++a; }
    const int b = a + 1 + pr;
    double ka[4], kb[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      ka[m] = p[((int64_t)m * N + a) * S_ + e];
      kb[m] = p[((int64_t)m * N + b) * S_ + e];
    }
    const double sgn = ((a < 2) != (b < 2)) ? -1.0 : 1.0;
    s_pair[el * S::NPAIR + it % S::NPAIR] =
        sgn * 2.0 * (ka[0] * kb[0] - ka[1] * kb[1] - ka[2] * kb[2] - ka[3] * kb[3]) * inv_sqrt_s * inv_sqrt_s;
  }
  __syncthreads();
  co_inverse_table<M, EB, NT, T>(s_pair, reinterpret_cast<double*>(smem + L::off_p2), s_inv, e0, B);

  // ---- phase 2: one group of six orderings per thread
  constexpr int TOTAL = EB * G;
  const T vfac = T(1.0 / double(1 << ((N - 2) / 2)) * (((N - 2) & 1) ? 0.70710678118654752440 : 1.0));
  for (int t = tid; t < TOTAL; t += NT) {
    const int el = t / G;
    const int gi = t - el * G;
    const int64_t e = e0 + el;
    if (e >= B) continue;
    const int packed = s_ord[gi];
    const T* ke = s_k + el * N * 4;
    const T* ee = s_e + el * N * 4;
    const T* inv = s_inv + el * S::NMASK;
    T J[M][M][4];
    T D[M][M][M];  // cached V3 dot products (co_bracket_dc)
    T Sp[N][4];
    int msk[N];
#pragma unroll
    for (int m = 0; m < 4; ++m) Sp[0][m] = T(0);
    msk[0] = 0;
    // positions 0 .. M-4 are common to the group
#pragma unroll
    for (int pos = 0; pos <= M - 4; ++pos) {
      const int g = (pos == 0) ? 0 : ((packed >> (4 * (pos - 1))) & 15);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        J[pos][pos][m] = ee[g * 4 + m];
        Sp[pos + 1][m] = Sp[pos][m] + ke[g * 4 + m];
      }
      msk[pos + 1] = msk[pos] | (1 << g);
    }
    // the three gluons of the last three positions, ascending
    const int tri[3] = {(packed >> (4 * (M - 4))) & 15, (packed >> (4 * (M - 3))) & 15,
                        (packed >> (4 * (M - 2))) & 15};
    T en[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) en[m] = ee[(N - 1) * 4 + m];
    // prefix columns 1 .. M-4
#pragma unroll
    for (int j = 1; j <= M - 4; ++j) {
#pragma unroll
      for (int i = j - 1; i >= 0; --i) {
        T br[4];
        co_bracket_dc<N, T>(J, Sp, D, i, j, br);
        const T ip = inv[msk[j + 1] ^ msk[i]];
        scale4(ip, br, J[i][j]);
      }
    }
    T* out = amps + (e * (int64_t)K + 6 * gi);
#pragma unroll 1
    for (int xi = 0; xi < 3; ++xi) {
      const int x = tri[xi];
      const int y0 = tri[xi == 0 ? 1 : 0];
      const int z0 = tri[xi == 2 ? 1 : 2];
      {
        constexpr int P = M - 3;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          J[P][P][m] = ee[x * 4 + m];
          Sp[P + 1][m] = Sp[P][m] + ke[x * 4 + m];
        }
        msk[P + 1] = msk[P] | (1 << x);
#pragma unroll
        for (int i = P - 1; i >= 0; --i) {
          T br[4];
          co_bracket_dc<N, T>(J, Sp, D, i, P, br);
          const T ip = inv[msk[P + 1] ^ msk[i]];
          scale4(ip, br, J[i][P]);
        }
      }
#pragma unroll 1
      for (int yi = 0; yi < 2; ++yi) {
        const int y = yi == 0 ? y0 : z0;
        const int z = yi == 0 ? z0 : y0;
        constexpr int P = M - 2;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          J[P][P][m] = ee[y * 4 + m];
          Sp[P + 1][m] = Sp[P][m] + ke[y * 4 + m];
          J[P + 1][P + 1][m] = ee[z * 4 + m];
          Sp[P + 2][m] = Sp[P + 1][m] + ke[z * 4 + m];
        }
        msk[P + 1] = msk[P] | (1 << y);
        msk[P + 2] = msk[P + 1] | (1 << z);
#pragma unroll
        for (int i = P - 1; i >= 0; --i) {
          T br[4];
          co_bracket_dc<N, T>(J, Sp, D, i, P, br);
          const T ip = inv[msk[P + 1] ^ msk[i]];
          scale4(ip, br, J[i][P]);
        }
        T amp = T(0);
#pragma unroll
        for (int i = P; i >= 0; --i) {
          T br[4];
          co_bracket_dc<N, T>(J, Sp, D, i, P + 1, br);
          if (i > 0) {
            const T ip = inv[msk[P + 2] ^ msk[i]];
            scale4(ip, br, J[i][P + 1]);
          } else {
            amp = mdot(en, br);
          }
        }
        out[2 * xi + yi] = amp * vfac;
      }
    }
  }
}

// Kernels of the depth-first variant: a block size with a minimum number of
// resident blocks (the register budget follows from it), or a block size
// with an explicit register cap MAXREG (the compiler spills what does not
// fit).  Both run co_dfs_body: the same arithmetic, bitwise identical.
template <int N, typename T, int NT_, int MINB_ = 1>
__global__ void __launch_bounds__(NT_, MINB_) co_kernel_dfs(int64_t S_, const int64_t* __restrict__ dB, double inv_sqrt_s,
                                                     const double* __restrict__ p, const int8_t* __restrict__ hel,
                                                     PolFrame F, T* __restrict__ amps, int* __restrict__ status) {
  co_dfs_body<N, T, NT_>(S_, dB, inv_sqrt_s, p, hel, F, amps, status);
}
template <int N, typename T, int NT_, int MAXREG_>
__global__ void __launch_bounds__(NT_) __maxnreg__(MAXREG_)
    co_kernel_dfs_r(int64_t S_, const int64_t* __restrict__ dB, double inv_sqrt_s, const double* __restrict__ p,
                    const int8_t* __restrict__ hel, PolFrame F, T* __restrict__ amps, int* __restrict__ status) {
  co_dfs_body<N, T, NT_>(S_, dB, inv_sqrt_s, p, hel, F, amps, status);
}

// MINB > 0: co_kernel_dfs<.., NT, MINB>; MINB < 0: co_kernel_dfs_r with at
// most -MINB registers per thread.
template <int N, typename T, int NT, int MINB>
constexpr auto co_dfs_kernel_ptr() {
  if constexpr (MINB > 0)
    return co_kernel_dfs<N, T, NT, MINB>;
  else
    return co_kernel_dfs_r<N, T, NT, -MINB>;
}

template <int N, typename T, int NT, int MINB = 1>
cudaError_t launch_co_dfs(int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q, T* amps,
                          int* status, cudaStream_t s, const int64_t* dB) {
  using S = CoDfsShape<N, NT>;
  using L = CoDfsSmem<N, T, NT>;
  auto kern = co_dfs_kernel_ptr<N, T, NT, MINB>();
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
  if (err != cudaSuccess) return err;
  const PolFrame F = make_pol_frame(q);
  const int64_t blocks = (B + S::EB - 1) / S::EB;
  kern<<<(unsigned)blocks, S::NT, L::bytes, s>>>(B, dB, 1.0 / sqrt_s, p, hel, F, amps, status);
  return cudaGetLastError();
}

// Variants (sampled helicities, n >= 6): 0 = one thread per ordering,
// 1 = depth-first groups of six orderings in blocks of 256 threads, 2 = the
// same in blocks of 128 threads (more resident blocks: the FP64 prologue of
// one block overlaps the recursion of another), 3 = 128-thread blocks with
// registers capped for three resident blocks per SM, 4 and 5 = 64-thread
// blocks with at most 200 and 184 registers per thread (10 and 11 resident
// warps per SM at n = 8, where the uncapped kernel takes 219 and allows 8).
// Defaults (GB300 timings): 2 for n = 6, 7; 1 for n = 8, 9.  The helicity
// sum and n < 6 have one variant.
inline int co_num_variants(int n, bool sum) { return (!sum && n >= 6) ? 6 : 1; }

template <typename T>
cudaError_t launch_co_t(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                        T* amps, int* status, cudaStream_t s, const int64_t* dB, int variant) {
  const bool sum = (hel == nullptr);
  const int v = (sum || n < 6) ? 0 : (variant < 0 || variant > 5 ? (n <= 7 ? 2 : 1) : variant);
#define BG_CO_CASE(NN)                                                                                   \
  case NN:                                                                                               \
    if (sum) return launch_co_n<NN, T, true>(B, sqrt_s, p, hel, q, amps, status, s, dB);                \
    if (v == 1) return launch_co_dfs<(NN >= 6 ? NN : 6), T, 256>(B, sqrt_s, p, hel, q, amps, status, s, dB); \
    if (v == 2) return launch_co_dfs<(NN >= 6 ? NN : 6), T, 128>(B, sqrt_s, p, hel, q, amps, status, s, dB); \
    if (v == 3) return launch_co_dfs<(NN >= 6 ? NN : 6), T, 128, 3>(B, sqrt_s, p, hel, q, amps, status, s, dB); \
    if (v == 4) return launch_co_dfs<(NN >= 6 ? NN : 6), T, 64, -200>(B, sqrt_s, p, hel, q, amps, status, s, dB); \
    if (v == 5) return launch_co_dfs<(NN >= 6 ? NN : 6), T, 64, -184>(B, sqrt_s, p, hel, q, amps, status, s, dB); \
    return launch_co_n<NN, T, false>(B, sqrt_s, p, hel, q, amps, status, s, dB);
  switch (n) {
    BG_CO_CASE(4)
    BG_CO_CASE(5)
    BG_CO_CASE(6)
    BG_CO_CASE(7)
    BG_CO_CASE(8)
    BG_CO_CASE(9)
    default: return cudaErrorInvalidValue;
  }
#undef BG_CO_CASE
}

// The tensor form (Eqs. 2.23-2.26) in the one-thread-per-ordering kernel,
// sampled or summed helicities, 4 <= n <= 9.
template <typename T>
cudaError_t launch_co_tensor_t(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                               T* amps, int* status, cudaStream_t s) {
  const bool sum = (hel == nullptr);
#define BG_COT_CASE(NN)                                                                      \
  case NN:                                                                                   \
    if (sum) return launch_co_n<NN, T, true, true>(B, sqrt_s, p, hel, q, amps, status, s, nullptr); \
    return launch_co_n<NN, T, false, true>(B, sqrt_s, p, hel, q, amps, status, s, nullptr);
  switch (n) {
    BG_COT_CASE(4)
    BG_COT_CASE(5)
    BG_COT_CASE(6)
    BG_COT_CASE(7)
    BG_COT_CASE(8)
    BG_COT_CASE(9)
    default: return cudaErrorInvalidValue;
  }
#undef BG_COT_CASE
}

}  // namespace bg
