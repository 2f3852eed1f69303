// co_grad.cuh -- reverse mode (adjoint) of the colour-ordered recursion, for
// the gradient of |M|^2 = scale * A^T C A (Eq. 2.16) with respect to the
// momenta and polarisation vectors of the gluons.
//
// One thread per (event, ordering).  Each thread owns slots in shared
// memory (thread index fastest, so accesses are bank-conflict free) for the
// currents J(i..j) of its ordering, their adjoints, the prefix sums S_p of
// the ordered momenta and their adjoints.  The forward sweep recomputes the
// currents (same arithmetic as co_recursion.cuh); the reverse sweep walks the
// segments from the longest to the shortest.  The adjoint of the amplitude
// with unit vertex factors is dA = 2 vfac (C A)_sigma, vfac = (1/sqrt2)^(n-2).
// For every segment the adjoint of its bracket is pushed to the sub-currents
// it was built from (V3 and V4 terms), to the prefix sums (V3 momentum terms
// and the propagator 1/P^2), and, for single-gluon segments, to the
// polarisation vectors.  The per-event adjoints of the momenta and
// polarisations are summed over the orderings (warp reductions and shared
// atomics) and written in FP64 as [B][n][4].
#pragma once

#include "co_recursion.cuh"

namespace bg {

template <int N, typename T>
struct GradShape {
  static constexpr int NT = sizeof(T) == 4 ? 128 : 64;
  static constexpr int M = N - 1;
  static constexpr int K = ct_fact(N - 2);
  static constexpr int EB0 = NT / ct_gcd(NT, K);
  static constexpr int EB = EB0 > 64 ? 64 : EB0;
  static constexpr int NSEG = M * (M + 1) / 2;
  static constexpr int NMASK = 1 << M;
  static constexpr int NPAIR = M * (M - 1) / 2;
  // per-thread slots: J, Jbar (NSEG x 4), S, Sbar (N x 4), scratch (5 x M)
  static constexpr int SLOTS = 2 * NSEG * 4 + 2 * N * 4 + 5 * M;
};

template <int N, typename T>
struct GradSmem {
  using S = GradShape<N, T>;
  static constexpr size_t off_pair = 0;                                              // double [EB][NPAIR]
  static constexpr size_t off_inv = off_pair + sizeof(double) * S::EB * S::NPAIR;    // T [EB][NMASK]
  static constexpr size_t off_k = off_inv + sizeof(T) * S::EB * S::NMASK;            // T [EB][N][4]
  static constexpr size_t off_e = off_k + sizeof(T) * S::EB * N * 4;                 // T [EB][N][4]
  static constexpr size_t off_acc = off_e + sizeof(T) * S::EB * N * 4;               // T [EB][2][N][4]
  static constexpr size_t off_slot = off_acc + sizeof(T) * S::EB * 2 * N * 4;        // T [SLOTS][NT]
  static constexpr size_t off_ord = off_slot + sizeof(T) * S::SLOTS * S::NT;         // int [K]
  static constexpr size_t bytes = off_ord + sizeof(int) * S::K;
};

// Per-thread view of the slots.
template <int N, typename T>
struct GradSlots {
  using S = GradShape<N, T>;
  T* base;
  int tid;
  __device__ __forceinline__ int seg(int i, int j) const { return i * S::M - i * (i - 1) / 2 + (j - i); }
  __device__ __forceinline__ T& J(int i, int j, int m) const { return base[((seg(i, j)) * 4 + m) * S::NT + tid]; }
  __device__ __forceinline__ T& Jb(int i, int j, int m) const {
    return base[((S::NSEG + seg(i, j)) * 4 + m) * S::NT + tid];
  }
  __device__ __forceinline__ T& Sp(int p, int m) const { return base[((2 * S::NSEG + p) * 4 + m) * S::NT + tid]; }
  __device__ __forceinline__ T& Sb(int p, int m) const {
    return base[((2 * S::NSEG + N + p) * 4 + m) * S::NT + tid];
  }
  // scratch arrays 0..4 of length M
  __device__ __forceinline__ T& X(int a, int s) const {
    return base[(8 * S::NSEG + 8 * N + a * S::M + s) * S::NT + tid];
  }
};

template <typename T>
__device__ __forceinline__ T dot4(const T* a, const T* b) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

template <int N, typename T>
__device__ __forceinline__ void loadJ(const GradSlots<N, T>& sl, int i, int j, T (&v)[4]) {
#pragma unroll
  for (int m = 0; m < 4; ++m) v[m] = sl.J(i, j, m);
}

// Forward sweep in the slots; returns the amplitude with unit vertex factors.
template <int N, typename T>
__device__ T grad_forward(const GradSlots<N, T>& sl, const int* msk, const T* __restrict__ inv, const T (&en)[4],
                          T (&brtop)[4]) {
  constexpr int M = N - 1;
  T amp = T(0);
  for (int len = 2; len <= M; ++len) {
    for (int i = 0; i + len - 1 < M; ++i) {
      const int j = i + len - 1;
      T P2[4], br[4], by[4], W[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        P2[m] = T(2) * (sl.Sp(j + 1, m) - sl.Sp(i, m));
        br[m] = T(0);
        by[m] = T(0);
        W[m] = T(0);
      }
      T sxy = T(0);
      for (int s = i; s < j; ++s) {
        T X[4], Y[4];
        loadJ(sl, i, s, X);
        loadJ(sl, s + 1, j, Y);
        const T xy = dot4(X, Y);
        sxy += xy;
#pragma unroll
        for (int m = 0; m < 4; ++m) W[m] = fma(xy, sl.Sp(s + 1, m), W[m]);
        sl.X(0, s) = -dot4(P2, Y);  // cX
        sl.X(1, s) = dot4(P2, X);   // cR
      }
      for (int s = i; s < j; ++s)
        for (int t = s + 1; t < j; ++t) {
          T X[4], Y[4], Z[4];
          loadJ(sl, i, s, X);
          loadJ(sl, s + 1, t, Y);
          loadJ(sl, t + 1, j, Z);
          sl.X(0, s) -= dot4(Y, Z);
          sl.X(1, t) -= dot4(X, Y);
          const T xz = dot4(X, Z);
#pragma unroll
          for (int m = 0; m < 4; ++m) by[m] = fma(xz, Y[m], by[m]);
        }
      for (int s = i; s < j; ++s) {
        const T cx = sl.X(0, s), cr = sl.X(1, s);
#pragma unroll
        for (int m = 0; m < 4; ++m) br[m] = fma(cx, sl.J(i, s, m), fma(cr, sl.J(s + 1, j, m), br[m]));
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) br[m] += T(2) * (W[m] + by[m]) - sxy * (sl.Sp(i, m) + sl.Sp(j + 1, m));
      if (len < M) {
        const T ip = inv[msk[j + 1] ^ msk[i]];
#pragma unroll
        for (int m = 0; m < 4; ++m) sl.J(i, j, m) = br[m] * ip;
      } else {
        amp = dot4(en, br);
#pragma unroll
        for (int m = 0; m < 4; ++m) brtop[m] = br[m];
      }
    }
  }
  return amp;
}

// Reverse sweep: adjoints of all currents (slots Jb), of the prefix sums
// (slots Sb) and of the last gluon's polarisation (enb).
template <int N, typename T>
__device__ void grad_reverse(const GradSlots<N, T>& sl, const int* msk, const T* __restrict__ inv, const T (&en)[4],
                             const T (&brtop)[4], T abar, T (&enb)[4]) {
  constexpr int M = N - 1;
  const T gm[4] = {T(1), T(-1), T(-1), T(-1)};
  for (int p = 0; p < N; ++p)
#pragma unroll
    for (int m = 0; m < 4; ++m) sl.Sb(p, m) = T(0);
  for (int i = 0; i < M; ++i)
    for (int j = i; j < M; ++j)
#pragma unroll
      for (int m = 0; m < 4; ++m) sl.Jb(i, j, m) = T(0);
#pragma unroll
  for (int m = 0; m < 4; ++m) enb[m] = abar * gm[m] * brtop[m];

  for (int len = M; len >= 2; --len) {
    for (int i = 0; i + len - 1 < M; ++i) {
      const int j = i + len - 1;
      T P2[4], bb[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) P2[m] = T(2) * (sl.Sp(j + 1, m) - sl.Sp(i, m));
      if (len == M) {
#pragma unroll
        for (int m = 0; m < 4; ++m) bb[m] = abar * gm[m] * en[m];
      } else {
        const T ip = inv[msk[j + 1] ^ msk[i]];
        T jbj = T(0);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const T v = sl.Jb(i, j, m);
          bb[m] = v * ip;
          jbj = fma(v, sl.J(i, j, m), jbj);
        }
        // J = br / P^2: d(1/P^2)/dP^mu = -2 g_mu P^mu / P^4, inv_bar = (Jbar . J) / inv
        const T c = T(-2) * jbj * ip;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const T pl = gm[m] * (sl.Sp(j + 1, m) - sl.Sp(i, m));
          sl.Sb(j + 1, m) = fma(c, pl, sl.Sb(j + 1, m));
          sl.Sb(i, m) = fma(-c, pl, sl.Sb(i, m));
        }
      }
      // recompute cX, cR (scratch 0, 1) and xy (scratch 2); sxy
      T sxy = T(0);
      for (int s = i; s < j; ++s) {
        T X[4], Y[4];
        loadJ(sl, i, s, X);
        loadJ(sl, s + 1, j, Y);
        const T xy = dot4(X, Y);
        sl.X(2, s) = xy;
        sxy += xy;
        sl.X(0, s) = -dot4(P2, Y);
        sl.X(1, s) = dot4(P2, X);
      }
      for (int s = i; s < j; ++s)
        for (int t = s + 1; t < j; ++t) {
          T X[4], Y[4], Z[4];
          loadJ(sl, i, s, X);
          loadJ(sl, s + 1, t, Y);
          loadJ(sl, t + 1, j, Z);
          sl.X(0, s) -= dot4(Y, Z);
          sl.X(1, t) -= dot4(X, Y);
        }
      // bracket = sum_s (cX X_s + cR Y_s) + 2 W + 2 by - sxy (S_i + S_{j+1})
      for (int s = i; s < j; ++s) {
        T a = T(0), b = T(0);
        const T cx = sl.X(0, s), cr = sl.X(1, s);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          a = fma(bb[m], sl.J(i, s, m), a);
          b = fma(bb[m], sl.J(s + 1, j, m), b);
          sl.Jb(i, s, m) = fma(cx, bb[m], sl.Jb(i, s, m));
          sl.Jb(s + 1, j, m) = fma(cr, bb[m], sl.Jb(s + 1, j, m));
        }
        sl.X(3, s) = a;  // cX bar
        sl.X(4, s) = b;  // cR bar
      }
      T sxyb = T(0);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        sxyb = fma(-bb[m], sl.Sp(i, m) + sl.Sp(j + 1, m), sxyb);
        sl.Sb(i, m) = fma(-sxy, bb[m], sl.Sb(i, m));
        sl.Sb(j + 1, m) = fma(-sxy, bb[m], sl.Sb(j + 1, m));
      }
      // V4: cX[s] -= Y.Z, cR[t] -= X.Y, by += (X.Z) Y with by_bar = 2 bb
      for (int s = i; s < j; ++s)
        for (int t = s + 1; t < j; ++t) {
          T X[4], Y[4], Z[4];
          loadJ(sl, i, s, X);
          loadJ(sl, s + 1, t, Y);
          loadJ(sl, t + 1, j, Z);
          const T xz = dot4(X, Z);
          const T yzb = -sl.X(3, s);
          const T xyb = -sl.X(4, t);
          T xzb = T(0);
#pragma unroll
          for (int m = 0; m < 4; ++m) xzb = fma(T(2) * bb[m], Y[m], xzb);
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            sl.Jb(i, s, m) += gm[m] * (xzb * Z[m] + xyb * Y[m]);
            sl.Jb(t + 1, j, m) += gm[m] * (xzb * X[m] + yzb * Y[m]);
            sl.Jb(s + 1, t, m) += T(2) * xz * bb[m] + gm[m] * (xyb * X[m] + yzb * Z[m]);
          }
        }
      // V3: xy = X.Y (sxy, W), cR = P2.X, cX = -P2.Y
      T P2b[4] = {T(0), T(0), T(0), T(0)};
      for (int s = i; s < j; ++s) {
        T X[4], Y[4];
        loadJ(sl, i, s, X);
        loadJ(sl, s + 1, j, Y);
        T xyb = sxyb;
        const T xy = sl.X(2, s);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          xyb = fma(T(2) * bb[m], sl.Sp(s + 1, m), xyb);
          sl.Sb(s + 1, m) = fma(xy, T(2) * bb[m], sl.Sb(s + 1, m));
        }
        const T pxb = sl.X(4, s);
        const T pyb = -sl.X(3, s);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          sl.Jb(i, s, m) += gm[m] * (xyb * Y[m] + pxb * P2[m]);
          sl.Jb(s + 1, j, m) += gm[m] * (xyb * X[m] + pyb * P2[m]);
          P2b[m] += gm[m] * (pxb * X[m] + pyb * Y[m]);
        }
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        sl.Sb(j + 1, m) = fma(T(2), P2b[m], sl.Sb(j + 1, m));
        sl.Sb(i, m) = fma(T(-2), P2b[m], sl.Sb(i, m));
      }
    }
  }
}

template <int N, typename T>
__global__ void __launch_bounds__(GradShape<N, T>::NT) co_grad_kernel(int64_t B, double inv_sqrt_s,
                                                                      const double* __restrict__ p,
                                                                      const int8_t* __restrict__ hel, Q4 q,
                                                                      const T* __restrict__ Y,
                                                                      double* __restrict__ kbar_out,
                                                                      double* __restrict__ ebar_out,
                                                                      int* __restrict__ status) {
  using S = GradShape<N, T>;
  using L = GradSmem<N, T>;
  constexpr int M = S::M, K = S::K, EB = S::EB, NT = S::NT;
  extern __shared__ __align__(16) unsigned char smem[];
  double* s_pair = reinterpret_cast<double*>(smem + L::off_pair);
  T* s_inv = reinterpret_cast<T*>(smem + L::off_inv);
  T* s_k = reinterpret_cast<T*>(smem + L::off_k);
  T* s_e = reinterpret_cast<T*>(smem + L::off_e);
  T* s_acc = reinterpret_cast<T*>(smem + L::off_acc);
  T* s_slot = reinterpret_cast<T*>(smem + L::off_slot);
  int* s_ord = reinterpret_cast<int*>(smem + L::off_ord);

  const int64_t e0 = (int64_t)blockIdx.x * EB;
  const int tid = threadIdx.x;

  // ---- per-event inputs (as in the forward kernel) ----
  for (int r = tid; r < K; r += NT) {
    int avail = (1 << (N - 2)) - 1;
    int rr = r, packed = 0;
    for (int pos = 0; pos < N - 2; ++pos) {
      const int f = ct_fact(N - 3 - pos);
      const int d = rr / f;
      rr -= d * f;
      int lab = 0, cnt = -1;
      for (int b = 0; b < N - 2; ++b) {
        const bool on = (avail >> b) & 1;
        cnt += on ? 1 : 0;
        if (on && cnt == d) lab = b;
      }
      avail &= ~(1 << lab);
      packed |= (lab + 1) << (4 * pos);
    }
    s_ord[r] = packed;
  }
  for (int it = tid; it < EB * 2 * N * 4; it += NT) s_acc[it] = T(0);
  for (int it = tid; it < EB * N; it += NT) {
    const int el = it / N, g = it % N;
    const int64_t e = e0 + el;
    if (e >= B) continue;
    double k[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) k[m] = p[((int64_t)m * N + g) * B + e] * inv_sqrt_s;
    if (g < 2) {
#pragma unroll
      for (int m = 0; m < 4; ++m) k[m] = -k[m];
    }
    double e1[4], e2[4];
    lc_polarisations(k, q.v, e1, e2);
    const int h = hel[(int64_t)g * B + e];
    if (h != 1 && h != -1) flag_status(status, BG_EINVAL);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      s_k[(el * N + g) * 4 + m] = T(k[m]);
      s_e[(el * N + g) * 4 + m] = T(h < 0 ? e2[m] : e1[m]);
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
      ka[m] = p[((int64_t)m * N + a) * B + e];
      kb[m] = p[((int64_t)m * N + b) * B + e];
    }
    const double sgn = ((a < 2) != (b < 2)) ? -1.0 : 1.0;
    s_pair[el * S::NPAIR + it % S::NPAIR] =
        sgn * 2.0 * (ka[0] * kb[0] - ka[1] * kb[1] - ka[2] * kb[2] - ka[3] * kb[3]) * inv_sqrt_s * inv_sqrt_s;
  }
  __syncthreads();
  for (int it = tid; it < EB * S::NMASK; it += NT) {
    const int el = it / S::NMASK, mask = it % S::NMASK;
    if (e0 + el >= B) continue;
    double p2 = 0.0;
    int idx = 0;
    for (int a = 0; a < M; ++a)
      for (int b = a + 1; b < M; ++b) {
        if (((mask >> a) & 1) && ((mask >> b) & 1)) p2 += s_pair[el * S::NPAIR + idx];
        ++idx;
      }
    s_inv[el * S::NMASK + mask] = (__popc(mask) >= 2 && mask != S::NMASK - 1) ? T(1) / T(p2) : T(0);
  }
  __syncthreads();

  // ---- one ordering per thread: forward, reverse, accumulate ----
  const GradSlots<N, T> sl{s_slot, tid};
  constexpr int TOTAL = EB * K;
  const T vfac = T(1.0 / double(1 << ((N - 2) / 2)) * (((N - 2) & 1) ? 0.70710678118654752440 : 1.0));
  for (int t = tid; t < TOTAL; t += NT) {
    const int el = t / K;
    const int r = t - el * K;
    const int64_t e = e0 + el;
    const bool live = e < B;
    int gl[N];
    int msk[N];
    if (live) {
      const int packed = s_ord[r];
      gl[0] = 0;
      for (int pos = 1; pos < N - 1; ++pos) gl[pos] = (packed >> (4 * (pos - 1))) & 15;
      gl[N - 1] = N - 1;
      const T* ke = s_k + el * N * 4;
      const T* ee = s_e + el * N * 4;
      msk[0] = 0;
#pragma unroll
      for (int m = 0; m < 4; ++m) sl.Sp(0, m) = T(0);
      for (int pos = 0; pos < M; ++pos) {
        const int g = gl[pos];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          sl.J(pos, pos, m) = ee[g * 4 + m];
          sl.Sp(pos + 1, m) = sl.Sp(pos, m) + ke[g * 4 + m];
        }
        msk[pos + 1] = msk[pos] | (1 << g);
      }
      T en[4], brtop[4], enb[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) en[m] = ee[(N - 1) * 4 + m];
      const T* inv = s_inv + el * S::NMASK;
      grad_forward<N, T>(sl, msk, inv, en, brtop);
      const T abar = T(2) * vfac * Y[e * (int64_t)K + r];
      grad_reverse<N, T>(sl, msk, inv, en, brtop, abar, enb);
      // momentum adjoint of the gluon at position q: sum of Sbar_p for p > q.
      // In place, shifted by one slot: afterwards Sb(q + 1) holds that sum.
      T run[4] = {T(0), T(0), T(0), T(0)};
      for (int pos = M - 1; pos >= 0; --pos)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          run[m] += sl.Sb(pos + 1, m);
          sl.Sb(pos + 1, m) = run[m];
        }
      // the last gluon's polarisation adjoint goes to a dead scratch slot
#pragma unroll
      for (int m = 0; m < 4; ++m) sl.X(0, m) = enb[m];
    }
    // sum over the orderings of each event, gluon by gluon
    const int el0 = __shfl_sync(0xffffffffu, el, 0);
    const bool uniform = __all_sync(0xffffffffu, el == el0);
    for (int g = 0; g < N; ++g) {
      // position of gluon g in this ordering
      int pos_g = -1;
      if (live) {
        for (int pos = 0; pos < N; ++pos)
          if (gl[pos] == g) pos_g = pos;
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        T a = T(0), b = T(0);
        if (live) {
          if (pos_g < M) {
            a = sl.Sb(pos_g + 1, m);
            b = sl.Jb(pos_g, pos_g, m);
          } else {
            b = sl.X(0, m);
          }
        }
        if (uniform) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
          }
          if ((tid & 31) == 0 && live) {
            atomicAdd(&s_acc[((el * 2 + 0) * N + g) * 4 + m], a);
            atomicAdd(&s_acc[((el * 2 + 1) * N + g) * 4 + m], b);
          }
        } else if (live) {
          atomicAdd(&s_acc[((el * 2 + 0) * N + g) * 4 + m], a);
          atomicAdd(&s_acc[((el * 2 + 1) * N + g) * 4 + m], b);
        }
      }
    }
  }
  __syncthreads();
  for (int it = tid; it < EB * N * 4; it += NT) {
    const int el = it / (N * 4), rem = it % (N * 4);
    const int64_t e = e0 + el;
    if (e >= B) continue;
    kbar_out[e * N * 4 + rem] = (double)s_acc[(el * 2 + 0) * N * 4 + rem];
    ebar_out[e * N * 4 + rem] = (double)s_acc[(el * 2 + 1) * N * 4 + rem];
  }
}

template <int N, typename T>
cudaError_t launch_co_grad_n(int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                             const T* Y, double* kbar, double* ebar, int* status, cudaStream_t s) {
  using S = GradShape<N, T>;
  using L = GradSmem<N, T>;
  auto kern = co_grad_kernel<N, T>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
  if (err != cudaSuccess) return err;
  Q4 qq;
  for (int m = 0; m < 4; ++m) qq.v[m] = q[m];
  const int64_t blocks = (B + S::EB - 1) / S::EB;
  kern<<<(unsigned)blocks, S::NT, L::bytes, s>>>(B, 1.0 / sqrt_s, p, hel, qq, Y, kbar, ebar, status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_co_grad_t(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                             const T* Y, double* kbar, double* ebar, int* status, cudaStream_t s) {
  switch (n) {
    case 4: return launch_co_grad_n<4, T>(B, sqrt_s, p, hel, q, Y, kbar, ebar, status, s);
    case 5: return launch_co_grad_n<5, T>(B, sqrt_s, p, hel, q, Y, kbar, ebar, status, s);
    case 6: return launch_co_grad_n<6, T>(B, sqrt_s, p, hel, q, Y, kbar, ebar, status, s);
    case 7: return launch_co_grad_n<7, T>(B, sqrt_s, p, hel, q, Y, kbar, ebar, status, s);
    case 8: return launch_co_grad_n<8, T>(B, sqrt_s, p, hel, q, Y, kbar, ebar, status, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bg
