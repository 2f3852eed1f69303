// co_grad.cuh -- reverse mode (adjoint) of the colour-ordered recursion, for
// the gradient of |M|^2 = scale * A^T C A (Eq. 2.16) with respect to the
// momenta and polarisation vectors of the gluons.
//
// One thread per (event, ordering).  As in the forward kernel the whole
// recursion is unrolled at compile time for each n and lives in registers:
// the forward sweep computes the currents J(i..j) (same arithmetic as
// co_recursion.cuh), the reverse sweep walks the segments from the longest
// to the shortest with the adjoints Jbar(i..j) of the currents and Sbar_p of
// the prefix sums of the ordered momenta, also in registers.  The adjoint of
// the amplitude with unit vertex factors is dA = 2 vfac (C A)_sigma,
// vfac = (1/sqrt2)^(n-2).  For every segment the adjoint of its bracket is
// pushed to the sub-currents it was built from (V3 and V4 terms), to the
// prefix sums (V3 momentum terms and the propagator 1/P^2), and, for
// single-gluon segments, to the polarisation vectors.
//
// Sums over the orderings of an event, in a fixed order (deterministic):
// the tasks of an event are padded to whole warps; each thread stores its
// per-gluon adjoints in shared memory (thread index fastest) at the slot of
// the gluon it holds at each position, each warp reduces them with shuffles,
// and the warp partials are added in warp order at the end.  Output: FP64
// [B][n][4] adjoints of the scaled momenta and of the polarisation vectors.
#pragma once

#include "co_recursion.cuh"

namespace bg {

template <int N, typename T>
struct GradShape {
  static constexpr int NT = 128;
  static constexpr int M = N - 1;
  static constexpr int K = ct_fact(N - 2);
  static constexpr int KP = (K + 31) / 32 * 32;   // tasks per event, whole warps
  static constexpr int WPE = KP / 32;             // warps per event
  static constexpr int EB = NT / ct_gcd(NT, KP);  // events per block: EB * KP % NT == 0
  static constexpr int NMASK = 1 << M;
  static constexpr int NPAIR = M * (M - 1) / 2;
  static constexpr int NVAL = 2 * N * 4;          // adjoint values per ordering
};

template <int N, typename T>
struct GradSmem {
  using S = GradShape<N, T>;
  static constexpr size_t off_pair = 0;                                               // double [EB][NPAIR]
  static constexpr size_t off_inv = off_pair + sizeof(double) * S::EB * S::NPAIR;     // T [EB][NMASK]
  static constexpr size_t off_k = off_inv + sizeof(T) * S::EB * S::NMASK;             // T [EB][N][4]
  static constexpr size_t off_e = off_k + sizeof(T) * S::EB * N * 4;                  // T [EB][N][4]
  static constexpr size_t off_part = off_e + sizeof(T) * S::EB * N * 4;               // T [EB][WPE][NVAL]
  static constexpr size_t off_scr = off_part + sizeof(T) * S::EB * S::WPE * S::NVAL;  // T [NVAL][NT]
  static constexpr size_t off_ord = off_scr + sizeof(T) * S::NVAL * S::NT;            // int [K]
  static constexpr size_t bytes = off_ord + sizeof(int) * S::K;
};

// acc += g o (a x + b z), g = (1, -1, -1, -1) component-wise (the metric
// applied to a gradient), as packed operations in FP32.
template <typename T>
__device__ __forceinline__ void gaxpby4(T a, const T (&x)[4], T b, const T (&z)[4], T (&acc)[4]) {
  T t[4];
  scale4(b, z, t);
  axpy4(a, x, t);
  const T gm[4] = {T(1), T(-1), T(-1), T(-1)};
#pragma unroll
  for (int m = 0; m < 4; ++m) acc[m] = fma(gm[m], t[m], acc[m]);
}
template <>
__device__ __forceinline__ void gaxpby4<float>(float a, const float (&x)[4], float b, const float (&z)[4],
                                               float (&acc)[4]) {
  float t[4];
  scale4(b, z, t);
  axpy4(a, x, t);
  unsigned long long a01 = pk2(acc[0], acc[1]), a23 = pk2(acc[2], acc[3]);
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(a01) : "l"(pk2(1.0f, -1.0f)), "l"(pk2(t[0], t[1])));
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(a23) : "l"(pk2(-1.0f, -1.0f)), "l"(pk2(t[2], t[3])));
  upk2(a01, acc[0], acc[1]);
  upk2(a23, acc[2], acc[3]);
}

// Euclidean dot product sum_m x[m] y[m] (no metric); in FP32 as one packed
// multiply, one packed FMA and an add.
template <typename T>
__device__ __forceinline__ T edot4(const T (&x)[4], const T (&y)[4]) {
  T r = T(0);
#pragma unroll
  for (int m = 0; m < 4; ++m) r = fma(x[m], y[m], r);
  return r;
}
template <>
__device__ __forceinline__ float edot4<float>(const float (&x)[4], const float (&y)[4]) {
  unsigned long long p;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(p) : "l"(pk2(x[0], x[1])), "l"(pk2(y[0], y[1])));
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(p) : "l"(pk2(x[2], x[3])), "l"(pk2(y[2], y[3])));
  float a, b;
  upk2(p, a, b);
  return a + b;
}

// Forward sweep: all currents of one ordering in registers (J[i][i] hold the
// polarisations); returns the top bracket (the amplitude is en . brtop).
template <int N, typename T>
__device__ __forceinline__ void grad_forward(T (&J)[N - 1][N - 1][4], const T (&Sp)[N][4], const int (&msk)[N],
                                             const T* __restrict__ inv, T (&brtop)[4]) {
  constexpr int M = N - 1;
#pragma unroll
  for (int len = 2; len <= M; ++len) {
    // keeps the block's warps on the same stretch of this long unrolled code,
    // so that one warp's instruction-cache miss serves the others
    __syncthreads();
#pragma unroll
    for (int i = 0; i + len - 1 < M; ++i) {
      const int j = i + len - 1;
      T br[4];
      co_bracket<N, T>(J, Sp, i, j, br);
      if (len < M) {
        const T ip = inv[msk[j + 1] ^ msk[i]];
#pragma unroll
        for (int m = 0; m < 4; ++m) J[i][j][m] = br[m] * ip;
      } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) brtop[m] = br[m];
      }
    }
  }
}

// Reverse sweep: adjoints of all currents (Jb), of the prefix sums (Sb) and
// of the last gluon's polarisation (enb), for the amplitude adjoint abar.
template <int N, typename T>
__device__ __forceinline__ void grad_reverse(const T (&J)[N - 1][N - 1][4], const T (&Sp)[N][4],
                                             const int (&msk)[N], const T* __restrict__ inv, const T (&en)[4],
                                             const T (&brtop)[4], T abar, T (&Jb)[N - 1][N - 1][4],
                                             T (&Sb)[N][4], T (&enb)[4]) {
  constexpr int M = N - 1;
  const T gm[4] = {T(1), T(-1), T(-1), T(-1)};
#pragma unroll
  for (int p = 0; p < N; ++p)
#pragma unroll
    for (int m = 0; m < 4; ++m) Sb[p][m] = T(0);
#pragma unroll
  for (int i = 0; i < M; ++i)
#pragma unroll
    for (int j = i; j < M; ++j)
#pragma unroll
      for (int m = 0; m < 4; ++m) Jb[i][j][m] = T(0);
#pragma unroll
  for (int m = 0; m < 4; ++m) enb[m] = abar * gm[m] * brtop[m];

#pragma unroll
  for (int len = M; len >= 2; --len) {
    __syncthreads();  // as in the forward sweep
#pragma unroll
    for (int i = 0; i + len - 1 < M; ++i) {
      const int j = i + len - 1;
      T P2[4], bb[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) P2[m] = T(2) * (Sp[j + 1][m] - Sp[i][m]);
      if (len == M) {
#pragma unroll
        for (int m = 0; m < 4; ++m) bb[m] = abar * gm[m] * en[m];
      } else {
        // J = br / P^2: bracket adjoint Jbar / P^2; d(1/P^2)/dP^mu = -2 g_mu P^mu / P^4
        const T ip = inv[msk[j + 1] ^ msk[i]];
        T jbj = T(0);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          bb[m] = Jb[i][j][m] * ip;
          jbj = fma(Jb[i][j][m], J[i][j][m], jbj);
        }
        const T c = T(-2) * jbj * ip;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const T pl = gm[m] * (Sp[j + 1][m] - Sp[i][m]);
          Sb[j + 1][m] = fma(c, pl, Sb[j + 1][m]);
          Sb[i][m] = fma(-c, pl, Sb[i][m]);
        }
      }
      // forward coefficients of the bracket: xy_s, cX_s = -P2.Y_s - sum Y.Z,
      // cR_t = P2.X_t - sum X.Y
      T xy[M], cX[M], cR[M], cXb[M], cRb[M];
      T sxy = T(0);
#pragma unroll
      for (int s = i; s < j; ++s) {
        xy[s] = mdot(J[i][s], J[s + 1][j]);
        sxy += xy[s];
        cX[s] = -mdot(P2, J[s + 1][j]);
        cR[s] = mdot(P2, J[i][s]);
      }
#pragma unroll
      for (int s = i; s < j; ++s)
#pragma unroll
        for (int t = s + 1; t < j; ++t) {
          cX[s] -= mdot(J[s + 1][t], J[t + 1][j]);
          cR[t] -= mdot(J[i][s], J[s + 1][t]);
        }
      // bracket = sum_s (cX_s X_s + cR_s Y_s) + 2 W + 2 by - sxy (S_i + S_{j+1})
#pragma unroll
      for (int s = i; s < j; ++s) {
        const T a = edot4(bb, J[i][s]);
        const T b = edot4(bb, J[s + 1][j]);
        axpy4(cX[s], bb, Jb[i][s]);
        axpy4(cR[s], bb, Jb[s + 1][j]);
        cXb[s] = a;
        cRb[s] = b;
      }
      T sxyb = T(0);
#pragma unroll
      for (int m = 0; m < 4; ++m) sxyb = fma(-bb[m], Sp[i][m] + Sp[j + 1][m], sxyb);
      axpy4(-sxy, bb, Sb[i]);
      axpy4(-sxy, bb, Sb[j + 1]);
      T bb2[4];
      add4(bb, bb, bb2);  // 2 bb
      // V4: cX_s -= Y.Z, cR_t -= X.Y, by += (X.Z) Y with by_bar = 2 bb
#pragma unroll
      for (int s = i; s < j; ++s)
#pragma unroll
        for (int t = s + 1; t < j; ++t) {
          const T xz = mdot(J[i][s], J[t + 1][j]);
          const T yzb = -cXb[s];
          const T xyb = -cRb[t];
          const T xzb = edot4(bb2, J[s + 1][t]);
          gaxpby4(xzb, J[t + 1][j], xyb, J[s + 1][t], Jb[i][s]);
          gaxpby4(xzb, J[i][s], yzb, J[s + 1][t], Jb[t + 1][j]);
          axpy4(xz, bb2, Jb[s + 1][t]);
          gaxpby4(xyb, J[i][s], yzb, J[t + 1][j], Jb[s + 1][t]);
        }
      // V3: xy_s enters sxy and W = sum_s xy_s S_{s+1}; cR_s = P2.X_s, cX_s = -P2.Y_s
      T P2b[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int s = i; s < j; ++s) {
        const T xyb = sxyb + edot4(bb2, Sp[s + 1]);
        axpy4(xy[s], bb2, Sb[s + 1]);
        const T pxb = cRb[s];
        const T pyb = -cXb[s];
        gaxpby4(xyb, J[s + 1][j], pxb, P2, Jb[i][s]);
        gaxpby4(xyb, J[i][s], pyb, P2, Jb[s + 1][j]);
        gaxpby4(pxb, J[i][s], pyb, J[s + 1][j], P2b);
      }
      axpy4(T(2), P2b, Sb[j + 1]);
      axpy4(T(-2), P2b, Sb[i]);
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
  constexpr int M = S::M, K = S::K, KP = S::KP, EB = S::EB, NT = S::NT, NVAL = S::NVAL;
  extern __shared__ __align__(16) unsigned char smem[];
  double* s_pair = reinterpret_cast<double*>(smem + L::off_pair);
  T* s_inv = reinterpret_cast<T*>(smem + L::off_inv);
  T* s_k = reinterpret_cast<T*>(smem + L::off_k);
  T* s_e = reinterpret_cast<T*>(smem + L::off_e);
  T* s_part = reinterpret_cast<T*>(smem + L::off_part);
  T* s_scr = reinterpret_cast<T*>(smem + L::off_scr);
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

  // ---- one ordering per thread: forward, reverse, per-warp sums ----
  const T vfac = T(1.0 / double(1 << ((N - 2) / 2)) * (((N - 2) & 1) ? 0.70710678118654752440 : 1.0));
  const int lane = tid & 31;
  for (int t = tid; t < EB * KP; t += NT) {  // EB * KP is a multiple of NT: uniform rounds
    const int el = t / KP;
    const int r = t - el * KP;
    const int64_t e = e0 + el;
    const bool live = (e < B) && (r < K);
    {
      // every thread runs the sweeps (they hold block barriers): the padding
      // tasks on a clamped ordering and event, with a zero seed
      const int rc = r < K ? r : K - 1;
      const int elc = e < B ? el : 0;
      const int packed = s_ord[rc];
      int gl[N];
      gl[0] = 0;
#pragma unroll
      for (int pos = 1; pos < N - 1; ++pos) gl[pos] = (packed >> (4 * (pos - 1))) & 15;
      gl[N - 1] = N - 1;
      const T* ke = s_k + elc * N * 4;
      const T* ee = s_e + elc * N * 4;
      T J[M][M][4], Jb[M][M][4], Sp[N][4], Sb[N][4];
      int msk[N];
      msk[0] = 0;
#pragma unroll
      for (int m = 0; m < 4; ++m) Sp[0][m] = T(0);
#pragma unroll
      for (int pos = 0; pos < M; ++pos) {
        const int g = gl[pos];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          J[pos][pos][m] = ee[g * 4 + m];
          Sp[pos + 1][m] = Sp[pos][m] + ke[g * 4 + m];
        }
        msk[pos + 1] = msk[pos] | (1 << g);
      }
      T en[4], brtop[4], enb[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) en[m] = ee[(N - 1) * 4 + m];
      const T* inv = s_inv + elc * S::NMASK;
      grad_forward<N, T>(J, Sp, msk, inv, brtop);
      const T abar = live ? T(2) * vfac * Y[e * (int64_t)K + rc] : T(0);
      grad_reverse<N, T>(J, Sp, msk, inv, en, brtop, abar, Jb, Sb, enb);
      // momentum adjoint of the gluon at position q: the sum of Sbar_p over
      // p > q (S_p holds the momenta of positions < p); polarisation adjoints
      // Jbar(q..q), and enb for the last gluon, whose momentum enters only
      // through its polarisation.  Stored at the gluon's slot.
      T run[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int pos = M - 1; pos >= 0; --pos) {
        const int g = gl[pos];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          run[m] += Sb[pos + 1][m];
          s_scr[((0 * N + g) * 4 + m) * NT + tid] = run[m];
          s_scr[((1 * N + g) * 4 + m) * NT + tid] = Jb[pos][pos][m];
        }
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        s_scr[((0 * N + N - 1) * 4 + m) * NT + tid] = T(0);
        s_scr[((1 * N + N - 1) * 4 + m) * NT + tid] = enb[m];
      }
    }
    // (dead tasks ran with a zero seed: their adjoints, stored above, are 0)
    // warp sums in a fixed order; a warp holds orderings of one event
    const int wglob = t >> 5;  // warp index among the block's tasks
    const int wel = wglob / S::WPE, wr = wglob % S::WPE;
#pragma unroll 4
    for (int v = 0; v < NVAL; ++v) {
      T a = s_scr[v * NT + tid];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
      if (lane == 0) s_part[(wel * S::WPE + wr) * NVAL + v] = a;
    }
  }
  __syncthreads();
  for (int it = tid; it < EB * NVAL; it += NT) {
    const int el = it / NVAL, v = it % NVAL;
    const int64_t e = e0 + el;
    if (e >= B) continue;
    T a = T(0);
    for (int w = 0; w < S::WPE; ++w) a += s_part[(el * S::WPE + w) * NVAL + v];
    const int which = v / (N * 4), rem = v % (N * 4);
    (which == 0 ? kbar_out : ebar_out)[e * N * 4 + rem] = (double)a;
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
