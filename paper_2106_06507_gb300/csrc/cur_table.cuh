// cur_table.cuh -- a per-thread table of off-shell currents in shared memory
// for the colour-ordered recursion (Eqs. 2.20-2.22) of one ordering, used
// where a register table of 4 n(n-1)/2 values would spill: the colour-flow
// evaluator at n >= 10 (FP64: n >= 8) and the forward sweep of the gradient.
// The bracket below has the same terms as the register form of the
// colour-ordered kernels (co_recursion.cuh).
#pragma once

#include "co_recursion.cuh"
#include "device_common.cuh"

namespace bg {

// Current table in shared memory: segment (i..j) of thread t at
// tab[(seg(i, j) * NT + t) * 4], four consecutive values (one 16-byte load in
// FP32), consecutive threads in consecutive slots, segments i <= j (or, with
// LEAF, i < j: the one-gluon currents J(p..p) are the polarisation vectors
// and are read from the event's record); the prefix sums S_p of the ordered
// momenta follow the segments (slot tab_nseg + p).
template <int N, bool LEAF>
__host__ __device__ constexpr int tab_seg(int i, int j) {
  return LEAF ? i * (N - 2) - i * (i - 1) / 2 + (j - i - 1) : i * (N - 1) - i * (i - 1) / 2 + (j - i);
}
template <int N, bool LEAF>
__host__ __device__ constexpr int tab_nseg() {
  return LEAF ? (N - 1) * (N - 2) / 2 : (N - 1) * N / 2;
}
// The loads are volatile asm statements so that the compiler keeps them in
// program order instead of hoisting the whole unrolled recursion's loads
// ahead of their use (which needs more than 255 registers and spills).  Such
// a statement does not tell the compiler which memory it reads, so the
// stores are volatile asm statements too: the compiler keeps volatile asm
// statements in their program order, and every table access is one of them.
template <int NT>
__device__ __forceinline__ void tab_ld(const float* __restrict__ tab, int seg, float (&v)[4]) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(tab + (size_t)seg * NT * 4);
  asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
               : "r"(a));
}
template <int NT>
__device__ __forceinline__ void tab_st(float* __restrict__ tab, int seg, const float (&v)[4]) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(tab + (size_t)seg * NT * 4);
  asm volatile("st.volatile.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v[0]), "f"(v[1]), "f"(v[2]),
               "f"(v[3]));
}
template <int NT>
__device__ __forceinline__ void tab_ld(const double* __restrict__ tab, int seg, double (&v)[4]) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(tab + (size_t)seg * NT * 4);
  asm volatile("ld.volatile.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "r"(a));
  asm volatile("ld.volatile.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v[2]), "=d"(v[3]) : "r"(a + 16));
}
template <int NT>
__device__ __forceinline__ void tab_st(double* __restrict__ tab, int seg, const double (&v)[4]) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(tab + (size_t)seg * NT * 4);
  asm volatile("st.volatile.shared.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v[0]), "d"(v[1]));
  asm volatile("st.volatile.shared.v2.f64 [%0], {%1, %2};" ::"r"(a + 16), "d"(v[2]), "d"(v[3]));
}

// J(a..b): with LEAF and a == b the polarisation vector of the gluon at
// position a from the record (ee, 16-byte aligned rows), else the table.
template <int N, int NT, bool LEAF>
__device__ __forceinline__ void tab_ldJ(const float* __restrict__ tab, const float* __restrict__ ee,
                                         const int (&gl)[N], int a, int b, float (&v)[4]) {
  if (LEAF && a == b) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(ee) + gl[a]);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  } else {
    tab_ld<NT>(tab, tab_seg<N, LEAF>(a, b), v);
  }
}
template <int N, int NT, bool LEAF>
__device__ __forceinline__ void tab_ldJ(const double* __restrict__ tab, const double* __restrict__ ee,
                                         const int (&gl)[N], int a, int b, double (&v)[4]) {
  if (LEAF && a == b) {
    const double2 q0 = __ldg(reinterpret_cast<const double2*>(ee) + 2 * gl[a]);
    const double2 q1 = __ldg(reinterpret_cast<const double2*>(ee) + 2 * gl[a] + 1);
    v[0] = q0.x;
    v[1] = q0.y;
    v[2] = q1.x;
    v[3] = q1.y;
  } else {
    tab_ld<NT>(tab, tab_seg<N, LEAF>(a, b), v);
  }
}

// Bracket of segment (i..j) (the V3 and V4 sums before the propagator, unit
// vertex factors) from the shared-memory table: the same terms as the
// register form of the colour-ordered kernels, with the loop over the second
// split point outermost so that only the row J(i..s) stays in registers:
// J(t+1..j) is loaded once per t, the interior J(s+1..t) as it is used, and
// the coefficient of J(t+1..j) is complete (and applied) at the end of
// iteration t.
template <int N, typename T, int NT, bool LEAF>
__device__ __forceinline__ void tab_bracket(const T* __restrict__ tab, const T* __restrict__ ee,
                                                 const int (&gl)[N], const int i, const int j, T (&br)[4]) {
  constexpr int M = N - 1, SP0 = tab_nseg<N, LEAF>();
  T X[M][4];
#pragma unroll
  for (int s = i; s < j; ++s) tab_ldJ<N, NT, LEAF>(tab, ee, gl, i, s, X[s]);
  T Si[4], Sj[4], P2[4];
  tab_ld<NT>(tab, SP0 + i, Si);
  tab_ld<NT>(tab, SP0 + j + 1, Sj);
  sub4(Sj, Si, P2);
  scale4(T(2), P2, P2);
  T by[4], W[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) { br[m] = T(0); by[m] = T(0); W[m] = T(0); }
  T sxy = T(0);
  T cX[M];
  // loads are issued one step ahead of their use (J(t+2..j) and S_{t+2}
  // during iteration t, J(s+2..t) during iteration s), so that the shared-
  // memory latency overlaps arithmetic; the arithmetic order is unchanged
  T Z[4], St[4];
  tab_ldJ<N, NT, LEAF>(tab, ee, gl, i + 1, j, Z);
  tab_ld<NT>(tab, SP0 + i + 1, St);
#pragma unroll
  for (int t = i; t < j; ++t) {
    T Zn[4], Stn[4], Y[4];
    if (t + 1 < j) {
      tab_ldJ<N, NT, LEAF>(tab, ee, gl, t + 2, j, Zn);
      tab_ld<NT>(tab, SP0 + t + 2, Stn);
    }
    if (i < t) tab_ldJ<N, NT, LEAF>(tab, ee, gl, i + 1, t, Y);
    // three-vertex term of the split at t
    const T xy0 = mdot(X[t], Z);
    sxy += xy0;
    axpy4(xy0, St, W);
    cX[t] = -mdot(P2, Z);
    T cR = mdot(P2, X[t]);
    // four-vertex terms (s, t): X = J(i..s), Y = J(s+1..t), Z = J(t+1..j)
#pragma unroll
    for (int s = i; s < t; ++s) {
      T Yn[4];
      if (s + 1 < t) tab_ldJ<N, NT, LEAF>(tab, ee, gl, s + 2, t, Yn);
      const T xz = mdot(X[s], Z);
      const T xy = mdot(X[s], Y);
      const T yz = mdot(Y, Z);
      cX[s] -= yz;
      cR -= xy;
      axpy4(xz, Y, by);
      if (s + 1 < t) {
#pragma unroll
        for (int m = 0; m < 4; ++m) Y[m] = Yn[m];
      }
    }
    axpy4(cR, Z, br);
    if (t + 1 < j) {
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        Z[m] = Zn[m];
        St[m] = Stn[m];
      }
    }
  }
#pragma unroll
  for (int s = i; s < j; ++s) axpy4(cX[s], X[s], br);
  T t4[4], u4[4];
  add4(W, by, t4);
  add4(Si, Sj, u4);
  add4(t4, t4, t4);
  axpy4(-sxy, u4, t4);
  add4(br, t4, br);
}


}  // namespace bg
