// comc.cuh -- colour-flow sampling evaluated with colour-ordered amplitudes:
// the colour-sampling variant of the colour-ordered algorithms (Sec. 4),
// with the colour-flow decomposition of Eq. (2.19).
//
// Each event carries a sampled colour flow, a pair (r_i, c_i) in {1,2,3}^2
// per gluon (external colour matrix |r_i><c_i|), and sampled helicities.  The
// flow amplitude is
//   A_flow = sum over orders (1, s_2, ..., s_n) of
//            delta(c_1, r_{s_2}) delta(c_{s_2}, r_{s_3}) ... delta(c_{s_n}, r_1)
//            x A(1, s_2, ..., s_n),
// and |M|^2 is estimated by 9^n 2^n g^(2n-4) |A_flow|^2.  Only orders whose
// delta chain closes contribute: on average (n-1)!/3^n per event, spread
// very unevenly (at n = 12 about 3 % of the flows have any, those have a
// few thousand).
//
// Work decomposition (one block per tile of EB events):
//   1. per event, in shared memory: scaled momenta and sampled polarisation
//      vectors in T, and the pair invariants 2 k_a.k_b for all pairs of the
//      n gluons, computed in FP64 and kept as an unevaluated sum of two
//      floats in the FP32 kernel (FP64 in the FP64 kernel);
//   2. one thread per event walks the orders whose chain closes (depth-first,
//      labels in increasing order) and counts them; a warp scan gives each
//      event its range of item indices;
//   3. in windows of CAP items: each event's walk is resumed where the last
//      window paused it, writing the packed orders of the window into shared
//      memory (an event is walked once in total), then every thread takes
//      items and evaluates the whole recursion of one order (same code path
//      for every item), and one thread per event adds its items' amplitudes
//      in item order (deterministic);
//   4. |M|^2 per event.
// The propagator denominators P(i..j)^2 of each order are accumulated from
// the pair invariants column by column, P(i..j)^2 = P(i..j-1)^2 +
// sum_{a=i}^{j-1} 2 k_{s_a}.k_{s_j}, in double-float arithmetic (Knuth's
// TwoSum, TAOCP vol. 2, 4.2.2) in the FP32 kernel: a plain FP32 sum of the
// invariants, or E^2 - |p|^2 of the FP32 momentum sum, loses up to ~1e-3 of
// P^2 to cancellation between incoming and outgoing momenta.
#pragma once

#include "bg_internal.h"
#include "co_recursion.cuh"
#include "device_common.cuh"

namespace bg {

struct ComcParams {
  int64_t B;                    // capacity (row stride of p, hel, colours)
  const int64_t* dB = nullptr;  // optional device-side event count
  double inv_sqrt_s;
  double scale;  // 9^n 2^n g^(2n-4) sqrt_s^(8-2n) 2^-(n-2)
};

// TAB (n >= 10; FP64 from n = 8): the current table of the order being
// evaluated lives in shared memory (one slice per thread) instead of
// registers: a register table of 4 n(n-1)/2 values spills there, and the
// spilled stacks of the resident threads outgrow L1.
template <int N, typename T>
struct ComcShape {
  static constexpr bool TAB = N >= 10 || (sizeof(T) == 8 && N >= 8);
  // 64 threads with the shared-memory table: two blocks per SM, so that one
  // block's per-event phases (walks, sums) overlap the other's recursions
  static constexpr int NT = TAB ? 64 : 128;
  static constexpr int M = N - 1;
  static constexpr int NPAIR = N * (N - 1) / 2;
  static constexpr int NSEG = M * (M + 1) / 2;  // segments (i..j), i <= j, of the off-shell current
  static constexpr int NSLOT = NSEG + N;         // + prefix sums S_0..S_M of the ordered momenta
  static constexpr int EB = N <= 8 ? 128 : N == 9 ? 64 : N <= 11 ? 32 : 16;
  static constexpr int CAP = TAB ? (sizeof(T) == 8 ? 512 : 1024) : 2048;  // items per window
};

// Pair invariants and running P^2 sums: two floats (value + error) for the
// FP32 kernel, one double for the FP64 kernel.
template <typename T>
struct ComcPair;
template <>
struct ComcPair<float> {
  using type = float2;
};
template <>
struct ComcPair<double> {
  using type = double;
};

__device__ __forceinline__ void p2_split(double v, float2& o) {
  o.x = (float)v;
  o.y = (float)(v - (double)o.x);
}
__device__ __forceinline__ void p2_split(double v, double& o) { o = v; }
__device__ __forceinline__ void p2_zero(float2& o) { o = make_float2(0.f, 0.f); }
__device__ __forceinline__ void p2_zero(double& o) { o = 0.0; }
// (a.x + a.y) + (b.x + b.y) as a normalised two-float sum.
__device__ __forceinline__ float2 p2_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bv = __fsub_rn(s, a.x);
  const float av = __fsub_rn(s, bv);
  float e = __fadd_rn(__fsub_rn(a.x, av), __fsub_rn(b.x, bv));
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  const float h = __fadd_rn(s, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ double p2_add(double a, double b) { return a + b; }
__device__ __forceinline__ float p2_value(float2 a) { return __fadd_rn(a.x, a.y); }
__device__ __forceinline__ double p2_value(double a) { return a; }


// Current table in shared memory: segment (i..j), i <= j, of thread t at
// tab[(seg(i, j) * NT + t) * 4], four consecutive values (one 16-byte load in
// FP32), consecutive threads in consecutive slots; the prefix sums S_p of the
// ordered momenta in slots NSEG + p.
template <int N>
__host__ __device__ constexpr int comc_seg(int i, int j) {
  return i * (N - 1) - i * (i - 1) / 2 + (j - i);
}
// The loads are volatile so that the compiler keeps them in program order
// instead of hoisting the whole unrolled recursion's loads ahead of their use
// (which needs more than 255 registers and spills).
template <int NT>
__device__ __forceinline__ void tab_ld(const float* __restrict__ tab, int seg, float (&v)[4]) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(tab + (size_t)seg * NT * 4);
  asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
               : "r"(a));
}
template <int NT>
__device__ __forceinline__ void tab_st(float* __restrict__ tab, int seg, const float (&v)[4]) {
  *reinterpret_cast<float4*>(tab + (size_t)seg * NT * 4) = make_float4(v[0], v[1], v[2], v[3]);
}
template <int NT>
__device__ __forceinline__ void tab_ld(const double* __restrict__ tab, int seg, double (&v)[4]) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(tab + (size_t)seg * NT * 4);
  asm volatile("ld.volatile.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "r"(a));
  asm volatile("ld.volatile.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v[2]), "=d"(v[3]) : "r"(a + 16));
}
template <int NT>
__device__ __forceinline__ void tab_st(double* __restrict__ tab, int seg, const double (&v)[4]) {
  *reinterpret_cast<double2*>(tab + (size_t)seg * NT * 4) = make_double2(v[0], v[1]);
  *reinterpret_cast<double2*>(tab + (size_t)seg * NT * 4 + 2) = make_double2(v[2], v[3]);
}

// Bracket of segment (i..j) (the V3 and V4 sums before the propagator, unit
// vertex factors) from the shared-memory table: the same terms as the
// register form of the colour-ordered kernels, with the loop over the second
// split point outermost so that only the row J(i..s) stays in registers:
// J(t+1..j) is loaded once per t, the interior J(s+1..t) as it is used, and
// the coefficient of J(t+1..j) is complete (and applied) at the end of
// iteration t.
template <int N, typename T, int NT>
__device__ __forceinline__ void comc_bracket_tab(const T* __restrict__ tab, const int i, const int j, T (&br)[4]) {
  constexpr int M = N - 1, NSEG = M * (M + 1) / 2;
  T X[M][4];
#pragma unroll
  for (int s = i; s < j; ++s) tab_ld<NT>(tab, comc_seg<N>(i, s), X[s]);
  T Si[4], Sj[4], P2[4];
  tab_ld<NT>(tab, NSEG + i, Si);
  tab_ld<NT>(tab, NSEG + j + 1, Sj);
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
  tab_ld<NT>(tab, comc_seg<N>(i + 1, j), Z);
  tab_ld<NT>(tab, NSEG + i + 1, St);
#pragma unroll
  for (int t = i; t < j; ++t) {
    T Zn[4], Stn[4], Y[4];
    if (t + 1 < j) {
      tab_ld<NT>(tab, comc_seg<N>(t + 2, j), Zn);
      tab_ld<NT>(tab, NSEG + t + 2, Stn);
    }
    if (i < t) tab_ld<NT>(tab, comc_seg<N>(i + 1, t), Y);
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
      if (s + 1 < t) tab_ld<NT>(tab, comc_seg<N>(s + 2, t), Yn);
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

// Depth-first walk over the orders (0, g_1, ..., g_{N-1}) (0-based labels)
// whose colour chain closes: the row colour of each gluon equals the column
// colour of the gluon before it, and the column colour of the last gluon
// equals the row colour of gluon 0.  rm[c]: mask of the gluons with row
// colour c; cp: column colours, 2 bits per gluon.  Orders are visited in
// lexicographic order of their labels; visit(packed) gets the labels of
// positions 1..N-1 packed 4 bits each and returns false to pause the walk
// after that order.  The state (depth, candidates left per depth, labels
// chosen, gluons still free) can be saved and the walk resumed where it
// paused, so that an event whose orders span several windows is walked once
// in total.
template <int N>
struct ComcWalk {
  // All state in scalars (no dynamically indexed arrays, which would live in
  // local memory): the candidates left at depth d are the 16-bit lane d & 3
  // of word d >> 2 of c[0..2]; the label chosen at depth d is nibble d - 1
  // of `packed`.
  uint64_t packed;
  uint64_t c0, c1, c2;
  uint32_t avail;
  int d;

  __device__ __forceinline__ static uint32_t rmask(const uint32_t (&rm)[3], uint32_t colour) {
    return colour == 0u ? rm[0] : (colour == 1u ? rm[1] : rm[2]);
  }
  __device__ __forceinline__ uint32_t cand(int k) const {
    const uint64_t w = k < 4 ? c0 : (k < 8 ? c1 : c2);
    return (uint32_t)((w >> (16 * (k & 3))) & 0xFFFFull);
  }
  __device__ __forceinline__ void set_cand(int k, uint32_t v) {
    const int sh = 16 * (k & 3);
    const uint64_t m = ~(0xFFFFull << sh), x = (uint64_t)(v & 0xFFFFu) << sh;
    if (k < 4)
      c0 = (c0 & m) | x;
    else if (k < 8)
      c1 = (c1 & m) | x;
    else
      c2 = (c2 & m) | x;
  }

  __device__ __forceinline__ void start(const uint32_t (&rm)[3], uint32_t cp) {
    packed = 0;
    c0 = c1 = c2 = 0;
    avail = ((1u << N) - 1u) & ~1u;
    d = 1;
    set_cand(1, avail & rmask(rm, cp & 3u));
  }
  // Returns the number of orders visited before the walk ended or paused.
  template <typename F>
  __device__ __forceinline__ int64_t run(const uint32_t (&rm)[3], uint32_t cp, F&& visit) {
    const int r0 = (rm[0] & 1u) ? 0 : ((rm[1] & 1u) ? 1 : 2);
    int64_t cnt = 0;
    while (d > 0) {
      const uint32_t cd = cand(d);
      if (cd) {
        const int g = __ffs(cd) - 1;
        set_cand(d, cd & (cd - 1u));
        const uint64_t pk = (packed & ~(0xFull << (4 * (d - 1)))) | ((uint64_t)g << (4 * (d - 1)));
        if (d == N - 1) {
          if ((int)((cp >> (2 * g)) & 3u) == r0) {
            ++cnt;
            if (!visit(pk)) return cnt;
          }
          continue;
        }
        packed = pk;
        avail &= ~(1u << g);
        ++d;
        set_cand(d, avail & rmask(rm, (cp >> (2 * g)) & 3u));
      } else {
        --d;
        if (d > 0) avail |= 1u << (int)((packed >> (4 * (d - 1))) & 0xFull);
      }
    }
    return cnt;
  }
};

template <int N, typename T>
struct ComcSmem {
  using S = ComcShape<N, T>;
  using PT = typename ComcPair<T>::type;
  static constexpr size_t a16(size_t x) { return (x + 15) & ~size_t(15); }
  static constexpr size_t off_k = 0;                                                 // T [EB][N][4]
  static constexpr size_t off_e = off_k + sizeof(T) * S::EB * N * 4;                 // T [EB][N][4]
  static constexpr size_t off_pair = a16(off_e + sizeof(T) * S::EB * N * 4);         // PT [EB][NPAIR]
  static constexpr size_t off_item = a16(off_pair + sizeof(PT) * S::EB * S::NPAIR);  // u64 [CAP]
  static constexpr size_t off_amp = off_item + 8 * S::CAP;                            // T [CAP]
  static constexpr size_t off_acc = a16(off_amp + sizeof(T) * S::CAP);               // double [EB]
  static constexpr size_t off_off = off_acc + 8 * S::EB;                              // i64 [EB+1]
  static constexpr size_t off_cf = a16(off_off + 8 * (S::EB + 1));                   // u32 [EB][4]
  static constexpr size_t off_iev = off_cf + 16 * S::EB;                              // u16 [CAP]
  static constexpr size_t off_walk = a16(off_iev + 2 * S::CAP);                       // walk states [EB]
  static constexpr size_t off_tab = a16(off_walk + sizeof(ComcWalk<N>) * S::EB);       // T [NSLOT][NT][4] (TAB)
  static constexpr size_t bytes = off_tab + (S::TAB ? sizeof(T) * S::NSLOT * S::NT * 4 : 0);
};

// Colour-ordered amplitude A(g_0, ..., g_{N-1}) of one order with unit vertex
// factors (Eqs. 2.20-2.22).  ke, ee: the event's momenta and polarisations
// [N][4]; pr: its pair invariants [NPAIR] (a < b lexicographic).  Currents
// are built column by column (right end j ascending, left end i
// descending), so that the running sums P(i..j)^2 need one column of
// partial sums.
template <int N, typename T, typename PT>
__device__ __forceinline__ T comc_amplitude(uint64_t packed, const T* __restrict__ ke, const T* __restrict__ ee,
                                            const PT* __restrict__ pr) {
  constexpr int M = N - 1;
  int gl[N];
  gl[0] = 0;
#pragma unroll
  for (int pos = 1; pos < N; ++pos) gl[pos] = (int)((packed >> (4 * (pos - 1))) & 15u);
  T J[M][M][4];
  T Sp[N][4];
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
  }
  T en[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) en[m] = ee[gl[N - 1] * 4 + m];
  PT p2[M];
#pragma unroll
  for (int i = 0; i < M; ++i) p2_zero(p2[i]);
  T amp = T(0);
#pragma unroll
  for (int j = 1; j < M; ++j) {
    PT c;
    p2_zero(c);
#pragma unroll
    for (int i = j - 1; i >= 0; --i) {
      T br[4];
      co_bracket<N, T>(J, Sp, i, j, br);
      if (i == 0 && j == M - 1) {
        amp = mdot(en, br);
      } else {
        const int a = min(gl[i], gl[j]), b = max(gl[i], gl[j]);
        c = p2_add(c, pr[a * N - a * (a + 1) / 2 + (b - a - 1)]);
        p2[i] = p2_add(p2[i], c);
        const T ip = T(1) / T(p2_value(p2[i]));
        scale4(ip, br, J[i][j]);
      }
    }
  }
  return amp;
}

// The same with the current table in shared memory (tab: this thread's
// slice, see tab_ld).
template <int N, typename T, typename PT, int NT>
__device__ __forceinline__ T comc_amplitude_tab(uint64_t packed, const T* __restrict__ ke, const T* __restrict__ ee,
                                                const PT* __restrict__ pr, T* __restrict__ tab) {
  constexpr int M = N - 1, NSEG = M * (M + 1) / 2;
  int gl[N];
  gl[0] = 0;
#pragma unroll
  for (int pos = 1; pos < N; ++pos) gl[pos] = (int)((packed >> (4 * (pos - 1))) & 15u);
  {
    T S[4] = {T(0), T(0), T(0), T(0)};
    tab_st<NT>(tab, NSEG, S);
#pragma unroll
    for (int pos = 0; pos < M; ++pos) {
      const int g = gl[pos];
      T v[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        v[m] = ee[g * 4 + m];
        S[m] += ke[g * 4 + m];
      }
      tab_st<NT>(tab, comc_seg<N>(pos, pos), v);
      tab_st<NT>(tab, NSEG + pos + 1, S);
    }
  }
  PT p2[M];
#pragma unroll
  for (int i = 0; i < M; ++i) p2_zero(p2[i]);
  T amp = T(0);
#pragma unroll
  for (int j = 1; j < M; ++j) {
    PT c;
    p2_zero(c);
#pragma unroll
    for (int i = j - 1; i >= 0; --i) {
      T br[4];
      comc_bracket_tab<N, T, NT>(tab, i, j, br);
      if (i == 0 && j == M - 1) {
        T en[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) en[m] = ee[gl[N - 1] * 4 + m];
        amp = mdot(en, br);
      } else {
        const int a = min(gl[i], gl[j]), b = max(gl[i], gl[j]);
        c = p2_add(c, pr[a * N - a * (a + 1) / 2 + (b - a - 1)]);
        p2[i] = p2_add(p2[i], c);
        const T ip = T(1) / T(p2_value(p2[i]));
        T J[4];
        scale4(ip, br, J);
        tab_st<NT>(tab, comc_seg<N>(i, j), J);
      }
      // table values are reloaded by each segment rather than kept live in
      // registers across segments (which would spill)
      asm volatile("" ::: "memory");
    }
  }
  return amp;
}

template <int N, typename T>
__global__ void __launch_bounds__(ComcShape<N, T>::NT)
    comc_kernel(ComcParams prm, const double* __restrict__ p, const int8_t* __restrict__ hel,
                const int8_t* __restrict__ col, const uint8_t* __restrict__ accept, PolFrame F,
                double* __restrict__ me2, int* __restrict__ status) {
  using S = ComcShape<N, T>;
  using L = ComcSmem<N, T>;
  using PT = typename ComcPair<T>::type;
  constexpr int EB = S::EB, NT = S::NT, CAP = S::CAP, NPAIR = S::NPAIR;
  const int64_t S_ = prm.B;
  const int64_t B = prm.dB ? (*prm.dB < S_ ? *prm.dB : S_) : S_;
  const int64_t e0 = (int64_t)blockIdx.x * EB;
  if (e0 >= B) return;
  extern __shared__ __align__(16) unsigned char smem[];
  T* s_k = reinterpret_cast<T*>(smem + L::off_k);
  T* s_e = reinterpret_cast<T*>(smem + L::off_e);
  PT* s_pair = reinterpret_cast<PT*>(smem + L::off_pair);
  uint64_t* s_item = reinterpret_cast<uint64_t*>(smem + L::off_item);
  T* s_amp = reinterpret_cast<T*>(smem + L::off_amp);
  double* s_acc = reinterpret_cast<double*>(smem + L::off_acc);
  long long* s_off = reinterpret_cast<long long*>(smem + L::off_off);
  uint32_t* s_cf = reinterpret_cast<uint32_t*>(smem + L::off_cf);
  uint16_t* s_iev = reinterpret_cast<uint16_t*>(smem + L::off_iev);
  ComcWalk<N>* s_walk = reinterpret_cast<ComcWalk<N>*>(smem + L::off_walk);
  const int tid = threadIdx.x;

  // ---- 1. momenta, polarisations, pair invariants, colour flows
  for (int it = tid; it < EB * N; it += NT) {
    const int el = it / N, g = it % N;
    const int64_t e = e0 + el;
    if (e >= B) continue;
    double k[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) k[m] = p[((int64_t)m * N + g) * S_ + e] * prm.inv_sqrt_s;
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
  for (int it = tid; it < EB * NPAIR; it += NT) {
    const int el = it / NPAIR;
    int pr = it % NPAIR;
    const int64_t e = e0 + el;
    if (e >= B) continue;
    int a = 0;
    while (pr >= N - 1 - a) {
      pr -= N - 1 - a;
      ++a;
    }
    const int b = a + 1 + pr;
    double ka[4], kb[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      ka[m] = p[((int64_t)m * N + a) * S_ + e];
      kb[m] = p[((int64_t)m * N + b) * S_ + e];
    }
    const double sgn = ((a < 2) != (b < 2)) ? -1.0 : 1.0;  // k = -p for gluons 1, 2
    const double v =
        sgn * 2.0 * (ka[0] * kb[0] - ka[1] * kb[1] - ka[2] * kb[2] - ka[3] * kb[3]) * prm.inv_sqrt_s * prm.inv_sqrt_s;
    p2_split(v, s_pair[el * NPAIR + it % NPAIR]);
  }
  for (int el = tid; el < EB; el += NT) {
    const int64_t e = e0 + el;
    uint32_t rm0 = 0, rm1 = 0, rm2 = 0, cp = 0, ok = e < B ? 1u : 0u;
    if (ok && accept != nullptr && accept[e] == 0) ok = 0;
    if (e < B) {
      for (int g = 0; g < N; ++g) {
        const int rr = col[(int64_t)(2 * g) * S_ + e], cc = col[(int64_t)(2 * g + 1) * S_ + e];
        if (rr < 1 || rr > 3 || cc < 1 || cc > 3) {
          flag_status(status, BG_EINVAL);
          ok = 0;
          continue;
        }
        const uint32_t bit = 1u << g;
        rm0 |= rr == 1 ? bit : 0u;
        rm1 |= rr == 2 ? bit : 0u;
        rm2 |= rr == 3 ? bit : 0u;
        cp |= (uint32_t)(cc - 1) << (2 * g);
      }
    }
    // a chain can close only if every colour is as often a row as a column
    // colour: other flows have no closing order and are not walked
    uint32_t bal = 1;
    if (ok) {
      int nc[3] = {0, 0, 0};
      for (int g = 0; g < N; ++g) ++nc[(cp >> (2 * g)) & 3u];
      bal = (__popc(rm0) == nc[0] && __popc(rm1) == nc[1] && __popc(rm2) == nc[2]) ? 1u : 0u;
    }
    s_cf[el * 4 + 0] = rm0;
    s_cf[el * 4 + 1] = rm1;
    s_cf[el * 4 + 2] = rm2;
    s_cf[el * 4 + 3] = cp | (ok << 30) | (bal << 29);
  }
  __syncthreads();

  // ---- 2. count the orders of each event, then a scan over the tile
  for (int el = tid; el < EB; el += NT) {
    const uint32_t rm[3] = {s_cf[el * 4 + 0], s_cf[el * 4 + 1], s_cf[el * 4 + 2]};
    const uint32_t w = s_cf[el * 4 + 3];
    int64_t cnt = 0;
    if (((w >> 30) & 1u) && ((w >> 29) & 1u)) {
      ComcWalk<N> wk;
      wk.start(rm, w & 0x00FFFFFFu);
      cnt = wk.run(rm, w & 0x00FFFFFFu, [](uint64_t) { return true; });
    }
    s_off[el + 1] = (long long)cnt;
    s_acc[el] = 0.0;
  }
  __syncthreads();
  if (tid < 32) {
    long long carry = 0;
    for (int base = 0; base < EB; base += 32) {
      const int el = base + tid;
      long long v = el < EB ? s_off[el + 1] : 0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, v, d);
        if (tid >= d) v += u;
      }
      if (el < EB) s_off[el + 1] = carry + v;
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
    if (tid == 0) s_off[0] = 0;
  }
  __syncthreads();
  const long long total = s_off[EB];

  // ---- 3. windows of CAP items: write the orders, evaluate, accumulate
  for (long long w0 = 0; w0 < total; w0 += CAP) {
    const long long w1 = (total - w0 < CAP) ? total : w0 + CAP;
    for (int el = tid; el < EB; el += NT) {
      // (events without items -- failing the cut, invalid or without a
      // closing order -- have lo == hi and are not walked)
      const long long lo = s_off[el], hi = s_off[el + 1];
      if (hi <= lo || hi <= w0 || lo >= w1) continue;
      // the event's orders lo + r, r = 0, 1, ..., are written from where its
      // walk paused at the end of the previous window
      const long long stop = hi < w1 ? hi : w1;
      const uint32_t rm[3] = {s_cf[el * 4 + 0], s_cf[el * 4 + 1], s_cf[el * 4 + 2]};
      const uint32_t cp = s_cf[el * 4 + 3] & 0x00FFFFFFu;
      ComcWalk<N> wk;
      if (lo >= w0) {
        wk.start(rm, cp);
      } else {
        wk = s_walk[el];
      }
      long long g = lo > w0 ? lo : w0;
      wk.run(rm, cp, [&](uint64_t pk) {
        s_item[g - w0] = pk;
        s_iev[g - w0] = (uint16_t)el;
        ++g;
        return g < stop;
      });
      if (hi > w1) s_walk[el] = wk;
    }
    __syncthreads();
    const int nw = (int)(w1 - w0);
    for (int it = tid; it < nw; it += NT) {
      const int el = s_iev[it];
      if constexpr (S::TAB)
        s_amp[it] = comc_amplitude_tab<N, T, PT, NT>(s_item[it], s_k + el * N * 4, s_e + el * N * 4,
                                                     s_pair + el * NPAIR,
                                                     reinterpret_cast<T*>(smem + L::off_tab) + tid * 4);
      else
        s_amp[it] = comc_amplitude<N, T, PT>(s_item[it], s_k + el * N * 4, s_e + el * N * 4, s_pair + el * NPAIR);
    }
    __syncthreads();
    for (int el = tid; el < EB; el += NT) {
      const long long lo = s_off[el] > w0 ? s_off[el] : w0;
      const long long hi = s_off[el + 1] < w1 ? s_off[el + 1] : w1;
      double a = s_acc[el];
      for (long long g = lo; g < hi; ++g) a += (double)s_amp[g - w0];
      s_acc[el] = a;
    }
    __syncthreads();
  }

  // ---- 4. |M|^2
  for (int el = tid; el < EB; el += NT) {
    const int64_t e = e0 + el;
    if (e >= B) continue;
    const double a = s_acc[el];
    me2[e] = ((s_cf[el * 4 + 3] >> 30) & 1u) ? prm.scale * a * a : 0.0;
  }
}

template <int N, typename T>
cudaError_t launch_comc_n(const ComcParams& prm, const double* p, const int8_t* hel, const int8_t* col,
                          const uint8_t* accept, const double* q, double* me2, int* status, cudaStream_t s) {
  using S = ComcShape<N, T>;
  using L = ComcSmem<N, T>;
  static_assert(L::bytes <= 200 * 1024, "shared memory of the colour-flow kernel");
  auto kern = comc_kernel<N, T>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
  if (err != cudaSuccess) return err;
  const PolFrame F = make_pol_frame(q);
  const int64_t blocks = (prm.B + S::EB - 1) / S::EB;
  kern<<<(unsigned)blocks, S::NT, L::bytes, s>>>(prm, p, hel, col, accept, F, me2, status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_comc_t(int n, const ComcParams& prm, const double* p, const int8_t* hel, const int8_t* col,
                          const uint8_t* accept, const double* q, double* me2, int* status, cudaStream_t s) {
  switch (n) {
    case 4: return launch_comc_n<4, T>(prm, p, hel, col, accept, q, me2, status, s);
    case 5: return launch_comc_n<5, T>(prm, p, hel, col, accept, q, me2, status, s);
    case 6: return launch_comc_n<6, T>(prm, p, hel, col, accept, q, me2, status, s);
    case 7: return launch_comc_n<7, T>(prm, p, hel, col, accept, q, me2, status, s);
    case 8: return launch_comc_n<8, T>(prm, p, hel, col, accept, q, me2, status, s);
    case 9: return launch_comc_n<9, T>(prm, p, hel, col, accept, q, me2, status, s);
    case 10: return launch_comc_n<10, T>(prm, p, hel, col, accept, q, me2, status, s);
    case 11: return launch_comc_n<11, T>(prm, p, hel, col, accept, q, me2, status, s);
    case 12: return launch_comc_n<12, T>(prm, p, hel, col, accept, q, me2, status, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bg
