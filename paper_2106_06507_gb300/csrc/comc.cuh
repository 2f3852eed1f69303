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
// very unevenly (at n = 12 about 3 % of the flows have any, those a few
// thousand on average and up to ~10^5).
//
// Every closing order of every event is one work item, so that the orders of
// a heavy event spread over the whole GPU:
//   1. comc_prep_kernel (a block per 256 events): each event's record --
//      scaled momenta, sampled polarisation vectors and the pair invariants
//      2 k_a.k_b of all pairs of gluons, computed in FP64 and kept as an
//      unevaluated sum of two floats in the FP32 kernel (FP64 in the FP64
//      kernel) -- its colour masks, and its number of closing orders (BEST
//      theorem, comc_rank.h); a block-wide scan of the counts;
//   2. comc_scan_kernel, comc_offsets_kernel: the events' item offsets
//      off[e] (exclusive prefix sums of the counts, off[B] the total) and the
//      chunk size CH (a multiple of the evaluator's block size, with at most
//      kComcMaxChunks chunks);
//   3. comc_eval_kernel, persistent: the blocks take the chunks of CH items
//      round-robin and their threads one item each per pass: the item's
//      event (galloping search from the event of the pass's first item), the
//      order of the item's rank in its event (comc_unrank), and the whole
//      recursion of that order.  The amplitudes of an event are added in
//      item order within the chunk; an event that a chunk boundary cuts
//      leaves the partial sum of its part of the chunk in one of the chunk's
//      two slots (first: the event that began before the chunk; last: the
//      event that goes on after it);
//   4. comc_final_kernel, one thread per event: the event's sum (from its
//      chunk, or its partial sums in chunk order) and |M|^2.
// The sums run in a fixed order: equal inputs give equal bits.
// The propagator denominators P(i..j)^2 of each order are accumulated from
// the pair invariants column by column, P(i..j)^2 = P(i..j-1)^2 +
// sum_{a=i}^{j-1} 2 k_{s_a}.k_{s_j}, in double-float arithmetic (Knuth's
// TwoSum, TAOCP vol. 2, 4.2.2) in the FP32 kernel: a plain FP32 sum of the
// invariants, or E^2 - |p|^2 of the FP32 momentum sum, loses up to ~1e-3 of
// P^2 to cancellation between incoming and outgoing momenta.
#pragma once

#include "bg_internal.h"
#include "co_recursion.cuh"
#include "comc_rank.h"
#include "cur_table.cuh"
#include "device_common.cuh"

namespace bg {

struct ComcParams {
  int64_t B;  // events (row stride of p, hel, colours)
  double inv_sqrt_s;
  double scale;  // 9^n 2^n g^(2n-4) sqrt_s^(8-2n) 2^-(n-2)
};

// At most this many chunks per launch (2 partial-sum slots each in the
// workspace); chunks grow beyond the evaluator's block size only past
// kComcMaxChunks x block size items.
constexpr int64_t kComcMaxChunks = 1 << 16;
constexpr int kComcPrepEvents = 256;

// TAB (n >= 10; FP64 from n = 8): the current table of the order being
// evaluated lives in shared memory (one slice per thread) instead of
// registers: a register table of 4 n(n-1)/2 values spills there, and the
// spilled stacks of the resident threads outgrow L1.
template <int N, typename T>
struct ComcShape {
  static constexpr bool TAB = N >= 10 || (sizeof(T) == 8 && N >= 8);
  // 64 threads with the shared-memory table: two blocks per SM, so that one
  // block's serial phases (the run sums) overlap the other's recursions
  static constexpr int NT = TAB ? 64 : 128;
  static constexpr int M = N - 1;
  static constexpr int NPAIR = N * (N - 1) / 2;
  // LEAF: the one-gluon currents are read from the event's record rather
  // than kept in the table (FP32 n = 10: a smaller table, one more resident
  // block per SM, 11 % faster; at n = 11, 12 the extra block's local-memory
  // stack outgrows L1 and it is slower)
  static constexpr bool LEAF = TAB && sizeof(T) == 4 && N == 10;
  static constexpr int NSEGT = LEAF ? M * (M - 1) / 2 : M * (M + 1) / 2;  // segments (i..j) in the table
  static constexpr int NSLOT = NSEGT + N;  // + prefix sums S_0..S_M of the ordered momenta
  static constexpr size_t tab_bytes = TAB ? sizeof(T) * NSLOT * NT * 4 : 0;
};

// The record of one event in the workspace: momenta k [N][4] and
// polarisations e [N][4] (type T), then the pair invariants [NPAIR] (a < b
// lexicographic; float2 value + error in FP32, double in FP64: 8 bytes each).
__host__ __device__ constexpr size_t comc_record_bytes(int n, size_t t_size) {
  return (2 * t_size * (size_t)n * 4 + 8 * (size_t)(n * (n - 1) / 2) + 15) & ~size_t(15);
}

// Workspace (caller-owned device memory, 256-byte aligned), carved in this
// order with 256-byte alignment between the arrays.
struct ComcWorkspace {
  long long* off;      // [B + 1] item offsets of the events
  long long* meta;     // [4]: total items, chunk size CH
  long long* bsum;     // [ceil(B / 256)] per-prep-block sums, then their exclusive prefix
  double* acc;         // [B] sums of the events that lie within one chunk
  double* part;        // [2 kComcMaxChunks] per chunk: first and last partial sums
  uint4* hdr;          // [B] colour masks (ComcFlow packed)
  unsigned char* rec;  // [B] records of comc_record_bytes(n) bytes
};

inline size_t comc_workspace_bytes(int n, int64_t B, size_t t_size, unsigned char* base = nullptr,
                                   ComcWorkspace* w = nullptr) {
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t nb = (size_t)((B + kComcPrepEvents - 1) / kComcPrepEvents);
  size_t o = 0;
  const size_t o_off = o;
  o = up(o + 8 * (size_t)(B + 1));
  const size_t o_meta = o;
  o = up(o + 8 * 4);
  const size_t o_bsum = o;
  o = up(o + 8 * (nb + 1));
  const size_t o_acc = o;
  o = up(o + 8 * (size_t)B);
  const size_t o_part = o;
  o = up(o + 8 * 2 * (size_t)kComcMaxChunks);
  const size_t o_hdr = o;
  o = up(o + 16 * (size_t)B);
  const size_t o_rec = o;
  o = up(o + comc_record_bytes(n, t_size) * (size_t)B);
  if (w && base) {
    w->off = reinterpret_cast<long long*>(base + o_off);
    w->meta = reinterpret_cast<long long*>(base + o_meta);
    w->bsum = reinterpret_cast<long long*>(base + o_bsum);
    w->acc = reinterpret_cast<double*>(base + o_acc);
    w->part = reinterpret_cast<double*>(base + o_part);
    w->hdr = reinterpret_cast<uint4*>(base + o_hdr);
    w->rec = base + o_rec;
  }
  return o;
}

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
template <int N, typename T, typename PT, int NT, bool LEAF>
__device__ __forceinline__ T comc_amplitude_tab(uint64_t packed, const T* __restrict__ ke, const T* __restrict__ ee,
                                                const PT* __restrict__ pr, T* __restrict__ tab) {
  constexpr int M = N - 1, SP0 = tab_nseg<N, LEAF>();
  int gl[N];
  gl[0] = 0;
#pragma unroll
  for (int pos = 1; pos < N; ++pos) gl[pos] = (int)((packed >> (4 * (pos - 1))) & 15u);
  {
    T S[4] = {T(0), T(0), T(0), T(0)};
    tab_st<NT>(tab, SP0, S);
#pragma unroll
    for (int pos = 0; pos < M; ++pos) {
      const int g = gl[pos];
#pragma unroll
      for (int m = 0; m < 4; ++m) S[m] += ke[g * 4 + m];
      if (!LEAF) {
        T v[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) v[m] = ee[g * 4 + m];
        tab_st<NT>(tab, tab_seg<N, LEAF>(pos, pos), v);
      }
      tab_st<NT>(tab, SP0 + pos + 1, S);
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
      tab_bracket<N, T, NT, LEAF>(tab, ee, gl, i, j, br);
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
        tab_st<NT>(tab, tab_seg<N, LEAF>(i, j), J);
      }
      // table values are reloaded by each segment rather than kept live in
      // registers across segments (which would spill)
      asm volatile("" ::: "memory");
    }
  }
  return amp;
}


__device__ __forceinline__ ComcFlow comc_decode(uint4 h) {
  ComcFlow f;
  f.rm0 = h.x & 0xFFFFu;
  f.rm1 = h.x >> 16;
  f.rm2 = h.y & 0xFFFFu;
  f.cm0 = h.y >> 16;
  f.cm1 = h.z & 0xFFFFu;
  f.cm2 = h.z >> 16;
  f.r0 = (int)(h.w & 3u);
  f.c0 = (int)((h.w >> 2) & 3u);
  return f;
}

__device__ __forceinline__ void comc_fact_table(uint32_t* s_fact) {
  if (threadIdx.x < 12) {
    uint32_t f = 1;
    for (int k = 2; k <= (int)threadIdx.x; ++k) f *= (uint32_t)k;
    s_fact[threadIdx.x] = f;
  }
}

// Inclusive scan of v over the warp.
__device__ __forceinline__ long long comc_warp_scan(long long v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long u = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += u;
  }
  return v;
}

// ---- 1. records, colour masks, counts; block-local inclusive scan
template <int N, typename T>
__global__ void __launch_bounds__(kComcPrepEvents)
    comc_prep_kernel(ComcParams prm, const double* __restrict__ p, const int8_t* __restrict__ hel,
                     const int8_t* __restrict__ col, const uint8_t* __restrict__ accept, PolFrame F, ComcWorkspace w,
                     int* __restrict__ status) {
  using PT = typename ComcPair<T>::type;
  constexpr int EB = kComcPrepEvents, NPAIR = N * (N - 1) / 2;
  constexpr size_t RB = comc_record_bytes(N, sizeof(T));
  const int64_t B = prm.B;
  const int64_t e0 = (int64_t)blockIdx.x * EB;
  const int tid = threadIdx.x;
  __shared__ uint32_t s_fact[12];
  __shared__ long long s_wsum[EB / 32];
  comc_fact_table(s_fact);

  for (int it = tid; it < EB * N; it += EB) {
    const int el = it / N, g = it % N;
    const int64_t e = e0 + el;
    if (e >= B) continue;
    double k[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) k[m] = p[((int64_t)m * N + g) * B + e] * prm.inv_sqrt_s;
    if (g < 2) {
#pragma unroll
      for (int m = 0; m < 4; ++m) k[m] = -k[m];
    }
    const int h = hel[(int64_t)g * B + e];
    if (h != 1 && h != -1) flag_status(status, BG_EINVAL);
    T ev[4];
    lc_polarisation_frame<T>(k, F, h >= 0, ev);
    T* rk = reinterpret_cast<T*>(w.rec + (size_t)e * RB);
    T* re = rk + N * 4;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      rk[g * 4 + m] = T(k[m]);
      re[g * 4 + m] = ev[m];
    }
  }
  for (int it = tid; it < EB * NPAIR; it += EB) {
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
      ka[m] = p[((int64_t)m * N + a) * B + e];
      kb[m] = p[((int64_t)m * N + b) * B + e];
    }
    const double sgn = ((a < 2) != (b < 2)) ? -1.0 : 1.0;  // k = -p for gluons 1, 2
    const double v =
        sgn * 2.0 * (ka[0] * kb[0] - ka[1] * kb[1] - ka[2] * kb[2] - ka[3] * kb[3]) * prm.inv_sqrt_s * prm.inv_sqrt_s;
    PT* rp = reinterpret_cast<PT*>(w.rec + (size_t)e * RB + 2 * sizeof(T) * N * 4);
    p2_split(v, rp[it % NPAIR]);
  }
  __syncthreads();

  const int64_t e = e0 + tid;
  long long cnt = 0;
  if (e < B) {
    ComcFlow f{0u, 0u, 0u, 0u, 0u, 0u, 0, 0};
    bool ok = accept == nullptr || accept[e] != 0;
    for (int g = 0; g < N; ++g) {
      const int rr = col[(int64_t)(2 * g) * B + e], cc = col[(int64_t)(2 * g + 1) * B + e];
      if (rr < 1 || rr > 3 || cc < 1 || cc > 3) {
        flag_status(status, BG_EINVAL);
        ok = false;
        continue;
      }
      if (g == 0) {
        f.r0 = rr - 1;
        f.c0 = cc - 1;
        continue;
      }
      const uint32_t bit = 1u << g;
      f.rm0 |= rr == 1 ? bit : 0u;
      f.rm1 |= rr == 2 ? bit : 0u;
      f.rm2 |= rr == 3 ? bit : 0u;
      f.cm0 |= cc == 1 ? bit : 0u;
      f.cm1 |= cc == 2 ? bit : 0u;
      f.cm2 |= cc == 3 ? bit : 0u;
    }
    // a chain can close only if every colour is as often a row as a column
    // colour (the BEST count assumes it)
    if (ok && comc_balanced(f)) cnt = (long long)comc_count(f, s_fact);
    w.hdr[e] = make_uint4(f.rm0 | (f.rm1 << 16), f.rm2 | (f.cm0 << 16), f.cm1 | (f.cm2 << 16),
                          (uint32_t)f.r0 | ((uint32_t)f.c0 << 2));
  }
  long long v = comc_warp_scan(cnt);
  if ((tid & 31) == 31) s_wsum[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    long long u = tid < EB / 32 ? s_wsum[tid] : 0;
    u = comc_warp_scan(u);
    if (tid < EB / 32) s_wsum[tid] = u;
  }
  __syncthreads();
  if (tid >= 32) v += s_wsum[(tid >> 5) - 1];
  if (e < B) w.off[e + 1] = v;
  if (tid == EB - 1) w.bsum[blockIdx.x] = v;
}

// (The kernels below that are not templates have internal linkage: this
// header is compiled into several translation units.)

// ---- 2a. exclusive prefix of the per-block sums (one block of 1024
// threads), the total and the chunk size
static __global__ void __launch_bounds__(1024)
    comc_scan_kernel(long long* __restrict__ bsum, int64_t nb, long long* __restrict__ meta, int nt) {
  __shared__ long long s_w[32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  long long carry = 0;
  for (int64_t base = 0; base < nb; base += 1024) {
    const int64_t i = base + tid;
    const long long v = i < nb ? bsum[i] : 0;
    const long long x = comc_warp_scan(v);
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) s_w[lane] = comc_warp_scan(s_w[lane]);
    __syncthreads();
    const long long incl = x + (warp ? s_w[warp - 1] : 0) + carry;
    if (i < nb) bsum[i] = incl - v;
    carry += s_w[31];
    __syncthreads();
  }
  if (tid == 0) {
    const long long per = (carry + kComcMaxChunks - 1) / kComcMaxChunks;
    long long ch = ((per + nt - 1) / nt) * nt;
    if (ch < nt) ch = nt;
    meta[0] = carry;
    meta[1] = ch;
  }
}

// ---- 2b. global offsets
static __global__ void __launch_bounds__(kComcPrepEvents)
    comc_offsets_kernel(long long* __restrict__ off, const long long* __restrict__ bsum, int64_t B) {
  const int64_t e = (int64_t)blockIdx.x * kComcPrepEvents + threadIdx.x;
  if (e < B) off[e + 1] += bsum[blockIdx.x];
  if (e == 0) off[0] = 0;
}

// Largest e in [lo, B) with off[e] <= g, i.e. the event of item g, given
// off[lo] <= g < off[B]: galloping from lo, then bisection.
__device__ __forceinline__ long long comc_find_event(const long long* __restrict__ off, long long B, long long g,
                                                     long long lo) {
  long long step = 1, hi = lo + 1;
  while (hi < B && off[hi] <= g) {
    lo = hi;
    step <<= 1;
    hi = lo + step;
  }
  if (hi > B) hi = B;
  while (hi - lo > 1) {
    const long long mid = (lo + hi) >> 1;
    if (off[mid] <= g)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// ---- 3. the items, chunk by chunk
template <int N, typename T>
__global__ void __launch_bounds__(ComcShape<N, T>::NT)
    comc_eval_kernel(ComcWorkspace w, int64_t B, int* __restrict__ status) {
  using S = ComcShape<N, T>;
  using PT = typename ComcPair<T>::type;
  constexpr int NT = S::NT;
  constexpr size_t RB = comc_record_bytes(N, sizeof(T));
  extern __shared__ __align__(16) unsigned char smem[];  // current tables (TAB)
  __shared__ T s_amp[NT];
  __shared__ long long s_ev[NT];
  __shared__ uint64_t s_pk[NT];
  __shared__ uint32_t s_fact[12];
  __shared__ long long s_e0;
  __shared__ double s_carry[2];
  __shared__ long long s_carry_ev[2];
  const int tid = threadIdx.x;
  comc_fact_table(s_fact);
  const long long total = w.meta[0], CH = w.meta[1];
  int par = 0;
  for (long long c = blockIdx.x; c * CH < total; c += gridDim.x) {
    const long long c0 = c * CH, c1 = (total - c0 < CH) ? total : c0 + CH;
    if (tid == 0) {
      s_e0 = comc_find_event(w.off, B, c0, 0);
      s_carry_ev[par] = -1;
    }
    __syncthreads();
    // passes of NT items: the sum phase of a pass reads the carry of slot
    // par (the run of an event continuing from the previous pass) and writes
    // slot par ^ 1
    for (long long w0 = c0; w0 < c1; w0 += NT) {
      const int nw = (c1 - w0 < NT) ? (int)(c1 - w0) : NT;
      long long e = -1;
      T amp = T(0);
      if (tid == 0) s_carry_ev[par ^ 1] = -1;
      // the item's event and order first, then (after a barrier) its
      // recursion: with the two back to back in one thread the FP32 n = 12
      // kernel gave wrong amplitudes for a tenth of the items.  Only the form
      // with the asm table loads did (plain or volatile C++ loads were right,
      // and slower); the cause was not found, and every variant that
      // separates the two steps agrees with the oracle.
      if (tid < nw) {
        const long long g = w0 + tid;
        e = comc_find_event(w.off, B, g, s_e0);
        s_pk[tid] = comc_unrank<N>((uint32_t)(g - w.off[e]), comc_decode(w.hdr[e]), s_fact);
      }
      __syncthreads();
      if (tid < nw) {
        const uint64_t pk = s_pk[tid];
        if (pk == ~0ull) {
          flag_status(status, BG_ECUDA);  // cannot happen: ranks lie below the count
        } else {
          const T* ke = reinterpret_cast<const T*>(w.rec + (size_t)e * RB);
          const T* ee = ke + N * 4;
          const PT* pr = reinterpret_cast<const PT*>(w.rec + (size_t)e * RB + 2 * sizeof(T) * N * 4);
          if constexpr (S::TAB)
            amp = comc_amplitude_tab<N, T, PT, NT, S::LEAF>(pk, ke, ee, pr, reinterpret_cast<T*>(smem) + tid * 4);
          else
            amp = comc_amplitude<N, T, PT>(pk, ke, ee, pr);
        }
      }
      s_amp[tid] = amp;
      s_ev[tid] = e;
      __syncthreads();
      // one thread per run of equal events adds the run in item order
      if (tid < nw && (tid == 0 || s_ev[tid - 1] != e)) {
        double a = (tid == 0 && s_carry_ev[par] == e) ? s_carry[par] : 0.0;
        int i = tid;
        for (; i < nw && s_ev[i] == e; ++i) a += (double)s_amp[i];
        const long long end = w0 + i, lo = w.off[e], hi = w.off[e + 1];
        if (hi <= end) {  // the event ends in this pass
          if (lo >= c0)
            w.acc[e] = a;
          else
            w.part[2 * c] = a;
        } else if (end < c1) {  // it goes on in the next pass of this chunk
          s_carry[par ^ 1] = a;
          s_carry_ev[par ^ 1] = e;
        } else {  // it goes on in the next chunk
          w.part[2 * c + (lo >= c0 ? 1 : 0)] = a;
        }
      }
      if (tid == 0) s_e0 = s_ev[nw - 1];
      par ^= 1;
      __syncthreads();
    }
  }
}

// ---- 4. per event: the sum and |M|^2
static __global__ void __launch_bounds__(256)
    comc_final_kernel(ComcWorkspace w, int64_t B, double scale, double* __restrict__ me2) {
  const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (e >= B) return;
  const long long lo = w.off[e], hi = w.off[e + 1];
  double a = 0.0;
  if (hi > lo) {
    const long long CH = w.meta[1];
    const long long cl = lo / CH, ch = (hi - 1) / CH;
    if (cl == ch) {
      a = w.acc[e];
    } else {
      a = w.part[2 * cl + 1];
      for (long long c = cl + 1; c <= ch; ++c) a += w.part[2 * c];
    }
  }
  me2[e] = scale * a * a;
}

template <int N, typename T>
cudaError_t launch_comc_n(const ComcParams& prm, const double* p, const int8_t* hel, const int8_t* col,
                          const uint8_t* accept, const double* q, double* me2, void* workspace, int sms, int* status,
                          cudaStream_t s) {
  using S = ComcShape<N, T>;
  static_assert(S::tab_bytes + S::NT * (sizeof(T) + 8) + 256 <= 227 * 1024, "shared memory of the colour-flow kernel");
  ComcWorkspace w;
  comc_workspace_bytes(N, prm.B, sizeof(T), static_cast<unsigned char*>(workspace), &w);
  const PolFrame F = make_pol_frame(q);
  const int64_t nb = (prm.B + kComcPrepEvents - 1) / kComcPrepEvents;
  comc_prep_kernel<N, T><<<(unsigned)nb, kComcPrepEvents, 0, s>>>(prm, p, hel, col, accept, F, w, status);
  comc_scan_kernel<<<1, 1024, 0, s>>>(w.bsum, nb, w.meta, S::NT);
  comc_offsets_kernel<<<(unsigned)nb, kComcPrepEvents, 0, s>>>(w.off, w.bsum, prm.B);
  auto kern = comc_eval_kernel<N, T>;
  static int occ = 0;
  if (occ == 0) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::tab_bytes);
    if (err != cudaSuccess) return err;
    int o = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, S::NT, S::tab_bytes);
    if (err != cudaSuccess) return err;
    occ = o > 0 ? o : 1;
  }
  kern<<<(unsigned)(sms * occ), S::NT, S::tab_bytes, s>>>(w, prm.B, status);
  comc_final_kernel<<<(unsigned)((prm.B + 255) / 256), 256, 0, s>>>(w, prm.B, prm.scale, me2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_comc_t(int n, const ComcParams& prm, const double* p, const int8_t* hel, const int8_t* col,
                          const uint8_t* accept, const double* q, double* me2, void* workspace, int sms, int* status,
                          cudaStream_t s) {
  switch (n) {
    case 4: return launch_comc_n<4, T>(prm, p, hel, col, accept, q, me2, workspace, sms, status, s);
    case 5: return launch_comc_n<5, T>(prm, p, hel, col, accept, q, me2, workspace, sms, status, s);
    case 6: return launch_comc_n<6, T>(prm, p, hel, col, accept, q, me2, workspace, sms, status, s);
    case 7: return launch_comc_n<7, T>(prm, p, hel, col, accept, q, me2, workspace, sms, status, s);
    case 8: return launch_comc_n<8, T>(prm, p, hel, col, accept, q, me2, workspace, sms, status, s);
    case 9: return launch_comc_n<9, T>(prm, p, hel, col, accept, q, me2, workspace, sms, status, s);
    case 10: return launch_comc_n<10, T>(prm, p, hel, col, accept, q, me2, workspace, sms, status, s);
    case 11: return launch_comc_n<11, T>(prm, p, hel, col, accept, q, me2, workspace, sms, status, s);
    case 12: return launch_comc_n<12, T>(prm, p, hel, col, accept, q, me2, workspace, sms, status, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bg
