// cd_recursion.cuh -- colour-dressed Berends-Giele recursion with sampled
// colours, Eqs. (2.28)-(2.32) of the paper, on the GPU.
//
// Currents are 3x3 colour matrices (colour-flow basis) of Lorentz vectors
// (gluon, Eq. 2.28) and of antisymmetric tensors (the auxiliary field of
// Eqs. 2.23-2.26), one per subset S of the first m = n-1 gluons.  With the
// sum over partitions with both colour orders (vertex 2.30) written as the
// sum over ordered partitions (S1, S2) and the colour product J(S1) J(S2):
//   br(S)_rc = sum_{(S1,S2)} sum_l [ V3(P1, P2; J1_rl, J2_lc)
//                                   + T2_lc . J1_rl + J2_lc . T1_rl ]
//   T(S)_rc  = sum_{(S1,S2)} sum_l J1_rl ^ J2_lc
//   J(S) = br(S) / P(S)^2,   A = sum_rc (E_n)_cr e_n . br(full)_rc,
// with unit vertex factors (the couplings (1/sqrt2)^(n-2) are applied to A).
// V3 uses current conservation: (X.Y)(P1 - P2) + 2(P.X)Y - 2(P.Y)X.
//
// Work decomposition.  Persistent CTAs fetch events from a global counter
// (dynamic scheduling: events rejected by the cut cost almost nothing, and
// the CTAs stay balanced).  A CTA evaluates one event at a time, subsets
// level by level (by size).  A task is (subset, chunk of its ordered
// partitions, colour row r) and computes the three entries (r, c) of the
// row: it reuses each left sub-current entry (r, l) for three products, and
// the three threads of one (subset, chunk), r fastest, walk the same
// partitions, so that their loads of the right sub-current (l, c) are
// broadcasts.  The colour products are computed
// dense and branch-free (exact zeros contribute exact zeros); a partition is
// skipped only when one of its sub-currents is zero in every entry.  Levels
// with few subsets split the partitions into chunks whose partial sums are
// reduced in a fixed order (deterministic results).
//
// Memory.  Each subset has one record (momentum, 9 gluon and 9 tensor
// colour entries), stored by rank (subsets ordered by size): the records of
// the first ranks -- the small subsets, which the partitions of every
// larger subset read -- sit in shared memory, the rest in a per-CTA slab of
// global memory that stays resident in L1/L2 (one or two CTAs per SM).  At
// n <= 10 in FP32 the whole table fits in shared memory.
#pragma once

#include "bg_internal.h"
#include "device_common.cuh"

namespace bg {

struct CdParams {
  int64_t B;              // capacity (row stride of p, hel, colours)
  const int64_t* dB = nullptr;  // optional device-side event count
  double inv_sqrt_s;
  double scale;  // g^(2n-4) sqrt_s^(8-2n) * colour and helicity weights * 2^-(n-2)
  int flow;      // 0: adjoint colours [n][B] in 1..8; 1: flow pairs [2n][B] in 1..3;
                 // 2: continuous colour and polarisation angles (ang)
  Q4 q;
  // flow == 2: [5n][B] per gluon g rows 5g..5g+4 = cos(theta), phi, cos(theta_bar),
  // phi_bar, phi_h (hel and col are not read)
  const double* ang = nullptr;
};

// Real external colour matrices of the adjoint generators T^a = lambda^a/sqrt2
// (a = 2, 5, 7 multiplied by -i, which changes only a phase of A).
__constant__ double c_adj_colour[8][3][3] = {
    {{0, 0.70710678118654752440, 0}, {0.70710678118654752440, 0, 0}, {0, 0, 0}},
    {{0, -0.70710678118654752440, 0}, {0.70710678118654752440, 0, 0}, {0, 0, 0}},
    {{0.70710678118654752440, 0, 0}, {0, -0.70710678118654752440, 0}, {0, 0, 0}},
    {{0, 0, 0.70710678118654752440}, {0, 0, 0}, {0.70710678118654752440, 0, 0}},
    {{0, 0, -0.70710678118654752440}, {0, 0, 0}, {0.70710678118654752440, 0, 0}},
    {{0, 0, 0}, {0, 0, 0.70710678118654752440}, {0, 0.70710678118654752440, 0}},
    {{0, 0, 0}, {0, 0, -0.70710678118654752440}, {0, 0.70710678118654752440, 0}},
    {{0.40824829046386301637, 0, 0}, {0, 0.40824829046386301637, 0}, {0, 0, -0.81649658092772603273}}};

// j-th submask (1-based, increasing order) of S: deposit the bits of j into
// the set positions of S.
__device__ __forceinline__ int submask_at(int S, int j) {
  int r = 0;
  for (int s = S; s; s &= s - 1) {
    const int low = s & -s;
    if (j & 1) r |= low;
    j >>= 1;
  }
  return r;
}


__host__ __device__ constexpr int cd_binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  int c = 1;
  for (int i = 1; i <= k; ++i) c = c * (n - k + i) / i;
  return c;
}

// Kernel variants: threads per CTA (one event per CTA) and the unrolling of
// the loop over partitions.  The task decomposition below depends on N only,
// so all variants compute every sum in the same order: bitwise identical
// results.
//   N <= 9:  0 = (128, 1), 1 = (256, 1), 2 = (128, 2), 3 = (256, 2)
//   N >= 10: 0 = (256, 1), 1 = (384, 1), 2 = (512, 1), 3 = (256, 2), 4 = (384, 2)
__host__ __device__ constexpr int cd_num_variants(int N) { return N <= 9 ? 4 : 5; }
__host__ __device__ constexpr int cd_variant_threads(int N, int v) {
  return N <= 9 ? ((v & 1) ? 256 : 128) : ((v == 0 || v == 3) ? 256 : (v == 1 || v == 4) ? 384 : 512);
}
__host__ __device__ constexpr int cd_variant_unroll(int N, int v) { return (v >= (N <= 9 ? 2 : 3)) ? 2 : 1; }
__host__ __device__ constexpr int cd_default_variant(int N) { return N <= 8 ? 0 : N == 9 ? 1 : 2; }
// Resident CTAs per SM the register allocation aims at: one for n >= 10
// (shared memory admits one), several for the small tables of n <= 9.
__host__ __device__ constexpr int cd_min_blocks(int N, int NT) { return N >= 10 ? 1 : 0 * NT; }

// For n >= 10: the number c of chunks of the npart ordered partitions of each
// of nsub subsets (3 colour rows each) that minimises the rounds of the
// 3 nsub c tasks on a 512-thread CTA times the partitions of a chunk (the
// threads of the CTA wait at the level's barrier for its last round), the
// fewest chunks on ties, at most four rounds.  The choice does not depend on
// the variant's CTA size, so that all variants add the same partial sums
// (bitwise identical results).  n <= 9: c0.
__host__ __device__ constexpr int cd_round_chunks(int N, int nsub, int npart, int c0) {
  if (N <= 9) return c0;
  constexpr int ref = 512;
  int best = 1;
  long long best_cost = -1;
  for (int c = 1; c <= npart && (c == 1 || 3LL * nsub * c <= 4LL * ref); ++c) {
    const long long rounds = (3LL * nsub * c + ref - 1) / ref;
    const long long cost = rounds * ((npart + c - 1) / c);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = c;
    }
  }
  return best;
}

template <int N, typename T>
struct CdShape {
  static constexpr int M = N - 1;
  static constexpr int NS = 1 << M;
  static constexpr int TARGET = (N <= 8) ? 256 : (N == 9) ? 512 : 1024;  // tasks wanted per level
  // subset record: P[4] | J[9][4] | T[9][6] | 1/P^2 | pad.  100 elements:
  // a multiple of 16 bytes whose word count is not a multiple of 32, so that
  // records read by different threads spread over the shared-memory banks.
  static constexpr int REC = 100;
  static constexpr int OFF_J = 4, OFF_T = 40, OFF_INV = 94;
  // static shared memory of the kernel (upper bound, bytes)
  static constexpr size_t STATIC_SMEM = (size_t)NS * (2 + 2 + 1) + (size_t)N * 4 * 8 * 2 +
                                        (size_t)N * 9 * 8 + (size_t)M * M * 8 + (N + 1) * 4 + 64;
  static constexpr size_t SMEM_LIMIT = 232448;  // opt-in shared memory per block
  static constexpr int NSM_FIT = (int)((SMEM_LIMIT - STATIC_SMEM - 1024) / (REC * sizeof(T)));
  static constexpr int NSM = NS < NSM_FIT ? NS : NSM_FIT;  // records (by rank) in shared memory
  static constexpr size_t DYN_SMEM = (size_t)NSM * REC * sizeof(T);
  // top level: chunks of the partitions of the full set, per colour row
  static constexpr int NPART_TOP = NS - 2;
  static constexpr int NCH_TOP = cd_round_chunks(N, 1, NPART_TOP, (TARGET + 2) / 3 < NPART_TOP ? (TARGET + 2) / 3 : NPART_TOP);
};

// Chunks of ordered partitions per (subset, colour row) at level L.  n <= 9
// (several CTAs per SM): about TARGET tasks per level.  n >= 10 (one CTA per
// SM, whose threads wait at the level's barrier for its last round of
// tasks): the count cd_round_chunks picks.
template <int N, typename T>
__host__ __device__ constexpr int cd_chunks(int L) {
  constexpr int M = N - 1;
  const int tasks = 3 * cd_binom(M, L);
  const int npart = (1 << L) - 2;
  int c = (CdShape<N, T>::TARGET + tasks - 1) / tasks;
  if (c < 1) c = 1;
  if (c > npart) c = npart;
  return cd_round_chunks(N, cd_binom(M, L), npart, c);
}

template <int N, typename T>
__host__ __device__ constexpr int cd_max_partial_tasks() {
  int mx = 0;
  for (int L = 2; L < N - 1; ++L) {
    const int c = cd_chunks<N, T>(L);
    if (c > 1 && 3 * cd_binom(N - 1, L) * c > mx) mx = 3 * cd_binom(N - 1, L) * c;
  }
  return mx;
}

constexpr size_t kCdHeader = 256;  // workspace header: the event counter

// Per-CTA slab of global memory (after the header): records of the ranks
// that do not fit in shared memory, then the partial sums of chunked tasks.
template <int N, typename T>
struct CdSlab {
  using S = CdShape<N, T>;
  static constexpr size_t off_rec = 0;
  static constexpr size_t off_part = off_rec + sizeof(T) * S::REC * (size_t)(S::NS - S::NSM);
  static constexpr size_t off_top = off_part + sizeof(T) * 30 * (size_t)(cd_max_partial_tasks<N, T>() + 1);
  static constexpr size_t bytes_raw = off_top + sizeof(double) * 3 * (size_t)S::NCH_TOP;
  static constexpr size_t bytes = (bytes_raw + 255) & ~size_t(255);
};

template <typename T>
__device__ __forceinline__ void cd_ld4(const T* p, T (&x)[4]);
template <>
__device__ __forceinline__ void cd_ld4<float>(const float* p, float (&x)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  x[0] = v.x, x[1] = v.y, x[2] = v.z, x[3] = v.w;
}
template <>
__device__ __forceinline__ void cd_ld4<double>(const double* p, double (&x)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  x[0] = a.x, x[1] = a.y, x[2] = b.x, x[3] = b.y;
}
template <typename T>
__device__ __forceinline__ void cd_ld6(const T* p, T (&x)[6]);
template <>
__device__ __forceinline__ void cd_ld6<float>(const float* p, float (&x)[6]) {
  const float2* q = reinterpret_cast<const float2*>(p);
  const float2 a = q[0], b = q[1], c = q[2];
  x[0] = a.x, x[1] = a.y, x[2] = b.x, x[3] = b.y, x[4] = c.x, x[5] = c.y;
}
template <>
__device__ __forceinline__ void cd_ld6<double>(const double* p, double (&x)[6]) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = q[0], b = q[1], c = q[2];
  x[0] = a.x, x[1] = a.y, x[2] = b.x, x[3] = b.y, x[4] = c.x, x[5] = c.y;
}

template <typename T>
struct CdPair;
template <>
struct CdPair<float> {
  using type = float2;
};
template <>
struct CdPair<double> {
  using type = double2;
};
__device__ __forceinline__ float2 cd_pair(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 cd_pair(double a, double b) { return make_double2(a, b); }

// Contribution of one ordered partition (S1 left, record A; S2 right,
// record B) to the colour entries (r, c), c = 0..2, of row r, summed over
// the inner colour index l.  Dense: zero entries contribute exact zeros.
template <typename T, bool TENSOR>
__device__ __forceinline__ void cd_partition(const T* __restrict__ A, const T* __restrict__ B, int r,
                                             const T (&P2)[4], T (&br)[3][4], T (&tc)[3][6]) {
  T p1[4], p2[4], dP[4];
  cd_ld4(A, p1);
  cd_ld4(B, p2);
#pragma unroll
  for (int i = 0; i < 4; ++i) dP[i] = p1[i] - p2[i];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    T X[4], T1[6];
    cd_ld4(A + 4 + 4 * (3 * r + l), X);
    cd_ld6(A + 40 + 6 * (3 * r + l), T1);
    const T px = mdot(P2, X);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T Y[4], T2[6];
      cd_ld4(B + 4 + 4 * (3 * l + c), Y);
      cd_ld6(B + 40 + 6 * (3 * l + c), T2);
      const T xy = mdot(X, Y);
      const T py = mdot(P2, Y);
#pragma unroll
      for (int i = 0; i < 4; ++i) br[c][i] += xy * dP[i] + px * Y[i] - py * X[i];
      if (TENSOR) {
        tc[c][0] += X[0] * Y[1] - X[1] * Y[0];
        tc[c][1] += X[0] * Y[2] - X[2] * Y[0];
        tc[c][2] += X[0] * Y[3] - X[3] * Y[0];
        tc[c][3] += X[1] * Y[2] - X[2] * Y[1];
        tc[c][4] += X[1] * Y[3] - X[3] * Y[1];
        tc[c][5] += X[2] * Y[3] - X[3] * Y[2];
      }
      ten_vec_acc(T2, X, br[c]);
      vec_ten_acc(Y, T1, br[c]);
    }
  }
}

// Rank of S among the subsets of its size in increasing order (colex):
// sum over its set bits p_1 < p_2 < ... of C(p_j, j).
__device__ __forceinline__ int cd_colex_rank(int S) {
  int r = 0, j = 0;
  for (int s = S; s; s &= s - 1) {
    ++j;
    r += cd_binom(__ffs(s) - 1, j);
  }
  return r;
}

template <int N, typename T>
__device__ __forceinline__ T* cd_rec(T* sRec, T* gRec, int rk) {
  constexpr int NSM = CdShape<N, T>::NSM, REC = CdShape<N, T>::REC;
  return rk < NSM ? sRec + (size_t)rk * REC : gRec + (size_t)(rk - NSM) * REC;
}

template <int N, typename T, int NT, int UR>
__global__ void __launch_bounds__(NT, cd_min_blocks(N, NT)) cd_kernel(CdParams prm, const double* __restrict__ p,
                                                                const int8_t* __restrict__ hel,
                                                                const int8_t* __restrict__ col,
                                                                const uint8_t* __restrict__ accept,
                                                                double* __restrict__ me2,
                                                                unsigned char* __restrict__ workspace,
                                                                int* __restrict__ status) {
  using Sh = CdShape<N, T>;
  using L = CdSlab<N, T>;
  constexpr int M = Sh::M, NS = Sh::NS;
  extern __shared__ __align__(16) unsigned char cd_smem[];
  T* const sRec = reinterpret_cast<T*>(cd_smem);
  unsigned long long* const counter = reinterpret_cast<unsigned long long*>(workspace);
  unsigned char* const slab = workspace + kCdHeader + (size_t)blockIdx.x * L::bytes;
  T* const gRec = reinterpret_cast<T*>(slab + L::off_rec);
  T* const part = reinterpret_cast<T*>(slab + L::off_part);
  double* const top = reinterpret_cast<double*>(slab + L::off_top);

  __shared__ uint16_t s_list[NS];  // rank -> subset
  __shared__ uint16_t s_rank[NS];  // subset -> rank
  __shared__ uint8_t s_nz[NS];     // record has a non-zero entry, by rank
  __shared__ int s_off[N + 1];     // first rank of each size
  __shared__ double s_k[N][4];     // scaled outgoing momenta (FP64)
  __shared__ double s_e[N][4];     // polarisations (FP64)
  __shared__ double s_E[N][3][3];  // external colour matrices
  __shared__ double s_pair[M][M];  // pair invariants 2 k_a.k_b / s (FP64)
  __shared__ long long s_ev;
  __shared__ int s_skip;

  const int tid = threadIdx.x;
  const int64_t S_ = prm.B;
  const int64_t Bn = prm.dB ? (*prm.dB < S_ ? *prm.dB : S_) : S_;
  // subsets ordered by size, then increasing (event independent)
  if (tid <= M + 1) {
    int o = 0;
    for (int i = 0; i < tid; ++i) o += cd_binom(M, i);
    s_off[tid] = o;
  }
  __syncthreads();
  for (int Sx = tid; Sx < NS; Sx += NT) {
    const int rk = s_off[__popc(Sx)] + cd_colex_rank(Sx);
    s_list[rk] = (uint16_t)Sx;
    s_rank[Sx] = (uint16_t)rk;
  }
  __syncthreads();

  for (;;) {
    if (tid == 0) s_ev = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t e = s_ev;
    if (e >= Bn) break;
    // ---- external states (FP64) ----
    if (tid < N) {
      const int g = tid;
      double k[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) k[m] = p[((int64_t)m * N + g) * S_ + e] * prm.inv_sqrt_s;
      if (g < 2) {
#pragma unroll
        for (int m = 0; m < 4; ++m) k[m] = -k[m];
      }
      double e1[4], e2[4];
      lc_polarisations(k, prm.q.v, e1, e2);
      if (prm.flow == 2) {
        // continuous sampling (Sec. 2.1): e = cos(phi_h) e1 + sin(phi_h) e2; the
        // colour matrix sum_a eta^a T^a of the colour polarisation
        // eta^a = eta T^a eta_bar is |eta_bar><eta| minus a multiple of the
        // identity, a U(1) gluon that decouples from all-gluon amplitudes,
        // so the outer product alone is used
        const double* a = prm.ang;
        double v[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] = a[(int64_t)(5 * g + j) * S_ + e];
        double sh, ch, eta[3], etab[3];
        sincos(v[4], &sh, &ch);
#pragma unroll
        for (int w = 0; w < 2; ++w) {
          const double ct = v[2 * w];
          const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
          double sp, cp;
          sincos(v[2 * w + 1], &sp, &cp);
          double* x = w ? etab : eta;
          x[0] = ct;
          x[1] = st * cp;
          x[2] = st * sp;
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          s_k[g][m] = k[m];
          s_e[g][m] = ch * e1[m] + sh * e2[m];
        }
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) s_E[g][i][j] = etab[i] * eta[j];
      } else {
        const int h = hel[(int64_t)g * S_ + e];
        if (h != 1 && h != -1) flag_status(status, BG_EINVAL);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          s_k[g][m] = k[m];
          s_e[g][m] = (h < 0) ? e2[m] : e1[m];
        }
        if (prm.flow) {
          const int rr = col[(int64_t)(2 * g) * S_ + e], cc = col[(int64_t)(2 * g + 1) * S_ + e];
          if (rr < 1 || rr > 3 || cc < 1 || cc > 3) flag_status(status, BG_EINVAL);
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) s_E[g][i][j] = (i == rr - 1 && j == cc - 1) ? 1.0 : 0.0;
        } else {
          int a = col[(int64_t)g * S_ + e];
          if (a < 1 || a > 8) {
            flag_status(status, BG_EINVAL);
            a = 1;
          }
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) s_E[g][i][j] = c_adj_colour[a - 1][i][j];
        }
      }
    }
    __syncthreads();
    if (tid == 0) {
      int skip = (accept != nullptr && accept[e] == 0) ? 1 : 0;
      if (prm.flow == 1 && !skip) {  // a colour flow with unequal row/column counts has A = 0
        int bal[3] = {0, 0, 0};
        for (int g = 0; g < N; ++g)
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
              if (s_E[g][i][j] != 0.0) {
                ++bal[i];
                --bal[j];
              }
        skip = (bal[0] | bal[1] | bal[2]) != 0;
      }
      s_skip = skip;
    }
    for (int it = tid; it < M * M; it += NT) {
      const int a = it / M, b = it % M;
      s_pair[a][b] = 2.0 * (s_k[a][0] * s_k[b][0] - s_k[a][1] * s_k[b][1] - s_k[a][2] * s_k[b][2] -
                            s_k[a][3] * s_k[b][3]);
    }
    __syncthreads();
    if (s_skip) {
      if (tid == 0) me2[e] = 0.0;
      __syncthreads();
      continue;
    }
    // ---- subset momenta, inverse propagators (FP64 -> T), level 1 ----
    for (int rk = tid; rk < NS; rk += NT) {
      const int Sx = s_list[rk];
      double P[4] = {0.0, 0.0, 0.0, 0.0}, p2 = 0.0;
      for (int a = 0; a < M; ++a) {
        if (!((Sx >> a) & 1)) continue;
#pragma unroll
        for (int m = 0; m < 4; ++m) P[m] += s_k[a][m];
        for (int b = a + 1; b < M; ++b)
          if ((Sx >> b) & 1) p2 += s_pair[a][b];
      }
      T* R = cd_rec<N, T>(sRec, gRec, rk);
#pragma unroll
      for (int m = 0; m < 4; ++m) R[m] = T(P[m]);
      R[Sh::OFF_INV] = (__popc(Sx) >= 2 && Sx != NS - 1) ? T(1.0 / p2) : T(0);
      if (__popc(Sx) == 1) {
        const int g = __ffs(Sx) - 1;
        bool any = false;
        for (int rc = 0; rc < 9; ++rc) {
          const double cf = s_E[g][rc / 3][rc % 3];
          any = any || (cf != 0.0);
#pragma unroll
          for (int m = 0; m < 4; ++m) R[Sh::OFF_J + 4 * rc + m] = T(cf * s_e[g][m]);
#pragma unroll
          for (int m = 0; m < 6; ++m) R[Sh::OFF_T + 6 * rc + m] = T(0);
        }
        s_nz[rk] = any ? 1 : 0;
      }
    }
    __syncthreads();

    // ---- levels 2 .. M-1 ----
    for (int Lv = 2; Lv < M; ++Lv) {
      const int nsub = s_off[Lv + 1] - s_off[Lv];
      const int nch = cd_chunks<N, T>(Lv);
      const int npart = (1 << Lv) - 2;
      const int ntask = nsub * nch * 3;
      for (int t = tid; t < ntask; t += NT) {
        const int r = t % 3;
        const int u = t / 3;
        const int ch = u % nch;
        const int rkS = s_off[Lv] + u / nch;
        const int Sx = s_list[rkS];
        T* RS = cd_rec<N, T>(sRec, gRec, rkS);
        T P2[4], br[3][4], tc[3][6];
#pragma unroll
        for (int m = 0; m < 4; ++m) P2[m] = T(2) * RS[m];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
#pragma unroll
          for (int m = 0; m < 4; ++m) br[c][m] = T(0);
#pragma unroll
          for (int m = 0; m < 6; ++m) tc[c][m] = T(0);
        }
        const int j0 = 1 + (int)((long)ch * npart / nch), j1 = 1 + (int)((long)(ch + 1) * npart / nch);
        int S1 = submask_at(Sx, j0);
#pragma unroll UR
        for (int j = j0; j < j1; ++j) {
          const int r1 = s_rank[S1], r2 = s_rank[Sx ^ S1];
          if (s_nz[r1] & s_nz[r2])
            cd_partition<T, true>(cd_rec<N, T>(sRec, gRec, r1), cd_rec<N, T>(sRec, gRec, r2), r, P2, br, tc);
          S1 = ((S1 | ~Sx) + 1) & Sx;
        }
        if (nch == 1) {
          const T ip = RS[Sh::OFF_INV];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
#pragma unroll
            for (int m = 0; m < 4; ++m) RS[Sh::OFF_J + 4 * (3 * r + c) + m] = br[c][m] * ip;
#pragma unroll
            for (int m = 0; m < 6; ++m) RS[Sh::OFF_T + 6 * (3 * r + c) + m] = tc[c][m];
          }
        } else {
          // 30 values as 15 aligned pairs (t * 30 is even, the slab
          // 16-byte aligned)
          using V2 = typename CdPair<T>::type;
          V2* q = reinterpret_cast<V2*>(part + (size_t)t * 30);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
#pragma unroll
            for (int m = 0; m < 4; m += 2) q[(10 * c + m) / 2] = cd_pair(br[c][m], br[c][m + 1]);
#pragma unroll
            for (int m = 0; m < 6; m += 2) q[(10 * c + 4 + m) / 2] = cd_pair(tc[c][m], tc[c][m + 1]);
          }
        }
      }
      __syncthreads();
      if (nch > 1) {
        for (int v = tid; v < nsub * 9; v += NT) {
          const int rc = v % 9, si = v / 9;
          const int r = rc / 3, c = rc % 3;
          const int rkS = s_off[Lv] + si;
          T acc[10];
#pragma unroll
          for (int m = 0; m < 10; ++m) acc[m] = T(0);
          for (int ch = 0; ch < nch; ++ch) {
            const size_t t = ((size_t)si * nch + ch) * 3 + r;
#pragma unroll
            for (int m = 0; m < 10; m += 2) {
              const typename CdPair<T>::type v =
                  reinterpret_cast<const typename CdPair<T>::type*>(part)[(t * 30 + 10 * c + m) / 2];
              acc[m] += v.x;
              acc[m + 1] += v.y;
            }
          }
          T* RS = cd_rec<N, T>(sRec, gRec, rkS);
          const T ip = RS[Sh::OFF_INV];
#pragma unroll
          for (int m = 0; m < 4; ++m) RS[Sh::OFF_J + 4 * rc + m] = acc[m] * ip;
#pragma unroll
          for (int m = 0; m < 6; ++m) RS[Sh::OFF_T + 6 * rc + m] = acc[4 + m];
        }
        __syncthreads();
      }
      // non-zero flags of this level
      for (int si = tid; si < nsub; si += NT) {
        const int rk = s_off[Lv] + si;
        const T* R = cd_rec<N, T>(sRec, gRec, rk);
        bool any = false;
        for (int i = Sh::OFF_J; i < Sh::OFF_T + 54; ++i) any = any || (R[i] != T(0));
        s_nz[rk] = any ? 1 : 0;
      }
      __syncthreads();
    }

    // ---- top level: A = sum_rc (E_n)_cr e_n . br(full)_rc ----
    {
      constexpr int FULL = NS - 1;
      constexpr int npart = NS - 2;
      constexpr int nch = Sh::NCH_TOP;
      const T* RF = cd_rec<N, T>(sRec, gRec, NS - 1);
      T en[4], P2[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        en[m] = T(s_e[N - 1][m]);
        P2[m] = T(2) * RF[m];
      }
      for (int t = tid; t < 3 * nch; t += NT) {
        const int r = t % 3, ch = t / 3;
        const double w0 = s_E[N - 1][0][r], w1 = s_E[N - 1][1][r], w2 = s_E[N - 1][2][r];
        double v = 0.0;
        if (w0 != 0.0 || w1 != 0.0 || w2 != 0.0) {
          const int j0 = 1 + (int)((long)ch * npart / nch), j1 = 1 + (int)((long)(ch + 1) * npart / nch);
          T br[3][4], tc[3][6];
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int m = 0; m < 4; ++m) br[c][m] = T(0);
          int S1 = submask_at(FULL, j0);
#pragma unroll UR
          for (int j = j0; j < j1; ++j) {
            const int r1 = s_rank[S1], r2 = s_rank[FULL ^ S1];
            if (s_nz[r1] & s_nz[r2])
              cd_partition<T, false>(cd_rec<N, T>(sRec, gRec, r1), cd_rec<N, T>(sRec, gRec, r2), r, P2, br, tc);
            S1 = ((S1 | ~FULL) + 1) & FULL;
          }
          v = w0 * (double)mdot(en, br[0]) + w1 * (double)mdot(en, br[1]) + w2 * (double)mdot(en, br[2]);
        }
        top[t] = v;
      }
      __syncthreads();
      // reduction in a fixed order (independent of the CTA size)
      if (tid < 32) {
        double a = 0.0;
        for (int t = tid; t < 3 * nch; t += 32) a += top[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (tid == 0) me2[e] = prm.scale * a * a;
      }
      __syncthreads();
    }
  }
}

template <int N, typename T, int V>
int cd_ctas_per_sm_v() {
  using Sh = CdShape<N, T>;
  constexpr int NT = cd_variant_threads(N, V), UR = cd_variant_unroll(N, V);
  if (cudaFuncSetAttribute(cd_kernel<N, T, NT, UR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)Sh::DYN_SMEM) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cd_kernel<N, T, NT, UR>, NT, Sh::DYN_SMEM) != cudaSuccess)
    return 0;
  return nb;
}

template <int N, typename T>
int cd_ctas_per_sm(int v) {
  switch (v) {
    case 0: return cd_ctas_per_sm_v<N, T, 0>();
    case 1: return cd_ctas_per_sm_v<N, T, 1>();
    case 2: return cd_ctas_per_sm_v<N, T, 2>();
    case 3: return cd_ctas_per_sm_v<N, T, 3>();
    case 4:
      if constexpr (cd_num_variants(N) > 4) return cd_ctas_per_sm_v<N, T, 4>();
      return 0;
    default: return 0;
  }
}

// Workspace for any variant: header + one slab per CTA of the largest grid.
template <int N, typename T>
size_t cd_workspace_bytes_n(int sms) {
  int nb = 0;
  for (int v = 0; v < cd_num_variants(N); ++v) {
    const int b = cd_ctas_per_sm<N, T>(v);
    if (b <= 0) return 0;
    nb = b > nb ? b : nb;
  }
  return kCdHeader + (size_t)sms * nb * CdSlab<N, T>::bytes;
}

template <int N, typename T, int V>
cudaError_t launch_cd_v(const CdParams& prm, const double* p, const int8_t* hel, const int8_t* col,
                        const uint8_t* accept, double* me2, void* workspace, int* status, int sms, cudaStream_t s) {
  constexpr int NT = cd_variant_threads(N, V), UR = cd_variant_unroll(N, V);
  const int nb = cd_ctas_per_sm_v<N, T, V>();
  if (nb <= 0) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)sms * nb;
  if (grid > prm.B) grid = prm.B;
  // the event counter starts at zero for every launch
  cudaError_t e = cudaMemsetAsync(workspace, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  cd_kernel<N, T, NT, UR><<<(unsigned)grid, NT, CdShape<N, T>::DYN_SMEM, s>>>(
      prm, p, hel, col, accept, me2, static_cast<unsigned char*>(workspace), status);
  return cudaGetLastError();
}

template <int N, typename T>
cudaError_t launch_cd_n(const CdParams& prm, const double* p, const int8_t* hel, const int8_t* col,
                        const uint8_t* accept, double* me2, void* workspace, int* status, int sms, cudaStream_t s,
                        int variant) {
  if (variant < 0 || variant >= cd_num_variants(N)) variant = cd_default_variant(N);
  switch (variant) {
    case 0: return launch_cd_v<N, T, 0>(prm, p, hel, col, accept, me2, workspace, status, sms, s);
    case 1: return launch_cd_v<N, T, 1>(prm, p, hel, col, accept, me2, workspace, status, sms, s);
    case 2: return launch_cd_v<N, T, 2>(prm, p, hel, col, accept, me2, workspace, status, sms, s);
    case 3: return launch_cd_v<N, T, 3>(prm, p, hel, col, accept, me2, workspace, status, sms, s);
    default:
      if constexpr (cd_num_variants(N) > 4)
        return launch_cd_v<N, T, 4>(prm, p, hel, col, accept, me2, workspace, status, sms, s);
      return cudaErrorInvalidValue;
  }
}

template <typename T>
size_t cd_workspace_bytes_t(int n, int sms) {
  switch (n) {
    case 4: return cd_workspace_bytes_n<4, T>(sms);
    case 5: return cd_workspace_bytes_n<5, T>(sms);
    case 6: return cd_workspace_bytes_n<6, T>(sms);
    case 7: return cd_workspace_bytes_n<7, T>(sms);
    case 8: return cd_workspace_bytes_n<8, T>(sms);
    case 9: return cd_workspace_bytes_n<9, T>(sms);
    case 10: return cd_workspace_bytes_n<10, T>(sms);
    case 11: return cd_workspace_bytes_n<11, T>(sms);
    case 12: return cd_workspace_bytes_n<12, T>(sms);
    default: return 0;
  }
}

template <typename T>
cudaError_t launch_cd_t(int n, const CdParams& prm, const double* p, const int8_t* hel, const int8_t* col,
                        const uint8_t* accept, double* me2, void* workspace, int* status, int sms, cudaStream_t s,
                        int variant) {
  switch (n) {
    case 4: return launch_cd_n<4, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s, variant);
    case 5: return launch_cd_n<5, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s, variant);
    case 6: return launch_cd_n<6, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s, variant);
    case 7: return launch_cd_n<7, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s, variant);
    case 8: return launch_cd_n<8, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s, variant);
    case 9: return launch_cd_n<9, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s, variant);
    case 10: return launch_cd_n<10, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s, variant);
    case 11: return launch_cd_n<11, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s, variant);
    case 12: return launch_cd_n<12, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s, variant);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bg
