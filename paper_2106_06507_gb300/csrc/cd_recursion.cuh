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
// Work decomposition: persistent CTAs, one event at a time per CTA.  The
// subsets are processed level by level (by size); a task is (subset, colour
// entry rc, chunk of its ordered partitions) and accumulates 4 + 6 values;
// levels with few subsets split the partitions into chunks whose partial sums
// are reduced in a fixed order (deterministic results).  The event's tables
// (gluon and tensor currents, momenta, inverse propagators) live in a per-CTA
// slab of global memory that stays resident in L1/L2; per-subset masks of
// the non-zero colour entries skip products that vanish exactly (most of
// them in the colour-flow basis).  In the colour-flow basis an event whose
// flow is not balanced (some colour appears more often as a row than as a
// column index) has amplitude zero and is skipped.
#pragma once

#include "bg_internal.h"
#include "device_common.cuh"

namespace bg {

template <int N, typename T>
struct CdShape {
  static constexpr int NT = 256;
  static constexpr int M = N - 1;
  static constexpr int NS = 1 << M;
  static constexpr int TARGET = 2 * NT;  // tasks wanted per level
};

__host__ __device__ constexpr int cd_binom(int n, int k) {
  return (k < 0 || k > n) ? 0 : (k == 0 || k == n) ? 1 : cd_binom(n - 1, k - 1) + cd_binom(n - 1, k);
}

// Chunks of ordered partitions per (subset, colour entry) at level L.
template <int N>
__host__ __device__ constexpr int cd_chunks(int L) {
  constexpr int M = N - 1;
  const int tasks = 9 * cd_binom(M, L);
  const int npart = (1 << L) - 2;
  int c = (2 * 256 + tasks - 1) / tasks;
  if (c < 1) c = 1;
  if (c > npart) c = npart;
  return c;
}

template <int N>
__host__ __device__ constexpr int cd_max_partial_tasks() {
  int mx = 0;
  for (int L = 2; L < N - 1; ++L) {
    const int c = cd_chunks<N>(L);
    if (c > 1 && 9 * cd_binom(N - 1, L) * c > mx) mx = 9 * cd_binom(N - 1, L) * c;
  }
  return mx;
}

// Per-CTA workspace slab layout (bytes), for arithmetic type T.
template <int N, typename T>
struct CdSlab {
  using S = CdShape<N, T>;
  static constexpr size_t off_J = 0;                                          // T [NS][9][4]
  static constexpr size_t off_T = off_J + sizeof(T) * S::NS * 36;             // T [NS][9][6]
  static constexpr size_t off_P = off_T + sizeof(T) * S::NS * 54;             // T [NS][4]
  static constexpr size_t off_inv = off_P + sizeof(T) * S::NS * 4;            // T [NS]
  static constexpr size_t off_part = off_inv + sizeof(T) * S::NS;             // T [tasks][10]
  static constexpr size_t bytes_raw = off_part + sizeof(T) * 10 * (cd_max_partial_tasks<N>() + 1);
  static constexpr size_t bytes = (bytes_raw + 255) & ~size_t(255);
};

struct CdParams {
  int64_t B;              // capacity (row stride of p, hel, colours)
  const int64_t* dB = nullptr;  // optional device-side event count
  double inv_sqrt_s;
  double scale;  // g^(2n-4) sqrt_s^(8-2n) * colour and helicity weights * 2^-(n-2)
  int flow;      // 0: adjoint colours [n][B] in 1..8; 1: flow pairs [2n][B] in 1..3
  Q4 q;
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

// Contribution of one ordered partition (S1 left, S2 right) to colour entry
// (r, c), summed over the inner colour index l.
template <typename T>
__device__ __forceinline__ void cd_partition(const T* __restrict__ J, const T* __restrict__ Tt,
                                             const T* __restrict__ Pt, const uint32_t* __restrict__ nz, int S1,
                                             int S2, int r, int c, const T (&P2)[4], T (&br)[4], T (&tc)[6],
                                             bool need_tensor) {
  const uint32_t m1 = nz[S1], m2 = nz[S2];  // bits 0..8: gluon entries, 9..17: tensor entries
  T dP[4];
  const T* p1 = Pt + 4 * S1;
  const T* p2 = Pt + 4 * S2;
#pragma unroll
  for (int i = 0; i < 4; ++i) dP[i] = p1[i] - p2[i];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const int e1 = 3 * r + l, e2 = 3 * l + c;
    const bool x = (m1 >> e1) & 1, y = (m2 >> e2) & 1;
    const bool tx = (m1 >> (9 + e1)) & 1, ty = (m2 >> (9 + e2)) & 1;
    if (!((x && (y || ty)) || (y && tx))) continue;
    const T* X = J + (size_t)S1 * 36 + 4 * e1;
    const T* Y = J + (size_t)S2 * 36 + 4 * e2;
    if (x && y) {
      const T xy = mdot(X, Y);
      const T px = mdot(P2, X);
      const T py = mdot(P2, Y);
#pragma unroll
      for (int i = 0; i < 4; ++i) br[i] += xy * dP[i] + px * Y[i] - py * X[i];
      if (need_tensor) {
        tc[0] += X[0] * Y[1] - X[1] * Y[0];
        tc[1] += X[0] * Y[2] - X[2] * Y[0];
        tc[2] += X[0] * Y[3] - X[3] * Y[0];
        tc[3] += X[1] * Y[2] - X[2] * Y[1];
        tc[4] += X[1] * Y[3] - X[3] * Y[1];
        tc[5] += X[2] * Y[3] - X[3] * Y[2];
      }
    }
    if (x && ty) ten_vec_acc(Tt + (size_t)S2 * 54 + 6 * e2, X, br);
    if (y && tx) vec_ten_acc(Y, Tt + (size_t)S1 * 54 + 6 * e1, br);
  }
}

template <int N, typename T>
__global__ void __launch_bounds__(256) cd_kernel(CdParams prm, const double* __restrict__ p,
                                                 const int8_t* __restrict__ hel, const int8_t* __restrict__ col,
                                                 const uint8_t* __restrict__ accept, double* __restrict__ me2,
                                                 unsigned char* __restrict__ workspace, int* __restrict__ status) {
  using Sh = CdShape<N, T>;
  using L = CdSlab<N, T>;
  constexpr int M = Sh::M, NS = Sh::NS, NT = Sh::NT;
  unsigned char* slab = workspace + (size_t)blockIdx.x * L::bytes;
  T* J = reinterpret_cast<T*>(slab + L::off_J);
  T* Tt = reinterpret_cast<T*>(slab + L::off_T);
  T* Pt = reinterpret_cast<T*>(slab + L::off_P);
  T* inv = reinterpret_cast<T*>(slab + L::off_inv);
  T* part = reinterpret_cast<T*>(slab + L::off_part);

  __shared__ double s_k[N][4];       // scaled outgoing momenta (FP64)
  __shared__ double s_e[N][4];       // polarisations (FP64)
  __shared__ double s_E[N][3][3];    // external colour matrices
  __shared__ double s_pair[M][M];    // pair invariants 2 k_a.k_b / s (FP64)
  __shared__ uint32_t s_nz[NS];      // non-zero colour entries per subset
  __shared__ uint16_t s_list[NS];    // subsets ordered by size
  __shared__ int s_off[N + 1];
  __shared__ int s_skip;
  __shared__ double s_red[NT / 32];

  const int tid = threadIdx.x;
  const int64_t S_ = prm.B;
  const int64_t Bn = prm.dB ? (*prm.dB < S_ ? *prm.dB : S_) : S_;
  // subsets grouped by size (event independent)
  if (tid == 0) {
    int pos = 0;
    for (int Lv = 0; Lv <= M; ++Lv) {
      s_off[Lv] = pos;
      for (int Sx = 0; Sx < NS; ++Sx)
        if (__popc(Sx) == Lv) s_list[pos++] = (uint16_t)Sx;
    }
    s_off[M + 1] = pos;
  }
  __syncthreads();

  for (int64_t e = blockIdx.x; e < Bn; e += gridDim.x) {
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
    __syncthreads();
    if (tid == 0) {
      int skip = (accept != nullptr && accept[e] == 0) ? 1 : 0;
      if (prm.flow && !skip) {  // a colour flow with unequal row/column counts has A = 0
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
    for (int Sx = tid; Sx < NS; Sx += NT) {
      double P[4] = {0.0, 0.0, 0.0, 0.0}, p2 = 0.0;
      for (int a = 0; a < M; ++a) {
        if (!((Sx >> a) & 1)) continue;
#pragma unroll
        for (int m = 0; m < 4; ++m) P[m] += s_k[a][m];
        for (int b = a + 1; b < M; ++b)
          if ((Sx >> b) & 1) p2 += s_pair[a][b];
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) Pt[4 * Sx + m] = T(P[m]);
      inv[Sx] = (__popc(Sx) >= 2 && Sx != NS - 1) ? T(1) / T(p2) : T(0);
      if (__popc(Sx) == 1) {
        const int g = __ffs(Sx) - 1;
        uint32_t mask = 0;
        for (int rc = 0; rc < 9; ++rc) {
          const double c = s_E[g][rc / 3][rc % 3];
          if (c != 0.0) mask |= 1u << rc;
#pragma unroll
          for (int m = 0; m < 4; ++m) J[(size_t)Sx * 36 + 4 * rc + m] = T(c * s_e[g][m]);
#pragma unroll
          for (int m = 0; m < 6; ++m) Tt[(size_t)Sx * 54 + 6 * rc + m] = T(0);
        }
        s_nz[Sx] = mask;
      }
    }
    __syncthreads();

    // ---- levels 2 .. M-1 ----
    for (int Lv = 2; Lv < M; ++Lv) {
      const int nsub = s_off[Lv + 1] - s_off[Lv];
      const int nch = cd_chunks<N>(Lv);
      const int npart = (1 << Lv) - 2;
      const int ntask = nsub * 9 * nch;
      for (int t = tid; t < ntask; t += NT) {
        const int ch = t % nch;
        const int rc = (t / nch) % 9;
        const int si = t / (nch * 9);
        const int Sx = s_list[s_off[Lv] + si];
        const int r = rc / 3, c = rc % 3;
        const int j0 = 1 + (int)((long)ch * npart / nch), j1 = 1 + (int)((long)(ch + 1) * npart / nch);
        T P2[4], br[4] = {T(0), T(0), T(0), T(0)}, tc[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int m = 0; m < 4; ++m) P2[m] = T(2) * Pt[4 * Sx + m];
        int S1 = submask_at(Sx, j0);
        for (int j = j0; j < j1; ++j) {
          cd_partition(J, Tt, Pt, s_nz, S1, Sx ^ S1, r, c, P2, br, tc, true);
          S1 = ((S1 | ~Sx) + 1) & Sx;
        }
        if (nch == 1) {
          const T ip = inv[Sx];
#pragma unroll
          for (int m = 0; m < 4; ++m) J[(size_t)Sx * 36 + 4 * rc + m] = br[m] * ip;
#pragma unroll
          for (int m = 0; m < 6; ++m) Tt[(size_t)Sx * 54 + 6 * rc + m] = tc[m];
        } else {
#pragma unroll
          for (int m = 0; m < 4; ++m) part[(size_t)t * 10 + m] = br[m];
#pragma unroll
          for (int m = 0; m < 6; ++m) part[(size_t)t * 10 + 4 + m] = tc[m];
        }
      }
      __syncthreads();
      if (nch > 1) {
        for (int u = tid; u < nsub * 9; u += NT) {
          const int rc = u % 9, si = u / 9;
          const int Sx = s_list[s_off[Lv] + si];
          T acc[10];
#pragma unroll
          for (int m = 0; m < 10; ++m) acc[m] = T(0);
          for (int ch = 0; ch < nch; ++ch)
#pragma unroll
            for (int m = 0; m < 10; ++m) acc[m] += part[((size_t)u * nch + ch) * 10 + m];
          const T ip = inv[Sx];
#pragma unroll
          for (int m = 0; m < 4; ++m) J[(size_t)Sx * 36 + 4 * rc + m] = acc[m] * ip;
#pragma unroll
          for (int m = 0; m < 6; ++m) Tt[(size_t)Sx * 54 + 6 * rc + m] = acc[4 + m];
        }
        __syncthreads();
      }
      // non-zero masks of this level
      for (int si = tid; si < nsub; si += NT) {
        const int Sx = s_list[s_off[Lv] + si];
        uint32_t mask = 0;
        for (int rc = 0; rc < 9; ++rc) {
          bool zj = true, zt = true;
#pragma unroll
          for (int m = 0; m < 4; ++m) zj = zj && (J[(size_t)Sx * 36 + 4 * rc + m] == T(0));
#pragma unroll
          for (int m = 0; m < 6; ++m) zt = zt && (Tt[(size_t)Sx * 54 + 6 * rc + m] == T(0));
          if (!zj) mask |= 1u << rc;
          if (!zt) mask |= 1u << (9 + rc);
        }
        s_nz[Sx] = mask;
      }
      __syncthreads();
    }

    // ---- top level: A = sum_rc (E_n)_cr e_n . br(full)_rc ----
    {
      constexpr int FULL = NS - 1;
      constexpr int npart = NS - 2;
      constexpr int nch = (2 * NT + 8) / 9 < npart ? (2 * NT + 8) / 9 : npart;
      T en[4], P2[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        en[m] = T(s_e[N - 1][m]);
        P2[m] = T(2) * Pt[4 * FULL + m];
      }
      double acc = 0.0;
      for (int t = tid; t < 9 * nch; t += NT) {
        const int rc = t / nch, ch = t % nch;
        const int r = rc / 3, c = rc % 3;
        const double w = s_E[N - 1][c][r];
        if (w == 0.0) continue;
        const int j0 = 1 + (int)((long)ch * npart / nch), j1 = 1 + (int)((long)(ch + 1) * npart / nch);
        T br[4] = {T(0), T(0), T(0), T(0)}, tc[6];
        int S1 = submask_at(FULL, j0);
        for (int j = j0; j < j1; ++j) {
          cd_partition(J, Tt, Pt, s_nz, S1, FULL ^ S1, r, c, P2, br, tc, false);
          S1 = ((S1 | ~FULL) + 1) & FULL;
        }
        acc += w * (double)mdot(en, br);
      }
      // block reduction (fixed order)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if ((tid & 31) == 0) s_red[tid >> 5] = acc;
      __syncthreads();
      if (tid == 0) {
        double a = 0.0;
        for (int w = 0; w < NT / 32; ++w) a += s_red[w];
        me2[e] = prm.scale * a * a;
      }
      __syncthreads();
    }
  }
}

template <int N, typename T>
size_t cd_slab_bytes() {
  return CdSlab<N, T>::bytes;
}

// Persistent grid: 2 CTAs per SM.
inline int cd_grid(int sms) { return 2 * sms; }

template <int N, typename T>
cudaError_t launch_cd_n(const CdParams& prm, const double* p, const int8_t* hel, const int8_t* col,
                        const uint8_t* accept, double* me2, void* workspace, int* status, int sms, cudaStream_t s) {
  int64_t grid = cd_grid(sms);
  if (grid > prm.B) grid = prm.B;
  cd_kernel<N, T><<<(unsigned)grid, CdShape<N, T>::NT, 0, s>>>(prm, p, hel, col, accept, me2,
                                                                 static_cast<unsigned char*>(workspace), status);
  return cudaGetLastError();
}

template <typename T>
size_t cd_slab_bytes_t(int n) {
  switch (n) {
    case 4: return cd_slab_bytes<4, T>();
    case 5: return cd_slab_bytes<5, T>();
    case 6: return cd_slab_bytes<6, T>();
    case 7: return cd_slab_bytes<7, T>();
    case 8: return cd_slab_bytes<8, T>();
    case 9: return cd_slab_bytes<9, T>();
    case 10: return cd_slab_bytes<10, T>();
    case 11: return cd_slab_bytes<11, T>();
    case 12: return cd_slab_bytes<12, T>();
    default: return 0;
  }
}

template <typename T>
cudaError_t launch_cd_t(int n, const CdParams& prm, const double* p, const int8_t* hel, const int8_t* col,
                        const uint8_t* accept, double* me2, void* workspace, int* status, int sms, cudaStream_t s) {
  switch (n) {
    case 4: return launch_cd_n<4, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s);
    case 5: return launch_cd_n<5, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s);
    case 6: return launch_cd_n<6, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s);
    case 7: return launch_cd_n<7, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s);
    case 8: return launch_cd_n<8, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s);
    case 9: return launch_cd_n<9, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s);
    case 10: return launch_cd_n<10, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s);
    case 11: return launch_cd_n<11, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s);
    case 12: return launch_cd_n<12, T>(prm, p, hel, col, accept, me2, workspace, status, sms, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bg
