// comc_rank.h -- counting and ranking the orders of a sampled colour flow
// whose chain of Kronecker deltas closes (the colour-flow decomposition,
// Eq. 2.19).
//
// Gluon i with the flow pair (r_i, c_i) is an edge r_i -> c_i of a directed
// multigraph on the three colours.  An order (1, s_2, ..., s_n) whose chain
// delta(c_1, r_{s_2}) delta(c_{s_2}, r_{s_3}) ... delta(c_{s_n}, r_1) closes
// is an Eulerian circuit of that graph which starts with gluon 1's edge.
// Their number is the BEST theorem's (de Bruijn, van Aardenne-Ehrenfest,
// Smith, Tutte):
//   ec(G) = t_w(G) prod_v (deg(v) - 1)!,
// the product over the vertices that have edges, deg the out-degree with
// loops counted, t_w(G) the number of spanning arborescences oriented
// towards a vertex w (matrix-tree theorem: the determinant of the
// out-degree Laplacian D - A, loops left out, with w's row and column
// removed).  It holds for balanced graphs (in-degree = out-degree at every
// vertex); t_w = 0 when the edges are not connected.
//
// A partial order that has used the trail r_1 -> ... -> x can be completed
// in as many ways as there are trails x -> r_1 over the remaining edges,
// i.e. Eulerian circuits of the remaining edges plus one edge r_1 -> x that
// start with that edge: ec of that graph.  Starting from a balanced flow,
// every such graph met below is balanced (removing the next edge x -> c and
// replacing r_1 -> x by r_1 -> c keeps every vertex's balance).  So the
// rank-th order, in lexicographic order of the gluon labels, is found
// position by position: the candidates for the next position are the free
// gluons with row colour x in increasing label order, each heading a block
// of completions whose size depends only on its column colour.
//
// All counts are at most (n-1)! < 2^31 for n <= 12 and fit 32 bits; every
// partial product below is bounded by the final count.  The code is
// compiled for the device and, by the host tests, for the CPU.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define COMC_HD __host__ __device__ __forceinline__
#define COMC_UNROLL _Pragma("unroll")
#define COMC_ROLLED _Pragma("unroll 1")
#else
#define COMC_HD inline
#define COMC_UNROLL
#define COMC_ROLLED
#endif

namespace bg {

// One event's flow with gluon 0 (labels 0-based) singled out.
struct ComcFlow {
  uint32_t rm0, rm1, rm2;  // gluons 1..n-1 with row colour 0, 1, 2 (bit g)
  uint32_t cm0, cm1, cm2;  // gluons 1..n-1 with column colour 0, 1, 2
  int r0, c0;              // gluon 0's pair
};

COMC_HD int comc_popc(uint32_t v) {
#if defined(__CUDA_ARCH__)
  return __popc(v);
#else
  return __builtin_popcount(v);
#endif
}
COMC_HD int comc_ctz(uint32_t v) {
#if defined(__CUDA_ARCH__)
  return __ffs((int)v) - 1;
#else
  return __builtin_ctz(v);
#endif
}

// Edge-type counts: field 3 r + c (4 bits) of a 64-bit word holds the number
// of edges r -> c (at most 12, one of which may be the added edge r_1 -> x).
COMC_HD uint64_t comc_unit(int r, int c) { return 1ull << (4 * (3 * r + c)); }
COMC_HD uint32_t comc_field(uint64_t m, int f) { return (uint32_t)(m >> (4 * f)) & 15u; }

COMC_HD uint64_t comc_types(const ComcFlow& f) {
  const uint32_t rm[3] = {f.rm0, f.rm1, f.rm2}, cm[3] = {f.cm0, f.cm1, f.cm2};
  uint64_t m = 0;
COMC_UNROLL
  for (int r = 0; r < 3; ++r)
COMC_UNROLL
    for (int c = 0; c < 3; ++c) m |= (uint64_t)comc_popc(rm[r] & cm[c]) << (4 * (3 * r + c));
  return m;
}

// ec(G) of the balanced graph with edge-type counts m; fact[k] = k!, k <= 11.
COMC_HD uint32_t comc_circuits(uint64_t m, const uint32_t* fact) {
  const uint32_t a00 = comc_field(m, 0), a01 = comc_field(m, 1), a02 = comc_field(m, 2);
  const uint32_t a10 = comc_field(m, 3), a11 = comc_field(m, 4), a12 = comc_field(m, 5);
  const uint32_t a20 = comc_field(m, 6), a21 = comc_field(m, 7), a22 = comc_field(m, 8);
  const uint32_t o0 = a00 + a01 + a02, o1 = a10 + a11 + a12, o2 = a20 + a21 + a22;
  const bool v0 = o0 != 0, v1 = o1 != 0, v2 = o2 != 0;
  uint32_t t;
  if (v0 && v1 && v2)
    t = (a10 + a12) * (a20 + a21) - a12 * a21;  // root 0: the 2x2 minor
  else if (v0 && v1)
    t = a10;  // root 0: vertex 1's edge towards it
  else if (v0 && v2)
    t = a20;
  else if (v1 && v2)
    t = a21;  // root 1
  else
    t = 1;  // one vertex (loops only)
  if (v0) t *= fact[o0 - 1];
  if (v1) t *= fact[o1 - 1];
  if (v2) t *= fact[o2 - 1];
  return t;
}

// Trails x -> r0 over the edges m: ec of m plus the edge r0 -> x.
COMC_HD uint32_t comc_trails(uint64_t m, int x, int r0, const uint32_t* fact) {
  return comc_circuits(m + comc_unit(r0, x), fact);
}

// Every colour as often a row as a column colour (gluon 0 included).
COMC_HD bool comc_balanced(const ComcFlow& f) {
  const int r0n = comc_popc(f.rm0) + (f.r0 == 0), r1n = comc_popc(f.rm1) + (f.r0 == 1);
  const int c0n = comc_popc(f.cm0) + (f.c0 == 0), c1n = comc_popc(f.cm1) + (f.c0 == 1);
  return r0n == c0n && r1n == c1n;  // the third colour follows from the totals
}

// Number of closing orders of a balanced flow: trails c0 -> r0 over the edges
// of gluons 1..n-1 (with gluon 0's edge r0 -> c0 this is ec of the flow).
COMC_HD uint32_t comc_count(const ComcFlow& f, const uint32_t* fact) {
  return comc_trails(comc_types(f), f.c0, f.r0, fact);
}

// The rank-th closing order (0 <= rank < comc_count) of a balanced flow of N
// gluons, in lexicographic order of the labels: positions 1..N-1 packed 4
// bits each (position p in bits 4 (p - 1)).  Returns ~0 if rank is out of
// range.
template <int N>
COMC_HD uint64_t comc_unrank(uint32_t rank, const ComcFlow& f, const uint32_t* fact) {
  uint64_t m = comc_types(f), packed = 0;
  uint32_t avail = ((1u << N) - 1u) & ~1u;
  int x = f.c0;
  // not unrolled: the unrolled form adds enough code to the colour-flow
  // evaluator to thrash its instruction cache (2-3x slower at n = 10..12)
COMC_ROLLED
  for (int pos = 1; pos < N; ++pos) {
    const uint32_t rowx = x == 0 ? f.rm0 : (x == 1 ? f.rm1 : f.rm2);
    const uint32_t t0 = comc_field(m, 3 * x + 0) ? comc_trails(m - comc_unit(x, 0), 0, f.r0, fact) : 0u;
    const uint32_t t1 = comc_field(m, 3 * x + 1) ? comc_trails(m - comc_unit(x, 1), 1, f.r0, fact) : 0u;
    const uint32_t t2 = comc_field(m, 3 * x + 2) ? comc_trails(m - comc_unit(x, 2), 2, f.r0, fact) : 0u;
    uint32_t cand = avail & rowx;
    int g = -1, c = 0;
    while (cand) {
      const int h = comc_ctz(cand);
      cand &= cand - 1u;
      const int ch = ((f.cm1 >> h) & 1u) ? 1 : (((f.cm2 >> h) & 1u) ? 2 : 0);
      const uint32_t sz = ch == 0 ? t0 : (ch == 1 ? t1 : t2);
      if (rank < sz) {
        g = h;
        c = ch;
        break;
      }
      rank -= sz;
    }
    if (g < 0) return ~0ull;
    packed |= (uint64_t)g << (4 * (pos - 1));
    avail &= ~(1u << g);
    m -= comc_unit(x, c);
    x = c;
  }
  return packed;
}

}  // namespace bg
