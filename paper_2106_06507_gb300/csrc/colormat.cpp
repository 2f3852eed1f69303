// colormat.cpp -- host generator of the adjoint (DDM) colour matrix, Eq. (2.17).
//
// C_{sigma tau} = sum_{a_1..a_n} (F^{a_s2} .. F^{a_s(n-1)})_{a1 an} (F^{a_t2} .. F^{a_t(n-1)})*_{a1 an}
// with F^b_{xy} = Tr(T^b [T^x, T^y]) and Tr(T^a T^b) = delta^ab (the
// normalisation of Eq. 2.27).
//
// Method (independent of any tabulated matrix): a chain of adjoint
// generators is a nested commutator in the fundamental representation,
//   (F^{b1} .. F^{bk})_{a a'} = Tr( [T^bk, .. [T^b2, [T^b1, T^a]] ..] T^a' ),
// which expands into 2^k signed words: each commutator puts T^bj either on
// the left (+) or on the right (-) of what it wraps.  The product of one
// trace with the complex conjugate of another, summed over all adjoint
// indices, is evaluated with the U(N) completeness relation
//   sum_a T^a_ij T^a_kl = delta_il delta_kj,
// which gives N^(number of closed index loops) for every pair of words.
// The U(1) part of U(N) drops out because every generator sits inside a
// commutator.  So every entry is a signed sum of powers of N = 3, an
// integer.  The matrix depends only on the relative permutation
// sigma^-1 o tau (the paper notes this relabelling property in Sec. 4.4), so
// only the first row is computed and the dense matrix is filled by
// relabelling.
#include <algorithm>
#include <cstdint>
#include <thread>
#include <vector>

#include "bg_internal.h"

namespace bg {

int64_t factorial(int m) {
  int64_t f = 1;
  for (int i = 2; i <= m; ++i) f *= i;
  return f;
}

// Permutation of 0..m-1 with lexicographic rank r (factorial number system).
static void perm_unrank(int64_t r, int m, int* perm) {
  int pool[16];
  for (int i = 0; i < m; ++i) pool[i] = i;
  int left = m;
  for (int pos = 0; pos < m; ++pos) {
    int64_t f = factorial(m - 1 - pos);
    int d = (int)(r / f);
    r %= f;
    perm[pos] = pool[d];
    for (int i = d; i < left - 1; ++i) pool[i] = pool[i + 1];
    --left;
  }
}

int64_t perm_rank(const int* perm, int m) {
  int64_t r = 0;
  for (int pos = 0; pos < m; ++pos) {
    int smaller = 0;
    for (int j = pos + 1; j < m; ++j) smaller += perm[j] < perm[pos];
    r += smaller * factorial(m - 1 - pos);
  }
  return r;
}

namespace {

// One expanded word: a cyclic sequence of n generator labels and its sign.
struct Word {
  int sign;
  int seq[kMaxNCO];
};

// Words of (F^{b_1}..F^{b_k})_{a1 an} for the chain labels b (labels 1..n-2;
// a1 is label 0 and an is label n-1), as traces Tr(L T^a1 R T^an).
static void expand(int n, const int* b, std::vector<Word>& out) {
  const int k = n - 2;
  out.resize((size_t)1 << k);
  for (int S = 0; S < (1 << k); ++S) {
    Word& w = out[S];
    int len = 0;
    int right = 0;
    for (int j = k - 1; j >= 0; --j)
      if (S >> j & 1) w.seq[len++] = b[j];  // left factors, last commutator outermost
    w.seq[len++] = 0;                        // T^{a1}
    for (int j = 0; j < k; ++j)
      if (!(S >> j & 1)) { w.seq[len++] = b[j]; ++right; }
    w.seq[len++] = n - 1;  // T^{an}
    w.sign = (right & 1) ? -1 : 1;
  }
}

// Number of closed index loops of sum_labels Tr(x) Tr(y) under the U(N)
// completeness relation; x and y contain each of the n labels once.
static int loops(int n, const int* x, const int* y) {
  int pos1[kMaxNCO], pos2[kMaxNCO];
  for (int p = 0; p < n; ++p) { pos1[x[p]] = p; pos2[y[p]] = p; }
  int seen = 0, cycles = 0;
  for (int p0 = 0; p0 < n; ++p0) {
    if (seen >> p0 & 1) continue;
    ++cycles;
    int p = p0;
    while (!(seen >> p & 1)) {
      seen |= 1 << p;
      int q = pos2[x[p]] + 1;
      if (q == n) q = 0;
      p = pos1[y[q]] + 1;
      if (p == n) p = 0;
    }
  }
  return cycles;
}

}  // namespace

void colour_row(int n, std::vector<double>& row) {
  const int k = n - 2;
  const int64_t nord = factorial(k);
  row.assign((size_t)nord, 0.0);
  int id[kMaxNCO];
  for (int j = 0; j < k; ++j) id[j] = j + 1;
  std::vector<Word> w1;
  expand(n, id, w1);
  double pw[kMaxNCO + 1];
  pw[0] = 1.0;
  for (int i = 1; i <= kMaxNCO; ++i) pw[i] = pw[i - 1] * 3.0;  // N_c = 3
  unsigned nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nth; ++t)
    th.emplace_back([&, t]() {
      std::vector<Word> w2;
      int perm[kMaxNCO], tau[kMaxNCO], rev[kMaxNCO];
      for (int64_t r = t; r < nord; r += nth) {
        perm_unrank(r, k, perm);
        for (int j = 0; j < k; ++j) tau[j] = perm[j] + 1;
        expand(n, tau, w2);
        double s = 0.0;
        for (const Word& b : w2) {
          for (int p = 0; p < n; ++p) rev[p] = b.seq[n - 1 - p];  // conjugate trace = reversed word
          for (const Word& a : w1) s += a.sign * b.sign * pw[loops(n, a.seq, rev)];
        }
        row[(size_t)r] = s;
      }
    });
  for (auto& x : th) x.join();
}

void colour_dense(int n, const std::vector<double>& row, std::vector<double>& dense) {
  const int k = n - 2;
  const int64_t nord = factorial(k);
  std::vector<int> perms((size_t)(nord * k));
  for (int64_t a = 0; a < nord; ++a) perm_unrank(a, k, &perms[(size_t)(a * k)]);
  dense.assign((size_t)(nord * nord), 0.0);
  unsigned nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nth; ++t)
    th.emplace_back([&, t]() {
      int pos[kMaxNCO], rho[kMaxNCO];
      for (int64_t a = t; a < nord; a += nth) {
        const int* s = &perms[(size_t)(a * k)];
        for (int j = 0; j < k; ++j) pos[s[j]] = j;
        for (int64_t b = 0; b < nord; ++b) {
          const int* u = &perms[(size_t)(b * k)];
          for (int j = 0; j < k; ++j) rho[j] = pos[u[j]];
          dense[(size_t)(a * nord + b)] = row[(size_t)perm_rank(rho, k)];
        }
      }
    });
  for (auto& x : th) x.join();
}

}  // namespace bg
