// Host driver for the closing-order counting and ranking of the colour-flow
// kernel (paper_2106_06507_gb300/csrc/comc_rank.h), compiled by
// tests/test_comc_rank_host.py.  Each input line holds n and the flow pairs
// r_0 c_0 r_1 c_1 ... (colours 0..2); the output line holds the balance flag,
// the count and the orders rank = 0, 1, ..., count - 1 (labels of positions
// 1..n-1, comma-separated), or "-" for an unbalanced flow.  A line that
// starts with -n asks for the count alone.
#include <cstdio>
#include <vector>

#include "comc_rank.h"

template <int N>
static void emit(const bg::ComcFlow& f, const uint32_t* fact, bool count_only) {
  const uint32_t cnt = bg::comc_count(f, fact);
  std::printf("1 %u", cnt);
  if (count_only) {
    std::printf("\n");
    return;
  }
  for (uint32_t r = 0; r < cnt; ++r) {
    const uint64_t pk = bg::comc_unrank<N>(r, f, fact);
    std::printf(" ");
    for (int p = 1; p < N; ++p) std::printf(p > 1 ? ",%d" : "%d", (int)((pk >> (4 * (p - 1))) & 15u));
  }
  // one rank past the end must be reported as out of range
  std::printf(" %s\n", bg::comc_unrank<N>(cnt, f, fact) == ~0ull ? "end" : "noend");
}

int main() {
  uint32_t fact[12];
  fact[0] = 1;
  for (int k = 1; k < 12; ++k) fact[k] = fact[k - 1] * (uint32_t)k;
  int n;
  while (std::scanf("%d", &n) == 1) {
    const bool count_only = n < 0;
    if (count_only) n = -n;
    if (n < 4 || n > 12) return 1;
    std::vector<int> r(n), c(n);
    for (int i = 0; i < n; ++i)
      if (std::scanf("%d %d", &r[i], &c[i]) != 2) return 1;
    bg::ComcFlow f{0, 0, 0, 0, 0, 0, r[0], c[0]};
    for (int g = 1; g < n; ++g) {
      const uint32_t b = 1u << g;
      (r[g] == 0 ? f.rm0 : r[g] == 1 ? f.rm1 : f.rm2) |= b;
      (c[g] == 0 ? f.cm0 : c[g] == 1 ? f.cm1 : f.cm2) |= b;
    }
    if (!bg::comc_balanced(f)) {
      std::printf("0 -\n");
      continue;
    }
    switch (n) {
      case 4: emit<4>(f, fact, count_only); break;
      case 5: emit<5>(f, fact, count_only); break;
      case 6: emit<6>(f, fact, count_only); break;
      case 7: emit<7>(f, fact, count_only); break;
      case 8: emit<8>(f, fact, count_only); break;
      case 9: emit<9>(f, fact, count_only); break;
      case 10: emit<10>(f, fact, count_only); break;
      case 11: emit<11>(f, fact, count_only); break;
      case 12: emit<12>(f, fact, count_only); break;
      default: std::printf("0 -\n");
    }
  }
  return 0;
}
