// Host driver for the colour-dressed kernel's chunk counts
// (paper_2106_06507_gb300/csrc/cd_recursion.cuh), compiled by
// tests/test_cd_chunks_host.py: for n = 4..12 prints, per level L = 2..n-2,
// the number of chunks of ordered partitions, then the top level's.  Runs on
// the host only (constant expressions; no device work).
#include <cstdio>

#include "cd_recursion.cuh"

template <int N>
static void emit() {
  std::printf("%d top %d levels", N, bg::CdShape<N, float>::NCH_TOP);
  for (int L = 2; L < N - 1; ++L) std::printf(" %d", bg::cd_chunks<N, float>(L));
  std::printf("\n");
}

int main() {
  emit<4>();
  emit<5>();
  emit<6>();
  emit<7>();
  emit<8>();
  emit<9>();
  emit<10>();
  emit<11>();
  emit<12>();
  return 0;
}
