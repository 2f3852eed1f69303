// Device counterpart of tests/comc_rank_driver.cpp: the same input lines
// (n and the flow pairs r_0 c_0 r_1 c_1 ..., colours 0..2) and the same
// output, with the count and every rank's order computed by a kernel (one
// thread per flow for the count, one thread per rank for the orders), so
// that tests/test_gpu_comc_rank.py can compare the device build of
// paper_2106_06507_gb300/csrc/comc_rank.h with the host build.
#include <cstdio>
#include <vector>

#include "comc_rank.h"

__constant__ uint32_t c_fact[12];

template <int N>
__global__ void count_kernel(const bg::ComcFlow* f, int nf, uint32_t* cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nf) cnt[i] = bg::comc_balanced(f[i]) ? bg::comc_count(f[i], c_fact) : 0xFFFFFFFFu;
}

template <int N>
__global__ void unrank_kernel(const bg::ComcFlow* f, const long long* first, const int* flow_of, long long total,
                              unsigned long long* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int k = flow_of[i];
  out[i] = bg::comc_unrank<N>((uint32_t)(i - first[k]), f[k], c_fact);
}

template <int N>
static int run(const std::vector<bg::ComcFlow>& flows) {
  const int nf = (int)flows.size();
  bg::ComcFlow* d_f = nullptr;
  uint32_t* d_cnt = nullptr;
  if (cudaMalloc(&d_f, sizeof(bg::ComcFlow) * nf) != cudaSuccess) return 1;
  if (cudaMalloc(&d_cnt, 4 * nf) != cudaSuccess) return 1;
  cudaMemcpy(d_f, flows.data(), sizeof(bg::ComcFlow) * nf, cudaMemcpyHostToDevice);
  count_kernel<N><<<(nf + 127) / 128, 128>>>(d_f, nf, d_cnt);
  std::vector<uint32_t> cnt(nf);
  if (cudaMemcpy(cnt.data(), d_cnt, 4 * nf, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
  std::vector<long long> first(nf);
  std::vector<int> flow_of;
  long long total = 0;
  for (int k = 0; k < nf; ++k) {
    first[k] = total;
    if (cnt[k] != 0xFFFFFFFFu) {
      total += cnt[k];
      for (uint32_t r = 0; r < cnt[k]; ++r) flow_of.push_back(k);
    }
  }
  std::vector<unsigned long long> out(total > 0 ? total : 1);
  if (total > 0) {
    long long* d_first = nullptr;
    int* d_of = nullptr;
    unsigned long long* d_out = nullptr;
    if (cudaMalloc(&d_first, 8 * nf) != cudaSuccess || cudaMalloc(&d_of, 4 * total) != cudaSuccess ||
        cudaMalloc(&d_out, 8 * total) != cudaSuccess)
      return 1;
    cudaMemcpy(d_first, first.data(), 8 * nf, cudaMemcpyHostToDevice);
    cudaMemcpy(d_of, flow_of.data(), 4 * total, cudaMemcpyHostToDevice);
    unrank_kernel<N><<<(unsigned)((total + 127) / 128), 128>>>(d_f, d_first, d_of, total, d_out);
    if (cudaMemcpy(out.data(), d_out, 8 * total, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    cudaFree(d_first);
    cudaFree(d_of);
    cudaFree(d_out);
  }
  for (int k = 0; k < nf; ++k) {
    if (cnt[k] == 0xFFFFFFFFu) {
      std::printf("0 -\n");
      continue;
    }
    std::printf("1 %u", cnt[k]);
    for (uint32_t r = 0; r < cnt[k]; ++r) {
      const unsigned long long pk = out[first[k] + r];
      std::printf(" ");
      for (int p = 1; p < N; ++p) std::printf(p > 1 ? ",%d" : "%d", (int)((pk >> (4 * (p - 1))) & 15u));
    }
    std::printf(" end\n");
  }
  cudaFree(d_f);
  cudaFree(d_cnt);
  return 0;
}

int main() {
  uint32_t fact[12];
  fact[0] = 1;
  for (int k = 1; k < 12; ++k) fact[k] = fact[k - 1] * (uint32_t)k;
  cudaMemcpyToSymbol(c_fact, fact, sizeof(fact));
  // all flows of one input share n
  std::vector<bg::ComcFlow> flows;
  int n = 0, m;
  while (std::scanf("%d", &m) == 1) {
    if (m < 4 || m > 12 || (n && m != n)) return 2;
    n = m;
    std::vector<int> r(n), c(n);
    for (int i = 0; i < n; ++i)
      if (std::scanf("%d %d", &r[i], &c[i]) != 2) return 2;
    bg::ComcFlow f{0, 0, 0, 0, 0, 0, r[0], c[0]};
    for (int g = 1; g < n; ++g) {
      const uint32_t b = 1u << g;
      (r[g] == 0 ? f.rm0 : r[g] == 1 ? f.rm1 : f.rm2) |= b;
      (c[g] == 0 ? f.cm0 : c[g] == 1 ? f.cm1 : f.cm2) |= b;
    }
    flows.push_back(f);
  }
  switch (n) {
    case 4: return run<4>(flows);
    case 5: return run<5>(flows);
    case 6: return run<6>(flows);
    case 7: return run<7>(flows);
    case 8: return run<8>(flows);
    case 9: return run<9>(flows);
    case 10: return run<10>(flows);
    case 11: return run<11>(flows);
    case 12: return run<12>(flows);
    default: return 2;
  }
}
