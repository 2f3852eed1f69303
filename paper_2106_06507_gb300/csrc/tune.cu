// tune.cu -- autotuner for the kernel variants of the two recursions.
//
// Variants compute the same sums in the same order (bitwise identical
// results) and differ only in how the work maps onto the GPU:
//   colour-ordered recursion, sampled helicities, n >= 6:
//     0 = one thread per ordering, 1 / 2 / 3 = depth-first groups of six
//     orderings in blocks of 256 / 128 / 128 threads (3: registers capped
//     for three resident blocks), 4 / 5 = blocks of 64 threads with at most
//     200 / 184 registers per thread;
//   colour-dressed recursion: threads per event (CTA size) and unrolling of
//     the partition loop, see cd_variant_threads() in cd_recursion.cuh.
// bg_autotune times every variant on a synthetic probe batch (Rambo points
// from a hash of the event index, no cut) and records the fastest in a
// process-wide table keyed by (device, algorithm, n, precision); launches
// that are not given a variant explicitly read the table.  The table can be
// saved to and loaded from a text file keyed by the device name.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "bg_internal.h"
#include "cd_recursion.cuh"

namespace bg {
namespace {

using Key = std::tuple<int, int, int, int>;  // device, family, n, prec
std::mutex g_tune_mutex;
std::map<Key, int> g_tune;

int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return d;
}

std::string device_name(int d) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, d) != cudaSuccess) {
    cudaGetLastError();
    return std::string();
  }
  return std::string(prop.name) + " sm_" + std::to_string(prop.major) + std::to_string(prop.minor);
}

int num_variants(int family, int n) {
  if (family == kTuneCO) return co_variants(n, false);
  if (family == kTuneCD) return cd_variants(n);
  return 0;
}

__device__ __forceinline__ uint64_t tune_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Probe inputs from a hash of the element index: uniforms in (0, 1),
// helicities +-1, adjoint colours 1..8.
__global__ void tune_fill_kernel(int64_t B, int n, double* u, int8_t* hel, int8_t* col) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  const int d = 4 * (n - 2);
  for (int j = 0; j < d; ++j) {
    const uint64_t r = tune_mix(0x9E3779B97F4A7C15ull * (uint64_t)(i * d + j + 1));
    u[i * d + j] = ((double)(r >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  }
  for (int g = 0; g < n; ++g) {
    const uint64_t r = tune_mix(0xD1B54A32D192ED03ull * (uint64_t)(i * n + g + 1));
    hel[(int64_t)g * B + i] = (r >> 63) ? 1 : -1;
    col[(int64_t)g * B + i] = (int8_t)(1 + ((r >> 20) & 7));
  }
}

}  // namespace

int tune_variant(int family, int n, int prec) {
  const int d = current_device();
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  auto it = g_tune.find(Key(d, family, n, prec));
  return it == g_tune.end() ? -1 : it->second;
}

}  // namespace bg

using namespace bg;

namespace {

int family_of(bg_algo algo) { return algo == BG_ALGO_CD ? kTuneCD : kTuneCO; }

bg_status check_args(const char* fn, bg_algo algo, int n, bg_prec prec) {
  if (algo != BG_ALGO_CO && algo != BG_ALGO_CD) return fail(BG_EINVAL, std::string(fn) + ": invalid algorithm");
  if (prec != BG_F32 && prec != BG_F64) return fail(BG_EINVAL, std::string(fn) + ": invalid precision");
  const int nmax = algo == BG_ALGO_CD ? kMaxN : kMaxNCO;
  if (n < 4 || n > nmax) return fail(BG_EINVAL, std::string(fn) + ": n outside the algorithm's range");
  return BG_OK;
}

struct ProbeBuffers {
  std::vector<void*> ptrs;
  ~ProbeBuffers() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename P>
  bool alloc(P** out, size_t bytes) {
    void* v = nullptr;
    if (device_alloc(&v, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    ptrs.push_back(v);
    *out = static_cast<P*>(v);
    return true;
  }
};

}  // namespace

extern "C" {

int bg_tune_num_variants(bg_algo algo, int n) {
  if (check_args("bg_tune_num_variants", algo, n, BG_F32) != BG_OK) return 0;
  return num_variants(family_of(algo), n);
}

bg_status bg_tune_set(bg_algo algo, int n, bg_prec prec, int variant) {
  bg_status st = check_args("bg_tune_set", algo, n, prec);
  if (st != BG_OK) return st;
  if (variant < -1 || variant >= num_variants(family_of(algo), n))
    return fail(BG_EINVAL, "bg_tune_set: variant out of range");
  const int d = current_device();
  if (d < 0) return fail(BG_ECUDA, "bg_tune_set: no CUDA device");
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  const Key k(d, family_of(algo), n, (int)prec);
  if (variant < 0)
    g_tune.erase(k);
  else
    g_tune[k] = variant;
  return BG_OK;
}

bg_status bg_tune_get(bg_algo algo, int n, bg_prec prec, int* variant) {
  bg_status st = check_args("bg_tune_get", algo, n, prec);
  if (st != BG_OK) return st;
  if (!variant) return fail(BG_EINVAL, "bg_tune_get: NULL");
  if (current_device() < 0) return fail(BG_ECUDA, "bg_tune_get: no CUDA device");
  *variant = tune_variant(family_of(algo), n, (int)prec);
  return BG_OK;
}

bg_status bg_autotune(bg_algo algo, int n, bg_prec prec, int64_t probe_batch, void* stream, int* best,
                      float* ms) {
  AllocScope scope;
  bg_status st = check_args("bg_autotune", algo, n, prec);
  if (st != BG_OK) return st;
  const int fam = family_of(algo);
  const int nv = num_variants(fam, n);
  int64_t B = probe_batch;
  if (B <= 0) B = (algo == BG_ALGO_CO) ? (n <= 8 ? 65536 : 16384) : (n <= 9 ? 16384 : (int64_t)32768 >> (n - 9));
  cudaStream_t s = (cudaStream_t)stream;
  const int sms = device_sms();
  if (sms <= 0) return fail(BG_ECUDA, "bg_autotune: no CUDA device");
  const size_t tsz = prec == BG_F32 ? 4 : 8;
  ProbeBuffers buf;
  double *u = nullptr, *p = nullptr, *me2 = nullptr;
  int8_t *hel = nullptr, *col = nullptr;
  void* work = nullptr;
  size_t work_bytes = 0;
  if (algo == BG_ALGO_CO) {
    work_bytes = (size_t)B * factorial(n - 2) * tsz;
  } else {
    work_bytes = prec == BG_F32 ? cd_workspace_bytes_f32(n, sms) : cd_workspace_bytes_f64(n, sms);
    if (work_bytes == 0) return fail(BG_ECUDA, "bg_autotune: colour-dressed kernel cannot launch");
  }
  if (!buf.alloc(&u, (size_t)B * 4 * (n - 2) * sizeof(double)) || !buf.alloc(&p, (size_t)B * 4 * n * sizeof(double)) ||
      !buf.alloc(&me2, (size_t)B * sizeof(double)) || !buf.alloc(&hel, (size_t)B * n) ||
      !buf.alloc(&col, (size_t)B * n) || !buf.alloc(&work, work_bytes))
    return fail(BG_ENOMEM, "bg_autotune: device allocation for the probe batch failed");
  tune_fill_kernel<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(B, n, u, hel, col);
  st = cuda_check(cudaGetLastError(), "bg_autotune: fill");
  if (st != BG_OK) return st;
  const double sqrt_s = 1000.0;
  st = cuda_check(launch_rambo(n, B, sqrt_s, u, p, -1.0, nullptr, s), "bg_autotune: rambo");
  if (st != BG_OK) return st;
  const double q[4] = {1.0, 0.0, 0.0, 1.0};
  CdParams prm;
  prm.B = B;
  prm.inv_sqrt_s = 1.0 / sqrt_s;
  prm.scale = 1.0;
  prm.flow = 0;
  for (int m = 0; m < 4; ++m) prm.q.v[m] = q[m];
  int* status = device_status_ptr();
  auto run = [&](int v) -> cudaError_t {
    if (algo == BG_ALGO_CO)
      return prec == BG_F32 ? launch_co_f32(n, B, sqrt_s, p, hel, q, static_cast<float*>(work), status, s, nullptr, v)
                            : launch_co_f64(n, B, sqrt_s, p, hel, q, static_cast<double*>(work), status, s, nullptr, v);
    return prec == BG_F32 ? launch_cd_f32(n, prm, p, hel, col, nullptr, me2, work, status, sms, s, v)
                          : launch_cd_f64(n, prm, p, hel, col, nullptr, me2, work, status, sms, s, v);
  };
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return fail(BG_ECUDA, "bg_autotune: events");
  }
  int arg = 0;
  float bestms = 0.0f;
  cudaError_t err = cudaSuccess;
  for (int v = 0; v < nv && err == cudaSuccess; ++v) {
    err = run(v);  // warm-up (first launch sets kernel attributes)
    float tmin = 0.0f;
    for (int r = 0; r < 3 && err == cudaSuccess; ++r) {
      cudaEventRecord(e0, s);
      err = run(v);
      cudaEventRecord(e1, s);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float t = 0.0f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
      if (r == 0 || t < tmin) tmin = t;
    }
    if (ms) ms[v] = tmin;
    if (v == 0 || tmin < bestms) {
      bestms = tmin;
      arg = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  st = cuda_check(err, "bg_autotune: probe launch");
  if (st != BG_OK) return st;
  st = bg_tune_set(algo, n, prec, arg);
  if (st == BG_OK && best) *best = arg;
  return st;
}

bg_status bg_tune_save(const char* path) {
  if (!path) return fail(BG_EINVAL, "bg_tune_save: NULL path");
  std::vector<std::pair<Key, int>> entries;
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    entries.assign(g_tune.begin(), g_tune.end());
  }
  FILE* f = std::fopen(path, "w");
  if (!f) return fail(BG_EINVAL, std::string("bg_tune_save: cannot open ") + path);
  std::fprintf(f, "bg-tune 1\n");
  for (const auto& kv : entries) {
    const std::string name = device_name(std::get<0>(kv.first));
    std::fprintf(f, "%s\t%d\t%d\t%d\t%d\n", name.c_str(), std::get<1>(kv.first), std::get<2>(kv.first),
                 std::get<3>(kv.first), kv.second);
  }
  const bool ok = std::fclose(f) == 0;
  return ok ? BG_OK : fail(BG_EINVAL, "bg_tune_save: write failed");
}

bg_status bg_tune_load(const char* path) {
  if (!path) return fail(BG_EINVAL, "bg_tune_load: NULL path");
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(BG_EINVAL, std::string("bg_tune_load: cannot open ") + path);
  char line[512];
  if (!std::fgets(line, sizeof line, f) || std::strncmp(line, "bg-tune 1", 9) != 0) {
    std::fclose(f);
    return fail(BG_EINVAL, "bg_tune_load: not a tuning file");
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    ndev = 0;
  }
  std::vector<std::string> names(ndev);
  for (int d = 0; d < ndev; ++d) names[d] = device_name(d);
  bg_status st = BG_OK;
  while (std::fgets(line, sizeof line, f)) {
    char* tab = std::strchr(line, '\t');
    int fam, n, prec, v;
    if (!tab || std::sscanf(tab + 1, "%d\t%d\t%d\t%d", &fam, &n, &prec, &v) != 4) {
      st = fail(BG_EINVAL, "bg_tune_load: malformed line");
      break;
    }
    *tab = '\0';
    if ((fam != kTuneCO && fam != kTuneCD) || n < 4 || n > kMaxN || (prec != BG_F32 && prec != BG_F64) || v < 0 ||
        v >= num_variants(fam, n)) {
      st = fail(BG_EINVAL, "bg_tune_load: entry out of range");
      break;
    }
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    for (int d = 0; d < ndev; ++d)
      if (names[d] == line) g_tune[Key(d, fam, n, prec)] = v;
  }
  std::fclose(f);
  return st;
}

}  // extern "C"
