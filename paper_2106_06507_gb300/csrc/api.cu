// api.cu -- the extern "C" entry points of libbg.so (declared in include/bg.h):
// argument checking, colour-matrix objects and kernel launches on the
// caller's stream.  No entry point allocates except the create calls.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "bg_internal.h"

namespace bg {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

bg_status fail(bg_status code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

bg_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return BG_OK;
  return fail(BG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Device status word: first invalid-label code seen by a kernel.
__device__ int g_device_status = 0;

int* device_status_ptr() {
  static std::mutex mu;
  static std::vector<int*> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if ((int)cache.size() <= dev) cache.resize(dev + 1, nullptr);
  if (!cache[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_device_status) != cudaSuccess) return nullptr;
    cache[dev] = static_cast<int*>(ptr);
  }
  return cache[dev];
}

static bool aligned(const void* ptr, size_t a) { return (reinterpret_cast<uintptr_t>(ptr) % a) == 0; }

}  // namespace bg

using namespace bg;

extern "C" {

const char* bg_last_error(void) { return g_last_error.c_str(); }

int64_t bg_num_orderings(int n) {
  if (n < 4 || n > kMaxN) return 0;
  return factorial(n - 2);
}

bg_status bg_colormat_row_host(int n, double* row) {
  if (n < 4 || n > kMaxNCO) return fail(BG_EINVAL, "bg_colormat_row_host: n must be in 4..9");
  if (!row) return fail(BG_EINVAL, "bg_colormat_row_host: row is NULL");
  std::vector<double> r;
  colour_row(n, r);
  std::memcpy(row, r.data(), r.size() * sizeof(double));
  return BG_OK;
}

bg_status bg_colormat_create(int n, bg_colormat** out) {
  if (!out) return fail(BG_EINVAL, "bg_colormat_create: out is NULL");
  *out = nullptr;
  if (n < 4 || n > kMaxN) return fail(BG_EINVAL, "bg_colormat_create: n must be in 4..12");
  if (n > kMaxNCO) return fail(BG_EUNSUPPORTED, "bg_colormat_create: the colour matrix is built for n <= 9");
  bg_colormat* C = new (std::nothrow) bg_colormat();
  if (!C) return fail(BG_ENOMEM, "bg_colormat_create: host allocation failed");
  C->n = n;
  C->k = (int)factorial(n - 2);
  C->C64 = nullptr;
  C->C32 = nullptr;
  cudaGetDevice(&C->device);
  colour_row(n, C->row);
  std::vector<double> dense;
  colour_dense(n, C->row, dense);
  std::vector<float> dense32(dense.size());
  for (size_t i = 0; i < dense.size(); ++i) dense32[i] = (float)dense[i];
  const size_t kk = (size_t)C->k * C->k;
  if (cudaMalloc(&C->C64, kk * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&C->C32, kk * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    bg_colormat_destroy(C);
    return fail(BG_ENOMEM, "bg_colormat_create: device allocation failed");
  }
  bg_status st = cuda_check(cudaMemcpy(C->C64, dense.data(), kk * sizeof(double), cudaMemcpyHostToDevice),
                            "bg_colormat_create: upload");
  if (st == BG_OK)
    st = cuda_check(cudaMemcpy(C->C32, dense32.data(), kk * sizeof(float), cudaMemcpyHostToDevice),
                    "bg_colormat_create: upload");
  if (st != BG_OK) {
    bg_colormat_destroy(C);
    return st;
  }
  *out = C;
  return BG_OK;
}

void bg_colormat_destroy(bg_colormat* C) {
  if (!C) return;
  if (C->C64) cudaFree(C->C64);
  if (C->C32) cudaFree(C->C32);
  delete C;
}

bg_status bg_colormat_row(const bg_colormat* C, double* row) {
  if (!C || !row) return fail(BG_EINVAL, "bg_colormat_row: NULL argument");
  std::memcpy(row, C->row.data(), C->row.size() * sizeof(double));
  return BG_OK;
}

bg_status bg_momenta_rambo(int n, int64_t B, double sqrt_s, const double* u, double* p, double pt_min,
                           uint8_t* accept, void* stream) {
  if (n < 4 || n > kMaxN) return fail(BG_EINVAL, "bg_momenta_rambo: n must be in 4..12");
  if (B < 0) return fail(BG_EINVAL, "bg_momenta_rambo: B < 0");
  if (!(sqrt_s > 0.0)) return fail(BG_EINVAL, "bg_momenta_rambo: sqrt_s must be > 0");
  if (B == 0) return BG_OK;
  if (!u || !p) return fail(BG_EINVAL, "bg_momenta_rambo: NULL u or p");
  if (!aligned(u, 8) || !aligned(p, 8)) return fail(BG_EINVAL, "bg_momenta_rambo: u, p must be 8-byte aligned");
  return cuda_check(launch_rambo(n, B, sqrt_s, u, p, pt_min, accept, (cudaStream_t)stream), "bg_momenta_rambo");
}

bg_status bg_currents_co(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                         bg_prec prec, void* amps, void* stream) {
  if (n < 4 || n > kMaxN) return fail(BG_EINVAL, "bg_currents_co: n must be in 4..12");
  if (n > kMaxNCO) return fail(BG_EUNSUPPORTED, "bg_currents_co: colour-ordered path supports n <= 9");
  if (B < 0) return fail(BG_EINVAL, "bg_currents_co: B < 0");
  if (!(sqrt_s > 0.0)) return fail(BG_EINVAL, "bg_currents_co: sqrt_s must be > 0");
  if (!q) return fail(BG_EINVAL, "bg_currents_co: q is NULL");
  const double qv = std::sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(q[0] > 0.0) || std::fabs(q[0] - qv) > 1e-12 * q[0])
    return fail(BG_EINVAL, "bg_currents_co: q must be light-like with q0 > 0");
  if (prec != BG_F32 && prec != BG_F64) return fail(BG_EINVAL, "bg_currents_co: invalid precision");
  if (B == 0) return BG_OK;
  if (!p || !amps) return fail(BG_EINVAL, "bg_currents_co: NULL p or amps");
  if (!aligned(p, 8) || !aligned(amps, prec == BG_F32 ? 4 : 8))
    return fail(BG_EINVAL, "bg_currents_co: misaligned p or amps");
  int* status = device_status_ptr();
  cudaError_t e = (prec == BG_F32)
                      ? launch_co_f32(n, B, sqrt_s, p, hel, q, static_cast<float*>(amps), status, (cudaStream_t)stream)
                      : launch_co_f64(n, B, sqrt_s, p, hel, q, static_cast<double*>(amps), status,
                                      (cudaStream_t)stream);
  return cuda_check(e, "bg_currents_co");
}

bg_status bg_color_sum(const bg_colormat* C, int64_t B, int H, const void* amps, bg_prec amp_prec,
                       bg_cs_mode mode, double g_s, double sqrt_s, int hel_sampled, const uint8_t* accept,
                       double* me2, void* stream) {
  if (!C) return fail(BG_EINVAL, "bg_color_sum: C is NULL");
  if (B < 0 || H < 1) return fail(BG_EINVAL, "bg_color_sum: B < 0 or H < 1");
  if (amp_prec != BG_F32 && amp_prec != BG_F64) return fail(BG_EINVAL, "bg_color_sum: invalid amp precision");
  if (mode != BG_CS_F64 && mode != BG_CS_F32) return fail(BG_EINVAL, "bg_color_sum: invalid mode");
  if (!(sqrt_s > 0.0)) return fail(BG_EINVAL, "bg_color_sum: sqrt_s must be > 0");
  if (B == 0) return BG_OK;
  if (!amps || !me2) return fail(BG_EINVAL, "bg_color_sum: NULL amps or me2");
  if (!aligned(amps, amp_prec == BG_F32 ? 4 : 8) || !aligned(me2, 8))
    return fail(BG_EINVAL, "bg_color_sum: misaligned amps or me2");
  const int n = C->n;
  ColourSumArgs a;
  a.n = n;
  a.B = B;
  a.H = H;
  a.k = C->k;
  a.amps = amps;
  a.amps_f32 = (amp_prec == BG_F32);
  a.C64 = C->C64;
  a.C32 = C->C32;
  a.scale = std::pow(g_s, 2 * n - 4) * std::pow(sqrt_s, 8 - 2 * n) * (hel_sampled ? std::ldexp(1.0, n) : 1.0);
  a.accept = accept;
  a.me2 = me2;
  cudaError_t e = (mode == BG_CS_F64) ? launch_color_sum_f64(a, (cudaStream_t)stream)
                                      : launch_color_sum_f32(a, (cudaStream_t)stream);
  return cuda_check(e, "bg_color_sum");
}

bg_status bg_device_status(int* status) {
  if (!status) return fail(BG_EINVAL, "bg_device_status: NULL");
  int* d = device_status_ptr();
  if (!d) return fail(BG_ECUDA, "bg_device_status: no device");
  bg_status st = cuda_check(cudaDeviceSynchronize(), "bg_device_status");
  if (st != BG_OK) return st;
  return cuda_check(cudaMemcpy(status, d, sizeof(int), cudaMemcpyDeviceToHost), "bg_device_status");
}

bg_status bg_device_status_reset(void) {
  int* d = device_status_ptr();
  if (!d) return fail(BG_ECUDA, "bg_device_status_reset: no device");
  return cuda_check(cudaMemset(d, 0, sizeof(int)), "bg_device_status_reset");
}

}  // extern "C"
