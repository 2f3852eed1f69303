// api.cu -- the extern "C" entry points of libbg.so (declared in include/bg.h):
// argument checking, colour-matrix objects and kernel launches on the
// caller's stream.  No entry point allocates except the create calls.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "bg_internal.h"
#include "cd_recursion.cuh"
#include "comc.cuh"

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

// Allocation counting for BG_FAIL_ALLOC (see bg_internal.h).
static thread_local int t_alloc_depth = 0;
static thread_local int t_alloc_count = 0;

AllocScope::AllocScope() {
  if (t_alloc_depth++ == 0) t_alloc_count = 0;
}
AllocScope::~AllocScope() { --t_alloc_depth; }

cudaError_t device_alloc(void** ptr, size_t bytes) {
  *ptr = nullptr;
  ++t_alloc_count;
  const char* inject = std::getenv("BG_FAIL_ALLOC");
  if (inject && std::atoi(inject) == t_alloc_count) return cudaErrorMemoryAllocation;
  return cudaMalloc(ptr, bytes);
}

bg_status alloc_failure(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a non-sticky error
  if (e == cudaErrorMemoryAllocation) return fail(BG_ENOMEM, std::string(what) + ": device allocation failed");
  return fail(BG_ECUDA, std::string(what) + ": device allocation failed: " + cudaGetErrorString(e));
}

}  // namespace bg

using namespace bg;

namespace bg {
int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms;
}
}  // namespace bg

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
  AllocScope scope;
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
  C->tc_tiles_raw = nullptr;
  C->tc_tiles = nullptr;
  C->tc_g = 0.0;
  C->tc_nt = C->tc_ntiles = C->tc_kchunks = 0;
  C->tc_cpl = 1;
  cudaGetDevice(&C->device);
  colour_row(n, C->row);
  std::vector<double> dense;
  colour_dense(n, C->row, dense);
  std::vector<float> dense32(dense.size());
  for (size_t i = 0; i < dense.size(); ++i) dense32[i] = (float)dense[i];
  const size_t kk = (size_t)C->k * C->k;
  cudaError_t ae = device_alloc((void**)&C->C64, kk * sizeof(double));
  if (ae == cudaSuccess) ae = device_alloc((void**)&C->C32, kk * sizeof(float));
  if (ae != cudaSuccess) {
    bg_colormat_destroy(C);
    return alloc_failure(ae, "bg_colormat_create");
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
  std::vector<uint16_t> tiles;
  if (build_tc_tiles(n, dense, C->k, tiles, C->tc_g, C->tc_nt, C->tc_ntiles, C->tc_kchunks, C->tc_cpl)) {
    ae = device_alloc((void**)&C->tc_tiles_raw, tiles.size() * 2);
    if (ae != cudaSuccess) {
      bg_colormat_destroy(C);
      return alloc_failure(ae, "bg_colormat_create");
    }
    st = cuda_check(cudaMemcpy(C->tc_tiles_raw, tiles.data(), tiles.size() * 2, cudaMemcpyHostToDevice),
                    "bg_colormat_create: upload");
    if (st != BG_OK) {
      bg_colormat_destroy(C);
      return st;
    }
    C->tc_tiles = reinterpret_cast<const __nv_bfloat16*>(C->tc_tiles_raw);
  }
  *out = C;
  return BG_OK;
}

void bg_colormat_destroy(bg_colormat* C) {
  if (!C) return;
  if (C->C64) cudaFree(C->C64);
  if (C->C32) cudaFree(C->C32);
  if (C->tc_tiles_raw) cudaFree(C->tc_tiles_raw);
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

bg_status bg_currents_co_tensor(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                                bg_prec prec, void* amps, void* stream) {
  if (n < 4 || n > kMaxN) return fail(BG_EINVAL, "bg_currents_co_tensor: n must be in 4..12");
  if (n > kMaxNCO) return fail(BG_EUNSUPPORTED, "bg_currents_co_tensor: colour-ordered path supports n <= 9");
  if (B < 0) return fail(BG_EINVAL, "bg_currents_co_tensor: B < 0");
  if (!(sqrt_s > 0.0)) return fail(BG_EINVAL, "bg_currents_co_tensor: sqrt_s must be > 0");
  if (!q) return fail(BG_EINVAL, "bg_currents_co_tensor: q is NULL");
  const double qv = std::sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(q[0] > 0.0) || std::fabs(q[0] - qv) > 1e-12 * q[0])
    return fail(BG_EINVAL, "bg_currents_co_tensor: q must be light-like with q0 > 0");
  if (prec != BG_F32 && prec != BG_F64) return fail(BG_EINVAL, "bg_currents_co_tensor: invalid precision");
  if (B == 0) return BG_OK;
  if (!p || !amps) return fail(BG_EINVAL, "bg_currents_co_tensor: NULL p or amps");
  if (!aligned(p, 8) || !aligned(amps, prec == BG_F32 ? 4 : 8))
    return fail(BG_EINVAL, "bg_currents_co_tensor: misaligned p or amps");
  int* status = device_status_ptr();
  cudaError_t e = (prec == BG_F32) ? launch_co_tensor_f32(n, B, sqrt_s, p, hel, q, static_cast<float*>(amps), status,
                                                          (cudaStream_t)stream)
                                   : launch_co_tensor_f64(n, B, sqrt_s, p, hel, q, static_cast<double*>(amps),
                                                          status, (cudaStream_t)stream);
  return cuda_check(e, "bg_currents_co_tensor");
}

bg_status bg_color_sum(const bg_colormat* C, int64_t B, int H, const void* amps, bg_prec amp_prec,
                       bg_cs_mode mode, double g_s, double sqrt_s, int hel_sampled, const uint8_t* accept,
                       double* me2, void* stream) {
  if (!C) return fail(BG_EINVAL, "bg_color_sum: C is NULL");
  if (B < 0 || H < 1) return fail(BG_EINVAL, "bg_color_sum: B < 0 or H < 1");
  if (amp_prec != BG_F32 && amp_prec != BG_F64) return fail(BG_EINVAL, "bg_color_sum: invalid amp precision");
  if (mode != BG_CS_F64 && mode != BG_CS_F32 && mode != BG_CS_TC_BF16)
    return fail(BG_EINVAL, "bg_color_sum: invalid mode");
  if (mode == BG_CS_TC_BF16 && (!C->tc_tiles || H != 1))
    return fail(BG_EUNSUPPORTED, "bg_color_sum: tensor-core mode needs 6 <= n <= 9 and H = 1");
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
  cudaError_t e = (mode == BG_CS_F64)   ? launch_color_sum_f64(a, (cudaStream_t)stream)
                  : (mode == BG_CS_F32) ? launch_color_sum_f32(a, (cudaStream_t)stream)
                                        : launch_color_sum_tc(a, C, device_status_ptr(), (cudaStream_t)stream);
  return cuda_check(e, "bg_color_sum");
}


bg_status bg_cd_workspace_bytes(int n, bg_prec prec, int64_t* bytes) {
  if (!bytes) return fail(BG_EINVAL, "bg_cd_workspace_bytes: NULL");
  if (n < 4 || n > kMaxN) return fail(BG_EINVAL, "bg_cd_workspace_bytes: n must be in 4..12");
  if (prec != BG_F32 && prec != BG_F64) return fail(BG_EINVAL, "bg_cd_workspace_bytes: invalid precision");
  const int sms = device_sms();
  if (sms <= 0) return fail(BG_ECUDA, "bg_cd_workspace_bytes: no device");
  const size_t ws = (prec == BG_F32) ? cd_workspace_bytes_f32(n, sms) : cd_workspace_bytes_f64(n, sms);
  if (ws == 0) return fail(BG_ECUDA, "bg_cd_workspace_bytes: kernel configuration not supported on this device");
  *bytes = (int64_t)ws;
  return BG_OK;
}

bg_status bg_currents_cd(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel,
                         const int8_t* colors, bg_color_mode cm, const double* q, bg_prec prec, double g_s,
                         const uint8_t* accept, double* me2, void* workspace, int64_t workspace_bytes,
                         void* stream) {
  if (n < 4 || n > kMaxN) return fail(BG_EINVAL, "bg_currents_cd: n must be in 4..12");
  if (B < 0) return fail(BG_EINVAL, "bg_currents_cd: B < 0");
  if (!(sqrt_s > 0.0)) return fail(BG_EINVAL, "bg_currents_cd: sqrt_s must be > 0");
  if (cm != BG_COL_ADJOINT && cm != BG_COL_FLOW) return fail(BG_EINVAL, "bg_currents_cd: invalid colour mode");
  if (prec != BG_F32 && prec != BG_F64) return fail(BG_EINVAL, "bg_currents_cd: invalid precision");
  if (!q) return fail(BG_EINVAL, "bg_currents_cd: q is NULL");
  const double qv = std::sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(q[0] > 0.0) || std::fabs(q[0] - qv) > 1e-12 * q[0])
    return fail(BG_EINVAL, "bg_currents_cd: q must be light-like with q0 > 0");
  if (B == 0) return BG_OK;
  if (!p || !hel || !colors || !me2 || !workspace) return fail(BG_EINVAL, "bg_currents_cd: NULL argument");
  int64_t need = 0;
  bg_status st = bg_cd_workspace_bytes(n, prec, &need);
  if (st != BG_OK) return st;
  if (workspace_bytes < need)
    return fail(BG_EINVAL, "bg_currents_cd: workspace smaller than bg_cd_workspace_bytes(n, prec)");
  if (!aligned(workspace, 256) || !aligned(p, 8) || !aligned(me2, 8))
    return fail(BG_EINVAL, "bg_currents_cd: misaligned pointer (workspace needs 256-byte alignment)");
  CdParams prm;
  prm.B = B;
  prm.inv_sqrt_s = 1.0 / sqrt_s;
  const double wcol = std::pow(cm == BG_COL_FLOW ? 9.0 : 8.0, n);
  prm.scale = wcol * std::ldexp(1.0, n) * std::pow(g_s, 2 * n - 4) * std::pow(sqrt_s, 8 - 2 * n) *
              std::ldexp(1.0, -(n - 2));
  prm.flow = (cm == BG_COL_FLOW) ? 1 : 0;
  for (int m = 0; m < 4; ++m) prm.q.v[m] = q[m];
  const int sms = device_sms();
  cudaError_t e = (prec == BG_F32) ? launch_cd_f32(n, prm, p, hel, colors, accept, me2, workspace,
                                                   device_status_ptr(), sms, (cudaStream_t)stream)
                                   : launch_cd_f64(n, prm, p, hel, colors, accept, me2, workspace,
                                                   device_status_ptr(), sms, (cudaStream_t)stream);
  return cuda_check(e, "bg_currents_cd");
}

bg_status bg_currents_cd_cont(int n, int64_t B, double sqrt_s, const double* p, const double* ang, const double* q,
                              bg_prec prec, double g_s, const uint8_t* accept, double* me2, void* workspace,
                              int64_t workspace_bytes, void* stream) {
  if (n < 4 || n > kMaxN) return fail(BG_EINVAL, "bg_currents_cd_cont: n must be in 4..12");
  if (B < 0) return fail(BG_EINVAL, "bg_currents_cd_cont: B < 0");
  if (!(sqrt_s > 0.0)) return fail(BG_EINVAL, "bg_currents_cd_cont: sqrt_s must be > 0");
  if (prec != BG_F32 && prec != BG_F64) return fail(BG_EINVAL, "bg_currents_cd_cont: invalid precision");
  if (!q) return fail(BG_EINVAL, "bg_currents_cd_cont: q is NULL");
  const double qv = std::sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(q[0] > 0.0) || std::fabs(q[0] - qv) > 1e-12 * q[0])
    return fail(BG_EINVAL, "bg_currents_cd_cont: q must be light-like with q0 > 0");
  if (B == 0) return BG_OK;
  if (!p || !ang || !me2 || !workspace) return fail(BG_EINVAL, "bg_currents_cd_cont: NULL argument");
  int64_t need = 0;
  bg_status st = bg_cd_workspace_bytes(n, prec, &need);
  if (st != BG_OK) return st;
  if (workspace_bytes < need)
    return fail(BG_EINVAL, "bg_currents_cd_cont: workspace smaller than bg_cd_workspace_bytes(n, prec)");
  if (!aligned(workspace, 256) || !aligned(p, 8) || !aligned(ang, 8) || !aligned(me2, 8))
    return fail(BG_EINVAL, "bg_currents_cd_cont: misaligned pointer (workspace needs 256-byte alignment)");
  CdParams prm;
  prm.B = B;
  prm.inv_sqrt_s = 1.0 / sqrt_s;
  prm.scale = std::pow(9.0, n) * std::ldexp(1.0, n) * std::pow(g_s, 2 * n - 4) * std::pow(sqrt_s, 8 - 2 * n) *
              std::ldexp(1.0, -(n - 2));
  prm.flow = 2;
  prm.ang = ang;
  for (int m = 0; m < 4; ++m) prm.q.v[m] = q[m];
  const int sms = device_sms();
  cudaError_t e = (prec == BG_F32) ? launch_cd_f32(n, prm, p, nullptr, nullptr, accept, me2, workspace,
                                                   device_status_ptr(), sms, (cudaStream_t)stream)
                                   : launch_cd_f64(n, prm, p, nullptr, nullptr, accept, me2, workspace,
                                                   device_status_ptr(), sms, (cudaStream_t)stream);
  return cuda_check(e, "bg_currents_cd_cont");
}

bg_status bg_comc_workspace_bytes(int n, int64_t B, bg_prec prec, int64_t* bytes) {
  if (!bytes) return fail(BG_EINVAL, "bg_comc_workspace_bytes: bytes is NULL");
  if (n < 4 || n > kMaxN) return fail(BG_EINVAL, "bg_comc_workspace_bytes: n must be in 4..12");
  if (B < 0) return fail(BG_EINVAL, "bg_comc_workspace_bytes: B < 0");
  if (prec != BG_F32 && prec != BG_F64) return fail(BG_EINVAL, "bg_comc_workspace_bytes: invalid precision");
  *bytes = (int64_t)comc_workspace_bytes(n, B, prec == BG_F32 ? 4 : 8);
  return BG_OK;
}

bg_status bg_currents_co_mc(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel,
                            const int8_t* colors, const double* q, bg_prec prec, double g_s, const uint8_t* accept,
                            double* me2, void* workspace, int64_t workspace_bytes, void* stream) {
  if (n < 4 || n > kMaxN) return fail(BG_EINVAL, "bg_currents_co_mc: n must be in 4..12");
  if (B < 0) return fail(BG_EINVAL, "bg_currents_co_mc: B < 0");
  if (!(sqrt_s > 0.0)) return fail(BG_EINVAL, "bg_currents_co_mc: sqrt_s must be > 0");
  if (prec != BG_F32 && prec != BG_F64) return fail(BG_EINVAL, "bg_currents_co_mc: invalid precision");
  if (!q) return fail(BG_EINVAL, "bg_currents_co_mc: q is NULL");
  const double qv = std::sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(q[0] > 0.0) || std::fabs(q[0] - qv) > 1e-12 * q[0])
    return fail(BG_EINVAL, "bg_currents_co_mc: q must be light-like with q0 > 0");
  if (B == 0) return BG_OK;
  if (!p || !hel || !colors || !me2 || !workspace) return fail(BG_EINVAL, "bg_currents_co_mc: NULL argument");
  if (workspace_bytes < (int64_t)comc_workspace_bytes(n, B, prec == BG_F32 ? 4 : 8))
    return fail(BG_EINVAL, "bg_currents_co_mc: workspace smaller than bg_comc_workspace_bytes(n, B, prec)");
  if (!aligned(p, 8) || !aligned(me2, 8) || !aligned(workspace, 256))
    return fail(BG_EINVAL, "bg_currents_co_mc: misaligned pointer (workspace needs 256-byte alignment)");
  ComcParams prm;
  prm.B = B;
  prm.inv_sqrt_s = 1.0 / sqrt_s;
  prm.scale = std::pow(9.0, n) * std::ldexp(1.0, n) * std::pow(g_s, 2 * n - 4) * std::pow(sqrt_s, 8 - 2 * n) *
              std::ldexp(1.0, -(n - 2));
  const int sms = device_sms();
  cudaError_t e = (prec == BG_F32) ? launch_comc_f32(n, prm, p, hel, colors, accept, q, me2, workspace, sms,
                                                     device_status_ptr(), (cudaStream_t)stream)
                                   : launch_comc_f64(n, prm, p, hel, colors, accept, q, me2, workspace, sms,
                                                     device_status_ptr(), (cudaStream_t)stream);
  return cuda_check(e, "bg_currents_co_mc");
}

// ---------------------------------------------------------------------------
// plans
// ---------------------------------------------------------------------------
static bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

void bg_plan_destroy(bg_plan* P) {
  if (!P) return;
  void* bufs[] = {P->u, P->hel, P->colors, P->p, P->accept, P->amps, P->me2, P->Y, P->kbar, P->ebar};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (P->C) bg_colormat_destroy(P->C);
  delete P;
}

int64_t bg_plan_workspace_bytes(const bg_plan* P) { return P ? P->bytes : 0; }

bg_status bg_plan_create(const bg_plan_desc* d, bg_plan** out) {
  AllocScope scope;
  if (!d || !out) return fail(BG_EINVAL, "bg_plan_create: NULL argument");
  *out = nullptr;
  const int n = d->n;
  if (n < 4 || n > kMaxN) return fail(BG_EINVAL, "bg_plan_create: n must be in 4..12");
  if (d->max_batch < 1) return fail(BG_EINVAL, "bg_plan_create: max_batch must be >= 1");
  if (!(d->sqrt_s > 0.0)) return fail(BG_EINVAL, "bg_plan_create: sqrt_s must be > 0");
  if (d->prec != BG_F32 && d->prec != BG_F64) return fail(BG_EINVAL, "bg_plan_create: invalid precision");
  if (d->algo != BG_ALGO_CO && d->algo != BG_ALGO_CD) return fail(BG_EINVAL, "bg_plan_create: invalid algorithm");
  if (d->algo == BG_ALGO_CD) return fail(BG_EUNSUPPORTED, "bg_plan_create: colour-dressed plans not available");
  if (n > kMaxNCO) return fail(BG_EUNSUPPORTED, "bg_plan_create: colour-ordered path supports n <= 9");
  if (d->cs_mode != BG_CS_F64 && d->cs_mode != BG_CS_F32 && d->cs_mode != BG_CS_TC_BF16)
    return fail(BG_EINVAL, "bg_plan_create: invalid cs_mode");
  if (d->grad && (n > 8 || !d->hel_sampled))
    return fail(BG_EUNSUPPORTED, "bg_plan_create: gradients need n <= 8 and sampled helicities");
  if (d->cs_mode == BG_CS_TC_BF16 && (n < 6 || !d->hel_sampled))
    return fail(BG_EUNSUPPORTED, "bg_plan_create: tensor-core colour sum needs 6 <= n <= 9, sampled helicities");
  const double qv = std::sqrt(d->q[1] * d->q[1] + d->q[2] * d->q[2] + d->q[3] * d->q[3]);
  if (!(d->q[0] > 0.0) || std::fabs(d->q[0] - qv) > 1e-12 * d->q[0])
    return fail(BG_EINVAL, "bg_plan_create: q must be light-like with q0 > 0");
  bg_plan* P = new (std::nothrow) bg_plan();
  if (!P) return fail(BG_ENOMEM, "bg_plan_create: host allocation failed");
  std::memset(static_cast<void*>(P), 0, sizeof(bg_plan));
  P->d = *d;
  P->k = (int)factorial(n - 2);
  P->H = d->hel_sampled ? 1 : (1 << n);
  cudaGetDevice(&P->device);
  bg_status st = bg_colormat_create(n, &P->C);
  if (st != BG_OK) {
    delete P;
    return st;
  }
  const int64_t B = d->max_batch;
  const size_t amp_bytes = (size_t)B * P->H * P->k * (d->prec == BG_F32 ? 4 : 8);
  struct Req {
    void** ptr;
    size_t bytes;
  } reqs[] = {{(void**)&P->u, (size_t)B * 4 * (n - 2) * sizeof(double)},
              {(void**)&P->hel, (size_t)B * n},
              {(void**)&P->colors, (size_t)B * 2 * n},
              {(void**)&P->p, (size_t)B * 4 * n * sizeof(double)},
              {(void**)&P->accept, (size_t)B},
              {&P->amps, amp_bytes},
              {(void**)&P->me2, (size_t)B * sizeof(double)},
              {&P->Y, d->grad ? amp_bytes : 0},
              {(void**)&P->kbar, d->grad ? (size_t)B * n * 4 * sizeof(double) : 0},
              {(void**)&P->ebar, d->grad ? (size_t)B * n * 4 * sizeof(double) : 0}};
  P->bytes = (int64_t)P->C->k * P->C->k * 12;
  for (auto& r : reqs) {
    if (r.bytes == 0) continue;
    cudaError_t ae = device_alloc(r.ptr, r.bytes);
    if (ae != cudaSuccess) {
      bg_plan_destroy(P);
      return alloc_failure(ae, "bg_plan_create");
    }
    P->bytes += (int64_t)r.bytes;
  }
  *out = P;
  return BG_OK;
}

// The whole path for one plan; `sync`: wait for a host output before
// returning (bg_me2_batch) or not (bg_me2_batch_async).
static bg_status me2_batch_impl(bg_plan* P, int64_t B, const double* u, const int8_t* hel, double* me2,
                                void* stream, bool sync) {
  if (!P) return fail(BG_EINVAL, "bg_me2_batch: plan is NULL");
  if (B < 0 || B > P->d.max_batch) return fail(BG_EINVAL, "bg_me2_batch: B outside 0..max_batch");
  if (B == 0) return BG_OK;
  if (!u || !me2) return fail(BG_EINVAL, "bg_me2_batch: NULL u or me2");
  if (P->d.hel_sampled && !hel) return fail(BG_EINVAL, "bg_me2_batch: hel is required for sampled helicities");
  const int n = P->d.n;
  cudaStream_t s = (cudaStream_t)stream;
  const double* ud = u;
  if (!is_device_ptr(u)) {
    bg_status st = cuda_check(cudaMemcpyAsync(P->u, u, (size_t)B * 4 * (n - 2) * sizeof(double),
                                              cudaMemcpyHostToDevice, s),
                              "bg_me2_batch: copy u");
    if (st != BG_OK) return st;
    ud = P->u;
  }
  const int8_t* hd = P->d.hel_sampled ? hel : nullptr;
  if (hd && !is_device_ptr(hd)) {
    // host layout [n][B] -> device [n][B] (row stride B in both)
    bg_status st = cuda_check(cudaMemcpyAsync(P->hel, hd, (size_t)B * n, cudaMemcpyHostToDevice, s),
                              "bg_me2_batch: copy hel");
    if (st != BG_OK) return st;
    hd = P->hel;
  }
  const bool host_out = !is_device_ptr(me2);
  double* md = host_out ? P->me2 : me2;
  bg_status st = bg_momenta_rambo(n, B, P->d.sqrt_s, ud, P->p, P->d.pt_min, P->accept, stream);
  if (st != BG_OK) return st;
  st = bg_currents_co(n, B, P->d.sqrt_s, P->p, hd, P->d.q, P->d.prec, P->amps, stream);
  if (st != BG_OK) return st;
  st = bg_color_sum(P->C, B, P->H, P->amps, P->d.prec, P->d.cs_mode, P->d.g_s, P->d.sqrt_s, P->d.hel_sampled,
                    P->accept, md, stream);
  if (st != BG_OK) return st;
  if (host_out) {
    st = cuda_check(cudaMemcpyAsync(me2, md, (size_t)B * sizeof(double), cudaMemcpyDeviceToHost, s),
                    "bg_me2_batch: copy me2");
    if (st != BG_OK) return st;
    if (sync) st = cuda_check(cudaStreamSynchronize(s), "bg_me2_batch: synchronise");
  }
  return st;
}

bg_status bg_me2_batch(bg_plan* P, int64_t B, const double* u, const int8_t* hel, const int8_t* colors,
                       double* me2, void* stream) {
  (void)colors;
  return me2_batch_impl(P, B, u, hel, me2, stream, true);
}

bg_status bg_me2_batch_async(bg_plan* P, int64_t B, const double* u, const int8_t* hel, double* me2, void* stream) {
  return me2_batch_impl(P, B, u, hel, me2, stream, false);
}

bg_status bg_me2_grad(bg_plan* P, int64_t B, const double* u, const int8_t* hel, const double* upstream,
                      double* me2, double* grad_u, void* stream) {
  if (!P) return fail(BG_EINVAL, "bg_me2_grad: plan is NULL");
  if (!P->d.grad || !P->kbar) return fail(BG_EINVAL, "bg_me2_grad: plan was not created with grad = 1");
  if (B < 0 || B > P->d.max_batch) return fail(BG_EINVAL, "bg_me2_grad: B outside 0..max_batch");
  if (B == 0) return BG_OK;
  if (!u || !hel || !grad_u) return fail(BG_EINVAL, "bg_me2_grad: NULL u, hel or grad_u");
  if (!is_device_ptr(u) || !is_device_ptr(hel) || !is_device_ptr(grad_u) || (me2 && !is_device_ptr(me2)) ||
      (upstream && !is_device_ptr(upstream)))
    return fail(BG_EINVAL, "bg_me2_grad: all buffers must be device memory");
  const int n = P->d.n;
  cudaStream_t s = (cudaStream_t)stream;
  bg_status st = bg_momenta_rambo(n, B, P->d.sqrt_s, u, P->p, P->d.pt_min, P->accept, stream);
  if (st != BG_OK) return st;
  st = bg_currents_co(n, B, P->d.sqrt_s, P->p, hel, P->d.q, P->d.prec, P->amps, stream);
  if (st != BG_OK) return st;
  ColourSumArgs a;
  a.n = n;
  a.B = B;
  a.H = 1;
  a.k = P->k;
  a.amps = P->amps;
  a.amps_f32 = (P->d.prec == BG_F32);
  a.C64 = P->C->C64;
  a.C32 = P->C->C32;
  a.scale = std::pow(P->d.g_s, 2 * n - 4) * std::pow(P->d.sqrt_s, 8 - 2 * n) * std::ldexp(1.0, n);
  a.accept = P->accept;
  a.me2 = me2 ? me2 : P->me2;
  a.Y = P->Y;
  cudaError_t e = (P->d.cs_mode == BG_CS_F64)   ? launch_color_sum_f64(a, s)
                  : (P->d.cs_mode == BG_CS_F32) ? launch_color_sum_f32(a, s)
                                                : launch_color_sum_tc(a, P->C, device_status_ptr(), s);
  st = cuda_check(e, "bg_me2_grad: colour sum");
  if (st != BG_OK) return st;
  e = (P->d.prec == BG_F32)
          ? launch_co_grad_f32(n, B, P->d.sqrt_s, P->p, hel, P->d.q, static_cast<const float*>(P->Y), P->kbar,
                               P->ebar, device_status_ptr(), s)
          : launch_co_grad_f64(n, B, P->d.sqrt_s, P->p, hel, P->d.q, static_cast<const double*>(P->Y), P->kbar,
                               P->ebar, device_status_ptr(), s);
  st = cuda_check(e, "bg_me2_grad: reverse recursion");
  if (st != BG_OK) return st;
  return cuda_check(launch_rambo_grad(n, B, P->d.sqrt_s, u, P->p, hel, P->d.q, P->kbar, P->ebar, a.scale, upstream,
                                      P->accept, grad_u, s),
                    "bg_me2_grad: polarisations and Rambo");
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
