// noalloc.cu -- bg_me2_batch_noalloc: the colour-ordered |M|^2 pipeline
// (Rambo -> cut -> polarisations -> recursion -> colour sum) for callers
// that cannot allocate device memory.
//
// The intermediate buffers (momenta, cut flags, amplitudes) live in one
// fixed-size array in device global memory, defined in this file.  It is
// part of the library's device image, so every GPU that loads libbg.so holds
// it (kNoallocScratchBytes) until the process exits.  Host code cannot use
// the array's name as a device address: at the first call on each device the
// entry point asks the runtime for the array's device address
// (cudaGetSymbolAddress, with that device current) and keeps it in a small
// per-device table.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "bg_internal.h"

namespace bg {
namespace {

constexpr size_t kNoallocScratchBytes = size_t(64) << 20;  // 64 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kMaxDevices];  // zero-initialised: not set up yet

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the scratch array on the current device (set up once,
// together with the device status word's address).
bg_status noalloc_scratch(cudaStream_t s, unsigned char** out) {
  int dev = 0;
  bg_status st = cuda_check(cudaGetDevice(&dev), "bg_me2_batch_noalloc: cudaGetDevice");
  if (st != BG_OK) return st;
  if (dev < 0 || dev >= kMaxDevices) return fail(BG_EUNSUPPORTED, "bg_me2_batch_noalloc: device index >= 64");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    // The first call on a device must not be captured into a graph: the
    // symbol lookup (and the status-word lookup below) are runtime calls.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap != cudaStreamCaptureStatusNone)
      return fail(BG_EINVAL,
                  "bg_me2_batch_noalloc: the first call on a device sets up the scratch address and must not run "
                  "during stream capture; make one call on this device (current) before capturing");
    void* ptr = nullptr;
    st = cuda_check(cudaGetSymbolAddress(&ptr, g_noalloc_scratch),
                    "bg_me2_batch_noalloc: cudaGetSymbolAddress of the scratch array (first call on this device; "
                    "the device must be current and no stream capture active)");
    if (st != BG_OK) return st;
    if (!device_status_ptr())
      return fail(BG_ECUDA, "bg_me2_batch_noalloc: cannot look up the device status word on this device");
    g_noalloc_ptr[dev] = static_cast<unsigned char*>(ptr);
  }
  *out = g_noalloc_ptr[dev];
  return BG_OK;
}

}  // namespace
}  // namespace bg

using namespace bg;

extern "C" bg_status bg_me2_batch_noalloc(const bg_colormat* C, int64_t B, double sqrt_s, double pt_min,
                                          double g_s, const double* q, bg_prec prec, bg_cs_mode cs_mode,
                                          const double* u, const int8_t* hel, double* me2, void* stream) {
  if (!C) return fail(BG_EINVAL, "bg_me2_batch_noalloc: C is NULL");
  const int n = C->n;
  if (n > kMaxNCO) return fail(BG_EUNSUPPORTED, "bg_me2_batch_noalloc: colour-ordered path supports n <= 9");
  if (B < 0) return fail(BG_EINVAL, "bg_me2_batch_noalloc: B < 0");
  if (prec != BG_F32 && prec != BG_F64) return fail(BG_EINVAL, "bg_me2_batch_noalloc: invalid precision");
  if (cs_mode != BG_CS_F64 && cs_mode != BG_CS_F32 && cs_mode != BG_CS_TC_BF16)
    return fail(BG_EINVAL, "bg_me2_batch_noalloc: invalid colour-sum mode");
  if (!(sqrt_s > 0.0)) return fail(BG_EINVAL, "bg_me2_batch_noalloc: sqrt_s must be > 0");
  if (!q) return fail(BG_EINVAL, "bg_me2_batch_noalloc: q is NULL");
  const double qv = std::sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(q[0] > 0.0) || std::fabs(q[0] - qv) > 1e-12 * q[0])
    return fail(BG_EINVAL, "bg_me2_batch_noalloc: q must be light-like with q0 > 0");
  const int H = hel ? 1 : (1 << n);
  if (cs_mode == BG_CS_TC_BF16 && (!C->tc_tiles || H != 1))
    return fail(BG_EUNSUPPORTED, "bg_me2_batch_noalloc: tensor-core mode needs 6 <= n <= 9 and sampled helicities");
  // scratch layout: momenta [4][n][B] double | amplitudes [B][H][k] | cut flags [B]
  const size_t amp_size = (prec == BG_F32) ? 4 : 8;
  const size_t per_event = 4 * (size_t)n * 8 + (size_t)H * C->k * amp_size + 1;
  const int64_t max_events = (int64_t)((kNoallocScratchBytes - 3 * 256) / per_event);
  if (B > max_events) {
    char msg[256];
    std::snprintf(msg, sizeof msg,
                  "bg_me2_batch_noalloc: B = %lld exceeds the fixed %zu MiB scratch: at most %lld events per call "
                  "for n = %d with this precision and helicity mode",
                  (long long)B, kNoallocScratchBytes >> 20, (long long)max_events, n);
    return fail(BG_EINVAL, msg);
  }
  if (B == 0) return BG_OK;
  if (!u || !me2) return fail(BG_EINVAL, "bg_me2_batch_noalloc: NULL u or me2");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* scratch = nullptr;
  bg_status st = noalloc_scratch(s, &scratch);
  if (st != BG_OK) return st;
  double* p = reinterpret_cast<double*>(scratch);
  void* amps = scratch + align256(4 * (size_t)n * 8 * B);
  uint8_t* accept = reinterpret_cast<uint8_t*>(static_cast<unsigned char*>(amps) +
                                               align256((size_t)B * H * C->k * amp_size));
  // Every scratch byte read below is written earlier in this same call, so
  // nothing has to start at zero and leftovers of an earlier call are harmless.
  // The device status word (a fixed library symbol, no allocation) receives
  // invalid helicity labels and a timed-out tensor-core wait, as for the
  // other entry points.
  int* status = device_status_ptr();
  st = cuda_check(launch_rambo(n, B, sqrt_s, u, p, pt_min, accept, s), "bg_me2_batch_noalloc: Rambo");
  if (st != BG_OK) return st;
  st = cuda_check(prec == BG_F32 ? launch_co_f32(n, B, sqrt_s, p, hel, q, static_cast<float*>(amps), status, s)
                                 : launch_co_f64(n, B, sqrt_s, p, hel, q, static_cast<double*>(amps), status, s),
                  "bg_me2_batch_noalloc: recursion");
  if (st != BG_OK) return st;
  ColourSumArgs a;
  a.n = n;
  a.B = B;
  a.H = H;
  a.k = C->k;
  a.amps = amps;
  a.amps_f32 = (prec == BG_F32);
  a.C64 = C->C64;
  a.C32 = C->C32;
  a.scale = std::pow(g_s, 2 * n - 4) * std::pow(sqrt_s, 8 - 2 * n) * (hel ? std::ldexp(1.0, n) : 1.0);
  a.accept = accept;
  a.me2 = me2;
  cudaError_t e = (cs_mode == BG_CS_F64)   ? launch_color_sum_f64(a, s)
                  : (cs_mode == BG_CS_F32) ? launch_color_sum_f32(a, s)
                                           : launch_color_sum_tc(a, C, status, s);
  return cuda_check(e, "bg_me2_batch_noalloc: colour sum");
}
