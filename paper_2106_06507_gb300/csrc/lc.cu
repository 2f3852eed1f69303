// lc.cu -- leading-colour |M|^2 (Sec. 4, the prefactor formula of the
// leading-colour algorithms):
//   |M|^2_LC = g^(2n-4) N^(n-2) (N^2 - 1) sum over the (n-1)! orders
//              (1, s_2, ..., s_n) of |A(1, s_2, ..., s_n)|^2,   N = 3.
// The colour-ordered kernels evaluate the (n-2)! orders (1, s, n) with gluon
// n last.  An order with gluon l last is an order of that form for the
// momenta with gluons l and n exchanged, so the (n-1)! orders come from n-1
// runs of the same recursion on relabelled inputs; each run's amplitudes are
// squared and added to a per-event FP64 sum in a fixed order (run by run,
// then ordering by ordering).  No colour matrix is involved.
#include <cmath>

#include "bg_internal.h"

namespace bg {
namespace {

// p2, hel2: the inputs with gluons l and n-1 (0-based) exchanged.  The
// recursion takes positions 0 and 1 as the incoming gluons (k = -p there), so
// a momentum that moves between an incoming and an outgoing position changes
// sign: every position then yields the all-outgoing momentum of the gluon
// it now holds.
__global__ void lc_relabel_kernel(int n, int l, int64_t B, const double* __restrict__ p,
                                  const int8_t* __restrict__ hel, double* __restrict__ p2,
                                  int8_t* __restrict__ hel2) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B) return;
  for (int g = 0; g < n; ++g) {
    const int src = g == l ? n - 1 : (g == n - 1 ? l : g);
    const double sg = ((g < 2) != (src < 2)) ? -1.0 : 1.0;
#pragma unroll
    for (int m = 0; m < 4; ++m) p2[((int64_t)m * n + g) * B + e] = sg * p[((int64_t)m * n + src) * B + e];
    if (hel) hel2[(int64_t)g * B + e] = hel[(int64_t)src * B + e];
  }
}

// acc[e] (+)= sum of the squares of the K amplitudes of event e: one warp per
// event, lane-strided partial sums and a fixed butterfly, so the result does
// not depend on scheduling.
template <typename T>
__global__ void lc_sumsq_kernel(int64_t B, int K, const T* __restrict__ amps, double* __restrict__ acc, int first) {
  const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (e >= B) return;
  const T* a = amps + e * (int64_t)K;
  double s = 0.0;
  for (int r = lane; r < K; r += 32) {
    const double v = (double)a[r];
    s = fma(v, v, s);
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  if (lane == 0) acc[e] = first ? s : acc[e] + s;
}

__global__ void lc_final_kernel(int64_t B, const double* __restrict__ acc, const uint8_t* __restrict__ accept,
                                double scale, double* __restrict__ me2) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B) return;
  me2[e] = (accept != nullptr && accept[e] == 0) ? 0.0 : scale * acc[e];
}

struct LcLayout {
  size_t off_p, off_hel, off_amps, off_acc, bytes;
};

LcLayout lc_layout(int n, int64_t B, bool sampled, bool f32) {
  auto a256 = [](size_t x) { return (x + 255) & ~size_t(255); };
  const int64_t H = sampled ? 1 : (int64_t(1) << n);
  LcLayout L;
  L.off_p = 0;
  L.off_hel = a256(L.off_p + sizeof(double) * 4 * (size_t)n * (size_t)B);
  L.off_amps = a256(L.off_hel + (size_t)n * (size_t)B);
  L.off_acc = a256(L.off_amps + (f32 ? 4 : 8) * (size_t)B * (size_t)H * (size_t)factorial(n - 2));
  L.bytes = a256(L.off_acc + sizeof(double) * (size_t)B);
  return L;
}

}  // namespace
}  // namespace bg

using namespace bg;

extern "C" {

bg_status bg_lc_workspace_bytes(int n, int64_t B, int hel_sampled, bg_prec prec, int64_t* bytes) {
  if (!bytes) return fail(BG_EINVAL, "bg_lc_workspace_bytes: bytes is NULL");
  if (n < 4 || n > kMaxNCO) return fail(BG_EINVAL, "bg_lc_workspace_bytes: n must be in 4..9");
  if (B < 0) return fail(BG_EINVAL, "bg_lc_workspace_bytes: B < 0");
  if (prec != BG_F32 && prec != BG_F64) return fail(BG_EINVAL, "bg_lc_workspace_bytes: invalid precision");
  *bytes = (int64_t)lc_layout(n, B, hel_sampled != 0, prec == BG_F32).bytes;
  return BG_OK;
}

bg_status bg_currents_lc(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                         bg_prec prec, double g_s, const uint8_t* accept, double* me2, void* workspace,
                         int64_t workspace_bytes, void* stream) {
  if (n < 4 || n > kMaxNCO) return fail(BG_EINVAL, "bg_currents_lc: n must be in 4..9");
  if (B < 0) return fail(BG_EINVAL, "bg_currents_lc: B < 0");
  if (!(sqrt_s > 0.0)) return fail(BG_EINVAL, "bg_currents_lc: sqrt_s must be > 0");
  if (prec != BG_F32 && prec != BG_F64) return fail(BG_EINVAL, "bg_currents_lc: invalid precision");
  if (!q) return fail(BG_EINVAL, "bg_currents_lc: q is NULL");
  const double qv = std::sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(q[0] > 0.0) || std::fabs(q[0] - qv) > 1e-12 * q[0])
    return fail(BG_EINVAL, "bg_currents_lc: q must be light-like with q0 > 0");
  if (B == 0) return BG_OK;
  if (!p || !me2 || !workspace) return fail(BG_EINVAL, "bg_currents_lc: NULL argument");
  const bool f32 = prec == BG_F32;
  const LcLayout L = lc_layout(n, B, hel != nullptr, f32);
  if (workspace_bytes < (int64_t)L.bytes)
    return fail(BG_EINVAL, "bg_currents_lc: workspace smaller than bg_lc_workspace_bytes");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) || (reinterpret_cast<uintptr_t>(p) & 7) ||
      (reinterpret_cast<uintptr_t>(me2) & 7))
    return fail(BG_EINVAL, "bg_currents_lc: misaligned pointer (workspace needs 256-byte alignment)");
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  double* p2 = reinterpret_cast<double*>(ws + L.off_p);
  int8_t* hel2 = hel ? reinterpret_cast<int8_t*>(ws + L.off_hel) : nullptr;
  void* amps = ws + L.off_amps;
  double* acc = reinterpret_cast<double*>(ws + L.off_acc);
  cudaStream_t s = (cudaStream_t)stream;
  int* status = device_status_ptr();
  const int K = (int)((hel ? 1 : (1 << n)) * factorial(n - 2));
  const unsigned eb = (unsigned)((B + 255) / 256);
  const unsigned wb = (unsigned)((B * 32 + 255) / 256);
  for (int l = n - 1; l >= 1; --l) {
    const double* pl = p;
    const int8_t* hl = hel;
    if (l != n - 1) {
      lc_relabel_kernel<<<eb, 256, 0, s>>>(n, l, B, p, hel, p2, hel2);
      bg_status st = cuda_check(cudaGetLastError(), "bg_currents_lc: relabel");
      if (st != BG_OK) return st;
      pl = p2;
      hl = hel2;
    }
    cudaError_t e = f32 ? launch_co_f32(n, B, sqrt_s, pl, hl, q, static_cast<float*>(amps), status, s)
                        : launch_co_f64(n, B, sqrt_s, pl, hl, q, static_cast<double*>(amps), status, s);
    bg_status st = cuda_check(e, "bg_currents_lc: recursion");
    if (st != BG_OK) return st;
    if (f32)
      lc_sumsq_kernel<float><<<wb, 256, 0, s>>>(B, K, static_cast<const float*>(amps), acc, l == n - 1);
    else
      lc_sumsq_kernel<double><<<wb, 256, 0, s>>>(B, K, static_cast<const double*>(amps), acc, l == n - 1);
    st = cuda_check(cudaGetLastError(), "bg_currents_lc: sum of squares");
    if (st != BG_OK) return st;
  }
  const double scale = std::pow(g_s, 2 * n - 4) * std::pow(3.0, n - 2) * 8.0 * (hel ? std::ldexp(1.0, n) : 1.0) *
                       std::pow(sqrt_s, 8 - 2 * n);
  lc_final_kernel<<<eb, 256, 0, s>>>(B, acc, accept, scale, me2);
  return cuda_check(cudaGetLastError(), "bg_currents_lc: final");
}

}  // extern "C"
