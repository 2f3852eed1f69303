// color_sum.cu -- the colour sum of Eq. (2.16) on CUDA cores:
//   |M|^2_e = scale * sum_h sum_{a,b} C_ab A_{e h a} A_{e h b}
// evaluated as a tiled product Y = C A_e (C symmetric, so column b of C is
// row b) followed by the per-event contraction sum_a A_{e h a} Y_{a e},
// all inside one kernel.  A block owns a tile of 64 events and walks all
// row tiles of C, so each event's quadratic form is finished in registers
// and written once (no atomics, no scratch memory, deterministic order).
// TC is the arithmetic type of C A; the per-event sum is accumulated in FP64.
// Colour matrices with k <= 24 take a one-thread-per-event kernel instead.
#include "bg_internal.h"
#include "device_common.cuh"

namespace bg {
namespace {

constexpr int TA = 64;   // rows of C per tile
constexpr int TE = 64;   // events per block
constexpr int KT = 16;   // reduction step
constexpr int NT = 256;  // threads: 16 x 16, each 4 rows x 4 events

template <typename TIn, typename TC>
__global__ void __launch_bounds__(NT) color_sum_kernel(int64_t Bcap, const int64_t* __restrict__ dB, int H, int k,
                                                       const TIn* __restrict__ A, const TC* __restrict__ C,
                                                       double scale, const uint8_t* __restrict__ accept,
                                                       double* __restrict__ me2, TIn* __restrict__ Y) {
  const int64_t B = dB ? (*dB < Bcap ? *dB : Bcap) : Bcap;
  if ((int64_t)blockIdx.x * 64 >= B) return;
  __shared__ __align__(16) TC Cs[KT][TA];
  __shared__ __align__(16) TC As[KT][TE];
  __shared__ double red[16][TE];
  const int tid = threadIdx.x;
  const int tx = tid & 15;   // event group (4 events)
  const int ty = tid >> 4;   // row group (4 rows)
  const int64_t e0 = (int64_t)blockIdx.x * TE;
  const int64_t strideE = (int64_t)H * k;
  double part[4] = {0.0, 0.0, 0.0, 0.0};

  for (int h = 0; h < H; ++h) {
    for (int a0 = 0; a0 < k; a0 += TA) {
      TC acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = TC(0);
      for (int b0 = 0; b0 < k; b0 += KT) {
        // C tile: Cs[kk][r] = C[b0+kk][a0+r]   (1024 elements, 4 per thread)
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const int idx = tid + l * NT;
          const int kk = idx / TA, r = idx % TA;
          const int b = b0 + kk, a = a0 + r;
          Cs[kk][r] = (b < k && a < k) ? C[(int64_t)b * k + a] : TC(0);
        }
        // A tile: As[kk][c] = A[e0+c][h][b0+kk]
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const int idx = tid + l * NT;
          const int c = idx / KT, kk = idx % KT;
          const int b = b0 + kk;
          const int64_t e = e0 + c;
          As[kk][c] = (b < k && e < B) ? TC(A[e * strideE + (int64_t)h * k + b]) : TC(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) {
          TC cv[4], av[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) cv[i] = Cs[kk][ty * 4 + i];
#pragma unroll
          for (int j = 0; j < 4; ++j) av[j] = As[kk][tx * 4 + j];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(cv[i], av[j], acc[i][j]);
        }
        __syncthreads();
      }
      // contract with A at the tile's rows: part_e += sum_a A_{e a} Y_{a e}
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t e = e0 + tx * 4 + j;
        if (e >= B) continue;
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int a = a0 + ty * 4 + i;
          if (a < k) {
            s += (double)A[e * strideE + (int64_t)h * k + a] * (double)acc[i][j];
            if (Y) Y[e * strideE + (int64_t)h * k + a] = (TIn)acc[i][j];
          }
        }
        part[j] += s;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) red[ty][tx * 4 + j] = part[j];
  __syncthreads();
  if (tid < TE) {
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < 16; ++r) s += red[r][tid];
    const int64_t e = e0 + tid;
    if (e < B) {
      const bool ok = (accept == nullptr) || (accept[e] != 0);
      me2[e] = ok ? scale * s : 0.0;
    }
  }
}

// Small colour matrices (k = 2, 6, 24: n = 4, 5, 6): one thread per event,
// C in shared memory, the event's k amplitudes in registers.  The same
// arithmetic per element as the tiled kernel: (C A)_a accumulated over b in
// increasing order in TC, then sum_a A_a (C A)_a in FP64 (over a in
// increasing order).  Consecutive threads read consecutive amplitude rows,
// so the loads are coalesced.
template <typename TIn, typename TC, int K>
__global__ void __launch_bounds__(128) color_sum_small_kernel(int64_t Bcap, const int64_t* __restrict__ dB, int H,
                                                              const TIn* __restrict__ A, const TC* __restrict__ C,
                                                              double scale, const uint8_t* __restrict__ accept,
                                                              double* __restrict__ me2, TIn* __restrict__ Y) {
  __shared__ TC Cs[K * K];
  for (int i = threadIdx.x; i < K * K; i += blockDim.x) Cs[i] = C[i];
  __syncthreads();
  const int64_t B = dB ? (*dB < Bcap ? *dB : Bcap) : Bcap;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B) return;
  double s = 0.0;
  for (int h = 0; h < H; ++h) {
    const TIn* a = A + (e * H + h) * (int64_t)K;
    TC x[K];
#pragma unroll
    for (int b = 0; b < K; ++b) x[b] = TC(a[b]);
#pragma unroll 2
    for (int i = 0; i < K; ++i) {
      TC acc = TC(0);
#pragma unroll
      for (int b = 0; b < K; ++b) acc = fma(Cs[b * K + i], x[b], acc);
      s += (double)a[i] * (double)acc;
      if (Y) Y[(e * H + h) * (int64_t)K + i] = (TIn)acc;
    }
  }
  const bool ok = (accept == nullptr) || (accept[e] != 0);
  me2[e] = ok ? scale * s : 0.0;
}

template <typename TIn, typename TC>
cudaError_t launch_cs(const ColourSumArgs& a, const TC* C, cudaStream_t s) {
  if (a.k == 2 || a.k == 6 || a.k == 24) {
    const int64_t blocks = (a.B + 127) / 128;
    const TIn* A = static_cast<const TIn*>(a.amps);
    TIn* Y = static_cast<TIn*>(a.Y);
    if (a.k == 2)
      color_sum_small_kernel<TIn, TC, 2><<<(unsigned)blocks, 128, 0, s>>>(a.B, a.dB, a.H, A, C, a.scale, a.accept,
                                                                         a.me2, Y);
    else if (a.k == 6)
      color_sum_small_kernel<TIn, TC, 6><<<(unsigned)blocks, 128, 0, s>>>(a.B, a.dB, a.H, A, C, a.scale, a.accept,
                                                                         a.me2, Y);
    else
      color_sum_small_kernel<TIn, TC, 24><<<(unsigned)blocks, 128, 0, s>>>(a.B, a.dB, a.H, A, C, a.scale,
                                                                          a.accept, a.me2, Y);
    return cudaGetLastError();
  }
  const int64_t blocks = (a.B + TE - 1) / TE;
  color_sum_kernel<TIn, TC><<<(unsigned)blocks, NT, 0, s>>>(a.B, a.dB, a.H, a.k, static_cast<const TIn*>(a.amps), C,
                                                           a.scale, a.accept, a.me2, static_cast<TIn*>(a.Y));
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_color_sum_f64(const ColourSumArgs& a, cudaStream_t s) {
  return a.amps_f32 ? launch_cs<float, double>(a, a.C64, s) : launch_cs<double, double>(a, a.C64, s);
}

cudaError_t launch_color_sum_f32(const ColourSumArgs& a, cudaStream_t s) {
  return a.amps_f32 ? launch_cs<float, float>(a, a.C32, s) : launch_cs<double, float>(a, a.C32, s);
}

}  // namespace bg
