// color_sum_tc.cu -- the colour sum of Eq. (2.16) on the 5th-generation
// tensor cores (tcgen05, sm_103a):
//   |M|^2_e = scale * sum_m A_{e m} (A C)_{e m},   C symmetric.
//
// Operands.  D = A C is a dense contraction: M = 128 events per CTA (TMEM
// lanes), N = a tile of NT orderings (TMEM columns), K = all orderings.  C is
// stored once per colour matrix as BF16 tiles of C/g (g = gcd of its
// entries; every C/g is exactly representable in BF16 for n <= 8, and as a
// sum of two BF16 planes hi + lo for n = 9, checked at creation), pre-arranged in the canonical no-swizzle K-major core-matrix
// layout so that a plain bulk copy lands a tile ready for the MMA.  The FP32
// amplitudes are split on the fly into three BF16 planes, A = hi + mid + lo
// (24 significant bits), so that D is accurate to FP32 rounding; the MMA
// accumulates in FP32 in tensor memory.
//
// Roles (10 warps, 11 with the staged amplitude path):
//   warp 0      one thread: bulk copies of C tiles (mbarrier complete_tx)
//   warp 1      allocates tensor memory; one thread issues tcgen05.mma and
//               tcgen05.commit
//   warps 2..5  converters: FP32 amplitudes -> 3 BF16 planes in shared memory
//   warps 6..9  epilogue: tcgen05.ld of D rows (one event per thread),
//               contraction with the FP32 amplitudes, FP64 accumulation
//   warp 10     (staged path) one thread: tensor-map bulk copies of the
//               amplitude tile, 128 events x 64 orderings of FP32 per K chunk
//               as two 128 x 32 boxes with 128-byte swizzle, into a ring of
//               2-3 staging buffers ahead of the converters
// The CTAs are persistent (one per SM, each looping over tiles of 128
// events).  Two pipeline stages for the BF16 operands and two accumulator
// buffers in tensor memory, so that the epilogue of one ordering tile
// overlaps the MMAs of the next -- also across the CTA's event tiles.  In the staged path the converters read their rows from
// shared memory (the swizzle makes the 32 rows of a warp hit distinct banks)
// instead of loading them from global memory row by row.  Every mbarrier
// wait is bounded (about 2 s of SM clocks); on expiry the kernel records
// BG_ETIMEOUT in the status word and the CTA drains and exits.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "bg_internal.h"
#include "device_common.cuh"

namespace bg {
namespace {

constexpr int TC_M = 128;         // events per CTA
constexpr int TC_KC = 64;         // K elements per pipeline stage
constexpr int TC_STAGES = 2;
constexpr int TC_THREADS = 320;
constexpr int TC_THREADS_STAGED = 352;
constexpr int TC_AF_BYTES = TC_M * TC_KC * 4;  // one FP32 amplitude stage: two 16 KB boxes
constexpr int TC_AF_MAX = 3;                   // FP32 staging buffers at most
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz
constexpr long long kTestWaitCycles = 2000000LL;  // ~1 ms: the stall test's limit

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                   smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; returns false (and records BG_ETIMEOUT) if the phase does not
// complete within `limit` SM clocks, or if another thread has already given up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* status, volatile int* abort_flag,
                                          long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      *abort_flag = 1;
      flag_status(status, BG_ETIMEOUT);
      return false;
    }
  }
  return true;
}

// After a producer stops (normally or because a wait gave up), it waits, with
// the same bound, for the bulk copies it issued into the last `depth` stages
// (iterations it_end-depth .. it_end-1 of a ring of `depth` stages), so that
// no copy is still writing shared memory when the CTA exits.  Returns at once
// when the consumers have already seen those copies complete.
__device__ __forceinline__ void drain_copies(uint64_t* full, int depth, int it_end) {
  for (int it = it_end - depth; it < it_end; ++it) {
    if (it < 0) continue;
    const long long t0 = clock64();
    while (!mbar_try_wait(&full[it % depth], (uint32_t)(it / depth) & 1))
      if (clock64() - t0 > kWaitCycles) break;
  }
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// 2-D tensor-map bulk copy of the box at (x, y) into shared memory.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension
// byte offset (between core matrices adjacent in K), stride-dimension byte
// offset (between 8-row groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row r, k) inside a K-major core-matrix tile whose
// rows hold TC_KC elements: 8x8 core matrices of 128 contiguous bytes, K-
// adjacent cores 128 B apart (LBO), 8-row groups 1024 B apart (SBO).
__host__ __device__ constexpr uint32_t tile_off(int r, int k) {
  return (uint32_t)(((r >> 3) * (TC_KC / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// 16 amplitudes of one row from column m0 (zeros beyond k or for rows past
// the batch).
template <typename TIn>
__device__ __forceinline__ void tc_load16(const TIn* row, bool live, int m0, int k, float (&x)[16]) {
#pragma unroll
  for (int j = 0; j < 16; ++j) x[j] = 0.0f;
  if (!live || m0 >= k) return;
  // vector loads only from 16-byte aligned addresses (the interface admits
  // amplitude arrays that are merely 4-byte aligned)
  if (sizeof(TIn) == 4 && m0 + 16 <= k && (reinterpret_cast<uintptr_t>(row + m0) & 15) == 0) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float4 f = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(row) + m0 + 4 * v);
      x[4 * v] = f.x, x[4 * v + 1] = f.y, x[4 * v + 2] = f.z, x[4 * v + 3] = f.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (m0 + j < k) x[j] = (float)row[m0 + j];
  }
}

// The TC_KC amplitudes of K chunk kc of one row.
template <typename TIn>
__device__ __forceinline__ void tc_load_chunk(const TIn* row, bool live, int kc, int k, float (&x)[TC_KC]) {
#pragma unroll
  for (int g = 0; g < TC_KC / 16; ++g) {
    float v[16];
    tc_load16<TIn>(row, live, kc * TC_KC + g * 16, k, v);
#pragma unroll
    for (int j = 0; j < 16; ++j) x[g * 16 + j] = v[j];
  }
}

struct TcParams {
  int64_t B;             // capacity
  const int64_t* dB;     // optional device-side event count
  int k;        // orderings
  int nt;       // orderings per N tile (multiple of 16, <= 240)
  int ntiles;   // N tiles
  int kchunks;  // K chunks of TC_KC
  double scale; // includes the gcd of C
  float g;      // gcd of C (Y = g D)
  int af_stages;  // staged path: FP32 staging buffers (2..TC_AF_MAX)
  long long wait_cycles;  // limit of every bounded wait (SM clocks)
  int stall_c;    // test hook: the C-tile producer issues nothing, so the waits run out
};

// Converter step `it` for row r: wait for stage it % 2 to be free, split the
// FP32 amplitudes x into hi / mid / lo BF16 planes in the stage's canonical
// layout, signal full_a.  Returns false if a wait gave up.
__device__ __forceinline__ bool tc_convert_chunk(const float (&x)[TC_KC], int it, int r, unsigned char* stage_base,
                                                 uint32_t stage_bytes, uint32_t a_plane_bytes, uint64_t* empty,
                                                 uint64_t* full_a, int* status, volatile int* abort_flag,
                                                 long long limit) {
  const int s = it & 1;
  const uint32_t use = (uint32_t)(it >> 1);
  if (it >= TC_STAGES && !mbar_wait(&empty[s], (use - 1) & 1, status, abort_flag, limit)) return false;
  unsigned char* st = stage_base + s * stage_bytes;
#pragma unroll
  for (int g = 0; g < TC_KC / 8; ++g) {
    uint32_t hi[4], mid[4], lo[4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      // pairs of elements converted by one packed instruction each (the same
      // round-to-nearest-even of each element as the scalar conversion)
      const float x0 = x[g * 8 + j], x1 = x[g * 8 + j + 1];
      const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
      const float2 hf = __bfloat1622float2(h);
      const float r0 = x0 - hf.x, r1 = x1 - hf.y;
      const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
      const float2 mf = __bfloat1622float2(m);
      const __nv_bfloat162 l = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
      hi[j / 2] = *reinterpret_cast<const uint32_t*>(&h);
      mid[j / 2] = *reinterpret_cast<const uint32_t*>(&m);
      lo[j / 2] = *reinterpret_cast<const uint32_t*>(&l);
    }
    const uint32_t off = tile_off(r, g * 8);
    *reinterpret_cast<uint4*>(st + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4*>(st + a_plane_bytes + off) = make_uint4(mid[0], mid[1], mid[2], mid[3]);
    *reinterpret_cast<uint4*>(st + 2 * a_plane_bytes + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  }
  fence_proxy_async();
  mbar_arrive(&full_a[s]);
  return true;
}

template <typename TIn, int CPL, bool STAGED>
__global__ void __launch_bounds__(STAGED ? TC_THREADS_STAGED : TC_THREADS, 1)
    color_sum_tc_kernel(TcParams P, const TIn* __restrict__ A, const __nv_bfloat16* __restrict__ Ct,
                        const uint8_t* __restrict__ accept, double* __restrict__ me2, int* __restrict__ status,
                        TIn* __restrict__ Y, const __grid_constant__ CUtensorMap amap) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned carve-up
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t a_plane_bytes = TC_M * TC_KC * 2;            // 16 KB
  const uint32_t c_tile_bytes = (uint32_t)P.nt * TC_KC * 2 * CPL;   // CPL planes of nt*128 B
  const uint32_t c_plane_bytes = (uint32_t)P.nt * TC_KC * 2;
  const uint32_t stage_bytes = 3 * a_plane_bytes + ((c_tile_bytes + 1023) & ~1023u);
  unsigned char* stage_base = smem;
  // staged path: FP32 amplitude staging ring (1024-byte aligned for the swizzle)
  unsigned char* af_base = smem + TC_STAGES * stage_bytes;
  const int af_stages = STAGED ? P.af_stages : 0;
  uint64_t* bars = reinterpret_cast<uint64_t*>(af_base + (size_t)af_stages * TC_AF_BYTES);
  uint64_t* full_c = bars;                  // [2]
  uint64_t* full_a = bars + 2;              // [2]
  uint64_t* empty = bars + 4;               // [2]
  uint64_t* dfull = bars + 6;               // [2]
  uint64_t* dempty = bars + 8;              // [2]
  uint64_t* full_af = bars + 10;            // [TC_AF_MAX]
  uint64_t* empty_af = bars + 10 + TC_AF_MAX;  // [TC_AF_MAX]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 10 + 2 * TC_AF_MAX);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 11 + 2 * TC_AF_MAX);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // Persistent CTAs: this CTA takes the event tiles blockIdx.x, + gridDim.x,
  // ...; the pipeline iterations (it) and the accumulator uses (g) count on
  // across its tiles, so that the epilogue of one tile overlaps the MMAs of
  // the next.
  int64_t nev = P.B;
  if (P.dB) nev = *P.dB < P.B ? *P.dB : P.B;
  const int64_t ntev = (nev + TC_M - 1) / TC_M;
  const int my_tiles = (int64_t)blockIdx.x < ntev ? (int)((ntev - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  if (my_tiles == 0) return;  // whole CTA without events in this launch
  P.B = nev;
  const int total = P.ntiles * P.kchunks;  // pipeline iterations per event tile
  const int all_it = my_tiles * total;
  const int all_g = my_tiles * P.ntiles;
  const uint32_t tmem_cols = (2 * P.nt <= 32) ? 32 : (2 * P.nt <= 64) ? 64 : (2 * P.nt <= 128) ? 128
                           : (2 * P.nt <= 256) ? 256 : 512;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full_c[s], 1);
      mbar_init(&full_a[s], 128);
      mbar_init(&empty[s], 1);
      mbar_init(&dfull[s], 1);
      mbar_init(&dempty[s], 128);
    }
    for (int s = 0; s < af_stages; ++s) {
      mbar_init(&full_af[s], 1);
      mbar_init(&empty_af[s], 128);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------- C tile producer ----------------
    if (lane == 0 && !P.stall_c) {
      int it = 0;
      for (; it < all_it; ++it) {
        const int s = it & 1;
        const uint32_t use = (uint32_t)(it >> 1);
        if (it >= TC_STAGES && !mbar_wait(&empty[s], (use - 1) & 1, status, abort_flag, P.wait_cycles)) break;
        const int local = it % total;
        const int ntile = local / P.kchunks, kc = local % P.kchunks;
        unsigned char* dst = stage_base + s * stage_bytes + 3 * a_plane_bytes;
        const unsigned char* src = reinterpret_cast<const unsigned char*>(Ct) +
                                   ((size_t)ntile * P.kchunks + kc) * (size_t)c_tile_bytes;
        mbar_arrive_expect_tx(&full_c[s], c_tile_bytes);
        bulk_g2s(dst, src, c_tile_bytes, &full_c[s]);
      }
      drain_copies(full_c, TC_STAGES, it);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(TC_M, P.nt);
      bool ok = true;
      for (int g = 0; g < all_g && ok; ++g) {
        const int b = g & 1;
        const uint32_t buse = (uint32_t)(g >> 1);
        if (g >= 2 && !mbar_wait(&dempty[b], (buse - 1) & 1, status, abort_flag, P.wait_cycles)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(b * P.nt);
        for (int kc = 0; kc < P.kchunks; ++kc) {
          const int it = g * P.kchunks + kc;
          const int s = it & 1;
          const uint32_t use = (uint32_t)(it >> 1);
          if (!mbar_wait(&full_c[s], use & 1, status, abort_flag, P.wait_cycles) ||
              !mbar_wait(&full_a[s], use & 1, status, abort_flag, P.wait_cycles)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(stage_base + s * stage_bytes);
          const uint32_t c0 = a0 + 3 * a_plane_bytes;
#pragma unroll
          for (int cp = 0; cp < CPL; ++cp) {
#pragma unroll
            for (int plane = 0; plane < 3; ++plane) {
#pragma unroll
              for (int ks = 0; ks < TC_KC / 16; ++ks) {
                const uint64_t ad = smem_desc(a0 + plane * a_plane_bytes + ks * 256, 128, 1024);
                const uint64_t bd = smem_desc(c0 + cp * c_plane_bytes + ks * 256, 128, 1024);
                mma_bf16(d_tmem, ad, bd, idesc, (kc > 0 || cp > 0 || plane > 0 || ks > 0) ? 1u : 0u);
              }
            }
          }
          mma_commit(&empty[s]);  // stage free once these MMAs have read it
        }
        if (ok) mma_commit(&dfull[b]);  // accumulator b complete
      }
    }
  } else if (warp < 6 && STAGED) {
    // ---------------- converters, staged path ----------------
    // Row r of the chunk sits in the two swizzled boxes of the staging
    // buffer: element j of box b at byte r*128 + ((j/4) ^ (r%8))*16 + (j%4)*4.
    const int r = threadIdx.x - 64;
    for (int it = 0; it < all_it; ++it) {
      const int sa = it % af_stages;
      const uint32_t ua = (uint32_t)(it / af_stages);
      if (!mbar_wait(&full_af[sa], ua & 1, status, abort_flag, P.wait_cycles)) break;
      const unsigned char* box = af_base + (size_t)sa * TC_AF_BYTES + r * 128;
      float x[TC_KC];
#pragma unroll
      for (int b = 0; b < 2; ++b) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4 v = *reinterpret_cast<const float4*>(box + b * (TC_AF_BYTES / 2) + ((c ^ (r & 7)) << 4));
          x[b * 32 + 4 * c] = v.x, x[b * 32 + 4 * c + 1] = v.y, x[b * 32 + 4 * c + 2] = v.z,
                         x[b * 32 + 4 * c + 3] = v.w;
        }
      }
      const bool ok =
          tc_convert_chunk(x, it, r, stage_base, stage_bytes, a_plane_bytes, empty, full_a, status, abort_flag,
                           P.wait_cycles);
      mbar_arrive(&empty_af[sa]);  // the staging buffer's rows are in registers and converted
      if (!ok) break;
    }
  } else if (warp == 10) {
    // ---------------- staged path: amplitude tile producer ----------------
    if (STAGED && lane == 0) {
      int it = 0;
      for (; it < all_it; ++it) {
        const int sa = it % af_stages;
        const uint32_t ua = (uint32_t)(it / af_stages);
        if (it >= af_stages && !mbar_wait(&empty_af[sa], (ua - 1) & 1, status, abort_flag, P.wait_cycles)) break;
        const int64_t e0 = ((int64_t)blockIdx.x + (int64_t)(it / total) * gridDim.x) * TC_M;
        const int kc = (it % total) % P.kchunks;
        unsigned char* dst = af_base + (size_t)sa * TC_AF_BYTES;
        mbar_arrive_expect_tx(&full_af[sa], TC_AF_BYTES);
        tma_load_2d(dst, &amap, kc * TC_KC, (int)e0, &full_af[sa]);
        tma_load_2d(dst + TC_AF_BYTES / 2, &amap, kc * TC_KC + 32, (int)e0, &full_af[sa]);
      }
      drain_copies(full_af, af_stages, it);
    }
  } else if (warp < 6) {
    // ---------------- converters: FP32 -> hi/mid/lo BF16 planes ----------------
    // The amplitudes of the next K chunk are loaded into registers before the
    // current chunk is converted (and before waiting for a free stage), so
    // the loads' latency overlaps the conversion and the MMAs.
    const int r = threadIdx.x - 64;  // row (event) of the tile, 0..127
    bool ok = true;
    for (int t = 0; t < my_tiles && ok; ++t) {
      const int64_t e = ((int64_t)blockIdx.x + (int64_t)t * gridDim.x) * TC_M + r;
      const TIn* row = A + e * (int64_t)P.k;
      const int ib = t * total;
      float xa[TC_KC], xb[TC_KC];
      tc_load_chunk<TIn>(row, e < P.B, 0, P.k, xa);
      for (int it = 0; it < total; it += 2) {
        if (it + 1 < total) tc_load_chunk<TIn>(row, e < P.B, (it + 1) % P.kchunks, P.k, xb);
        if (!tc_convert_chunk(xa, ib + it, r, stage_base, stage_bytes, a_plane_bytes, empty, full_a, status,
                              abort_flag, P.wait_cycles)) {
          ok = false;
          break;
        }
        if (it + 1 >= total) break;
        if (it + 2 < total) tc_load_chunk<TIn>(row, e < P.B, (it + 2) % P.kchunks, P.k, xa);
        if (!tc_convert_chunk(xb, ib + it + 1, r, stage_base, stage_bytes, a_plane_bytes, empty, full_a, status,
                              abort_flag, P.wait_cycles)) {
          ok = false;
          break;
        }
      }
    }
  } else {
    // ---------------- epilogue: one event per thread ----------------
    const int q = warp & 3;  // TMEM lane quarter accessible to this warp
    const int r = q * 32 + lane;
    bool ok = true;
    for (int t = 0; t < my_tiles && ok; ++t) {
      const int64_t e = ((int64_t)blockIdx.x + (int64_t)t * gridDim.x) * TC_M + r;
      const TIn* row = A + e * (int64_t)P.k;
      double acc = 0.0;
      for (int ntile = 0; ntile < P.ntiles; ++ntile) {
        const int g = t * P.ntiles + ntile;
        const int b = g & 1;
        const uint32_t buse = (uint32_t)(g >> 1);
        // warp-uniform decision: tcgen05.ld below is .sync.aligned
        const bool ready = mbar_wait(&dfull[b], buse & 1, status, abort_flag, P.wait_cycles);
        if (!__all_sync(0xffffffffu, ready)) {
          ok = false;
          break;
        }
        tc_fence_after();
        float part = 0.0f;
        float an[16];
        tc_load16<TIn>(row, e < P.B, ntile * P.nt, P.k, an);
        for (int c0 = 0; c0 < P.nt; c0 += 16) {
          float ac[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) ac[j] = an[j];
          if (c0 + 16 < P.nt) tc_load16<TIn>(row, e < P.B, ntile * P.nt + c0 + 16, P.k, an);
          float d[16];
          tmem_ld16(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * P.nt + c0), d);
          const int m0 = ntile * P.nt + c0;
#pragma unroll
          for (int j = 0; j < 16; ++j) part = fmaf(ac[j], d[j], part);  // ac is 0 beyond k and B
          if (Y && e < P.B) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (m0 + j < P.k) Y[e * (int64_t)P.k + m0 + j] = (TIn)(P.g * d[j]);
          }
        }
        acc += (double)part;
        tc_fence_before();
        mbar_arrive(&dempty[b]);
      }
      if (e < P.B) {
        const bool keep = ok && ((accept == nullptr) || (accept[e] != 0));
        me2[e] = (keep && !*abort_flag) ? P.scale * acc : 0.0;
      }
    }
    if (!ok) {
      // the events of this CTA's remaining tiles get 0 (a wait gave up)
      for (int t = 0; t < my_tiles; ++t) {
        const int64_t e = ((int64_t)blockIdx.x + (int64_t)t * gridDim.x) * TC_M + r;
        if (e < P.B) me2[e] = 0.0;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(tmem_cols)
                 : "memory");
  }
}

}  // namespace

// Host: BF16 tiles of C / g in the layout of tile_off.  C/g is split into
// cpl = 1 or 2 exactly representable BF16 planes (hi + lo): for n <= 8 one
// plane suffices; at n = 9, 22 entries per row need 9-10 significant bits and
// a second plane carries the low bits.  Each tile stores its planes back to
// back.  Returns false if two planes are not enough or n is outside 6..9.
static bool bf16_exact(float v, uint16_t& bits) {
  uint32_t u;
  std::memcpy(&u, &v, 4);
  bits = (uint16_t)(u >> 16);
  return (u & 0xFFFFu) == 0;
}

bool build_tc_tiles(int n, const std::vector<double>& dense, int k, std::vector<uint16_t>& tiles, double& g,
                    int& nt, int& ntiles, int& kchunks, int& cpl) {
  if (n < 6 || n > 9) return false;
  long long gg = 0;
  for (double v : dense) {
    long long x = (long long)(v < 0 ? -v : v);
    if ((double)x != (v < 0 ? -v : v)) return false;
    long long a = gg, b = x;
    while (b) { long long t = a % b; a = b; b = t; }
    gg = a;
  }
  if (gg == 0) return false;
  g = (double)gg;
  // planes: hi = C/g rounded to BF16, lo = remainder (must be exact)
  cpl = 1;
  for (double v : dense) {
    uint16_t bits;
    if (!bf16_exact((float)(v / g), bits)) { cpl = 2; break; }
  }
  nt = k < 240 ? ((k + 15) / 16) * 16 : 240;
  ntiles = (k + nt - 1) / nt;
  kchunks = (k + TC_KC - 1) / TC_KC;
  const size_t plane_elems = (size_t)nt * TC_KC;
  tiles.assign((size_t)ntiles * kchunks * plane_elems * cpl, 0);
  for (int t = 0; t < ntiles; ++t)
    for (int kc = 0; kc < kchunks; ++kc) {
      uint16_t* base = &tiles[((size_t)t * kchunks + kc) * plane_elems * cpl];
      for (int rr = 0; rr < nt; ++rr)
        for (int kk = 0; kk < TC_KC; ++kk) {
          const int m = t * nt + rr, c = kc * TC_KC + kk;
          const double v = (m < k && c < k) ? dense[(size_t)m * k + c] / g : 0.0;
          const float hi = __bfloat162float(__float2bfloat16_rn((float)v));
          uint16_t hb, lb;
          if (!bf16_exact(hi, hb)) return false;
          const double rem = v - (double)hi;
          if (cpl == 1) {
            if (rem != 0.0) return false;
          } else {
            if (!bf16_exact((float)rem, lb) || (double)(float)rem != rem) return false;
            base[plane_elems + tile_off(rr, kk) / 2] = lb;
          }
          base[tile_off(rr, kk) / 2] = hb;
        }
    }
  return true;
}

size_t tc_smem_bytes(int nt, int cpl, int af_stages) {
  const size_t a_plane = TC_M * TC_KC * 2;
  const size_t c_tile = ((size_t)nt * TC_KC * 2 * cpl + 1023) & ~size_t(1023);
  return 1024 + TC_STAGES * (3 * a_plane + c_tile) + (size_t)af_stages * TC_AF_BYTES + 256;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link against the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
    else
      cudaGetLastError();
  });
  return fn;
}

// Tensor map of the FP32 amplitudes A [B][k] (row stride k): boxes of 32
// orderings x 128 events with 128-byte swizzle; out-of-range boxes are
// zero-filled.  False if the layout does not allow it (base or row stride
// not a multiple of 16 bytes, sizes out of range).
bool amp_tensor_map(const float* A, int64_t B, int k, CUtensorMap* map) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn || (reinterpret_cast<uintptr_t>(A) & 15) || ((size_t)k * 4) % 16 || B < 1 || B > (int64_t(1) << 31))
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)B};
  const cuuint64_t strides[1] = {(cuuint64_t)k * 4};
  const cuuint32_t box[2] = {32, (cuuint32_t)TC_M};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

constexpr size_t kSmemOptIn = 232448;  // shared memory per block (opt-in)

cudaError_t launch_color_sum_tc(const ColourSumArgs& a, const bg_colormat* C, int* status, cudaStream_t s) {
  TcParams P;
  P.B = a.B;
  P.dB = a.dB;
  P.k = a.k;
  P.nt = C->tc_nt;
  P.ntiles = C->tc_ntiles;
  P.kchunks = C->tc_kchunks;
  P.scale = a.scale * C->tc_g;
  P.g = (float)C->tc_g;
  P.af_stages = 0;
  // BG_TC_TEST_STALL (tests only): the C tiles are never copied, every wait
  // runs out after ~1 ms, the kernel records BG_ETIMEOUT and writes 0.
  const char* stall = std::getenv("BG_TC_TEST_STALL");
  P.stall_c = (stall && stall[0] == '1') ? 1 : 0;
  P.wait_cycles = P.stall_c ? kTestWaitCycles : kWaitCycles;
  // persistent CTAs: one per SM (a CTA fills the SM's shared memory), each
  // looping over event tiles of 128
  const int64_t tiles = (a.B + TC_M - 1) / TC_M;
  if (tiles == 0) return cudaSuccess;
  const int sms = device_sms();
  const unsigned blocks = (unsigned)(sms > 0 && tiles > sms ? sms : tiles);
  // The staged amplitude path: FP32 amplitudes, one BF16 plane of C, a
  // tensor map for A, and room for at least two staging buffers.
  CUtensorMap amap;
  std::memset(&amap, 0, sizeof amap);
  if (a.amps_f32 && C->tc_cpl == 1) {
    int st = TC_AF_MAX;
    while (st >= 2 && tc_smem_bytes(P.nt, 1, st) > kSmemOptIn) --st;
    if (st >= 2 && amp_tensor_map(static_cast<const float*>(a.amps), a.B, a.k, &amap)) P.af_stages = st;
  }
  const size_t smem = tc_smem_bytes(P.nt, C->tc_cpl, P.af_stages);
#define BG_TC_LAUNCH(TIN, CPL, STG)                                                                            \
  {                                                                                                            \
    auto kern = color_sum_tc_kernel<TIN, CPL, STG>;                                                            \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);       \
    if (e != cudaSuccess) return e;                                                                            \
    kern<<<blocks, STG ? TC_THREADS_STAGED : TC_THREADS, smem, s>>>(                                           \
        P, static_cast<const TIN*>(a.amps), C->tc_tiles, a.accept, a.me2, status, static_cast<TIN*>(a.Y), amap); \
  }
  if (a.amps_f32) {
    if (C->tc_cpl == 1) {
      if (P.af_stages) BG_TC_LAUNCH(float, 1, true) else BG_TC_LAUNCH(float, 1, false)
    } else {
      BG_TC_LAUNCH(float, 2, false)
    }
  } else {
    if (C->tc_cpl == 1) BG_TC_LAUNCH(double, 1, false) else BG_TC_LAUNCH(double, 2, false)
  }
#undef BG_TC_LAUNCH
  return cudaGetLastError();
}

}  // namespace bg
