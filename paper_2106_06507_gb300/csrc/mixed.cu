// mixed.cu -- mixed-multiplicity batches (each event has its own n in
// n_min..n_max) in one CUDA-graph launch.
//
// The graph, recorded once per plan:
//   1. (before the graph, on the caller's stream) the batch size is copied
//      to the device;
//   2. bin the events by multiplicity on the device (counts, offsets and a
//      permutation grouping the events of each n) and derive the number of
//      events of every (n, chunk) pipeline;
//   3. one branch per multiplicity, on its own stream so that the branches
//      run concurrently: for each chunk of at most cap_n events, gather the
//      chunk's uniforms, helicities and colours, then Rambo -> cut ->
//      colour-ordered recursion + colour sum (n <= n_co_max) or colour-dressed
//      recursion with sampled colours (n > n_co_max), then scatter |M|^2 back
//      to the events' positions;
//   4. join.
// Every kernel reads its event count from device memory, so the recorded
// launches serve any batch of up to max_batch events; launches for empty
// chunks return at once.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "bg_internal.h"
#include "cd_recursion.cuh"

namespace bg {
namespace {

constexpr int kNIdx = 13;  // multiplicities 0..12
constexpr int kMaxChunks = 64;

__global__ void bin_count_kernel(const int64_t* __restrict__ dB, const int32_t* __restrict__ nev, int n_min,
                                 int n_max, int64_t* __restrict__ counts, int* __restrict__ status) {
  const int64_t B = *dB;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < B; e += (int64_t)gridDim.x * blockDim.x) {
    const int n = nev[e];
    if (n < n_min || n > n_max) {
      flag_status(status, BG_EINVAL);
      continue;
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(&counts[n]), 1ull);
  }
}

// counts -> offsets, cursors and per-(n, chunk) event counts
__global__ void bin_offsets_kernel(const int64_t* __restrict__ counts, int64_t* __restrict__ offsets,
                                   int64_t* __restrict__ cursor, int64_t* __restrict__ chunk_cnt,
                                   const int64_t* __restrict__ cap) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t acc = 0;
  for (int n = 0; n < kNIdx; ++n) {
    offsets[n] = acc;
    cursor[n] = 0;
    acc += counts[n];
    for (int c = 0; c < kMaxChunks; ++c) {
      const int64_t left = (cap[n] > 0) ? counts[n] - (int64_t)c * cap[n] : 0;
      chunk_cnt[n * kMaxChunks + c] = left <= 0 ? 0 : (left < cap[n] ? left : cap[n]);
    }
  }
}

__global__ void bin_perm_kernel(const int64_t* __restrict__ dB, const int32_t* __restrict__ nev, int n_min,
                                int n_max, const int64_t* __restrict__ offsets, int64_t* __restrict__ cursor,
                                int64_t* __restrict__ perm) {
  const int64_t B = *dB;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < B; e += (int64_t)gridDim.x * blockDim.x) {
    const int n = nev[e];
    if (n < n_min || n > n_max) continue;
    const int64_t pos = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(&cursor[n]), 1ull);
    perm[offsets[n] + pos] = e;
  }
}

struct ChunkRef {
  int n, c;
  int64_t cap;
  const int64_t* cnt;      // events of this chunk (device)
  const int64_t* offsets;  // first permutation slot of each n (device)
  const int64_t* perm;
};

// Gather the inputs of chunk (n, c) into the branch's contiguous buffers.
__global__ void gather_kernel(ChunkRef ch, int n_max, int64_t stride_in, const double* __restrict__ u,
                              const int8_t* __restrict__ hel, const int8_t* __restrict__ col, int col_rows,
                              double* __restrict__ un, int8_t* __restrict__ hn, int8_t* __restrict__ cn) {
  const int64_t B = *ch.cnt;
  const int64_t* base = ch.perm + ch.offsets[ch.n] + (int64_t)ch.c * ch.cap;
  const int n = ch.n;
  const int d = 4 * (n - 2), dmax = 4 * (n_max - 2);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = base[i];
    for (int j = 0; j < d; ++j) un[i * d + j] = u[e * dmax + j];
    for (int g = 0; g < n; ++g) hn[(int64_t)g * ch.cap + i] = hel[(int64_t)g * stride_in + e];
    for (int r = 0; r < col_rows; ++r) cn[(int64_t)r * ch.cap + i] = col[(int64_t)r * stride_in + e];
  }
}

__global__ void scatter_kernel(ChunkRef ch, const double* __restrict__ me2n, double* __restrict__ me2) {
  const int64_t B = *ch.cnt;
  const int64_t* base = ch.perm + ch.offsets[ch.n] + (int64_t)ch.c * ch.cap;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B; i += (int64_t)gridDim.x * blockDim.x)
    me2[base[i]] = me2n[i];
}

}  // namespace
}  // namespace bg

using namespace bg;

struct bg_mixed {
  bg_mixed_desc d;
  int device = 0, sms = 0;
  int64_t cap[kNIdx] = {0};
  int nchunks[kNIdx] = {0};
  bg_colormat* C[kNIdx] = {nullptr};
  // inputs / outputs (plan-owned)
  int32_t* nev = nullptr;
  double* u = nullptr;
  int8_t* hel = nullptr;
  int8_t* col = nullptr;
  double* me2 = nullptr;
  // binning
  int64_t* dB = nullptr;
  int64_t* counts = nullptr;
  int64_t* offsets = nullptr;
  int64_t* cursor = nullptr;
  int64_t* chunk_cnt = nullptr;
  int64_t* dcap = nullptr;
  int64_t* perm = nullptr;
  // per-multiplicity buffers
  double* un[kNIdx] = {nullptr};
  int8_t* hn[kNIdx] = {nullptr};
  int8_t* cn[kNIdx] = {nullptr};
  double* p[kNIdx] = {nullptr};
  uint8_t* acc[kNIdx] = {nullptr};
  void* amps[kNIdx] = {nullptr};
  double* me2n[kNIdx] = {nullptr};
  void* cdws[kNIdx] = {nullptr};
  int64_t cdws_bytes[kNIdx] = {0};
  std::vector<void*> allocs;
  cudaStream_t main_s = nullptr;
  cudaStream_t br_s[kNIdx] = {nullptr};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[kNIdx] = {nullptr};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t bytes = 0;
};

namespace {

bg_status mixed_alloc(bg_mixed* P, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) return BG_OK;
  cudaError_t e = device_alloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return alloc_failure(e, "bg_mixed_create");
  }
  P->allocs.push_back(*ptr);
  P->bytes += (int64_t)bytes;
  return BG_OK;
}

// Records the whole DAG on P->main_s (stream capture in progress).
cudaError_t mixed_record(bg_mixed* P) {
  const bg_mixed_desc& d = P->d;
  cudaStream_t ms = P->main_s;
  int* status = device_status_ptr();
  const unsigned bin_blocks = (unsigned)std::min<int64_t>((d.max_batch + 255) / 256, 4 * (int64_t)P->sms);
  cudaError_t e = cudaMemsetAsync(P->counts, 0, kNIdx * sizeof(int64_t), ms);
  if (e != cudaSuccess) return e;
  bin_count_kernel<<<bin_blocks, 256, 0, ms>>>(P->dB, P->nev, d.n_min, d.n_max, P->counts, status);
  bin_offsets_kernel<<<1, 32, 0, ms>>>(P->counts, P->offsets, P->cursor, P->chunk_cnt, P->dcap);
  bin_perm_kernel<<<bin_blocks, 256, 0, ms>>>(P->dB, P->nev, d.n_min, d.n_max, P->offsets, P->cursor, P->perm);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaEventRecord(P->fork_ev, ms)) != cudaSuccess) return e;
  for (int n = d.n_min; n <= d.n_max; ++n) {
    cudaStream_t s = P->br_s[n];
    if ((e = cudaStreamWaitEvent(s, P->fork_ev, 0)) != cudaSuccess) return e;
    const bool co = n <= d.n_co_max;
    const int col_rows = co ? 0 : (d.color_mode == BG_COL_FLOW ? 2 * n : n);
    const int64_t cap = P->cap[n];
    const unsigned gblocks = (unsigned)std::min<int64_t>((cap + 255) / 256, 4 * (int64_t)P->sms);
    for (int c = 0; c < P->nchunks[n]; ++c) {
      ChunkRef ch{n, c, cap, P->chunk_cnt + n * kMaxChunks + c, P->offsets, P->perm};
      gather_kernel<<<gblocks, 256, 0, s>>>(ch, d.n_max, d.max_batch, P->u, P->hel, P->col, col_rows, P->un[n],
                                            P->hn[n], P->cn[n]);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = launch_rambo(n, cap, d.sqrt_s, P->un[n], P->p[n], d.pt_min, P->acc[n], s, ch.cnt)) != cudaSuccess)
        return e;
      if (co) {
        e = (d.prec == BG_F32) ? launch_co_f32(n, cap, d.sqrt_s, P->p[n], P->hn[n], d.q,
                                               static_cast<float*>(P->amps[n]), status, s, ch.cnt)
                               : launch_co_f64(n, cap, d.sqrt_s, P->p[n], P->hn[n], d.q,
                                               static_cast<double*>(P->amps[n]), status, s, ch.cnt);
        if (e != cudaSuccess) return e;
        ColourSumArgs a;
        a.n = n;
        a.B = cap;
        a.H = 1;
        a.k = P->C[n]->k;
        a.amps = P->amps[n];
        a.amps_f32 = (d.prec == BG_F32);
        a.C64 = P->C[n]->C64;
        a.C32 = P->C[n]->C32;
        a.scale = std::pow(d.g_s, 2 * n - 4) * std::pow(d.sqrt_s, 8 - 2 * n) * std::ldexp(1.0, n);
        a.accept = P->acc[n];
        a.me2 = P->me2n[n];
        a.dB = ch.cnt;
        const bool tc = (d.cs_mode == BG_CS_TC_BF16) && P->C[n]->tc_tiles;
        e = tc ? launch_color_sum_tc(a, P->C[n], status, s)
               : (d.cs_mode == BG_CS_F64 ? launch_color_sum_f64(a, s) : launch_color_sum_f32(a, s));
        if (e != cudaSuccess) return e;
      } else {
        CdParams prm;
        prm.B = cap;
        prm.dB = ch.cnt;
        prm.inv_sqrt_s = 1.0 / d.sqrt_s;
        const double wcol = std::pow(d.color_mode == BG_COL_FLOW ? 9.0 : 8.0, n);
        prm.scale = wcol * std::ldexp(1.0, n) * std::pow(d.g_s, 2 * n - 4) * std::pow(d.sqrt_s, 8 - 2 * n) *
                    std::ldexp(1.0, -(n - 2));
        prm.flow = (d.color_mode == BG_COL_FLOW) ? 1 : 0;
        for (int m = 0; m < 4; ++m) prm.q.v[m] = d.q[m];
        e = (d.prec == BG_F32) ? launch_cd_f32(n, prm, P->p[n], P->hn[n], P->cn[n], P->acc[n], P->me2n[n],
                                               P->cdws[n], status, P->sms, s)
                               : launch_cd_f64(n, prm, P->p[n], P->hn[n], P->cn[n], P->acc[n], P->me2n[n],
                                               P->cdws[n], status, P->sms, s);
        if (e != cudaSuccess) return e;
      }
      scatter_kernel<<<gblocks, 256, 0, s>>>(ch, P->me2n[n], P->me2);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = cudaEventRecord(P->join_ev[n], s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(ms, P->join_ev[n], 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" {

void bg_mixed_destroy(bg_mixed* P) {
  if (!P) return;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  for (void* a : P->allocs) cudaFree(a);
  for (int n = 0; n < kNIdx; ++n) {
    if (P->C[n]) bg_colormat_destroy(P->C[n]);
    if (P->br_s[n]) cudaStreamDestroy(P->br_s[n]);
    if (P->join_ev[n]) cudaEventDestroy(P->join_ev[n]);
  }
  if (P->fork_ev) cudaEventDestroy(P->fork_ev);
  if (P->main_s) cudaStreamDestroy(P->main_s);
  delete P;
}

bg_status bg_mixed_create(const bg_mixed_desc* d, bg_mixed** out) {
  AllocScope scope;
  if (!d || !out) return fail(BG_EINVAL, "bg_mixed_create: NULL argument");
  *out = nullptr;
  if (d->n_min < 4 || d->n_max > kMaxN || d->n_min > d->n_max)
    return fail(BG_EINVAL, "bg_mixed_create: need 4 <= n_min <= n_max <= 12");
  if (d->max_batch < 1) return fail(BG_EINVAL, "bg_mixed_create: max_batch must be >= 1");
  if (!(d->sqrt_s > 0.0)) return fail(BG_EINVAL, "bg_mixed_create: sqrt_s must be > 0");
  if (d->prec != BG_F32 && d->prec != BG_F64) return fail(BG_EINVAL, "bg_mixed_create: invalid precision");
  if (d->cs_mode != BG_CS_F64 && d->cs_mode != BG_CS_F32 && d->cs_mode != BG_CS_TC_BF16)
    return fail(BG_EINVAL, "bg_mixed_create: invalid colour-sum mode");
  if (d->color_mode != BG_COL_ADJOINT && d->color_mode != BG_COL_FLOW)
    return fail(BG_EINVAL, "bg_mixed_create: invalid colour mode");
  if (d->n_co_max > kMaxNCO) return fail(BG_EINVAL, "bg_mixed_create: n_co_max must be <= 9");
  const double qv = std::sqrt(d->q[1] * d->q[1] + d->q[2] * d->q[2] + d->q[3] * d->q[3]);
  if (!(d->q[0] > 0.0) || std::fabs(d->q[0] - qv) > 1e-12 * d->q[0])
    return fail(BG_EINVAL, "bg_mixed_create: q must be light-like with q0 > 0");
  const int64_t chunk_budget = d->chunk_bytes > 0 ? d->chunk_bytes : (int64_t(8) << 30);
  bg_mixed* P = new (std::nothrow) bg_mixed();
  if (!P) return fail(BG_ENOMEM, "bg_mixed_create: host allocation failed");
  P->d = *d;
  cudaGetDevice(&P->device);
  cudaDeviceGetAttribute(&P->sms, cudaDevAttrMultiProcessorCount, P->device);
  const int64_t MB = d->max_batch;
  bg_status st = BG_OK;
#define MX_ALLOC(ptr, bytes)                                                      \
  do {                                                                           \
    void* tmp_ = nullptr;                                                        \
    st = mixed_alloc(P, &tmp_, (size_t)(bytes));                                 \
    if (st != BG_OK) {                                                           \
      bg_mixed_destroy(P);                                                       \
      return st;                                                                 \
    }                                                                            \
    ptr = reinterpret_cast<decltype(ptr)>(tmp_);                                 \
  } while (0)
  MX_ALLOC(P->nev, MB * sizeof(int32_t));
  MX_ALLOC(P->u, MB * 4 * (d->n_max - 2) * sizeof(double));
  MX_ALLOC(P->hel, MB * d->n_max);
  MX_ALLOC(P->col, MB * 2 * d->n_max);
  MX_ALLOC(P->me2, MB * sizeof(double));
  MX_ALLOC(P->dB, sizeof(int64_t));
  MX_ALLOC(P->counts, kNIdx * sizeof(int64_t));
  MX_ALLOC(P->offsets, kNIdx * sizeof(int64_t));
  MX_ALLOC(P->cursor, kNIdx * sizeof(int64_t));
  MX_ALLOC(P->chunk_cnt, kNIdx * kMaxChunks * sizeof(int64_t));
  MX_ALLOC(P->dcap, kNIdx * sizeof(int64_t));
  MX_ALLOC(P->perm, MB * sizeof(int64_t));
  const size_t amp_size = d->prec == BG_F32 ? 4 : 8;
  for (int n = d->n_min; n <= d->n_max; ++n) {
    const bool co = n <= d->n_co_max;
    int64_t per_event = 4 * (n - 2) * 8 + n + 2 * n + 4 * n * 8 + 1 + 8;
    if (co) per_event += (int64_t)factorial(n - 2) * amp_size;
    int64_t cap = std::min<int64_t>(MB, std::max<int64_t>(256, chunk_budget / per_event));
    if (cap < MB) cap = std::max<int64_t>(256, (cap / 256) * 256);
    const int64_t nch = (MB + cap - 1) / cap;
    if (nch > kMaxChunks) {
      bg_mixed_destroy(P);
      return fail(BG_EINVAL, "bg_mixed_create: max_batch too large for the chunk budget (more than 64 chunks)");
    }
    P->cap[n] = cap;
    P->nchunks[n] = (int)nch;
    MX_ALLOC(P->un[n], cap * 4 * (n - 2) * sizeof(double));
    MX_ALLOC(P->hn[n], cap * n);
    MX_ALLOC(P->cn[n], co ? 0 : cap * 2 * n);
    MX_ALLOC(P->p[n], cap * 4 * n * sizeof(double));
    MX_ALLOC(P->acc[n], cap);
    MX_ALLOC(P->me2n[n], cap * sizeof(double));
    if (co) {
      MX_ALLOC(P->amps[n], cap * (int64_t)factorial(n - 2) * amp_size);
      st = bg_colormat_create(n, &P->C[n]);
      if (st != BG_OK) {
        bg_mixed_destroy(P);
        return st;
      }
      P->bytes += (int64_t)P->C[n]->k * P->C[n]->k * 12;
    } else {
      int64_t wsb = 0;
      st = bg_cd_workspace_bytes(n, d->prec, &wsb);
      if (st != BG_OK) {
        bg_mixed_destroy(P);
        return st;
      }
      MX_ALLOC(P->cdws[n], wsb);
      P->cdws_bytes[n] = wsb;
    }
  }
#undef MX_ALLOC
  if (d->autotune) {
    for (int n = d->n_min; n <= d->n_max; ++n) {
      const bg_algo algo = n <= d->n_co_max ? BG_ALGO_CO : BG_ALGO_CD;
      if (bg_tune_num_variants(algo, n) < 2) continue;
      st = bg_autotune(algo, n, d->prec, 0, nullptr, nullptr, nullptr);
      if (st != BG_OK) {
        bg_mixed_destroy(P);
        return st;
      }
    }
  }
  st = cuda_check(cudaMemcpy(P->dcap, P->cap, sizeof(P->cap), cudaMemcpyHostToDevice), "bg_mixed_create: upload");
  if (st != BG_OK) {
    bg_mixed_destroy(P);
    return st;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&P->main_s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->fork_ev, cudaEventDisableTiming);
  for (int n = d->n_min; n <= d->n_max && e == cudaSuccess; ++n) {
    e = cudaStreamCreateWithFlags(&P->br_s[n], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->join_ev[n], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    bg_mixed_destroy(P);
    return cuda_check(e, "bg_mixed_create: streams");
  }
  // Run the DAG once uncaptured with an empty batch: every kernel returns at
  // once, and the launchers' one-time set-up (shared-memory attributes)
  // happens outside the capture.
  e = cudaMemsetAsync(P->dB, 0, sizeof(int64_t), P->main_s);
  if (e == cudaSuccess) e = mixed_record(P);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->main_s);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(P->main_s, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaError_t er = mixed_record(P);
    e = cudaStreamEndCapture(P->main_s, &P->graph);
    if (er != cudaSuccess) e = er;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&P->exec, P->graph, 0);
  if (e != cudaSuccess) {
    bg_mixed_destroy(P);
    return cuda_check(e, "bg_mixed_create: graph capture");
  }
  *out = P;
  return BG_OK;
}

bg_status bg_mixed_buffers(bg_mixed* P, int32_t** n_per_event, double** u, int8_t** hel, int8_t** colors,
                           double** me2) {
  if (!P) return fail(BG_EINVAL, "bg_mixed_buffers: NULL plan");
  if (n_per_event) *n_per_event = P->nev;
  if (u) *u = P->u;
  if (hel) *hel = P->hel;
  if (colors) *colors = P->col;
  if (me2) *me2 = P->me2;
  return BG_OK;
}

int64_t bg_mixed_workspace_bytes(const bg_mixed* P) { return P ? P->bytes : 0; }

bg_status bg_mixed_run(bg_mixed* P, int64_t B, void* stream) {
  if (!P) return fail(BG_EINVAL, "bg_mixed_run: NULL plan");
  if (B < 0 || B > P->d.max_batch) return fail(BG_EINVAL, "bg_mixed_run: B outside 0..max_batch");
  cudaStream_t s = (cudaStream_t)stream;
  // B is copied from pageable memory: the copy is staged before the call
  // returns, and it is ordered before the graph on the caller's stream
  bg_status st = cuda_check(cudaMemcpyAsync(P->dB, &B, sizeof(int64_t), cudaMemcpyHostToDevice, s),
                            "bg_mixed_run: batch size");
  if (st != BG_OK) return st;
  return cuda_check(cudaGraphLaunch(P->exec, s), "bg_mixed_run: graph launch");
}

bg_status bg_mixed_kernel_nodes(const bg_mixed* P, int64_t* kernels) {
  if (!P || !kernels) return fail(BG_EINVAL, "bg_mixed_kernel_nodes: NULL argument");
  if (!P->graph) return fail(BG_EINVAL, "bg_mixed_kernel_nodes: plan has no graph");
  size_t num = 0;
  bg_status st = cuda_check(cudaGraphGetNodes(P->graph, nullptr, &num), "bg_mixed_kernel_nodes");
  if (st != BG_OK) return st;
  std::vector<cudaGraphNode_t> nodes(num);
  if (num) {
    st = cuda_check(cudaGraphGetNodes(P->graph, nodes.data(), &num), "bg_mixed_kernel_nodes");
    if (st != BG_OK) return st;
  }
  int64_t k = 0;
  for (size_t i = 0; i < num; ++i) {
    cudaGraphNodeType t;
    st = cuda_check(cudaGraphNodeGetType(nodes[i], &t), "bg_mixed_kernel_nodes");
    if (st != BG_OK) return st;
    k += t == cudaGraphNodeTypeKernel ? 1 : 0;
  }
  *kernels = k;
  return BG_OK;
}

bg_status bg_mixed_counts(bg_mixed* P, int64_t* counts) {
  if (!P || !counts) return fail(BG_EINVAL, "bg_mixed_counts: NULL argument");
  // the counts of the last run: wait for it on the device
  bg_status st = cuda_check(cudaDeviceSynchronize(), "bg_mixed_counts: synchronise");
  if (st != BG_OK) return st;
  return cuda_check(cudaMemcpy(counts, P->counts, kNIdx * sizeof(int64_t), cudaMemcpyDeviceToHost),
                    "bg_mixed_counts");
}

}  // extern "C"
