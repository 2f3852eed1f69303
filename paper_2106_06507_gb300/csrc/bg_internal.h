// bg_internal.h -- declarations shared by the translation units of libbg.so.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bg.h"

namespace bg {

// Thread-local last-error message (bg_last_error).
void set_error(const std::string& msg);
bg_status fail(bg_status code, const std::string& msg);
bg_status cuda_check(cudaError_t e, const char* what);

constexpr int kMaxN = 12;
constexpr int kMaxNCO = 9;  // colour-ordered path: (n-2)! orderings

int64_t factorial(int m);

// Host colour-matrix generator (colormat.cpp).
// First row C[id][tau] of Eq. (2.17), tau in lexicographic order.
void colour_row(int n, std::vector<double>& row);
// Lexicographic rank of a permutation of 0..m-1.
int64_t perm_rank(const int* perm, int m);
// Dense matrix from the row: C[s][t] = row[rank(sigma_s^-1 o sigma_t)].
void colour_dense(int n, const std::vector<double>& row, std::vector<double>& dense);

// Device allocation of the create calls (api.cu).  It returns
// cudaErrorMemoryAllocation without allocating when the environment variable
// BG_FAIL_ALLOC=k is set and this is the k-th allocation of the current
// top-level create call (counted from 1 across nested creates): a host-side
// hook that lets the tests reach every BG_ENOMEM path.  AllocScope marks a
// create call; nested scopes share the outer count.
cudaError_t device_alloc(void** ptr, size_t bytes);
struct AllocScope {
  AllocScope();
  ~AllocScope();
};
// BG_ENOMEM for an out-of-memory error, BG_ECUDA with the runtime's message
// for any other failed allocation (no device, an earlier sticky error).
bg_status alloc_failure(cudaError_t e, const char* what);

// Device status word and SM count of the current device (api.cu; 0 if
// there is no device).
int* device_status_ptr();
int device_sms();

// Kernel launchers (one per .cu file).
// Kernels take a capacity B (row stride of event-indexed SoA arrays) and an
// optional device-side event count dB (<= B; NULL means B), so that a launch
// can be recorded once in a CUDA graph and replayed for varying counts.
cudaError_t launch_rambo(int n, int64_t B, double sqrt_s, const double* u, double* p, double pt_min,
                         uint8_t* accept, cudaStream_t s, const int64_t* dB = nullptr);

// variant < 0: the autotuner's choice for (n, precision) on the current
// device, else the default (tune.cu).
cudaError_t launch_co_f32(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                          float* amps, int* status, cudaStream_t s, const int64_t* dB = nullptr, int variant = -1);
cudaError_t launch_co_f64(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                          double* amps, int* status, cudaStream_t s, const int64_t* dB = nullptr, int variant = -1);
int co_variants(int n, bool helicity_sum);  // number of recursion variants
// The same currents with the auxiliary tensor field in place of the
// four-gluon vertex (co_tensor.cu).
cudaError_t launch_co_tensor_f32(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel,
                                 const double* q, float* amps, int* status, cudaStream_t s);
cudaError_t launch_co_tensor_f64(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel,
                                 const double* q, double* amps, int* status, cudaStream_t s);

// Autotuner table (tune.cu): the chosen variant of a kernel family for
// (n, precision) on the current device, or -1 (default).
enum TuneFamily { kTuneCO = 0, kTuneCD = 1 };
int tune_variant(int family, int n, int prec);

struct ColourSumArgs {
  int n;
  int64_t B;
  int H;
  int k;
  const void* amps;
  bool amps_f32;
  const double* C64;  // [k][k]
  const float* C32;   // [k][k]
  double scale;       // g^(2n-4) sqrt_s^(8-2n) w
  const uint8_t* accept;
  double* me2;
  void* Y = nullptr;   // optional output (C A)[B][H][k], same type as amps
  const int64_t* dB = nullptr;  // optional device-side event count (<= B)
};
cudaError_t launch_color_sum_f64(const ColourSumArgs& a, cudaStream_t s);

// Colour-dressed recursion (cd_f32.cu, cd_f64.cu): workspace bytes and
// launchers; CdParams is defined in cd_recursion.cuh.
struct CdParams;
size_t cd_workspace_bytes_f32(int n, int sms);  // 0 if the kernel cannot launch
size_t cd_workspace_bytes_f64(int n, int sms);
cudaError_t launch_cd_f32(int n, const CdParams& prm, const double* p, const int8_t* hel, const int8_t* col,
                          const uint8_t* accept, double* me2, void* workspace, int* status, int sms, cudaStream_t s,
                          int variant = -1);
cudaError_t launch_cd_f64(int n, const CdParams& prm, const double* p, const int8_t* hel, const int8_t* col,
                          const uint8_t* accept, double* me2, void* workspace, int* status, int sms, cudaStream_t s,
                          int variant = -1);
int cd_variants(int n);  // number of kernel variants (threads per event)
// (CdParams carries the capacity B and an optional device-side count dB.)

// Colour-flow sampling with colour-ordered amplitudes (comc_f32.cu,
// comc_f64.cu); ComcParams is defined in comc.cuh.
struct ComcParams;
cudaError_t launch_comc_f32(int n, const ComcParams& prm, const double* p, const int8_t* hel, const int8_t* col,
                            const uint8_t* accept, const double* q, double* me2, void* workspace, int sms, int* status,
                            cudaStream_t s);
cudaError_t launch_comc_f64(int n, const ComcParams& prm, const double* p, const int8_t* hel, const int8_t* col,
                            const uint8_t* accept, const double* q, double* me2, void* workspace, int sms, int* status,
                            cudaStream_t s);

// Gradient (co_grad.cu, grad_rambo.cu).
cudaError_t launch_co_grad_f32(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                               const float* Y, double* kbar, double* ebar, int* status, cudaStream_t s);
cudaError_t launch_co_grad_f64(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                               const double* Y, double* kbar, double* ebar, int* status, cudaStream_t s);
cudaError_t launch_rambo_grad(int n, int64_t B, double sqrt_s, const double* u, const double* p, const int8_t* hel,
                              const double* q, const double* kbar, const double* ebar, double scale,
                              const double* upstream, const uint8_t* accept, double* grad_u, cudaStream_t s);

// Tensor-core colour sum (color_sum_tc.cu).
bool build_tc_tiles(int n, const std::vector<double>& dense, int k, std::vector<uint16_t>& tiles, double& g, int& nt,
                    int& ntiles, int& kchunks, int& cpl);
cudaError_t launch_color_sum_f32(const ColourSumArgs& a, cudaStream_t s);

}  // namespace bg

struct bg_plan {
  bg_plan_desc d;
  int k;       // orderings
  int H;       // polarisation configurations per event
  int device;
  bg_colormat* C;
  // device workspace
  double* u;        // [max_batch][4(n-2)] staging for host uniforms
  int8_t* hel;      // [n][max_batch] staging for host helicities
  int8_t* colors;   // [2n][max_batch] staging for host colours
  double* p;        // [4][n][max_batch]
  uint8_t* accept;  // [max_batch]
  void* amps;       // [max_batch][H][k]
  double* me2;      // [max_batch] staging for a host output
  void* Y;          // [max_batch][k] (C A), gradient plans only
  double* kbar;     // [max_batch][n][4] momentum adjoints, gradient plans only
  double* ebar;     // [max_batch][n][4] polarisation adjoints, gradient plans only
  int64_t bytes;
};

struct bg_colormat {
  int n;
  int k;
  int device;
  std::vector<double> row;  // host copy of the first row
  double* C64;              // device [k][k]
  float* C32;               // device [k][k]
  // tensor-core operand: BF16 tiles of C / tc_g (NULL if not available)
  uint16_t* tc_tiles_raw;
  const __nv_bfloat16* tc_tiles;
  double tc_g;
  int tc_nt, tc_ntiles, tc_kchunks, tc_cpl;
};

namespace bg {
cudaError_t launch_color_sum_tc(const ColourSumArgs& a, const bg_colormat* C, int* status, cudaStream_t s);
}
