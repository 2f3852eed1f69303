/* bg.h -- C ABI of the GB300 Berends-Giele library (libbg.so).
 *
 * Per-event colour- and helicity-summed (or sampled) squared tree amplitudes
 * |M|^2 for n-gluon scattering, gg -> (n-2) g, computed with the
 * Berends-Giele recursion of "Many-gluon tree amplitudes on modern GPUs"
 * (Bothmann, Giele, Hoeche, Isaacson, Knobbe), in two forms:
 *   - colour-ordered currents (Sec. 2.3, Eqs. 2.20-2.22) for all (n-2)!
 *     orderings of the adjoint (DDM) basis, Eq. (2.15), followed by the
 *     colour sum A^T C A of Eq. (2.16) with the colour matrix of Eq. (2.17);
 *   - colour-dressed currents (Eqs. 2.28-2.32) for sampled colours.
 * Inputs are Rambo phase-space points (Sec. 3) and helicity / colour labels;
 * the output is |M|^2 per event, as in the paper's statement of the problem
 * (Eqs. 2.1, 2.4).
 *
 * Conventions shared by every call
 *   - n is the total number of gluons (gg -> gg is n = 4); 4 <= n <= 12.
 *   - All array arguments are caller-owned DEVICE pointers unless stated
 *     otherwise; the library never frees them.  Nothing here allocates
 *     memory except bg_colormat_create and bg_plan_create.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     are asynchronous on it: argument errors are returned synchronously,
 *     launch errors as BG_ECUDA; data-dependent device errors (an invalid
 *     helicity or colour label) are recorded in a device status word that
 *     bg_device_status() reads after a synchronisation.
 *   - Momenta are in GeV, metric (+,-,-,-).  Event-indexed arrays are
 *     structure-of-arrays with the event index fastest, so that consecutive
 *     GPU threads read consecutive addresses.
 *   - Polarisations: real light-cone-gauge vectors e1, e2 of Eq. (2.7) with
 *     reference vector q (Eq. 2.2); helicity label +1 selects e1, -1 selects
 *     e2.  Sums over both labels equal the helicity sums (Eq. 2.3).  The
 *     gauge frame: with n = q_vec/|q_vec|, a and b are x^ and y^ rotated by
 *     the rotation taking z^ to n (for n_z < 0: a(-n) and -b(-n)); e1 =
 *     A - (A.k/q.k) q, e2 = B - (B.k/q.k) q with A = (0,a), B = (0,b).  If a
 *     gluon momentum k is parallel to q (|k.q| <= 1e-9 |k0| q0), q is
 *     replaced by (q0, -q_vec) for that gluon.
 *   - Couplings: |M|^2 includes g_s^(2n-4).  It is summed (not averaged)
 *     over colours and helicities; no symmetry factor is applied.
 *   - Errors never abort and never throw.
 */
#ifndef BG_H
#define BG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BG_OK = 0,
  BG_EINVAL = 1,        /* invalid argument (size, pointer, alignment, enum) */
  BG_ENOMEM = 2,        /* device or host allocation failed (create calls only) */
  BG_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
  BG_EUNSUPPORTED = 4,  /* valid but not supported (e.g. n out of range for a mode) */
  BG_ETIMEOUT = 5       /* a bounded device wait gave up */
} bg_status;

/* Arithmetic type of the recursion (currents and amplitudes). */
typedef enum { BG_F64 = 0, BG_F32 = 1 } bg_prec;

/* Colour-sum arithmetic: FP64 CUDA cores; FP32 CUDA cores; tensor cores
 * (tcgen05, BF16 inputs: C/gcd exact in BF16, amplitudes split into three
 * BF16 planes hi+mid+lo carrying 24 significant bits; FP32 accumulation in
 * tensor memory; FP64 per-event accumulation).  At n = 9 some C/gcd entries
 * need 9-10 significant bits and C is split into two exact BF16 planes
 * (hi + lo).  BG_CS_TC_BF16 needs 6 <= n <= 9 and one polarisation
 * configuration per event. */
typedef enum { BG_CS_F64 = 0, BG_CS_F32 = 1, BG_CS_TC_BF16 = 2 } bg_cs_mode;

/* Sampled-colour representation for the colour-dressed recursion. */
typedef enum { BG_COL_ADJOINT = 0, BG_COL_FLOW = 1 } bg_color_mode;

/* Last error message of the calling thread ("" if none). */
const char* bg_last_error(void);

/* Number of colour orderings (n-2)! of the adjoint basis, Eq. (2.15);
 * 0 if n is outside 4..12. */
int64_t bg_num_orderings(int n);

/* ---------------------------------------------------------------------------
 * Colour matrix C_{sigma sigma'} of Eq. (2.17), sigma, sigma' in S_{n-2}
 * (orderings of gluons 2..n-1 in lexicographic order), normalised with
 * Tr(T^a T^b) = delta^ab so that F^a_bc = Tr(T^a [T^b, T^c]).  Built on the
 * host by expanding each chain of adjoint generators into fundamental
 * traces and contracting with the U(N) completeness relation (each term is
 * +-N^loops), then uploaded to the current device.  The object is
 * library-owned: free it with bg_colormat_destroy.  Supported: 4 <= n <= 9.
 * Errors: BG_EINVAL (n, out), BG_EUNSUPPORTED (n > 9), BG_ENOMEM, BG_ECUDA.
 * ------------------------------------------------------------------------- */
typedef struct bg_colormat bg_colormat;
bg_status bg_colormat_create(int n, bg_colormat** out);
void bg_colormat_destroy(bg_colormat* C);
/* Copies the first row C_{id, tau} (length (n-2)!) to HOST memory `row`. */
bg_status bg_colormat_row(const bg_colormat* C, double* row);
/* Same first row computed on the host only (no device is touched), for
 * 4 <= n <= 9; `row` is HOST memory of length (n-2)!. */
bg_status bg_colormat_row_host(int n, double* row);

/* ---------------------------------------------------------------------------
 * bg_momenta_rambo -- Rambo flat massless phase space (Sec. 3; Kleiss,
 * Stirling, Ellis), FP64.
 *   u       [B][4(n-2)]  uniforms in (0,1): per final-state gluon i,
 *                        u[e][4i+0..3] = (cos-theta, phi, energy, energy)
 *                        variables of the Rambo construction.
 *   p       [4][n][B]    output lab momenta (component, gluon, event);
 *                        p1 = (E,0,0,E), p2 = (E,0,0,-E), E = sqrt_s/2.
 *   accept  [B] or NULL  output 1 if every final-state gluon has
 *                        pT > pt_min (Sec. 5 cut), else 0.
 * Errors: BG_EINVAL (n outside 4..12, B < 0, NULL u/p, sqrt_s <= 0).
 * B = 0 is a no-op.
 * ------------------------------------------------------------------------- */
bg_status bg_momenta_rambo(int n, int64_t B, double sqrt_s, const double* u, double* p, double pt_min,
                           uint8_t* accept, void* stream);

/* ---------------------------------------------------------------------------
 * bg_apply_cuts -- the paper's kinematic constraints (Sec. 5) on the final-
 * state gluons 3..n of momenta written by bg_momenta_rambo: p_T > pt_min,
 * |eta| < eta_max and Delta R > dr_min for every pair, with eta =
 * asinh(p_z / p_T), phi = atan2(p_y, p_x), Delta R^2 = (Delta eta)^2 +
 * (Delta phi)^2, Delta phi in [0, pi].  eta_max <= 0 or dr_min <= 0 drop that
 * constraint.  The paper's setup: sqrt_s = 14000, pt_min = 20,
 * eta_max = 2.5, dr_min = 0.4.
 *   p       [4][n][B]    lab momenta
 *   accept  [B]          output 1 if the event passes every constraint, else 0
 * Errors: BG_EINVAL.  B = 0 is a no-op.
 * ------------------------------------------------------------------------- */
bg_status bg_apply_cuts(int n, int64_t B, const double* p, double pt_min, double eta_max, double dr_min,
                        uint8_t* accept, void* stream);

/* ---------------------------------------------------------------------------
 * bg_currents_co -- colour-ordered Berends-Giele currents, Eqs. (2.20)-(2.22),
 * for every ordering sigma in S_{n-2}: A(1, sigma_2..sigma_{n-1}, n).
 *   p       [4][n][B]    lab momenta (as written by bg_momenta_rambo).
 *   hel     [n][B] int8  helicity labels +-1 (sampled helicities), or NULL
 *                        to evaluate all H = 2^n polarisation configurations
 *                        (configuration h: gluon i takes label -1 iff bit i
 *                        of h is set).
 *   q       [4] HOST     light-like reference vector with q0 > 0.
 *   prec                 BG_F32: currents in FP32 (polarisations built in
 *                        FP64); BG_F64: all FP64.
 *   amps    [B][H][k]    output, float or double per prec, k = (n-2)!,
 *                        orderings lexicographic.  Amplitudes carry unit
 *                        coupling (g_s = 1) and are in units of sqrt_s:
 *                        A[GeV^(4-n)] = amps * sqrt_s^(4-n).
 * Momenta are divided by sqrt_s before the recursion (FP32 range).
 * Supported: 4 <= n <= 9.  Errors: BG_EINVAL, BG_EUNSUPPORTED, BG_ECUDA.
 * ------------------------------------------------------------------------- */
bg_status bg_currents_co(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                         bg_prec prec, void* amps, void* stream);

/* ---------------------------------------------------------------------------
 * bg_currents_co_tensor -- the colour-ordered currents of bg_currents_co with
 * the four-gluon vertex replaced by the auxiliary antisymmetric tensor field
 * of Eqs. (2.23)-(2.26): every segment (i..j) also carries the tensor
 * current T(i..j) = sum_s J(i..s) ^ J(s+1..j), which enters the brackets of
 * the longer segments through T(s+1..j) J(i..s) + J(s+1..j) T(i..s).  The
 * amplitudes equal those of bg_currents_co up to rounding (not bit for bit:
 * the sums run in another order).  Arguments, layouts and errors as for
 * bg_currents_co (one thread per ordering; 4 <= n <= 9).  It performs more
 * arithmetic than the four-vertex form for n <= 9 and is kept for the
 * comparison of the two forms.
 * ------------------------------------------------------------------------- */
bg_status bg_currents_co_tensor(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                                bg_prec prec, void* amps, void* stream);

/* ---------------------------------------------------------------------------
 * bg_color_sum -- |M|^2 = g_s^(2n-4) sqrt_s^(8-2n) w sum_h sum_{s,s'}
 * C_{s s'} A_{h s} A_{h s'}, Eq. (2.16), with w = 2^n if hel_sampled (one
 * sampled polarisation configuration per event, H = 1) else 1.
 *   amps    [B][H][k]    as written by bg_currents_co (amp_prec its type).
 *   accept  [B] or NULL  events with accept == 0 get |M|^2 = 0.
 *   me2     [B] double   output in GeV^(8-2n).
 * mode BG_CS_F64 accumulates in FP64; BG_CS_F32 forms C A in FP32 (C's
 * integer entries are exact in FP32) and accumulates the quadratic form
 * per event in FP64.  BG_CS_TC_BF16: every wait of the tensor-core kernel
 * on its pipeline is bounded (~2 s); if one runs out, the kernel records
 * BG_ETIMEOUT in the device status word and writes 0 for its events.  (The
 * environment variable BG_TC_TEST_STALL=1 makes the waits run out on purpose
 * after ~1 ms; it exists for the tests of that path.)
 * Errors: BG_EINVAL (NULL C/amps/me2, B < 0, H < 1), BG_ECUDA.
 * ------------------------------------------------------------------------- */
bg_status bg_color_sum(const bg_colormat* C, int64_t B, int H, const void* amps, bg_prec amp_prec,
                       bg_cs_mode mode, double g_s, double sqrt_s, int hel_sampled, const uint8_t* accept,
                       double* me2, void* stream);

/* ---------------------------------------------------------------------------
 * Plans: the whole hot path for one multiplicity behind one call.
 * bg_plan_create allocates the plan's device workspace (momenta, cut flags,
 * amplitudes, staging buffers for host inputs) for up to max_batch events
 * and, for the colour-ordered algorithm, the colour matrix; bg_me2_batch
 * then runs Rambo -> cut -> polarisations -> recursion -> colour sum without
 * allocating.
 *   algo BG_ALGO_CO: colour-ordered currents + exact colour sum (n <= 9).
 *   hel_sampled: 1 = one helicity configuration per event (hel given,
 *   weight 2^n); 0 = sum over all 2^n configurations (hel ignored).
 * ------------------------------------------------------------------------- */
typedef enum { BG_ALGO_CO = 0, BG_ALGO_CD = 1 } bg_algo;
typedef struct {
  int n;
  int64_t max_batch;
  double sqrt_s;
  double pt_min;      /* final-state pT cut in GeV (< 0: none) */
  double g_s;         /* strong coupling, e.g. sqrt(4 pi 0.118) */
  double q[4];        /* light-like reference vector of the polarisations */
  bg_prec prec;       /* recursion arithmetic */
  bg_cs_mode cs_mode; /* colour-sum arithmetic (BG_ALGO_CO) */
  bg_algo algo;
  bg_color_mode color_mode; /* BG_ALGO_CD */
  int hel_sampled;
  int grad;           /* 1: also allocate the workspace of bg_me2_grad */
} bg_plan_desc;
typedef struct bg_plan bg_plan;
/* Errors: BG_EINVAL (desc), BG_EUNSUPPORTED, BG_ENOMEM, BG_ECUDA. */
bg_status bg_plan_create(const bg_plan_desc* desc, bg_plan** out);
void bg_plan_destroy(bg_plan* plan);
/* Bytes of device workspace the plan holds (colour matrix included). */
int64_t bg_plan_workspace_bytes(const bg_plan* plan);

/* ---------------------------------------------------------------------------
 * bg_me2_batch -- |M|^2 for B <= max_batch events of the plan's
 * multiplicity.
 *   u       [B][4(n-2)] double   Rambo uniforms
 *   hel     [n][B] int8 (+-1)    sampled helicities (hel_sampled = 1), else NULL
 *   colors  unused by BG_ALGO_CO (NULL)
 *   me2     [B] double           output, GeV^(8-2n)
 * Each of u, hel, me2 may be device memory or host memory (pinned or
 * pageable); host buffers are staged through the plan's workspace with
 * copies on `stream`.  If me2 is host memory the call synchronises `stream`
 * before returning, so the values are ready.  Calls on one plan must not
 * overlap (they share its workspace).
 * ------------------------------------------------------------------------- */
bg_status bg_me2_batch(bg_plan* plan, int64_t B, const double* u, const int8_t* hel, const int8_t* colors,
                       double* me2, void* stream);

/* bg_me2_batch_async -- as bg_me2_batch, but it never waits: every copy and
 * kernel is enqueued on `stream` and the call returns.  With PINNED host
 * buffers the copies are asynchronous, so that calls of several plans on
 * several streams overlap their host<->device transfers with each other's
 * kernels; |M|^2 in a host `me2` is valid once `stream` has completed (for
 * example after cudaStreamSynchronize).  Host buffers must stay unchanged
 * and alive until then.  (Pageable host buffers work too, but their copies
 * are synchronous with the host.)  Errors: as bg_me2_batch. */
bg_status bg_me2_batch_async(bg_plan* plan, int64_t B, const double* u, const int8_t* hel, double* me2,
                             void* stream);

/* ---------------------------------------------------------------------------
 * bg_me2_batch_noalloc -- the same pipeline as bg_me2_batch (Rambo -> cut ->
 * polarisations -> colour-ordered recursion -> colour sum) for callers that
 * cannot allocate device memory when they need |M|^2: for example a host
 * program whose memory pool has already reserved the GPU's memory, an event
 * loop that must not stall on the device-wide synchronisation cudaMalloc
 * and cudaFree imply, or a plug-in that a host framework calls through this
 * C interface and that owns no memory of its own.  The paper has no
 * counterpart; it is a deployment variant of the same computation.
 *   C       colour matrix from bg_colormat_create (made once, at set-up)
 *   u       [B][4(n-2)] double DEVICE   Rambo uniforms
 *   hel     [n][B] int8 DEVICE (+-1)    sampled helicities, or NULL for the
 *                                       sum over all 2^n configurations
 *   me2     [B] double DEVICE           output, GeV^(8-2n)
 * prec, cs_mode as for bg_currents_co / bg_color_sum; n = C's multiplicity.
 * The momenta, cut flags and amplitudes between the kernels live in one
 * fixed 64 MiB array of device memory that is part of the library image:
 * every GPU that loads libbg.so holds it until the process exits.  B is
 * limited by that size (at n = 8 with FP32 amplitudes and sampled
 * helicities, about 21000 events per call); a larger B returns BG_EINVAL
 * with the limit in bg_last_error().  The call allocates nothing.  Its first
 * call on each device looks up the array's device address with the runtime
 * (that device must be current); make that first call before any stream
 * capture (a first call made during capture returns BG_EINVAL and says so).
 * All calls share the one array: calls that overlap on the GPU (different
 * streams or threads without ordering between them) race on it and give
 * wrong results.  Nothing in the array needs to start at zero: a call writes
 * every byte it reads.  As for the other entry points, an invalid helicity
 * label or a tensor-core wait that gave up is recorded in the device status
 * word (bg_device_status); in that case me2 is not valid.
 * Errors: BG_EINVAL, BG_EUNSUPPORTED, BG_ECUDA.
 * ------------------------------------------------------------------------- */
bg_status bg_me2_batch_noalloc(const bg_colormat* C, int64_t B, double sqrt_s, double pt_min, double g_s,
                               const double* q, bg_prec prec, bg_cs_mode cs_mode, const double* u,
                               const int8_t* hel, double* me2, void* stream);

/* ---------------------------------------------------------------------------
 * bg_me2_grad -- |M|^2 and its gradient with respect to the 4(n-2) Rambo
 * uniforms of each event, d|M|^2/du, by reverse mode through the colour sum
 * (Eq. 2.16: d|M|^2/dA = 2 scale C A), the colour-ordered recursion (Eqs.
 * 2.20-2.22, one ordering per thread, currents and their adjoints in
 * registers),
 * the light-cone polarisations (Eq. 2.7) and Rambo (forward-mode Jacobian,
 * FP64).  The paper computes no gradients; this serves gradient-trained
 * phase-space mappings.
 *   plan      created with algo BG_ALGO_CO, hel_sampled = 1, grad = 1, n <= 8
 *   u         [B][4(n-2)] double DEVICE
 *   hel       [n][B] int8 DEVICE
 *   upstream  [B] double DEVICE, dL/d|M|^2 per event, or NULL for 1
 *   me2       [B] double DEVICE output, or NULL
 *   grad_u    [B][4(n-2)] double DEVICE output: upstream * d|M|^2/du
 * Events failing the cut get |M|^2 = 0 and a zero gradient (the cut is a
 * step function).  The sums over orderings are taken in a fixed order:
 * repeated calls give bitwise identical results.
 * Errors: BG_EINVAL, BG_EUNSUPPORTED, BG_ECUDA.
 * ------------------------------------------------------------------------- */
bg_status bg_me2_grad(bg_plan* plan, int64_t B, const double* u, const int8_t* hel, const double* upstream,
                      double* me2, double* grad_u, void* stream);

/* ---------------------------------------------------------------------------
 * bg_currents_cd -- colour-dressed Berends-Giele recursion with sampled
 * colours, Eqs. (2.28)-(2.32) (auxiliary tensor field of Eqs. 2.23-2.26 for
 * the four-gluon vertex), one sampled helicity and colour configuration per
 * event, returning the Monte-Carlo estimate of the colour- and
 * helicity-summed |M|^2:
 *   me2 = w_col * 2^n * g_s^(2n-4) * |A(colours, helicities)|^2,
 *   w_col = 8^n (adjoint) or 9^n (colour flow).
 *   p       [4][n][B]    lab momenta (bg_momenta_rambo)
 *   hel     [n][B] int8  helicity labels +-1
 *   colors  BG_COL_ADJOINT: [n][B] int8 adjoint index 1..8 (external colour
 *           matrix T^a, with -i T^a for a = 2, 5, 7: a phase only);
 *           BG_COL_FLOW: [2n][B] int8, rows 2i and 2i+1 the pair (r_i, c_i)
 *           in 1..3 (external colour matrix |r_i><c_i|)
 *   accept  [B] or NULL  events with accept == 0 get 0
 *   me2     [B] double   output, GeV^(8-2n)
 *   workspace, workspace_bytes: caller-owned device scratch of at least
 *           bg_cd_workspace_bytes(n, prec) bytes (per-CTA tables of the
 *           subset currents); nothing needs to be zeroed.
 * Supported: 4 <= n <= 12.  Errors: BG_EINVAL, BG_ECUDA.
 * ------------------------------------------------------------------------- */
bg_status bg_cd_workspace_bytes(int n, bg_prec prec, int64_t* bytes);
bg_status bg_currents_cd(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel,
                         const int8_t* colors, bg_color_mode cm, const double* q, bg_prec prec, double g_s,
                         const uint8_t* accept, double* me2, void* workspace, int64_t workspace_bytes,
                         void* stream);

/* ---------------------------------------------------------------------------
 * bg_currents_cd_cont -- the colour-dressed recursion of bg_currents_cd with
 * continuous colour and helicity sampling (Sec. 2.1): per gluon two real
 * unit colour vectors eta = (cos t, sin t cos f, sin t sin f) and eta_bar,
 * the gluon colour polarisation eta^a = eta T^a eta_bar, and the
 * polarisation vector e = cos(phi_h) e1 + sin(phi_h) e2 (e1, e2 of Eq. 2.7);
 *   me2 = 9^n * 2^n * g_s^(2n-4) * |A(colour vectors, angles)|^2
 * for cos t, cos t_bar uniform in (-1, 1) and the angles uniform in
 * (0, 2 pi) (colour weight N_c per sphere, polarisation weight 2).
 *   p       [4][n][B]    lab momenta (bg_momenta_rambo)
 *   ang     [5n][B]      double; rows 5g..5g+4 for gluon g: cos(theta),
 *                        phi, cos(theta_bar), phi_bar, phi_h
 *   accept  [B] or NULL  events with accept == 0 get 0
 *   me2     [B] double   output, GeV^(8-2n)
 *   workspace: as for bg_currents_cd (bg_cd_workspace_bytes(n, prec)).
 * Supported: 4 <= n <= 12.  Errors: BG_EINVAL, BG_ECUDA.
 * ------------------------------------------------------------------------- */
bg_status bg_currents_cd_cont(int n, int64_t B, double sqrt_s, const double* p, const double* ang, const double* q,
                              bg_prec prec, double g_s, const uint8_t* accept, double* me2, void* workspace,
                              int64_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * bg_currents_co_mc -- colour sampling with colour-ordered amplitudes (the
 * colour-sampling variant of the colour-ordered algorithms, Sec. 4, with the
 * colour-flow decomposition of Eq. 2.19): per event one sampled colour flow
 * and helicity configuration; the flow amplitude is the sum, over the
 * (n-1)! orders (1, s_2, ..., s_n) whose chain of Kronecker deltas
 * delta(c_1, r_{s_2}) delta(c_{s_2}, r_{s_3}) ... delta(c_{s_n}, r_1) closes,
 * of the colour-ordered amplitudes A(1, s_2, ..., s_n) (Eqs. 2.20-2.22);
 *   me2 = 9^n * 2^n * g_s^(2n-4) * |A_flow|^2,
 * the same estimator as bg_currents_cd with BG_COL_FLOW (equal event by
 * event up to rounding).
 *   p       [4][n][B]    lab momenta (bg_momenta_rambo)
 *   hel     [n][B] int8  helicity labels +-1
 *   colors  [2n][B] int8 rows 2i and 2i+1 the pair (r_i, c_i) in 1..3
 *           (external colour matrix |r_i><c_i|)
 *   accept  [B] or NULL  events with accept == 0 get 0
 *   me2     [B] double   output, GeV^(8-2n)
 *   workspace, workspace_bytes: caller-owned device scratch of at least
 *           bg_comc_workspace_bytes(n, B, prec) bytes, 256-byte aligned (the
 *           events' momenta, polarisations, pair invariants and colour
 *           masks, the item offsets, partial sums); nothing needs to be
 *           zeroed.  About 1 KB per event at n = 12.
 * Every closing order of every event is one work item: the orders are
 * counted per event in closed form (the BEST theorem for the Eulerian
 * circuits of the flow's colour graph), and a persistent kernel evaluates
 * the items, so that an event with many orders spreads over the GPU.  The
 * work per event is the number of closing orders, (n-1)!/3^n on average and
 * up to (n-1)! for degenerate flows.  The sums run in a fixed order (equal
 * inputs give equal bits).  Events with a colour label outside 1..3 get 0
 * and set BG_EINVAL in the device status word.  Supported: 4 <= n <= 12.
 * Errors: BG_EINVAL, BG_ECUDA.
 * ------------------------------------------------------------------------- */
bg_status bg_comc_workspace_bytes(int n, int64_t B, bg_prec prec, int64_t* bytes);
bg_status bg_currents_co_mc(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel,
                            const int8_t* colors, const double* q, bg_prec prec, double g_s, const uint8_t* accept,
                            double* me2, void* workspace, int64_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * bg_currents_lc -- leading-colour |M|^2 (Sec. 4, the prefactor formula of
 * the leading-colour algorithms):
 *   me2 = g_s^(2n-4) N^(n-2) (N^2-1) sum over the (n-1)! orders
 *         (1, s_2, ..., s_n) of |A(1, s_2, ..., s_n)|^2   (N = 3),
 * times 2^n for sampled helicities (hel != NULL) or summed over all 2^n
 * polarisation configurations (hel == NULL).  Exact for n = 4, 5; an
 * O(1/N^2) approximation of the colour sum beyond.
 *   p       [4][n][B]    lab momenta (bg_momenta_rambo)
 *   hel     [n][B] int8 or NULL
 *   accept  [B] or NULL  events with accept == 0 get 0
 *   me2     [B] double   output, GeV^(8-2n)
 *   workspace, workspace_bytes: caller-owned device scratch of at least
 *           bg_lc_workspace_bytes(n, B, hel != NULL, prec) bytes, 256-byte
 *           aligned (relabelled inputs, one run's amplitudes, per-event
 *           sums); nothing needs to be zeroed.
 * Runs the colour-ordered recursion n-1 times (once per gluon placed last)
 * on `stream`.  Supported: 4 <= n <= 9.  Errors: BG_EINVAL, BG_ECUDA.
 * ------------------------------------------------------------------------- */
bg_status bg_lc_workspace_bytes(int n, int64_t B, int hel_sampled, bg_prec prec, int64_t* bytes);
bg_status bg_currents_lc(int n, int64_t B, double sqrt_s, const double* p, const int8_t* hel, const double* q,
                         bg_prec prec, double g_s, const uint8_t* accept, double* me2, void* workspace,
                         int64_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Mixed multiplicities: a batch whose events each have their own n in
 * n_min..n_max (Sec. 5 times every n from 4 to 12; a generator of events
 * with several jet multiplicities feeds such batches).  bg_mixed_create
 * allocates input, output and per-multiplicity buffers for up to max_batch
 * events and records the whole path as one CUDA graph: binning of the
 * events by n on the device, then one branch per multiplicity (concurrent
 * streams), each Rambo -> cut -> colour-ordered recursion + colour sum
 * (n <= n_co_max, Eqs. 2.16-2.22, sampled helicities) or colour-dressed
 * recursion with sampled colours (n > n_co_max, Eqs. 2.28-2.32), then a
 * scatter of |M|^2 back to the events' positions.  A branch handles its
 * events in chunks of at most cap_n events, cap_n chosen so that a chunk's
 * buffers stay within chunk_bytes (0: 8 GiB; at most 64 chunks).
 * bg_mixed_run replays the graph with one launch for B <= max_batch events.
 *   n_co_max: largest n on the colour-ordered path (<= 9; below n_min: all
 *             events on the colour-dressed path)
 *   cs_mode:  colour-sum arithmetic of the colour-ordered branches; the
 *             tensor-core mode applies to 6 <= n <= 9, smaller n use FP32
 *   color_mode: colour sampling of the colour-dressed branches
 *   autotune: run bg_autotune for every branch's recursion before the graph
 *             is recorded (the graph keeps the variants chosen then)
 * The paper has no single-launch counterpart: it runs one multiplicity at
 * a time.
 * ------------------------------------------------------------------------- */
typedef struct {
  int n_min, n_max;
  int64_t max_batch;
  double sqrt_s;
  double pt_min;
  double g_s;
  double q[4];
  bg_prec prec;
  bg_cs_mode cs_mode;
  bg_color_mode color_mode;
  int n_co_max;
  int64_t chunk_bytes;
  int autotune;       /* 1: bg_autotune each branch's recursion at creation */
} bg_mixed_desc;
typedef struct bg_mixed bg_mixed;
/* Errors: BG_EINVAL (desc), BG_ENOMEM, BG_ECUDA.  Synchronises the device. */
bg_status bg_mixed_create(const bg_mixed_desc* desc, bg_mixed** out);
void bg_mixed_destroy(bg_mixed* plan);
/* The plan-owned DEVICE buffers the graph reads and writes (any pointer may
 * be NULL):
 *   n_per_event [max_batch] int32               multiplicity of each event
 *   u           [max_batch][4(n_max-2)] double  Rambo uniforms; event e uses
 *                                               its first 4(n_e-2)
 *   hel         [n_max][max_batch] int8 (+-1)   sampled helicities, rows
 *                                               0..n_e-1
 *   colors      [2 n_max][max_batch] int8       sampled colours of the
 *                                               colour-dressed branches, as
 *                                               for bg_currents_cd (rows
 *                                               0..n_e-1 adjoint, 0..2n_e-1
 *                                               flow)
 *   me2         [max_batch] double              output, GeV^(8-2n_e) */
bg_status bg_mixed_buffers(bg_mixed* plan, int32_t** n_per_event, double** u, int8_t** hel, int8_t** colors,
                           double** me2);
int64_t bg_mixed_workspace_bytes(const bg_mixed* plan);
/* Runs the graph for the first B events of the buffers on `stream` (copies
 * B to the device, then one graph launch).  Events with n outside
 * n_min..n_max set BG_EINVAL in the device status word and keep their me2
 * entry unchanged.  Runs on one plan must be ordered (one stream): they
 * share its buffers. */
bg_status bg_mixed_run(bg_mixed* plan, int64_t B, void* stream);
/* counts[13]: events of each n in the last run (synchronises the device). */
bg_status bg_mixed_counts(bg_mixed* plan, int64_t* counts);
/* *kernels: the number of kernels one bg_mixed_run launches (the kernel
 * nodes of the plan's CUDA graph; its other nodes are memory copies and
 * sets).  Host only, no device work.  Errors: BG_EINVAL, BG_ECUDA. */
bg_status bg_mixed_kernel_nodes(const bg_mixed* plan, int64_t* kernels);

/* ---------------------------------------------------------------------------
 * Autotuning (no counterpart in the paper).  Each recursion has kernel
 * variants that compute the same sums in the same order -- bitwise identical
 * results -- and differ in how the work maps onto the GPU:
 *   BG_ALGO_CO (sampled helicities, n >= 6): 0 = one thread per ordering,
 *     1 = depth-first groups of six orderings sharing prefix currents in
 *     blocks of 256 threads, 2 = the same in blocks of 128, 3 = blocks of
 *     128 with registers capped for three blocks per SM, 4 and 5 = blocks
 *     of 64 with at most 200 and 184 registers per thread (defaults: 2 for
 *     n = 6, 7; 1 for n = 8, 9);
 *     helicity sums and n < 6 have one variant;
 *   BG_ALGO_CD: (threads per event, unrolling of the partition loop):
 *     n <= 9: 0 = (128, 1), 1 = (256, 1), 2 = (128, 2), 3 = (256, 2);
 *     n >= 10: 0 = (256, 1), 1 = (384, 1), 2 = (512, 1), 3 = (256, 2),
 *     4 = (384, 2); defaults 0 for n <= 8, 1 for n = 9, 2 for n >= 10.
 * bg_autotune times every variant of (algo, n, prec) on a synthetic probe
 * batch of probe_batch events (<= 0: a size chosen by n) on `stream`, stores
 * the fastest in a process-wide table for the current device and returns it
 * in *best (ms[v], if not NULL, receives the time of variant v; give it
 * bg_tune_num_variants entries).  It allocates and frees the probe buffers,
 * synchronises `stream`, and must not run during stream capture.  Calls that
 * launch a recursion (bg_currents_co, bg_currents_cd, bg_me2_batch, the
 * mixed graph at creation) use the table's entry for the current device.
 * bg_tune_set forces a variant (-1 restores the default); bg_tune_get reads
 * it (-1 = default).  bg_tune_save / bg_tune_load write and read the table
 * as text keyed by the device name (entries for other devices are ignored
 * on load).  Errors: BG_EINVAL, BG_ENOMEM, BG_ECUDA.
 * ------------------------------------------------------------------------- */
int bg_tune_num_variants(bg_algo algo, int n);
bg_status bg_autotune(bg_algo algo, int n, bg_prec prec, int64_t probe_batch, void* stream, int* best, float* ms);
bg_status bg_tune_set(bg_algo algo, int n, bg_prec prec, int variant);
bg_status bg_tune_get(bg_algo algo, int n, bg_prec prec, int* variant);
bg_status bg_tune_save(const char* path);
bg_status bg_tune_load(const char* path);

/* Device status word of the current device: 0 if no kernel has seen an
 * invalid label since the last reset, else a BG_* code.  Synchronises the
 * device.  bg_device_status_reset clears it. */
bg_status bg_device_status(int* status);
bg_status bg_device_status_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* BG_H */
