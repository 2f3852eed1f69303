// bg_oracle.cpp -- plain, slow, FP64 CPU oracle for the n-gluon Berends-Giele
// hot path of "Many-gluon tree amplitudes on modern GPUs" (Bothmann, Giele,
// Hoeche, Isaacson, Knobbe).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
// calls this file; only tests/, __graft_entry__.smoke() and the CPU-baseline
// leg of bench.py use it.  It shares no code, header, table or constant
// generator with the CUDA path.
//
// Every function follows the paper's definitions literally, one event at a
// time, with no blocking, fusion or reordering beyond what the equations say:
//   * Rambo flat phase space (Sec. 3 intro, the paper's cited generator)
//   * real polarisation vectors, Eq. (2.7) and the projector Eq. (2.2)
//   * colour-ordered Berends-Giele currents with V3/V4, Eqs. (2.20)-(2.22)
//   * the tensor-field form of the same recursion, Eqs. (2.23)-(2.26)
//   * the adjoint (DDM) colour matrix, Eq. (2.17), by explicit SU(3)
//     contraction of 8x8 matrices F^a_{bc} = Tr(T^a [T^b, T^c])
//   * the colour sum A^T C A, Eq. (2.16)
//   * colour-dressed currents, Eqs. (2.28)-(2.32)
//   * colour-flow sampling with colour-ordered amplitudes, Eq. (2.19)
//   * the leading-colour sum of Sec. 4
//   * continuous colour and helicity sampling for the colour-dressed
//     recursion (Sec. 2.1: colour polarisation vectors, polarisation angle)
// Equation numbers count the paper's numbered equations within Sec. 2.
//
// Conventions (the paper leaves these open; each reading is listed in the
// design notes):  metric (+,-,-,-); all momenta outgoing, k1 = -p1,
// k2 = -p2; couplings stripped (g = 1 inside the recursion, the factor
// g^(2n-4) multiplies |M|^2 at the end); generators normalised as
// Tr(T^a T^b) = delta^ab.
//
// Parity pins (tests/test_oracle_pins.py): 4-gluon closed form, Parke-Taylor
// MHV magnitudes, vanishing of all-plus / one-minus amplitudes, gauge
// invariance, cyclic / reflection / photon-decoupling identities, current
// conservation, tensor form == V4 form, linear == helicity polarisation sums,
// colour-dressed == colour-ordered x colour matrix by brute force over all
// colours at n = 4, 5, colour-matrix diagonal closed form and symmetry;
// colour-flow amplitude from colour-ordered amplitudes == colour-dressed
// amplitude for the same flow, and its average over all 9^n flows == the
// colour sum; leading-colour sum == full colour sum at n = 4, 5 (the
// subleading terms vanish there).

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

typedef std::complex<double> cplx;
const double kPi = 3.14159265358979323846;
const double kInvSqrt2 = 0.70710678118654752440;

// ---------------------------------------------------------------------------
// Forward-mode dual number with up to kMaxDir directions: used to pin the
// gradient of |M|^2 with respect to the Rambo uniforms exactly (to rounding).
// ---------------------------------------------------------------------------
const int kMaxDir = 40;
struct Dual {
  double v;
  double d[kMaxDir];
  Dual() : v(0) { std::memset(d, 0, sizeof d); }
  Dual(double x) : v(x) { std::memset(d, 0, sizeof d); }  // NOLINT
};
inline Dual operator+(const Dual& a, const Dual& b) { Dual r; r.v = a.v + b.v; for (int i = 0; i < kMaxDir; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
inline Dual operator-(const Dual& a, const Dual& b) { Dual r; r.v = a.v - b.v; for (int i = 0; i < kMaxDir; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
inline Dual operator-(const Dual& a) { Dual r; r.v = -a.v; for (int i = 0; i < kMaxDir; ++i) r.d[i] = -a.d[i]; return r; }
inline Dual operator*(const Dual& a, const Dual& b) { Dual r; r.v = a.v * b.v; for (int i = 0; i < kMaxDir; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
inline Dual operator/(const Dual& a, const Dual& b) { Dual r; r.v = a.v / b.v; for (int i = 0; i < kMaxDir; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v); return r; }
inline Dual& operator+=(Dual& a, const Dual& b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, const Dual& b) { a = a - b; return a; }
inline Dual sqrt(const Dual& a) { Dual r; r.v = std::sqrt(a.v); for (int i = 0; i < kMaxDir; ++i) r.d[i] = a.d[i] / (2.0 * r.v); return r; }
inline Dual log(const Dual& a) { Dual r; r.v = std::log(a.v); for (int i = 0; i < kMaxDir; ++i) r.d[i] = a.d[i] / a.v; return r; }
inline Dual cos(const Dual& a) { Dual r; r.v = std::cos(a.v); double s = -std::sin(a.v); for (int i = 0; i < kMaxDir; ++i) r.d[i] = s * a.d[i]; return r; }
inline Dual sin(const Dual& a) { Dual r; r.v = std::sin(a.v); double c = std::cos(a.v); for (int i = 0; i < kMaxDir; ++i) r.d[i] = c * a.d[i]; return r; }
inline double value(double x) { return x; }
inline double value(long double x) { return (double)x; }
inline double value(const Dual& x) { return x.v; }
using std::cos;
using std::log;
using std::sin;
using std::sqrt;

// ---------------------------------------------------------------------------
// Minkowski 4-vectors and antisymmetric rank-2 tensors, metric (+,-,-,-).
// Components are stored contravariant.
// ---------------------------------------------------------------------------
template <class T> struct Vec { T c[4]; };
template <class T> struct Ten { T c[4][4]; };  // antisymmetric tensor T^{mu nu}

const double kMetric[4] = {1.0, -1.0, -1.0, -1.0};

template <class T> Vec<T> vzero() { Vec<T> r; for (int m = 0; m < 4; ++m) r.c[m] = T(0.0); return r; }
template <class T> Ten<T> tzero() { Ten<T> r; for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) r.c[a][b] = T(0.0); return r; }
template <class T> T mdot(const Vec<T>& a, const Vec<T>& b) { return a.c[0] * b.c[0] - a.c[1] * b.c[1] - a.c[2] * b.c[2] - a.c[3] * b.c[3]; }
template <class T> Vec<T> vadd(const Vec<T>& a, const Vec<T>& b) { Vec<T> r; for (int m = 0; m < 4; ++m) r.c[m] = a.c[m] + b.c[m]; return r; }
template <class T> Vec<T> vsub(const Vec<T>& a, const Vec<T>& b) { Vec<T> r; for (int m = 0; m < 4; ++m) r.c[m] = a.c[m] - b.c[m]; return r; }
template <class T, class S> Vec<T> vscale(const S& s, const Vec<T>& a) { Vec<T> r; for (int m = 0; m < 4; ++m) r.c[m] = T(s) * a.c[m]; return r; }

// The colour-ordered three-gluon vertex of Eq. (2.21) contracted with two
// currents, with the factor i g/sqrt(2) and the propagator's -i taken out:
//   V3(p, q; X, Y) = (X.Y)(p - q) + ((2q + p).X) Y - ((2p + q).Y) X.
template <class T> Vec<T> V3(const Vec<T>& p, const Vec<T>& q, const Vec<T>& X, const Vec<T>& Y) {
  Vec<T> two_q_plus_p, two_p_plus_q, p_minus_q;
  for (int m = 0; m < 4; ++m) {
    two_q_plus_p.c[m] = T(2.0) * q.c[m] + p.c[m];
    two_p_plus_q.c[m] = T(2.0) * p.c[m] + q.c[m];
    p_minus_q.c[m] = p.c[m] - q.c[m];
  }
  T xy = mdot(X, Y), ax = mdot(two_q_plus_p, X), by = mdot(two_p_plus_q, Y);
  Vec<T> r;
  for (int m = 0; m < 4; ++m) r.c[m] = xy * p_minus_q.c[m] + ax * Y.c[m] - by * X.c[m];
  return r;
}

// The colour-ordered four-gluon vertex of Eq. (2.21) contracted with three
// currents, with the factor i g^2/2 and the propagator's -i taken out:
//   V4(X, Y, Z) = 2 (X.Z) Y - (X.Y) Z - (Y.Z) X.
template <class T> Vec<T> V4(const Vec<T>& X, const Vec<T>& Y, const Vec<T>& Z) {
  T xz = mdot(X, Z), xy = mdot(X, Y), yz = mdot(Y, Z);
  Vec<T> r;
  for (int m = 0; m < 4; ++m) r.c[m] = T(2.0) * xz * Y.c[m] - xy * Z.c[m] - yz * X.c[m];
  return r;
}

// Antisymmetric wedge (X ^ Y)^{ab} = X^a Y^b - X^b Y^a  (tensor current, Eq. 2.25).
template <class T> Ten<T> wedge(const Vec<T>& X, const Vec<T>& Y) {
  Ten<T> r;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) r.c[a][b] = X.c[a] * Y.c[b] - X.c[b] * Y.c[a];
  return r;
}
template <class T> void tacc(Ten<T>& acc, const T& s, const Ten<T>& t) {
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) acc.c[a][b] += s * t.c[a][b];
}
// (T X)^nu = T^{nu beta} X_beta   (tensor on the right of the gluon in Eq. 2.24)
template <class T> Vec<T> ten_vec(const Ten<T>& t, const Vec<T>& X) {
  Vec<T> r;
  for (int nu = 0; nu < 4; ++nu) {
    T s = T(0.0);
    for (int b = 0; b < 4; ++b) s += t.c[nu][b] * T(kMetric[b]) * X.c[b];
    r.c[nu] = s;
  }
  return r;
}
// (Y T)^nu = Y_alpha T^{alpha nu}   (tensor on the left of the gluon in Eq. 2.24)
template <class T> Vec<T> vec_ten(const Vec<T>& Y, const Ten<T>& t) {
  Vec<T> r;
  for (int nu = 0; nu < 4; ++nu) {
    T s = T(0.0);
    for (int a = 0; a < 4; ++a) s += Y.c[a] * T(kMetric[a]) * t.c[a][nu];
    r.c[nu] = s;
  }
  return r;
}

// ---------------------------------------------------------------------------
// Rambo (Kleiss, Stirling, Ellis), the phase-space generator the paper uses
// (Sec. 3 intro).  n_out massless momenta at fixed sqrt(s) from 4 n_out
// uniforms u[4i+0..3] per final-state gluon i.
// Output: lab-frame momenta p[n][4], incoming p1 = (E,0,0,E), p2 = (E,0,0,-E).
// ---------------------------------------------------------------------------
template <class T> void rambo(int n, double sqrt_s, const T* u, Vec<T>* p) {
  const int n_out = n - 2;
  std::vector<Vec<T>> q(n_out);
  for (int i = 0; i < n_out; ++i) {
    T c = T(2.0) * u[4 * i + 0] - T(1.0);
    T phi = T(2.0 * kPi) * u[4 * i + 1];
    T q0 = -log(u[4 * i + 2] * u[4 * i + 3]);
    T st = sqrt(T(1.0) - c * c);
    q[i].c[0] = q0;
    q[i].c[1] = q0 * st * cos(phi);
    q[i].c[2] = q0 * st * sin(phi);
    q[i].c[3] = q0 * c;
  }
  Vec<T> Q = vzero<T>();
  for (int i = 0; i < n_out; ++i) Q = vadd(Q, q[i]);
  T M = sqrt(mdot(Q, Q));
  T b[3] = {-Q.c[1] / M, -Q.c[2] / M, -Q.c[3] / M};
  T x = T(sqrt_s) / M;
  T gamma = Q.c[0] / M;
  T a = T(1.0) / (T(1.0) + gamma);
  const double E = 0.5 * sqrt_s;
  p[0].c[0] = T(E); p[0].c[1] = T(0.0); p[0].c[2] = T(0.0); p[0].c[3] = T(E);
  p[1].c[0] = T(E); p[1].c[1] = T(0.0); p[1].c[2] = T(0.0); p[1].c[3] = T(-E);
  for (int i = 0; i < n_out; ++i) {
    T bq = b[0] * q[i].c[1] + b[1] * q[i].c[2] + b[2] * q[i].c[3];
    p[2 + i].c[0] = x * (gamma * q[i].c[0] + bq);
    for (int j = 0; j < 3; ++j) p[2 + i].c[1 + j] = x * (q[i].c[1 + j] + b[j] * q[i].c[0] + a * bq * b[j]);
  }
}

// All-outgoing convention: k1 = -p1, k2 = -p2, k_i = p_i (sum k = 0).
template <class T> void outgoing(int n, const Vec<T>* p, Vec<T>* k) {
  for (int i = 0; i < n; ++i) k[i] = (i < 2) ? vscale(T(-1.0), p[i]) : p[i];
}

// ---------------------------------------------------------------------------
// Real polarisation vectors e1, e2 in the light-cone gauge of Eq. (2.2):
// e.e = -1, e.k = 0, e.q = 0, so that sum_lambda e e = -g + (kq + qk)/(k.q).
// Gauge frame: for the reference direction n = q_vec/|q_vec| take the two
// unit vectors a, b orthogonal to n obtained by rotating x^, y^ with the
// rotation that maps z^ to n (for n_z < 0: a(-n), -b(-n)).  Then
//   e1 = A - (A.k / q.k) q,   e2 = B - (B.k / q.k) q,  A = (0,a), B = (0,b).
// If k is parallel to q (|k.q| <= 1e-9 |k0| q0) the reference vector is
// replaced by (q0, -q_vec).
// ---------------------------------------------------------------------------
void gauge_pair(const double* nvec, double* a, double* b) {
  double nx = nvec[0], ny = nvec[1], nz = nvec[2];
  double sgn = 1.0;
  if (nz < 0.0) { nx = -nx; ny = -ny; nz = -nz; sgn = -1.0; }
  double h = 1.0 / (1.0 + nz);
  a[0] = 1.0 - nx * nx * h; a[1] = -nx * ny * h; a[2] = -nx;
  b[0] = -nx * ny * h;      b[1] = 1.0 - ny * ny * h; b[2] = -ny;
  for (int j = 0; j < 3; ++j) b[j] *= sgn;
}

template <class T> void polarisations(const Vec<T>& k, const double* q_in, Vec<T>* e1, Vec<T>* e2) {
  double q[4] = {q_in[0], q_in[1], q_in[2], q_in[3]};
  double kq = value(k.c[0]) * q[0] - value(k.c[1]) * q[1] - value(k.c[2]) * q[2] - value(k.c[3]) * q[3];
  if (std::fabs(kq) <= 1e-9 * std::fabs(value(k.c[0])) * q[0]) { q[1] = -q[1]; q[2] = -q[2]; q[3] = -q[3]; }
  double qn = std::sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double nvec[3] = {q[1] / qn, q[2] / qn, q[3] / qn};
  double a[3], b[3];
  gauge_pair(nvec, a, b);
  Vec<T> Q, A, B;
  for (int m = 0; m < 4; ++m) Q.c[m] = T(q[m]);
  A.c[0] = T(0.0); B.c[0] = T(0.0);
  for (int j = 0; j < 3; ++j) { A.c[1 + j] = T(a[j]); B.c[1 + j] = T(b[j]); }
  T qk = mdot(Q, k);
  T ca = mdot(A, k) / qk, cb = mdot(B, k) / qk;
  for (int m = 0; m < 4; ++m) {
    e1->c[m] = A.c[m] - ca * Q.c[m];
    e2->c[m] = B.c[m] - cb * Q.c[m];
  }
}

// ---------------------------------------------------------------------------
// Colour-ordered Berends-Giele recursion, Eqs. (2.20) and (2.22).
// `ord` lists the n gluon labels in colour order; ord[n-1] is the leg whose
// current is put on shell.  eps[label] is that gluon's external current.
//   J(i..j) = 1/P(i..j)^2 [ sum_s (1/sqrt2) V3(P(i..s), P(s+1..j); J(i..s), J(s+1..j))
//                         + sum_{s<t} (1/2) V4(J(i..s), J(s+1..t), J(t+1..j)) ]
//   A = eps_n . [bracket for J(1..n-1)]     (the P^2 of Eq. 2.22 amputates the
//                                            propagator; P(1..n-1)^2 = 0)
// With tensor_form = 1 the V4 terms are replaced by the auxiliary
// antisymmetric tensor field of Eqs. (2.23)-(2.26):
//   J^{ab}(i..j) = (1/sqrt2) sum_s J(i..s) ^ J(s+1..j),
//   bracket += (1/sqrt2) [ J^{.b}(s+1..j) J_b(i..s) + J_a(s+1..j) J^{a.}(i..s) ].
// Returns the current table through J_out (segment [i][j], may be NULL).
// ---------------------------------------------------------------------------
template <class T>
T amp_co(int n, const Vec<T>* k, const Vec<T>* eps, const int* ord, int tensor_form,
         std::vector<Vec<T>>* J_out = nullptr, std::vector<Vec<T>>* P_out = nullptr) {
  const int m = n - 1;  // legs in the off-shell current
  std::vector<Vec<T>> J(m * m), P(m * m);
  std::vector<Ten<T>> Tt(tensor_form ? m * m : 0);
  for (int i = 0; i < m; ++i) {
    J[i * m + i] = eps[ord[i]];
    P[i * m + i] = k[ord[i]];
    if (tensor_form) Tt[i * m + i] = tzero<T>();
  }
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) P[i * m + j] = vadd(P[i * m + j - 1], k[ord[j]]);
  T amp = T(0.0);
  for (int len = 2; len <= m; ++len) {
    for (int i = 0; i + len - 1 < m; ++i) {
      const int j = i + len - 1;
      Vec<T> br = vzero<T>();
      for (int s = i; s < j; ++s)
        br = vadd(br, vscale(T(kInvSqrt2), V3(P[i * m + s], P[(s + 1) * m + j], J[i * m + s], J[(s + 1) * m + j])));
      if (!tensor_form) {
        for (int s = i; s < j; ++s)
          for (int t = s + 1; t < j; ++t)
            br = vadd(br, vscale(T(0.5), V4(J[i * m + s], J[(s + 1) * m + t], J[(t + 1) * m + j])));
      } else {
        Ten<T> tc = tzero<T>();
        for (int s = i; s < j; ++s) {
          br = vadd(br, vscale(T(kInvSqrt2), ten_vec(Tt[(s + 1) * m + j], J[i * m + s])));
          br = vadd(br, vscale(T(kInvSqrt2), vec_ten(J[(s + 1) * m + j], Tt[i * m + s])));
          tacc(tc, T(kInvSqrt2), wedge(J[i * m + s], J[(s + 1) * m + j]));
        }
        Tt[i * m + j] = tc;
      }
      if (len < m) {
        J[i * m + j] = vscale(T(1.0) / mdot(P[i * m + j], P[i * m + j]), br);
      } else {
        J[i * m + j] = br;  // amputated top current (bracket)
        amp = mdot(eps[ord[n - 1]], br);
      }
    }
  }
  if (J_out) *J_out = J;
  if (P_out) *P_out = P;
  return amp;
}

// ---------------------------------------------------------------------------
// Orderings sigma in S_{n-2} of the labels {2..n-1} (0-based {1..n-2}),
// enumerated in lexicographic order.  Ordering index r <-> permutation via
// the factorial number system.
// ---------------------------------------------------------------------------
long long factorial(int m) { long long f = 1; for (int i = 2; i <= m; ++i) f *= i; return f; }

void ordering_from_index(int n, long long r, int* sigma /* n-2 labels, 0-based in 1..n-2 */) {
  const int m = n - 2;
  std::vector<int> pool(m);
  for (int i = 0; i < m; ++i) pool[i] = i + 1;
  for (int pos = 0; pos < m; ++pos) {
    long long f = factorial(m - 1 - pos);
    long long d = r / f;
    r %= f;
    sigma[pos] = pool[d];
    pool.erase(pool.begin() + d);
  }
}

// ---------------------------------------------------------------------------
// SU(3) generators with Tr(T^a T^b) = delta^ab (T = lambda / sqrt 2), the
// normalisation the paper uses for Eq. (2.27).
// ---------------------------------------------------------------------------
void gell_mann(cplx lam[8][3][3]) {
  for (int a = 0; a < 8; ++a)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) lam[a][i][j] = 0.0;
  const cplx I(0.0, 1.0);
  lam[0][0][1] = 1.0; lam[0][1][0] = 1.0;
  lam[1][0][1] = -I;  lam[1][1][0] = I;
  lam[2][0][0] = 1.0; lam[2][1][1] = -1.0;
  lam[3][0][2] = 1.0; lam[3][2][0] = 1.0;
  lam[4][0][2] = -I;  lam[4][2][0] = I;
  lam[5][1][2] = 1.0; lam[5][2][1] = 1.0;
  lam[6][1][2] = -I;  lam[6][2][1] = I;
  const double r3 = 1.0 / std::sqrt(3.0);
  lam[7][0][0] = r3; lam[7][1][1] = r3; lam[7][2][2] = -2.0 * r3;
}

void generators(cplx T[8][3][3]) {
  gell_mann(T);
  for (int a = 0; a < 8; ++a)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) T[a][i][j] *= kInvSqrt2;
}

// F^a_{bc} = Tr(T^a [T^b, T^c]), the adjoint generators of Eq. (2.15)
// (= i f^abc in the paper's normalisation, Eq. 2.27).
void adjoint_F(cplx F[8][8][8]) {
  cplx T[8][3][3];
  generators(T);
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b)
      for (int c = 0; c < 8; ++c) {
        cplx tr = 0.0;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            for (int l = 0; l < 3; ++l)
              tr += T[a][i][j] * (T[b][j][l] * T[c][l][i] - T[c][j][l] * T[b][l][i]);
        F[a][b][c] = tr;
      }
}

// Chain tensor G[a1][b1..bk][an] = (F^{b1} ... F^{bk})_{a1 an}, k = n-2,
// stored with a1 as the most significant base-8 digit and an the least.
void chain_tensor(int n, std::vector<cplx>& G) {
  static cplx F[8][8][8];
  adjoint_F(F);
  const int k = n - 2;
  long long inner = 1;
  for (int i = 0; i < k; ++i) inner *= 8;
  G.assign((size_t)(64 * inner), cplx(0.0));
  std::vector<int> b(k);
  for (long long bi = 0; bi < inner; ++bi) {
    long long r = bi;
    for (int i = k - 1; i >= 0; --i) { b[i] = (int)(r % 8); r /= 8; }
    // M = F^{b1} ... F^{bk}
    cplx M[8][8], Tm[8][8];
    for (int x = 0; x < 8; ++x)
      for (int y = 0; y < 8; ++y) M[x][y] = F[b[0]][x][y];
    for (int i = 1; i < k; ++i) {
      for (int x = 0; x < 8; ++x)
        for (int y = 0; y < 8; ++y) {
          cplx s = 0.0;
          for (int z = 0; z < 8; ++z) s += M[x][z] * F[b[i]][z][y];
          Tm[x][y] = s;
        }
      std::memcpy(M, Tm, sizeof M);
    }
    for (int x = 0; x < 8; ++x)
      for (int y = 0; y < 8; ++y) G[((size_t)x * inner + bi) * 8 + y] = M[x][y];
  }
}

// Colour coefficient of Eq. (2.17) for a pair of orderings, by the explicit
// sum over all adjoint colours a1..an.  sigma, tau: n-2 labels in 1..n-2
// (0-based gluon labels 2..n-1).
double colour_coefficient(int n, const std::vector<cplx>& G, const int* sigma, const int* tau) {
  const int k = n - 2;
  long long inner = 1;
  for (int i = 0; i < k; ++i) inner *= 8;
  std::vector<int> a(n);
  double sum = 0.0;
  for (long long x = 0; x < 8; ++x)
    for (long long y = 0; y < 8; ++y)
      for (long long ai = 0; ai < inner; ++ai) {
        long long r = ai;
        for (int i = k; i >= 1; --i) { a[i] = (int)(r % 8); r /= 8; }  // a[label] for labels 1..n-2
        long long is = 0, it = 0;
        for (int i = 0; i < k; ++i) { is = is * 8 + a[sigma[i]]; it = it * 8 + a[tau[i]]; }
        cplx v = G[((size_t)x * inner + is) * 8 + y] * std::conj(G[((size_t)x * inner + it) * 8 + y]);
        sum += v.real();
      }
  return sum;
}

// ---------------------------------------------------------------------------
// Colour-dressed currents in the colour-flow basis, Eqs. (2.28)-(2.32).
// Currents are 3x3 colour matrices of Lorentz vectors (gluon) and of
// antisymmetric tensors (tensor pseudo-particle), one per subset S of the
// first n-1 gluons (bitmask).  The sum over partitions with both colour
// orders of the vertex (2.30) is the sum over ordered partitions (S1, S2)
// with the colour product J(S1) J(S2); the gluon-tensor terms run over
// ordered partitions as well.
// External colour matrix of gluon i: Ecol[i] (3x3, real).
// ---------------------------------------------------------------------------
template <class T> struct CMat { Vec<T> e[3][3]; };
template <class T> struct CTen { Ten<T> e[3][3]; };

template <class T>
T amp_cd(int n, const Vec<T>* k, const Vec<T>* eps, const double (*Ecol)[3][3],
         std::vector<CMat<T>>* J_out = nullptr) {
  const int m = n - 1;
  const int full = (1 << m) - 1;
  std::vector<CMat<T>> J(full + 1);
  std::vector<CTen<T>> Tt(full + 1);
  std::vector<Vec<T>> P(full + 1);
  for (int S = 1; S <= full; ++S) {
    P[S] = vzero<T>();
    for (int i = 0; i < m; ++i)
      if (S >> i & 1) P[S] = vadd(P[S], k[i]);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) { J[S].e[r][c] = vzero<T>(); Tt[S].e[r][c] = tzero<T>(); }
  }
  for (int i = 0; i < m; ++i)
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) J[1 << i].e[r][c] = vscale(T(Ecol[i][r][c]), eps[i]);
  // subsets in order of increasing size
  std::vector<int> order;
  for (int sz = 2; sz <= m; ++sz)
    for (int S = 1; S <= full; ++S)
      if (__builtin_popcount(S) == sz) order.push_back(S);
  T amp = T(0.0);
  for (int S : order) {
    CMat<T> br;
    CTen<T> tc;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) { br.e[r][c] = vzero<T>(); tc.e[r][c] = tzero<T>(); }
    for (int S1 = (S - 1) & S; S1 > 0; S1 = (S1 - 1) & S) {  // ordered partitions (S1, S2)
      const int S2 = S ^ S1;
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
          for (int l = 0; l < 3; ++l) {
            const Vec<T>& X = J[S1].e[r][l];
            const Vec<T>& Y = J[S2].e[l][c];
            br.e[r][c] = vadd(br.e[r][c], vscale(T(kInvSqrt2), V3(P[S1], P[S2], X, Y)));
            br.e[r][c] = vadd(br.e[r][c], vscale(T(kInvSqrt2), ten_vec(Tt[S2].e[l][c], X)));
            br.e[r][c] = vadd(br.e[r][c], vscale(T(kInvSqrt2), vec_ten(Y, Tt[S1].e[r][l])));
            tacc(tc.e[r][c], T(kInvSqrt2), wedge(X, Y));
          }
    }
    if (S != full) {
      T inv = T(1.0) / mdot(P[S], P[S]);
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) J[S].e[r][c] = vscale(inv, br.e[r][c]);
      Tt[S] = tc;
    } else {
      // amplitude = Tr(E_n . (eps_n . bracket))
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) amp += T(Ecol[n - 1][c][r]) * mdot(eps[n - 1], br.e[r][c]);
      J[S] = br;
    }
  }
  if (J_out) *J_out = J;
  return amp;
}

// Real external colour matrices.  Adjoint index a in 1..8: T^a, with the
// imaginary generators (a = 2, 5, 7) replaced by the real antisymmetric
// -i T^a (|amplitude| is unchanged since the amplitude is multilinear in
// the external colour matrices).  Colour flow (r, c) in {1,2,3}^2: |r><c|.
void colour_matrix_adjoint(int a, double E[3][3]) {
  cplx T[8][3][3];
  generators(T);
  const bool imag = (a == 2 || a == 5 || a == 7);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx v = T[a - 1][i][j];
      E[i][j] = imag ? (v * cplx(0.0, -1.0)).real() : v.real();
    }
}
void colour_matrix_flow(int r, int c, double E[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) E[i][j] = (i == r - 1 && j == c - 1) ? 1.0 : 0.0;
}

template <class T> void load_vecs(int n, const double* src, Vec<T>* dst) {
  for (int i = 0; i < n; ++i)
    for (int m = 0; m < 4; ++m) dst[i].c[m] = T(src[4 * i + m]);
}
template <class T> void store_vecs(int n, const Vec<T>* src, double* dst) {
  for (int i = 0; i < n; ++i)
    for (int m = 0; m < 4; ++m) dst[4 * i + m] = value(src[i].c[m]);
}

// External polarisation of gluon i for helicity label lam (+1 -> e1, -1 -> e2).
template <class T> void pols_for(int n, const Vec<T>* k, const double* q, const int8_t* hel, Vec<T>* eps) {
  for (int i = 0; i < n; ++i) {
    Vec<T> e1, e2;
    polarisations(k[i], q, &e1, &e2);
    eps[i] = (hel[i] > 0) ? e1 : e2;
  }
}

// Colour-ordered amplitudes A(1, sigma, n) for all (n-2)! orderings
// (lexicographic), for one event and one helicity configuration.
template <class T> void all_amps(int n, const Vec<T>* k, const Vec<T>* eps, T* amps, int tensor_form = 0) {
  const long long nord = factorial(n - 2);
  std::vector<int> sigma(n - 2), ord(n);
  for (long long r = 0; r < nord; ++r) {
    ordering_from_index(n, r, sigma.data());
    ord[0] = 0;
    for (int i = 0; i < n - 2; ++i) ord[1 + i] = sigma[i];
    ord[n - 1] = n - 1;
    amps[r] = amp_co(n, k, eps, ord.data(), tensor_form);
  }
}

// Colour sum of Eq. (2.16) for one helicity configuration: sum C A A.
template <class T> T colour_sum(int nord, const double* C, const T* A) {
  T s = T(0.0);
  for (int a = 0; a < nord; ++a) {
    T row = T(0.0);
    for (int b = 0; b < nord; ++b) row += T(C[(size_t)a * nord + b]) * A[b];
    s += A[a] * row;
  }
  return s;
}

// |M|^2 for one event from its uniforms: Rambo -> k -> polarisations ->
// all orderings -> colour sum, times g^(2n-4) (and 2^n if helicities are
// sampled, hel != NULL).  Returns 0 for events failing the pT cut.
template <class T>
T me2_co_event(int n, double sqrt_s, const T* u, const double* q, const double* C, const int8_t* hel,
               double g, double pt_min, int tensor_form = 0) {
  std::vector<Vec<T>> p(n), k(n), eps(n);
  rambo(n, sqrt_s, u, p.data());
  for (int i = 2; i < n; ++i)
    if (std::sqrt(value(p[i].c[1]) * value(p[i].c[1]) + value(p[i].c[2]) * value(p[i].c[2])) <= pt_min) return T(0.0);
  outgoing(n, p.data(), k.data());
  const int nord = (int)factorial(n - 2);
  std::vector<T> A(nord);
  T me2 = T(0.0);
  std::vector<int8_t> h(n);
  const int nconf = hel ? 1 : (1 << n);
  for (int conf = 0; conf < nconf; ++conf) {
    for (int i = 0; i < n; ++i) h[i] = hel ? hel[i] : (((conf >> i) & 1) ? -1 : 1);
    pols_for(n, k.data(), q, h.data(), eps.data());
    all_amps(n, k.data(), eps.data(), A.data(), tensor_form);
    me2 += colour_sum(nord, C, A.data());
  }
  double fac = std::pow(g, 2 * n - 4) * (hel ? std::pow(2.0, n) : 1.0);
  return T(fac) * me2;
}

// Batch colour-dressed |M|^2 estimator with sampled colours and helicities:
// mode 0 adjoint (colors[B][n] in 1..8, weight 8^n), mode 1 colour flow
// (colors[B][2n] pairs in 1..3, weight 9^n); helicity weight 2^n; times
// g^(2n-4).  Events failing the pT cut get 0.  T = double, or long double
// for the extended-precision reference.
template <class T>
void me2_cd_batch(int n, long long B, double sqrt_s, const double* u, const double* q, const int8_t* hel,
                  const int8_t* colors, int mode, double g, double pt_min, double* me2, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  std::vector<std::thread> th;
  const int d = 4 * (n - 2);
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t]() {
      std::vector<Vec<T>> p(n), k(n), eps(n);
      std::vector<T> ul(d);
      std::vector<double> E(n * 9);
      for (long long e = t; e < B; e += nthreads) {
        for (int i = 0; i < d; ++i) ul[i] = T(u[e * d + i]);
        rambo(n, sqrt_s, ul.data(), p.data());
        bool cut = false;
        for (int i = 2; i < n; ++i)
          if (std::sqrt(value(p[i].c[1]) * value(p[i].c[1]) + value(p[i].c[2]) * value(p[i].c[2])) <= pt_min)
            cut = true;
        if (cut) { me2[e] = 0.0; continue; }
        outgoing(n, p.data(), k.data());
        pols_for(n, k.data(), q, hel + e * n, eps.data());
        for (int i = 0; i < n; ++i) {
          double M[3][3];
          if (mode == 0) colour_matrix_adjoint(colors[e * n + i], M);
          else colour_matrix_flow(colors[e * 2 * n + 2 * i], colors[e * 2 * n + 2 * i + 1], M);
          for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) E[i * 9 + r * 3 + c] = M[r][c];
        }
        T a = amp_cd(n, k.data(), eps.data(), reinterpret_cast<const double(*)[3][3]>(E.data()));
        double w = std::pow(mode == 0 ? 8.0 : 9.0, n) * std::pow(2.0, n) * std::pow(g, 2 * n - 4);
        me2[e] = (double)(T(w) * a * a);
      }
    });
  for (auto& x : th) x.join();
}

// Common start of the per-event sampled evaluations below: Rambo, the pT
// cut, all-outgoing momenta and the sampled polarisations.  Returns false
// for events failing the cut.
template <class T>
bool event_setup(int n, double sqrt_s, const T* u, const double* q, const int8_t* hel, double pt_min,
                 Vec<T>* k, Vec<T>* eps) {
  std::vector<Vec<T>> p(n);
  rambo(n, sqrt_s, u, p.data());
  for (int i = 2; i < n; ++i)
    if (std::sqrt(value(p[i].c[1]) * value(p[i].c[1]) + value(p[i].c[2]) * value(p[i].c[2])) <= pt_min)
      return false;
  outgoing(n, p.data(), k);
  pols_for(n, k, q, hel, eps);
  return true;
}

// Colour-flow amplitude of Eq. (2.19) for one sampled flow, from the
// colour-ordered partial amplitudes: the sum over the (n-1)! orders
// (1, s_2, ..., s_n) of the product of Kronecker deltas around the cycle
// times A(1, s_2, ..., s_n).  Gluon i carries the flow pair (r_i, c_i), its
// colour matrix is |r_i><c_i|, so the trace of the ordered product is
// delta(c_1, r_{s_2}) delta(c_{s_2}, r_{s_3}) ... delta(c_{s_n}, r_1).
// Orders whose delta product vanishes are skipped (their term is zero).
template <class T>
T amp_colour_flow(int n, const Vec<T>* k, const Vec<T>* eps, const int8_t* flow) {
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  T a = T(0.0);
  do {
    bool on = true;
    for (int t = 0; t < n && on; ++t) {
      const int from = ord[t], to = ord[(t + 1) % n];
      on = flow[2 * from + 1] == flow[2 * to];
    }
    if (on) a += amp_co(n, k, eps, ord.data(), 0);
  } while (std::next_permutation(ord.begin() + 1, ord.end()));
  return a;
}

// Leading-colour sum of Sec. 4 (the prefactor formula for the leading
// colour algorithms): N^(n-2) (N^2 - 1) sum over the (n-1)! orders
// (1, s_2, ..., s_n) of |A(1, s_2, ..., s_n)|^2, N = 3.
template <class T>
T leading_colour_sum(int n, const Vec<T>* k, const Vec<T>* eps) {
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  T s = T(0.0);
  do {
    const T a = amp_co(n, k, eps, ord.data(), 0);
    s += a * a;
  } while (std::next_permutation(ord.begin() + 1, ord.end()));
  return T(std::pow(3.0, n - 2) * 8.0) * s;
}

// Batch |M|^2 estimator with sampled colour flows evaluated from
// colour-ordered amplitudes (the colour-sampling variant of Sec. 4, with the
// colour-flow decomposition of Eq. 2.19): colors[B][2n] flow pairs
// (r_i, c_i) in 1..3, hel[B][n]; me2 = 9^n 2^n g^(2n-4) |A_flow|^2.  Events
// failing the pT cut get 0.  T = double, or long double for the
// extended-precision reference.
template <class T>
void me2_co_mc_batch(int n, long long B, double sqrt_s, const double* u, const double* q, const int8_t* hel,
                     const int8_t* colors, double g, double pt_min, double* me2, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  std::vector<std::thread> th;
  const int d = 4 * (n - 2);
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t]() {
      std::vector<Vec<T>> k(n), eps(n);
      std::vector<T> ul(d);
      for (long long e = t; e < B; e += nthreads) {
        for (int i = 0; i < d; ++i) ul[i] = T(u[e * d + i]);
        if (!event_setup(n, sqrt_s, ul.data(), q, hel + e * n, pt_min, k.data(), eps.data())) {
          me2[e] = 0.0;
          continue;
        }
        const T a = amp_colour_flow(n, k.data(), eps.data(), colors + e * 2 * n);
        me2[e] = (double)(T(std::pow(9.0, n) * std::pow(2.0, n) * std::pow(g, 2 * n - 4)) * a * a);
      }
    });
  for (auto& x : th) x.join();
}

// Continuous colour and helicity sampling (Sec. 2.1): per gluon two real unit
// colour vectors eta(theta, phi), eta_bar(theta_bar, phi_bar) in the angle
// form of the paper, the gluon colour polarisation eta^a = eta_i T^a_ij
// eta_bar_j (Eq. of the gluon colour polarisation), and the polarisation
// vector e(phi_h) = cos(phi_h) e1 + sin(phi_h) e2.  The external colour matrix
// of the colour-dressed recursion is sum_a eta^a T^a, built here from the
// Gell-Mann generators (complex arithmetic; the result is real).
// ang[5]: cos(theta), phi, cos(theta_bar), phi_bar, phi_h.
void continuous_external(const double* ang, double E[3][3]) {
  cplx T[8][3][3];
  generators(T);
  double eta[3], etab[3];
  for (int v = 0; v < 2; ++v) {
    const double ct = ang[2 * v], ph = ang[2 * v + 1];
    const double st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
    double* x = v ? etab : eta;
    x[0] = ct;
    x[1] = st * std::cos(ph);
    x[2] = st * std::sin(ph);
  }
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      cplx acc = 0.0;
      for (int a = 0; a < 8; ++a) {
        cplx ea = 0.0;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) ea += eta[i] * T[a][i][j] * etab[j];
        acc += ea * T[a][k][l];
      }
      E[k][l] = acc.real();
    }
}

// Batch |M|^2 estimator with continuous colour and helicity sampling:
// ang[B][5n] (per gluon the five angles of continuous_external); weight per
// gluon N_c^2 = 9 for the two colour spheres (measure N_c / 4 pi each) and 2
// for the polarisation angle (the average over phi_h of e e is half the
// polarisation sum); times g^(2n-4).  Events failing the pT cut get 0.
template <class T>
void me2_cd_cont_batch(int n, long long B, double sqrt_s, const double* u, const double* q, const double* ang,
                       double g, double pt_min, double* me2, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  std::vector<std::thread> th;
  const int d = 4 * (n - 2);
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t]() {
      std::vector<Vec<T>> p(n), k(n), eps(n);
      std::vector<T> ul(d);
      std::vector<double> E(n * 9);
      for (long long e = t; e < B; e += nthreads) {
        for (int i = 0; i < d; ++i) ul[i] = T(u[e * d + i]);
        rambo(n, sqrt_s, ul.data(), p.data());
        bool cut = false;
        for (int i = 2; i < n; ++i)
          if (std::sqrt(value(p[i].c[1]) * value(p[i].c[1]) + value(p[i].c[2]) * value(p[i].c[2])) <= pt_min)
            cut = true;
        if (cut) { me2[e] = 0.0; continue; }
        outgoing(n, p.data(), k.data());
        for (int i = 0; i < n; ++i) {
          const double* a = ang + (e * n + i) * 5;
          Vec<T> e1, e2;
          polarisations(k[i], q, &e1, &e2);
          const T c = T(std::cos(a[4])), sn = T(std::sin(a[4]));
          for (int m = 0; m < 4; ++m) eps[i].c[m] = c * e1.c[m] + sn * e2.c[m];
          double M[3][3];
          continuous_external(a, M);
          for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) E[i * 9 + r * 3 + cc] = M[r][cc];
        }
        T a = amp_cd(n, k.data(), eps.data(), reinterpret_cast<const double(*)[3][3]>(E.data()));
        const double w = std::pow(9.0, n) * std::pow(2.0, n) * std::pow(g, 2 * n - 4);
        me2[e] = (double)(T(w) * a * a);
      }
    });
  for (auto& x : th) x.join();
}

}  // namespace

// ===========================================================================
// C ABI of the oracle (called from oracle/oracle.py through ctypes).
// All arrays are host arrays in the layouts stated; FP64 throughout.
// ===========================================================================
extern "C" {

// Rambo for one event: u[4(n-2)] -> lab momenta p[n][4].
void or_rambo(int n, double sqrt_s, const double* u, double* p) {
  std::vector<Vec<double>> pv(n);
  rambo(n, sqrt_s, u, pv.data());
  store_vecs(n, pv.data(), p);
}

// Polarisation pair for one momentum k[4] and reference q[4].
void or_polarisations(const double* k, const double* q, double* e1, double* e2) {
  Vec<double> kv, a, b;
  load_vecs(1, k, &kv);
  polarisations(kv, q, &a, &b);
  store_vecs(1, &a, e1);
  store_vecs(1, &b, e2);
}

// Colour-ordered amplitude for an arbitrary colour order of all n gluons.
// k[n][4] outgoing momenta, eps[n][4] external currents (real), ord[n]
// 0-based labels (ord[n-1] is put on shell).  tensor_form selects Eq. (2.24).
double or_amp_co(int n, const double* k, const double* eps, const int* ord, int tensor_form) {
  std::vector<Vec<double>> kv(n), ev(n);
  load_vecs(n, k, kv.data());
  load_vecs(n, eps, ev.data());
  return amp_co(n, kv.data(), ev.data(), ord, tensor_form);
}

// Same with complex external currents (eps_re, eps_im), for helicity
// amplitudes (Parke-Taylor pins).  Result written to out[2] = (re, im).
void or_amp_co_cplx(int n, const double* k, const double* eps_re, const double* eps_im, const int* ord,
                    int tensor_form, double* out) {
  std::vector<Vec<cplx>> kv(n), ev(n);
  for (int i = 0; i < n; ++i)
    for (int m = 0; m < 4; ++m) {
      kv[i].c[m] = cplx(k[4 * i + m], 0.0);
      ev[i].c[m] = cplx(eps_re[4 * i + m], eps_im[4 * i + m]);
    }
  cplx a = amp_co(n, kv.data(), ev.data(), ord, tensor_form);
  out[0] = a.real();
  out[1] = a.imag();
}

// Off-shell current table of one colour order: J[i][j] (segment i..j of the
// first n-1 legs, 0-based, i <= j), written as J[(i*(n-1)+j)*4 + mu]; also
// the segment momenta P in the same layout.  Segment [0][n-2] holds the
// amputated bracket.
void or_currents_co(int n, const double* k, const double* eps, const int* ord, int tensor_form, double* J,
                    double* P) {
  std::vector<Vec<double>> kv(n), ev(n), Jt, Pt;
  load_vecs(n, k, kv.data());
  load_vecs(n, eps, ev.data());
  amp_co(n, kv.data(), ev.data(), ord, tensor_form, &Jt, &Pt);
  const int m = n - 1;
  for (int i = 0; i < m; ++i)
    for (int j = i; j < m; ++j)
      for (int mu = 0; mu < 4; ++mu) {
        J[(i * m + j) * 4 + mu] = Jt[i * m + j].c[mu];
        P[(i * m + j) * 4 + mu] = Pt[i * m + j].c[mu];
      }
}

// Ordering index -> labels (n-2 entries, 0-based labels 1..n-2).
void or_ordering(int n, long long r, int* sigma) { ordering_from_index(n, r, sigma); }

// All (n-2)! amplitudes A(1, sigma, n) for one event and helicity config.
void or_amps_all(int n, const double* k, const double* eps, double* amps) {
  std::vector<Vec<double>> kv(n), ev(n);
  load_vecs(n, k, kv.data());
  load_vecs(n, eps, ev.data());
  all_amps(n, kv.data(), ev.data(), amps);
}

// Adjoint generators F[a][b][c] = Tr(T^a [T^b, T^c]) as (re, im) pairs.
void or_adjoint_generators(double* F) {
  static cplx Fc[8][8][8];
  adjoint_F(Fc);
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b)
      for (int c = 0; c < 8; ++c) {
        F[((a * 8 + b) * 8 + c) * 2 + 0] = Fc[a][b][c].real();
        F[((a * 8 + b) * 8 + c) * 2 + 1] = Fc[a][b][c].imag();
      }
}

// Colour matrix entries C_{sigma tau} of Eq. (2.17) by explicit contraction.
// pairs[2*i], pairs[2*i+1] are ordering indices (lexicographic).  Work per
// entry is 8^n, so this is for n <= 8.
void or_colour_entries(int n, int npairs, const long long* pairs, double* out, int nthreads) {
  std::vector<cplx> G;
  chain_tensor(n, G);
  if (nthreads < 1) nthreads = 1;
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t]() {
      std::vector<int> s(n - 2), u(n - 2);
      for (int i = t; i < npairs; i += nthreads) {
        ordering_from_index(n, pairs[2 * i], s.data());
        ordering_from_index(n, pairs[2 * i + 1], u.data());
        out[i] = colour_coefficient(n, G, s.data(), u.data());
      }
    });
  for (auto& x : th) x.join();
}

// External colour matrix (3x3 row-major) for an adjoint index (mode 0,
// c0 in 1..8) or a colour-flow pair (mode 1, (c0, c1) in {1,2,3}^2).
void or_colour_external(int mode, int c0, int c1, double* E) {
  double M[3][3];
  if (mode == 0) colour_matrix_adjoint(c0, M); else colour_matrix_flow(c0, c1, M);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) E[i * 3 + j] = M[i][j];
}

// Colour-dressed amplitude for explicit external colour matrices
// E[n][3][3] (row-major), momenta k[n][4], currents eps[n][4].
double or_amp_cd(int n, const double* k, const double* eps, const double* E) {
  std::vector<Vec<double>> kv(n), ev(n);
  load_vecs(n, k, kv.data());
  load_vecs(n, eps, ev.data());
  return amp_cd(n, kv.data(), ev.data(), reinterpret_cast<const double(*)[3][3]>(E));
}

// Colour-dressed current of one subset S (bitmask over the first n-1
// gluons): Jc[3][3][4].
void or_current_cd(int n, const double* k, const double* eps, const double* E, int S, double* Jc) {
  std::vector<Vec<double>> kv(n), ev(n);
  std::vector<CMat<double>> J;
  load_vecs(n, k, kv.data());
  load_vecs(n, eps, ev.data());
  amp_cd(n, kv.data(), ev.data(), reinterpret_cast<const double(*)[3][3]>(E), &J);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      for (int mu = 0; mu < 4; ++mu) Jc[(r * 3 + c) * 4 + mu] = J[S].e[r][c].c[mu];
}

// Batch |M|^2, colour-ordered with the full colour sum, from uniforms
// u[B][4(n-2)].  C[k][k] colour matrix (k = (n-2)!), hel[B][n] (+-1) or
// NULL for the sum over all 2^n polarisation configurations.  me2[B] in
// GeV^(8-2n).  Work is split over nthreads std::threads by event.
// tensor_form = 1 evaluates the amplitudes with the tensor-field form of
// the recursion (Eq. 2.24): the same mathematics in a different operation
// order, used to measure the FP64 rounding floor of each event.
void or_me2_co_batch(int n, long long B, double sqrt_s, const double* u, const double* q, const double* C,
                     const int8_t* hel, double g, double pt_min, double* me2, int nthreads, int tensor_form) {
  if (nthreads < 1) nthreads = 1;
  std::vector<std::thread> th;
  const int d = 4 * (n - 2);
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t]() {
      for (long long e = t; e < B; e += nthreads)
        me2[e] = me2_co_event<double>(n, sqrt_s, u + e * d, q, C, hel ? hel + e * n : nullptr, g, pt_min,
                                      tensor_form);
    });
  for (auto& x : th) x.join();
}

// Same as or_me2_co_batch in extended precision (long double: 64-bit
// significand on x86-64, IEEE binary128 on AArch64).  Serves as the
// reference for FP64 parity: the plain FP64 evaluation of the definition
// itself carries rounding errors above 1e-12 on ill-conditioned events.
void or_me2_co_batch_ext(int n, long long B, double sqrt_s, const double* u, const double* q, const double* C,
                         const int8_t* hel, double g, double pt_min, double* me2, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  std::vector<std::thread> th;
  const int d = 4 * (n - 2);
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t]() {
      std::vector<long double> ul(d);
      for (long long e = t; e < B; e += nthreads) {
        for (int i = 0; i < d; ++i) ul[i] = u[e * d + i];
        me2[e] = (double)me2_co_event<long double>(n, sqrt_s, ul.data(), q, C, hel ? hel + e * n : nullptr, g,
                                                   pt_min);
      }
    });
  for (auto& x : th) x.join();
}

void or_me2_cd_batch(int n, long long B, double sqrt_s, const double* u, const double* q, const int8_t* hel,
                     const int8_t* colors, int mode, double g, double pt_min, double* me2, int nthreads) {
  me2_cd_batch<double>(n, B, sqrt_s, u, q, hel, colors, mode, g, pt_min, me2, nthreads);
}

void or_me2_cd_batch_ext(int n, long long B, double sqrt_s, const double* u, const double* q, const int8_t* hel,
                         const int8_t* colors, int mode, double g, double pt_min, double* me2, int nthreads) {
  me2_cd_batch<long double>(n, B, sqrt_s, u, q, hel, colors, mode, g, pt_min, me2, nthreads);
}

// Batch |M|^2 estimator with sampled colour flows (me2_co_mc_batch).
void or_me2_co_mc_batch(int n, long long B, double sqrt_s, const double* u, const double* q, const int8_t* hel,
                        const int8_t* colors, double g, double pt_min, double* me2, int nthreads) {
  me2_co_mc_batch<double>(n, B, sqrt_s, u, q, hel, colors, g, pt_min, me2, nthreads);
}

void or_me2_co_mc_batch_ext(int n, long long B, double sqrt_s, const double* u, const double* q,
                            const int8_t* hel, const int8_t* colors, double g, double pt_min, double* me2,
                            int nthreads) {
  me2_co_mc_batch<long double>(n, B, sqrt_s, u, q, hel, colors, g, pt_min, me2, nthreads);
}

// Batch leading-colour |M|^2 (Sec. 4): g^(2n-4) N^(n-2) (N^2-1) sum over the
// (n-1)! orders of |A|^2, for sampled helicities hel[B][n] (weight 2^n) or,
// with hel = NULL, summed over all 2^n polarisation configurations.  Events
// failing the pT cut get 0.
void or_me2_lc_batch(int n, long long B, double sqrt_s, const double* u, const double* q, const int8_t* hel,
                     double g, double pt_min, double* me2, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  std::vector<std::thread> th;
  const int d = 4 * (n - 2);
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t]() {
      std::vector<Vec<double>> k(n), eps(n);
      std::vector<int8_t> h(n);
      for (long long e = t; e < B; e += nthreads) {
        const int nconf = hel ? 1 : (1 << n);
        double s = 0.0;
        bool cut = false;
        for (int conf = 0; conf < nconf && !cut; ++conf) {
          for (int i = 0; i < n; ++i) h[i] = hel ? hel[e * n + i] : (((conf >> i) & 1) ? -1 : 1);
          if (!event_setup(n, sqrt_s, u + e * d, q, h.data(), pt_min, k.data(), eps.data())) {
            cut = true;
            break;
          }
          s += leading_colour_sum(n, k.data(), eps.data());
        }
        me2[e] = cut ? 0.0 : std::pow(g, 2 * n - 4) * (hel ? std::pow(2.0, n) : 1.0) * s;
      }
    });
  for (auto& x : th) x.join();
}

// Continuous colour and helicity sampling (me2_cd_cont_batch).
void or_me2_cd_cont_batch(int n, long long B, double sqrt_s, const double* u, const double* q, const double* ang,
                          double g, double pt_min, double* me2, int nthreads) {
  me2_cd_cont_batch<double>(n, B, sqrt_s, u, q, ang, g, pt_min, me2, nthreads);
}

void or_me2_cd_cont_batch_ext(int n, long long B, double sqrt_s, const double* u, const double* q,
                              const double* ang, double g, double pt_min, double* me2, int nthreads) {
  me2_cd_cont_batch<long double>(n, B, sqrt_s, u, q, ang, g, pt_min, me2, nthreads);
}

// Continuous external colour matrix of one gluon from its five angles.
void or_continuous_external(const double* ang, double* E) {
  double M[3][3];
  continuous_external(ang, M);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) E[i * 3 + j] = M[i][j];
}

// The paper's kinematic constraints (Sec. 5) on the final-state gluons of
// the Rambo event of each row of u[B][4(n-2)]: pT > pt_min, |eta| < eta_max,
// Delta R > dr_min for every pair (eta_max <= 0 or dr_min <= 0 drop that
// constraint).  Pseudorapidity from the polar angle, eta = -ln tan(theta/2);
// azimuth difference folded into [0, pi].  acc[B] = 1 if the event passes.
void or_accept_cuts(int n, long long B, double sqrt_s, const double* u, double pt_min, double eta_max,
                    double dr_min, uint8_t* acc) {
  const int d = 4 * (n - 2);
  std::vector<Vec<double>> p(n);
  std::vector<double> eta(n), phi(n);
  for (long long e = 0; e < B; ++e) {
    rambo(n, sqrt_s, u + e * d, p.data());
    bool ok = true;
    for (int i = 2; i < n; ++i) {
      const double px = p[i].c[1], py = p[i].c[2], pz = p[i].c[3];
      const double pt = std::sqrt(px * px + py * py);
      if (!(pt > pt_min)) ok = false;
      const double theta = std::atan2(pt, pz);
      eta[i] = -std::log(std::tan(0.5 * theta));
      phi[i] = std::atan2(py, px);
      if (eta_max > 0.0 && !(std::fabs(eta[i]) < eta_max)) ok = false;
    }
    if (dr_min > 0.0)
      for (int i = 2; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
          double dphi = std::fabs(phi[i] - phi[j]);
          if (dphi > M_PI) dphi = 2.0 * M_PI - dphi;
          const double dr = std::sqrt((eta[i] - eta[j]) * (eta[i] - eta[j]) + dphi * dphi);
          if (!(dr > dr_min)) ok = false;
        }
    acc[e] = ok ? 1 : 0;
  }
}

// Gradient of the colour-summed |M|^2 (sampled helicity hel[n]) with
// respect to the 4(n-2) Rambo uniforms of one event, by forward-mode dual
// numbers through Rambo, the polarisations, the recursion and the colour
// sum.  Returns |M|^2; grad[4(n-2)].
double or_me2_co_grad(int n, double sqrt_s, const double* u, const double* q, const double* C, const int8_t* hel,
                      double g, double* grad) {
  const int d = 4 * (n - 2);
  std::vector<Dual> ud(d);
  for (int i = 0; i < d; ++i) { ud[i] = Dual(u[i]); ud[i].d[i] = 1.0; }
  Dual r = me2_co_event<Dual>(n, sqrt_s, ud.data(), q, C, hel, g, -1.0);
  for (int i = 0; i < d; ++i) grad[i] = r.d[i];
  return r.v;
}

}  // extern "C"
