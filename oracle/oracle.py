"""Python front end of the FP64 CPU oracle (test infrastructure only).

The oracle is a plain, slow, obviously-correct restatement of the paper's
definitions (see bg_oracle.cpp for the per-function citations).  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this module; the product library never does, and the two share
no code.

Layouts used here (host numpy arrays, float64):
  u      [B, 4(n-2)]  Rambo uniforms, per final-state gluon (u1..u4)
  p, k   [n, 4]       lab momenta / all-outgoing momenta of one event
  hel    [B, n] int8  +1 -> polarisation e1, -1 -> e2
  colors [B, n] int8  adjoint index 1..8   |  [B, 2n] colour-flow pairs 1..3
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from functools import lru_cache

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bg_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libbg_oracle.so")
_GOLDEN = os.path.join(os.path.dirname(_HERE), "tests", "golden")

_lock = threading.Lock()
_lib = None

DEFAULT_Q = (1.0, 0.0, 0.0, 1.0)
G_S_DEFAULT = math.sqrt(4.0 * math.pi * 0.118)  # alpha_s = 0.118 (Sec. 5)


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (no GPU, no CUDA)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i8p = ctypes.POINTER(ctypes.c_int8)
            llp = ctypes.POINTER(ctypes.c_longlong)
            c_int, c_dbl, c_ll = ctypes.c_int, ctypes.c_double, ctypes.c_longlong
            L.or_rambo.argtypes = [c_int, c_dbl, dp, dp]
            L.or_polarisations.argtypes = [dp, dp, dp, dp]
            L.or_amp_co.argtypes = [c_int, dp, dp, ip, c_int]
            L.or_amp_co.restype = c_dbl
            L.or_amp_co_cplx.argtypes = [c_int, dp, dp, dp, ip, c_int, dp]
            L.or_currents_co.argtypes = [c_int, dp, dp, ip, c_int, dp, dp]
            L.or_ordering.argtypes = [c_int, c_ll, ip]
            L.or_amps_all.argtypes = [c_int, dp, dp, dp]
            L.or_adjoint_generators.argtypes = [dp]
            L.or_colour_entries.argtypes = [c_int, c_int, llp, dp, c_int]
            L.or_colour_external.argtypes = [c_int, c_int, c_int, dp]
            L.or_amp_cd.argtypes = [c_int, dp, dp, dp]
            L.or_amp_cd.restype = c_dbl
            L.or_current_cd.argtypes = [c_int, dp, dp, dp, c_int, dp]
            L.or_me2_co_batch.argtypes = [c_int, c_ll, c_dbl, dp, dp, dp, i8p, c_dbl, c_dbl, dp, c_int, c_int]
            L.or_me2_co_batch_ext.argtypes = [c_int, c_ll, c_dbl, dp, dp, dp, i8p, c_dbl, c_dbl, dp, c_int]
            L.or_me2_cd_batch.argtypes = [c_int, c_ll, c_dbl, dp, dp, i8p, i8p, c_int, c_dbl, c_dbl, dp, c_int]
            L.or_me2_cd_batch_ext.argtypes = [c_int, c_ll, c_dbl, dp, dp, i8p, i8p, c_int, c_dbl, c_dbl, dp, c_int]
            L.or_me2_co_mc_batch.argtypes = [c_int, c_ll, c_dbl, dp, dp, i8p, i8p, c_dbl, c_dbl, dp, c_int]
            L.or_me2_co_mc_batch_ext.argtypes = [c_int, c_ll, c_dbl, dp, dp, i8p, i8p, c_dbl, c_dbl, dp, c_int]
            L.or_me2_lc_batch.argtypes = [c_int, c_ll, c_dbl, dp, dp, i8p, c_dbl, c_dbl, dp, c_int]
            L.or_me2_cd_cont_batch.argtypes = [c_int, c_ll, c_dbl, dp, dp, dp, c_dbl, c_dbl, dp, c_int]
            L.or_me2_cd_cont_batch_ext.argtypes = [c_int, c_ll, c_dbl, dp, dp, dp, c_dbl, c_dbl, dp, c_int]
            L.or_continuous_external.argtypes = [dp, dp]
            L.or_accept_cuts.argtypes = [c_int, c_ll, c_dbl, dp, c_dbl, c_dbl, c_dbl, ctypes.POINTER(ctypes.c_uint8)]
            L.or_me2_co_grad.argtypes = [c_int, c_dbl, dp, dp, dp, i8p, c_dbl, dp]
            L.or_me2_co_grad.restype = c_dbl
            _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _i8(a):
    a = np.ascontiguousarray(a, dtype=np.int8)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))


def n_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


# --------------------------------------------------------------------------
# kinematics
# --------------------------------------------------------------------------
def rambo(n: int, sqrt_s: float, u) -> np.ndarray:
    """Lab momenta [n,4] of one event from its 4(n-2) uniforms."""
    u, up = _d(u)
    p = np.zeros((n, 4))
    _, pp = _d(p)
    lib().or_rambo(n, sqrt_s, up, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return p


def outgoing(p: np.ndarray) -> np.ndarray:
    """All-outgoing momenta: k1 = -p1, k2 = -p2, k_i = p_i."""
    k = np.array(p, dtype=np.float64, copy=True)
    k[:2] *= -1.0
    return k


def polarisations(k, q=DEFAULT_Q):
    k, kp = _d(k)
    q, qp = _d(q)
    e1 = np.zeros(4)
    e2 = np.zeros(4)
    lib().or_polarisations(kp, qp, e1.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           e2.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return e1, e2


def pols_for(k: np.ndarray, hel, q=DEFAULT_Q) -> np.ndarray:
    """External currents [n,4] for helicity labels hel[n] (+1 -> e1, -1 -> e2)."""
    eps = np.zeros_like(k)
    for i in range(k.shape[0]):
        e1, e2 = polarisations(k[i], q)
        eps[i] = e1 if hel[i] > 0 else e2
    return eps


def mdot(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return a[..., 0] * b[..., 0] - a[..., 1] * b[..., 1] - a[..., 2] * b[..., 2] - a[..., 3] * b[..., 3]


# --------------------------------------------------------------------------
# colour-ordered amplitudes
# --------------------------------------------------------------------------
def amp_co(k, eps, order, tensor_form=False) -> float:
    n = len(order)
    k, kp = _d(k)
    eps, ep = _d(eps)
    o, op = _i(order)
    return lib().or_amp_co(n, kp, ep, op, int(tensor_form))


def amp_co_complex(k, eps_c, order, tensor_form=False) -> complex:
    n = len(order)
    k, kp = _d(k)
    er, erp = _d(np.real(eps_c))
    ei, eip = _d(np.imag(eps_c))
    o, op = _i(order)
    out = np.zeros(2)
    lib().or_amp_co_cplx(n, kp, erp, eip, op, int(tensor_form), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return complex(out[0], out[1])


def currents_co(k, eps, order, tensor_form=False):
    """Current table J[i,j,4] and segment momenta P[i,j,4] of one colour order."""
    n = len(order)
    m = n - 1
    k, kp = _d(k)
    eps, ep = _d(eps)
    o, op = _i(order)
    J = np.zeros((m, m, 4))
    P = np.zeros((m, m, 4))
    lib().or_currents_co(n, kp, ep, op, int(tensor_form), J.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         P.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return J, P


def ordering(n: int, r: int) -> np.ndarray:
    """Labels (0-based, in 1..n-2) of lexicographic ordering index r."""
    s = np.zeros(n - 2, dtype=np.int32)
    lib().or_ordering(n, r, s.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return s


@lru_cache(maxsize=None)
def orderings(n: int) -> np.ndarray:
    return np.stack([ordering(n, r) for r in range(math.factorial(n - 2))])


def amps_all(k, eps) -> np.ndarray:
    """A(1, sigma, n) for all (n-2)! orderings in lexicographic order."""
    n = k.shape[0]
    k, kp = _d(k)
    eps, ep = _d(eps)
    out = np.zeros(math.factorial(n - 2))
    lib().or_amps_all(n, kp, ep, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


# --------------------------------------------------------------------------
# colour matrix (Eq. 2.17)
# --------------------------------------------------------------------------
def adjoint_generators() -> np.ndarray:
    F = np.zeros((8, 8, 8, 2))
    lib().or_adjoint_generators(F.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return F[..., 0] + 1j * F[..., 1]


def colour_entries(n: int, pairs, nthreads: int | None = None) -> np.ndarray:
    """C_{sigma tau} for ordering-index pairs by explicit SU(3) contraction."""
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int64).reshape(-1, 2))
    out = np.zeros(pairs.shape[0])
    lib().or_colour_entries(n, pairs.shape[0], pairs.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nthreads or n_cores())
    return out


def colour_row_explicit(n: int, nthreads: int | None = None) -> np.ndarray:
    """First row C_{id, tau} by explicit contraction (8^n work per entry)."""
    k = math.factorial(n - 2)
    pairs = np.stack([np.zeros(k, dtype=np.int64), np.arange(k, dtype=np.int64)], axis=1)
    return colour_entries(n, pairs, nthreads)


def golden_row_path(n: int) -> str:
    return os.path.join(_GOLDEN, f"colour_row_n{n}.txt")


@lru_cache(maxsize=None)
def colour_row(n: int) -> np.ndarray:
    """First row of C, from the committed golden file (written by
    tests/golden/make_colour_rows.py from this oracle) if present, else by
    explicit contraction."""
    path = golden_row_path(n)
    if os.path.exists(path):
        vals = np.loadtxt(path, comments="#")
        return np.atleast_1d(vals).astype(np.float64)
    return colour_row_explicit(n)


def relabel_index(n: int) -> np.ndarray:
    """R[s, t] = index of the relative ordering rho = sigma_s^-1 o sigma_t,
    rho_j = position in sigma_s of the label sigma_t[j].

    The index of rho is looked up in a table addressed by the digits of rho
    in base m+1 (m = n-2), filled from the list of orderings itself, so the
    lookup needs no ranking formula; rows are done in blocks with numpy
    (5040 x 5040 at n = 9 in seconds)."""
    ords = orderings(n).astype(np.int64)          # [k, m], labels 1..m
    kk, m = ords.shape
    base = m + 1
    weights = base ** np.arange(m - 1, -1, -1, dtype=np.int64)
    table = np.full(base ** m, -1, dtype=np.int64)
    table[ords @ weights] = np.arange(kk)
    pos = np.zeros((kk, base), dtype=np.int64)    # pos[s, label] = position (1..m) in sigma_s
    pos[np.arange(kk)[:, None], ords] = np.arange(1, m + 1)[None, :]
    R = np.empty((kk, kk), dtype=np.int64)
    block = max(1, (1 << 22) // (kk * m))
    for s0 in range(0, kk, block):
        s1 = min(kk, s0 + block)
        rho = pos[s0:s1][:, ords]                 # [blk, k, m]: rho[s, t, j] = pos_s[sigma_t[j]]
        R[s0:s1] = table[rho @ weights]
    assert R.min() >= 0
    return R


def relabel_index_loop(n: int) -> np.ndarray:
    """relabel_index written as the plain double loop over (s, t) with a
    dictionary lookup (slow; kept as the definition it is checked against)."""
    ords = orderings(n)
    kk = ords.shape[0]
    m = n - 2
    lookup = {tuple(o): i for i, o in enumerate(ords)}
    R = np.zeros((kk, kk), dtype=np.int64)
    for s in range(kk):
        pos = np.zeros(n, dtype=np.int64)
        pos[ords[s]] = np.arange(1, m + 1)
        for t in range(kk):
            R[s, t] = lookup[tuple(pos[ords[t]])]
    return R


@lru_cache(maxsize=None)
def colour_matrix(n: int) -> np.ndarray:
    """Full (n-2)! x (n-2)! colour matrix from its first row, using that C
    depends only on the relative permutation (checked directly at n = 5, 6)."""
    row = colour_row(n)
    return row[relabel_index(n)]


# --------------------------------------------------------------------------
# colour-dressed amplitudes (Eqs. 2.28-2.32)
# --------------------------------------------------------------------------
def colour_external(mode: int, c0: int, c1: int = 0) -> np.ndarray:
    E = np.zeros((3, 3))
    lib().or_colour_external(mode, c0, c1, E.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return E


def externals_for(colors, mode: int) -> np.ndarray:
    colors = np.asarray(colors)
    if mode == 0:
        return np.stack([colour_external(0, int(c)) for c in colors])
    n = colors.shape[0] // 2
    return np.stack([colour_external(1, int(colors[2 * i]), int(colors[2 * i + 1])) for i in range(n)])


def amp_cd(k, eps, E) -> float:
    n = k.shape[0]
    k, kp = _d(k)
    eps, ep = _d(eps)
    E, Ep = _d(E)
    return lib().or_amp_cd(n, kp, ep, Ep)


def current_cd(k, eps, E, S: int) -> np.ndarray:
    n = k.shape[0]
    k, kp = _d(k)
    eps, ep = _d(eps)
    E, Ep = _d(E)
    J = np.zeros((3, 3, 4))
    lib().or_current_cd(n, kp, ep, Ep, S, J.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return J


# --------------------------------------------------------------------------
# batched |M|^2
# --------------------------------------------------------------------------
def me2_co(n, u, sqrt_s=1000.0, hel=None, q=DEFAULT_Q, g=G_S_DEFAULT, pt_min=-1.0, C=None,
           nthreads=None, tensor_form=False) -> np.ndarray:
    """Colour-summed |M|^2 (GeV^(8-2n)) per event; hel=None sums all 2^n
    polarisation configurations, else hel[B,n] is sampled (weight 2^n).
    tensor_form evaluates the amplitudes with the auxiliary tensor field."""
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1, 4 * (n - 2)))
    B = u.shape[0]
    C = colour_matrix(n) if C is None else np.ascontiguousarray(C, dtype=np.float64)
    q, qp = _d(q)
    _, Cp = _d(C)
    me2 = np.zeros(B)
    hp = None
    if hel is not None:
        hel, hp = _i8(np.asarray(hel).reshape(B, n))
    lib().or_me2_co_batch(n, B, sqrt_s, u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), qp, Cp, hp, g,
                          pt_min, me2.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nthreads or n_cores(),
                          int(tensor_form))
    return me2


def me2_co_ext(n, u, sqrt_s=1000.0, hel=None, q=DEFAULT_Q, g=G_S_DEFAULT, pt_min=-1.0, C=None,
               nthreads=None) -> np.ndarray:
    """me2_co evaluated in extended precision (long double), rounded to FP64."""
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1, 4 * (n - 2)))
    B = u.shape[0]
    C = colour_matrix(n) if C is None else np.ascontiguousarray(C, dtype=np.float64)
    q, qp = _d(q)
    _, Cp = _d(C)
    me2 = np.zeros(B)
    hp = None
    if hel is not None:
        hel, hp = _i8(np.asarray(hel).reshape(B, n))
    lib().or_me2_co_batch_ext(n, B, sqrt_s, u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), qp, Cp, hp, g,
                              pt_min, me2.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nthreads or n_cores())
    return me2


def fp64_noise_floor(n, u, hel=None, sqrt_s=1000.0, q=DEFAULT_Q, g=G_S_DEFAULT, pt_min=-1.0) -> np.ndarray:
    """Per-event relative FP64 rounding floor of |M|^2: the spread between
    two mathematically identical evaluations (V4 form vs tensor-field form of
    the recursion; for helicity-summed |M|^2 also a second gauge vector,
    since the sum is exactly independent of q)."""
    a = me2_co(n, u, sqrt_s=sqrt_s, hel=hel, q=q, g=g, pt_min=pt_min)
    b = me2_co(n, u, sqrt_s=sqrt_s, hel=hel, q=q, g=g, pt_min=pt_min, tensor_form=True)
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.where(a != 0, np.abs(b / a - 1.0), 0.0)
        if hel is None:
            c = me2_co(n, u, sqrt_s=sqrt_s, q=(1.0, 0.6, 0.0, 0.8), g=g, pt_min=pt_min)
            r = np.maximum(r, np.where(a != 0, np.abs(c / a - 1.0), 0.0))
    return r


def me2_cd(n, u, hel, colors, mode=0, sqrt_s=1000.0, q=DEFAULT_Q, g=G_S_DEFAULT, pt_min=-1.0,
           nthreads=None, ext=False) -> np.ndarray:
    """Colour-dressed |M|^2 estimator per event with sampled colours
    (ext: evaluated in extended precision)."""
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1, 4 * (n - 2)))
    B = u.shape[0]
    q, qp = _d(q)
    hel, hp = _i8(np.asarray(hel).reshape(B, n))
    colors, cp = _i8(np.asarray(colors).reshape(B, -1))
    me2 = np.zeros(B)
    fn = lib().or_me2_cd_batch_ext if ext else lib().or_me2_cd_batch
    fn(n, B, sqrt_s, u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), qp, hp, cp, mode, g,
       pt_min, me2.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nthreads or n_cores())
    return me2


def me2_co_mc(n, u, hel, colors, sqrt_s=1000.0, q=DEFAULT_Q, g=G_S_DEFAULT, pt_min=-1.0,
              nthreads=None, ext=False) -> np.ndarray:
    """|M|^2 estimator per event for sampled colour flows colors[B, 2n],
    evaluated from colour-ordered amplitudes with Eq. (2.19) (ext: in
    extended precision)."""
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1, 4 * (n - 2)))
    B = u.shape[0]
    q, qp = _d(q)
    hel, hp = _i8(np.asarray(hel).reshape(B, n))
    colors, cp = _i8(np.asarray(colors).reshape(B, 2 * n))
    me2 = np.zeros(B)
    fn = lib().or_me2_co_mc_batch_ext if ext else lib().or_me2_co_mc_batch
    fn(n, B, sqrt_s, u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), qp, hp, cp, g,
       pt_min, me2.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nthreads or n_cores())
    return me2


def me2_lc(n, u, hel=None, sqrt_s=1000.0, q=DEFAULT_Q, g=G_S_DEFAULT, pt_min=-1.0, nthreads=None) -> np.ndarray:
    """Leading-colour |M|^2 per event (Sec. 4): hel[B, n] sampled (weight
    2^n) or None (all 2^n polarisation configurations)."""
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1, 4 * (n - 2)))
    B = u.shape[0]
    q, qp = _d(q)
    hp = None
    if hel is not None:
        hel, hp = _i8(np.asarray(hel).reshape(B, n))
    me2 = np.zeros(B)
    lib().or_me2_lc_batch(n, B, sqrt_s, u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), qp, hp, g, pt_min,
                          me2.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nthreads or n_cores())
    return me2


def continuous_external(ang) -> np.ndarray:
    """External colour matrix sum_a eta^a T^a of one gluon from its five
    angles (cos theta, phi, cos theta_bar, phi_bar, phi_h)."""
    a, ap = _d(np.asarray(ang, dtype=np.float64).reshape(5))
    E = np.zeros((3, 3))
    lib().or_continuous_external(ap, E.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return E


def me2_cd_cont(n, u, ang, sqrt_s=1000.0, q=DEFAULT_Q, g=G_S_DEFAULT, pt_min=-1.0, nthreads=None,
                ext=False) -> np.ndarray:
    """Colour-dressed |M|^2 estimator with continuous colour and helicity
    sampling, ang[B, n, 5] = (cos theta, phi, cos theta_bar, phi_bar, phi_h)
    per gluon (ext: extended precision)."""
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1, 4 * (n - 2)))
    B = u.shape[0]
    q, qp = _d(q)
    ang, angp = _d(np.asarray(ang, dtype=np.float64).reshape(B, n, 5))
    me2 = np.zeros(B)
    fn = lib().or_me2_cd_cont_batch_ext if ext else lib().or_me2_cd_cont_batch
    fn(n, B, sqrt_s, u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), qp, angp, g, pt_min,
       me2.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nthreads or n_cores())
    return me2


def accept_cuts(n, u, sqrt_s=1000.0, pt_min=20.0, eta_max=2.5, dr_min=0.4) -> np.ndarray:
    """Per-event acceptance [B] uint8 of the paper's kinematic constraints
    (Sec. 5) for the Rambo events of u[B, 4(n-2)]."""
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1, 4 * (n - 2)))
    acc = np.zeros(u.shape[0], dtype=np.uint8)
    lib().or_accept_cuts(n, u.shape[0], sqrt_s, u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), pt_min, eta_max,
                         dr_min, acc.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return acc


def me2_co_grad(n, u, hel, sqrt_s=1000.0, q=DEFAULT_Q, g=G_S_DEFAULT, C=None):
    """(|M|^2, d|M|^2/du) for one event by forward-mode dual numbers."""
    u, up = _d(np.asarray(u).reshape(-1))
    C = colour_matrix(n) if C is None else np.ascontiguousarray(C, dtype=np.float64)
    _, Cp = _d(C)
    q, qp = _d(q)
    hel, hp = _i8(np.asarray(hel).reshape(-1))
    grad = np.zeros(4 * (n - 2))
    v = lib().or_me2_co_grad(n, sqrt_s, up, qp, Cp, hp, g, grad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return v, grad
