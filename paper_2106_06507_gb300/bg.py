"""Thin ctypes binding of libbg.so (include/bg.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  Tensors are torch CUDA tensors (device memory and
streams come from PyTorch); the calls enqueue work on the current torch
stream unless `stream` is given.  Raises if the library is missing: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbg.so")

BG_OK, BG_EINVAL, BG_ENOMEM, BG_ECUDA, BG_EUNSUPPORTED, BG_ETIMEOUT = range(6)
BG_F64, BG_F32 = 0, 1
BG_CS_F64, BG_CS_F32, BG_CS_TC_BF16 = 0, 1, 2
BG_COL_ADJOINT, BG_COL_FLOW = 0, 1

G_S_DEFAULT = math.sqrt(4.0 * math.pi * 0.118)  # alpha_s = 0.118
DEFAULT_Q = (1.0, 0.0, 0.0, 1.0)

_lib = None


BG_ALGO_CO, BG_ALGO_CD = 0, 1


class PlanDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("max_batch", ctypes.c_int64), ("sqrt_s", ctypes.c_double),
                ("pt_min", ctypes.c_double), ("g_s", ctypes.c_double), ("q", ctypes.c_double * 4),
                ("prec", ctypes.c_int), ("cs_mode", ctypes.c_int), ("algo", ctypes.c_int),
                ("color_mode", ctypes.c_int), ("hel_sampled", ctypes.c_int), ("grad", ctypes.c_int)]


class MixedDesc(ctypes.Structure):
    _fields_ = [("n_min", ctypes.c_int), ("n_max", ctypes.c_int), ("max_batch", ctypes.c_int64),
                ("sqrt_s", ctypes.c_double), ("pt_min", ctypes.c_double), ("g_s", ctypes.c_double),
                ("q", ctypes.c_double * 4), ("prec", ctypes.c_int), ("cs_mode", ctypes.c_int),
                ("color_mode", ctypes.c_int), ("n_co_max", ctypes.c_int), ("chunk_bytes", ctypes.c_int64),
                ("autotune", ctypes.c_int)]


class BGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bg status {code}: {msg}")
        self.code = code


def lib() -> ctypes.CDLL:
    """Load libbg.so (built by build_lib.build()); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libbg.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        c_int, c_dbl, c_i64, vp = ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        L.bg_last_error.restype = ctypes.c_char_p
        L.bg_num_orderings.argtypes = [c_int]
        L.bg_num_orderings.restype = c_i64
        L.bg_colormat_create.argtypes = [c_int, ctypes.POINTER(vp)]
        L.bg_colormat_destroy.argtypes = [vp]
        L.bg_colormat_destroy.restype = None
        L.bg_colormat_row.argtypes = [vp, dp]
        L.bg_colormat_row_host.argtypes = [c_int, dp]
        L.bg_momenta_rambo.argtypes = [c_int, c_i64, c_dbl, vp, vp, c_dbl, vp, vp]
        L.bg_currents_co.argtypes = [c_int, c_i64, c_dbl, vp, vp, dp, c_int, vp, vp]
        L.bg_currents_co_tensor.argtypes = [c_int, c_i64, c_dbl, vp, vp, dp, c_int, vp, vp]
        L.bg_color_sum.argtypes = [vp, c_i64, c_int, vp, c_int, c_int, c_dbl, c_dbl, c_int, vp, vp, vp]
        L.bg_plan_create.argtypes = [ctypes.POINTER(PlanDesc), ctypes.POINTER(vp)]
        L.bg_plan_destroy.argtypes = [vp]
        L.bg_plan_destroy.restype = None
        L.bg_plan_workspace_bytes.argtypes = [vp]
        L.bg_plan_workspace_bytes.restype = c_i64
        L.bg_me2_batch.argtypes = [vp, c_i64, vp, vp, vp, vp, vp]
        L.bg_me2_batch_async.argtypes = [vp, c_i64, vp, vp, vp, vp]
        L.bg_me2_grad.argtypes = [vp, c_i64, vp, vp, vp, vp, vp, vp]
        L.bg_cd_workspace_bytes.argtypes = [c_int, c_int, ctypes.POINTER(c_i64)]
        L.bg_currents_cd.argtypes = [c_int, c_i64, c_dbl, vp, vp, vp, c_int, dp, c_int, c_dbl, vp, vp, vp, c_i64, vp]
        L.bg_apply_cuts.argtypes = [c_int, c_i64, vp, c_dbl, c_dbl, c_dbl, vp, vp]
        L.bg_currents_cd_cont.argtypes = [c_int, c_i64, c_dbl, vp, vp, dp, c_int, c_dbl, vp, vp, vp, c_i64, vp]
        L.bg_comc_workspace_bytes.argtypes = [c_int, c_i64, c_int, ctypes.POINTER(c_i64)]
        L.bg_currents_co_mc.argtypes = [c_int, c_i64, c_dbl, vp, vp, vp, dp, c_int, c_dbl, vp, vp, vp, c_i64, vp]
        L.bg_lc_workspace_bytes.argtypes = [c_int, c_i64, c_int, c_int, ctypes.POINTER(c_i64)]
        L.bg_currents_lc.argtypes = [c_int, c_i64, c_dbl, vp, vp, dp, c_int, c_dbl, vp, vp, vp, c_i64, vp]
        L.bg_mixed_create.argtypes = [ctypes.POINTER(MixedDesc), ctypes.POINTER(vp)]
        L.bg_mixed_destroy.argtypes = [vp]
        L.bg_mixed_destroy.restype = None
        L.bg_mixed_buffers.argtypes = [vp] + [ctypes.POINTER(vp)] * 5
        L.bg_mixed_workspace_bytes.argtypes = [vp]
        L.bg_mixed_workspace_bytes.restype = c_i64
        L.bg_mixed_run.argtypes = [vp, c_i64, vp]
        L.bg_mixed_counts.argtypes = [vp, ctypes.POINTER(c_i64)]
        L.bg_mixed_kernel_nodes.argtypes = [vp, ctypes.POINTER(c_i64)]
        L.bg_tune_num_variants.argtypes = [c_int, c_int]
        L.bg_tune_num_variants.restype = c_int
        L.bg_autotune.argtypes = [c_int, c_int, c_int, c_i64, vp, ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_float)]
        L.bg_tune_set.argtypes = [c_int, c_int, c_int, c_int]
        L.bg_tune_get.argtypes = [c_int, c_int, c_int, ctypes.POINTER(c_int)]
        L.bg_tune_save.argtypes = [ctypes.c_char_p]
        L.bg_tune_load.argtypes = [ctypes.c_char_p]
        L.bg_device_status.argtypes = [ctypes.POINTER(c_int)]
        L.bg_device_status_reset.argtypes = []
        for name in ("bg_colormat_create", "bg_colormat_row", "bg_colormat_row_host", "bg_momenta_rambo",
                     "bg_currents_co", "bg_currents_co_tensor", "bg_color_sum", "bg_device_status", "bg_device_status_reset",
                     "bg_plan_create", "bg_me2_batch", "bg_me2_batch_async", "bg_cd_workspace_bytes",
                     "bg_currents_cd", "bg_currents_cd_cont", "bg_apply_cuts", "bg_comc_workspace_bytes", "bg_currents_co_mc", "bg_lc_workspace_bytes", "bg_currents_lc", "bg_me2_grad", "bg_mixed_create", "bg_mixed_buffers", "bg_mixed_run",
                     "bg_mixed_counts", "bg_mixed_kernel_nodes", "bg_autotune", "bg_tune_set", "bg_tune_get", "bg_tune_save",
                     "bg_tune_load"):
            getattr(L, name).restype = c_int
        _lib = L
    return _lib


def _check(code: int) -> None:
    if code != BG_OK:
        raise BGError(code, lib().bg_last_error().decode())


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _q(q) -> ctypes.Array:
    return (ctypes.c_double * 4)(*[float(x) for x in q])


def num_orderings(n: int) -> int:
    return int(lib().bg_num_orderings(n))


class ColourMatrix:
    """Device colour matrix of Eq. (2.17) (library-owned; freed on close)."""

    def __init__(self, n: int):
        self.n = n
        self.k = num_orderings(n)
        h = ctypes.c_void_p()
        _check(lib().bg_colormat_create(n, ctypes.byref(h)))
        self._h = h

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def row(self):
        import numpy as np
        out = np.zeros(self.k)
        _check(lib().bg_colormat_row(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().bg_colormat_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def colour_row_host(n: int):
    import numpy as np
    out = np.zeros(math.factorial(n - 2))
    _check(lib().bg_colormat_row_host(n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def momenta_rambo(n: int, u: torch.Tensor, sqrt_s: float = 1000.0, pt_min: float = -1.0, p=None, accept=None,
                  stream=None):
    """u [B, 4(n-2)] float64 CUDA -> (p [4, n, B] float64, accept [B] uint8)."""
    B = u.shape[0]
    assert u.dtype == torch.float64 and u.is_cuda and u.is_contiguous()
    if p is None:
        p = torch.empty((4, n, B), dtype=torch.float64, device=u.device)
    if accept is None:
        accept = torch.empty((B,), dtype=torch.uint8, device=u.device)
    _check(lib().bg_momenta_rambo(n, B, sqrt_s, _ptr(u), _ptr(p), pt_min, _ptr(accept), _stream(stream)))
    return p, accept


def apply_cuts(n: int, p: torch.Tensor, pt_min: float = 20.0, eta_max: float = 2.5, dr_min: float = 0.4,
               accept=None, stream=None) -> torch.Tensor:
    """The paper's kinematic constraints (Sec. 5) on p [4, n, B] -> accept [B]
    uint8 (eta_max <= 0 or dr_min <= 0 drop that constraint)."""
    B = p.shape[2]
    if accept is None:
        accept = torch.empty((B,), dtype=torch.uint8, device=p.device)
    _check(lib().bg_apply_cuts(n, B, _ptr(p), pt_min, eta_max, dr_min, _ptr(accept), _stream(stream)))
    return accept


def currents_co(n: int, p: torch.Tensor, hel: torch.Tensor | None = None, q=DEFAULT_Q, prec: int = BG_F32,
                sqrt_s: float = 1000.0, amps=None, stream=None, tensor_form: bool = False) -> torch.Tensor:
    """p [4, n, B] float64, hel [n, B] int8 or None (all 2^n configurations)
    -> amps [B, H, (n-2)!] (float32 or float64).  tensor_form: the auxiliary
    tensor field in place of the four-gluon vertex (bg_currents_co_tensor)."""
    B = p.shape[2]
    H = 1 if hel is not None else 2**n
    k = num_orderings(n)
    dt = torch.float32 if prec == BG_F32 else torch.float64
    if amps is None:
        amps = torch.empty((B, H, k), dtype=dt, device=p.device)
    if hel is not None:
        assert hel.dtype == torch.int8 and hel.is_contiguous() and tuple(hel.shape) == (n, B)
    fn = lib().bg_currents_co_tensor if tensor_form else lib().bg_currents_co
    _check(fn(n, B, sqrt_s, _ptr(p), _ptr(hel), _q(q), prec, _ptr(amps), _stream(stream)))
    return amps


def color_sum(C: ColourMatrix, amps: torch.Tensor, hel_sampled: bool, mode: int = BG_CS_F64,
              g_s: float = G_S_DEFAULT, sqrt_s: float = 1000.0, accept: torch.Tensor | None = None, me2=None,
              stream=None) -> torch.Tensor:
    """amps [B, H, k] -> me2 [B] float64 (GeV^(8-2n))."""
    B, H, k = amps.shape
    assert k == C.k and amps.is_contiguous()
    prec = BG_F32 if amps.dtype == torch.float32 else BG_F64
    if me2 is None:
        me2 = torch.empty((B,), dtype=torch.float64, device=amps.device)
    _check(lib().bg_color_sum(C.handle, B, H, _ptr(amps), prec, mode, g_s, sqrt_s, int(bool(hel_sampled)),
                              _ptr(accept), _ptr(me2), _stream(stream)))
    return me2


_cd_ws_cache: dict = {}


def cd_workspace_bytes(n: int, prec: int = BG_F32) -> int:
    b = ctypes.c_int64(0)
    _check(lib().bg_cd_workspace_bytes(n, prec, ctypes.byref(b)))
    return int(b.value)


def currents_cd(n: int, p: torch.Tensor, hel: torch.Tensor, colors: torch.Tensor, flow: bool = False,
                prec: int = BG_F32, sqrt_s: float = 1000.0, g_s: float = G_S_DEFAULT, q=DEFAULT_Q,
                accept: torch.Tensor | None = None, me2=None, workspace: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """Colour-dressed |M|^2 estimator per event: p [4, n, B] float64, hel [n, B]
    int8, colors [n, B] (adjoint, 1..8) or [2n, B] (flow pairs, 1..3) int8.
    The workspace (bg_cd_workspace_bytes) is cached per (n, prec, device) if
    not given."""
    B = p.shape[2]
    if me2 is None:
        me2 = torch.empty((B,), dtype=torch.float64, device=p.device)
    if workspace is None:
        key = (n, prec, p.device.index)
        workspace = _cd_ws_cache.get(key)
        if workspace is None:
            workspace = torch.empty((cd_workspace_bytes(n, prec),), dtype=torch.uint8, device=p.device)
            _cd_ws_cache[key] = workspace
    _check(lib().bg_currents_cd(n, B, sqrt_s, _ptr(p), _ptr(hel), _ptr(colors),
                                BG_COL_FLOW if flow else BG_COL_ADJOINT, _q(q), prec, g_s, _ptr(accept), _ptr(me2),
                                _ptr(workspace), workspace.numel(), _stream(stream)))
    return me2


def currents_cd_cont(n: int, p: torch.Tensor, ang: torch.Tensor, prec: int = BG_F32, sqrt_s: float = 1000.0,
                     g_s: float = G_S_DEFAULT, q=DEFAULT_Q, accept: torch.Tensor | None = None, me2=None,
                     workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Colour-dressed |M|^2 estimator with continuous colour and helicity
    sampling: p [4, n, B] float64, ang [5n, B] float64 (per gluon cos theta,
    phi, cos theta_bar, phi_bar, phi_h)."""
    B = p.shape[2]
    if me2 is None:
        me2 = torch.empty((B,), dtype=torch.float64, device=p.device)
    if workspace is None:
        key = (n, prec, p.device.index)
        workspace = _cd_ws_cache.get(key)
        if workspace is None:
            workspace = torch.empty((cd_workspace_bytes(n, prec),), dtype=torch.uint8, device=p.device)
            _cd_ws_cache[key] = workspace
    assert ang.dtype == torch.float64 and ang.is_contiguous() and tuple(ang.shape) == (5 * n, B)
    _check(lib().bg_currents_cd_cont(n, B, sqrt_s, _ptr(p), _ptr(ang), _q(q), prec, g_s, _ptr(accept), _ptr(me2),
                                     _ptr(workspace), workspace.numel(), _stream(stream)))
    return me2


def comc_workspace_bytes(n: int, B: int, prec: int = BG_F32) -> int:
    b = ctypes.c_int64()
    _check(lib().bg_comc_workspace_bytes(n, B, prec, ctypes.byref(b)))
    return b.value


def currents_co_mc(n: int, p: torch.Tensor, hel: torch.Tensor, colors: torch.Tensor, prec: int = BG_F32,
                   sqrt_s: float = 1000.0, g_s: float = G_S_DEFAULT, q=DEFAULT_Q,
                   accept: torch.Tensor | None = None, me2=None, workspace: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
    """|M|^2 estimator per event for sampled colour flows, evaluated from
    colour-ordered amplitudes (Eq. 2.19): p [4, n, B] float64, hel [n, B]
    int8, colors [2n, B] int8 flow pairs in 1..3."""
    B = p.shape[2]
    if me2 is None:
        me2 = torch.empty((B,), dtype=torch.float64, device=p.device)
    if workspace is None:
        workspace = torch.empty((max(comc_workspace_bytes(n, B, prec), 1),), dtype=torch.uint8, device=p.device)
    _check(lib().bg_currents_co_mc(n, B, sqrt_s, _ptr(p), _ptr(hel), _ptr(colors), _q(q), prec, g_s, _ptr(accept),
                                   _ptr(me2), _ptr(workspace), workspace.numel(), _stream(stream)))
    return me2


def lc_workspace_bytes(n: int, B: int, hel_sampled: bool = True, prec: int = BG_F32) -> int:
    b = ctypes.c_int64()
    _check(lib().bg_lc_workspace_bytes(n, B, int(hel_sampled), prec, ctypes.byref(b)))
    return b.value


def currents_lc(n: int, p: torch.Tensor, hel: torch.Tensor | None, prec: int = BG_F32, sqrt_s: float = 1000.0,
                g_s: float = G_S_DEFAULT, q=DEFAULT_Q, accept: torch.Tensor | None = None, me2=None,
                workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Leading-colour |M|^2 per event (Sec. 4): p [4, n, B] float64, hel
    [n, B] int8 (sampled, weight 2^n) or None (all 2^n configurations)."""
    B = p.shape[2]
    if me2 is None:
        me2 = torch.empty((B,), dtype=torch.float64, device=p.device)
    if workspace is None:
        workspace = torch.empty((max(lc_workspace_bytes(n, B, hel is not None, prec), 1),), dtype=torch.uint8,
                                device=p.device)
    _check(lib().bg_currents_lc(n, B, sqrt_s, _ptr(p), _ptr(hel), _q(q), prec, g_s, _ptr(accept), _ptr(me2),
                                _ptr(workspace), workspace.numel(), _stream(stream)))
    return me2


class Plan:
    """The whole hot path for one multiplicity (bg_plan_create / bg_me2_batch)."""

    def __init__(self, n: int, max_batch: int, sqrt_s: float = 1000.0, pt_min: float = -1.0,
                 g_s: float = G_S_DEFAULT, q=DEFAULT_Q, prec: int = BG_F32, cs_mode: int = BG_CS_F32,
                 algo: int = BG_ALGO_CO, color_mode: int = BG_COL_ADJOINT, hel_sampled: bool = True,
                 grad: bool = False):
        d = PlanDesc()
        d.grad = int(grad)
        d.n, d.max_batch, d.sqrt_s, d.pt_min, d.g_s = n, max_batch, sqrt_s, pt_min, g_s
        for i in range(4):
            d.q[i] = float(q[i])
        d.prec, d.cs_mode, d.algo, d.color_mode, d.hel_sampled = prec, cs_mode, algo, color_mode, int(hel_sampled)
        self.desc = d
        self.n = n
        self.hel_sampled = bool(hel_sampled)
        h = ctypes.c_void_p()
        _check(lib().bg_plan_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h

    @property
    def workspace_bytes(self) -> int:
        return int(lib().bg_plan_workspace_bytes(self._h))

    def me2(self, u, hel=None, colors=None, out=None, stream=None, wait=True):
        """u [B, 4(n-2)] float64, hel [n, B] int8 (device or host tensors or
        numpy arrays) -> me2 [B] float64 (on the device of `out`, or a new
        CUDA tensor if out is None).  wait=False: bg_me2_batch_async (a host
        `out` is valid after the stream completes; use pinned buffers)."""
        B = u.shape[0]
        if out is None:
            out = torch.empty((B,), dtype=torch.float64, device="cuda")
        if wait:
            _check(lib().bg_me2_batch(self._h, B, _vptr(u), _vptr(hel), _vptr(colors), _vptr(out), _stream(stream)))
        else:
            _check(lib().bg_me2_batch_async(self._h, B, _vptr(u), _vptr(hel), _vptr(out), _stream(stream)))
        return out

    def grad(self, u: torch.Tensor, hel: torch.Tensor, upstream: torch.Tensor | None = None,
             me2: torch.Tensor | None = None, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """d|M|^2/du (times `upstream`) for u [B, 4(n-2)] float64 CUDA, hel
        [n, B] int8 CUDA; optionally also writes |M|^2 into `me2`."""
        B = u.shape[0]
        if out is None:
            out = torch.empty_like(u)
        _check(lib().bg_me2_grad(self._h, B, _vptr(u), _vptr(hel), _vptr(upstream), _vptr(me2), _vptr(out),
                                 _stream(stream)))
        return out

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().bg_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class _DeviceArray:
    """A plan-owned device buffer exposed through __cuda_array_interface__
    (torch.as_tensor makes a view without copying)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


class Mixed:
    """Mixed-multiplicity batches in one CUDA-graph launch (bg_mixed_*).
    The inputs live in plan-owned device buffers, exposed as tensors:
    n_per_event [max_batch] int32, u [max_batch, 4(n_max-2)] float64,
    hel [n_max, max_batch] int8, colors [2 n_max, max_batch] int8, and the
    output me2 [max_batch] float64."""

    def __init__(self, n_min: int, n_max: int, max_batch: int, sqrt_s: float = 1000.0, pt_min: float = -1.0,
                 g_s: float = G_S_DEFAULT, q=DEFAULT_Q, prec: int = BG_F32, cs_mode: int = BG_CS_F32,
                 color_mode: int = BG_COL_ADJOINT, n_co_max: int = 9, chunk_bytes: int = 0,
                 autotune: bool = False):
        d = MixedDesc()
        d.n_min, d.n_max, d.max_batch, d.sqrt_s, d.pt_min, d.g_s = n_min, n_max, max_batch, sqrt_s, pt_min, g_s
        for i in range(4):
            d.q[i] = float(q[i])
        d.prec, d.cs_mode, d.color_mode, d.n_co_max, d.chunk_bytes = prec, cs_mode, color_mode, n_co_max, chunk_bytes
        d.autotune = int(autotune)
        self.desc = d
        h = ctypes.c_void_p()
        _check(lib().bg_mixed_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        ptrs = [ctypes.c_void_p() for _ in range(5)]
        _check(lib().bg_mixed_buffers(h, *[ctypes.byref(x) for x in ptrs]))
        dev = torch.device("cuda", torch.cuda.current_device())
        shapes = [((max_batch,), "<i4"), ((max_batch, 4 * (n_max - 2)), "<f8"), ((n_max, max_batch), "|i1"),
                  ((2 * n_max, max_batch), "|i1"), ((max_batch,), "<f8")]
        views = [torch.as_tensor(_DeviceArray(p.value, sh, ts), device=dev) for p, (sh, ts) in zip(ptrs, shapes)]
        self.n_per_event, self.u, self.hel, self.colors, self.me2 = views

    @property
    def workspace_bytes(self) -> int:
        return int(lib().bg_mixed_workspace_bytes(self._h))

    def run(self, B: int, stream=None) -> torch.Tensor:
        """Replays the graph for the first B events; returns the me2 view."""
        _check(lib().bg_mixed_run(self._h, B, _stream(stream)))
        return self.me2[:B]

    def counts(self) -> list[int]:
        c = (ctypes.c_int64 * 13)()
        _check(lib().bg_mixed_counts(self._h, c))
        return list(c)

    def kernel_nodes(self) -> int:
        """Kernels one run launches (the kernel nodes of the plan's graph)."""
        k = ctypes.c_int64()
        _check(lib().bg_mixed_kernel_nodes(self._h, ctypes.byref(k)))
        return k.value

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self.n_per_event = self.u = self.hel = self.colors = self.me2 = None
            lib().bg_mixed_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class Me2Function(torch.autograd.Function):
    """|M|^2(u) as a differentiable function of the Rambo uniforms: forward
    runs bg_me2_batch, backward bg_me2_grad with the incoming gradient."""

    @staticmethod
    def forward(ctx, u, hel, plan):
        ctx.plan = plan
        ctx.save_for_backward(u, hel)
        return plan.me2(u.contiguous(), hel)

    @staticmethod
    def backward(ctx, grad_out):
        u, hel = ctx.saved_tensors
        g = ctx.plan.grad(u.contiguous(), hel, upstream=grad_out.contiguous())
        return g, None, None


def me2_autograd(u: torch.Tensor, hel: torch.Tensor, plan: "Plan") -> torch.Tensor:
    return Me2Function.apply(u, hel, plan)


def _vptr(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        assert x.is_contiguous()
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)  # numpy array (host memory)


def tune_num_variants(algo: int, n: int) -> int:
    return int(lib().bg_tune_num_variants(algo, n))


def autotune(algo: int, n: int, prec: int = BG_F32, probe_batch: int = 0, stream=None):
    """Times every kernel variant of (algo, n, prec), records the fastest for
    the current device; returns (best variant, [ms per variant])."""
    nv = tune_num_variants(algo, n)
    ms = (ctypes.c_float * max(nv, 1))()
    best = ctypes.c_int(-1)
    _check(lib().bg_autotune(algo, n, prec, probe_batch, _stream(stream), ctypes.byref(best), ms))
    return best.value, [float(ms[i]) for i in range(nv)]


def tune_set(algo: int, n: int, prec: int, variant: int) -> None:
    _check(lib().bg_tune_set(algo, n, prec, variant))


def tune_get(algo: int, n: int, prec: int) -> int:
    v = ctypes.c_int(-1)
    _check(lib().bg_tune_get(algo, n, prec, ctypes.byref(v)))
    return v.value


def tune_save(path: str) -> None:
    _check(lib().bg_tune_save(path.encode()))


def tune_load(path: str) -> None:
    _check(lib().bg_tune_load(path.encode()))


def device_status() -> int:
    s = ctypes.c_int(0)
    _check(lib().bg_device_status(ctypes.byref(s)))
    return s.value


def device_status_reset() -> None:
    _check(lib().bg_device_status_reset())
