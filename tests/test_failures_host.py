"""Failure paths of the create calls, reached on the host without a GPU.

The library routes every device allocation of bg_colormat_create,
bg_plan_create, bg_mixed_create and bg_autotune through one function that
fails, without allocating, on the k-th allocation of a create call when the
environment variable BG_FAIL_ALLOC=k is set.  With k = 1 the first allocation
fails before any device is touched, so these tests run on a machine without
a GPU: each create call must return BG_ENOMEM, leave its output NULL and set
a message.  (The GPU tests repeat this for every k, with a leak check.)"""
import ctypes

import pytest

BG_ENOMEM = 2


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


@pytest.fixture(scope="module")
def libbg():
    from paper_2106_06507_gb300 import build_lib
    L = ctypes.CDLL(build_lib.build())
    L.bg_last_error.restype = ctypes.c_char_p
    L.bg_colormat_create.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    L.bg_plan_create.argtypes = [ctypes.POINTER(PlanDesc), ctypes.POINTER(ctypes.c_void_p)]
    L.bg_mixed_create.argtypes = [ctypes.POINTER(MixedDesc), ctypes.POINTER(ctypes.c_void_p)]
    return L


@pytest.fixture
def fail_first_alloc(monkeypatch):
    monkeypatch.setenv("BG_FAIL_ALLOC", "1")


def q_light_like(d):
    for i, v in enumerate((1.0, 0.0, 0.0, 1.0)):
        d.q[i] = v


@pytest.mark.parametrize("n", [4, 6, 9])
def test_colormat_create_reports_enomem(libbg, fail_first_alloc, n):
    out = ctypes.c_void_p(12345)
    assert libbg.bg_colormat_create(n, ctypes.byref(out)) == BG_ENOMEM
    assert not out.value
    assert b"device allocation failed" in libbg.bg_last_error()


@pytest.mark.parametrize("n,grad", [(5, 0), (8, 1)])
def test_plan_create_reports_enomem(libbg, fail_first_alloc, n, grad):
    d = PlanDesc(n=n, max_batch=1024, sqrt_s=1000.0, pt_min=20.0, g_s=1.2, prec=1, cs_mode=1, algo=0,
                 color_mode=0, hel_sampled=1, grad=grad)
    q_light_like(d)
    out = ctypes.c_void_p(12345)
    assert libbg.bg_plan_create(ctypes.byref(d), ctypes.byref(out)) == BG_ENOMEM
    assert not out.value
    assert b"device allocation failed" in libbg.bg_last_error()


def test_mixed_create_reports_enomem(libbg, fail_first_alloc):
    d = MixedDesc(n_min=4, n_max=12, max_batch=4096, sqrt_s=1000.0, pt_min=20.0, g_s=1.2, prec=1, cs_mode=1,
                  color_mode=0, n_co_max=9, chunk_bytes=0, autotune=0)
    q_light_like(d)
    out = ctypes.c_void_p(12345)
    assert libbg.bg_mixed_create(ctypes.byref(d), ctypes.byref(out)) == BG_ENOMEM
    assert not out.value


def test_argument_errors_come_before_allocation(libbg, fail_first_alloc):
    # an invalid descriptor is BG_EINVAL even when an allocation would fail
    d = PlanDesc(n=3, max_batch=1024, sqrt_s=1000.0, pt_min=20.0, g_s=1.2, prec=1, cs_mode=1, algo=0,
                 color_mode=0, hel_sampled=1, grad=0)
    q_light_like(d)
    out = ctypes.c_void_p()
    assert libbg.bg_plan_create(ctypes.byref(d), ctypes.byref(out)) == 1
