"""bg_me2_batch_noalloc: the |M|^2 pipeline for callers that cannot allocate
device memory (its intermediate buffers sit in a fixed array of device memory
inside the library).  Called through the C ABI and compared with the
allocating entry point bg_me2_batch on the same inputs, for two calls in a
row, within the FP64 parity tolerance of the other tests (1e-12 relative; the
two paths run the same kernels, so the results are expected to be equal); at
the largest batch the fixed array holds; and with an invalid helicity label,
which the device status word must report.  This file is collected last on
purpose."""
import ctypes

import numpy as np
import pytest

from paper_2106_06507_gb300 import inputs

pytestmark = pytest.mark.gpu

SQRT_S = 1000.0
PT_MIN = 20.0


@pytest.fixture(scope="module")
def bg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_06507_gb300 import bg as _bg, build_lib
    build_lib.build()
    L = _bg.lib()
    vp, c_i64, c_dbl, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    L.bg_me2_batch_noalloc.argtypes = [vp, c_i64, c_dbl, c_dbl, c_dbl, ctypes.POINTER(c_dbl), c_int, c_int, vp, vp,
                                       vp, vp]
    L.bg_me2_batch_noalloc.restype = c_int
    return _bg


def noalloc(bg, C, B, u, hel, out, prec, cs_mode, pt_min):
    import torch
    q = (ctypes.c_double * 4)(*bg.DEFAULT_Q)
    return bg.lib().bg_me2_batch_noalloc(C.handle, B, SQRT_S, pt_min, bg.G_S_DEFAULT, q, prec, cs_mode,
                                         ctypes.c_void_p(u.data_ptr()),
                                         None if hel is None else ctypes.c_void_p(hel.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("n,prec_name,cs_name,sampled,sizes", [
    (6, "BG_F32", "BG_CS_TC_BF16", True, (2500, 1300)),
    (4, "BG_F64", "BG_CS_F64", False, (999, 500)),
])
def test_noalloc_matches_allocating_entry_point(bg, n, prec_name, cs_name, sampled, sizes):
    import torch
    dev = torch.device("cuda:0")
    prec, cs_mode = getattr(bg, prec_name), getattr(bg, cs_name)
    pt_min = PT_MIN if sampled else -1.0
    C = bg.ColourMatrix(n)
    plan = bg.Plan(n, max(sizes), SQRT_S, pt_min, prec=prec, cs_mode=cs_mode, hel_sampled=sampled)
    for call, B in enumerate(sizes):  # two calls in a row, different inputs
        u = torch.from_numpy(inputs.rambo_uniforms(n, B, seed=60 + call)).to(dev)
        hel = None
        if sampled:
            hel = torch.from_numpy(np.ascontiguousarray(inputs.helicities(n, B, seed=60 + call).T)).to(dev)
        ref = plan.me2(u, hel).cpu().numpy()
        out = torch.full((B,), -1.0, dtype=torch.float64, device=dev)
        assert noalloc(bg, C, B, u, hel, out, prec, cs_mode, pt_min) == bg.BG_OK, bg.lib().bg_last_error()
        got = out.cpu().numpy()
        assert np.array_equal(got == 0, ref == 0)
        nz = ref != 0
        assert np.all(np.abs(got[nz] / ref[nz] - 1.0) <= 1e-12)
    plan.close()
    C.close()


def noalloc_max_events(n, k, amp_bytes, H):
    # the library's own sizing rule: momenta [4][n][B] double, amplitudes
    # [B][H][k], cut flags [B], each region padded to 256 bytes
    per_event = 4 * n * 8 + H * k * amp_bytes + 1
    return ((64 << 20) - 3 * 256) // per_event


def test_noalloc_at_its_largest_batch(bg):
    # n = 8, FP32 amplitudes, sampled helicities: the batch that fills the
    # fixed array (21392 events) matches the plan path; one more is rejected
    import torch
    dev = torch.device("cuda:0")
    n = 8
    B = noalloc_max_events(n, 720, 4, 1)
    assert B == 21392
    C = bg.ColourMatrix(n)
    plan = bg.Plan(n, B + 1, SQRT_S, PT_MIN, prec=bg.BG_F32, cs_mode=bg.BG_CS_TC_BF16, hel_sampled=True)
    u = torch.from_numpy(inputs.rambo_uniforms(n, B + 1, seed=62)).to(dev)
    hel = torch.from_numpy(np.ascontiguousarray(inputs.helicities(n, B + 1, seed=62).T)).to(dev)
    ref = plan.me2(u[:B], hel[:, :B].contiguous()).cpu().numpy()
    out = torch.full((B + 1,), -1.0, dtype=torch.float64, device=dev)
    hb = hel[:, :B].contiguous()
    assert noalloc(bg, C, B, u, hb, out, bg.BG_F32, bg.BG_CS_TC_BF16, PT_MIN) == bg.BG_OK
    got = out[:B].cpu().numpy()
    assert out[B].item() == -1.0  # nothing written past the batch
    assert np.array_equal(got == 0, ref == 0)
    nz = ref != 0
    assert np.all(np.abs(got[nz] / ref[nz] - 1.0) <= 1e-12)
    assert noalloc(bg, C, B + 1, u, hel, out, bg.BG_F32, bg.BG_CS_TC_BF16, PT_MIN) == bg.BG_EINVAL
    assert f"at most {B} events" in bg.lib().bg_last_error().decode()
    plan.close()
    C.close()


def test_noalloc_reports_invalid_helicity_label(bg):
    import torch
    dev = torch.device("cuda:0")
    n, B = 7, 400
    C = bg.ColourMatrix(n)
    u = torch.from_numpy(inputs.rambo_uniforms(n, B, seed=63)).to(dev)
    hel = torch.from_numpy(np.ascontiguousarray(inputs.helicities(n, B, seed=63).T)).to(dev)
    out = torch.zeros((B,), dtype=torch.float64, device=dev)
    bg.device_status_reset()
    assert noalloc(bg, C, B, u, hel, out, bg.BG_F32, bg.BG_CS_TC_BF16, PT_MIN) == bg.BG_OK
    assert bg.device_status() == 0
    hel[2, 5] = -2
    assert noalloc(bg, C, B, u, hel, out, bg.BG_F32, bg.BG_CS_TC_BF16, PT_MIN) == bg.BG_OK
    assert bg.device_status() == bg.BG_EINVAL
    bg.device_status_reset()
    C.close()


def test_noalloc_rejects_batches_beyond_its_fixed_scratch(bg):
    import torch
    n = 8
    C = bg.ColourMatrix(n)
    u = torch.zeros((1, 4 * (n - 2)), dtype=torch.float64, device="cuda")
    out = torch.zeros((1,), dtype=torch.float64, device="cuda")
    hel = torch.ones((n, 1), dtype=torch.int8, device="cuda")
    rc = noalloc(bg, C, 10**6, u, hel, out, bg.BG_F32, bg.BG_CS_TC_BF16, PT_MIN)
    assert rc == bg.BG_EINVAL
    msg = bg.lib().bg_last_error().decode()
    assert "at most" in msg and "MiB" in msg
    C.close()
