"""Failure paths on the GPU machine, made on the host (no GPU fault):

- every device allocation of bg_colormat_create, bg_plan_create and
  bg_mixed_create in turn is made to fail (BG_FAIL_ALLOC=k): the call
  returns BG_ENOMEM, leaves its output NULL and frees what it had allocated
  (the device's free memory is unchanged), and with k past the last
  allocation the call succeeds;
- an invalid helicity label is recorded in the device status word by the
  plan path."""
import numpy as np
import pytest

from paper_2106_06507_gb300 import inputs

pytestmark = pytest.mark.gpu

LEAK_TOL = 8 << 20  # bytes: the driver's bookkeeping, far below any plan buffer


@pytest.fixture(scope="module")
def bg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_06507_gb300 import bg as _bg, build_lib
    build_lib.build()
    _bg.lib()
    return _bg


def free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def each_allocation_fails(monkeypatch, bg, create, max_k=120):
    """create() raises BGError(BG_ENOMEM) for k = 1.. until it succeeds."""
    base = free_bytes()
    for k in range(1, max_k + 1):
        monkeypatch.setenv("BG_FAIL_ALLOC", str(k))
        try:
            obj = create()
        except bg.BGError as e:
            assert e.code == bg.BG_ENOMEM, (k, str(e))
            assert "device allocation failed" in str(e)
            assert abs(free_bytes() - base) <= LEAK_TOL, k
            continue
        monkeypatch.delenv("BG_FAIL_ALLOC")
        obj.close()
        assert abs(free_bytes() - base) <= LEAK_TOL
        return k - 1
    raise AssertionError("create() never succeeded")


def test_colormat_create_every_allocation(bg, monkeypatch):
    # n = 8: C in FP64 and FP32 and the tensor-core tiles
    assert each_allocation_fails(monkeypatch, bg, lambda: bg.ColourMatrix(8)) == 3


def test_plan_create_every_allocation(bg, monkeypatch):
    # large enough that a leaked buffer shows in the device's free memory
    def make():
        return bg.Plan(7, 1 << 18, 1000.0, 20.0, prec=bg.BG_F32, cs_mode=bg.BG_CS_TC_BF16, hel_sampled=True,
                       grad=True)
    assert each_allocation_fails(monkeypatch, bg, make) >= 10


def test_mixed_create_every_allocation(bg, monkeypatch):
    def make():
        # colour-ordered branches n = 4..7, colour-dressed n = 8..11 (74
        # allocations; the n = 9 colour matrix is left out to keep it quick)
        return bg.Mixed(4, 11, 1 << 16, 1000.0, 20.0, prec=bg.BG_F32, cs_mode=bg.BG_CS_TC_BF16,
                        color_mode=bg.BG_COL_ADJOINT, n_co_max=7)
    assert each_allocation_fails(monkeypatch, bg, make) >= 60


def test_plan_reports_invalid_helicity_label(bg):
    import torch
    n, B = 6, 300
    plan = bg.Plan(n, B, 1000.0, 20.0, prec=bg.BG_F32, cs_mode=bg.BG_CS_TC_BF16, hel_sampled=True)
    u = torch.from_numpy(inputs.rambo_uniforms(n, B, seed=70)).cuda()
    hel = torch.from_numpy(np.ascontiguousarray(inputs.helicities(n, B, seed=70).T)).cuda()
    bg.device_status_reset()
    plan.me2(u, hel)
    assert bg.device_status() == 0
    hel[3, 17] = 2
    plan.me2(u, hel)
    assert bg.device_status() == bg.BG_EINVAL
    bg.device_status_reset()
    plan.close()
