"""GPU parity of the leading-colour |M|^2 (bg_currents_lc, Sec. 4) against
the oracle on identical host-generated inputs; at n = 4, 5, where the
leading-colour formula is exact, against the GPU's own colour-summed path.

The leading-colour sum is a sum of squares (no cancellation), so the
tolerances are those of a single colour-ordered amplitude squared: FP64
within 1e-11 relative per event (median < 1e-13), FP32 median < 2e-6 and
worst < 1e-3 (the FP32 recursion's own spread, as in test_gpu_co.py).
"""
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
    _bg.lib()
    return _bg


def run(bg, n, u, hel, prec, pt_min=PT_MIN):
    import torch
    dev = torch.device("cuda:0")
    p, acc = bg.momenta_rambo(n, torch.from_numpy(u).to(dev), SQRT_S, pt_min)
    h = None if hel is None else torch.from_numpy(np.ascontiguousarray(hel.T)).to(dev)
    return bg.currents_lc(n, p, h, prec=prec, sqrt_s=SQRT_S, accept=acc).cpu().numpy()


@pytest.mark.parametrize("n,B", [(4, 300), (5, 300), (6, 200), (7, 100), (8, 30)])
def test_lc_fp64_parity(bg, oracle, n, B):
    u = inputs.rambo_uniforms(n, B, seed=160 + n)
    hel = inputs.helicities(n, B, seed=160 + n)
    got = run(bg, n, u, hel, bg.BG_F64)
    ref = oracle.me2_lc(n, u, hel=hel, sqrt_s=SQRT_S, pt_min=PT_MIN)
    assert np.all(got[ref == 0] == 0.0)
    nz = ref > 0
    assert nz.sum() >= B // 4
    rel = np.abs(got[nz] / ref[nz] - 1.0)
    assert np.median(rel) < 1e-13 and rel.max() < 1e-11


@pytest.mark.parametrize("n,B", [(6, 1000), (8, 200), (9, 20)])
def test_lc_fp32_parity(bg, oracle, n, B):
    u = inputs.rambo_uniforms(n, B, seed=170 + n)
    hel = inputs.helicities(n, B, seed=170 + n)
    got = run(bg, n, u, hel, bg.BG_F32)
    ref = oracle.me2_lc(n, u, hel=hel, sqrt_s=SQRT_S, pt_min=PT_MIN)
    assert np.all(got[ref == 0] == 0.0)
    nz = ref > 0
    rel = np.abs(got[nz] / ref[nz] - 1.0)
    assert np.median(rel) < 2e-6 and rel.max() < 1e-3


@pytest.mark.parametrize("n", [4, 5])
def test_lc_exact_at_four_and_five_gluons(bg, oracle, n):
    # helicity-summed: the leading-colour formula equals the colour sum
    import torch
    dev = torch.device("cuda:0")
    B = 64
    u = inputs.rambo_uniforms(n, B, seed=180 + n)
    got = run(bg, n, u, None, bg.BG_F64, pt_min=-1.0)
    C = bg.ColourMatrix(n)
    p, _ = bg.momenta_rambo(n, torch.from_numpy(u).to(dev), SQRT_S)
    amps = bg.currents_co(n, p, None, prec=bg.BG_F64, sqrt_s=SQRT_S)
    co = bg.color_sum(C, amps, False, mode=bg.BG_CS_F64, sqrt_s=SQRT_S).cpu().numpy()
    C.close()
    assert np.allclose(got, co, rtol=1e-12, atol=0)
    assert np.allclose(got, oracle.me2_lc(n, u, sqrt_s=SQRT_S), rtol=1e-12, atol=0)


def test_lc_edge_cases(bg):
    import torch
    dev = torch.device("cuda:0")
    n = 6
    z = torch.zeros((4, n, 0), dtype=torch.float64, device=dev)
    assert bg.currents_lc(n, z, torch.zeros((n, 0), dtype=torch.int8, device=dev)).numel() == 0
    u = inputs.rambo_uniforms(n, 4, seed=190)
    hel = inputs.helicities(n, 4, seed=190)
    assert np.all(run(bg, n, u, hel, bg.BG_F32, pt_min=450.0) == 0.0)
    p, _ = bg.momenta_rambo(n, torch.from_numpy(u).to(dev), SQRT_S)
    with pytest.raises(bg.BGError) as ei:
        bg.currents_lc(n, p, None, workspace=torch.empty(16, dtype=torch.uint8, device=dev))
    assert ei.value.code == bg.BG_EINVAL
    with pytest.raises(bg.BGError):
        bg.currents_lc(10, torch.zeros((4, 10, 1), dtype=torch.float64, device=dev), None)
