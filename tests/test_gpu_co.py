"""GPU parity of the colour-ordered path (Rambo -> currents -> colour sum)
against the oracle on identical host-generated inputs.

Tolerances (written here, derived in the design notes):
  FP64 path: |M|^2 is compared with the oracle evaluated in extended
  precision.  The median relative error is below max(1e-13, 8x the plain FP64 oracle's
  median error); the number of events
  above 1e-12 is at most 2 + 4x the number for which the plain FP64 oracle
  itself is above 1e-12 (the GPU sums in a different, equally valid FP64
  order, so its count of ill-conditioned events follows the oracle's; the 2
  covers samples where the oracle has none); the worst event is within
  max(5e-11, 8x the plain FP64 oracle's worst error).  The FP64 evaluation
  of the definition itself loses up to ~2e-11 on ill-conditioned events
  (large cancellations between diagrams), so a per-event 1e-12 bound is not
  a property of FP64 arithmetic; the GPU path is required to be as accurate
  as an FP64 evaluation of the definition.
  Amplitudes agree to 1e-11 of the event's largest ordering amplitude.
  FP32 currents: median relative error below 2e-6, 99.9% of events below
  1e-4, all below 1e-3 (the tail is nearly collinear phase space, where
  cancellations amplify FP32 rounding).
"""
import math

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


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    return torch.device("cuda:0")


def to_dev(x, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


def assert_fp64_parity(oracle, got, n, u, hel, pt_min=-1.0):
    ext = oracle.me2_co_ext(n, u, sqrt_s=SQRT_S, hel=hel, pt_min=pt_min)
    f64 = oracle.me2_co(n, u, sqrt_s=SQRT_S, hel=hel, pt_min=pt_min)
    assert np.array_equal(got == 0, ext == 0)
    nz = ext != 0
    rel = np.abs(got[nz] / ext[nz] - 1.0)
    floor = np.abs(f64[nz] / ext[nz] - 1.0)
    assert np.median(rel) <= max(1e-13, 8.0 * np.median(floor))
    assert np.sum(rel > 1e-12) <= 2 + 4 * np.sum(floor > 1e-12)
    assert rel.max() <= max(5e-11, 8.0 * floor.max())


@pytest.mark.parametrize("n", [4, 5, 6, 8, 10, 12])
def test_rambo_parity(bg, oracle, torch_dev, n):
    B = 1000
    u = inputs.rambo_uniforms(n, B, seed=21)
    p, acc = bg.momenta_rambo(n, to_dev(u, torch_dev), SQRT_S, PT_MIN)
    p = p.cpu().numpy()
    acc = acc.cpu().numpy()
    for e in range(0, B, 7):
        ref = oracle.rambo(n, SQRT_S, u[e])
        assert np.allclose(p[:, :, e].T, ref, rtol=0, atol=1e-12 * SQRT_S)
        pt = np.hypot(ref[2:, 1], ref[2:, 2])
        assert acc[e] == int(np.all(pt > PT_MIN))


@pytest.mark.parametrize("n", [4, 5, 6, 7, 8])
def test_amplitudes_fp64_parity(bg, oracle, torch_dev, n):
    B = {4: 300, 5: 300, 6: 100, 7: 40, 8: 12}[n]
    u = inputs.rambo_uniforms(n, B, seed=22)
    hel = inputs.helicities(n, B, seed=22)
    p, _ = bg.momenta_rambo(n, to_dev(u, torch_dev), SQRT_S)
    amps = bg.currents_co(n, p, to_dev(hel.T, torch_dev), prec=bg.BG_F64, sqrt_s=SQRT_S).cpu().numpy()
    unit = SQRT_S ** (4 - n)
    for e in range(B):
        k = oracle.outgoing(oracle.rambo(n, SQRT_S, u[e]))
        ref = oracle.amps_all(k, oracle.pols_for(k, hel[e]))
        got = amps[e, 0] * unit
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_helicity_summed_fp64_n4_full_config(bg, oracle, torch_dev):
    # gg -> gg, 10^4 Rambo points at sqrt(s) = 1 TeV, all 16 polarisation
    # configurations, exact colour matrix, FP64 (the 4-gluon workload).
    n, B = 4, 10000
    u = inputs.rambo_uniforms(n, B, seed=0)
    C = bg.ColourMatrix(n)
    p, acc = bg.momenta_rambo(n, to_dev(u, torch_dev), SQRT_S)
    amps = bg.currents_co(n, p, None, prec=bg.BG_F64, sqrt_s=SQRT_S)
    assert tuple(amps.shape) == (B, 16, 2)
    me2 = bg.color_sum(C, amps, hel_sampled=False, mode=bg.BG_CS_F64, sqrt_s=SQRT_S).cpu().numpy()
    assert_fp64_parity(oracle, me2, n, u, None)


@pytest.mark.parametrize("n", [5, 6, 7, 8])
def test_me2_fp64_parity_sampled_helicity(bg, oracle, torch_dev, n):
    B = {5: 4001, 6: 1501, 7: 401, 8: 101}[n]  # ragged: not a multiple of the event tile
    u = inputs.rambo_uniforms(n, B, seed=23)
    hel = inputs.helicities(n, B, seed=23)
    C = bg.ColourMatrix(n)
    p, acc = bg.momenta_rambo(n, to_dev(u, torch_dev), SQRT_S, PT_MIN)
    amps = bg.currents_co(n, p, to_dev(hel.T, torch_dev), prec=bg.BG_F64, sqrt_s=SQRT_S)
    me2 = bg.color_sum(C, amps, hel_sampled=True, mode=bg.BG_CS_F64, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    assert_fp64_parity(oracle, me2, n, u, hel, PT_MIN)


@pytest.mark.parametrize("n", [5, 6, 7, 8])
def test_me2_fp32_parity_sampled_helicity(bg, oracle, torch_dev, n):
    B = {5: 4000, 6: 1500, 7: 400, 8: 100}[n]
    u = inputs.rambo_uniforms(n, B, seed=24)
    hel = inputs.helicities(n, B, seed=24)
    C = bg.ColourMatrix(n)
    p, acc = bg.momenta_rambo(n, to_dev(u, torch_dev), SQRT_S, PT_MIN)
    amps = bg.currents_co(n, p, to_dev(hel.T, torch_dev), prec=bg.BG_F32, sqrt_s=SQRT_S)
    ref = oracle.me2_co(n, u, sqrt_s=SQRT_S, hel=hel, pt_min=PT_MIN)
    nz = ref != 0
    for mode in (bg.BG_CS_F32, bg.BG_CS_F64):
        me2 = bg.color_sum(C, amps, hel_sampled=True, mode=mode, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
        assert np.array_equal(me2 == 0, ref == 0)
        rel = np.abs(me2[nz] / ref[nz] - 1.0)
        assert np.median(rel) < 2e-6
        assert np.quantile(rel, 0.999) < 1e-4
        assert rel.max() < 1e-3


def test_edge_cases(bg, torch_dev):
    import torch
    n = 6
    C = bg.ColourMatrix(n)
    # empty batch
    u = torch.empty((0, 4 * (n - 2)), dtype=torch.float64, device=torch_dev)
    p, acc = bg.momenta_rambo(n, u, SQRT_S)
    amps = bg.currents_co(n, p, torch.empty((n, 0), dtype=torch.int8, device=torch_dev), sqrt_s=SQRT_S)
    me2 = bg.color_sum(C, amps, hel_sampled=True, sqrt_s=SQRT_S)
    assert me2.numel() == 0
    # single event, all events rejected by an impossible cut
    u1 = torch.from_numpy(inputs.rambo_uniforms(n, 1, seed=5)).to(torch_dev)
    p1, acc1 = bg.momenta_rambo(n, u1, SQRT_S, pt_min=1e9)
    assert acc1.item() == 0
    hel1 = torch.ones((n, 1), dtype=torch.int8, device=torch_dev)
    me21 = bg.color_sum(C, bg.currents_co(n, p1, hel1, sqrt_s=SQRT_S), True, accept=acc1, sqrt_s=SQRT_S)
    assert me21.item() == 0.0
    # unsupported multiplicity for the colour-ordered path, invalid arguments
    with pytest.raises(bg.BGError) as ei:
        bg.currents_co(10, torch.zeros((4, 10, 1), dtype=torch.float64, device=torch_dev), None)
    assert ei.value.code == bg.BG_EUNSUPPORTED
    with pytest.raises(bg.BGError) as ei:
        bg.currents_co(n, p1, hel1, q=(1.0, 0.0, 0.0, 0.5), sqrt_s=SQRT_S)
    assert ei.value.code == bg.BG_EINVAL


def test_invalid_helicity_label_sets_device_status(bg, torch_dev):
    import torch
    n = 5
    bg.device_status_reset()
    u = torch.from_numpy(inputs.rambo_uniforms(n, 4, seed=6)).to(torch_dev)
    p, _ = bg.momenta_rambo(n, u, SQRT_S)
    hel = torch.ones((n, 4), dtype=torch.int8, device=torch_dev)
    bg.currents_co(n, p, hel, sqrt_s=SQRT_S)
    assert bg.device_status() == 0
    hel[2, 1] = 3
    bg.currents_co(n, p, hel, sqrt_s=SQRT_S)
    assert bg.device_status() == bg.BG_EINVAL
    bg.device_status_reset()
    assert bg.device_status() == 0


def test_colour_matrix_device_row(bg, oracle):
    for n in (4, 6, 8):
        C = bg.ColourMatrix(n)
        assert np.allclose(C.row(), oracle.colour_row(n), rtol=0, atol=1e-6)
        C.close()
