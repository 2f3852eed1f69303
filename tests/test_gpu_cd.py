"""GPU parity of the colour-dressed recursion with sampled colours
(bg_currents_cd) against the oracle on identical host-generated inputs, and
the brute-force identity sum over all colours = colour-ordered |M|^2 on the
GPU itself.

Colour assignments whose amplitude vanishes by colour algebra come out as
rounding noise (~1e-33 of a typical |M|^2 in FP64) rather than exactly 0:
events whose reference value is below 1e-16 of the batch's largest |M|^2 are
treated as zeros and must stay below 1e-10 (FP64) or 1e-6 (FP32: the squared
FP32 noise of an amplitude that cancels) of it.

Tolerances (derived in the design notes):
  FP64: compared with the oracle in extended precision; as accurate as the
  plain FP64 oracle (median below max(1e-13, 8x the FP64 oracle's median), events above 1e-12 at most 2 + 4x
  the FP64 oracle's count, worst within max(5e-11, 8x the FP64 oracle's)).
  FP32: median relative error < 1e-5; 99% of events within 1e-3 of
  max(|M|^2, 1e-2 x the sample's median |M|^2).  The colour-dressed
  amplitude of one colour sample is a sum of many colour-ordered amplitudes
  with colour weights of both signs, so cancellations amplify FP32 rounding
  more than in the colour-summed |M|^2; an event whose amplitude cancels to
  a small fraction of the typical one keeps an absolute error of the size of
  the cancelling terms.
"""
import itertools

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


def run_cd(bg, n, u, hel, cols, flow, prec, pt_min=PT_MIN):
    import torch
    dev = torch.device("cuda:0")
    p, acc = bg.momenta_rambo(n, torch.from_numpy(u).to(dev), SQRT_S, pt_min)
    h = torch.from_numpy(np.ascontiguousarray(hel.T)).to(dev)
    c = torch.from_numpy(np.ascontiguousarray(cols.T)).to(dev)
    return bg.currents_cd(n, p, h, c, flow=flow, prec=prec, sqrt_s=SQRT_S, accept=acc).cpu().numpy()


def colours(n, B, seed, flow):
    return inputs.flow_colours(n, B, seed=seed) if flow else inputs.adjoint_colours(n, B, seed=seed)


def split_zeros(got, ref, tol=1e-10):
    """Mask of the events that are not structural zeros; checks the zeros."""
    scale = ref.max() if ref.size and ref.max() > 0 else 1.0
    zero = ref <= 1e-16 * scale
    assert np.all(np.abs(got[zero]) <= tol * scale)
    return ~zero


def fp32_rel(got, ref):
    """Error of FP32 results relative to max(|M|^2, 1e-2 x the sample's median
    |M|^2): an event whose amplitude cancels to a small fraction of the
    typical amplitude keeps an absolute FP32 error of the size of the terms
    that cancel, so its own relative error is unbounded."""
    return np.abs(got - ref) / np.maximum(ref, 1e-2 * np.median(ref))


def assert_fp64_like(got, ext, f64):
    nz = split_zeros(got, ext)
    if not nz.any():
        return
    rel = np.abs(got[nz] / ext[nz] - 1.0)
    floor = np.abs(f64[nz] / ext[nz] - 1.0)
    assert np.median(rel) <= max(1e-13, 8.0 * np.median(floor))
    assert np.sum(rel > 1e-12) <= 2 + 4 * np.sum(floor > 1e-12)
    assert rel.max() <= max(5e-11, 8.0 * floor.max())


@pytest.mark.parametrize("flow", [False, True])
@pytest.mark.parametrize("n,B", [(4, 301), (5, 300), (6, 200), (7, 120), (8, 60)])
def test_cd_fp64_parity(bg, oracle, n, B, flow):
    # only 3-7 % of sampled colour flows are balanced (others give exactly 0)
    B = 20 * B if flow else B
    u = inputs.rambo_uniforms(n, B, seed=70 + n)
    hel = inputs.helicities(n, B, seed=70 + n)
    cols = colours(n, B, 70 + n, flow)
    got = run_cd(bg, n, u, hel, cols, flow, bg.BG_F64)
    mode = 1 if flow else 0
    ext = oracle.me2_cd(n, u, hel, cols, mode, sqrt_s=SQRT_S, pt_min=PT_MIN, ext=True)
    f64 = oracle.me2_cd(n, u, hel, cols, mode, sqrt_s=SQRT_S, pt_min=PT_MIN)
    assert_fp64_like(got, ext, f64)


@pytest.mark.parametrize("flow", [False, True])
@pytest.mark.parametrize("n,B", [(6, 400), (8, 200), (10, 64), (12, 96)])
def test_cd_fp32_parity(bg, oracle, n, B, flow):
    # colour flows drawn balanced (unbalanced ones give exactly 0); no cut, so
    # that the few-event high-multiplicity samples have non-zero |M|^2 (at
    # n = 12 only ~6 % of adjoint colour samples do)
    u = inputs.rambo_uniforms(n, B, seed=80 + n)
    hel = inputs.helicities(n, B, seed=80 + n)
    cols = inputs.balanced_flow_colours(n, B, seed=80 + n) if flow else colours(n, B, 80 + n, False)
    got = run_cd(bg, n, u, hel, cols, flow, bg.BG_F32, pt_min=-1.0)
    ref = oracle.me2_cd(n, u, hel, cols, 1 if flow else 0, sqrt_s=SQRT_S, pt_min=-1.0)
    nz = split_zeros(got, ref, tol=1e-6)
    assert nz.sum() >= 2
    assert np.median(np.abs(got[nz] / ref[nz] - 1.0)) < 1e-5
    rel = fp32_rel(got[nz], ref[nz])
    assert np.quantile(rel, 0.99) < 1e-3


@pytest.mark.parametrize("flow", [False, True])
def test_cd_fp64_n10(bg, oracle, flow):
    n, B = 10, 64
    u = inputs.rambo_uniforms(n, B, seed=90)
    hel = inputs.helicities(n, B, seed=90)
    cols = inputs.balanced_flow_colours(n, B, seed=90) if flow else colours(n, B, 90, False)
    got = run_cd(bg, n, u, hel, cols, flow, bg.BG_F64, pt_min=-1.0)
    mode = 1 if flow else 0
    ext = oracle.me2_cd(n, u, hel, cols, mode, sqrt_s=SQRT_S, pt_min=-1.0, ext=True)
    f64 = oracle.me2_cd(n, u, hel, cols, mode, sqrt_s=SQRT_S, pt_min=-1.0)
    assert (ext > 1e-16 * ext.max()).sum() >= 2
    assert_fp64_like(got, ext, f64)


@pytest.mark.parametrize("flow", [False, True])
def test_cd_sum_over_all_colours_equals_colour_ordered(bg, flow):
    # sum over every colour assignment of the CD estimator / (number of
    # assignments) = the colour-summed |M|^2 of the colour-ordered path
    import torch
    n = 4
    u1 = inputs.rambo_uniforms(n, 1, seed=95)
    h1 = inputs.helicities(n, 1, seed=95)
    cols = np.array(list(itertools.product(range(1, 4), repeat=2 * n) if flow
                         else itertools.product(range(1, 9), repeat=n)), dtype=np.int8)
    B = cols.shape[0]
    est = run_cd(bg, n, np.repeat(u1, B, axis=0), np.repeat(h1, B, axis=0), cols, flow, bg.BG_F64, pt_min=-1.0)
    C = bg.ColourMatrix(n)
    dev = torch.device("cuda:0")
    p, _ = bg.momenta_rambo(n, torch.from_numpy(u1).to(dev), SQRT_S)
    amps = bg.currents_co(n, p, torch.from_numpy(np.ascontiguousarray(h1.T)).to(dev), prec=bg.BG_F64,
                          sqrt_s=SQRT_S)
    co = bg.color_sum(C, amps, True, mode=bg.BG_CS_F64, sqrt_s=SQRT_S).cpu().numpy()[0]
    assert abs(est.mean() / co - 1.0) < 1e-11
    C.close()


def test_cd_edge_cases(bg):
    import torch
    dev = torch.device("cuda:0")
    n = 6
    # empty batch
    z = torch.zeros((4, n, 0), dtype=torch.float64, device=dev)
    out = bg.currents_cd(n, z, torch.zeros((n, 0), dtype=torch.int8, device=dev),
                         torch.zeros((n, 0), dtype=torch.int8, device=dev))
    assert out.numel() == 0
    # an unbalanced colour flow gives exactly zero
    u = inputs.rambo_uniforms(n, 1, seed=96)
    hel = np.ones((1, n), dtype=np.int8)
    cols = np.array([[1, 2] * n], dtype=np.int8)  # every gluon |1><2|
    assert run_cd(bg, n, u, hel, cols, True, bg.BG_F32)[0] == 0.0
    # invalid colour label -> device status
    bg.device_status_reset()
    cols = np.full((1, n), 9, dtype=np.int8)
    run_cd(bg, n, u, hel, cols, False, bg.BG_F32)
    assert bg.device_status() == bg.BG_EINVAL
    bg.device_status_reset()
    # workspace too small
    p, acc = bg.momenta_rambo(n, torch.from_numpy(u).to(dev), SQRT_S)
    ws = torch.empty(16, dtype=torch.uint8, device=dev)
    with pytest.raises(bg.BGError) as ei:
        bg.currents_cd(n, p, torch.ones((n, 1), dtype=torch.int8, device=dev),
                       torch.ones((n, 1), dtype=torch.int8, device=dev), workspace=ws)
    assert ei.value.code == bg.BG_EINVAL


# --------------------------------------------------------------------------
# continuous colour and helicity sampling (Sec. 2.1)
# --------------------------------------------------------------------------
def run_cd_cont(bg, n, u, ang, prec, pt_min=PT_MIN):
    import torch
    dev = torch.device("cuda:0")
    p, acc = bg.momenta_rambo(n, torch.from_numpy(u).to(dev), SQRT_S, pt_min)
    a = torch.from_numpy(np.ascontiguousarray(ang.reshape(ang.shape[0], 5 * n).T)).to(dev)
    return bg.currents_cd_cont(n, p, a, prec=prec, sqrt_s=SQRT_S, accept=acc).cpu().numpy()


@pytest.mark.parametrize("n,B", [(4, 300), (5, 300), (6, 200), (7, 120), (8, 60)])
def test_cd_cont_fp64_parity(bg, oracle, n, B):
    u = inputs.rambo_uniforms(n, B, seed=200 + n)
    ang = inputs.continuous_angles(n, B, seed=200 + n)
    got = run_cd_cont(bg, n, u, ang, bg.BG_F64)
    ext = oracle.me2_cd_cont(n, u, ang, sqrt_s=SQRT_S, pt_min=PT_MIN, ext=True)
    f64 = oracle.me2_cd_cont(n, u, ang, sqrt_s=SQRT_S, pt_min=PT_MIN)
    assert_fp64_like(got, ext, f64)


@pytest.mark.parametrize("n,B", [(6, 400), (8, 200), (10, 64), (12, 24)])
def test_cd_cont_fp32_parity(bg, oracle, n, B):
    u = inputs.rambo_uniforms(n, B, seed=210 + n)
    ang = inputs.continuous_angles(n, B, seed=210 + n)
    got = run_cd_cont(bg, n, u, ang, bg.BG_F32, pt_min=-1.0)
    ref = oracle.me2_cd_cont(n, u, ang, sqrt_s=SQRT_S, pt_min=-1.0)
    nz = split_zeros(got, ref, tol=1e-6)
    assert nz.sum() >= B // 2
    # continuous colour vectors make every colour structure of the amplitude
    # contribute (no zero entries), with both signs: at n >= 10 the
    # cancellation leaves a median FP32 error of ~1.5e-5
    med = 1e-5 if n <= 9 else 5e-5
    assert np.median(np.abs(got[nz] / ref[nz] - 1.0)) < med
    assert np.quantile(fp32_rel(got[nz], ref[nz]), 0.99) < 1e-3


def test_cd_cont_design_average_equals_colour_ordered(bg):
    # exact average over colour vectors from the cube design (4 x 4 per
    # gluon) at polarisation angle 0 = the GPU's colour-ordered |M|^2 with the
    # colour sum, for e1 on every gluon
    import math
    import torch
    n = 4
    cube = np.array([[1, 1, 1], [1, 1, -1], [1, -1, 1], [-1, 1, 1]], dtype=np.float64) / math.sqrt(3.0)
    ang1 = [(v[0], math.atan2(v[2], v[1])) for v in cube]
    states = np.array([[a[0], a[1], b[0], b[1], 0.0] for a in ang1 for b in ang1])
    combos = np.array(list(itertools.product(range(len(states)), repeat=n)))
    A = states[combos]
    u1 = inputs.rambo_uniforms(n, 1, seed=220)
    est = run_cd_cont(bg, n, np.repeat(u1, A.shape[0], axis=0), A, bg.BG_F64, pt_min=-1.0)
    dev = torch.device("cuda:0")
    C = bg.ColourMatrix(n)
    p, _ = bg.momenta_rambo(n, torch.from_numpy(u1).to(dev), SQRT_S)
    amps = bg.currents_co(n, p, torch.ones((n, 1), dtype=torch.int8, device=dev), prec=bg.BG_F64, sqrt_s=SQRT_S)
    co = bg.color_sum(C, amps, True, mode=bg.BG_CS_F64, sqrt_s=SQRT_S).cpu().numpy()[0]
    C.close()
    assert abs(est.mean() / co - 1.0) < 1e-11
