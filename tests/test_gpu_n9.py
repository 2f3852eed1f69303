"""n = 9 (k = 5040 orderings) on the GPU against the oracle.

n = 9 is the largest colour-ordered multiplicity: the (n-2)! = 5040 orderings,
the 5040 x 5040 colour matrix (Eq. 2.17), whose tensor-core form needs two
BF16 planes, and the n <= 9 branch of mixed batches.  The oracle builds the
full matrix from its first row through the relabelling C_{s,t} =
C_{id, s^-1 t} and evaluates the definition (Eq. 2.16) per event.

Tolerances (the same rules as at n <= 8, written here):
  FP64 amplitudes: element-wise within 1e-11 of the event's largest ordering
  amplitude.
  FP64 |M|^2 (FP64 recursion, FP64 colour sum): the FP64 parity rule of
  test_gpu_co.py against the extended-precision oracle.
  FP32 currents + FP64 colour sum: median relative error below 2e-6, all
  below 1e-3 (the FP32 criterion of n <= 8).
  FP32 currents + tensor-core colour sum: the tensor-core rounding bound of
  test_gpu_tc.py at n = 9 (U = 1890 FP32 accumulator updates per element:
  median below 5.7e-5, all below 1.9e-3) on top of the FP32 currents.
Batch 130: two CTAs of the 128-event tensor-core tile, the second ragged
(events 127, 128, 129 sit at the tile edge); 33 events for the FP64 checks."""
import math

import numpy as np
import pytest

from paper_2106_06507_gb300 import inputs

from test_gpu_co import assert_fp64_parity
from test_gpu_tc import tc_tolerances

pytestmark = pytest.mark.gpu

SQRT_S = 1000.0
PT_MIN = 20.0
N = 9


@pytest.fixture(scope="module")
def bg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_06507_gb300 import bg as _bg, build_lib
    build_lib.build()
    _bg.lib()
    return _bg


def dev_arr(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def test_colour_matrix_n9_relabelling(oracle):
    # the dense matrix the oracle uses: symmetric, closed-form diagonal
    # 8 (2N)^(n-2), first row equal to the golden row.  The golden row is the
    # oracle's floating-point SU(3) contraction (8^9 terms per entry), so its
    # integer entries carry rounding of ~1e-16 relative: compare within 1e-13.
    C = oracle.colour_matrix(N)
    assert C.shape == (5040, 5040)
    big = np.abs(C).max()
    assert np.abs(C - C.T).max() <= 1e-13 * big
    assert np.abs(np.diag(C) - 8 * 6 ** 7).max() <= 1e-13 * big
    assert np.array_equal(C[0], oracle.colour_row(N))
    assert np.abs(C - np.round(C)).max() <= 1e-13 * big


def test_amplitudes_fp64_n9(bg, oracle):
    B = 33
    u = inputs.rambo_uniforms(N, B, seed=90)
    hel = inputs.helicities(N, B, seed=90)
    p, _ = bg.momenta_rambo(N, dev_arr(u), SQRT_S)
    amps = bg.currents_co(N, p, dev_arr(hel.T), prec=bg.BG_F64, sqrt_s=SQRT_S).cpu().numpy()
    assert amps.shape == (B, 1, 5040)
    unit = SQRT_S ** (4 - N)
    for e in range(B):
        k = oracle.outgoing(oracle.rambo(N, SQRT_S, u[e]))
        ref = oracle.amps_all(k, oracle.pols_for(k, hel[e]))
        got = amps[e, 0] * unit
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), e


def test_me2_fp64_n9(bg, oracle):
    B = 33
    u = inputs.rambo_uniforms(N, B, seed=91)
    hel = inputs.helicities(N, B, seed=91)
    C = bg.ColourMatrix(N)
    p, acc = bg.momenta_rambo(N, dev_arr(u), SQRT_S, PT_MIN)
    amps = bg.currents_co(N, p, dev_arr(hel.T), prec=bg.BG_F64, sqrt_s=SQRT_S)
    me2 = bg.color_sum(C, amps, True, mode=bg.BG_CS_F64, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    assert_fp64_parity(oracle, me2, N, u, hel, PT_MIN)
    C.close()


def test_me2_fp32_tensor_core_n9(bg, oracle):
    B = 130
    u = inputs.rambo_uniforms(N, B, seed=92)
    hel = inputs.helicities(N, B, seed=92)
    C = bg.ColourMatrix(N)
    p, acc = bg.momenta_rambo(N, dev_arr(u), SQRT_S, PT_MIN)
    amps = bg.currents_co(N, p, dev_arr(hel.T), prec=bg.BG_F32, sqrt_s=SQRT_S)
    ref = oracle.me2_co(N, u, sqrt_s=SQRT_S, hel=hel, pt_min=PT_MIN)
    nz = ref != 0
    assert nz.sum() >= 40
    assert nz[127:130].any()  # tile-edge events take part
    bg.device_status_reset()
    f64 = bg.color_sum(C, amps, True, mode=bg.BG_CS_F64, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    tc = bg.color_sum(C, amps, True, mode=bg.BG_CS_TC_BF16, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    assert bg.device_status() == 0
    for got in (f64, tc):
        assert np.array_equal(got == 0, ref == 0)
    rel64 = np.abs(f64[nz] / ref[nz] - 1.0)
    assert np.median(rel64) < 2e-6 and rel64.max() < 1e-3
    med_tol, max_tol = tc_tolerances(N)
    reltc = np.abs(tc[nz] / ref[nz] - 1.0)
    assert np.median(reltc) < med_tol + 2e-6 and reltc.max() < max_tol + 1e-3
    C.close()


def test_plan_n9_tensor_core_matches_oracle(bg, oracle):
    # the whole path behind one call (bg_me2_batch) at n = 9
    B = 129
    u = inputs.rambo_uniforms(N, B, seed=93)
    hel = inputs.helicities(N, B, seed=93)
    plan = bg.Plan(N, B, SQRT_S, PT_MIN, prec=bg.BG_F32, cs_mode=bg.BG_CS_TC_BF16, hel_sampled=True)
    got = plan.me2(dev_arr(u), dev_arr(hel.T)).cpu().numpy()
    plan.close()
    ref = oracle.me2_co(N, u, sqrt_s=SQRT_S, hel=hel, pt_min=PT_MIN)
    assert np.array_equal(got == 0, ref == 0)
    nz = ref != 0
    med_tol, max_tol = tc_tolerances(N)
    rel = np.abs(got[nz] / ref[nz] - 1.0)
    assert np.median(rel) < med_tol + 2e-6 and rel.max() < max_tol + 1e-3
    assert math.factorial(N - 2) == 5040
