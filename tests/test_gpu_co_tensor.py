"""The colour-ordered recursion in the tensor form (auxiliary antisymmetric
tensor field in place of the four-gluon vertex, Eqs. 2.23-2.26) on the GPU,
bg_currents_co_tensor, against the oracle.

The two forms are mathematically equal, so the GPU tensor form is compared
with the oracle's four-vertex amplitudes and with the oracle's own tensor
form, under the tolerances of test_gpu_co.py:
  FP64 amplitudes: element-wise within 1e-11 of the event's largest ordering
  amplitude (n = 4..8, and n = 9 for a few events);
  FP64 helicity-summed |M|^2 at n = 4 (all 16 configurations): the FP64
  parity rule against the extended-precision oracle, with the rounding floor
  of the oracle's two FP64 evaluations (four-vertex and tensor form);
  FP32 |M|^2 with the exact colour sum (FP64 CUDA cores): median relative
  error below 2e-6, all below 1e-3."""
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


def dev_arr(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


@pytest.mark.parametrize("n,B", [(4, 200), (5, 120), (6, 60), (7, 20), (8, 6), (9, 3)])
def test_tensor_form_amplitudes_fp64(bg, oracle, n, B):
    u = inputs.rambo_uniforms(n, B, seed=130 + n)
    hel = inputs.helicities(n, B, seed=130 + n)
    p, _ = bg.momenta_rambo(n, dev_arr(u), SQRT_S)
    amps = bg.currents_co(n, p, dev_arr(hel.T), prec=bg.BG_F64, sqrt_s=SQRT_S, tensor_form=True).cpu().numpy()
    unit = SQRT_S ** (4 - n)
    ords = oracle.orderings(n)
    for e in range(B):
        k = oracle.outgoing(oracle.rambo(n, SQRT_S, u[e]))
        eps = oracle.pols_for(k, hel[e])
        ref = oracle.amps_all(k, eps)  # four-vertex form
        got = amps[e, 0] * unit
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), (n, e)
        # the oracle's own tensor form on a few orderings
        for r in (0, len(ords) // 2, len(ords) - 1):
            order = np.concatenate([[0], ords[r], [n - 1]]).astype(np.int32)
            ref_t = oracle.amp_co(k, eps, order, tensor_form=True)
            assert abs(got[r] - ref_t) <= 1e-11 * np.abs(ref).max(), (n, e, r)


def test_tensor_form_helicity_sum_n4(bg, oracle):
    # The FP64 rule of test_gpu_co.py with the rounding floor of both FP64
    # evaluations of the definition in the oracle, the four-vertex and the
    # tensor form: the GPU tensor form sums in the latter's order.
    n, B = 4, 2000
    u = inputs.rambo_uniforms(n, B, seed=140)
    C = bg.ColourMatrix(n)
    p, _ = bg.momenta_rambo(n, dev_arr(u), SQRT_S)
    amps = bg.currents_co(n, p, None, prec=bg.BG_F64, sqrt_s=SQRT_S, tensor_form=True)
    got = bg.color_sum(C, amps, hel_sampled=False, mode=bg.BG_CS_F64, sqrt_s=SQRT_S).cpu().numpy()
    C.close()
    ext = oracle.me2_co_ext(n, u, sqrt_s=SQRT_S)
    f64 = oracle.me2_co(n, u, sqrt_s=SQRT_S)
    f64t = oracle.me2_co(n, u, sqrt_s=SQRT_S, tensor_form=True)
    assert np.array_equal(got == 0, ext == 0)
    nz = ext != 0
    rel = np.abs(got[nz] / ext[nz] - 1.0)
    floor = np.maximum(np.abs(f64[nz] / ext[nz] - 1.0), np.abs(f64t[nz] / ext[nz] - 1.0))
    assert np.median(rel) <= max(1e-13, 8.0 * np.median(floor))
    assert np.sum(rel > 1e-12) <= 2 + 4 * np.sum(floor > 1e-12)
    assert rel.max() <= max(5e-11, 8.0 * floor.max())


@pytest.mark.parametrize("n,B", [(6, 1001), (7, 301), (8, 67)])
def test_tensor_form_me2_fp32(bg, oracle, n, B):
    u = inputs.rambo_uniforms(n, B, seed=150 + n)
    hel = inputs.helicities(n, B, seed=150 + n)
    C = bg.ColourMatrix(n)
    p, acc = bg.momenta_rambo(n, dev_arr(u), SQRT_S, PT_MIN)
    amps = bg.currents_co(n, p, dev_arr(hel.T), prec=bg.BG_F32, sqrt_s=SQRT_S, tensor_form=True)
    got = bg.color_sum(C, amps, True, mode=bg.BG_CS_F64, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    ref = oracle.me2_co(n, u, sqrt_s=SQRT_S, hel=hel, pt_min=PT_MIN)
    assert np.array_equal(got == 0, ref == 0)
    nz = ref != 0
    rel = np.abs(got[nz] / ref[nz] - 1.0)
    assert np.median(rel) < 2e-6 and rel.max() < 1e-3
    C.close()


def test_tensor_form_argument_errors(bg):
    import torch
    with pytest.raises(bg.BGError) as ei:
        bg.currents_co(10, torch.zeros((4, 10, 1), dtype=torch.float64, device="cuda"), None, tensor_form=True)
    assert ei.value.code == bg.BG_EUNSUPPORTED
