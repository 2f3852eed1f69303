"""GPU parity of the tensor-core (tcgen05) colour sum against the FP64
CUDA-core colour sum on the same amplitudes, and against the oracle.

Tolerance: the amplitudes enter as three BF16 planes (24 significant bits)
and C/gcd is exact in BF16, so every product is exact; the error is the
tensor cores' FP32 accumulation, U = 3 * planes(C) * ceil(k/16) accumulator
updates per element of A C (135 at n = 8; 1890 at n = 9, where C needs two
BF16 planes), each rounding at ~2^-24 of the running sum.  Bound: median
relative error of |M|^2 below max(5e-6, 3e-8 U) and every event below
max(2e-4, 1e-6 U) (measured: median 1.3e-6 at n = 8, 1.0e-5 at n = 9)."""


def tc_tolerances(n):
    k = math.factorial(n - 2)
    U = 3 * (2 if n == 9 else 1) * math.ceil(k / 16)
    return max(5e-6, 3e-8 * U), max(2e-4, 1e-6 * U)
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


def amps_for(bg, n, B, seed, prec):
    import torch
    dev = torch.device("cuda:0")
    u = inputs.rambo_uniforms(n, B, seed=seed)
    hel = inputs.helicities(n, B, seed=seed)
    p, acc = bg.momenta_rambo(n, torch.from_numpy(u).to(dev), SQRT_S, PT_MIN)
    amps = bg.currents_co(n, p, torch.from_numpy(np.ascontiguousarray(hel.T)).to(dev), prec=prec, sqrt_s=SQRT_S)
    return u, hel, acc, amps


@pytest.mark.parametrize("n,B", [(6, 1), (6, 1000), (7, 129), (7, 3000), (8, 127), (8, 1500), (9, 130)])
def test_tc_colour_sum_matches_fp64_colour_sum(bg, n, B):
    C = bg.ColourMatrix(n)
    u, hel, acc, amps = amps_for(bg, n, B, 41 + n, bg.BG_F32)
    ref = bg.color_sum(C, amps, True, mode=bg.BG_CS_F64, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    got = bg.color_sum(C, amps, True, mode=bg.BG_CS_TC_BF16, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    assert bg.device_status() == 0
    assert np.array_equal(got == 0, ref == 0)
    nz = ref != 0
    if nz.any():
        rel = np.abs(got[nz] / ref[nz] - 1.0)
        med_tol, max_tol = tc_tolerances(n)
        assert np.median(rel) < med_tol
        assert rel.max() < max_tol
    C.close()


def test_tc_colour_sum_fp64_amplitudes_and_oracle(bg, oracle):
    n, B = 7, 300
    C = bg.ColourMatrix(n)
    u, hel, acc, amps = amps_for(bg, n, B, 47, bg.BG_F64)
    got = bg.color_sum(C, amps, True, mode=bg.BG_CS_TC_BF16, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    ref = oracle.me2_co(n, u, sqrt_s=SQRT_S, hel=hel, pt_min=PT_MIN)
    assert np.array_equal(got == 0, ref == 0)
    nz = ref != 0
    rel = np.abs(got[nz] / ref[nz] - 1.0)
    assert np.median(rel) < 5e-6 and rel.max() < 2e-4
    C.close()


def test_tc_repeated_calls_are_deterministic(bg):
    n, B = 8, 700
    C = bg.ColourMatrix(n)
    _, _, acc, amps = amps_for(bg, n, B, 48, bg.BG_F32)
    a = bg.color_sum(C, amps, True, mode=bg.BG_CS_TC_BF16, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    b = bg.color_sum(C, amps, True, mode=bg.BG_CS_TC_BF16, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    assert np.array_equal(a, b)
    C.close()


@pytest.mark.parametrize("n,B", [(6, 1000), (7, 300), (8, 129), (8, 1500)])
def test_tc_staged_path_matches_register_path(bg, n, B):
    # FP32 amplitudes at a 16-byte aligned address go through the staged
    # path (tensor-map copies of the amplitude tile into shared memory); the
    # same amplitudes at an address that is only 4-byte aligned go through
    # the per-thread loads.  Both convert and multiply the same numbers in the
    # same order: the results must be bit for bit equal.
    import torch
    C = bg.ColourMatrix(n)
    _, _, acc, amps = amps_for(bg, n, B, 60 + n, bg.BG_F32)
    k = amps.shape[2]
    flat = torch.empty((B * k + 4,), dtype=torch.float32, device=amps.device)
    shifted = flat[1:1 + B * k].view(B, 1, k)
    shifted.copy_(amps)
    assert shifted.data_ptr() % 16 != 0 and amps.data_ptr() % 16 == 0
    a = bg.color_sum(C, amps, True, mode=bg.BG_CS_TC_BF16, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    b = bg.color_sum(C, shifted, True, mode=bg.BG_CS_TC_BF16, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    assert bg.device_status() == 0
    assert np.array_equal(a, b)
    C.close()


@pytest.mark.parametrize("staged", [True, False])
def test_tc_bounded_wait_runs_out(bg, monkeypatch, staged):
    # BG_TC_TEST_STALL=1 makes the colour-matrix tile producer issue no copy,
    # so the MMA issuer's wait for the first tile (and then every other wait)
    # runs out after ~1 ms: the kernel must record BG_ETIMEOUT in the device
    # status word, write |M|^2 = 0, leave no copy or MMA in flight, and the
    # device must stay usable (the next call gives the normal result).
    import torch
    n, B = 8, 300
    C = bg.ColourMatrix(n)
    _, _, acc, amps = amps_for(bg, n, B, 70, bg.BG_F32)
    if not staged:  # a 4-byte aligned copy takes the per-thread load path
        flat = torch.empty((B * 720 + 4,), dtype=torch.float32, device=amps.device)
        amps = flat[1:1 + B * 720].view(B, 1, 720).copy_(amps)
    bg.device_status_reset()
    ref = bg.color_sum(C, amps, True, mode=bg.BG_CS_TC_BF16, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    assert bg.device_status() == 0 and (ref > 0).any()
    monkeypatch.setenv("BG_TC_TEST_STALL", "1")
    got = bg.color_sum(C, amps, True, mode=bg.BG_CS_TC_BF16, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    assert bg.device_status() == bg.BG_ETIMEOUT
    assert np.all(got == 0.0)
    monkeypatch.delenv("BG_TC_TEST_STALL")
    bg.device_status_reset()
    again = bg.color_sum(C, amps, True, mode=bg.BG_CS_TC_BF16, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    assert bg.device_status() == 0
    assert np.array_equal(again, ref)
    C.close()


def test_tc_unsupported_cases(bg):
    import torch
    for n in (5,):
        C = bg.ColourMatrix(n)
        amps = torch.zeros((4, 1, math.factorial(n - 2)), dtype=torch.float32, device="cuda")
        with pytest.raises(bg.BGError) as ei:
            bg.color_sum(C, amps, True, mode=bg.BG_CS_TC_BF16)
        assert ei.value.code == bg.BG_EUNSUPPORTED
        C.close()
    C = bg.ColourMatrix(6)
    amps = torch.zeros((4, 64, 24), dtype=torch.float32, device="cuda")
    with pytest.raises(bg.BGError):
        bg.color_sum(C, amps, False, mode=bg.BG_CS_TC_BF16)
    C.close()
