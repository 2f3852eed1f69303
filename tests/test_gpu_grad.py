"""GPU gradient d|M|^2/du (bg_me2_grad, the hand-written adjoint) against the
oracle's dual-number gradient and against central differences of the GPU's
own |M|^2.

Tolerances: FP64 path, per-event relative error of the gradient vector
(Euclidean norm) below 1e-9 (the dual-number oracle is exact to rounding;
the reverse sweep re-associates sums over up to 8! terms).  FP32 path:
median below 1e-5, 95 % below 1e-4, 99 % below 1e-3 and every event below
5e-3, on 400 (n = 6) and 200 (n = 8) events (the gradient is a difference of
large contributions, so its FP32 error is larger than that of |M|^2; measured
at n = 6 / 8: median 7.8e-7 / 1.9e-6, 99 % 1.1e-4 / 2.8e-5, worst 5.0e-4 /
4.5e-5).
Central differences (h = 1e-6, FP64): agreement to 1e-6 of the gradient
norm.  The per-event sums over orderings are taken in a fixed order, so
repeated calls agree bit for bit; an upstream weight w changes the result
only by the FP64 rounding of w x scale x gradient (1e-13 relative here)."""
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


def dev_inputs(n, B, seed):
    import torch
    dev = torch.device("cuda:0")
    u = inputs.rambo_uniforms(n, B, seed=seed)
    hel = inputs.helicities(n, B, seed=seed)
    return u, hel, torch.from_numpy(u).to(dev), torch.from_numpy(np.ascontiguousarray(hel.T)).to(dev)


def plan_for(bg, n, B, prec, pt_min=PT_MIN):
    cs = bg.BG_CS_F64 if prec == bg.BG_F64 else (bg.BG_CS_TC_BF16 if 6 <= n <= 8 else bg.BG_CS_F32)
    return bg.Plan(n, B, SQRT_S, pt_min, prec=prec, cs_mode=cs, hel_sampled=True, grad=True)


@pytest.mark.parametrize("n,B", [(4, 7), (5, 7), (6, 6), (7, 4), (8, 3)])
def test_grad_fp64_matches_dual_numbers(bg, oracle, n, B):
    u, hel, ut, ht = dev_inputs(n, B, 100 + n)
    plan = plan_for(bg, n, B, bg.BG_F64, pt_min=-1.0)
    import torch
    me2 = torch.empty(B, dtype=torch.float64, device="cuda")
    g = plan.grad(ut, ht, me2=me2).cpu().numpy()
    for e in range(B):
        v, ref = oracle.me2_co_grad(n, u[e], hel[e], sqrt_s=SQRT_S)
        assert abs(me2[e].item() / v - 1.0) < 1e-11
        assert np.linalg.norm(g[e] - ref) <= 1e-9 * np.linalg.norm(ref)
    plan.close()


@pytest.mark.parametrize("n,B", [(6, 400), (8, 200)])
def test_grad_fp32_matches_dual_numbers(bg, oracle, n, B):
    # the oracle's dual-number gradients on all host cores (each call is one
    # event; ctypes releases the interpreter lock)
    from concurrent.futures import ThreadPoolExecutor
    u, hel, ut, ht = dev_inputs(n, B, 110 + n)
    plan = plan_for(bg, n, B, bg.BG_F32, pt_min=-1.0)
    g = plan.grad(ut, ht).cpu().numpy()
    plan.close()
    oracle.colour_matrix(n)
    with ThreadPoolExecutor(oracle.n_cores()) as ex:
        refs = list(ex.map(lambda e: oracle.me2_co_grad(n, u[e], hel[e], sqrt_s=SQRT_S)[1], range(B)))
    rel = np.array([np.linalg.norm(g[e] - refs[e]) / np.linalg.norm(refs[e]) for e in range(B)])
    assert np.median(rel) < 1e-5
    assert np.quantile(rel, 0.95) < 1e-4
    assert np.quantile(rel, 0.99) < 1e-3
    assert rel.max() < 5e-3


def test_grad_central_differences_fp64(bg):
    import torch
    n, B = 6, 4
    u, hel, ut, ht = dev_inputs(n, B, 120)
    plan = plan_for(bg, n, B, bg.BG_F64, pt_min=-1.0)
    g = plan.grad(ut, ht).cpu().numpy()
    h = 1e-6
    d = 4 * (n - 2)
    for j in range(d):
        up = ut.clone()
        up[:, j] += h
        um = ut.clone()
        um[:, j] -= h
        fd = ((plan.me2(up, ht) - plan.me2(um, ht)) / (2 * h)).cpu().numpy()
        assert np.all(np.abs(fd - g[:, j]) <= 1e-6 * np.linalg.norm(g, axis=1))
    plan.close()


def test_grad_upstream_cut_and_autograd(bg):
    import torch
    n, B = 6, 64
    u, hel, ut, ht = dev_inputs(n, B, 130)
    plan = plan_for(bg, n, B, bg.BG_F32)
    me2 = torch.empty(B, dtype=torch.float64, device="cuda")
    g1 = plan.grad(ut, ht, me2=me2)
    assert torch.equal(me2, plan.me2(ut, ht))
    up = torch.full((B,), 2.5, dtype=torch.float64, device="cuda")
    g2 = plan.grad(ut, ht, upstream=up)
    assert torch.allclose(g2, 2.5 * g1, rtol=1e-13, atol=0.0)
    assert torch.equal(plan.grad(ut, ht, me2=me2), g1)  # deterministic
    cut = (me2 == 0).cpu().numpy()
    assert cut.any() and (~cut).any()
    assert np.all(g1.cpu().numpy()[cut] == 0)
    # torch.autograd: d(sum w_e |M|^2_e)/du = w_e d|M|^2_e/du
    uu = ut.clone().requires_grad_(True)
    w = torch.linspace(0.5, 1.5, B, dtype=torch.float64, device="cuda")
    (bg.me2_autograd(uu, ht, plan) * w).sum().backward()
    assert torch.allclose(uu.grad, w[:, None] * g1, rtol=1e-13, atol=0.0)
    plan.close()


def test_grad_plan_errors(bg):
    with pytest.raises(bg.BGError) as ei:
        bg.Plan(9, 8, grad=True)
    assert ei.value.code == bg.BG_EUNSUPPORTED
    plan = bg.Plan(5, 8)
    import torch
    u = torch.zeros((2, 12), dtype=torch.float64, device="cuda")
    h = torch.ones((5, 2), dtype=torch.int8, device="cuda")
    with pytest.raises(bg.BGError) as ei:
        plan.grad(u, h)
    assert ei.value.code == bg.BG_EINVAL
    plan.close()
