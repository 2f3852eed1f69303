"""GPU tests of the plan API (bg_plan_create / bg_me2_batch): the whole hot
path in one call, with device buffers and with host buffers (staged through
the plan's workspace), checked against the stage-by-stage calls and the
oracle."""
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


def test_plan_device_and_host_buffers_agree_with_stages(bg, oracle):
    import torch
    dev = torch.device("cuda:0")
    n, B = 6, 3001
    u = inputs.rambo_uniforms(n, B, seed=31)
    hel = np.ascontiguousarray(inputs.helicities(n, B, seed=31).T)
    plan = bg.Plan(n, 4096, SQRT_S, PT_MIN, prec=bg.BG_F32, cs_mode=bg.BG_CS_F32, hel_sampled=True)
    ut, ht = torch.from_numpy(u).to(dev), torch.from_numpy(hel).to(dev)
    dev_out = plan.me2(ut, ht).cpu().numpy()
    # stage by stage
    C = bg.ColourMatrix(n)
    p, acc = bg.momenta_rambo(n, ut, SQRT_S, PT_MIN)
    amps = bg.currents_co(n, p, ht, prec=bg.BG_F32, sqrt_s=SQRT_S)
    ref_stages = bg.color_sum(C, amps, True, mode=bg.BG_CS_F32, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    assert np.array_equal(dev_out, ref_stages)
    # host buffers: numpy (pageable) and pinned torch tensors, host output
    out_np = np.zeros(B)
    plan.me2(u, hel, out=out_np)
    assert np.array_equal(out_np, ref_stages)
    out_pin = torch.zeros(B, dtype=torch.float64).pin_memory()
    plan.me2(torch.from_numpy(u).pin_memory(), torch.from_numpy(hel).pin_memory(), out=out_pin)
    assert np.array_equal(out_pin.numpy(), ref_stages)
    # against the oracle (FP32 tolerance of the colour-ordered path)
    ref = oracle.me2_co(n, u, sqrt_s=SQRT_S, hel=hel.T, pt_min=PT_MIN)
    nz = ref != 0
    assert np.array_equal(out_np == 0, ref == 0)
    rel = np.abs(out_np[nz] / ref[nz] - 1.0)
    assert np.median(rel) < 2e-6 and rel.max() < 1e-3
    plan.close()
    C.close()


def test_plan_helicity_summed_fp64(bg, oracle):
    n, B = 4, 777
    u = inputs.rambo_uniforms(n, B, seed=32)
    plan = bg.Plan(n, B, SQRT_S, -1.0, prec=bg.BG_F64, cs_mode=bg.BG_CS_F64, hel_sampled=False)
    out = np.zeros(B)
    plan.me2(u, None, out=out)
    ext = oracle.me2_co_ext(n, u, sqrt_s=SQRT_S)
    rel = np.abs(out / ext - 1.0)
    assert np.median(rel) < 1e-13 and rel.max() < 5e-11
    plan.close()


def test_plan_errors(bg):
    with pytest.raises(bg.BGError) as ei:
        bg.Plan(10, 16, algo=bg.BG_ALGO_CO)
    assert ei.value.code == bg.BG_EUNSUPPORTED
    with pytest.raises(bg.BGError) as ei:
        bg.Plan(6, 0)
    assert ei.value.code == bg.BG_EINVAL
    plan = bg.Plan(5, 8, SQRT_S, hel_sampled=True)
    u = inputs.rambo_uniforms(5, 9, seed=1)
    hel = np.ones((5, 9), dtype=np.int8)
    with pytest.raises(bg.BGError) as ei:
        plan.me2(u, hel, out=np.zeros(9))
    assert ei.value.code == bg.BG_EINVAL
    with pytest.raises(bg.BGError) as ei:
        plan.me2(u[:4], None, out=np.zeros(4))  # sampled helicities need hel
    assert ei.value.code == bg.BG_EINVAL
    assert plan.workspace_bytes > 0
    plan.close()


def test_plan_async_host_buffers_on_streams(bg):
    # bg_me2_batch_async with pinned host buffers on several streams gives
    # the same |M|^2 as the synchronous call
    import torch
    res = []
    plans, hosts, outs, streams = [], [], [], []
    for n in (6, 7):
        B = 2000
        u = torch.from_numpy(inputs.rambo_uniforms(n, B, seed=60 + n)).pin_memory()
        h = torch.from_numpy(np.ascontiguousarray(inputs.helicities(n, B, seed=60 + n).T)).pin_memory()
        plan = bg.Plan(n, B, SQRT_S, PT_MIN, prec=bg.BG_F32, cs_mode=bg.BG_CS_TC_BF16, hel_sampled=True)
        ref = plan.me2(u, h, out=torch.empty(B, dtype=torch.float64).pin_memory())
        res.append(ref.clone())
        plans.append(plan)
        hosts.append((u, h))
        outs.append(torch.full((B,), -1.0, dtype=torch.float64).pin_memory())
        streams.append(torch.cuda.Stream())
    for plan, (u, h), out, st in zip(plans, hosts, outs, streams):
        plan.me2(u, h, out=out, stream=st, wait=False)
    for st in streams:
        st.synchronize()
    for ref, out, plan in zip(res, outs, plans):
        assert torch.equal(ref, out)
        plan.close()


@pytest.mark.parametrize("n", [4, 6, 8, 10, 12])
def test_apply_cuts_matches_oracle(bg, oracle, n):
    # the paper's constraints at sqrt(s) = 14 TeV, and each constraint alone:
    # acceptance flags bit for bit equal to the oracle's
    import torch
    B = 1 << 14
    u = inputs.rambo_uniforms(n, B, seed=230 + n)
    p, _ = bg.momenta_rambo(n, torch.from_numpy(u).to(torch.device("cuda:0")), 14000.0)
    for cuts in ((20.0, 2.5, 0.4), (20.0, 0.0, 0.0), (-1.0, 2.5, 0.0), (-1.0, 0.0, 0.4)):
        got = bg.apply_cuts(n, p, *cuts).cpu().numpy()
        ref = oracle.accept_cuts(n, u, sqrt_s=14000.0, pt_min=cuts[0], eta_max=cuts[1], dr_min=cuts[2])
        assert np.array_equal(got, ref), (cuts, int((got != ref).sum()))
