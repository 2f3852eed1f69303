"""Parity at the full benchmark sizes, in the launch configuration the bench
times, on sampled events that the oracle evaluates one by one.

- colour-ordered, n = 5..8, 2^20 events, FP32 currents, tensor-core colour
  sum for n = 6..8 (FP32 CUDA cores for n = 5), pT > 20 GeV: FP32 tolerances
  of the recursion plus those of the tensor-core colour sum (median < 7e-6,
  worst < 1.2e-3; see test_gpu_co.py and test_gpu_tc.py);
- colour-dressed, n = 8, 10, 12, 2^20 events, FP32, sampled adjoint colours:
  the FP32 colour-dressed criterion of test_gpu_cd.py;
- gradient, n = 6, 8, 2^18 events, FP32: the FP32 gradient criterion of
  test_gpu_grad.py;
- mixed batch, 10^7 events with n uniform in 4..12 in one graph launch: the
  criteria above per branch (the colour-dressed samples, 8 per n, each
  within 1e-3 of max(|M|^2, 1e-2 x the sample median)); at n = 9, bit for bit
  equal to the single-multiplicity path and against the oracle within the
  n = 9 tensor-core bound (median < 5.9e-5, worst < 2.9e-3: the two-plane
  colour matrix, see test_gpu_n9.py);
- colour-flow sampling with colour-ordered amplitudes, n = 12, 2^20 events,
  uniform flows; colour-dressed with continuous colour and polarisation-angle
  sampling, n = 12, 2^20 events; leading colour, n = 8, 2^20 events: the FP32
  criteria of test_gpu_comc.py, test_gpu_cd.py and test_gpu_lc.py.

The sample always contains the first and last events and the events at the
edges of 128-event tiles, plus seeded random picks.
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


def sample_indices(B, count, seed):
    rng = np.random.default_rng(seed)
    fixed = [0, 1, 127, 128, 255, 256, B // 2, B - 129, B - 128, B - 2, B - 1]
    idx = np.unique(np.concatenate([np.array(fixed), rng.integers(0, B, count)]))
    return idx[(idx >= 0) & (idx < B)]


def check_fp32(got, ref, med, worst):
    nz = ref > 0
    assert np.all(got[~nz] == 0.0)  # events failing the cut
    rel = np.abs(got[nz] / ref[nz] - 1.0)
    assert np.median(rel) < med, np.median(rel)
    assert rel.max() < worst, rel.max()


def fp32_rel_cd(got, ref):
    return np.abs(got - ref) / np.maximum(ref, 1e-2 * np.median(ref))


@pytest.mark.parametrize("n", [5, 6, 7, 8])
def test_co_fp32_tc_full_size(bg, oracle, n):
    import torch
    dev = torch.device("cuda:0")
    B = 1 << 20
    u = inputs.rambo_uniforms(n, B, seed=0)
    hel = inputs.helicities(n, B, seed=0)
    ut = torch.from_numpy(u).to(dev)
    ht = torch.from_numpy(np.ascontiguousarray(hel.T)).to(dev)
    cs = bg.BG_CS_TC_BF16 if n >= 6 else bg.BG_CS_F32
    C = bg.ColourMatrix(n)
    p, acc = bg.momenta_rambo(n, ut, SQRT_S, PT_MIN)
    amps = bg.currents_co(n, p, ht, prec=bg.BG_F32, sqrt_s=SQRT_S)
    got = bg.color_sum(C, amps, True, mode=cs, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    C.close()
    idx = sample_indices(B, 150 if n <= 7 else 60, 10 + n)
    ref = oracle.me2_co(n, u[idx], SQRT_S, hel=hel[idx], pt_min=PT_MIN)
    check_fp32(got[idx], ref, 7e-6, 1.2e-3)


@pytest.mark.parametrize("n,count", [(8, 60), (10, 24), (12, 8)])
def test_cd_fp32_full_size(bg, oracle, n, count):
    import torch
    dev = torch.device("cuda:0")
    B = 1 << 20
    u = inputs.rambo_uniforms(n, B, seed=0)
    hel = inputs.helicities(n, B, seed=0)
    cols = inputs.adjoint_colours(n, B, seed=0)
    ut = torch.from_numpy(u).to(dev)
    ht = torch.from_numpy(np.ascontiguousarray(hel.T)).to(dev)
    ct = torch.from_numpy(np.ascontiguousarray(cols.T)).to(dev)
    p, acc = bg.momenta_rambo(n, ut, SQRT_S, PT_MIN)
    got = bg.currents_cd(n, p, ht, ct, prec=bg.BG_F32, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    # sample among events that pass the cut and have a non-zero colour
    # factor, plus the fixed edges.  An event whose colour factor vanishes
    # can come out of the FP32 recursion as rounding noise (at most 1e-6 of
    # the largest |M|^2, checked below for the zeros in the sample) rather
    # than exactly 0, depending on the order of the partial sums: the sample
    # is drawn above 1e-3 of the median non-zero |M|^2
    acc_np = acc.cpu().numpy().astype(bool)
    rng = np.random.default_rng(20 + n)
    pos = acc_np & (got > 0)
    live = np.nonzero(pos & (got > 1e-3 * np.median(got[pos])))[0]
    idx = np.unique(np.concatenate([sample_indices(B, 0, 0), rng.choice(live, count, replace=False)]))
    ref = oracle.me2_cd(n, u[idx], hel[idx], cols[idx], 0, sqrt_s=SQRT_S, pt_min=PT_MIN)
    g, r = got[idx], ref
    scale = r.max()
    zero = r <= 1e-16 * scale
    assert np.all(np.abs(g[zero]) <= 1e-6 * scale)
    nz = ~zero
    assert nz.sum() >= count // 2
    assert np.median(np.abs(g[nz] / r[nz] - 1.0)) < 1e-5
    assert np.quantile(fp32_rel_cd(g[nz], r[nz]), 0.99) < 1e-3


@pytest.mark.parametrize("n,count", [(6, 12), (8, 4)])
def test_grad_fp32_full_size(bg, oracle, n, count):
    import torch
    dev = torch.device("cuda:0")
    B = 1 << 18
    u = inputs.rambo_uniforms(n, B, seed=0)
    hel = inputs.helicities(n, B, seed=0)
    ut = torch.from_numpy(u).to(dev)
    ht = torch.from_numpy(np.ascontiguousarray(hel.T)).to(dev)
    plan = bg.Plan(n, B, SQRT_S, PT_MIN, prec=bg.BG_F32, cs_mode=bg.BG_CS_F32, hel_sampled=True, grad=True)
    me2 = torch.empty(B, dtype=torch.float64, device=dev)
    g = plan.grad(ut, ht, me2=me2).cpu().numpy()
    me2 = me2.cpu().numpy()
    plan.close()
    rng = np.random.default_rng(30 + n)
    live = np.nonzero(me2 > 0)[0]
    idx = np.concatenate([[live[0], live[-1]], rng.choice(live, count, replace=False)])
    C = oracle.colour_matrix(n)
    rel = []
    for e in idx:
        v, gr = oracle.me2_co_grad(n, u[e], hel[e], SQRT_S, C=C)
        rel.append(np.linalg.norm(g[e] - gr) / np.linalg.norm(gr))
    rel = np.array(rel)
    assert np.median(rel) < 1e-4, rel
    assert np.quantile(rel, 0.95) < 1e-2, rel


def test_mixed_full_size(bg, oracle):
    import torch
    dev = torch.device("cuda:0")
    B = 10_000_000
    ev = inputs.mixed_events(B, 4, 12, seed=0, colours="adjoint")
    mx = bg.Mixed(4, 12, B, SQRT_S, PT_MIN, prec=bg.BG_F32, cs_mode=bg.BG_CS_TC_BF16,
                  color_mode=bg.BG_COL_ADJOINT, n_co_max=9)
    mx.n_per_event.copy_(torch.from_numpy(ev["nev"]))
    mx.u.copy_(torch.from_numpy(ev["u"]))
    mx.hel.copy_(torch.from_numpy(np.ascontiguousarray(ev["hel"].T)))
    mx.colors.copy_(torch.from_numpy(np.ascontiguousarray(ev["colors"].T)))
    got = mx.run(B).cpu().numpy()
    assert mx.counts()[4:] == list(np.bincount(ev["nev"], minlength=13)[4:])
    mx.close()
    rng = np.random.default_rng(40)
    for n in range(4, 13):
        sel = np.nonzero(ev["nev"] == n)[0]
        count = 12 if n <= 9 else 8
        live = sel[got[sel] > 0]
        idx = np.concatenate([[sel[0], sel[-1]], rng.choice(live, count, replace=False)])
        u = np.ascontiguousarray(ev["u"][idx, :4 * (n - 2)])
        hel = np.ascontiguousarray(ev["hel"][idx, :n])
        g = got[idx]
        if n == 9:
            # the n = 9 branch: bit for bit the single-multiplicity path (same
            # kernels) and, against the oracle, the tensor-core rule at n = 9
            # (two BF16 planes of C) on top of the FP32 currents
            plan = bg.Plan(9, idx.size, SQRT_S, PT_MIN, prec=bg.BG_F32, cs_mode=bg.BG_CS_TC_BF16, hel_sampled=True)
            single = plan.me2(torch.from_numpy(u).to(dev), torch.from_numpy(np.ascontiguousarray(hel.T)).to(dev))
            plan.close()
            assert np.array_equal(g, single.cpu().numpy())
            ref = oracle.me2_co(n, u, SQRT_S, hel=hel, pt_min=PT_MIN)
            nz = ref > 0
            assert np.all(g[~nz] == 0.0)
            rel = np.abs(g[nz] / ref[nz] - 1.0)
            assert np.median(rel) < 5.9e-5, (n, rel)
            assert rel.max() < 2.9e-3, (n, rel)
        elif n <= 8:
            ref = oracle.me2_co(n, u, SQRT_S, hel=hel, pt_min=PT_MIN)
            nz = ref > 0
            assert np.all(g[~nz] == 0.0)
            rel = np.abs(g[nz] / ref[nz] - 1.0)
            assert np.median(rel) < 7e-6, (n, rel)
            assert rel.max() < 1.2e-3, (n, rel)
        else:
            ref = oracle.me2_cd(n, u, hel, ev["colors"][idx, :n], 0, sqrt_s=SQRT_S, pt_min=PT_MIN)
            scale = ref.max()
            zero = ref <= 1e-16 * scale
            assert np.all(np.abs(g[zero]) <= 1e-6 * scale)
            nz = ~zero
            assert np.all(fp32_rel_cd(g[nz], ref[nz]) < 1e-3), (n, g, ref)


def test_comc_fp32_full_size(bg, oracle):
    # colour-flow sampling with colour-ordered amplitudes, n = 12, 2^20 events,
    # uniform flows (the bench workload): sampled events with a non-zero
    # estimate against the oracle, the colour-flow FP32 criterion of
    # test_gpu_comc.py at n >= 10
    import torch
    dev = torch.device("cuda:0")
    n, B = 12, 1 << 20
    u = inputs.rambo_uniforms(n, B, seed=0)
    hel = inputs.helicities(n, B, seed=0)
    cols = inputs.flow_colours(n, B, seed=0)
    p, acc = bg.momenta_rambo(n, torch.from_numpy(u).to(dev), SQRT_S, PT_MIN)
    got = bg.currents_co_mc(n, p, torch.from_numpy(np.ascontiguousarray(hel.T)).to(dev),
                            torch.from_numpy(np.ascontiguousarray(cols.T)).to(dev), prec=bg.BG_F32,
                            sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    live = np.nonzero(got > 0)[0]
    rng = np.random.default_rng(50)
    idx = np.unique(np.concatenate([sample_indices(B, 0, 0), rng.choice(live, 24, replace=False)]))
    ref = oracle.me2_co_mc(n, u[idx], hel[idx], cols[idx], sqrt_s=SQRT_S, pt_min=PT_MIN)
    g, r = got[idx], ref
    scale = r.max()
    zero = r <= 1e-16 * scale
    assert np.all(np.abs(g[zero]) <= 1e-6 * scale)
    nz = ~zero
    assert nz.sum() >= 12
    assert np.median(np.abs(g[nz] / r[nz] - 1.0)) < 5e-5
    assert np.quantile(fp32_rel_cd(g[nz], r[nz]), 0.99) < 2e-3


def test_cd_continuous_fp32_full_size(bg, oracle):
    # colour-dressed with continuous colour and polarisation-angle sampling,
    # n = 12, 2^20 events: sampled events against the oracle
    import torch
    dev = torch.device("cuda:0")
    n, B = 12, 1 << 20
    u = inputs.rambo_uniforms(n, B, seed=0)
    ang = inputs.continuous_angles(n, B, seed=0)
    p, acc = bg.momenta_rambo(n, torch.from_numpy(u).to(dev), SQRT_S, PT_MIN)
    a = torch.from_numpy(np.ascontiguousarray(ang.reshape(B, 5 * n).T)).to(dev)
    got = bg.currents_cd_cont(n, p, a, prec=bg.BG_F32, sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    acc_np = acc.cpu().numpy().astype(bool)
    rng = np.random.default_rng(51)
    idx = np.unique(np.concatenate([sample_indices(B, 0, 0), rng.choice(np.nonzero(acc_np)[0], 8, replace=False)]))
    ref = oracle.me2_cd_cont(n, u[idx], ang[idx], sqrt_s=SQRT_S, pt_min=PT_MIN)
    assert np.all(got[idx][ref == 0] == 0.0)
    nz = ref > 0
    assert nz.sum() >= 4
    assert np.all(fp32_rel_cd(got[idx][nz], ref[nz]) < 2e-3)


def test_lc_fp32_full_size(bg, oracle):
    # leading-colour sum, n = 8, 2^20 events: sampled events against the
    # oracle (a sum of squares: the FP32 colour-ordered criterion)
    import torch
    dev = torch.device("cuda:0")
    n, B = 8, 1 << 20
    u = inputs.rambo_uniforms(n, B, seed=0)
    hel = inputs.helicities(n, B, seed=0)
    p, acc = bg.momenta_rambo(n, torch.from_numpy(u).to(dev), SQRT_S, PT_MIN)
    got = bg.currents_lc(n, p, torch.from_numpy(np.ascontiguousarray(hel.T)).to(dev), prec=bg.BG_F32,
                         sqrt_s=SQRT_S, accept=acc).cpu().numpy()
    idx = sample_indices(B, 40, 52)
    ref = oracle.me2_lc(n, u[idx], hel=hel[idx], sqrt_s=SQRT_S, pt_min=PT_MIN)
    check_fp32(got[idx], ref, 2e-6, 1e-3)
