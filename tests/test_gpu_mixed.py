"""GPU tests of the mixed-multiplicity graph (bg_mixed_*): a batch whose
events each have their own n, binned on the device and evaluated by one
branch per multiplicity in one CUDA-graph launch.

Each event's |M|^2 is checked against the single-multiplicity path on the
same inputs (bit for bit: the same kernels run on the same per-event data,
only the event's position in its chunk differs, and no kernel mixes events)
and, in FP64, against the oracle."""
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


def load(mx, ev, B):
    import torch
    mx.n_per_event[:B].copy_(torch.from_numpy(ev["nev"][:B]))
    mx.u[:B].copy_(torch.from_numpy(ev["u"][:B]))
    n_max = mx.hel.shape[0]
    mx.hel[:, :B].copy_(torch.from_numpy(np.ascontiguousarray(ev["hel"][:B, :n_max].T)))
    mx.colors[:, :B].copy_(torch.from_numpy(np.ascontiguousarray(ev["colors"][:B].T)))


def single_n(bg, n, ev, idx, prec, cs_mode, n_co_max, flow):
    """|M|^2 of events idx (all of multiplicity n) by the single-n path."""
    import torch
    dev = torch.device("cuda:0")
    u = torch.from_numpy(np.ascontiguousarray(ev["u"][idx, :4 * (n - 2)])).to(dev)
    hel = torch.from_numpy(np.ascontiguousarray(ev["hel"][idx, :n].T)).to(dev)
    if n <= n_co_max:
        cs = cs_mode if (cs_mode != bg.BG_CS_TC_BF16 or n >= 6) else bg.BG_CS_F32
        plan = bg.Plan(n, len(idx), SQRT_S, PT_MIN, prec=prec, cs_mode=cs, hel_sampled=True)
        out = plan.me2(u, hel).cpu().numpy()
        plan.close()
        return out
    rows = 2 * n if flow else n
    col = torch.from_numpy(np.ascontiguousarray(ev["colors"][idx, :rows].T)).to(dev)
    p, acc = bg.momenta_rambo(n, u, SQRT_S, PT_MIN)
    return bg.currents_cd(n, p, hel, col, flow=flow, prec=prec, sqrt_s=SQRT_S, accept=acc).cpu().numpy()


@pytest.mark.parametrize("chunk_bytes", [1, 0])
def test_mixed_fp32_tc_matches_single_n_paths(bg, chunk_bytes):
    # n = 4..12, tensor-core colour sum for n <= 9, colour-dressed above;
    # chunk_bytes = 1 forces the smallest chunks (256 events: several chunks
    # per multiplicity)
    B = 2500
    ev = inputs.mixed_events(B, 4, 12, seed=41, colours="adjoint")
    mx = bg.Mixed(4, 12, B, SQRT_S, PT_MIN, prec=bg.BG_F32, cs_mode=bg.BG_CS_TC_BF16,
                  color_mode=bg.BG_COL_ADJOINT, n_co_max=9, chunk_bytes=chunk_bytes)
    load(mx, ev, B)
    bg.device_status_reset()
    got = mx.run(B).cpu().numpy()
    assert bg.device_status() == 0
    counts = mx.counts()
    assert counts == list(np.bincount(ev["nev"], minlength=13))
    for n in range(4, 13):
        idx = np.nonzero(ev["nev"] == n)[0]
        ref = single_n(bg, n, ev, idx, bg.BG_F32, bg.BG_CS_TC_BF16, 9, False)
        assert np.array_equal(got[idx], ref), n
    assert np.all(got >= 0.0)
    assert np.count_nonzero(got) > B // 4  # the pT cut removes a fraction only
    mx.close()


def test_mixed_fp64_against_oracle(bg, oracle):
    # n = 4..8 with the colour-ordered path up to n = 6 and colour-dressed
    # colour-flow sampling (balanced flows) for n = 7, 8
    B = 360
    ev = inputs.mixed_events(B, 4, 8, seed=42, colours="balanced_flow")
    mx = bg.Mixed(4, 8, B, SQRT_S, PT_MIN, prec=bg.BG_F64, cs_mode=bg.BG_CS_F64,
                  color_mode=bg.BG_COL_FLOW, n_co_max=6)
    load(mx, ev, B)
    got = mx.run(B).cpu().numpy()
    for n in range(4, 9):
        idx = np.nonzero(ev["nev"] == n)[0]
        u = ev["u"][idx, :4 * (n - 2)]
        hel = ev["hel"][idx, :n]
        if n <= 6:
            ref = oracle.me2_co_ext(n, u, SQRT_S, hel=hel, pt_min=PT_MIN)
        else:
            ref = oracle.me2_cd(n, u, hel, ev["colors"][idx, :2 * n], mode=1, sqrt_s=SQRT_S, pt_min=PT_MIN,
                                ext=True)
        g = got[idx]
        scale = ref.max()
        zero = ref <= 1e-16 * scale
        assert np.all(np.abs(g[zero]) <= 1e-10 * scale), n
        assert np.all(np.abs(g[~zero] / ref[~zero] - 1.0) < 1e-9), n
    mx.close()


def test_mixed_replay_and_edge_cases(bg):
    import torch
    B = 1200
    ev = inputs.mixed_events(B, 5, 10, seed=43, colours="adjoint")
    mx = bg.Mixed(5, 10, B, SQRT_S, PT_MIN, prec=bg.BG_F32, cs_mode=bg.BG_CS_F32, n_co_max=8, chunk_bytes=1)
    load(mx, ev, B)
    first = mx.run(B).cpu().numpy().copy()
    # the graph's kernels: per multiplicity at least Rambo and a recursion
    # (n = 5..10: six), plus the binning kernels
    assert 2 * 6 < mx.kernel_nodes() < 400
    # a shorter replay of the same graph: the first events bin differently
    # but get the same values
    mx.me2.fill_(-1.0)
    part = mx.run(700).cpu().numpy()
    assert np.array_equal(part, first[:700])
    assert np.all(mx.me2[700:].cpu().numpy() == -1.0)
    assert mx.counts() == list(np.bincount(ev["nev"][:700], minlength=13))
    # empty batch
    mx.run(0)
    torch.cuda.synchronize()
    assert mx.counts() == [0] * 13
    # out-of-range batch
    with pytest.raises(bg.BGError):
        mx.run(B + 1)
    # an event with n outside n_min..n_max: reported, the others computed
    bg.device_status_reset()
    mx.n_per_event[3] = 11
    mx.me2.fill_(-1.0)
    got = mx.run(B).cpu().numpy()
    assert bg.device_status() == bg.BG_EINVAL
    bg.device_status_reset()
    assert got[3] == -1.0
    keep = np.arange(B) != 3
    assert np.array_equal(got[keep], first[keep])
    mx.close()


def test_mixed_invalid_descriptors(bg):
    with pytest.raises(bg.BGError):
        bg.Mixed(3, 8, 100)
    with pytest.raises(bg.BGError):
        bg.Mixed(4, 13, 100)
    with pytest.raises(bg.BGError):
        bg.Mixed(8, 6, 100)
    with pytest.raises(bg.BGError):
        bg.Mixed(4, 8, 0)
    with pytest.raises(bg.BGError):
        bg.Mixed(4, 12, 100, n_co_max=10)
    with pytest.raises(bg.BGError):
        bg.Mixed(4, 8, 100, q=(1.0, 0.0, 0.0, 0.5))
