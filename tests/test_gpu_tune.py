"""GPU tests of the autotuner (bg_autotune / bg_tune_*): every kernel
variant of a recursion gives bitwise identical results (the variants differ
only in the mapping of the same sums onto the GPU), the tuner records a
valid choice, and its table survives a save / load round trip."""
import numpy as np
import pytest

from paper_2106_06507_gb300 import inputs

pytestmark = pytest.mark.gpu

SQRT_S = 1000.0


@pytest.fixture(scope="module")
def bg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_06507_gb300 import bg as _bg, build_lib
    build_lib.build()
    _bg.lib()
    return _bg


def cd_all_variants(bg, n, B, prec, flow):
    import torch
    dev = torch.device("cuda:0")
    u = torch.from_numpy(inputs.rambo_uniforms(n, B, seed=90 + n)).to(dev)
    hel = torch.from_numpy(np.ascontiguousarray(inputs.helicities(n, B, seed=90 + n).T)).to(dev)
    c = inputs.balanced_flow_colours(n, B, seed=90 + n) if flow else inputs.adjoint_colours(n, B, seed=90 + n)
    col = torch.from_numpy(np.ascontiguousarray(c.T)).to(dev)
    p, acc = bg.momenta_rambo(n, u, SQRT_S, -1.0)
    outs = []
    for v in range(bg.tune_num_variants(bg.BG_ALGO_CD, n)):
        bg.tune_set(bg.BG_ALGO_CD, n, prec, v)
        outs.append(bg.currents_cd(n, p, hel, col, flow=flow, prec=prec, sqrt_s=SQRT_S, accept=acc).cpu().numpy())
    bg.tune_set(bg.BG_ALGO_CD, n, prec, -1)
    return outs


@pytest.mark.parametrize("n,B,prec,flow", [(5, 300, 1, False), (9, 200, 1, True), (10, 120, 1, False),
                                           (12, 40, 1, True), (8, 100, 0, False), (11, 24, 0, True)])
def test_cd_variants_bitwise_identical(bg, n, B, prec, flow):
    outs = cd_all_variants(bg, n, B, prec, flow)
    assert len(outs) == (4 if n <= 9 else 5)
    assert np.count_nonzero(outs[0]) > 0
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


@pytest.mark.parametrize("n,prec", [(6, 1), (7, 1), (8, 0), (9, 1)])
def test_co_variants_bitwise_identical(bg, n, prec):
    import torch
    dev = torch.device("cuda:0")
    B = 1000 if n <= 8 else 200
    u = torch.from_numpy(inputs.rambo_uniforms(n, B, seed=95)).to(dev)
    hel = torch.from_numpy(np.ascontiguousarray(inputs.helicities(n, B, seed=95).T)).to(dev)
    p, _ = bg.momenta_rambo(n, u, SQRT_S, -1.0)
    outs = []
    for v in range(bg.tune_num_variants(bg.BG_ALGO_CO, n)):
        bg.tune_set(bg.BG_ALGO_CO, n, prec, v)
        outs.append(bg.currents_co(n, p, hel, prec=prec, sqrt_s=SQRT_S).cpu().numpy())
    bg.tune_set(bg.BG_ALGO_CO, n, prec, -1)
    assert len(outs) == 6
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)


def test_autotune_table_and_cache(bg, tmp_path):
    best_cd, ms_cd = bg.autotune(bg.BG_ALGO_CD, 10, bg.BG_F32, probe_batch=2048)
    assert 0 <= best_cd < 5 and len(ms_cd) == 5 and min(ms_cd) > 0
    assert ms_cd[best_cd] == min(ms_cd)
    assert bg.tune_get(bg.BG_ALGO_CD, 10, bg.BG_F32) == best_cd
    best_co, ms_co = bg.autotune(bg.BG_ALGO_CO, 7, bg.BG_F32)
    assert best_co in range(6) and len(ms_co) == 6
    path = str(tmp_path / "tune.txt")
    bg.tune_save(path)
    bg.tune_set(bg.BG_ALGO_CD, 10, bg.BG_F32, -1)
    bg.tune_set(bg.BG_ALGO_CO, 7, bg.BG_F32, -1)
    assert bg.tune_get(bg.BG_ALGO_CD, 10, bg.BG_F32) == -1
    bg.tune_load(path)
    assert bg.tune_get(bg.BG_ALGO_CD, 10, bg.BG_F32) == best_cd
    assert bg.tune_get(bg.BG_ALGO_CO, 7, bg.BG_F32) == best_co
    # the default is restored explicitly; a single-variant case tunes trivially
    bg.tune_set(bg.BG_ALGO_CD, 10, bg.BG_F32, -1)
    bg.tune_set(bg.BG_ALGO_CO, 7, bg.BG_F32, -1)
    assert bg.autotune(bg.BG_ALGO_CO, 5, bg.BG_F32)[0] == 0
    bg.tune_set(bg.BG_ALGO_CO, 5, bg.BG_F32, -1)
    with pytest.raises(bg.BGError):
        bg.tune_set(bg.BG_ALGO_CD, 10, bg.BG_F32, 5)
    with pytest.raises(bg.BGError):
        bg.autotune(bg.BG_ALGO_CO, 10, bg.BG_F32)
    bad = tmp_path / "bad.txt"
    bad.write_text("something else\n")
    with pytest.raises(bg.BGError):
        bg.tune_load(str(bad))


def test_mixed_autotuned_graph_matches_default(bg):
    import torch
    B = 1500
    ev = inputs.mixed_events(B, 6, 11, seed=44, colours="adjoint")
    res = []
    for tune in (False, True):
        mx = bg.Mixed(6, 11, B, SQRT_S, 20.0, prec=bg.BG_F32, cs_mode=bg.BG_CS_F32, n_co_max=8, autotune=tune)
        mx.n_per_event.copy_(torch.from_numpy(ev["nev"]))
        mx.u.copy_(torch.from_numpy(ev["u"]))
        mx.hel.copy_(torch.from_numpy(np.ascontiguousarray(ev["hel"].T)))
        mx.colors.copy_(torch.from_numpy(np.ascontiguousarray(ev["colors"].T)))
        res.append(mx.run(B).cpu().numpy())
        mx.close()
    for n in range(6, 12):
        bg.tune_set(bg.BG_ALGO_CO if n <= 8 else bg.BG_ALGO_CD, n, bg.BG_F32, -1)
    assert np.array_equal(res[0], res[1])
