"""Host logic of bench.py on CPU: the max-over-ranks timing reduction with a
world_size-2 gloo group, the ncu-figure and roofline helpers, the flop and
colour-flow order counts, and the reference arm's JSON line."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(1.5 + rank)
        bench.barrier()
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=5) for _ in range(2))
    assert res == {0: 2.5, 1: 2.5}


def test_ncu_figures_line(tmp_path):
    # the bench reads the dominant kernel's ncu figures from the summary's
    # "bench-figures:" line, and uses them only for the sources they name
    sys.path.insert(0, ROOT)
    import bench
    f = tmp_path / "summary.md"
    f.write_text("# x\n\nbench-figures: sources_sha1=abc executed_flops_per_event=123.5 "
                 "dram_bytes_per_event=2880\n")
    assert bench.ncu_figures(str(f)) == {"sources_sha1": "abc", "executed_flops_per_event": 123.5,
                                         "dram_bytes_per_event": 2880.0}
    assert bench.ncu_figures(str(tmp_path / "missing.md")) is None


def test_roofline_helper():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.roofline("k", "alu", 40.0, 80.0, "TFLOP/s", "src", traffic=5, extra=1)
    assert r["frac"] == 0.5 and r["traffic"] == 5 and r["extra"] == 1 and r["bound"] == "alu"
    assert bench.fp32_peak_tflops(152) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)


def test_canonical_flop_model():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.canonical_recursion_flops(8) == 720 * 7119
    assert bench.canonical_recursion_flops(4) == 2 * (65 * 4 + 46 * 1 + 12 * 3 + 7)
    assert bench.colour_sum_flops(8) == 2 * 720 * 720 + 2 * 720


def test_tensor_form_flop_model():
    # n = 4 by hand: segments of length 2 (two of them): V3 65 + wedge 24 +
    # propagator 12; the full current (length 3): two splits of V3 (130) and
    # one contraction on each side (2 x 24); final contraction 7; 2 orderings
    sys.path.insert(0, ROOT)
    import bench
    assert bench.tensor_form_flops(4) == 2 * (7 + 2 * (65 + 24 + 12) + (130 + 48))


def test_flow_order_counts_brute_force():
    # the bench's count of closing colour-flow orders (by colour types) against
    # the direct enumeration of the (n-1)! orders
    import itertools

    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from paper_2106_06507_gb300 import inputs
    for n in (4, 6, 7):
        cols = inputs.flow_colours(n, 400, seed=7)
        cols[::2] = inputs.balanced_flow_colours(n, 400, seed=7)[::2]
        got = bench.flow_order_counts(cols, n)
        for e in range(0, 400, 7):
            r, c = cols[e, 0::2], cols[e, 1::2]
            ref = sum(all(c[o[t]] == r[o[(t + 1) % n]] for t in range(n))
                      for o in ((0,) + p for p in itertools.permutations(range(1, n))))
            assert got[e] == ref, (n, e)
        assert got.max() > 0


def test_reference_arm_json_contract(monkeypatch, capsys):
    # the reference arm (the oracle on the host cores) prints one JSON line
    # with the contract's keys; tiny per-step samples keep this quick
    import json
    import types
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "REF_STEP_PER_N", 4)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    bench.run_reference(types.SimpleNamespace(gpus=1, steps=2, warmup=0))
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == "events/s" and line["value"] > 0
    assert line["higher_is_better"] is True and line["steps"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "events/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    # the step time is the time actually spent: events per step / rate
    assert line["ms_per_step"] == pytest.approx(1e3 * 16 / line["value"])
    # the same workload keys as the GPU arm's line
    for k, v in bench.ref_arm_config().items():
        assert line["config"][k] == v


def test_gradient_roofline_uses_the_committed_figures_only_for_their_sources():
    # the executed-FLOP figures the bench reads apply only while the kernel
    # sources are those of the capture: with matching sources the roofline is
    # figures x events/s, with other sources (or no n = 8 rate) there is none
    sys.path.insert(0, ROOT)
    import bench
    for summary in (bench.NCU_SUMMARY, bench.GRAD_SUMMARY):
        fig = bench.ncu_figures(summary)
        assert fig and fig["executed_flops_per_event"] > 0 and len(fig["sources_sha1"]) == 40

    class Dev:
        pass

    orig = bench.device_sms
    bench.device_sms = lambda dev: 152
    try:
        r = bench.grad_roofline({"6": 1.0, "8": 1.0e6}, Dev())
        assert bench.grad_roofline({"6": 1.0}, Dev()) is None
    finally:
        bench.device_sms = orig
    fig = bench.ncu_figures(bench.GRAD_SUMMARY)
    if fig["sources_sha1"] != bench.sources_sha1(bench.GRAD_SOURCES):
        assert r is None
    else:
        assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
        assert abs(r["achieved"] - fig["executed_flops_per_event"] * 1e6 / 1e12) < 1e-9


def test_mixed_roofline_counts_accepted_colour_dressed_events():
    # dense-model FLOPs of the accepted events with n >= 10 only
    sys.path.insert(0, ROOT)
    import bench
    orig = bench.device_sms
    bench.device_sms = lambda dev: 152
    try:
        r = bench.mixed_roofline({10: 1, 11: 1, 12: 2}, batch=7, events_per_s=7.0e6, dev=None)
    finally:
        bench.device_sms = orig
    flops = bench.cd_dense_flops(10) + bench.cd_dense_flops(11) + 2 * bench.cd_dense_flops(12)
    assert abs(r["achieved"] - flops * 1.0e6 / 1e12) < 1e-9
    assert r["bound"] == "alu" and r["frac"] == r["achieved"] / r["peak"]
    assert r["events_computed"] == {"10": 1, "11": 1, "12": 2}
