#!/usr/bin/env python
"""Throughput of the colour-ordered Berends-Giele hot path on GB300.

Workload (one "step"): for each multiplicity n = 5, 6, 7, 8 gluons, one batch
of 2^20 Rambo phase-space points at sqrt(s) = 1 TeV with a final-state
pT > 20 GeV cut, one sampled helicity configuration per event, FP32
colour-ordered currents for all (n-2)! orderings, and the full colour sum
A^T C A with the exact SU(3) colour matrix; FP64 Rambo and FP64 per-event
accumulation.  Metric: events/s (all generated events of all four
multiplicities; per-n figures are in "per_n").

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload co|cd|grad|mixed|comc|lc|paper]

The default workload (co) is the one above.  The others measure the other
parts of the path with the same timing rules:
  cd     colour-dressed recursion with sampled adjoint colours, n = 8, 10, 12,
         2^20 events per n, FP32 currents, pT > 20 GeV;
  grad   |M|^2 and d|M|^2/du (colour-ordered, FP32, full colour sum), n = 6
         and 8, 2^18 events per n;
  mixed  10^7 events with n uniform in 4..12 in one CUDA-graph launch: tensor-
         core colour sum for n = 6..9 (FP32 CUDA cores for n = 4, 5),
         colour-dressed recursion with sampled adjoint colours for n = 10..12,
         FP32 currents, pT > 20 GeV, autotuned kernel variants;
  comc   colour-flow sampling with colour-ordered amplitudes (Eq. 2.19),
         flows uniform in {1,2,3}^2, n = 8, 10, 12, 2^20 events per n;
  lc     leading-colour |M|^2 (Sec. 4) on the default events, n = 5..8;
  paper  the paper's own setup: sqrt(s) = 14 TeV, pT > 20 GeV, |eta| < 2.5,
         Delta R > 0.4, colour-ordered n = 5..8 (acceptance, recursion /
         colour-sum time split, device bytes per event);
  forms  the colour-ordered recursion with the four-gluon vertex against the
         tensor form (Eqs. 2.23-2.26), n = 6..9, kernel times and FLOP counts.

Prints ONE JSON line on rank 0.  N > 1 runs under torch.distributed.run, one
process per GPU, each with its own events (weak scaling, no collective on the
data path; a barrier and a max-reduction of the timings only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NS = (5, 6, 7, 8)
BATCH = 1 << 20
SQRT_S = 1000.0
PT_MIN = 20.0
SEED = 0
FP32_LANES_PER_SM = 128
MAX_SM_MHZ = 2070.0
L2_BYTES = 129 * 1024 * 1024

WORKLOAD = ("colour-ordered BG, n=5,6,7,8 gluons, 2^20 Rambo points per n at sqrt(s)=1 TeV, pT>20 GeV, "
            "sampled helicities, FP32 currents for all (n-2)! orderings, exact colour sum A^T C A")

# The ncu figures of the dominant kernel (executed FP32 operations per event
# and DRAM bytes per event) are read from the committed summary of the capture,
# which states the kernel sources it was taken on; they are used only while
# those sources are unchanged.
NCU_SUMMARY = os.path.join(ROOT, "profiles", "co_kernel_dfs_n8.md")
DOMINANT_SOURCES = ("paper_2106_06507_gb300/csrc/co_recursion.cuh", "paper_2106_06507_gb300/csrc/co_f32.cu",
                    "paper_2106_06507_gb300/csrc/device_common.cuh")
# the same for the gradient kernel at n = 8
GRAD_SUMMARY = os.path.join(ROOT, "profiles", "co_grad_kernel_n8.md")
GRAD_SOURCES = ("paper_2106_06507_gb300/csrc/co_grad.cuh", "paper_2106_06507_gb300/csrc/co_grad.cu",
                "paper_2106_06507_gb300/csrc/co_recursion.cuh", "paper_2106_06507_gb300/csrc/device_common.cuh")


def ncu_figures(path: str = NCU_SUMMARY) -> dict | None:
    """The `bench-figures:` line of an ncu summary: key=value pairs
    (sources_sha1, executed_flops_per_event, dram_bytes_per_event, ...)."""
    try:
        with open(path) as f:
            for line in f:
                if line.startswith("bench-figures:"):
                    out = {}
                    for kv in line.split(":", 1)[1].split():
                        k, v = kv.split("=", 1)
                        out[k] = v if k == "sources_sha1" else float(v)
                    return out
    except OSError:
        return None
    return None


def fp32_peak_tflops(sms: int) -> float:
    """FP32 pipe peak from unit counts: SMs x 128 lanes x 2 FLOP x max clock."""
    return sms * FP32_LANES_PER_SM * 2 * MAX_SM_MHZ * 1e6 / 1e12


def fp32_peak_source(sms: int) -> str:
    return f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 FLOP x {MAX_SM_MHZ:.0f} MHz (unit counts, max clock)"


def roofline(kernel: str, bound: str, achieved: float, peak: float, unit: str, peak_source: str,
             traffic=None, **extra) -> dict:
    """The roofline object of a bench line: achieved / peak of one kernel."""
    d = {"kernel": kernel, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
         "frac": (achieved / peak) if (achieved is not None and peak) else None, "traffic": traffic,
         "peak_source": peak_source}
    d.update(extra)
    return d


def device_sms(dev) -> int:
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def cs_mode_for(bg, n: int) -> int:
    """Colour-sum arithmetic per multiplicity: tensor cores (tcgen05) where
    available (6 <= n <= 9), FP32 CUDA cores for the 6x6 matrix of n = 5."""
    return bg.BG_CS_TC_BF16 if 6 <= n <= 9 else bg.BG_CS_F32


def canonical_recursion_flops(n: int) -> int:
    """Canonical FLOPs per event of the colour-ordered recursion (all (n-2)!
    orderings, one polarisation configuration): V3 = 65, V4 = 46,
    propagator = 12, final contraction = 7 per ordering."""
    per_order = 65 * math.comb(n, 3) + 46 * math.comb(n, 4) + 12 * math.comb(n - 1, 2) + 7
    return math.factorial(n - 2) * per_order


def colour_sum_flops(n: int) -> int:
    k = math.factorial(n - 2)
    return 2 * k * k + 2 * k


def sources_sha1(files=DOMINANT_SOURCES) -> str:
    h = hashlib.sha1()
    for rel in files:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


# ---------------------------------------------------------------------------
# distributed helpers (host logic; covered by a gloo test on CPU)
# ---------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        load = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on a bounded sample
# ---------------------------------------------------------------------------
CPU_SAMPLE_PER_N = 1 << 17  # cpu_baseline: events of each n (about 10 s of the oracle on 16 Arm cores)
REF_STEP_PER_N = 8192       # reference arm: events of each n per step


def oracle_step(per_n: int) -> tuple[dict, int]:
    """The oracle on the first `per_n` events of each multiplicity of the
    default workload (its own seeded inputs, made before the clock starts),
    on all host cores; returns the seconds per n and the core count."""
    from oracle import oracle as O
    from paper_2106_06507_gb300 import inputs
    secs = {}
    for n in NS:
        u = inputs.rambo_uniforms(n, per_n, seed=SEED)
        hel = inputs.helicities(n, per_n, seed=SEED)
        O.colour_matrix(n)
        t0 = time.perf_counter()
        O.me2_co(n, u, sqrt_s=SQRT_S, hel=hel, pt_min=PT_MIN)
        secs[n] = time.perf_counter() - t0
    return secs, O.n_cores()


def cpu_baseline() -> dict:
    secs, cores = oracle_step(CPU_SAMPLE_PER_N)
    total = sum(secs.values())
    return {"value": len(NS) * CPU_SAMPLE_PER_N / total, "unit": "events/s", "cores": cores, "kind": "oracle",
            "sample": (f"FP64 C++ oracle on all host threads, the first {CPU_SAMPLE_PER_N} events of each n of the "
                       f"default workload (n = 5..8 in equal numbers, as in the workload): {total:.1f} s"),
            "per_n": {str(n): CPU_SAMPLE_PER_N / secs[n] for n in NS}}


def run_reference(args) -> None:
    """The oracle as the reference arm: each step runs it on REF_STEP_PER_N
    events of each multiplicity of the default workload (equal numbers per n,
    as in the workload), so that events/s is directly the workload's rate."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_step(REF_STEP_PER_N)
    t_total = 0.0
    per_n_secs = {n: 0.0 for n in NS}
    cores = 0
    for _ in range(args.steps):
        secs, cores = oracle_step(REF_STEP_PER_N)
        t_total += sum(secs.values())
        for n in NS:
            per_n_secs[n] += secs[n]
    events = len(NS) * REF_STEP_PER_N * args.steps
    value = events / t_total
    sample = (f"FP64 C++ oracle on all host threads; each step the first {REF_STEP_PER_N} events of each n = 5..8 "
              "of the default workload")
    print(json.dumps({
        "impl": "reference", "metric": "events/s", "value": value, "unit": "events/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": ref_arm_config() | {"events_per_step": len(NS) * REF_STEP_PER_N},
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "per_n": {str(n): REF_STEP_PER_N * args.steps / per_n_secs[n] for n in NS},
    }), flush=True)


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def run_ours(args) -> None:
    import numpy as np
    import torch
    import torch.distributed as dist

    world, rank, local = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2106_06507_gb300 import bg, build_lib, inputs
    build_lib.build()
    bg.lib()
    sms = device_sms(dev)

    stream = torch.cuda.current_stream(dev)
    f64 = args.precision == "f64"
    prec = bg.BG_F64 if f64 else bg.BG_F32

    def csm(n):
        return bg.BG_CS_F64 if f64 else cs_mode_for(bg, n)

    # inputs: resident in HBM before the timed region; each rank its own events
    first = rank * BATCH
    U, HEL, P, ACC, AMPS, ME2, CM = {}, {}, {}, {}, {}, {}, {}
    h2d = 0
    for n in NS:
        u = inputs.rambo_uniforms(n, BATCH, seed=SEED, first_event=first)
        h = np.ascontiguousarray(inputs.helicities(n, BATCH, seed=SEED, first_event=first).T)
        U[n] = torch.from_numpy(u).to(dev)
        HEL[n] = torch.from_numpy(h).to(dev)
        P[n] = torch.empty((4, n, BATCH), dtype=torch.float64, device=dev)
        ACC[n] = torch.empty((BATCH,), dtype=torch.uint8, device=dev)
        AMPS[n] = torch.empty((BATCH, 1, math.factorial(n - 2)), dtype=torch.float64 if f64 else torch.float32,
                              device=dev)
        ME2[n] = torch.empty((BATCH,), dtype=torch.float64, device=dev)
        CM[n] = bg.ColourMatrix(n)
        h2d += u.nbytes + h.nbytes
    input_bytes = sum(U[n].numel() * 8 for n in NS)

    ev = {n: [torch.cuda.Event(enable_timing=True) for _ in range(4)] for n in NS}
    launches_per_step = 3 * len(NS)
    def step(record: bool):
        for n in NS:
            if record:
                ev[n][0].record(stream)
            bg.momenta_rambo(n, U[n], SQRT_S, PT_MIN, p=P[n], accept=ACC[n], stream=stream)
            if record:
                ev[n][1].record(stream)
            bg.currents_co(n, P[n], HEL[n], prec=prec, sqrt_s=SQRT_S, amps=AMPS[n], stream=stream)
            if record:
                ev[n][2].record(stream)
            bg.color_sum(CM[n], AMPS[n], True, mode=csm(n), sqrt_s=SQRT_S, accept=ACC[n],
                         me2=ME2[n], stream=stream)
            if record:
                ev[n][3].record(stream)

    # FP32 / FP64 pipe rates of the FMA probe (measured, for context)
    probe_f32 = fma_probe_tflops(True, sms, stream, dev, 20000)
    probe_f64 = fma_probe_tflops(False, sms, stream, dev, 500)
    # kernel variants of the recursion chosen by the library's autotuner on
    # this GPU (they give bitwise identical results)
    probe_batch = (1 << 14) if f64 else (1 << 18)
    tuned = {n: bg.autotune(bg.BG_ALGO_CO, n, prec, probe_batch=probe_batch, stream=stream)[0] for n in NS if n >= 6}

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize(dev)
    barrier()

    clocks = ClockSampler(gpu_uuid(dev, local))
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    kernel_ms = {n: [0.0, 0.0, 0.0] for n in NS}
    torch.cuda.synchronize(dev)
    t0.record(stream)
    for _ in range(args.steps):
        step(False)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    elapsed = t0.elapsed_time(t1) * 1e-3
    barrier()
    elapsed = max_over_ranks(elapsed, dev)
    events = world * len(NS) * BATCH * args.steps
    value = events / elapsed
    # per-kernel times: the same step serialised on one stream, CUDA events
    # between the kernels
    for _ in range(args.steps):
        step(True)
        torch.cuda.synchronize(dev)
        for n in NS:
            for j in range(3):
                kernel_ms[n][j] += ev[n][j].elapsed_time(ev[n][j + 1])

    # e2e: the public plan API with HOST buffers, copies inside the timed region.
    # Two sets of plans (and pinned output buffers) alternate between steps,
    # one stream per multiplicity and set: the calls of step s+1 are issued
    # before the host waits for the results of step s, so that the
    # host-to-device copies of one step overlap the kernels of the other.
    # Every step copies its inputs in and its |M|^2 out, and the host has
    # every step's results before the clock stops.
    plan_sets = [{n: bg.Plan(n, BATCH, SQRT_S, PT_MIN, prec=prec, cs_mode=csm(n), hel_sampled=True) for n in NS}
                 for _ in range(2)]
    host_u = {n: U[n].cpu().pin_memory() for n in NS}
    host_h = {n: HEL[n].cpu().pin_memory() for n in NS}
    host_m = [{n: torch.empty((BATCH,), dtype=torch.float64).pin_memory() for n in NS} for _ in range(2)]
    d2h = sum(host_m[0][n].numel() * 8 for n in NS)
    e2e_streams = [{n: torch.cuda.Stream(dev) for n in NS} for _ in range(2)]

    def e2e_issue(b):
        for n in reversed(NS):  # the longest recursion first
            plan_sets[b][n].me2(host_u[n], host_h[n], out=host_m[b][n], stream=e2e_streams[b][n], wait=False)

    def e2e_wait(b):
        for n in NS:
            e2e_streams[b][n].synchronize()

    def e2e_run(steps):
        for i in range(steps):
            e2e_issue(i & 1)
            if i > 0:
                e2e_wait((i - 1) & 1)
        e2e_wait((steps - 1) & 1)

    e2e_run(max(2, args.warmup))
    torch.cuda.synchronize(dev)
    barrier()
    w0 = time.perf_counter()
    e2e_run(args.steps)
    torch.cuda.synchronize(dev)
    e2e_elapsed = max_over_ranks(time.perf_counter() - w0, dev)
    e2e_value = world * len(NS) * BATCH * args.steps / e2e_elapsed
    # the e2e results must equal the device-resident results
    for b in range(2):
        for n in NS:
            if not torch.equal(host_m[b][n], ME2[n].cpu()):
                raise RuntimeError(f"e2e |M|^2 differs from the device-resident run at n={n}")
    for b in range(2):
        for n in NS:
            plan_sets[b][n].close()
    del host_u, host_h, host_m

    # roofline of the dominant kernel (the colour-ordered recursion at n = 8)
    n_dom = max(NS, key=lambda n: kernel_ms[n][1])
    dom_s = kernel_ms[n_dom][1] / args.steps * 1e-3
    dfs = tuned.get(n_dom, 0) != 0  # the ncu figures are for the depth-first kernel
    kname = (f"{'co_kernel_dfs' if dfs else 'co_kernel'}<{n_dom},{'double' if f64 else 'float'}> "
             f"(colour-ordered recursion, tuned variant {tuned.get(n_dom, 0)})")
    canonical = canonical_recursion_flops(n_dom) * BATCH
    canon = {"achieved": canonical / dom_s / 1e12, "flops_per_launch": canonical,
             "flops_model": "canonical (V3=65, V4=46, prop=12, final=7 per ordering)"}
    if f64:  # FP64 pipe: the FMA probe's measured rate
        canon["frac"] = canon["achieved"] / probe_f64
        roof = roofline(kname, "alu", canon["achieved"], probe_f64, "TFLOP/s", "FP64 FMA probe (measured)",
                        canonical=canon)
    else:
        peak = fp32_peak_tflops(sms)
        canon["frac"] = canon["achieved"] / peak
        fig = ncu_figures()
        valid = bool(fig) and fig.get("sources_sha1") == sources_sha1() and n_dom == 8 and dfs
        if valid:
            ex_flops = fig["executed_flops_per_event"] * BATCH
            roof = roofline(kname, "alu", ex_flops / dom_s / 1e12, peak, "TFLOP/s", fp32_peak_source(sms),
                            traffic=fig["dram_bytes_per_event"] * BATCH,
                            flops_per_launch=ex_flops,
                            flops_model=("executed FP32 operations counted by ncu on these kernel sources: "
                                         "2 FFMA + FADD + FMUL + 2 (2 FFMA2 + FADD2 + FMUL2) per event x events"),
                            ncu_summary=os.path.relpath(NCU_SUMMARY, ROOT), sources_sha1=fig["sources_sha1"],
                            canonical=canon, probe_fp32_tflops=probe_f32, probe_fp64_tflops=probe_f64)
        else:
            roof = roofline(kname, "alu", canon["achieved"], peak, "TFLOP/s", fp32_peak_source(sms),
                            flops_per_launch=canonical,
                            flops_model=("canonical (no ncu count of executed operations for these kernel "
                                         "sources)"), canonical=canon,
                            probe_fp32_tflops=probe_f32, probe_fp64_tflops=probe_f64)
    total_ms = sum(sum(v) for v in kernel_ms.values()) / args.steps
    shares = {f"n{n}_{name}": kernel_ms[n][j] / args.steps / total_ms
              for n in NS for j, name in enumerate(("rambo", "co_recursion", "colour_sum"))}
    per_n = {str(n): BATCH * world / (sum(kernel_ms[n]) / args.steps * 1e-3) for n in NS}
    for n in NS:  # free the headline's buffers before the other workloads
        CM[n].close()
    del U, HEL, P, ACC, AMPS, ME2
    torch.cuda.empty_cache()

    # the other workloads of the scope table, measured in the same run with
    # the same rules (CUDA events on the launching stream, warm-up steps, L2
    # flushed between timed steps): the plain FP64 GPU form of this workload,
    # the colour-dressed recursion, the gradient and a mixed batch
    extra_launches = 0
    per_precision = workloads = None
    side_clk = None
    if not f64 and not args.headline_only:
        side_clocks = ClockSampler(gpu_uuid(dev, local))
        side_clocks.start()
        per_precision, l0 = side_fp64(bg, inputs, dev, stream, rank, value, per_n)
        cd, l1 = side_cd(bg, inputs, dev, stream, rank, sms)
        grad, l2 = side_grad(bg, inputs, dev, stream, rank)
        mixed, l3 = side_mixed(bg, inputs, dev, stream, rank)
        side_clk = side_clocks.stop()
        workloads = {"cd": cd, "grad": grad, "mixed": mixed}
        extra_launches = l0 + l1 + l2 + l3

    if rank == 0:
        line = {
            "metric": "events/s", "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if f64 else "f32", "data": "synthetic",
            "config": ref_arm_config() | {
                "precision": ("FP64 currents and FP64 colour sum (CUDA cores)" if f64 else
                              "FP32 currents; colour sum on tcgen05 tensor cores (BF16x3 amplitude split, "
                              "FP32 accumulate) for n=6..8, FP32 CUDA cores for n=5; "
                              "FP64 Rambo/polarisations/per-event accumulation"),
                "parallelism": f"replicas x{world}",
                "l2": f"inputs larger than L2: {input_bytes / 2**20:.0f} MiB of uniforms per step",
                "tuned_variants": {str(n): v for n, v in tuned.items()}},
            "per_n": per_n,
            "kernel_ms_per_step": {f"n{n}": [round(x / args.steps, 4) for x in kernel_ms[n]] for n in NS},
            "schedule": ("one stream: Rambo, recursion, colour sum per n in turn; kernel_ms_per_step and "
                         "kernel_share from the same step with CUDA events between the kernels"),
            "kernel_share": {k: round(v, 4) for k, v in shares.items()},
            "roofline": roof,
            "cpu_baseline": None,
            "e2e": {"value": e2e_value, "unit": "events/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
        }
        if per_precision is not None:
            line["per_precision"] = per_precision
            line["workloads"] = workloads
            line["workloads_clocks"] = side_clk
            line["workloads_gpu_launches"] = extra_launches
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    if world > 1 and dist.is_initialized():
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# the other workloads, reported beside the headline in the default line
# ---------------------------------------------------------------------------
SIDE_WARMUP = 3
SIDE_STEPS = 3
FP64_BATCH = 1 << 18     # plain FP64 GPU form of the default workload, per n
CD_SIDE_BATCH = 1 << 17  # colour-dressed, per n
MIXED_SIDE_EVENTS = 1_000_000


def flush_l2(dev):
    import torch
    buf = getattr(flush_l2, "buf", None)
    if buf is None or buf.device != dev:
        buf = flush_l2.buf = torch.empty((2 * L2_BYTES,), dtype=torch.uint8, device=dev)
    buf.fill_(1)


def timed_side(step, dev, stream) -> float:
    """SIDE_WARMUP untimed steps, then SIDE_STEPS steps each between CUDA events
    on `stream`, with L2 flushed (outside the events) before each; returns the
    seconds per step (max over ranks)."""
    import torch
    for _ in range(SIDE_WARMUP):
        step()
    torch.cuda.synchronize(dev)
    barrier()
    total = 0.0
    for _ in range(SIDE_STEPS):
        flush_l2(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize(dev)
        total += a.elapsed_time(b) * 1e-3
    return max_over_ranks(total / SIDE_STEPS, dev)


def side_fp64(bg, inputs, dev, stream, rank, value32, per_n32):
    """The plain FP64 GPU form of the default workload (FP64 currents, FP64
    colour sum on CUDA cores), FP64_BATCH events per n."""
    import numpy as np
    import torch
    B = FP64_BATCH
    first = rank * BATCH
    bufs = {}
    for n in NS:
        u = torch.from_numpy(inputs.rambo_uniforms(n, B, seed=SEED, first_event=first)).to(dev)
        h = torch.from_numpy(np.ascontiguousarray(inputs.helicities(n, B, seed=SEED, first_event=first).T)).to(dev)
        bufs[n] = (u, h, torch.empty((4, n, B), dtype=torch.float64, device=dev),
                   torch.empty((B,), dtype=torch.uint8, device=dev),
                   torch.empty((B, 1, math.factorial(n - 2)), dtype=torch.float64, device=dev),
                   torch.empty((B,), dtype=torch.float64, device=dev), bg.ColourMatrix(n))

    def one(n):
        u, h, p, acc, amps, me2, C = bufs[n]
        bg.momenta_rambo(n, u, SQRT_S, PT_MIN, p=p, accept=acc, stream=stream)
        bg.currents_co(n, p, h, prec=bg.BG_F64, sqrt_s=SQRT_S, amps=amps, stream=stream)
        bg.color_sum(C, amps, True, mode=bg.BG_CS_F64, sqrt_s=SQRT_S, accept=acc, me2=me2, stream=stream)

    for n in NS:
        if n >= 6:
            bg.autotune(bg.BG_ALGO_CO, n, bg.BG_F64, probe_batch=1 << 14, stream=stream)
    per_n = {str(n): B / timed_side(lambda n=n: one(n), dev, stream) for n in NS}
    value = len(NS) * B / sum(B / per_n[str(n)] for n in NS)
    for n in NS:
        bufs[n][-1].close()
    launches = (SIDE_WARMUP + SIDE_STEPS) * 3 * len(NS)
    return {"f64": {"value": value, "unit": "events/s", "per_n": per_n, "batch_per_n": B,
                    "precision": "FP64 currents, FP64 colour sum (CUDA cores), FP64 Rambo",
                    "steps": SIDE_STEPS, "warmup": SIDE_WARMUP, "l2": "flushed before each timed step"},
            "f32": {"value": value32, "unit": "events/s", "per_n": per_n32,
                    "precision": "the headline (FP32 currents, tensor-core colour sum)"},
            "f32_over_f64": value32 / value,
            "f32_over_f64_per_n": {str(n): per_n32[str(n)] / per_n[str(n)] for n in NS}}, launches


def side_cd(bg, inputs, dev, stream, rank, sms):
    """Colour-dressed recursion with sampled adjoint colours, n = 8, 10, 12,
    FP32 currents, CD_SIDE_BATCH events per n (the 2^20-event workload at an
    eighth of its batch)."""
    import numpy as np
    import torch
    B = CD_SIDE_BATCH
    first = rank * BATCH
    bufs = {}
    for n in CD_NS:
        u = torch.from_numpy(inputs.rambo_uniforms(n, B, seed=SEED, first_event=first)).to(dev)
        h = torch.from_numpy(np.ascontiguousarray(inputs.helicities(n, B, seed=SEED, first_event=first).T)).to(dev)
        c = torch.from_numpy(np.ascontiguousarray(inputs.adjoint_colours(n, B, seed=SEED, first_event=first).T)).to(dev)
        bufs[n] = (u, h, c, torch.empty((4, n, B), dtype=torch.float64, device=dev),
                   torch.empty((B,), dtype=torch.uint8, device=dev), torch.empty((B,), dtype=torch.float64, device=dev))
    times = {}
    for n in CD_NS:
        u, h, c, p, acc, me2 = bufs[n]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

        def full_step(n=n, u=u, h=h, c=c, p=p, acc=acc, me2=me2, ev=ev):
            bg.momenta_rambo(n, u, SQRT_S, PT_MIN, p=p, accept=acc, stream=stream)
            ev[0].record(stream)
            bg.currents_cd(n, p, h, c, prec=bg.BG_F32, sqrt_s=SQRT_S, accept=acc, me2=me2, stream=stream)
            ev[1].record(stream)

        step_s = timed_side(full_step, dev, stream)
        times[n] = (step_s, ev[0].elapsed_time(ev[1]) * 1e-3)  # kernel time of the last timed step
    per_n = {str(n): B / times[n][0] for n in CD_NS}
    value = len(CD_NS) * B / sum(times[n][0] for n in CD_NS)
    n_dom = 12
    accepted = int(bufs[n_dom][4].sum().item())
    flops = cd_dense_flops(n_dom) * accepted
    peak = fp32_peak_tflops(sms)
    roof = roofline(f"cd_kernel<{n_dom},float> (colour-dressed recursion)", "alu", flops / times[n_dom][1] / 1e12,
                    peak, "TFLOP/s", fp32_peak_source(sms),
                    flops_model=("dense 3x3x3 colour products per ordered partition (56 FMA per (r,l,c), 4 per "
                                 "(r,l)) x events passing the cut"),
                    flops_per_event=cd_dense_flops(n_dom), events_computed=accepted,
                    kernel_ms=times[n_dom][1] * 1e3)
    launches = (SIDE_WARMUP + SIDE_STEPS) * 2 * len(CD_NS)
    return {"workload": ("colour-dressed BG with sampled adjoint colours (1..8), n=8,10,12, "
                         f"{B} Rambo points per n at sqrt(s)=1 TeV, pT>20 GeV, sampled helicities, FP32 currents "
                         "(the 2^20-event configuration at an eighth of the batch)"),
            "value": value, "unit": "events/s", "per_n": per_n, "batch_per_n": B, "steps": SIDE_STEPS,
            "warmup": SIDE_WARMUP, "l2": "flushed before each timed step", "roofline": roof}, launches


def side_grad(bg, inputs, dev, stream, rank):
    """|M|^2 and d|M|^2/du with respect to the Rambo uniforms, n = 6, 8, 2^18
    events per n, FP32 currents with the full colour sum."""
    import numpy as np
    import torch
    B = GRAD_BATCH
    first = rank * B
    per_n, launches = {}, 0
    for n in GRAD_NS:
        u = torch.from_numpy(inputs.rambo_uniforms(n, B, seed=SEED, first_event=first)).to(dev)
        h = torch.from_numpy(np.ascontiguousarray(inputs.helicities(n, B, seed=SEED, first_event=first).T)).to(dev)
        g = torch.empty_like(u)
        m = torch.empty((B,), dtype=torch.float64, device=dev)
        plan = bg.Plan(n, B, SQRT_S, PT_MIN, prec=bg.BG_F32, cs_mode=bg.BG_CS_F32, hel_sampled=True, grad=True)
        per_n[str(n)] = B / timed_side(lambda: plan.grad(u, h, me2=m, out=g, stream=stream), dev, stream)
        plan.close()
        launches += (SIDE_WARMUP + SIDE_STEPS) * 5
    value = len(GRAD_NS) * B / sum(B / per_n[str(n)] for n in GRAD_NS)
    return {"workload": ("|M|^2 and d|M|^2/du (4(n-2) Rambo uniforms), colour-ordered FP32 with full colour sum, "
                         "n=6,8, 2^18 events per n, pT>20 GeV, sampled helicities"),
            "value": value, "unit": "events/s", "per_n": per_n, "batch_per_n": B, "steps": SIDE_STEPS,
            "warmup": SIDE_WARMUP, "l2": "flushed before each timed step",
            "roofline": grad_roofline(per_n, dev)}, launches


def side_mixed(bg, inputs, dev, stream, rank):
    """A mixed batch of MIXED_SIDE_EVENTS events with n uniform in 4..12 (the
    10^7-event mixed workload at a tenth of its size), one launch per step."""
    import numpy as np
    import torch
    B = MIXED_SIDE_EVENTS
    evs = inputs.mixed_events(B, 4, 12, seed=SEED + rank, colours="adjoint")
    mx = bg.Mixed(4, 12, B, SQRT_S, PT_MIN, prec=bg.BG_F32, cs_mode=bg.BG_CS_TC_BF16,
                  color_mode=bg.BG_COL_ADJOINT, n_co_max=9, autotune=True)
    mx.n_per_event.copy_(torch.from_numpy(evs["nev"]))
    mx.u.copy_(torch.from_numpy(evs["u"]))
    mx.hel.copy_(torch.from_numpy(np.ascontiguousarray(evs["hel"].T)))
    mx.colors.copy_(torch.from_numpy(np.ascontiguousarray(evs["colors"].T)))
    t = timed_side(lambda: mx.run(B, stream=stream), dev, stream)
    counts = mx.counts()[4:]
    kernels = mx.kernel_nodes()
    mx.close()
    rl = mixed_roofline(mixed_accepted(bg, evs["nev"], evs["u"], dev), B, B / t, dev)
    return {"workload": ("mixed batch: 10^6 events (the 10^7-event configuration at a tenth of its size) with n "
                         "uniform in 4..12 in one launch: colour-ordered + tensor-core colour sum for n=6..9 (FP32 "
                         "CUDA cores n=4,5), colour-dressed with sampled adjoint colours for n=10..12, FP32 currents, "
                         "FP64 Rambo and accumulation, pT>20 GeV, autotuned kernel variants"),
            "value": B / t, "unit": "events/s", "events": B, "counts_per_n": counts, "seconds_per_step": t,
            "steps": SIDE_STEPS, "warmup": SIDE_WARMUP, "l2": "flushed before each timed step",
            "launch": "one CUDA-graph launch per step", "kernels_per_graph": kernels,
            "roofline": rl}, (SIDE_WARMUP + SIDE_STEPS) * kernels


def timed_steps(step, args, dev, stream) -> tuple[float, dict]:
    """W untimed steps, then K steps between CUDA events on `stream` with a
    barrier and a synchronisation on both sides; returns (seconds, max over
    ranks) and the clock record of the timed region."""
    import torch
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    barrier()
    clocks = ClockSampler(gpu_uuid(dev, dev.index))
    clocks.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    barrier()
    return max_over_ranks(t0.elapsed_time(t1) * 1e-3, dev), clk


def timed_host(step, args, dev) -> float:
    """Wall-clock seconds of K steps that include host<->device copies."""
    import torch
    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    barrier()
    w0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize(dev)
    return max_over_ranks(time.perf_counter() - w0, dev)


def fma_probe_tflops(f32: bool, sms: int, stream, dev, iters: int) -> float:
    """Measured FMA-pipe rate (TFLOP/s) of the probe kernel of libbg_probe.so
    (8 blocks of 256 threads per SM)."""
    import ctypes

    import torch
    from paper_2106_06507_gb300 import build_lib
    lib = ctypes.CDLL(build_lib.PROBE_LIB)
    lib.bgprobe_fma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                ctypes.c_void_p]
    flops = ctypes.c_double(0.0)
    sp = ctypes.c_void_p(stream.cuda_stream)
    if lib.bgprobe_fma(int(f32), sms * 8, 64, ctypes.byref(flops), sp) != 0:
        raise RuntimeError("FMA probe launch failed")
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    if lib.bgprobe_fma(int(f32), sms * 8, iters, ctypes.byref(flops), sp) != 0:
        raise RuntimeError("FMA probe launch failed")
    s1.record(stream)
    torch.cuda.synchronize(dev)
    return flops.value / (s0.elapsed_time(s1) * 1e-3) / 1e12


def gpu_uuid(dev, local: int) -> str:
    import torch
    props = torch.cuda.get_device_properties(dev)
    gpu_id = str(getattr(props, "uuid", "")) or str(local)
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) > 8:
        gpu_id = "GPU-" + gpu_id
    return gpu_id


def ref_arm_config() -> dict:
    """The workload keys of the default line, shared by both arms."""
    return {"workload": WORKLOAD, "n": list(NS), "batch_per_n": BATCH, "sqrt_s_gev": SQRT_S, "pt_min_gev": PT_MIN,
            "helicities": "sampled, weight 2^n"}


def cd_dense_flops(n: int) -> int:
    """FLOPs per event of the colour-dressed recursion as implemented: every
    ordered partition (S1, S2) of every subset takes the dense 3x3x3 colour
    products; per (r, l, c) 56 FMA (X.Y, P.Y, the V3 update, the tensor
    product and both tensor contractions), per (r, l) 4 FMA (P.X); the top
    level skips the tensor product (44 FMA)."""
    m = n - 1
    inner = sum(math.comb(m, L) * (2 ** L - 2) for L in range(2, m))
    top = 2 ** m - 2
    return 2 * (inner * 9 * (4 + 3 * 56) + top * 9 * (4 + 3 * 44))


def setup_gpu():
    import torch
    import torch.distributed as dist
    world, rank, local = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2106_06507_gb300 import bg, build_lib
    build_lib.build()
    bg.lib()
    return world, rank, dev, bg


def finish_gpu(world):
    import torch.distributed as dist
    if world > 1 and dist.is_initialized():
        dist.destroy_process_group()


CD_NS = (8, 10, 12)


def run_cd(args) -> None:
    import numpy as np
    import torch
    from paper_2106_06507_gb300 import inputs
    world, rank, dev, bg = setup_gpu()
    stream = torch.cuda.current_stream(dev)
    cd_prec = bg.BG_F64 if args.precision == "f64" else bg.BG_F32
    batch = BATCH if args.precision == "f32" else BATCH >> 4  # FP64 on GB300 is ~1/64 of FP32
    first = rank * batch
    U, HEL, COL, P, ACC, ME2 = {}, {}, {}, {}, {}, {}
    host = {}
    for n in CD_NS:
        u = inputs.rambo_uniforms(n, batch, seed=SEED, first_event=first)
        h = np.ascontiguousarray(inputs.helicities(n, batch, seed=SEED, first_event=first).T)
        if args.colour_sampling == "continuous":
            c = np.ascontiguousarray(inputs.continuous_angles(n, batch, seed=SEED, first_event=first)
                                     .reshape(batch, 5 * n).T)
        else:
            c = np.ascontiguousarray(inputs.adjoint_colours(n, batch, seed=SEED, first_event=first).T)
        U[n], HEL[n], COL[n] = (torch.from_numpy(x).to(dev) for x in (u, h, c))
        host[n] = tuple(torch.from_numpy(x).pin_memory() for x in (u, h, c))
        P[n] = torch.empty((4, n, batch), dtype=torch.float64, device=dev)
        ACC[n] = torch.empty((batch,), dtype=torch.uint8, device=dev)
        ME2[n] = torch.empty((batch,), dtype=torch.float64, device=dev)
    ev = {n: [torch.cuda.Event(enable_timing=True) for _ in range(3)] for n in CD_NS}
    kernel_ms = {n: [0.0, 0.0] for n in CD_NS}

    def cd_call(n, p, hel, col, me2):
        if args.colour_sampling == "continuous":
            bg.currents_cd_cont(n, p, col, prec=cd_prec, sqrt_s=SQRT_S, accept=ACC[n], me2=me2, stream=stream)
        else:
            bg.currents_cd(n, p, hel, col, prec=cd_prec, sqrt_s=SQRT_S, accept=ACC[n], me2=me2, stream=stream)

    def step(record=False):
        for n in CD_NS:
            if record:
                ev[n][0].record(stream)
            bg.momenta_rambo(n, U[n], SQRT_S, PT_MIN, p=P[n], accept=ACC[n], stream=stream)
            if record:
                ev[n][1].record(stream)
            cd_call(n, P[n], HEL[n], COL[n], ME2[n])
            if record:
                ev[n][2].record(stream)

    elapsed, clk = timed_steps(step, args, dev, stream)
    value = world * len(CD_NS) * batch * args.steps / elapsed
    for _ in range(args.steps):  # per-kernel times (separate pass)
        step(True)
        torch.cuda.synchronize(dev)
        for n in CD_NS:
            for j in range(2):
                kernel_ms[n][j] += ev[n][j].elapsed_time(ev[n][j + 1]) / args.steps
    ref = {n: ME2[n].cpu() for n in CD_NS}
    out_h = {n: torch.empty((batch,), dtype=torch.float64).pin_memory() for n in CD_NS}
    d_in = {n: tuple(torch.empty_like(x, device=dev) for x in host[n]) for n in CD_NS}

    def e2e_step():
        for n in CD_NS:
            for dst, src in zip(d_in[n], host[n]):
                dst.copy_(src, non_blocking=True)
            bg.momenta_rambo(n, d_in[n][0], SQRT_S, PT_MIN, p=P[n], accept=ACC[n], stream=stream)
            cd_call(n, P[n], d_in[n][1], d_in[n][2], ME2[n])
            out_h[n].copy_(ME2[n], non_blocking=True)

    e2e_s = timed_host(e2e_step, args, dev)
    for n in CD_NS:
        if not torch.equal(out_h[n], ref[n]):
            raise RuntimeError(f"e2e colour-dressed |M|^2 differs from the device-resident run at n={n}")
    h2d = sum(sum(x.numel() * x.element_size() for x in host[n]) for n in CD_NS)
    n_dom = max(CD_NS, key=lambda n: kernel_ms[n][1])
    accepted = int(ACC[n_dom].sum().item())  # events failing the cut are skipped by the kernel
    flops = cd_dense_flops(n_dom) * accepted
    achieved = flops / (kernel_ms[n_dom][1] * 1e-3) / 1e12
    sms = device_sms(dev)
    peak, peak_source = fp32_peak_tflops(sms), fp32_peak_source(sms)
    if cd_prec == bg.BG_F64:
        peak, peak_source = fma_probe_tflops(False, sms, stream, dev, 500), "FP64 FMA probe (measured)"
    if rank == 0:
        print(json.dumps({
            "metric": "events/s", "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": (("colour-dressed BG with continuous colour (two unit vectors per gluon) and "
                                     "polarisation-angle sampling, n=8,10,12, "
                                     if args.colour_sampling == "continuous" else
                                     "colour-dressed BG with sampled adjoint colours (1..8), n=8,10,12, ") +
                                    f"{batch} Rambo points per n at sqrt(s)=1 TeV, pT>20 GeV, sampled helicities, "
                                    f"{args.precision.upper()} currents"),
                       "n": list(CD_NS), "batch_per_n": batch, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2"},
            "per_n": {str(n): batch * world / (sum(kernel_ms[n]) * 1e-3) for n in CD_NS},
            "kernel_ms_per_step": {f"n{n}": [round(x, 3) for x in kernel_ms[n]] for n in CD_NS},
            "roofline": roofline(f"cd_kernel<{n_dom},{'double' if args.precision == 'f64' else 'float'}>",
                                 "alu", achieved, peak, "TFLOP/s", peak_source,
                                 flops_model=("dense 3x3x3 colour products per ordered partition (56 FMA per "
                                              "(r,l,c), 4 per (r,l)) x events passing the cut"),
                                 flops_per_event=cd_dense_flops(n_dom), events_computed=accepted),
            "e2e": {"value": world * len(CD_NS) * batch * args.steps / e2e_s, "unit": "events/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": len(CD_NS) * batch * 8},
            "gpu_launches": 2 * len(CD_NS) * args.steps, "clocks": clk}), flush=True)
    finish_gpu(world)


def flow_order_counts(cols, n: int):
    """Number of orders (1, s_2, ..., s_n) whose colour-flow chain closes, per
    event (cols [B, 2n] flow pairs in 1..3): the work of the colour-flow
    kernel.  Counted by colour types -- the gluons of one (row, column) type
    are interchangeable -- with a memoised recursion over the remaining
    types, times the permutations within each type."""
    import numpy as np
    r = cols[:, 0::2].astype(np.int64) - 1
    c = cols[:, 1::2].astype(np.int64) - 1
    bal = np.all(np.stack([(r == k).sum(1) == (c == k).sum(1) for k in range(3)]), axis=0)
    out = np.zeros(cols.shape[0], dtype=np.int64)
    idx = np.nonzero(bal)[0]
    if idx.size == 0:
        return out
    types = r[idx, 1:] * 3 + c[idx, 1:]
    m = np.stack([(types == t).sum(1) for t in range(9)], axis=1)
    sig = np.concatenate([r[idx, :1], c[idx, :1], m], axis=1)
    uniq, inv = np.unique(sig, axis=0, return_inverse=True)
    from functools import lru_cache
    vals = np.zeros(len(uniq), dtype=np.int64)
    for i, row in enumerate(uniq):
        r0, c0, mm = int(row[0]), int(row[1]), tuple(int(x) for x in row[2:])

        @lru_cache(maxsize=None)
        def f(cur, rem):
            if not any(rem):
                return 1 if cur == r0 else 0
            tot = 0
            for cc in range(3):
                t = cur * 3 + cc
                if rem[t]:
                    tot += f(cc, rem[:t] + (rem[t] - 1,) + rem[t + 1:])
            return tot

        vals[i] = f(c0, mm) * math.prod(math.factorial(x) for x in mm)
    out[idx] = vals[inv.reshape(-1)]
    return out


COMC_NS = (8, 10, 12)


def run_comc(args) -> None:
    """Colour-flow sampling with colour-ordered amplitudes (Eq. 2.19), uniform
    flows in {1,2,3}^2 per gluon, the colour-dressed workload's n, batch, cut
    and arithmetic."""
    import numpy as np
    import torch
    from paper_2106_06507_gb300 import inputs
    world, rank, dev, bg = setup_gpu()
    stream = torch.cuda.current_stream(dev)
    prec = bg.BG_F64 if args.precision == "f64" else bg.BG_F32
    batch = BATCH if args.precision == "f32" else BATCH >> 4
    first = rank * batch
    U, HEL, COL, P, ACC, ME2, WS, host, orders = {}, {}, {}, {}, {}, {}, {}, {}, {}
    for n in COMC_NS:
        u = inputs.rambo_uniforms(n, batch, seed=SEED, first_event=first)
        h = inputs.helicities(n, batch, seed=SEED, first_event=first)
        c = inputs.flow_colours(n, batch, seed=SEED, first_event=first)
        orders[n] = flow_order_counts(c, n)
        h, c = np.ascontiguousarray(h.T), np.ascontiguousarray(c.T)
        U[n], HEL[n], COL[n] = (torch.from_numpy(x).to(dev) for x in (u, h, c))
        host[n] = tuple(torch.from_numpy(x).pin_memory() for x in (u, h, c))
        P[n] = torch.empty((4, n, batch), dtype=torch.float64, device=dev)
        ACC[n] = torch.empty((batch,), dtype=torch.uint8, device=dev)
        ME2[n] = torch.empty((batch,), dtype=torch.float64, device=dev)
        WS[n] = torch.empty((bg.comc_workspace_bytes(n, batch, prec),), dtype=torch.uint8, device=dev)
    ev = {n: [torch.cuda.Event(enable_timing=True) for _ in range(3)] for n in COMC_NS}
    kernel_ms = {n: [0.0, 0.0] for n in COMC_NS}

    def step(record=False):
        for n in COMC_NS:
            if record:
                ev[n][0].record(stream)
            bg.momenta_rambo(n, U[n], SQRT_S, PT_MIN, p=P[n], accept=ACC[n], stream=stream)
            if record:
                ev[n][1].record(stream)
            bg.currents_co_mc(n, P[n], HEL[n], COL[n], prec=prec, sqrt_s=SQRT_S, accept=ACC[n], me2=ME2[n],
                              workspace=WS[n], stream=stream)
            if record:
                ev[n][2].record(stream)

    elapsed, clk = timed_steps(step, args, dev, stream)
    value = world * len(COMC_NS) * batch * args.steps / elapsed
    for _ in range(args.steps):
        step(True)
        torch.cuda.synchronize(dev)
        for n in COMC_NS:
            for j in range(2):
                kernel_ms[n][j] += ev[n][j].elapsed_time(ev[n][j + 1]) / args.steps
    ref = {n: ME2[n].cpu() for n in COMC_NS}
    out_h = {n: torch.empty((batch,), dtype=torch.float64).pin_memory() for n in COMC_NS}
    d_in = {n: tuple(torch.empty_like(x, device=dev) for x in host[n]) for n in COMC_NS}

    def e2e_step():
        for n in COMC_NS:
            for dst, src in zip(d_in[n], host[n]):
                dst.copy_(src, non_blocking=True)
            bg.momenta_rambo(n, d_in[n][0], SQRT_S, PT_MIN, p=P[n], accept=ACC[n], stream=stream)
            bg.currents_co_mc(n, P[n], d_in[n][1], d_in[n][2], prec=prec, sqrt_s=SQRT_S, accept=ACC[n],
                              me2=ME2[n], workspace=WS[n], stream=stream)
            out_h[n].copy_(ME2[n], non_blocking=True)

    e2e_s = timed_host(e2e_step, args, dev)
    for n in COMC_NS:
        if not torch.equal(out_h[n], ref[n]):
            raise RuntimeError(f"e2e colour-flow |M|^2 differs from the device-resident run at n={n}")
    h2d = sum(sum(x.numel() * x.element_size() for x in host[n]) for n in COMC_NS)
    n_dom = max(COMC_NS, key=lambda n: kernel_ms[n][1])
    acc_np = ACC[n_dom].cpu().numpy().astype(bool)
    n_orders = int(orders[n_dom][acc_np].sum())
    per_order = canonical_recursion_flops(n_dom) // math.factorial(n_dom - 2)
    flops = per_order * n_orders
    achieved = flops / (kernel_ms[n_dom][1] * 1e-3) / 1e12
    sms = device_sms(dev)
    peak, peak_source = fp32_peak_tflops(sms), fp32_peak_source(sms)
    if prec == bg.BG_F64:
        peak, peak_source = fma_probe_tflops(False, sms, stream, dev, 500), "FP64 FMA probe (measured)"
    if rank == 0:
        print(json.dumps({
            "metric": "events/s", "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": ("colour-flow sampling with colour-ordered amplitudes (Eq. 2.19), flows uniform "
                                    f"in {{1,2,3}}^2 per gluon, n=8,10,12, {batch} Rambo points per n at "
                                    f"sqrt(s)=1 TeV, pT>20 GeV, sampled helicities, {args.precision.upper()} "
                                    "currents"),
                       "n": list(COMC_NS), "batch_per_n": batch, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2"},
            "per_n": {str(n): batch * world / (sum(kernel_ms[n]) * 1e-3) for n in COMC_NS},
            "kernel_ms_per_step": {f"n{n}": [round(x, 3) for x in kernel_ms[n]] for n in COMC_NS},
            "orders_per_event": {str(n): float(orders[n].mean()) for n in COMC_NS},
            "roofline": roofline(f"comc_eval_kernel<{n_dom},{'double' if args.precision == 'f64' else 'float'}>",
                                 "alu", achieved, peak, "TFLOP/s", peak_source,
                                 flops_model=("canonical recursion FLOPs of one order x closing orders of the "
                                              "events passing the cut"),
                                 flops_per_order=per_order, orders_computed=n_orders,
                                 timed_span=("the whole bg_currents_co_mc call: prep, scan, offsets, eval and "
                                             "final kernels")),
            "e2e": {"value": world * len(COMC_NS) * batch * args.steps / e2e_s, "unit": "events/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": len(COMC_NS) * batch * 8},
            "gpu_launches": 6 * len(COMC_NS) * args.steps, "clocks": clk}), flush=True)
    finish_gpu(world)


def run_lc(args) -> None:
    """Leading-colour |M|^2 (Sec. 4) on the default workload's events: n = 5..8,
    2^20 events per n, sampled helicities, FP32 currents, (n-1)! orders."""
    import numpy as np
    import torch
    from paper_2106_06507_gb300 import inputs
    world, rank, dev, bg = setup_gpu()
    stream = torch.cuda.current_stream(dev)
    prec = bg.BG_F64 if args.precision == "f64" else bg.BG_F32
    batch = BATCH if args.precision == "f32" else BATCH >> 4
    first = rank * batch
    U, HEL, P, ACC, ME2, WS, host = {}, {}, {}, {}, {}, {}, {}
    for n in NS:
        u = inputs.rambo_uniforms(n, batch, seed=SEED, first_event=first)
        h = np.ascontiguousarray(inputs.helicities(n, batch, seed=SEED, first_event=first).T)
        U[n], HEL[n] = torch.from_numpy(u).to(dev), torch.from_numpy(h).to(dev)
        host[n] = (torch.from_numpy(u).pin_memory(), torch.from_numpy(h).pin_memory())
        P[n] = torch.empty((4, n, batch), dtype=torch.float64, device=dev)
        ACC[n] = torch.empty((batch,), dtype=torch.uint8, device=dev)
        ME2[n] = torch.empty((batch,), dtype=torch.float64, device=dev)
        WS[n] = torch.empty((bg.lc_workspace_bytes(n, batch, True, prec),), dtype=torch.uint8, device=dev)
    ev = {n: [torch.cuda.Event(enable_timing=True) for _ in range(3)] for n in NS}
    kernel_ms = {n: [0.0, 0.0] for n in NS}

    def step(record=False):
        for n in NS:
            if record:
                ev[n][0].record(stream)
            bg.momenta_rambo(n, U[n], SQRT_S, PT_MIN, p=P[n], accept=ACC[n], stream=stream)
            if record:
                ev[n][1].record(stream)
            bg.currents_lc(n, P[n], HEL[n], prec=prec, sqrt_s=SQRT_S, accept=ACC[n], me2=ME2[n], workspace=WS[n],
                           stream=stream)
            if record:
                ev[n][2].record(stream)

    elapsed, clk = timed_steps(step, args, dev, stream)
    value = world * len(NS) * batch * args.steps / elapsed
    for _ in range(args.steps):
        step(True)
        torch.cuda.synchronize(dev)
        for n in NS:
            for j in range(2):
                kernel_ms[n][j] += ev[n][j].elapsed_time(ev[n][j + 1]) / args.steps
    ref = {n: ME2[n].cpu() for n in NS}
    out_h = {n: torch.empty((batch,), dtype=torch.float64).pin_memory() for n in NS}
    d_in = {n: tuple(torch.empty_like(x, device=dev) for x in host[n]) for n in NS}

    def e2e_step():
        for n in NS:
            for dst, src in zip(d_in[n], host[n]):
                dst.copy_(src, non_blocking=True)
            bg.momenta_rambo(n, d_in[n][0], SQRT_S, PT_MIN, p=P[n], accept=ACC[n], stream=stream)
            bg.currents_lc(n, P[n], d_in[n][1], prec=prec, sqrt_s=SQRT_S, accept=ACC[n], me2=ME2[n],
                           workspace=WS[n], stream=stream)
            out_h[n].copy_(ME2[n], non_blocking=True)

    e2e_s = timed_host(e2e_step, args, dev)
    for n in NS:
        if not torch.equal(out_h[n], ref[n]):
            raise RuntimeError(f"e2e leading-colour |M|^2 differs from the device-resident run at n={n}")
    h2d = sum(sum(x.numel() * x.element_size() for x in host[n]) for n in NS)
    n_dom = max(NS, key=lambda n: kernel_ms[n][1])
    flops = canonical_recursion_flops(n_dom) * (n_dom - 1) * batch  # (n-1)! orders = (n-1) x (n-2)!
    achieved = flops / (kernel_ms[n_dom][1] * 1e-3) / 1e12
    sms = device_sms(dev)
    peak, peak_source = fp32_peak_tflops(sms), fp32_peak_source(sms)
    if prec == bg.BG_F64:
        peak, peak_source = fma_probe_tflops(False, sms, stream, dev, 500), "FP64 FMA probe (measured)"
    if rank == 0:
        print(json.dumps({
            "metric": "events/s", "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": ("leading-colour |M|^2 (Sec. 4), n=5,6,7,8, 2^20 Rambo points per n at "
                                    f"sqrt(s)=1 TeV, pT>20 GeV, sampled helicities, {args.precision.upper()} "
                                    "currents for all (n-1)! orders"),
                       "n": list(NS), "batch_per_n": batch, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2"},
            "per_n": {str(n): batch * world / (sum(kernel_ms[n]) * 1e-3) for n in NS},
            "kernel_ms_per_step": {f"n{n}": [round(x, 3) for x in kernel_ms[n]] for n in NS},
            "roofline": roofline(f"bg_currents_lc at n={n_dom} ({n_dom - 1} recursion launches)", "alu",
                                 achieved, peak, "TFLOP/s", peak_source,
                                 flops_model="canonical recursion FLOPs per order x (n-1)! orders x events",
                                 flops_per_event=canonical_recursion_flops(n_dom) * (n_dom - 1)),
            "e2e": {"value": world * len(NS) * batch * args.steps / e2e_s, "unit": "events/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": len(NS) * batch * 8},
            "gpu_launches": sum(1 + 3 * (n - 1) for n in NS) * args.steps, "clocks": clk}), flush=True)
    finish_gpu(world)


def run_paper(args) -> None:
    """The paper's own setup (Sec. 5): sqrt(s) = 14 TeV, pT > 20 GeV, |eta| < 2.5,
    Delta R > 0.4, colour-ordered n = 5..8, 2^20 events per n, sampled
    helicities, FP32 currents and the exact colour sum (tcgen05 for n >= 6).
    Reports the acceptance, the time split between the recursion and the
    colour sum, and the device bytes per event."""
    import numpy as np
    import torch
    from paper_2106_06507_gb300 import inputs
    world, rank, dev, bg = setup_gpu()
    stream = torch.cuda.current_stream(dev)
    sqrt_s, first = 14000.0, rank * BATCH
    U, HEL, P, ACC, AMPS, ME2, CM, host = {}, {}, {}, {}, {}, {}, {}, {}
    for n in NS:
        u = inputs.rambo_uniforms(n, BATCH, seed=SEED, first_event=first)
        h = np.ascontiguousarray(inputs.helicities(n, BATCH, seed=SEED, first_event=first).T)
        U[n], HEL[n] = torch.from_numpy(u).to(dev), torch.from_numpy(h).to(dev)
        host[n] = (torch.from_numpy(u).pin_memory(), torch.from_numpy(h).pin_memory())
        P[n] = torch.empty((4, n, BATCH), dtype=torch.float64, device=dev)
        ACC[n] = torch.empty((BATCH,), dtype=torch.uint8, device=dev)
        AMPS[n] = torch.empty((BATCH, 1, math.factorial(n - 2)), dtype=torch.float32, device=dev)
        ME2[n] = torch.empty((BATCH,), dtype=torch.float64, device=dev)
        CM[n] = bg.ColourMatrix(n)
    ev = {n: [torch.cuda.Event(enable_timing=True) for _ in range(4)] for n in NS}
    kernel_ms = {n: [0.0, 0.0, 0.0] for n in NS}

    def one(n, u, h, record=False):
        if record:
            ev[n][0].record(stream)
        bg.momenta_rambo(n, u, sqrt_s, PT_MIN, p=P[n], accept=ACC[n], stream=stream)
        bg.apply_cuts(n, P[n], PT_MIN, 2.5, 0.4, accept=ACC[n], stream=stream)
        if record:
            ev[n][1].record(stream)
        bg.currents_co(n, P[n], h, prec=bg.BG_F32, sqrt_s=sqrt_s, amps=AMPS[n], stream=stream)
        if record:
            ev[n][2].record(stream)
        bg.color_sum(CM[n], AMPS[n], True, mode=cs_mode_for(bg, n), sqrt_s=sqrt_s, accept=ACC[n], me2=ME2[n],
                     stream=stream)
        if record:
            ev[n][3].record(stream)

    def step(record=False):
        for n in NS:
            one(n, U[n], HEL[n], record)

    elapsed, clk = timed_steps(step, args, dev, stream)
    value = world * len(NS) * BATCH * args.steps / elapsed
    for _ in range(args.steps):
        step(True)
        torch.cuda.synchronize(dev)
        for n in NS:
            for j in range(3):
                kernel_ms[n][j] += ev[n][j].elapsed_time(ev[n][j + 1]) / args.steps
    ref = {n: ME2[n].cpu() for n in NS}
    out_h = {n: torch.empty((BATCH,), dtype=torch.float64).pin_memory() for n in NS}
    d_in = {n: tuple(torch.empty_like(x, device=dev) for x in host[n]) for n in NS}

    def e2e_step():
        for n in NS:
            for dst, src in zip(d_in[n], host[n]):
                dst.copy_(src, non_blocking=True)
            one(n, d_in[n][0], d_in[n][1])
            out_h[n].copy_(ME2[n], non_blocking=True)

    e2e_s = timed_host(e2e_step, args, dev)
    for n in NS:
        if not torch.equal(out_h[n], ref[n]):
            raise RuntimeError(f"e2e |M|^2 differs from the device-resident run at n={n}")
    acceptance = {str(n): float(ACC[n].float().mean().item()) for n in NS}
    h2d = sum(sum(x.numel() * x.element_size() for x in host[n]) for n in NS)
    n_dom = max(NS, key=lambda n: kernel_ms[n][1])
    achieved = canonical_recursion_flops(n_dom) * BATCH / (kernel_ms[n_dom][1] * 1e-3) / 1e12
    sms = device_sms(dev)
    peak = fp32_peak_tflops(sms)
    # uniforms, momenta, helicities, cut flags, FP32 amplitudes, |M|^2
    bytes_per_event = {str(n): 32 * (n - 2) + 32 * n + n + 1 + 4 * math.factorial(n - 2) + 8 for n in NS}
    for n in NS:
        CM[n].close()
    if rank == 0:
        print(json.dumps({
            "metric": "events/s", "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": ("the paper's setup: colour-ordered BG n=5,6,7,8, 2^20 Rambo points per n at "
                                    "sqrt(s)=14 TeV, pT>20 GeV, |eta|<2.5, Delta R>0.4, sampled helicities, FP32 "
                                    "currents, exact colour sum (tcgen05 for n>=6)"),
                       "n": list(NS), "batch_per_n": BATCH, "sqrt_s_gev": sqrt_s, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2"},
            "per_n": {str(n): BATCH * world / (sum(kernel_ms[n]) * 1e-3) for n in NS},
            "acceptance": acceptance,
            "kernel_ms_per_step": {f"n{n}": {"rambo+cuts": round(kernel_ms[n][0], 3),
                                             "recursion": round(kernel_ms[n][1], 3),
                                             "colour_sum": round(kernel_ms[n][2], 3)} for n in NS},
            "device_bytes_per_event": bytes_per_event,
            "roofline": roofline(f"colour-ordered recursion n={n_dom}", "alu", achieved, peak, "TFLOP/s",
                                 fp32_peak_source(sms), flops_model="canonical recursion FLOPs x events"),
            "e2e": {"value": world * len(NS) * BATCH * args.steps / e2e_s, "unit": "events/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": len(NS) * BATCH * 8},
            "gpu_launches": 4 * len(NS) * args.steps, "clocks": clk}), flush=True)
    finish_gpu(world)


GRAD_NS = (6, 8)
GRAD_BATCH = 1 << 18


def grad_roofline(per_n: dict, dev) -> dict | None:
    """Roofline of the gradient kernel at n = 8: executed FP32 FLOPs per event
    (ncu counters, valid while the kernel sources are those of the capture) x
    the n = 8 events/s of the whole gradient call (Rambo, recursion, colour
    sum, adjoint, Rambo adjoint: a conservative span for the kernel)."""
    fig = ncu_figures(GRAD_SUMMARY)
    if not fig or fig.get("sources_sha1") != sources_sha1(GRAD_SOURCES) or "8" not in per_n:
        return None
    sms = device_sms(dev)
    achieved = fig["executed_flops_per_event"] * per_n["8"] / 1e12
    return roofline("co_grad_kernel<8,float> (reverse-mode gradient)", "alu", achieved, fp32_peak_tflops(sms),
                    "TFLOP/s", fp32_peak_source(sms), flops_model="executed FP32 operations per event (ncu)",
                    executed_flops_per_event=fig["executed_flops_per_event"],
                    ncu_summary=os.path.relpath(GRAD_SUMMARY, ROOT),
                    timed_span="the whole n = 8 gradient call: Rambo, recursion, colour sum, adjoint, Rambo adjoint")


def run_grad(args) -> None:
    import numpy as np
    import torch
    from paper_2106_06507_gb300 import inputs
    world, rank, dev, bg = setup_gpu()
    stream = torch.cuda.current_stream(dev)
    first = rank * GRAD_BATCH
    plans, U, HEL, G, M = {}, {}, {}, {}, {}
    host = {}
    for n in GRAD_NS:
        u = inputs.rambo_uniforms(n, GRAD_BATCH, seed=SEED, first_event=first)
        h = np.ascontiguousarray(inputs.helicities(n, GRAD_BATCH, seed=SEED, first_event=first).T)
        U[n], HEL[n] = torch.from_numpy(u).to(dev), torch.from_numpy(h).to(dev)
        host[n] = (torch.from_numpy(u).pin_memory(), torch.from_numpy(h).pin_memory())
        G[n] = torch.empty_like(U[n])
        M[n] = torch.empty((GRAD_BATCH,), dtype=torch.float64, device=dev)
        plans[n] = bg.Plan(n, GRAD_BATCH, SQRT_S, PT_MIN, prec=bg.BG_F32, cs_mode=bg.BG_CS_F32, hel_sampled=True,
                           grad=True)

    def step():
        for n in GRAD_NS:
            plans[n].grad(U[n], HEL[n], me2=M[n], out=G[n], stream=stream)

    elapsed, clk = timed_steps(step, args, dev, stream)
    value = world * len(GRAD_NS) * GRAD_BATCH * args.steps / elapsed
    per_n = {}
    for n in GRAD_NS:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plans[n].grad(U[n], HEL[n], me2=M[n], out=G[n], stream=stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        per_n[str(n)] = GRAD_BATCH * world / (a.elapsed_time(b) * 1e-3)
    ref = {n: G[n].cpu() for n in GRAD_NS}
    d_in = {n: (torch.empty_like(U[n]), torch.empty_like(HEL[n])) for n in GRAD_NS}
    out_h = {n: (torch.empty((GRAD_BATCH, 4 * (n - 2)), dtype=torch.float64).pin_memory(),
                 torch.empty((GRAD_BATCH,), dtype=torch.float64).pin_memory()) for n in GRAD_NS}

    def e2e_step():
        for n in GRAD_NS:
            d_in[n][0].copy_(host[n][0], non_blocking=True)
            d_in[n][1].copy_(host[n][1], non_blocking=True)
            plans[n].grad(d_in[n][0], d_in[n][1], me2=M[n], out=G[n], stream=stream)
            out_h[n][0].copy_(G[n], non_blocking=True)
            out_h[n][1].copy_(M[n], non_blocking=True)

    e2e_s = timed_host(e2e_step, args, dev)
    for n in GRAD_NS:
        if not (torch.equal(out_h[n][0], ref[n]) and torch.equal(out_h[n][1], M[n].cpu())):
            raise RuntimeError(f"e2e gradient differs from the device-resident run at n={n}")
    h2d = sum(sum(x.numel() * x.element_size() for x in host[n]) for n in GRAD_NS)
    d2h = sum(sum(x.numel() * x.element_size() for x in out_h[n]) for n in GRAD_NS)
    if rank == 0:
        print(json.dumps({
            "metric": "events/s", "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": ("|M|^2 and d|M|^2/du (4(n-2) Rambo uniforms), colour-ordered FP32 with full "
                                    "colour sum, n=6,8, 2^18 events per n, pT>20 GeV, sampled helicities"),
                       "n": list(GRAD_NS), "batch_per_n": GRAD_BATCH, "parallelism": f"replicas x{world}"},
            "per_n": per_n, "roofline": grad_roofline(per_n, dev),
            "e2e": {"value": world * len(GRAD_NS) * GRAD_BATCH * args.steps / e2e_s, "unit": "events/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": 5 * len(GRAD_NS) * args.steps, "clocks": clk}), flush=True)
    for n in GRAD_NS:
        plans[n].close()
    finish_gpu(world)


MIXED_EVENTS = 10_000_000


def mixed_accepted(bg, nev, u, dev) -> dict:
    """Events with n >= 10 of a mixed batch that pass the cut, per n: the
    library's own Rambo and cut on their uniforms (outside any timed region)."""
    import numpy as np
    import torch
    out = {}
    for n in (10, 11, 12):
        idx = np.nonzero(np.asarray(nev) == n)[0]
        if idx.size == 0:
            out[n] = 0
            continue
        un = torch.from_numpy(np.ascontiguousarray(np.asarray(u)[idx, :4 * (n - 2)])).to(dev)
        _, acc = bg.momenta_rambo(n, un, SQRT_S, PT_MIN)
        out[n] = int(acc.sum().item())
    return out


def mixed_roofline(accepted: dict, batch: int, events_per_s: float, dev) -> dict:
    """Roofline of the colour-dressed kernel, which carries most of a mixed
    batch: its dense-model FLOPs for the events with n >= 10 that pass the cut
    (every such event is computed, whether or not its sampled colours give a
    non-zero amplitude) x batches per second of the whole graph (a
    conservative span: every other kernel of the batch runs in that time
    too)."""
    flops = sum(cd_dense_flops(n) * accepted.get(n, 0) for n in (10, 11, 12))
    sms = device_sms(dev)
    achieved = flops * events_per_s / batch / 1e12
    return roofline("cd_kernel<10..12,float> in the mixed batch", "alu", achieved, fp32_peak_tflops(sms), "TFLOP/s",
                    fp32_peak_source(sms), flops_model="dense-model FLOPs of the events with n >= 10 passing the cut",
                    events_computed={str(n): accepted.get(n, 0) for n in (10, 11, 12)},
                    timed_span="the whole graph launch (every multiplicity's kernels)")


def run_mixed(args) -> None:
    import numpy as np
    import torch
    from paper_2106_06507_gb300 import inputs
    world, rank, dev, bg = setup_gpu()
    stream = torch.cuda.current_stream(dev)
    B = MIXED_EVENTS
    ev = inputs.mixed_events(B, 4, 12, seed=SEED + rank, colours="adjoint")
    mx = bg.Mixed(4, 12, B, SQRT_S, PT_MIN, prec=bg.BG_F32, cs_mode=bg.BG_CS_TC_BF16,
                  color_mode=bg.BG_COL_ADJOINT, n_co_max=9, autotune=True)
    host = (torch.from_numpy(ev["nev"]).pin_memory(), torch.from_numpy(ev["u"]).pin_memory(),
            torch.from_numpy(np.ascontiguousarray(ev["hel"].T)).pin_memory(),
            torch.from_numpy(np.ascontiguousarray(ev["colors"].T)).pin_memory())
    dst = (mx.n_per_event, mx.u, mx.hel, mx.colors)
    for d, h in zip(dst, host):
        d.copy_(h)
    torch.cuda.synchronize(dev)

    def step():
        mx.run(B, stream=stream)

    elapsed, clk = timed_steps(step, args, dev, stream)
    value = world * B * args.steps / elapsed
    ref = mx.me2.cpu()
    counts = mx.counts()
    out_h = torch.empty((B,), dtype=torch.float64).pin_memory()

    def e2e_step():
        for d, h in zip(dst, host):
            d.copy_(h, non_blocking=True)
        mx.run(B, stream=stream)
        out_h.copy_(mx.me2, non_blocking=True)

    e2e_s = timed_host(e2e_step, args, dev)
    if not torch.equal(out_h, ref):
        raise RuntimeError("e2e mixed |M|^2 differs from the device-resident run")
    h2d = sum(h.numel() * h.element_size() for h in host)
    tuned = {str(n): bg.tune_get(bg.BG_ALGO_CO if n <= 9 else bg.BG_ALGO_CD, n, bg.BG_F32) for n in range(6, 13)}
    kernels = mx.kernel_nodes()
    rl = mixed_roofline(mixed_accepted(bg, ev["nev"], ev["u"], dev), B, value / world, dev)
    if rank == 0:
        print(json.dumps({
            "metric": "events/s", "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": ("mixed batch, 10^7 events with n uniform in 4..12 in one CUDA-graph launch: "
                                    "colour-ordered + tensor-core colour sum for n=6..9 (FP32 CUDA cores n=4,5), "
                                    "colour-dressed with sampled adjoint colours for n=10..12, FP32 currents, "
                                    "FP64 Rambo and accumulation, pT>20 GeV, autotuned kernel variants"),
                       "events": B, "counts_per_n": counts[4:], "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2", "tuned_variants": tuned,
                       "workspace_gb": mx.workspace_bytes / 1e9},
            "roofline": rl,
            "e2e": {"value": world * B * args.steps / e2e_s, "unit": "events/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": B * 8},
            "gpu_launches": kernels * args.steps, "graph_launches": args.steps, "kernels_per_graph": kernels,
            "clocks": clk}), flush=True)
    mx.close()
    finish_gpu(world)


FORMS_NS = (6, 7, 8, 9)
FORMS_BATCH = {6: 1 << 18, 7: 1 << 18, 8: 1 << 18, 9: 1 << 15}


def tensor_form_flops(n: int) -> int:
    """Canonical FLOPs per event of the tensor form of the colour-ordered
    recursion (all (n-2)! orderings): per split V3 = 65, each tensor
    contraction T X or Y T = 24 (present unless the tensor belongs to a
    single gluon), the wedge into the segment's tensor = 24 (not for the full
    current); propagator = 12, final contraction = 7."""
    m = n - 1
    per_order = 7
    for L in range(2, m + 1):
        segs = m - L + 1
        splits = L - 1
        f = 65 * splits + 24 * 2 * (L - 2)
        if L < m:
            f += 24 * splits + 12
        per_order += segs * f
    return math.factorial(n - 2) * per_order


def run_forms(args) -> None:
    """Four-vertex form against the tensor form (Eqs. 2.23-2.26) of the
    colour-ordered recursion, FP32, sampled helicities: kernel time per event
    of the one-thread-per-ordering kernel with each form, and of the tuned
    depth-first four-vertex kernel.  One JSON line."""
    import numpy as np
    import torch
    from paper_2106_06507_gb300 import inputs
    world, rank, dev, bg = setup_gpu()
    stream = torch.cuda.current_stream(dev)
    rows = {}
    for n in FORMS_NS:
        B = FORMS_BATCH[n]
        u = torch.from_numpy(inputs.rambo_uniforms(n, B, seed=SEED)).to(dev)
        h = torch.from_numpy(np.ascontiguousarray(inputs.helicities(n, B, seed=SEED).T)).to(dev)
        p, acc = bg.momenta_rambo(n, u, SQRT_S, PT_MIN)
        amps = torch.empty((B, 1, math.factorial(n - 2)), dtype=torch.float32, device=dev)
        tuned = bg.autotune(bg.BG_ALGO_CO, n, bg.BG_F32, probe_batch=min(B, 1 << 16), stream=stream)[0]

        def timed(fn):
            for _ in range(args.warmup):
                fn()
            total = 0.0
            for _ in range(args.steps):
                flush_l2(dev)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                torch.cuda.synchronize(dev)
                total += a.elapsed_time(b)
            return total / args.steps

        bg.tune_set(bg.BG_ALGO_CO, n, bg.BG_F32, 0)
        t_v4 = timed(lambda: bg.currents_co(n, p, h, prec=bg.BG_F32, sqrt_s=SQRT_S, amps=amps, stream=stream))
        ref = amps.clone()
        bg.tune_set(bg.BG_ALGO_CO, n, bg.BG_F32, tuned)
        t_dfs = timed(lambda: bg.currents_co(n, p, h, prec=bg.BG_F32, sqrt_s=SQRT_S, amps=amps, stream=stream))
        t_tf = timed(lambda: bg.currents_co(n, p, h, prec=bg.BG_F32, sqrt_s=SQRT_S, amps=amps, stream=stream,
                                            tensor_form=True))
        diff = float(((amps - ref).abs().amax(dim=2) / ref.abs().amax(dim=2).clamp_min(1e-300)).median().item())
        rows[str(n)] = {"batch": B, "tuned_variant": tuned,
                        "ms_per_2^20_events": {"four_vertex_one_thread_per_ordering": t_v4 * (1 << 20) / B,
                                               "four_vertex_depth_first_tuned": t_dfs * (1 << 20) / B,
                                               "tensor_form_one_thread_per_ordering": t_tf * (1 << 20) / B},
                        "canonical_flops_per_event": {"four_vertex": canonical_recursion_flops(n),
                                                      "tensor_form": tensor_form_flops(n)},
                        "tensor_over_four_vertex_time": t_tf / t_v4,
                        "median_rel_amplitude_difference": diff}
    if rank == 0:
        n8 = rows["8"]["ms_per_2^20_events"]
        sms = device_sms(dev)
        achieved = tensor_form_flops(8) * (1 << 20) / (n8["tensor_form_one_thread_per_ordering"] * 1e-3) / 1e12
        rl = roofline("co_kernel<8,float,tensor form>", "alu", achieved, fp32_peak_tflops(sms), "TFLOP/s",
                      fp32_peak_source(sms), flops_model="canonical FLOPs of the tensor form (tensor_form_flops)",
                      flops_per_event=tensor_form_flops(8))
        print(json.dumps({
            "metric": "events/s", "value": (1 << 20) / (n8["tensor_form_one_thread_per_ordering"] * 1e-3),
            "unit": "events/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": n8["tensor_form_one_thread_per_ordering"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": ("colour-ordered recursion alone, four-vertex form against the tensor form, FP32, "
                                    "sampled helicities, pT>20 GeV, n=6..9; value: tensor form at n=8")},
            "forms": rows, "roofline": rl, "e2e": None,
            "gpu_launches": 3 * args.steps * len(FORMS_NS)}), flush=True)
    finish_gpu(world)


def run_profile_case(args) -> None:
    """A small case of one multiplicity for ncu captures: `warmup` steps, then
    one step (Rambo, recursion, colour sum; with --workload cd or comc: Rambo
    once, then the colour-dressed or colour-flow recursion; with --workload
    grad: the plan's gradient call), on cuda:0."""
    import numpy as np
    import torch

    from paper_2106_06507_gb300 import bg, build_lib, inputs
    build_lib.build()
    n, B = args.profile_n, args.profile_batch
    dev = torch.device("cuda", 0)
    if args.workload == "cd":
        u = torch.from_numpy(inputs.rambo_uniforms(n, B, seed=SEED)).to(dev)
        h = torch.from_numpy(np.ascontiguousarray(inputs.helicities(n, B, seed=SEED).T)).to(dev)
        c = torch.from_numpy(np.ascontiguousarray(inputs.adjoint_colours(n, B, seed=SEED).T)).to(dev)
        p, acc = bg.momenta_rambo(n, u, SQRT_S, PT_MIN)
        for _ in range(args.warmup + 1):
            me2 = bg.currents_cd(n, p, h, c, prec=bg.BG_F32, sqrt_s=SQRT_S, accept=acc)
        torch.cuda.synchronize(dev)
        print(json.dumps({"profile_case": {"workload": "cd", "n": n, "batch": B,
                                           "sum_me2": float(me2.sum().item())}}), flush=True)
        return
    if args.workload == "comc":
        u = torch.from_numpy(inputs.rambo_uniforms(n, B, seed=SEED)).to(dev)
        h = torch.from_numpy(np.ascontiguousarray(inputs.helicities(n, B, seed=SEED).T)).to(dev)
        c = torch.from_numpy(np.ascontiguousarray(inputs.flow_colours(n, B, seed=SEED).T)).to(dev)
        p, acc = bg.momenta_rambo(n, u, SQRT_S, PT_MIN)
        for _ in range(args.warmup + 1):
            me2 = bg.currents_co_mc(n, p, h, c, prec=bg.BG_F32, sqrt_s=SQRT_S, accept=acc)
        torch.cuda.synchronize(dev)
        print(json.dumps({"profile_case": {"workload": "comc", "n": n, "batch": B,
                                           "sum_me2": float(me2.sum().item())}}), flush=True)
        return
    if args.workload == "grad":
        u = torch.from_numpy(inputs.rambo_uniforms(n, B, seed=SEED)).to(dev)
        h = torch.from_numpy(np.ascontiguousarray(inputs.helicities(n, B, seed=SEED).T)).to(dev)
        plan = bg.Plan(n, B, SQRT_S, PT_MIN, prec=bg.BG_F32, cs_mode=bg.BG_CS_F32, hel_sampled=True, grad=True)
        for _ in range(args.warmup + 1):
            g = plan.grad(u, h)
        torch.cuda.synchronize(dev)
        print(json.dumps({"profile_case": {"workload": "grad", "n": n, "batch": B,
                                           "sum_abs_grad": float(g.abs().sum().item())}}), flush=True)
        plan.close()
        return
    u = torch.from_numpy(inputs.rambo_uniforms(n, B, seed=SEED)).to(dev)
    h = torch.from_numpy(np.ascontiguousarray(inputs.helicities(n, B, seed=SEED).T)).to(dev)
    C = bg.ColourMatrix(n)
    p = torch.empty((4, n, B), dtype=torch.float64, device=dev)
    acc = torch.empty((B,), dtype=torch.uint8, device=dev)
    amps = torch.empty((B, 1, math.factorial(n - 2)), dtype=torch.float32, device=dev)
    me2 = torch.empty((B,), dtype=torch.float64, device=dev)
    for _ in range(args.warmup + 1):
        bg.momenta_rambo(n, u, SQRT_S, PT_MIN, p=p, accept=acc)
        bg.currents_co(n, p, h, prec=bg.BG_F32, sqrt_s=SQRT_S, amps=amps)
        bg.color_sum(C, amps, True, mode=cs_mode_for(bg, n), sqrt_s=SQRT_S, accept=acc, me2=me2)
    torch.cuda.synchronize(dev)
    print(json.dumps({"profile_case": {"n": n, "batch": B, "sum_me2": float(me2.sum().item())}}), flush=True)
    C.close()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="default workload only: skip the FP64 form and the other workloads in the line")
    ap.add_argument("--workload", choices=("co", "cd", "grad", "mixed", "comc", "lc", "paper", "forms"), default="co")
    ap.add_argument("--precision", choices=("f32", "f64"), default="f32",
                    help="recursion arithmetic of the co and cd workloads (f64: the plain FP64 GPU form)")
    ap.add_argument("--colour-sampling", choices=("adjoint", "continuous"), default="adjoint",
                    help="colour sampling of the cd workload (continuous: colour vectors and polarisation angles)")
    ap.add_argument("--profile-n", type=int, default=0,
                    help="profiling case: run only multiplicity n (warm-up steps, then one step)")
    ap.add_argument("--profile-batch", type=int, default=1 << 16)
    args = ap.parse_args(argv)
    if args.profile_n:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "cd":
        run_cd(args)
    elif args.workload == "grad":
        run_grad(args)
    elif args.workload == "mixed":
        run_mixed(args)
    elif args.workload == "comc":
        run_comc(args)
    elif args.workload == "lc":
        run_lc(args)
    elif args.workload == "paper":
        run_paper(args)
    elif args.workload == "forms":
        run_forms(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
