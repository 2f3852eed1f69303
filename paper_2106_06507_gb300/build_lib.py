"""Build libbg.so in-tree for sm_103a (nvcc; translation units compiled in
parallel, then linked).  Output: paper_2106_06507_gb300/_build/libbg.so, and
beside it libbg_probe.so, the FMA-throughput probe the benchmark uses to
measure the pipe peaks (include/bg_probe.h; not part of libbg.so).

    python -m paper_2106_06507_gb300.build_lib [--verbose-ptxas]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libbg.so")
PROBE_LIB = os.path.join(BUILD, "libbg_probe.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-I", INCLUDE, "-I", CSRC] + ARCH

PROBE_SOURCE = "probe.cu"

SOURCES = [
    "api.cu",
    "rambo.cu",
    "co_f32.cu",
    "co_f64.cu",
    "co_tensor.cu",
    "color_sum.cu",
    "color_sum_tc.cu",
    "cd_f32.cu",
    "cd_f64.cu",
    "colormat.cpp",
    "noalloc.cu",
    "co_grad.cu",
    "grad_rambo.cu",
    "mixed.cu",
    "tune.cu",
    "comc_f32.cu",
    "comc_f64.cu",
    "lc.cu",
    "cuts.cu",
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbg.so")


def _deps() -> list[str]:
    out = []
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cuh", ".h", ".cpp")):
                out.append(os.path.join(d, f))
    return out


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(PROBE_LIB):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(PROBE_LIB))
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None) -> str:
    if not force and not verbose_ptxas and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    tool = nvcc()
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []

    def compile_one(src: str) -> tuple[str, str]:
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        path = os.path.join(CSRC, src)
        if src.endswith(".cpp"):
            cmd = [tool, "-x", "c++", "-O2", "-std=c++17", "-Xcompiler", "-fPIC,-pthread", "-I", INCLUDE,
                   "-I", CSRC, "-c", path, "-o", obj]
        else:
            cmd = [tool] + NVCC_FLAGS + extra + ["-c", path, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
        return obj, res.stderr

    srcs = SOURCES + [PROBE_SOURCE]
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose_ptxas:
        for src, (_, log) in zip(srcs, results):
            sys.stdout.write(f"==== {src}\n{log}")

    def link(out: str, objs: list[str]) -> None:
        tmp = out + f".tmp{os.getpid()}"
        cmd = [tool] + ARCH + ["-shared", "-Xcompiler", "-pthread", "-o", tmp] + objs
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, out)

    link(LIB, [o for o, _ in results[:-1]])
    link(PROBE_LIB, [results[-1][0]])
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose_ptxas="--verbose-ptxas" in sys.argv))
