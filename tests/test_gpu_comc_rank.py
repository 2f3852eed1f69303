"""The closing-order counting and ranking (csrc/comc_rank.h) built for the
device equals its host build: tests/comc_rank_device.cu computes every
flow's count and every rank's order in kernels, tests/comc_rank_driver.cpp
on the CPU (itself checked against brute force by test_comc_rank_host.py);
the two outputs must be identical, for random balanced flows at n = 4..12
and the degenerate flows of test_comc_rank_host.py."""
import shutil
import subprocess

import pytest

from test_comc_rank_host import ROOT, random_flows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def exes(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if shutil.which("nvcc") is None:
        pytest.skip("no nvcc")
    d = tmp_path_factory.mktemp("comc_rank_dev")
    inc = str(ROOT / "paper_2106_06507_gb300" / "csrc")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", inc, str(ROOT / "tests" / "comc_rank_driver.cpp"),
                    "-o", str(d / "host")], check=True)
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I", inc,
                    str(ROOT / "tests" / "comc_rank_device.cu"), "-o", str(d / "dev")], check=True)
    return d / "host", d / "dev"


def lines(exe, flows):
    text = "".join(f"{len(f)} " + " ".join(f"{r} {c}" for r, c in f) + "\n" for f in flows)
    return subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True).stdout.splitlines()


@pytest.mark.parametrize("n", [4, 5, 6, 7, 8, 9, 10, 11, 12])
def test_device_ranking_equals_host(exes, n):
    host, dev = exes
    flows = random_flows(n, 40, seed=500 + n)
    if n <= 9:
        flows.append([(1, 1)] * n)  # every order closes
    flows.append([(0, 1), (1, 0)] + [(0, 0)] * (n - 2) if n <= 10 else [(0, 1), (1, 0)] + [(0, 0)] * 7 +
                 [(2, 2)] * (n - 9))  # a flow whose colour lines fall apart: no order at n > 10
    a, b = lines(host, flows), lines(dev, flows)
    assert len(a) == len(flows)
    assert a == b
