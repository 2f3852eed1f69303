"""Chunk counts of the colour-dressed kernel (csrc/cd_recursion.cuh), on the
host: the level of subsets of size L has nsub = C(n-1, L) subsets with
npart = 2^L - 2 ordered partitions each, split into c chunks per subset and
colour row (3 c nsub tasks).  For n >= 10 c minimises the rounds of tasks on
a 512-thread CTA times the partitions per chunk, the fewest chunks on ties,
at most four rounds (c = 1 always allowed); the top level likewise with one
subset.  For n <= 9 c is the count that gives about TARGET tasks per level
(256 for n <= 8, 512 for n = 9).  tests/cd_chunks_driver.cu prints the
header's constant expressions; they must equal a brute-force evaluation of
these definitions."""
import math
import shutil
import subprocess

import pytest

from test_comc_rank_host import ROOT


def brute_round(nsub, npart, ref=512):
    best, best_cost = 1, None
    for c in range(1, npart + 1):
        if c > 1 and 3 * nsub * c > 4 * ref:
            break
        cost = math.ceil(3 * nsub * c / ref) * math.ceil(npart / c)
        if best_cost is None or cost < best_cost:
            best, best_cost = c, cost
    return best


def target_rule(n, nsub, npart):
    target = 256 if n <= 8 else 512 if n == 9 else 1024
    tasks = 3 * nsub
    return max(1, min(npart, (target + tasks - 1) // tasks))


@pytest.fixture(scope="module")
def counts(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not shutil.which(nvcc) and not __import__("os").path.exists(nvcc):
        pytest.skip("no nvcc")
    exe = tmp_path_factory.mktemp("cd_chunks") / "cd_chunks_driver"
    csrc = ROOT / "paper_2106_06507_gb300" / "csrc"
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", str(csrc), "-I",
                    str(ROOT / "include"), str(ROOT / "tests" / "cd_chunks_driver.cu"), "-o", str(exe)], check=True)
    out = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        tok = line.split()
        out[int(tok[0])] = (int(tok[2]), [int(x) for x in tok[4:]])
    return out


@pytest.mark.parametrize("n", range(4, 13))
def test_chunk_counts_follow_their_definition(counts, n):
    top, levels = counts[n]
    m = n - 1
    assert len(levels) == max(0, m - 2)
    for L, c in zip(range(2, m), levels):
        nsub, npart = math.comb(m, L), 2 ** L - 2
        want = brute_round(nsub, npart) if n >= 10 else target_rule(n, nsub, npart)
        assert c == want, (n, L)
        assert 1 <= c <= npart
    npart_top = 2 ** m - 2
    target = 256 if n <= 8 else 512 if n == 9 else 1024
    want_top = brute_round(1, npart_top) if n >= 10 else min((target + 2) // 3, npart_top)
    assert top == want_top


def test_round_rule_fills_the_rounds_at_n10(counts):
    # the case that motivated the rule: ~1024 tasks per level on 512 threads
    # left the last of three rounds nearly empty
    _, levels = counts[10]
    for L, c in zip(range(2, 9), levels):
        tasks = 3 * math.comb(9, L) * c
        if tasks > 512:
            assert tasks / (512 * math.ceil(tasks / 512)) > 0.6, (L, c, tasks)
