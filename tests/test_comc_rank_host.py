"""Counting and ranking of the closing orders of a colour flow (the
colour-flow kernel's work list, Eq. 2.19), on the host.

The kernel counts each event's orders (1, s_2, ..., s_n) whose delta chain
closes with the BEST theorem and finds the rank-th of them directly, so that
every order is an independent work item.  tests/comc_rank_driver.cpp compiles
that code (csrc/comc_rank.h) for the CPU; here its count and its full ranked
list are compared with brute force over all (n-1)! orders, in lexicographic
order of the labels: equal, element by element, for random flows at
n = 4..8, for the degenerate flows (all gluons on one colour line: every
order closes; two colours only; a flow whose colour lines fall apart into
two components); at n = 9..12 the full ranked list against a depth-first
search over the colour chain (flows with up to a few thousand orders), and
the count alone against a type-level enumeration.  One rank past the end
must be reported as out of range."""
import itertools
import math
import subprocess

import numpy as np
import pytest

ROOT = __import__("pathlib").Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    exe = tmp_path_factory.mktemp("comc_rank") / "comc_rank_driver"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", str(ROOT / "paper_2106_06507_gb300" / "csrc"),
                    str(ROOT / "tests" / "comc_rank_driver.cpp"), "-o", str(exe)], check=True)
    return exe


def run_driver(exe, flows):
    text = "".join(f"{len(f)} " + " ".join(f"{r} {c}" for r, c in f) + "\n" for f in flows)
    out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True).stdout
    res = []
    for line in out.splitlines():
        tok = line.split()
        if tok[0] == "0":
            res.append(None)
            continue
        cnt = int(tok[1])
        orders = [tuple(int(v) for v in t.split(",")) for t in tok[2:2 + cnt]]
        assert tok[2 + cnt] == "end", line[:200]
        res.append((cnt, orders))
    return res


def closes(flow, order):
    seq = (0,) + order
    return all(flow[seq[k]][1] == flow[seq[(k + 1) % len(seq)]][0] for k in range(len(seq)))


def brute(flow):
    n = len(flow)
    return [o for o in itertools.permutations(range(1, n)) if closes(flow, o)]


def balanced(flow):
    return all(sum(r == c for r, _ in flow) == sum(cc == c for _, cc in flow) for c in range(3))


def random_flows(n, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        f = [tuple(int(x) for x in rng.integers(0, 3, 2)) for _ in range(n)]
        if balanced(f):
            out.append(f)
    return out


@pytest.mark.parametrize("n", [4, 5, 6, 7, 8])
def test_ranked_orders_equal_brute_force(driver, n):
    flows = random_flows(n, {4: 60, 5: 60, 6: 40, 7: 25, 8: 12}[n], seed=300 + n)
    got = run_driver(driver, flows)
    nonzero = 0
    for f, g in zip(flows, got):
        ref = brute(f)
        assert g is not None
        assert g[0] == len(ref), f
        assert g[1] == ref, f
        nonzero += len(ref) > 0
    assert nonzero >= len(flows) // 3


def test_degenerate_flows(driver):
    one_line = [(1, 1)] * 7  # every order closes: (n-1)!
    two_colours = [(0, 1), (1, 0), (0, 1), (1, 0), (0, 0), (1, 1)]
    apart = [(0, 0), (0, 0), (1, 1), (1, 1), (2, 2)]  # no edge joins the colours: no order
    cycle = [(0, 1), (1, 2), (2, 0), (0, 1), (1, 2), (2, 0)]
    flows = [one_line, two_colours, apart, cycle]
    got = run_driver(driver, flows)
    assert got[0][0] == math.factorial(6)
    assert got[2][0] == 0
    for f, g in zip(flows, got):
        ref = brute(f)
        assert (g[0], g[1]) == (len(ref), ref), f


def test_unbalanced_flow_is_reported(driver):
    assert run_driver(driver, [[(0, 1), (0, 0), (1, 1), (2, 2)]]) == [None]


def type_level_count(flow):
    """Closing orders counted over sequences of edge types (gluons with the
    same pair are interchangeable: each type sequence stands for prod m! orders)."""
    from collections import Counter
    r0, c0 = flow[0]
    rest = Counter(flow[1:])

    def walk(x, left):
        if not left:
            return 1 if x == r0 else 0
        tot = 0
        for (r, c), m in list(left.items()):
            if r == x and m > 0:
                left[(r, c)] -= 1
                if left[(r, c)] == 0:
                    del left[(r, c)]
                tot += walk(c, left)
                left[(r, c)] = left.get((r, c), 0) + 1
        return tot

    return walk(c0, dict(rest)) * math.prod(math.factorial(m) for m in rest.values())


@pytest.mark.parametrize("n", [9, 10, 12])
def test_counts_at_large_n(driver, n):
    flows = random_flows(n, 6, seed=400 + n)
    # a heavily degenerate flow: few types, many orders
    flows.append([(0, 0)] * (n // 2) + [(0, 1), (1, 0)] * ((n - n // 2) // 2) + [(1, 1)] * ((n - n // 2) % 2))
    exe_out = run_driver_counts(driver, flows)
    for f, cnt in zip(flows, exe_out):
        assert cnt == type_level_count(f), f


def run_driver_counts(exe, flows):
    text = "".join(f"-{len(f)} " + " ".join(f"{r} {c}" for r, c in f) + "\n" for f in flows)
    out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True).stdout
    return [int(line.split()[1]) if line.split()[0] == "1" else None for line in out.splitlines()]


def dfs_orders(flow):
    """Closing orders in lexicographic label order by depth-first search over
    the colour chain (no (n-1)! enumeration: usable at n = 9..12)."""
    n = len(flow)
    r0 = flow[0][0]
    out, seq, used = [], [], [False] * n

    def rec(x):
        if len(seq) == n - 1:
            if x == r0:
                out.append(tuple(seq))
            return
        for g in range(1, n):
            if not used[g] and flow[g][0] == x:
                used[g] = True
                seq.append(g)
                rec(flow[g][1])
                seq.pop()
                used[g] = False

    rec(flow[0][1])
    return out


@pytest.mark.parametrize("n", [9, 10, 11, 12])
def test_ranked_orders_equal_dfs_at_large_n(driver, n):
    # every order, in order, for random balanced flows with at most a few
    # thousand closing orders each (about 2 * 10^4 orders per n in all)
    flows, total = [], 0
    for f in random_flows(n, 200, seed=600 + n):
        c = type_level_count(f)
        if c <= 5000 and total + c <= 20000:
            flows.append(f)
            total += c
    assert sum(type_level_count(f) > 0 for f in flows) >= 5
    for f, g in zip(flows, run_driver(driver, flows)):
        ref = dfs_orders(f)
        assert g[0] == len(ref) and g[1] == ref, f
