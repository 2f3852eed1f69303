"""Host-side checks of libbg.so that need no GPU: the library builds for
sm_103a, loads, exports every symbol declared in include/bg.h, and its host
colour-matrix generator (U(N) loop counting) agrees with the oracle's
explicit SU(3) contraction."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libbg():
    from paper_2106_06507_gb300 import build_lib
    path = build_lib.build()
    return ctypes.CDLL(path)


def declared_symbols(header: str = "bg.h"):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted({m.group(1) for m in re.finditer(r"\b(bg[a-z0-9_]*_[a-z0-9_]+)\s*\(", text)})


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("bg_momenta_rambo", "bg_currents_co", "bg_color_sum", "bg_colormat_create", "bg_currents_cd",
                     "bg_me2_batch", "bg_me2_grad"):
        assert required in names
    assert sorted(os.listdir(os.path.join(ROOT, "include"))) == ["bg.h", "bg_probe.h"]


def test_library_exports_every_declared_symbol(libbg):
    missing = [n for n in declared_symbols() if not hasattr(libbg, n)]
    assert not missing, missing


def test_binding_loads_without_gpu(libbg):
    # the ctypes binding resolves every entry point it declares (a stale name
    # would fail here, on the CPU, rather than on the GPU machine)
    from paper_2106_06507_gb300 import bg
    L = bg.lib()
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_probe_library_is_separate(libbg):
    # the FMA probe is a measurement utility in its own library, not part of
    # the product ABI
    from paper_2106_06507_gb300 import build_lib
    probe = ctypes.CDLL(build_lib.PROBE_LIB)
    names = declared_symbols("bg_probe.h")
    assert names == ["bgprobe_fma"]
    assert all(hasattr(probe, n) for n in names)
    assert not hasattr(libbg, "bgprobe_fma") and not hasattr(libbg, "bg_probe_fma")


def test_num_orderings(libbg):
    libbg.bg_num_orderings.restype = ctypes.c_int64
    assert [libbg.bg_num_orderings(n) for n in range(3, 14)] == [0, 2, 6, 24, 120, 720, 5040, 40320, 362880,
                                                                  3628800, 0]


@pytest.mark.parametrize("n", [4, 5, 6, 7, 8, 9])
def test_library_colour_row_matches_oracle(libbg, oracle, n):
    # n = 9: the golden row (5040 entries by explicit SU(3) contraction, 8^9
    # terms each, about two hours of the oracle on 8 cores) is read from
    # tests/golden
    import math
    row = np.zeros(math.factorial(n - 2))
    rc = libbg.bg_colormat_row_host(n, row.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert rc == 0
    assert np.array_equal(row, np.round(row))
    assert np.allclose(row, oracle.colour_row(n), rtol=0, atol=1e-6)


def test_library_colour_row_n9_closed_forms(libbg):
    # the closed-form diagonal 8 (2N)^(n-2), integrality and the gcd of the
    # entries at n = 9
    row = np.zeros(5040)
    assert libbg.bg_colormat_row_host(9, row.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == 0
    assert row[0] == 8 * 6**7
    assert np.array_equal(row, np.round(row))
    g = np.gcd.reduce(np.abs(row).astype(np.int64))
    assert g == 432
    assert row.sum() != 0


def test_argument_errors_without_gpu(libbg):
    libbg.bg_last_error.restype = ctypes.c_char_p
    vp = ctypes.c_void_p
    libbg.bg_momenta_rambo.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, vp, vp, ctypes.c_double, vp,
                                       vp]
    assert libbg.bg_momenta_rambo(3, 10, 1000.0, None, None, 0.0, None, None) == 1
    assert b"n must be" in libbg.bg_last_error()
    assert libbg.bg_momenta_rambo(5, -1, 1000.0, None, None, 0.0, None, None) == 1
    assert libbg.bg_momenta_rambo(5, 0, 1000.0, None, None, 0.0, None, None) == 0  # empty batch is a no-op
    assert libbg.bg_momenta_rambo(5, 10, 1000.0, None, None, 0.0, None, None) == 1
    row = np.zeros(10)
    assert libbg.bg_colormat_row_host(10, row.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == 1
    # colour-flow workspace size: argument errors, and the size grows with the batch
    ws = ctypes.c_int64()
    libbg.bg_comc_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
    assert libbg.bg_comc_workspace_bytes(13, 10, 1, ctypes.byref(ws)) == 1
    assert libbg.bg_comc_workspace_bytes(8, -1, 1, ctypes.byref(ws)) == 1
    assert libbg.bg_comc_workspace_bytes(12, 1000, 1, ctypes.byref(ws)) == 0
    small = ws.value
    assert libbg.bg_comc_workspace_bytes(12, 2000, 1, ctypes.byref(ws)) == 0
    assert ws.value - small >= 1000 * (2 * 4 * 12 * 4 + 8 * 66) and ws.value % 256 == 0
    # a mixed plan's kernel count needs a plan
    libbg.bg_mixed_kernel_nodes.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    assert libbg.bg_mixed_kernel_nodes(None, ctypes.byref(ws)) == 1


def test_tune_variant_counts_without_gpu(libbg):
    # colour-ordered: sampled-helicity variants exist from n = 6; colour-
    # dressed: four (CTA size, unrolling) pairs up to n = 9, five above;
    # out of range: 0
    CO, CD = 0, 1
    assert [libbg.bg_tune_num_variants(CO, n) for n in range(4, 10)] == [1, 1, 6, 6, 6, 6]
    assert [libbg.bg_tune_num_variants(CD, n) for n in range(4, 13)] == [4] * 6 + [5] * 3
    assert libbg.bg_tune_num_variants(CO, 10) == 0
    assert libbg.bg_tune_num_variants(CD, 3) == 0
    assert libbg.bg_tune_num_variants(7, 6) == 0
