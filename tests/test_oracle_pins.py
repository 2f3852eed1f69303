"""Pins of the FP64 oracle against facts fixed by the paper and by the
mathematics, independent of the oracle's own formulas (CPU only).

Each test is chosen so that a plausible slip in the oracle (a dropped
vertex term, a wrong sign or sqrt(2), a transposed colour product, a wrong
boost) fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2106_06507_gb300 import inputs

SQRT_S = 1000.0
Q = (1.0, 0.0, 0.0, 1.0)


def event(O, n, seed=0, i=0):
    u = inputs.rambo_uniforms(n, i + 1, seed=seed)[i]
    p = O.rambo(n, SQRT_S, u)
    return u, p, O.outgoing(p)


def helicity_vector(O, k, t, q=Q):
    """Definite-helicity vector (e1 + i e2)/sqrt2 or its conjugate, labelled by
    the sign of i (p^ x eps_T).eps_T* for the positive-energy momentum p = +-k."""
    e1, e2 = O.polarisations(k, q)
    v = (e1 + 1j * e2) / math.sqrt(2.0)
    p = k if k[0] > 0 else -k
    eT = v[1:] - (v[0] / p[0]) * p[1:]
    ph = p[1:] / np.linalg.norm(p[1:])
    h = (1j * np.dot(np.cross(ph, eT), np.conj(eT)) / np.dot(eT, np.conj(eT))).real
    assert abs(abs(h) - 1.0) < 1e-9
    return v if np.sign(h) == t else np.conj(v)


# --------------------------------------------------------------------------
# Rambo (P7) and flatness
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [4, 5, 6, 8, 10, 12])
def test_rambo_conservation_and_masslessness(oracle, n):
    for i in range(20):
        _, p, k = event(oracle, n, seed=1, i=i)
        assert np.allclose(k.sum(axis=0), 0.0, atol=1e-12 * SQRT_S)
        assert np.all(np.abs(oracle.mdot(k, k)) <= 1e-9 * SQRT_S**2)
        assert abs(p[2:, 0].sum() - SQRT_S) <= 1e-12 * SQRT_S
        assert np.all(p[:, 0] > 0)


def test_rambo_flat_energy_spectrum(oracle):
    # Flat massless n_out-body phase space: x = 2E/sqrt(s) has density
    # (m-1)(m-2) x (1-x)^(m-3), m = n_out, so <x^2> = 6/(m(m+1)); directions
    # are isotropic, <cos^2 theta> = 1/3.
    n = 6
    m = n - 2
    B = 20000
    u = inputs.rambo_uniforms(n, B, seed=7)
    x2 = []
    c2 = []
    for e in range(B):
        p = oracle.rambo(n, SQRT_S, u[e])
        x = 2.0 * p[2:, 0] / SQRT_S
        x2.extend(x * x)
        c2.extend((p[2:, 3] / p[2:, 0]) ** 2)
    assert abs(np.mean(x2) / (6.0 / (m * (m + 1))) - 1.0) < 0.01
    assert abs(np.mean(c2) * 3.0 - 1.0) < 0.01


# --------------------------------------------------------------------------
# polarisations, Eq. (2.2)
# --------------------------------------------------------------------------
def test_polarisation_projector(oracle):
    g = np.diag([1.0, -1.0, -1.0, -1.0])
    for n in (4, 7):
        _, _, k = event(oracle, n, seed=2)
        for i in range(n):
            e1, e2 = oracle.polarisations(k[i], Q)
            for e in (e1, e2):
                assert abs(oracle.mdot(e, e) + 1.0) < 1e-12
                assert abs(oracle.mdot(e, k[i])) < 1e-12 * abs(k[i][0])
            assert abs(oracle.mdot(e1, e2)) < 1e-12
            q = np.array(Q) if abs(oracle.mdot(k[i], Q)) > 1e-9 * abs(k[i][0]) else np.array([1.0, 0, 0, -1.0])
            assert abs(oracle.mdot(e1, q)) < 1e-12 and abs(oracle.mdot(e2, q)) < 1e-12
            # sum_l e_l^mu e_l^nu = -g^{mu nu} + (k^mu q^nu + q^mu k^nu)/(k.q)
            lhs = np.outer(e1, e1) + np.outer(e2, e2)
            rhs = -np.linalg.inv(g) + (np.outer(k[i], q) + np.outer(q, k[i])) / oracle.mdot(k[i], q)
            assert np.allclose(lhs, rhs, atol=1e-9)


# --------------------------------------------------------------------------
# P1: the 4-gluon colour- and helicity-summed |M|^2
# --------------------------------------------------------------------------
def test_four_gluon_closed_form(oracle):
    # sum over all 256 colour and helicity states of |M(gg->gg)|^2 =
    # 256 * (9/2) g^4 (3 - tu/s^2 - su/t^2 - st/u^2)
    g = 1.2
    B = 50
    u = inputs.rambo_uniforms(4, B, seed=3)
    me2 = oracle.me2_co(4, u, sqrt_s=SQRT_S, g=g)
    for e in range(B):
        k = oracle.outgoing(oracle.rambo(4, SQRT_S, u[e]))
        s = oracle.mdot(k[0] + k[1], k[0] + k[1])
        t = oracle.mdot(k[0] + k[2], k[0] + k[2])
        uu = oracle.mdot(k[0] + k[3], k[0] + k[3])
        ref = 1152.0 * g**4 * (3.0 - t * uu / s**2 - s * uu / t**2 - s * t / uu**2)
        assert abs(me2[e] / ref - 1.0) < 1e-12


# --------------------------------------------------------------------------
# P2: Parke-Taylor MHV magnitudes, vanishing all-plus / one-minus
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [4, 5, 6, 7, 8])
def test_parke_taylor(oracle, n):
    _, _, k = event(oracle, n, seed=4)
    order = list(range(n))
    rng = np.random.default_rng(n)
    rng.shuffle(order)

    def s(a, b):
        return 2.0 * oracle.mdot(k[a], k[b])

    den = abs(np.prod([s(order[i], order[(i + 1) % n]) for i in range(n)]))
    pairs = list(itertools.combinations(range(n), 2))
    mags = []
    for (i, j) in pairs[:12]:
        for t0 in (1, -1):
            t = [t0] * n
            t[i] = t[j] = -t0
            eps = np.stack([helicity_vector(oracle, k[a], t[a]) for a in range(n)])
            A = oracle.amp_co_complex(k, eps, order)
            mags.append(abs(A))
            assert abs(abs(A) ** 2 / (s(i, j) ** 4 / den) - 1.0) < 1e-8
    scale = max(mags)
    for t in ([1] * n, [-1] * n, [-1] + [1] * (n - 1), [1, -1] + [-1] * (n - 2)):
        eps = np.stack([helicity_vector(oracle, k[a], t[a]) for a in range(n)])
        assert abs(oracle.amp_co_complex(k, eps, order)) < 1e-10 * scale


# --------------------------------------------------------------------------
# P3: gauge invariance
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [4, 5, 6, 7])
def test_ward_identity(oracle, n):
    _, _, k = event(oracle, n, seed=5)
    hel = inputs.helicities(n, 1, seed=5)[0]
    eps = oracle.pols_for(k, hel)
    order = list(range(n))
    ref = abs(oracle.amp_co(k, eps, order))
    for r in range(min(6, math.factorial(n - 2))):
        o = [0] + list(oracle.ordering(n, r)) + [n - 1]
        a0 = oracle.amp_co(k, eps, o)
        ref = max(ref, abs(a0))
        for i in range(n):
            e2 = eps.copy()
            e2[i] = k[i] * (np.linalg.norm(eps[i]) / abs(k[i][0]))
            assert abs(oracle.amp_co(k, e2, o)) < 1e-10 * max(ref, abs(a0))


@pytest.mark.parametrize("n", [4, 5, 6])
def test_summed_me2_independent_of_reference_vector(oracle, n):
    u = inputs.rambo_uniforms(n, 3, seed=6)
    a = oracle.me2_co(n, u, sqrt_s=SQRT_S, q=(1.0, 0.0, 0.0, 1.0))
    b = oracle.me2_co(n, u, sqrt_s=SQRT_S, q=(1.0, 0.6, 0.0, 0.8))
    c = oracle.me2_co(n, u, sqrt_s=SQRT_S, q=(2.0, -1.2, 1.6, 0.0))
    assert np.allclose(a, b, rtol=1e-11, atol=0)
    assert np.allclose(a, c, rtol=1e-11, atol=0)


# --------------------------------------------------------------------------
# P4: cyclic, reflection, photon decoupling; linear == helicity sums
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [4, 5, 6, 7])
def test_cyclic_reflection_decoupling(oracle, n):
    _, _, k = event(oracle, n, seed=8)
    hel = inputs.helicities(n, 1, seed=8)[0]
    eps = oracle.pols_for(k, hel)
    base = list(range(n))
    a = oracle.amp_co(k, eps, base)
    scale = abs(a)
    for c in range(1, n):
        cyc = base[c:] + base[:c]
        scale = max(scale, abs(oracle.amp_co(k, eps, cyc)))
    for c in range(1, n):
        cyc = base[c:] + base[:c]
        assert abs(oracle.amp_co(k, eps, cyc) - a) < 1e-10 * scale
    assert abs(oracle.amp_co(k, eps, base[::-1]) - (-1) ** n * a) < 1e-10 * scale
    # U(1) decoupling: gluon 1 inserted at every place of the cyclic order of 2..n
    rest = base[1:]
    terms = [oracle.amp_co(k, eps, rest[:j] + [0] + rest[j:]) for j in range(1, n)]
    assert abs(sum(terms)) < 1e-10 * max(abs(t) for t in terms)


@pytest.mark.parametrize("n", [4, 5, 6])
def test_linear_sum_equals_helicity_sum(oracle, n):
    _, _, k = event(oracle, n, seed=9)
    order = list(range(n))
    lin = 0.0
    hel = 0.0
    for conf in range(2**n):
        h = [1 if (conf >> i) & 1 == 0 else -1 for i in range(n)]
        lin += oracle.amp_co(k, oracle.pols_for(k, h), order) ** 2
        eps = np.stack([helicity_vector(oracle, k[a], h[a]) for a in range(n)])
        hel += abs(oracle.amp_co_complex(k, eps, order)) ** 2
    assert abs(lin / hel - 1.0) < 1e-11


# --------------------------------------------------------------------------
# P7: tensor form == V4 form; current conservation
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [4, 5, 6, 7, 8])
def test_tensor_form_equals_v4_form(oracle, n):
    _, _, k = event(oracle, n, seed=10)
    hel = inputs.helicities(n, 1, seed=10)[0]
    eps = oracle.pols_for(k, hel)
    for r in range(min(5, math.factorial(n - 2))):
        o = [0] + list(oracle.ordering(n, r)) + [n - 1]
        Jv, _ = oracle.currents_co(k, eps, o, tensor_form=False)
        Jt, _ = oracle.currents_co(k, eps, o, tensor_form=True)
        assert np.allclose(Jv, Jt, rtol=1e-10, atol=1e-12 * np.abs(Jv).max())


@pytest.mark.parametrize("n", [5, 6, 7, 8])
def test_current_conservation(oracle, n):
    _, _, k = event(oracle, n, seed=11)
    hel = inputs.helicities(n, 1, seed=11)[0]
    eps = oracle.pols_for(k, hel)
    o = [0] + list(oracle.ordering(n, 3)) + [n - 1]
    J, P = oracle.currents_co(k, eps, o)
    m = n - 1
    for i in range(m):
        for j in range(i, m - (1 if i == 0 else 0)):
            scale = np.abs(J[i, j]).max() * np.abs(P[i, j]).max()
            assert abs(oracle.mdot(P[i, j], J[i, j])) <= 1e-10 * scale


# --------------------------------------------------------------------------
# P5: colour matrix, Eq. (2.17)
# --------------------------------------------------------------------------
def test_adjoint_generators(oracle):
    F = oracle.adjoint_generators()
    assert np.abs(F.real).max() < 1e-14  # F = i f with f real
    f = F.imag
    assert np.allclose(f, -np.swapaxes(f, 1, 2), atol=1e-14)
    assert np.allclose(f, -np.swapaxes(f, 0, 1), atol=1e-14)
    # sum_{bc} f^abc f^a'bc = 2 N delta^aa'  (C_A = N with Tr(T^a T^b) = delta)
    assert np.allclose(np.einsum("abc,dbc->ad", f, f), 6.0 * np.eye(8), atol=1e-12)


@pytest.mark.parametrize("n", [4, 5, 6, 7, 8])
def test_colour_matrix_closed_forms(oracle, n):
    C = oracle.colour_matrix(n)
    k = math.factorial(n - 2)
    assert C.shape == (k, k)
    # diagonal: sum_a |(F..F)_{a1 an}|^2 = Tr((sum_b F^b F^b)^(n-2)) = 8 (2N)^(n-2)
    assert np.allclose(np.diag(C), 8.0 * 6.0 ** (n - 2), rtol=1e-12)
    assert np.allclose(C, C.T, rtol=0, atol=1e-9 * C.max())
    # entries are integers (each term of the U(N) expansion is +-N^loops)
    assert np.abs(C - np.round(C)).max() < 1e-6
    # symmetric positive definite
    np.linalg.cholesky(C)


@pytest.mark.parametrize("n", [5, 6, 7, 8, 9])
def test_colour_row_integer_scaling(oracle, n):
    # every entry is a multiple of 432 = 2 N^2 (N^2 - 1) (N = 3); the scaled
    # entries are integers of at most 8 significant bits up to n = 8 (exact in
    # BF16, which the tensor-core colour sum relies on) and within the
    # diagonal 8 (2N)^(n-2) / 432 in magnitude
    row = np.round(oracle.colour_row(n)).astype(np.int64)
    assert np.gcd.reduce(np.abs(row)) == 432
    v = row // 432
    assert np.all(v * 432 == row)
    assert np.abs(v).max() == v[0] == 8 * 6 ** (n - 2) // 432
    nz = np.abs(v[v != 0])
    sh = np.maximum(np.floor(np.log2(nz)).astype(np.int64) - 7, 0)
    exact8 = np.all(((nz >> sh) << sh) == nz)
    # up to n = 8 one BF16 plane holds C / 432 exactly; at n = 9 it does not
    # (the tensor-core path splits C / 432 into two BF16 planes there)
    assert exact8 == (n <= 8)


def test_colour_matrix_depends_on_relative_permutation(oracle):
    for n in (5, 6):
        k = math.factorial(n - 2)
        pairs = np.array([(s, t) for s in range(k) for t in range(k)], dtype=np.int64)
        direct = oracle.colour_entries(n, pairs).reshape(k, k)
        assert np.allclose(direct, oracle.colour_matrix(n), rtol=0, atol=1e-9)


def test_colour_golden_rows_reproduce(oracle):
    for n in (4, 5, 6):
        assert np.allclose(oracle.colour_row_explicit(n), oracle.colour_row(n), rtol=0, atol=1e-9)


# --------------------------------------------------------------------------
# P6: colour-dressed == colour-ordered x colour matrix (brute force)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [4, 5])
def test_colour_dressed_bruteforce_adjoint(oracle, n):
    u = inputs.rambo_uniforms(n, 1, seed=12)
    hel = inputs.helicities(n, 1, seed=12)
    cols = np.array(list(itertools.product(range(1, 9), repeat=n)), dtype=np.int8)
    B = cols.shape[0]
    est = oracle.me2_cd(n, np.repeat(u, B, axis=0), np.repeat(hel, B, axis=0), cols, mode=0, sqrt_s=SQRT_S)
    co = oracle.me2_co(n, u, sqrt_s=SQRT_S, hel=hel)
    assert abs(est.mean() / co[0] - 1.0) < 1e-11


@pytest.mark.parametrize("n", [4, 5])
def test_colour_dressed_bruteforce_flow(oracle, n):
    u = inputs.rambo_uniforms(n, 1, seed=13)
    hel = inputs.helicities(n, 1, seed=13)
    cols = np.array(list(itertools.product(range(1, 4), repeat=2 * n)), dtype=np.int8)
    B = cols.shape[0]
    est = oracle.me2_cd(n, np.repeat(u, B, axis=0), np.repeat(hel, B, axis=0), cols, mode=1, sqrt_s=SQRT_S)
    co = oracle.me2_co(n, u, sqrt_s=SQRT_S, hel=hel)
    assert abs(est.mean() / co[0] - 1.0) < 1e-11


@pytest.mark.parametrize("n", [4, 5, 6])
def test_colour_dressed_current_is_ordering_sum(oracle, n):
    # Eq. (2.28): J(S) = sum over orderings of S of (E_s1 ... E_sL) J(s1..sL)
    _, _, k = event(oracle, n, seed=14)
    hel = inputs.helicities(n, 1, seed=14)[0]
    eps = oracle.pols_for(k, hel)
    E = oracle.externals_for(inputs.adjoint_colours(n, 1, seed=14)[0], 0)
    m = n - 1
    for S in range(1, 2**m):
        labels = [i for i in range(m) if S >> i & 1]
        L = len(labels)
        ref = np.zeros((3, 3, 4))
        mag = 0.0
        for perm in itertools.permutations(labels):
            rest = [i for i in range(n) if i not in perm]
            o = list(perm) + rest
            J, _ = oracle.currents_co(k, eps, o)
            col = np.eye(3)
            for i in perm:
                col = col @ E[i]
            ref += col[:, :, None] * J[0, L - 1][None, None, :]
            mag = max(mag, np.abs(col).max() * np.abs(J[0, L - 1]).max())
        got = oracle.current_cd(k, eps, E, S)
        assert np.allclose(got, ref, rtol=1e-10, atol=1e-12 * mag)


def test_colour_dressed_current_conservation(oracle):
    n = 7
    _, _, k = event(oracle, n, seed=15)
    hel = inputs.helicities(n, 1, seed=15)[0]
    eps = oracle.pols_for(k, hel)
    E = oracle.externals_for(inputs.flow_colours(n, 1, seed=15)[0], 1)
    for S in (0b11, 0b111, 0b10110, 0b111101):
        J = oracle.current_cd(k, eps, E, S)
        P = k[[i for i in range(n - 1) if S >> i & 1]].sum(axis=0)
        scale = np.abs(J).max() * np.abs(P).max() + 1e-300
        assert np.abs(oracle.mdot(P[None, None, :], J)).max() < 1e-10 * scale


# --------------------------------------------------------------------------
# Colour-flow sampling with colour-ordered amplitudes (Eq. 2.19) and the
# leading-colour sum (Sec. 4)
# --------------------------------------------------------------------------
def matched_flows(n, count, seed):
    """Flow pairs whose row colours are a permutation of the column colours
    (the only flows with a non-zero amplitude), plus uniform ones."""
    rng = np.random.default_rng(seed)
    f = np.zeros((count, 2 * n), dtype=np.int8)
    for b in range(count):
        c = rng.integers(1, 4, n)
        r = c[rng.permutation(n)] if b % 4 else rng.integers(1, 4, n)
        f[b, 0::2], f[b, 1::2] = r, c
    return f


@pytest.mark.parametrize("n", [4, 5, 6, 7])
def test_colour_flow_from_ordered_equals_colour_dressed(oracle, n):
    # Eq. (2.19) summed from colour-ordered amplitudes against the
    # independent colour-dressed recursion with the same flow externals
    count = 40
    u = np.repeat(inputs.rambo_uniforms(n, 1, seed=16), count, axis=0)
    hel = np.repeat(inputs.helicities(n, 1, seed=16), count, axis=0)
    fl = matched_flows(n, count, 16 + n)
    a = oracle.me2_co_mc(n, u, hel, fl, sqrt_s=SQRT_S)
    b = oracle.me2_cd(n, u, hel, fl, mode=1, sqrt_s=SQRT_S)
    assert (b > 0).sum() >= count // 2
    # (flows such as all-equal colours cancel to zero by photon decoupling:
    # exact in one form, rounding-level in the other)
    assert np.abs(a - b).max() < 1e-10 * b.max()
    # flows whose rows are not a permutation of the columns vanish exactly
    bad = fl.copy()
    bad[:, 0] = bad[:, 1] % 3 + 1
    bad[:, 2::2] = bad[:, 3::2]
    assert np.all(oracle.me2_co_mc(n, u, hel, bad, sqrt_s=SQRT_S) == 0.0)


@pytest.mark.parametrize("n", [4, 5])
def test_colour_flow_from_ordered_bruteforce(oracle, n):
    # the average over all 9^n flows (weight 9^n each) is the colour sum
    u = inputs.rambo_uniforms(n, 1, seed=17)
    hel = inputs.helicities(n, 1, seed=17)
    cols = np.array(list(itertools.product(range(1, 4), repeat=2 * n)), dtype=np.int8)
    B = cols.shape[0]
    est = oracle.me2_co_mc(n, np.repeat(u, B, axis=0), np.repeat(hel, B, axis=0), cols, sqrt_s=SQRT_S)
    co = oracle.me2_co(n, u, sqrt_s=SQRT_S, hel=hel)
    assert abs(est.mean() / co[0] - 1.0) < 1e-11


@pytest.mark.parametrize("n", [4, 5])
def test_leading_colour_exact_for_four_and_five_gluons(oracle, n):
    # the subleading colour terms of the all-gluon colour sum vanish for
    # n = 4, 5: the leading-colour formula equals the full colour sum
    u = inputs.rambo_uniforms(n, 4, seed=18)
    hel = inputs.helicities(n, 4, seed=18)
    assert np.allclose(oracle.me2_lc(n, u, sqrt_s=SQRT_S), oracle.me2_co(n, u, sqrt_s=SQRT_S), rtol=1e-12, atol=0)
    assert np.allclose(oracle.me2_lc(n, u, hel=hel, sqrt_s=SQRT_S), oracle.me2_co(n, u, hel=hel, sqrt_s=SQRT_S),
                       rtol=1e-12, atol=0)


def test_leading_colour_gauge_invariant_and_subleading_at_six(oracle):
    n = 6
    u = inputs.rambo_uniforms(n, 3, seed=19)
    a = oracle.me2_lc(n, u, sqrt_s=SQRT_S, q=(1.0, 0.0, 0.0, 1.0))
    b = oracle.me2_lc(n, u, sqrt_s=SQRT_S, q=(1.0, 0.6, 0.0, 0.8))
    assert np.allclose(a, b, rtol=1e-11, atol=0)
    # from n = 6 on the formula is an approximation: O(1/N^2) away
    r = a / oracle.me2_co(n, u, sqrt_s=SQRT_S)
    assert np.all(np.abs(r - 1.0) > 1e-8) and np.all(np.abs(r - 1.0) < 0.3)


# --------------------------------------------------------------------------
# Continuous colour and helicity sampling (Sec. 2.1)
# --------------------------------------------------------------------------
# Representatives of the 4 antipodal pairs of cube vertices: the average of
# x_i x_j over them is delta_ij / 3, as over the sphere (|A|^2 is of degree
# two in every colour vector, so this average is exact).
CUBE = np.array([[1, 1, 1], [1, 1, -1], [1, -1, 1], [-1, 1, 1]], dtype=np.float64) / math.sqrt(3.0)


def unit_vector(ct, ph):
    """(cos theta, sin theta cos phi, sin theta sin phi)."""
    st = math.sqrt(max(0.0, 1.0 - ct * ct))
    return np.array([ct, st * math.cos(ph), st * math.sin(ph)])


def angles_of(v):
    """(cos theta, phi) with v = (cos theta, sin theta cos phi, sin theta sin phi)."""
    return float(v[0]), float(math.atan2(v[2], v[1]))


def test_continuous_external_is_fierz_outer_product(oracle):
    # sum_a (eta T^a eta_bar) T^a = |eta_bar><eta| - (eta.eta_bar / N) 1
    rng = np.random.default_rng(20)
    for _ in range(5):
        a = np.array([rng.uniform(-1, 1), rng.uniform(0, 6.28), rng.uniform(-1, 1), rng.uniform(0, 6.28), 0.0])
        eta, etab = unit_vector(a[0], a[1]), unit_vector(a[2], a[3])
        ref = np.outer(etab, eta) - np.dot(eta, etab) / 3.0 * np.eye(3)
        assert np.abs(oracle.continuous_external(a) - ref).max() < 1e-14


@pytest.mark.parametrize("n", [4, 6])
def test_continuous_trace_part_decouples(oracle, n):
    # the -1/N trace part of sum_a eta^a T^a is a U(1) gluon, which decouples
    # from all-gluon amplitudes: the outer product |eta_bar><eta| alone gives
    # the same amplitude
    _, _, k = event(oracle, n, seed=23)
    hel = inputs.helicities(n, 1, seed=23)[0]
    eps = oracle.pols_for(k, hel)
    ang = inputs.continuous_angles(n, 1, seed=23)[0]
    E = np.stack([oracle.continuous_external(a) for a in ang])
    outer = np.stack([np.outer(unit_vector(a[2], a[3]), unit_vector(a[0], a[1])) for a in ang])
    a1 = oracle.amp_cd(k, eps, E)
    a2 = oracle.amp_cd(k, eps, outer)
    assert abs(a1 - a2) <= 1e-12 * abs(a1)


def test_continuous_colour_average_is_colour_sum(oracle):
    # exact average over colour vectors from the cube design (4 x 4 per
    # gluon) at a fixed polarisation angle 0 (e1 for every gluon) = the
    # colour-summed |M|^2 of that polarisation configuration
    n = 4
    u = inputs.rambo_uniforms(n, 1, seed=21)
    states = [angles_of(x) + angles_of(y) for x in CUBE for y in CUBE]
    ang = np.array([[s[0], s[1], s[2], s[3], 0.0] for s in states])
    combos = np.array(list(itertools.product(range(len(states)), repeat=n)))
    A = ang[combos]  # [B, n, 5]
    est = oracle.me2_cd_cont(n, np.repeat(u, A.shape[0], axis=0), A, sqrt_s=SQRT_S)
    co = oracle.me2_co(n, u, sqrt_s=SQRT_S, hel=np.ones((1, n), dtype=np.int8))
    assert abs(est.mean() / co[0] - 1.0) < 1e-11


@pytest.mark.parametrize("n", [4, 5])
def test_continuous_polarisation_average_is_helicity_sum(oracle, n):
    # the polarisation angle averaged over {0, 2pi/3, 4pi/3} per gluon (exact
    # for cos^2, sin^2, cos sin) with weight 2 each = the sum over the two
    # linear polarisations, here for one fixed colour-vector assignment
    u = inputs.rambo_uniforms(n, 1, seed=22 + n)
    base = inputs.continuous_angles(n, 1, seed=22 + n)[0]
    combos = np.array(list(itertools.product(range(3), repeat=n)))
    A = np.repeat(base[None], combos.shape[0], axis=0).copy()
    A[:, :, 4] = combos * (2.0 * math.pi / 3.0)
    est = oracle.me2_cd_cont(n, np.repeat(u, A.shape[0], axis=0), A, sqrt_s=SQRT_S).mean()
    ref = 0.0
    for lam in itertools.product((0.0, 0.5 * math.pi), repeat=n):
        B1 = base.copy()
        B1[:, 4] = lam
        ref += oracle.me2_cd_cont(n, u, B1[None], sqrt_s=SQRT_S)[0] / 2 ** n
    assert abs(est / ref - 1.0) < 1e-11


# --------------------------------------------------------------------------
# The paper's kinematic constraints (Sec. 5)
# --------------------------------------------------------------------------
def test_eta_cut_acceptance_closed_form(oracle):
    # isotropic back-to-back gluons (n = 4): |eta| < eta_max <=> |cos theta| <
    # tanh(eta_max), so the acceptance is tanh(eta_max); pT and Delta R cuts off
    n, B = 4, 200000
    u = inputs.rambo_uniforms(n, B, seed=30)
    for eta_max in (0.5, 2.5):
        acc = oracle.accept_cuts(n, u, sqrt_s=14000.0, pt_min=-1.0, eta_max=eta_max, dr_min=0.0)
        p = math.tanh(eta_max)
        assert abs(acc.mean() - p) < 4.0 * math.sqrt(p * (1 - p) / B)
    # back to back: Delta eta = 2 |eta|, Delta phi = pi > 0.4, every event passes
    assert oracle.accept_cuts(n, u[:1000], sqrt_s=14000.0, pt_min=-1.0, eta_max=0.0, dr_min=0.4).all()


@pytest.mark.parametrize("n", [5, 7])
def test_cuts_against_direct_evaluation(oracle, n):
    # eta from arctanh(p_z/|p|) and Delta phi from the angle between the
    # transverse momenta (a route independent of the oracle's polar-angle
    # form and of its folding of the azimuth difference)
    B = 3000
    u = inputs.rambo_uniforms(n, B, seed=31)
    got = oracle.accept_cuts(n, u, sqrt_s=14000.0, pt_min=20.0, eta_max=2.5, dr_min=0.4)
    ref = np.zeros(B, dtype=np.uint8)
    for e in range(B):
        p = oracle.rambo(n, 14000.0, u[e])[2:]
        pt = np.hypot(p[:, 1], p[:, 2])
        eta = np.arctanh(p[:, 3] / np.linalg.norm(p[:, 1:], axis=1))
        ok = np.all(pt > 20.0) and np.all(np.abs(eta) < 2.5)
        for i in range(n - 2):
            for j in range(i + 1, n - 2):
                c = np.dot(p[i, 1:3], p[j, 1:3]) / (pt[i] * pt[j])
                dphi = math.acos(max(-1.0, min(1.0, c)))
                ok = ok and (eta[i] - eta[j]) ** 2 + dphi ** 2 > 0.16
        ref[e] = ok
    assert np.array_equal(got, ref)
    assert 0.05 < got.mean() < 0.95


# --------------------------------------------------------------------------
# P8: gradient with respect to the Rambo uniforms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [4, 5])
def test_gradient_dual_vs_central_differences(oracle, n):
    u = inputs.rambo_uniforms(n, 1, seed=16)[0]
    hel = inputs.helicities(n, 1, seed=16)[0]
    v, grad = oracle.me2_co_grad(n, u, hel, sqrt_s=SQRT_S)
    assert abs(v / oracle.me2_co(n, u[None], sqrt_s=SQRT_S, hel=hel[None])[0] - 1.0) < 1e-12
    h = 1e-6
    for j in range(u.size):
        up = u.copy(); up[j] += h
        um = u.copy(); um[j] -= h
        fd = (oracle.me2_co(n, up[None], sqrt_s=SQRT_S, hel=hel[None])[0]
              - oracle.me2_co(n, um[None], sqrt_s=SQRT_S, hel=hel[None])[0]) / (2 * h)
        assert abs(fd - grad[j]) <= 1e-5 * np.abs(grad).max()
