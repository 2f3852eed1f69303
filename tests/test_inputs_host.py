"""Host tests of the seeded input generators: the mixed-multiplicity batch
draws, for every event, the same numbers as the single-multiplicity
generators at that event's position, and its padding is inert."""
import numpy as np
import pytest

from paper_2106_06507_gb300 import inputs


@pytest.mark.parametrize("colours", ["adjoint", "flow", "balanced_flow"])
def test_mixed_events_match_single_n_generators(colours):
    B = 3000
    ev = inputs.mixed_events(B, 4, 12, seed=5, colours=colours)
    nev = ev["nev"]
    assert np.array_equal(nev, inputs.multiplicities(B, 4, 12, seed=5))
    single_col = {"adjoint": inputs.adjoint_colours, "flow": inputs.flow_colours,
                  "balanced_flow": inputs.balanced_flow_colours}[colours]
    for n in range(4, 13):
        idx = np.nonzero(nev == n)[0]
        assert idx.size > 200
        for e in idx[[0, 1, idx.size // 2, -1]]:
            d = 4 * (n - 2)
            assert np.array_equal(ev["u"][e, :d], inputs.rambo_uniforms(n, 1, seed=5, first_event=e)[0])
            assert np.all(ev["u"][e, d:] == 0.5)
            assert np.array_equal(ev["hel"][e, :n], inputs.helicities(n, 1, seed=5, first_event=e)[0])
            assert np.all(ev["hel"][e, n:] == 1)
            c = single_col(n, 1, seed=5, first_event=e)[0]
            assert np.array_equal(ev["colors"][e, :c.size], c)
            assert np.all(ev["colors"][e, c.size:] == 1)


def test_balanced_flows_are_balanced():
    ev = inputs.mixed_events(2000, 4, 12, seed=6, colours="balanced_flow")
    for e in range(0, 2000, 37):
        n = ev["nev"][e]
        c = ev["colors"][e, :2 * n]
        assert sorted(c[0::2]) == sorted(c[1::2])


def test_multiplicities_uniform():
    nev = inputs.multiplicities(90000, 4, 12, seed=0)
    cnt = np.bincount(nev, minlength=13)[4:]
    assert nev.min() == 4 and nev.max() == 12
    # 9 equally likely values: 10000 expected each, sd ~ 95
    assert np.all(np.abs(cnt - 10000) < 600)
