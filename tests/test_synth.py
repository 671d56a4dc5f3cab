"""The seeded input generator: mechanism structure and states."""
import numpy as np
import pytest

from paper_2411_02640_gb300 import synth

SHAPES = {  # species, reactions, three-body, falloff
    "h2o2_9_21": (9, 21, 4, 2),
    "gri_53_325": (53, 325, 30, 29),
    "large_160_900": (160, 900, 72, 54),
}


@pytest.mark.parametrize("name", list(SHAPES))
def test_mechanism_shape_balance_and_coverage(name):
    m = synth.mechanism(name)
    ns, nr, n3, nf = SHAPES[name]
    c = m.counts()
    assert (m.n_species, m.n_reactions, c["three_body"], c["falloff"]) == (ns, nr, n3, nf)
    assert len(set(map(tuple, m.composition))) == ns
    seen = set()
    keys = set()
    for r in m.reactions:
        a = sum(nu * m.composition[k] for k, nu in r.reactants)
        b = sum(nu * m.composition[k] for k, nu in r.products)
        assert np.array_equal(a, b)
        assert len(r.reactants) <= 3 and len(r.products) <= 3
        assert all(nu in (1, 2) for _, nu in r.reactants + r.products)
        assert r.reversible
        lo, hi = r.rate[0], r.rate[0]
        assert 1e6 <= r.rate[0] <= 1e14 and -2 <= r.rate[1] <= 3 and 0 <= r.rate[2] <= 3e4
        if r.kind == "falloff":
            al, t3, t1, t2 = r.troe
            assert 0.4 <= al <= 0.8 and 10 <= t3 <= 1e3 and 1e3 <= t1 <= 1e4 and 1e3 <= t2 <= 1e4
        if r.kind == "three_body":
            assert 1 <= len(r.efficiencies) <= 4
            assert all(0.5 <= a <= 12 for a in r.efficiencies.values())
        key = (tuple(r.reactants), tuple(r.products))
        assert key not in keys
        keys.add(key)
        seen.update(k for k, _ in r.reactants + r.products)
    reactive = set(np.nonzero(~m.inert)[0])
    assert reactive <= seen


@pytest.mark.parametrize("name", list(SHAPES))
def test_mechanism_file_round_trip_is_exact(name, tmp_path):
    m = synth.mechanism(name)
    path = str(tmp_path / "m.kxmech")
    synth.write_mechanism(m, path)
    m2 = synth.read_mechanism(path)
    for f in ("W", "nasa_T", "nasa_lo", "nasa_hi", "eta_fit", "lam_fit", "diff_fit", "composition"):
        assert np.array_equal(getattr(m, f), getattr(m2, f)), f
    for a, b in zip(m.reactions, m2.reactions):
        assert a == b


def test_mechanism_is_deterministic():
    a = synth.make_mechanism(synth.SPECS["gri_53_325"])
    b = synth.make_mechanism(synth.SPECS["gri_53_325"])
    assert np.array_equal(a.nasa_lo, b.nasa_lo) and a.reactions == b.reactions


@pytest.mark.parametrize("name", list(SHAPES))
def test_transport_fits_follow_their_curves(name):
    """The degree-4 fits in ln T reproduce the seeded smooth curves closely
    over 300-3000 K (the curves are smooth, so the residual is small)."""
    m = synth.mechanism(name)
    L = np.log(np.linspace(300, 3000, 50))
    P = np.polynomial.polynomial
    for k in range(m.n_species):
        v = P.polyval(L, m.eta_fit[k])
        assert np.all(np.isfinite(v)) and np.all(np.exp(v) > 1e-7) and np.all(np.exp(v) < 1e-2)
    assert np.array_equal(m.diff_fit, m.diff_fit.transpose(1, 0, 2))


@pytest.mark.parametrize("name", list(SHAPES))
def test_states(name):
    m = synth.mechanism(name)
    sp = synth.STATE_SPECS[name]
    T, p, Y = synth.make_states(m.n_species, sp, 0, 3000)
    assert T.min() >= sp.T_range[0] and T.max() <= sp.T_range[1]
    assert np.all(p >= sp.p_atm_range[0] * synth.P_ATM * (1 - 1e-12))
    assert np.all(p <= sp.p_atm_range[1] * synth.P_ATM * (1 + 1e-12))
    np.testing.assert_allclose(Y.sum(axis=0), 1.0, rtol=1e-14)
    assert np.all(Y > 0)
    # any sub-range is reproducible on its own, across chunk boundaries
    T2, p2, Y2 = synth.make_states(m.n_species, sp, 65530, 20)
    T3, p3, Y3 = synth.make_states(m.n_species, sp, 0, 65550)
    assert np.array_equal(T2, T3[65530:]) and np.array_equal(Y2, Y3[:, 65530:])
