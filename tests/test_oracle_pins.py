"""Pins of the FP64 oracle against what the paper and the mathematics fix.

The paper prints no property values and its mechanisms are not available,
so the oracle is pinned by hand-worked closed forms (constant-cp species,
power-law transport fits, special Troe parameters), thermodynamic identities
(dH/dT = cp, dS/dT = cp/T, Gibbs-Helmholtz, continuity at Tmid), chemical
equilibrium built from element potentials (every atom-balanced reaction must
then have zero net rate), conservation of mass and elements, the
mass-action orders, the limits of the third-body, falloff and mixing rules,
and the Jacobian against finite differences.  Each pin is chosen so that a
plausible slip (a dropped term, a wrong sign, a swapped index, an inverted
ratio) breaks at least one of them.
"""
import math
import tempfile

import numpy as np
import pytest

import oracle
from paper_2411_02640_gb300 import synth
from paper_2411_02640_gb300.synth import P_ATM, R_U, Reaction
from tests import toys

MECHS = ["h2o2_9_21", "gri_53_325"]


def states(name, n, start=0):
    m = synth.mechanism(name)
    return synth.make_states(m.n_species, synth.STATE_SPECS[name], start, n)


# ------------------------------------------------------------------ thermo (A.1)

def test_constant_cp_species_by_hand(tmp_path):
    """Species with a0 = 3.5, a5 = -1000 K, a6 = 5 at T = 800 K:
    cp/R = 3.5, H/RT = 3.5 - 1000/800 = 2.25,
    S/R = 3.5 ln 800 + 5 = 3.5 * 6.684611727667927 + 5 = 28.396141046837744,
    G/RT = 2.25 - 28.396141046837744 = -26.146141046837744."""
    specs = [("A", {"H": 1}, 3.5, -1000.0, 5.0), ("B", {"O": 1}, 2.5, 0.0, 0.0)]
    _, path = toys.toy("cc", [], str(tmp_path), specs=specs)
    o = oracle.Oracle(path)
    t = o.species_thermo(800.0)
    assert t["cp_R"][0] == pytest.approx(3.5, rel=1e-15)
    assert t["h_RT"][0] == pytest.approx(2.25, rel=1e-15)
    assert t["s_R"][0] == pytest.approx(28.396141046837744, rel=1e-14)
    assert t["g_RT"][0] == pytest.approx(-26.146141046837744, rel=1e-14)
    assert t["g_closed"][0] == pytest.approx(-26.146141046837744, rel=1e-14)


@pytest.mark.parametrize("name", MECHS + ["large_160_900"])
def test_gibbs_closed_form_matches_h_minus_s(oracle_for, name):
    o = oracle_for(name)
    for T in (300.0, 650.0, 999.0, 1000.0, 1700.0, 2800.0):
        t = o.species_thermo(T)
        scale = np.maximum(np.abs(t["h_RT"]), np.abs(t["s_R"]))
        assert np.all(np.abs(t["g_RT"] - t["g_closed"]) <= 1e-13 * scale)


@pytest.mark.parametrize("name", MECHS)
def test_thermo_identities_by_finite_difference(oracle_for, name):
    """d(H/R)/dT = cp/R, d(S/R)/dT = cp/(RT) and d(G/RT)/dT = -H/(RT^2)."""
    o = oracle_for(name)
    for T in (400.0, 800.0, 1500.0, 2500.0):
        d = 1e-3
        a, b, c = o.species_thermo(T - d), o.species_thermo(T), o.species_thermo(T + d)
        dH = ((T + d) * c["h_RT"] - (T - d) * a["h_RT"]) / (2 * d)
        dS = (c["s_R"] - a["s_R"]) / (2 * d)
        dG = (c["g_RT"] - a["g_RT"]) / (2 * d)
        np.testing.assert_allclose(dH, b["cp_R"], rtol=1e-7)
        np.testing.assert_allclose(dS, b["cp_R"] / T, rtol=1e-7)
        np.testing.assert_allclose(dG, -b["h_RT"] / T, rtol=1e-7, atol=1e-9 * np.abs(b["g_RT"]).max() / T)


@pytest.mark.parametrize("name", MECHS + ["large_160_900"])
def test_nasa_blocks_continuous_at_tmid(oracle_for, name):
    o = oracle_for(name)
    below, above = o.species_thermo(np.nextafter(1000.0, 0.0)), o.species_thermo(1000.0)
    for key in ("cp_R", "h_RT", "s_R", "g_RT"):
        np.testing.assert_allclose(below[key], above[key], rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("name", MECHS)
def test_mixture_cp_h_pure_species_and_linearity(oracle_for, name):
    o = oracle_for(name)
    m = synth.mechanism(name)
    ns = m.n_species
    T = np.full(ns, 1234.5); p = np.full(ns, P_ATM)
    cp, h = o.thermo(T, p, np.eye(ns))
    t = o.species_thermo(1234.5)
    np.testing.assert_allclose(cp, t["cp_R"] * R_U / m.W, rtol=1e-14)
    np.testing.assert_allclose(h, t["h_RT"] * R_U * 1234.5 / m.W, rtol=1e-13, atol=1e-9)
    T2, p2, Y = states(name, 2)
    Tm = np.array([T2[0]] * 3); pm = np.array([p2[0]] * 3)
    Ym = np.stack([Y[:, 0], Y[:, 1], 0.3 * Y[:, 0] + 0.7 * Y[:, 1]], axis=1)
    cpm, hm = o.thermo(Tm, pm, Ym)
    assert cpm[2] == pytest.approx(0.3 * cpm[0] + 0.7 * cpm[1], rel=1e-13)
    assert hm[2] == pytest.approx(0.3 * hm[0] + 0.7 * hm[1], rel=1e-12, abs=1e-6 * max(abs(hm[0]), abs(hm[1])))


# ------------------------------------------------------------------ kinetics (A.2)

def equilibrium_state(o, mech, T, seed=0):
    """A composition at chemical equilibrium: chemical potentials
    mu_k/(RT) = G_k/(RT) + ln(p_k/p_atm) built as sum_e n_ke lambda_e, so
    that sum_k nu_ki mu_k = 0 for every atom-balanced reaction."""
    g = o.species_thermo(T)["g_RT"]
    n = mech.composition.astype(float)
    lam, *_ = np.linalg.lstsq(n, g, rcond=None)
    rng = np.random.default_rng(seed)
    lam = lam + rng.uniform(-3.0, 1.0, lam.shape)
    ln_pk = n @ lam - g
    ln_pk = np.clip(ln_pk, -60.0, 8.0)           # clip moves only the inert-free residual directions
    # clipping breaks equilibrium for clipped species; recompute lambda-consistent values instead
    ln_pk = n @ lam - g
    pk = P_ATM * np.exp(ln_pk)
    p = pk.sum()
    X = pk / p
    Y = X * mech.W / (X * mech.W).sum()
    return p, Y


@pytest.mark.parametrize("name", MECHS)
@pytest.mark.parametrize("T", [600.0, 1200.0, 2400.0])
def test_equilibrium_from_element_potentials_has_zero_net_rates(oracle_for, name, T):
    o = oracle_for(name)
    m = synth.mechanism(name)
    p, Y = equilibrium_state(o, m, T)
    d = o.reaction_detail(T, p, Y)
    gross = np.abs(d["c"]) * np.maximum(np.abs(d["Rf"]), np.abs(d["Rr"]))
    assert np.all(gross > 0)
    assert np.all(np.abs(d["q"]) <= 1e-10 * gross), np.max(np.abs(d["q"]) / gross)
    # kf / kr = Kc by construction of kr
    np.testing.assert_allclose(d["kf"] / d["kr"], d["Kc"], rtol=1e-13)


@pytest.mark.parametrize("name", MECHS)
def test_away_from_equilibrium_rates_are_not_zero(oracle_for, name):
    """Guards the equilibrium pin against a trivially zero q."""
    o = oracle_for(name)
    m = synth.mechanism(name)
    p, Y = equilibrium_state(o, m, 1200.0)
    Y2 = Y.copy(); Y2[0] *= 3.0
    d = o.reaction_detail(1200.0, p, Y2)
    gross = np.abs(d["c"]) * np.maximum(np.abs(d["Rf"]), np.abs(d["Rr"]))
    assert np.max(np.abs(d["q"]) / gross) > 1e-3


@pytest.mark.parametrize("name", MECHS + ["large_160_900"])
def test_mass_and_element_conservation(oracle_for, name):
    o = oracle_for(name)
    m = synth.mechanism(name)
    T, p, Y = states(name, 256)
    w = o.production_rates(T, p, Y)
    gross = o.gross_scale(T, p, Y)
    mass = np.abs((m.W[:, None] * w).sum(axis=0))
    assert np.all(mass <= 1e-13 * gross)
    for e in range(len(m.elements)):
        me = synth.ATOMIC_MASS[m.elements[e]]
        el = np.abs((m.composition[:, e][:, None] * w).sum(axis=0)) * me
        assert np.all(el <= 1e-13 * gross)


@pytest.mark.parametrize("name", MECHS)
def test_mass_action_orders_under_pressure_scaling(oracle_for, name):
    """At fixed T and Y, scaling p by s scales every C_k by s, so an
    elementary reaction's k_f prod C^nu' scales by s^(sum nu') and its
    k_r prod C^nu'' by s^(sum nu''); a three-body modifier scales by s."""
    o = oracle_for(name)
    m = synth.mechanism(name)
    T, p, Y = states(name, 1)
    s = 3.0
    a = o.reaction_detail(T[0], p[0], Y[:, 0])
    b = o.reaction_detail(T[0], s * p[0], Y[:, 0])
    for i, r in enumerate(m.reactions):
        if r.kind not in ("elementary", "three_body"):
            continue
        nf = sum(nu for _, nu in r.reactants); nr = sum(nu for _, nu in r.products)
        assert b["Rf"][i] == pytest.approx(a["Rf"][i] * s ** nf, rel=1e-13)
        assert b["Rr"][i] == pytest.approx(a["Rr"][i] * s ** nr, rel=1e-13)
        if r.kind == "three_body":
            assert b["c"][i] == pytest.approx(a["c"][i] * s, rel=1e-13)


@pytest.mark.parametrize("name", MECHS)
def test_arrhenius_parameters_recovered_from_kf(oracle_for, name):
    """ln k_f = ln A + beta ln T - E/T: three temperatures determine (A, beta, E)."""
    o = oracle_for(name)
    m = synth.mechanism(name)
    Ts = [500.0, 1100.0, 2300.0]
    T, p, Y = states(name, 1)
    ks = [o.reaction_detail(t, p[0], Y[:, 0])["kf"] for t in Ts]
    M = np.array([[1.0, math.log(t), -1.0 / t] for t in Ts])
    for i, r in enumerate(m.reactions):
        if r.kind != "elementary" and r.kind != "three_body":
            continue
        sol = np.linalg.solve(M, np.log([k[i] for k in ks]))
        assert math.exp(sol[0]) == pytest.approx(r.rate[0], rel=1e-8)
        assert sol[1] == pytest.approx(r.rate[1], abs=1e-9)
        assert sol[2] == pytest.approx(r.rate[2], rel=1e-8, abs=1e-6)


def test_worked_recombination_by_hand(tmp_path):
    """H + O <=> HO, A = 1e10, beta = 0.5, E/R = 1000 K, at T = 1000 K:
    k_f = 1e10 * sqrt(1000) * e^-1 = 1.16333693845168e11.
    Constant-cp species (a0, a5, a6): H (2.5, 2.5e4, -0.5), O (2.5, 3e4, 2),
    HO (3.5, 4e3, 1.5) give G/RT = a0 (1 - ln T) + a5/T - a6:
    g_H = 2.5(1 - 6.907755278982137) + 25 + 0.5 = 10.730611802544657,
    g_O = 2.5(1 - 6.907755278982137) + 30 - 2 = 13.230611802544657,
    g_HO = 3.5(1 - 6.907755278982137) + 4 - 1.5 = -18.17714347643748,
    ln K_p = -(g_HO - g_H - g_O) = 42.13836708152679, sum nu = -1, so
    K_c = K_p R T / p_atm."""
    _, path = toys.toy("rec", [toys.recomb("elementary")], str(tmp_path))
    o = oracle.Oracle(path)
    T, p = 1000.0, P_ATM
    Y = np.array([0.2, 0.3, 0.4, 0.1])
    d = o.reaction_detail(T, p, Y)
    kf = 1.16333693845167958e11
    assert d["kf"][0] == pytest.approx(kf, rel=1e-14)
    Kc = math.exp(42.13836708152679) * R_U * T / P_ATM
    assert d["Kc"][0] == pytest.approx(Kc, rel=1e-13)
    W = np.array([1.008, 15.999, 1.008 + 15.999, 28.014])
    C = (p / (R_U * T)) * (Y / W) / (Y / W).sum()
    q = kf * C[0] * C[1] - kf / Kc * C[2]
    assert d["q"][0] == pytest.approx(q, rel=1e-13)
    w = o.production_rates([T], [p], Y[:, None])[:, 0]
    np.testing.assert_allclose(w, [-q, -q, q, 0.0], rtol=1e-13)


def test_third_body_unit_and_single_efficiency(tmp_path):
    """All efficiencies 1: [X] = [M] = p/(R T).  A pure species k with
    efficiency alpha: [X] = alpha p/(R T)."""
    r1 = toys.recomb("three_body")
    r2 = toys.recomb("three_body", efficiencies={3: 4.5}, rate=(2e9, 0.0, 0.0))
    _, path = toys.toy("tb", [r1, r2], str(tmp_path))
    o = oracle.Oracle(path)
    T, p = 900.0, 2.5 * P_ATM
    d = o.reaction_detail(T, p, np.array([0.1, 0.2, 0.3, 0.4]))
    assert d["c"][0] == pytest.approx(p / (R_U * T), rel=1e-14)
    d = o.reaction_detail(T, p, np.array([0.0, 0.0, 0.0, 1.0]))
    assert d["c"][1] == pytest.approx(4.5 * p / (R_U * T), rel=1e-14)
    assert d["c"][0] == pytest.approx(p / (R_U * T), rel=1e-14)


def test_single_species_collider(tmp_path):
    r = toys.recomb("three_body", collider=3)
    _, path = toys.toy("col", [r], str(tmp_path))
    o = oracle.Oracle(path)
    T, p = 900.0, P_ATM
    Y = np.array([0.1, 0.2, 0.3, 0.4])
    W = np.array([1.008, 15.999, 17.007, 28.014])
    C = (p / (R_U * T)) * (Y / W) / (Y / W).sum()
    assert o.reaction_detail(T, p, Y)["c"][0] == pytest.approx(C[3], rel=1e-14)


def test_lindemann_limits(tmp_path):
    """Pr -> infinity: k_f -> k_inf; Pr -> 0: k_f -> k_0 [X]."""
    r = toys.recomb("falloff", rate=(1e9, 0.0, 500.0), rate_low=(1e12, 0.0, 0.0))
    _, path = toys.toy("lind", [r], str(tmp_path))
    o = oracle.Oracle(path)
    T = 1000.0
    Y = np.array([0.25, 0.25, 0.25, 0.25])
    kinf = 1e9 * math.exp(-0.5)
    hi = o.reaction_detail(T, 1e4 * P_ATM, Y)
    assert hi["Pr"][0] > 1e5
    assert abs(hi["kf"][0] / kinf - 1.0) <= 1.0 / hi["Pr"][0] * 1.01
    lo = o.reaction_detail(T, 1e-6 * P_ATM, Y)
    assert lo["Pr"][0] < 1e-4
    k0X = 1e12 * lo["X"][0]
    assert abs(lo["kf"][0] / k0X - 1.0) <= lo["Pr"][0] * 1.01
    assert lo["F"][0] == 1.0 and hi["F"][0] == 1.0


def test_troe_center_and_limits(tmp_path):
    """alpha = 0 and T** = 1e30 reduce Fcent to exp(-T/T***); with T*** = T
    that is 1/e.  log F = log Fcent / (1 + f^2) with
    f = (log Pr + c)/(n - d (log Pr + c)) equals log Fcent where
    log Pr = -c (f = 0) and half of it where f = +1 or f = -1, i.e. at
    log Pr = -c + n/(1 + d) and log Pr = -c - n/(1 - d)."""
    T = 1000.0
    r = toys.recomb("falloff", rate=(1e9, 0.0, 0.0), rate_low=(1e12, 0.0, 0.0), troe=(0.0, T, 5000.0, 1e30))
    _, path = toys.toy("troe", [r], str(tmp_path))
    o = oracle.Oracle(path)
    Y = np.array([0.25, 0.25, 0.25, 0.25])
    logFc = math.log10(math.exp(-1.0))
    c = -0.4 - 0.67 * logFc
    n = 0.75 - 1.27 * logFc
    d = 0.14
    # [X] = p/(RT) with unit efficiencies, so Pr = (k0/kinf) p/(RT) = 1e3 p/(RT)
    for lp, F in ((-c, math.exp(-1.0)), (-c + n / (1 + d), math.exp(-0.5)), (-c - n / (1 - d), math.exp(-0.5))):
        pp = 10.0 ** lp / 1e3 * R_U * T
        det = o.reaction_detail(T, pp, Y)
        assert math.log10(det["Pr"][0]) == pytest.approx(lp, abs=1e-12)
        assert det["F"][0] == pytest.approx(F, rel=1e-11)


def _sri_pin_errors(o, T, sri):
    """Largest relative deviation of the oracle's SRI blending factor F from
    the values the SRI form (App. A.2.2) fixes exactly.  With
    X = 1/(1 + (log10 Pr)^2): at log10 Pr = 0, X = 1 and
    F = d T^e (a e^(-b/T) + e^(-T/c)); at log10 Pr = +-1, X = 1/2 (the square
    root of that base); at log10 Pr = +-3, X = 1/10; and as Pr grows without
    bound X -> 0 and F -> d T^e (at log10 Pr = 100, X = 1/10001).
    k_inf = 1e9 and k_0 = 1e12 with unit efficiencies give
    Pr = 1e3 p/(R T), so each log10 Pr is set through p."""
    a, b, c, d, e = sri
    base = a * math.exp(-b / T) + math.exp(-T / c)
    Y = np.array([0.25, 0.25, 0.25, 0.25])
    worst = 0.0
    for lp in (0.0, 1.0, -1.0, 3.0, -3.0, 100.0):
        X = 1.0 / (1.0 + lp * lp)
        want = d * T ** e * base ** X
        det = o.reaction_detail(T, 10.0 ** lp / 1e3 * R_U * T, Y)
        assert math.log10(det["Pr"][0]) == pytest.approx(lp, abs=1e-12)
        dev = abs(det["F"][0] / want - 1.0)
        worst = max(worst, dev if math.isfinite(dev) else math.inf)
    return worst


SRI_CASES = [(1000.0, (0.5, 200.0, 1000.0, 1.2, 0.1)),   # base 0.78
             (1500.0, (3.0, 0.0, 800.0, 0.9, -0.4)),     # a = 3, b = 0: base = 3 + e^(-T/c)
             (700.0, (1.0, 0.0, 300.0, 1.0, 0.0))]      # a = 1, b = 0, d = 1, e = 0: F = (1 + e^(-T/c))^X


def _sri_toy(tmp_path, sri):
    r = toys.recomb("falloff", rate=(1e9, 0.0, 0.0), rate_low=(1e12, 0.0, 0.0), sri=sri)
    return toys.toy("sri", [r], str(tmp_path))[1]


@pytest.mark.parametrize("T,sri", SRI_CASES)
def test_sri_blend_exact_points(tmp_path, T, sri):
    """The SRI factor at the points where X = 1, 1/2, 1/10 and X -> 0."""
    o = oracle.Oracle(_sri_toy(tmp_path, sri))
    assert _sri_pin_errors(o, T, sri) <= 1e-14


SRI_MUTANTS = [
    ("log10(Pr)", "log(Pr)"),   # natural log where the SRI form takes log10 of Pr
    ("d * pow(T, e) * pow(a * exp(-b / T) + exp(-T / c), X)",   # the exponent X over d T^e as well
     "pow(d * pow(T, e) * (a * exp(-b / T) + exp(-T / c)), X)"),
    ("1.0 / (1.0 + lp * lp)", "1.0 / (1.0 + lp)"),   # X without the square
]


@pytest.mark.parametrize("old,new", SRI_MUTANTS)
def test_sri_pins_catch_planted_mistakes(tmp_path, old, new):
    """Planted mistakes in the oracle's SRI factor, compiled on the CPU from a
    copy of its source: the exact points above must reject each."""
    src = open(oracle._SRC).read()
    at = src.index("R sri_F(")
    end = src.index("\n}\n", at)
    body = src[at:end]
    assert body.count(old) == 1
    mutant = src[:at] + body.replace(old, new) + src[end:]
    L = oracle.build_variant(mutant, str(tmp_path / "liboracle_mutant.so"))
    T, sri = SRI_CASES[0]
    o = oracle.Oracle(_sri_toy(tmp_path, sri), library=L)
    assert _sri_pin_errors(o, T, sri) > 1e-3


def test_chemically_activated_and_plog_limits(tmp_path):
    """Chemically activated: k_f -> k_0 as Pr -> 0 (Lindemann F = 1).
    PLOG: at a tabulated pressure k_f is that pressure's Arrhenius rate; at
    the geometric mean of two neighbours ln k_f is the mean of theirs."""
    ca = toys.recomb("chem_act", rate=(1e9, 0.0, 0.0), rate_low=(1e12, 0.0, 800.0))
    pl = Reaction(kind="plog", reversible=True, reactants=[(0, 1), (1, 1)], products=[(2, 1)],
                  rate=(0.0, 0.0, 0.0), plog=[(0.1 * P_ATM, 1e9, 0.2, 300.0), (10 * P_ATM, 1e11, -0.3, 900.0)])
    _, path = toys.toy("capl", [ca, pl], str(tmp_path))
    o = oracle.Oracle(path)
    T = 1000.0
    Y = np.array([0.25, 0.25, 0.25, 0.25])
    d = o.reaction_detail(T, 1e-8 * P_ATM, Y)
    assert abs(d["kf"][0] / (1e12 * math.exp(-0.8)) - 1.0) <= 1.01 * d["Pr"][0]
    k1 = 1e9 * T ** 0.2 * math.exp(-0.3)
    k2 = 1e11 * T ** -0.3 * math.exp(-0.9)
    assert o.reaction_detail(T, 0.1 * P_ATM, Y)["kf"][1] == pytest.approx(k1, rel=1e-13)
    assert o.reaction_detail(T, 10 * P_ATM, Y)["kf"][1] == pytest.approx(k2, rel=1e-13)
    assert o.reaction_detail(T, P_ATM, Y)["kf"][1] == pytest.approx(math.sqrt(k1 * k2), rel=1e-12)


@pytest.mark.parametrize("name", MECHS)
def test_rates_homogeneous_of_degree_zero_in_Y(oracle_for, name):
    o = oracle_for(name)
    T, p, Y = states(name, 16)
    a = o.production_rates(T, p, Y)
    b = o.production_rates(T, p, 3.7 * Y)
    scale = np.abs(a).max(axis=0)
    assert np.all(np.abs(a - b) <= 1e-13 * scale)


@pytest.mark.parametrize("name", ["h2o2_9_21", "gri_53_325"])
def test_jacobian_against_central_differences_and_euler(oracle_for, name):
    o = oracle_for(name)
    m = synth.mechanism(name)
    T, p, Y = states(name, 3, start=7)
    # add cold states, where K_c spans hundreds of decades and its square underflows
    T = np.concatenate([T, [320.0, 380.0, 441.10673386162404]])
    p = np.concatenate([p, p[:3]])
    Y = np.concatenate([Y, Y], axis=1)
    for i in range(6):
        J = o.jacobian(T[i], p[i], Y[:, i])
        # Euler: rates are homogeneous of degree 0 in Y
        eul = J[:, 1:] @ Y[:, i]
        assert np.all(np.abs(eul) <= 1e-10 * (np.abs(J[:, 1:]) @ Y[:, i]) + 1e-300)
        # central differences, h = 1e-6 relative
        h = 1e-6 * T[i]
        fd = (o.production_rates([T[i] + h], [p[i]], Y[:, i:i + 1]) -
              o.production_rates([T[i] - h], [p[i]], Y[:, i:i + 1]))[:, 0] / (2 * h)
        sc = np.abs(J[:, 0]).max()
        assert np.all(np.abs(fd - J[:, 0]) <= 1e-5 * sc)
        for j in range(0, m.n_species, max(1, m.n_species // 7)):
            hy = 1e-6 * max(Y[j, i], 1e-3)
            Yp = Y[:, i].copy(); Yp[j] += hy
            Ym = Y[:, i].copy(); Ym[j] -= hy
            fd = (o.production_rates([T[i]], [p[i]], Yp[:, None]) -
                  o.production_rates([T[i]], [p[i]], Ym[:, None]))[:, 0] / (2 * hy)
            sc = np.abs(J[:, 1 + j]).max()
            assert np.all(np.abs(fd - J[:, 1 + j]) <= 1e-5 * sc + 1e-300)


# ------------------------------------------------------------------ transport (A.3)

def test_power_law_fits_and_pressure_scaling(tmp_path):
    """ln eta = ln eta0 + s ln T gives eta = eta0 T^s exactly; D_kj scales
    as p_atm/p."""
    _, path = toys.toy("tr", [], str(tmp_path), eta0=[2e-5, 3e-5, 4e-5, 5e-5], s_eta=0.7,
                       lam0=[0.03, 0.04, 0.05, 0.06], s_lam=0.8, d0=2e-5)
    o = oracle.Oracle(path)
    eta, lam, D = o.species_transport(1500.0, 2 * P_ATM)
    np.testing.assert_allclose(eta, np.array([2e-5, 3e-5, 4e-5, 5e-5]) * 1500.0 ** 0.7, rtol=1e-13)
    np.testing.assert_allclose(lam, np.array([0.03, 0.04, 0.05, 0.06]) * 1500.0 ** 0.8, rtol=1e-13)
    assert D[1, 2] == pytest.approx(2e-5 * 1.3 * 1500.0 ** 1.75 / 2, rel=1e-13)
    np.testing.assert_allclose(D, D.T, rtol=0)


def test_direct_fits_closed_form(tmp_path):
    """Direct fits (transport_fit direct): eta, lambda and 1/D_kj are the
    polynomials in ln T themselves, no exponential: eta = a + b ln T + c ln^2 T,
    lambda likewise, D_kj = (p_atm/p) / (e0 + e1 ln T); a pure species has
    mu = eta_k, a trace species k in pure j has D_k = D_kj."""
    import dataclasses
    from paper_2411_02640_gb300.synth import write_mechanism
    mech, _ = toys.toy("dir0", [], str(tmp_path))
    ns = mech.n_species
    eta = np.array([[1e-5 * (1 + k), 2e-6, 3e-7, 0, 0] for k in range(ns)])
    lam = np.array([[0.01 * (1 + k), 4e-3, -1e-4, 0, 0] for k in range(ns)])
    dif = np.zeros((ns, ns, 5))
    for j in range(ns):
        for k in range(ns):
            dif[j, k] = [3e4 * (1 + 0.1 * (j + k)), -2e3, 0, 0, 0]
    d = dataclasses.replace(mech, name="dir", eta_fit=eta, lam_fit=lam, diff_fit=dif, transport_fit="direct")
    path = str(tmp_path / "dir.kxmech")
    write_mechanism(d, path)
    o = oracle.Oracle(path)
    T, p = 1234.5, 2.5 * P_ATM
    L = math.log(T)
    e, la, D = o.species_transport(T, p)
    for k in range(ns):
        assert e[k] == pytest.approx(1e-5 * (1 + k) + 2e-6 * L + 3e-7 * L * L, rel=1e-14)
        assert la[k] == pytest.approx(0.01 * (1 + k) + 4e-3 * L - 1e-4 * L * L, rel=1e-14)
    assert D[1, 3] == pytest.approx((P_ATM / p) / (3e4 * 1.4 - 2e3 * L), rel=1e-14)
    mu, lm, Dk = o.transport(np.full(ns, T), np.full(ns, p), np.eye(ns))
    np.testing.assert_allclose(mu, e, rtol=1e-14)
    np.testing.assert_allclose(lm, la, rtol=1e-14)
    Y = np.zeros((ns, 1)); Y[2, 0] = 1.0
    _, _, Dk = o.transport([T], [p], Y)
    assert Dk[0, 0] == pytest.approx(D[0, 2], rel=1e-13)


def test_direct_fits_describe_the_same_curves():
    """The generator's direct fits are least-squares refits of the curves its
    ln fits describe: eta and lambda agree to the refit residual (< 0.5 %)
    between the two forms of the 53/325 mechanism, so reading direct
    coefficients as logarithms (or the reverse) cannot pass."""
    ln_m, dir_m = synth.mechanism("gri_53_325"), synth.mechanism("gri_53_325_direct")
    d = tempfile.mkdtemp()
    o_ln = oracle.Oracle(synth.mechanism_file("gri_53_325", d))
    o_dir = oracle.Oracle(synth.mechanism_file("gri_53_325_direct", d))
    for T in (400.0, 900.0, 1700.0, 2600.0):
        e1, l1, D1 = o_ln.species_transport(T, P_ATM)
        e2, l2, D2 = o_dir.species_transport(T, P_ATM)
        np.testing.assert_allclose(e2, e1, rtol=5e-3)
        np.testing.assert_allclose(l2, l1, rtol=5e-3)
        assert np.all(D2 > 0) and np.all(np.abs(np.log(D2 / D1)) < np.log(2.5))


@pytest.mark.parametrize("name", MECHS)
def test_pure_species_limits(oracle_for, name):
    """A pure species: mu = eta_k (phi_kk = 1), lambda = lambda_k, D_k = D_kk;
    a trace species k in pure j: D_k = D_kj."""
    o = oracle_for(name)
    m = synth.mechanism(name)
    ns = m.n_species
    T, p = 1300.0, 3 * P_ATM
    eta, lam, D = o.species_transport(T, p)
    mu, la, Dk = o.transport(np.full(ns, T), np.full(ns, p), np.eye(ns))
    np.testing.assert_allclose(mu, eta, rtol=1e-14)
    np.testing.assert_allclose(la, lam, rtol=1e-14)
    np.testing.assert_allclose(np.diag(Dk), np.diag(D), rtol=1e-14)
    for k in range(ns):
        for j in range(ns):
            if j != k:
                assert Dk[k, j] == pytest.approx(D[k, j], rel=1e-14)


def test_identical_species_mixture(tmp_path):
    """Species with equal W and equal property fits mix to the same
    property: every phi_kj = 1."""
    specs = [("A", {"H": 1}, 2.5, 0, 0), ("B", {"H": 1}, 2.5, 0, 0), ("C", {"H": 1}, 2.5, 0, 0)]
    _, path = toys.toy("same", [], str(tmp_path), specs=specs, eta0=[3e-5] * 3, lam0=[0.05] * 3)
    o = oracle.Oracle(path)
    Y = np.array([[0.2], [0.5], [0.3]])
    mu, la, _ = o.transport([900.0], [P_ATM], Y)
    eta, lam, _ = o.species_transport(900.0, P_ATM)
    assert mu[0] == pytest.approx(eta[0], rel=1e-14)
    assert la[0] == pytest.approx(lam[0], rel=1e-14)


@pytest.mark.parametrize("name", MECHS)
def test_wilke_phi_reciprocity_and_diagonal(oracle_for, name):
    """phi_kk = 1 and phi_jk = phi_kj (eta_j/eta_k)(W_k/W_j) (Bird, Stewart
    and Lightfoot's reciprocity of Wilke's interaction factors)."""
    o = oracle_for(name)
    m = synth.mechanism(name)
    T = 1400.0
    phi = o.wilke_phi(T)
    eta, _, _ = o.species_transport(T, P_ATM)
    np.testing.assert_allclose(np.diag(phi), 1.0, rtol=1e-15)
    rhs = phi * (eta[None, :] / eta[:, None]) * (m.W[:, None] / m.W[None, :])
    np.testing.assert_allclose(phi.T, rhs, rtol=1e-13)


def test_wilke_binary_by_hand(tmp_path):
    """W = (2, 32), eta = (1e-5, 2e-5) Pa s at T = 1 K (power law with
    s = 0): phi_12 = (1 + sqrt(1/2) * 16^(1/4))^2 / sqrt(8 * (1 + 1/16))
    = (1 + 1.4142135623730951)^2 / sqrt(8.5) = 1.9991340110003848,
    phi_21 = (1 + sqrt(2) * (1/16)^(1/4))^2 / sqrt(8 * 17)
    = (1 + 0.7071067811865476)^2 / sqrt(136) = 0.2498917513750481;
    X = (1/2, 1/2): mu = 1e-5/(1 + phi_12) + 2e-5/(phi_21 + 1)."""
    specs = [("A", {"H": 2}, 3.5, 0, 0), ("B", {"O": 2}, 3.5, 0, 0)]
    _, path = toys.toy("wb", [], str(tmp_path), specs=specs, W=[2.0, 32.0], eta0=[1e-5, 2e-5], s_eta=0.0)
    o = oracle.Oracle(path)
    phi = o.wilke_phi(1.0)
    assert phi[0, 1] == pytest.approx(1.9991340110003848, rel=1e-14)
    assert phi[1, 0] == pytest.approx(0.2498917513750481, rel=1e-14)
    Y = np.array([[2.0 / 34.0], [32.0 / 34.0]])          # equal mole fractions
    mu, _, _ = o.transport([1.0], [P_ATM], Y)
    assert mu[0] == pytest.approx(1e-5 / (1 + 1.9991340110003848) + 2e-5 / (0.2498917513750481 + 1), rel=1e-14)


def test_binary_mixture_diffusion(tmp_path):
    """Two species: D_1 = (W_2 / Wbar) D_12 and D_2 = (W_1 / Wbar) D_12."""
    specs = [("A", {"H": 2}, 3.5, 0, 0), ("B", {"O": 2}, 3.5, 0, 0)]
    _, path = toys.toy("bin", [], str(tmp_path), specs=specs)
    o = oracle.Oracle(path)
    T, p = 1100.0, 0.7 * P_ATM
    Y = np.array([[0.3], [0.7]])
    _, _, D = o.species_transport(T, p)
    _, _, Dk = o.transport([T], [p], Y)
    W = np.array([2.016, 31.998])
    X = (Y[:, 0] / W) / (Y[:, 0] / W).sum()
    Wbar = (X * W).sum()
    assert Dk[0, 0] == pytest.approx(W[1] / Wbar * D[0, 1], rel=1e-13)
    assert Dk[1, 0] == pytest.approx(W[0] / Wbar * D[0, 1], rel=1e-13)


@pytest.mark.parametrize("name", MECHS)
def test_mathur_between_harmonic_and_arithmetic_and_permutation(oracle_for, name, tmp_path):
    o = oracle_for(name)
    m = synth.mechanism(name)
    T, p, Y = states(name, 64)
    mu, la, Dk = o.transport(T, p, Y)
    for i in range(0, 64, 9):
        _, lam, _ = o.species_transport(T[i], p[i])
        X = (Y[:, i] / m.W) / (Y[:, i] / m.W).sum()
        arith, harm = (X * lam).sum(), 1.0 / (X / lam).sum()
        assert harm * (1 - 1e-14) <= la[i] <= arith * (1 + 1e-14)
        assert la[i] == pytest.approx(0.5 * (arith + harm), rel=1e-13)
    # species order is irrelevant to the mixture values
    perm = np.random.default_rng(5).permutation(m.n_species)
    inv = np.argsort(perm)
    pm = synth.Mechanism(m.name, m.elements, [m.species[k] for k in perm], m.composition[perm], m.W[perm],
                         m.inert[perm], m.nasa_T[perm], m.nasa_lo[perm], m.nasa_hi[perm], m.eta_fit[perm],
                         m.lam_fit[perm], m.diff_fit[perm][:, perm], [])
    path = str(tmp_path / "perm.kxmech")
    synth.write_mechanism(pm, path)
    o2 = oracle.Oracle(path)
    mu2, la2, Dk2 = o2.transport(T, p, Y[perm])
    np.testing.assert_allclose(mu2, mu, rtol=1e-13)
    np.testing.assert_allclose(la2, la, rtol=1e-13)
    np.testing.assert_allclose(Dk2[inv], Dk, rtol=1e-13)
