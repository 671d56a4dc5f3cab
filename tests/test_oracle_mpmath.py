"""Pin of the whole oracle against an independent restatement of the method
at 50 significant digits (mpmath).

The restatement below is written in Python from the appendix formulas, one
quantity at a time, with none of the oracle's code: NASA-7 properties
(Appendix A.1), concentrations, Arrhenius rates, third-body
concentrations, the Lindemann / Troe / SRI blending of falloff and
chemically activated reactions, PLOG interpolation, equilibrium constants
from the Gibbs energies (Eq. K_p and the K_c conversion), rates of progress
and their stoichiometric sum (Appendix A.2), the pure-species transport fits
and the Wilke, Mathur and mixture-averaged diffusion rules (Appendix A.3.4,
A.3.5).  Every operation runs at 50 digits, so the restatement is exact to
far below float64 rounding: the differences measured here are the oracle's
own float64 rounding, and any slip in the oracle (a dropped term, a wrong
index, sign or unit) shows up as a disagreement many orders above it.

The readings of the paper where it is silent or garbled are the same on
both sides: log10 in the Troe and SRI forms, Pr floored at 1e-300 before
its logarithm, the T** term of F_cent kept, falloff k_f = k_inf Pr/(1+Pr) F
with c_i = 1, chemically activated k_f = k_0 F/(1+Pr), the efficiency-
weighted mixture (or the named collider) as the falloff third body,
(W_j/W_k)^(1/4) in Wilke's phi_kj, D_jk at one atmosphere scaled by p_atm/p,
the self-diffusion coefficient where the diffusion sum is empty, the low
NASA block below T_mid, kmol-SI units, and concentrations
C_k = (p/RT)(Y_k/W_k)/sum_j Y_j/W_j.

Error measures: production rates per species against the gross rate that
passes through it, sum_i |nu_ki| |c_i| (|k_f prod C^nu'| + |k_r prod C^nu''|)
(the size of the terms whose float64 rounding the oracle carries), as the
largest W_k-weighted value per state; thermo against sum_k |Y_k c_p,k| and
sum_k |Y_k h_k|; transport elementwise relative."""
import math

import numpy as np
import pytest

from paper_2411_02640_gb300 import synth
from paper_2411_02640_gb300.synth import P_ATM, R_U, Reaction
from tests import toys

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp

DPS = 50


def _f(x):
    return mpmath.mpf(float(x))


def _nasa(mech, k, T):
    """cp/R, H/RT, S/R, G/RT of species k at T (Appendix A.1)."""
    a = mech.nasa_lo[k] if T < _f(mech.nasa_T[k][1]) else mech.nasa_hi[k]
    a = [_f(v) for v in a]
    cp = a[0] + a[1] * T + a[2] * T ** 2 + a[3] * T ** 3 + a[4] * T ** 4
    h = a[0] + a[1] * T / 2 + a[2] * T ** 2 / 3 + a[3] * T ** 3 / 4 + a[4] * T ** 4 / 5 + a[5] / T
    s = a[0] * mpmath.log(T) + a[1] * T + a[2] * T ** 2 / 2 + a[3] * T ** 3 / 3 + a[4] * T ** 4 / 4 + a[6]
    return cp, h, s, h - s


def _arrh(abe, T):
    A, beta, E = (_f(v) for v in abe)
    return A * T ** beta * mpmath.exp(-E / T)


def _third_body(r: Reaction, C):
    if r.collider is not None:
        return C[r.collider]
    return mpmath.fsum((_f(r.efficiencies[k]) if k in r.efficiencies else _f(r.default_eff)) * C[k]
                       for k in range(len(C)))


def _blend(r: Reaction, T, Pr):
    """Falloff blending factor F (Lindemann 1, Troe, SRI) with log10."""
    lPr = mpmath.log10(max(Pr, mpmath.mpf("1e-300")))
    if r.troe is not None:
        alpha, T3, T1, T2 = (_f(v) for v in r.troe)
        Fc = (1 - alpha) * mpmath.exp(-T / T3) + alpha * mpmath.exp(-T / T1) + mpmath.exp(-T2 / T)
        lFc = mpmath.log10(Fc)
        c = -mpmath.mpf("0.4") - mpmath.mpf("0.67") * lFc
        n = mpmath.mpf("0.75") - mpmath.mpf("1.27") * lFc
        d = mpmath.mpf("0.14")
        f = (lPr + c) / (n - d * (lPr + c))
        return mpmath.power(10, lFc / (1 + f * f))
    if r.sri is not None:
        a, b, c, d, e = (_f(v) for v in r.sri)
        X = 1 / (1 + lPr * lPr)
        return d * T ** e * (a * mpmath.exp(-b / T) + mpmath.exp(-T / c)) ** X
    return mpmath.mpf(1)


def _plog(r: Reaction, T, p):
    """ln k_f interpolated linearly in ln p between the bracketing pressures;
    the end rates outside the table."""
    tab = sorted(r.plog, key=lambda e: e[0])
    lk = [mpmath.log(_arrh(e[1:], T)) for e in tab]
    lp = [mpmath.log(_f(e[0])) for e in tab]
    x = mpmath.log(p)
    if x <= lp[0]:
        return mpmath.exp(lk[0])
    if x >= lp[-1]:
        return mpmath.exp(lk[-1])
    for m in range(len(tab) - 1):
        if lp[m] <= x <= lp[m + 1]:
            return mpmath.exp(lk[m] + (lk[m + 1] - lk[m]) * (x - lp[m]) / (lp[m + 1] - lp[m]))
    raise AssertionError("pressure not bracketed")


def rates(mech, T, p, Y):
    """Net production rates and the per-species gross rate at one state."""
    ns = mech.n_species
    T, p = _f(T), _f(p)
    Y = [_f(v) for v in Y]
    R, patm = _f(R_U), _f(P_ATM)
    W = [_f(v) for v in mech.W]
    sig = mpmath.fsum(Y[k] / W[k] for k in range(ns))
    CM = p / (R * T)
    C = [CM * (Y[k] / W[k]) / sig for k in range(ns)]
    g = [_nasa(mech, k, T)[3] for k in range(ns)]
    wdot = [mpmath.mpf(0)] * ns
    gross = [mpmath.mpf(0)] * ns
    for r in mech.reactions:
        c = mpmath.mpf(1)
        if r.kind == "elementary":
            kf = _arrh(r.rate, T)
        elif r.kind == "three_body":
            kf = _arrh(r.rate, T)
            c = _third_body(r, C)
        elif r.kind in ("falloff", "chem_act"):
            kinf, k0 = _arrh(r.rate, T), _arrh(r.rate_low, T)
            Pr = k0 * _third_body(r, C) / kinf
            F = _blend(r, T, Pr)
            kf = kinf * Pr / (1 + Pr) * F if r.kind == "falloff" else k0 * F / (1 + Pr)
        elif r.kind == "plog":
            kf = _plog(r, T, p)
        else:
            raise AssertionError(r.kind)
        Rf = kf
        for k, nu in r.reactants:
            Rf *= C[k] ** nu
        Rr = mpmath.mpf(0)
        if r.reversible:
            dnu = sum(nu for _, nu in r.products) - sum(nu for _, nu in r.reactants)
            Kp = mpmath.exp(-(mpmath.fsum(nu * g[k] for k, nu in r.products)
                              - mpmath.fsum(nu * g[k] for k, nu in r.reactants)))
            Kc = Kp * (patm / (R * T)) ** dnu
            Rr = kf / Kc
            for k, nu in r.products:
                Rr *= C[k] ** nu
        q = c * (Rf - Rr)
        G = abs(c) * (abs(Rf) + abs(Rr))
        for k, nu in r.reactants:
            wdot[k] -= nu * q
            gross[k] += nu * G
        for k, nu in r.products:
            wdot[k] += nu * q
            gross[k] += nu * G
    return wdot, gross


def thermo(mech, T, Y):
    """Mass-based mixture c_p and h with the scales sum |Y_k c_p,k|, sum |Y_k h_k|."""
    T = _f(T)
    R = _f(R_U)
    cpk, hk = [], []
    for k in range(mech.n_species):
        cp, h, _, _ = _nasa(mech, k, T)
        cpk.append(_f(Y[k]) * cp * R / _f(mech.W[k]))
        hk.append(_f(Y[k]) * h * R * T / _f(mech.W[k]))
    return mpmath.fsum(cpk), mpmath.fsum(hk), mpmath.fsum(abs(v) for v in cpk), mpmath.fsum(abs(v) for v in hk)


def _poly(c, L):
    return mpmath.fsum(_f(c[n]) * L ** n for n in range(len(c)))


def transport(mech, T, p, Y):
    """Wilke viscosity, Mathur conductivity and mixture-averaged D_k."""
    ns = mech.n_species
    T, p = _f(T), _f(p)
    L = mpmath.log(T)
    W = [_f(v) for v in mech.W]
    direct = mech.transport_fit == "direct"
    if direct:
        eta = [_poly(mech.eta_fit[k], L) for k in range(ns)]
        lam = [_poly(mech.lam_fit[k], L) for k in range(ns)]
        D = [[(1 / _poly(mech.diff_fit[k, j], L)) * _f(P_ATM) / p for j in range(ns)] for k in range(ns)]
    else:
        eta = [mpmath.exp(_poly(mech.eta_fit[k], L)) for k in range(ns)]
        lam = [mpmath.exp(_poly(mech.lam_fit[k], L)) for k in range(ns)]
        D = [[mpmath.exp(_poly(mech.diff_fit[k, j], L)) * _f(P_ATM) / p for j in range(ns)] for k in range(ns)]
    y = [_f(Y[k]) / W[k] for k in range(ns)]
    sig = mpmath.fsum(y)
    X = [v / sig for v in y]
    Wbar = mpmath.fsum(X[k] * W[k] for k in range(ns))
    mu = mpmath.mpf(0)
    for k in range(ns):
        den = mpmath.fsum(X[j] * (1 + mpmath.sqrt(eta[k] / eta[j]) * (W[j] / W[k]) ** mpmath.mpf(0.25)) ** 2
                          / (mpmath.sqrt(8) * mpmath.sqrt(1 + W[k] / W[j])) for j in range(ns))
        mu += X[k] * eta[k] / den
    lm = (mpmath.fsum(X[k] * lam[k] for k in range(ns)) + 1 / mpmath.fsum(X[k] / lam[k] for k in range(ns))) / 2
    Dk = []
    for k in range(ns):
        s = mpmath.fsum(X[j] / D[k][j] for j in range(ns) if j != k)
        Dk.append(D[k][k] if s == 0 else (Wbar - X[k] * W[k]) / Wbar / s)
    return mu, lm, Dk


def _oracle(path):
    import oracle as ora
    return ora.Oracle(path)


def _kinds_mechanism(directory):
    rx = [toys.recomb("elementary"), toys.recomb("three_body", efficiencies={3: 2.0, 0: 0.7}),
          toys.recomb("three_body", collider=3, rate=(3e9, -0.5, 200.0)),
          toys.recomb("falloff", rate=(1e9, 0.3, 400.0), rate_low=(1e12, 0.1, 100.0)),
          toys.recomb("falloff", rate=(5e8, 0.0, 800.0), rate_low=(1e13, -1.1, 100.0), troe=(0.5, 100.0, 2000.0, 3000.0),
                      efficiencies={2: 3.0}),
          toys.recomb("falloff", rate=(2e9, 0.2, 300.0), rate_low=(4e12, 0.1, 500.0), sri=(0.5, 200.0, 1000.0, 1.2, 0.1)),
          toys.recomb("chem_act", rate=(1e9, 0.0, 0.0), rate_low=(1e12, 0.1, 100.0), troe=(0.6, 300.0, 2500.0, 4000.0)),
          toys.recomb("falloff", rate=(1e9, 0.0, 0.0), rate_low=(1e12, 0.0, 0.0), collider=1),
          Reaction(kind="plog", reversible=True, reactants=[(0, 1), (1, 1)], products=[(2, 1)], rate=(0, 0, 0),
                   plog=[(0.1 * P_ATM, 1e9, 0.2, 300.0), (1.0 * P_ATM, 3e9, 0.0, 500.0), (10 * P_ATM, 1e11, -0.3, 900.0)]),
          Reaction(kind="elementary", reversible=False, reactants=[(2, 1)], products=[(0, 1), (1, 1)],
                   rate=(1e13, 0.0, 2e4)),
          Reaction(kind="elementary", reversible=True, reactants=[(2, 2)], products=[(0, 2), (1, 2)],
                   rate=(1e8, 1.5, 5e3)),
          Reaction(kind="elementary", reversible=True, reactants=[(2, 3)], products=[(0, 3), (1, 3)],
                   rate=(1e7, 0.5, 1000.0))]
    return toys.toy("kinds", rx, directory)


def _cases(name, tmp_path, n, seed):
    if name == "kinds":
        mech, path = _kinds_mechanism(str(tmp_path))
        rng = np.random.default_rng(seed)
        T = rng.uniform(300.0, 2800.0, n)
        p = P_ATM * np.exp(rng.uniform(math.log(0.02), math.log(50.0), n))   # below, inside and above the PLOG table
        Y = rng.dirichlet(np.full(mech.n_species, 0.5), n).T.copy()
        return mech, path, T, p, Y
    mech = synth.mechanism(name)
    path = synth.mechanism_file(name, str(tmp_path))
    T, p, Y = synth.make_states(mech.n_species, synth.STATE_SPECS[name], 7 * seed, n)
    return mech, path, T, p, Y


CASES = [("h2o2_9_21", 32), ("kinds", 24), ("gri_53_325", 3)]


@pytest.mark.parametrize("name,n", CASES)
def test_production_rates_match_50_digit_restatement(name, n, tmp_path):
    mp.dps = DPS
    mech, path, T, p, Y = _cases(name, tmp_path, n, seed=5)
    w_ora = _oracle(path).production_rates(T, p, Y)
    W = np.asarray(mech.W)
    worst = 0.0
    for i in range(n):
        w, gross = rates(mech, T[i], p[i], Y[:, i])
        scale = max(float(W[k] * gross[k]) for k in range(mech.n_species))
        err = max(float(W[k] * abs(_f(w_ora[k, i]) - w[k])) for k in range(mech.n_species)) / scale
        worst = max(worst, err)
    assert worst <= 3e-13, worst


@pytest.mark.parametrize("name,n", CASES)
def test_thermo_matches_50_digit_restatement(name, n, tmp_path):
    mp.dps = DPS
    mech, path, T, p, Y = _cases(name, tmp_path, n, seed=6)
    cp_o, h_o = _oracle(path).thermo(T, p, Y)
    for i in range(n):
        cp, h, scp, sh = thermo(mech, T[i], Y[:, i])
        assert abs(_f(cp_o[i]) - cp) <= 1e-14 * scp
        assert abs(_f(h_o[i]) - h) <= 1e-14 * sh


@pytest.mark.parametrize("name,n", CASES + [("h2o2_9_21_direct", 32)])
def test_transport_matches_50_digit_restatement(name, n, tmp_path):
    mp.dps = DPS
    mech, path, T, p, Y = _cases(name, tmp_path, n, seed=8)
    mu_o, lam_o, D_o = _oracle(path).transport(T, p, Y)
    worst = 0.0
    for i in range(n):
        mu, lm, Dk = transport(mech, T[i], p[i], Y[:, i])
        errs = [abs(_f(mu_o[i]) / mu - 1), abs(_f(lam_o[i]) / lm - 1)]
        errs += [abs(_f(D_o[k, i]) / Dk[k] - 1) for k in range(mech.n_species)]
        worst = max(worst, max(float(e) for e in errs))
    assert worst <= 1e-13, worst
