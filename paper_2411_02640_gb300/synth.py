"""Seeded synthetic reaction mechanisms and thermochemical states.

This module is the one source of inputs shared by the CPU oracle and the
GPU path.  It builds *inputs* only: species, atom-balanced reactions,
Arrhenius/Troe/third-body parameters, NASA-7 and transport-fit coefficients,
and batches of states (T, p, Y_k).  It evaluates none of the quantities the
method computes (rates of progress, production rates, equilibrium constants,
mixture properties); the few integrals it takes to make the NASA-7 blocks
consistent use numpy's polynomial primitives on the drawn cp curve.

The paper's benchmark mechanisms (H2/O2, GRI-Mech 3.0, ethanol; Table 1) are
not available here, so mechanisms of the same size and reaction-type mix are
drawn from a seed:

* species: distinct elemental compositions within per-element ranges,
  molecular weights from standard atomic masses;
* reactions: reversible, atom-balanced, at most three species per side and
  stoichiometric coefficients in {1, 2}; three-body and falloff reactions are
  recombinations A + B (+M) <=> AB;
* Arrhenius A log-uniform in [1e6, 1e14] (SI, kmol), beta U[-2, 3],
  E/R U[0, 3e4] K; Troe alpha U[0.4, 0.8], T*** U[10, 1e3] K,
  T*, T** U[1e3, 1e4] K; third-body efficiencies U[0.5, 12] on 1-4 species;
* NASA-7 (Appendix A.1) blocks on [300, 1000] and [1000, 3000] K fitted by
  constrained least squares to cp/R = a + b tanh((T - T0)/w), continuous in
  cp, h and s at 1000 K, with h_f U[-3e5, 5e5] J/mol and s(298.15)
  U[100, 250] J/mol/K;
* transport (Appendix A.3.5): degree-4 fits in ln T of ln eta_k, ln lambda_k
  and ln D_jk (at one atmosphere) to smooth seeded curves over 300-3000 K.

Units are SI with kmol throughout: W in kg/kmol, concentrations in kmol/m^3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from itertools import combinations_with_replacement
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

R_U = 8314.46261815324        # J/(kmol K), universal gas constant
P_ATM = 101325.0              # Pa

ATOMIC_MASS = {"H": 1.008, "C": 12.011, "N": 14.007, "O": 15.999, "Ar": 39.95}

KINDS = ("elementary", "three_body", "falloff", "chem_act", "plog")


@dataclass
class Reaction:
    """One reaction.  ``rate`` is k_f (elementary, three-body), k_inf
    (falloff) or the high-pressure constant of a chemically activated
    reaction; ``rate_low`` is k_0 for falloff and chemically activated
    reactions (Sec. A.2.2)."""
    kind: str
    reversible: bool
    reactants: List[Tuple[int, int]]
    products: List[Tuple[int, int]]
    rate: Tuple[float, float, float]
    rate_low: Optional[Tuple[float, float, float]] = None
    default_eff: float = 1.0
    efficiencies: Dict[int, float] = field(default_factory=dict)
    collider: Optional[int] = None          # single-species third body [X_m]
    troe: Optional[Tuple[float, float, float, float]] = None   # alpha, T***, T*, T**
    sri: Optional[Tuple[float, float, float, float, float]] = None  # a, b, c, d, e
    plog: Optional[List[Tuple[float, float, float, float]]] = None  # (p, A, beta, E/R)

    def uses_third_body(self) -> bool:
        return self.kind in ("three_body", "falloff", "chem_act")


@dataclass
class Mechanism:
    name: str
    elements: List[str]
    species: List[str]
    composition: np.ndarray          # [Ns, Ne] int
    W: np.ndarray                    # [Ns] kg/kmol
    inert: np.ndarray                # [Ns] bool
    nasa_T: np.ndarray               # [Ns, 3]  Tlow, Tmid, Thigh
    nasa_lo: np.ndarray              # [Ns, 7]
    nasa_hi: np.ndarray              # [Ns, 7]
    eta_fit: np.ndarray              # [Ns, 5]  ln eta   = sum c_n (ln T)^n, Pa s
    lam_fit: np.ndarray              # [Ns, 5]  ln lambda = ..., W/(m K)
    diff_fit: np.ndarray             # [Ns, Ns, 5] ln D_jk at p_atm, m^2/s (symmetric)
    reactions: List[Reaction]
    # "ln": the three fits are of ln eta, ln lambda, ln D_jk; "direct": of eta, lambda and of the
    # reciprocal 1/D_jk themselves (the paper's polynomial fits, evaluated without exponentials)
    transport_fit: str = "ln"

    @property
    def n_species(self) -> int:
        return len(self.species)

    @property
    def n_reactions(self) -> int:
        return len(self.reactions)

    def counts(self) -> Dict[str, int]:
        out = {k: 0 for k in KINDS}
        for r in self.reactions:
            out[r.kind] += 1
        return out


# --------------------------------------------------------------------------
# mechanism file (text, one record per line; doubles written with repr so
# that strtod reads them back bit-exactly)
# --------------------------------------------------------------------------

def _f(x: float) -> str:
    return repr(float(x))


def write_mechanism(mech: Mechanism, path: str) -> None:
    ns = mech.n_species
    lines = ["KXMECH 1", f"name {mech.name}",
             f"elements {len(mech.elements)} " + " ".join(mech.elements),
             f"species {ns}"]
    for k in range(ns):
        comp = " ".join(str(int(c)) for c in mech.composition[k])
        lines.append(f"species_data {k} {mech.species[k]} {_f(mech.W[k])} {int(mech.inert[k])} {comp}")
    for k in range(ns):
        t = " ".join(_f(v) for v in mech.nasa_T[k])
        lo = " ".join(_f(v) for v in mech.nasa_lo[k])
        hi = " ".join(_f(v) for v in mech.nasa_hi[k])
        lines.append(f"nasa {k} {t} {lo} {hi}")
    if mech.transport_fit != "ln":
        lines.append(f"transport_fit {mech.transport_fit}")
    for k in range(ns):
        lines.append(f"eta {k} " + " ".join(_f(v) for v in mech.eta_fit[k]))
    for k in range(ns):
        lines.append(f"lambda {k} " + " ".join(_f(v) for v in mech.lam_fit[k]))
    for j in range(ns):
        for k in range(j, ns):
            lines.append(f"diff {j} {k} " + " ".join(_f(v) for v in mech.diff_fit[j, k]))
    lines.append(f"reactions {mech.n_reactions}")
    for i, r in enumerate(mech.reactions):
        lines.append(f"reaction {i} {r.kind} {int(r.reversible)}")
        lines.append(f"reactants {len(r.reactants)} " + " ".join(f"{k} {nu}" for k, nu in r.reactants))
        lines.append(f"products {len(r.products)} " + " ".join(f"{k} {nu}" for k, nu in r.products))
        lines.append("rate " + " ".join(_f(v) for v in r.rate))
        if r.rate_low is not None:
            lines.append("rate_low " + " ".join(_f(v) for v in r.rate_low))
        if r.uses_third_body():
            if r.collider is not None:
                lines.append(f"collider {r.collider}")
            else:
                effs = sorted(r.efficiencies.items())
                lines.append(f"third_body {_f(r.default_eff)} {len(effs)} "
                             + " ".join(f"{k} {_f(a)}" for k, a in effs))
        if r.troe is not None:
            lines.append("troe " + " ".join(_f(v) for v in r.troe))
        if r.sri is not None:
            lines.append("sri " + " ".join(_f(v) for v in r.sri))
        if r.plog is not None:
            lines.append(f"plog {len(r.plog)} " + " ".join(" ".join(_f(v) for v in e) for e in r.plog))
        lines.append("end")
    lines.append("end_mechanism")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")


def read_mechanism(path: str) -> Mechanism:
    with open(path) as fh:
        toks = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    assert toks[0] == ["KXMECH", "1"], "not a KXMECH 1 file"
    it = iter(toks[1:])
    name = next(it)[1]
    el = next(it)
    elements = el[2:2 + int(el[1])]
    ns = int(next(it)[1])
    ne = len(elements)
    species, W, inert = [None] * ns, np.zeros(ns), np.zeros(ns, bool)
    comp = np.zeros((ns, ne), int)
    nasa_T, lo, hi = np.zeros((ns, 3)), np.zeros((ns, 7)), np.zeros((ns, 7))
    eta, lam, dif = np.zeros((ns, 5)), np.zeros((ns, 5)), np.zeros((ns, ns, 5))
    reactions: List[Reaction] = []
    fit_kind = "ln"
    for t in it:
        key = t[0]
        if key == "transport_fit":
            fit_kind = t[1]
            continue
        if key == "species_data":
            k = int(t[1]); species[k] = t[2]; W[k] = float(t[3]); inert[k] = bool(int(t[4]))
            comp[k] = [int(v) for v in t[5:5 + ne]]
        elif key == "nasa":
            k = int(t[1]); v = [float(x) for x in t[2:]]
            nasa_T[k] = v[0:3]; lo[k] = v[3:10]; hi[k] = v[10:17]
        elif key == "eta":
            eta[int(t[1])] = [float(x) for x in t[2:7]]
        elif key == "lambda":
            lam[int(t[1])] = [float(x) for x in t[2:7]]
        elif key == "diff":
            j, k = int(t[1]), int(t[2]); c = [float(x) for x in t[3:8]]
            dif[j, k] = c; dif[k, j] = c
        elif key == "reactions":
            pass
        elif key == "reaction":
            reactions.append(Reaction(kind=t[2], reversible=bool(int(t[3])), reactants=[], products=[],
                                      rate=(0.0, 0.0, 0.0)))
        elif key in ("reactants", "products"):
            n = int(t[1]); lst = [(int(t[2 + 2 * m]), int(t[3 + 2 * m])) for m in range(n)]
            setattr(reactions[-1], key, lst)
        elif key == "rate":
            reactions[-1].rate = tuple(float(x) for x in t[1:4])
        elif key == "rate_low":
            reactions[-1].rate_low = tuple(float(x) for x in t[1:4])
        elif key == "third_body":
            r = reactions[-1]; r.default_eff = float(t[1]); n = int(t[2])
            r.efficiencies = {int(t[3 + 2 * m]): float(t[4 + 2 * m]) for m in range(n)}
        elif key == "collider":
            reactions[-1].collider = int(t[1])
        elif key == "troe":
            reactions[-1].troe = tuple(float(x) for x in t[1:5])
        elif key == "sri":
            reactions[-1].sri = tuple(float(x) for x in t[1:6])
        elif key == "plog":
            n = int(t[1]); v = [float(x) for x in t[2:2 + 4 * n]]
            reactions[-1].plog = [tuple(v[4 * m:4 * m + 4]) for m in range(n)]
        elif key in ("end", "end_mechanism"):
            pass
        else:
            raise ValueError(f"unknown record {key}")
    return Mechanism(name, elements, species, comp, W, inert, nasa_T, lo, hi, eta, lam, dif, reactions, transport_fit=fit_kind)


# --------------------------------------------------------------------------
# mechanism specs shaped like the paper's three workloads
# --------------------------------------------------------------------------

@dataclass
class MechSpec:
    name: str
    elements: List[str]
    ranges: Dict[str, Tuple[int, int]]
    n_species: int
    n_reactions: int
    n_three_body: int
    n_falloff: int
    inert: List[Dict[str, int]]
    seed: int
    n_chem_act: int = 0
    n_plog: int = 0
    n_sri: int = 0
    n_collider: int = 0        # three-body reactions with a single-species collider
    n_lindemann: int = 0       # falloff reactions without Troe blending


SPECS = {
    # 9 species / 21 reactions: H2/O2-like, H and O 0-2 plus inert N2
    "h2o2_9_21": MechSpec("h2o2_9_21", ["H", "O", "N"], {"H": (0, 2), "O": (0, 2), "N": (0, 0)},
                          9, 21, 4, 2, [{"N": 2}], seed=1),
    # 53 species / 325 reactions: GRI-sized, C 0-3, H 0-8, O 0-2, N 0-2, inert Ar
    "gri_53_325": MechSpec("gri_53_325", ["C", "H", "O", "N", "Ar"],
                           {"C": (0, 3), "H": (0, 8), "O": (0, 2), "N": (0, 2), "Ar": (0, 0)},
                           53, 325, 30, 29, [{"Ar": 1}], seed=2),
    # 160 species / 900 reactions, 8 % three-body, 6 % Troe falloff
    "large_160_900": MechSpec("large_160_900", ["C", "H", "O", "N", "Ar"],
                              {"C": (0, 4), "H": (0, 10), "O": (0, 3), "N": (0, 2), "Ar": (0, 0)},
                              160, 900, 72, 54, [{"Ar": 1}], seed=3),
}


# --------------------------------------------------------------------------
# drawing
# --------------------------------------------------------------------------

_STEPS = [{"H": 1}, {"H": -1}, {"H": 2}, {"O": 1}, {"C": 1}, {"C": 1, "H": 2}, {"C": 1, "H": 3},
          {"O": 1, "H": 1}, {"N": 1}, {"N": 1, "O": 1}, {"N": 1, "H": 1}, {"C": 1, "O": 1}, {"O": -1}]
_CORE = [{"H": 1}, {"H": 2}, {"O": 1}, {"O": 2}, {"O": 1, "H": 1}, {"H": 2, "O": 1}, {"H": 1, "O": 2},
         {"H": 2, "O": 2}, {"N": 2}, {"C": 1, "O": 1}, {"C": 1, "O": 2}, {"C": 1, "H": 4}, {"C": 1, "H": 3},
         {"N": 1, "O": 1}, {"N": 1}]


def _formula(elements: Sequence[str], c: Sequence[int]) -> str:
    s = "".join(f"{e}{'' if n == 1 else n}" for e, n in zip(elements, c) if n > 0)
    return s or "X"


def _draw_species(spec: MechSpec, rng: np.random.Generator) -> List[Tuple[int, ...]]:
    el = spec.elements
    lo = np.array([spec.ranges[e][0] for e in el])
    hi = np.array([spec.ranges[e][1] for e in el])
    n_reactive = spec.n_species - len(spec.inert)

    def vec(d):
        return tuple(int(d.get(e, 0)) for e in el)

    def ok(c):
        a = np.array(c)
        return a.sum() > 0 and np.all(a >= lo) and np.all(a <= hi)

    inert = [vec(d) for d in spec.inert]
    comps: List[Tuple[int, ...]] = []
    seen = set(inert)
    for d in _CORE:
        c = vec(d)
        if ok(c) and c not in seen and len(comps) < n_reactive and all(e in el for e in d):
            comps.append(c); seen.add(c)
    steps = [vec(d) for d in _STEPS if all(e in el for e in d)]
    guard = 0
    while len(comps) < n_reactive:
        guard += 1
        if guard > 200000:
            raise RuntimeError("cannot draw enough distinct species")
        base = comps[rng.integers(len(comps))]
        st = steps[rng.integers(len(steps))]
        c = tuple(b + s for b, s in zip(base, st))
        if ok(c) and c not in seen:
            comps.append(c); seen.add(c)
    return comps + inert


class _Index:
    """Multisets of reactive species (size 1-3, multiplicity <= 2) grouped by
    total elemental composition; two multisets in one group balance."""

    def __init__(self, comps: np.ndarray, reactive: np.ndarray):
        self.comps = comps
        base = int(comps.max()) * 3 + 1
        self.key1 = (comps * (base ** np.arange(comps.shape[1]))).sum(axis=1).astype(np.int64)
        self.groups: Dict[int, List[Tuple[int, ...]]] = {}
        ids = [int(i) for i in np.nonzero(reactive)[0]]
        for size in (1, 2, 3):
            for ms in combinations_with_replacement(ids, size):
                if size == 3 and ms[0] == ms[2]:
                    continue
                key = int(sum(self.key1[m] for m in ms))
                self.groups.setdefault(key, []).append(ms)

    def key(self, ms) -> int:
        return int(sum(self.key1[m] for m in ms))

    def partners(self, ms) -> List[Tuple[int, ...]]:
        s = set(ms)
        return [o for o in self.groups.get(self.key(ms), []) if not (set(o) & s)]


def _to_nu(ms: Sequence[int]) -> List[Tuple[int, int]]:
    out: Dict[int, int] = {}
    for m in ms:
        out[m] = out.get(m, 0) + 1
    return sorted(out.items())


def _arrhenius(rng) -> Tuple[float, float, float]:
    return (float(10.0 ** rng.uniform(6.0, 14.0)), float(rng.uniform(-2.0, 3.0)), float(rng.uniform(0.0, 3.0e4)))


def _nasa_fit(rng, n_atoms: int, T_lo=300.0, T_mid=1000.0, T_hi=3000.0):
    """Constrained least-squares NASA-7 blocks for cp/R = a + b tanh((T-T0)/w)."""
    a = rng.uniform(2.5, 2.5 + 1.5 * (n_atoms - 1)) if n_atoms > 1 else 2.5
    b = rng.uniform(0.0, 1.5 * n_atoms) if n_atoms > 1 else 0.0
    T0 = rng.uniform(600.0, 1800.0)
    w = rng.uniform(300.0, 1000.0)

    def cp(T):
        return a + b * np.tanh((T - T0) / w)

    target = cp(T_mid)
    P = np.polynomial.polynomial
    blocks = []
    for (t0, t1) in ((T_lo, T_mid), (T_mid, T_hi)):
        T = np.linspace(t0, t1, 64)
        V = np.vander(T, 5, increasing=True)
        # KKT system for min |V c - cp|^2 subject to [1, Tm, Tm^2, Tm^3, Tm^4] c = cp(Tm)
        cvec = np.vander([T_mid], 5, increasing=True)[0]
        K = np.zeros((6, 6))
        K[:5, :5] = 2 * V.T @ V
        K[:5, 5] = cvec
        K[5, :5] = cvec
        rhs = np.concatenate([2 * V.T @ cp(T), [target]])
        sol = np.linalg.solve(K, rhs)
        blocks.append(sol[:5])
    h_f = rng.uniform(-3.0e5, 5.0e5) * 1.0e3          # J/kmol
    s298 = rng.uniform(100.0, 250.0) * 1.0e3           # J/(kmol K)
    Tref = 298.15
    # H/R = integral of cp/R dT + a5 ;  S/R = integral of cp/(R T) dT + a6
    def h_int(c, T):
        return P.polyval(T, P.polyint(c))

    def s_int(c, T):
        return c[0] * math.log(T) + P.polyval(T, P.polyint(c[1:]))

    lo, hi = blocks
    a5_lo = h_f / R_U - h_int(lo, Tref)
    a6_lo = s298 / R_U - s_int(lo, Tref)
    a5_hi = a5_lo + h_int(lo, T_mid) - h_int(hi, T_mid)
    a6_hi = a6_lo + s_int(lo, T_mid) - s_int(hi, T_mid)
    return (np.array([T_lo, T_mid, T_hi]), np.concatenate([lo, [a5_lo, a6_lo]]),
            np.concatenate([hi, [a5_hi, a6_hi]]))


def _fit_ln(rng_curve, T):
    L = np.log(T)
    c = np.polyfit(L, rng_curve, 4)[::-1]
    return c


def _transport(rng, W: np.ndarray):
    ns = len(W)
    T = np.exp(np.linspace(math.log(300.0), math.log(3000.0), 64))
    eta = np.zeros((ns, 5)); lam = np.zeros((ns, 5)); dif = np.zeros((ns, ns, 5))
    for k in range(ns):
        e0 = rng.uniform(1e-5, 5e-5); s = rng.uniform(0.6, 0.8); c = rng.uniform(0.0, 150.0)
        eta[k] = _fit_ln(None, T) if False else np.polyfit(np.log(T), math.log(e0) + s * np.log(T / 300.0) - c / T, 4)[::-1]
        l0 = rng.uniform(0.01, 0.2); s2 = rng.uniform(0.7, 1.0); c2 = rng.uniform(0.0, 150.0)
        lam[k] = np.polyfit(np.log(T), math.log(l0) + s2 * np.log(T / 300.0) - c2 / T, 4)[::-1]
    for j in range(ns):
        for k in range(j, ns):
            d0 = rng.uniform(0.5, 2.0) * 1.5e-5 * math.sqrt(0.5 * (1.0 / W[j] + 1.0 / W[k]) * 28.0)
            cc = rng.uniform(0.0, 200.0)
            f = np.polyfit(np.log(T), math.log(d0) + 1.75 * np.log(T / 300.0) - cc / T, 4)[::-1]
            dif[j, k] = f; dif[k, j] = f
    return eta, lam, dif


def make_mechanism(spec: MechSpec) -> Mechanism:
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    comps_t = _draw_species(spec, rng)
    ns = len(comps_t)
    comps = np.array(comps_t, dtype=int)
    el = spec.elements
    W = np.array([sum(ATOMIC_MASS[e] * n for e, n in zip(el, c)) for c in comps_t])
    inert = np.zeros(ns, bool)
    inert[ns - len(spec.inert):] = True
    names = [_formula(el, c) for c in comps_t]

    nasa_T = np.zeros((ns, 3)); lo = np.zeros((ns, 7)); hi = np.zeros((ns, 7))
    for k in range(ns):
        nasa_T[k], lo[k], hi[k] = _nasa_fit(rng, int(comps[k].sum()))
    eta, lam, dif = _transport(rng, W)

    idx = _Index(comps, ~inert)
    reactive = [int(i) for i in np.nonzero(~inert)[0]]
    used_keys = set()
    reactions: List[Reaction] = []
    covered = set()

    def canon(R, P):
        a, b = tuple(sorted(R)), tuple(sorted(P))
        return (a, b) if a <= b else (b, a)

    def add(kind, R, P, swap):
        if swap:
            R, P = P, R
        key = canon(R, P)
        if key in used_keys:
            return False
        used_keys.add(key)
        r = Reaction(kind=kind, reversible=True, reactants=_to_nu(R), products=_to_nu(P), rate=_arrhenius(rng))
        reactions.append(r)
        covered.update(R); covered.update(P)
        return r

    # recombinations A + B (+M) <=> AB for three-body / falloff reactions
    recomb = []
    for p in reactive:
        pairs = [ms for ms in idx.groups.get(idx.key((p,)), []) if len(ms) == 2 and p not in ms]
        if pairs:
            recomb.append((p, pairs))
    if not recomb:
        raise RuntimeError("no recombination candidates")

    def add_special(kind):
        for _ in range(10000):
            p, pairs = recomb[rng.integers(len(recomb))]
            R = pairs[rng.integers(len(pairs))]
            r = add(kind, R, (p,), False)
            if r:
                return r
        raise RuntimeError("cannot draw recombination reaction")

    n_special = spec.n_three_body + spec.n_falloff + spec.n_chem_act
    third = []
    for m in range(spec.n_three_body):
        third.append(add_special("three_body"))
    for m in range(spec.n_falloff):
        r = add_special("falloff")
        r.rate_low = _arrhenius(rng)
        if m >= spec.n_lindemann + spec.n_sri:
            r.troe = (float(rng.uniform(0.4, 0.8)), float(rng.uniform(10.0, 1e3)),
                      float(rng.uniform(1e3, 1e4)), float(rng.uniform(1e3, 1e4)))
        elif m >= spec.n_lindemann:
            r.sri = (float(rng.uniform(0.2, 2.0)), float(rng.uniform(100.0, 1000.0)),
                     float(rng.uniform(300.0, 3000.0)), float(rng.uniform(0.5, 2.0)), float(rng.uniform(-0.5, 0.5)))
        third.append(r)
    for m in range(spec.n_chem_act):
        r = add_special("chem_act")
        r.rate_low = _arrhenius(rng)
        r.troe = (float(rng.uniform(0.4, 0.8)), float(rng.uniform(10.0, 1e3)),
                  float(rng.uniform(1e3, 1e4)), float(rng.uniform(1e3, 1e4)))
        third.append(r)
    for j, r in enumerate(third):
        if r.kind == "three_body" and j < spec.n_collider:
            r.collider = reactive[rng.integers(len(reactive))]
            continue
        nsel = int(rng.integers(1, 5))
        pool = list(range(ns))
        sel = rng.choice(pool, size=min(nsel, ns), replace=False)
        r.efficiencies = {int(k): float(rng.uniform(0.5, 12.0)) for k in sel}

    n_elem = spec.n_reactions - n_special
    # coverage: every reactive species appears at least once
    order = list(rng.permutation(reactive))
    for s in order:
        if s in covered:
            continue
        cands = []
        for o in reactive:
            for ms in (tuple(sorted((s, o))),):
                if idx.partners(ms):
                    cands.append(ms)
        for ms in ((s,), (s, s)):
            if idx.partners(ms):
                cands.append(ms)
        rng.shuffle(cands)
        done = False
        for ms in cands:
            parts = idx.partners(ms)
            P = parts[rng.integers(len(parts))]
            if add("elementary", ms, P, bool(rng.integers(2))):
                done = True
                break
        if not done:
            raise RuntimeError(f"species {names[s]} cannot be placed in a balanced reaction")
    bimol = [ms for g in idx.groups.values() for ms in g if len(ms) == 2]
    guard = 0
    n_plog_left = spec.n_plog
    while len(reactions) < n_special + n_elem:
        guard += 1
        if guard > 500000:
            raise RuntimeError("cannot draw enough elementary reactions")
        u = rng.random()
        if u < 0.9:
            R = bimol[rng.integers(len(bimol))]
        else:
            grp = list(idx.groups.values())[rng.integers(len(idx.groups))]
            R = grp[rng.integers(len(grp))]
        parts = idx.partners(R)
        if not parts:
            continue
        P = parts[rng.integers(len(parts))]
        add("elementary", R, P, bool(rng.integers(2)))
    for r in reactions:
        if n_plog_left and r.kind == "elementary":
            n_plog_left -= 1
            r.kind = "plog"
            r.plog = []
            for pa in (0.1, 1.0, 10.0, 100.0):
                A, b, E = _arrhenius(rng)
                r.plog.append((pa * P_ATM, A, b, E))
    if len(covered & set(reactive)) != len(reactive):
        raise RuntimeError("coverage failed")
    return Mechanism(spec.name, el, names, comps, W, inert, nasa_T, lo, hi, eta, lam, dif, reactions)


# --------------------------------------------------------------------------
# states
# --------------------------------------------------------------------------

@dataclass
class StateSpec:
    T_range: Tuple[float, float]
    p_atm_range: Tuple[float, float]    # equal ends -> constant pressure
    alpha: float                        # Dirichlet concentration
    seed: int


STATE_SPECS = {
    "h2o2_9_21": StateSpec((300.0, 2500.0), (1.0, 1.0), 0.5, 101),
    "gri_53_325": StateSpec((300.0, 2800.0), (0.5, 40.0), 0.2, 102),
    "large_160_900": StateSpec((500.0, 2800.0), (1.0, 60.0), 0.2, 103),
}

CHUNK = 1 << 16


for _n in list(STATE_SPECS):
    STATE_SPECS[_n + "_direct"] = STATE_SPECS[_n]
    STATE_SPECS[_n + "_special"] = STATE_SPECS[_n]


def make_states(ns: int, spec: StateSpec, start: int, count: int, dtype=np.float64):
    """States ``start .. start+count-1`` of the seeded stream: SoA arrays
    T[count], p[count], Y[ns, count].  Point i is drawn in chunk i // 2^16
    from SeedSequence([seed, chunk]), so any range is reproducible alone."""
    T = np.empty(count, dtype); p = np.empty(count, dtype); Y = np.empty((ns, count), dtype)
    pos = 0
    i = start
    while pos < count:
        c = i // CHUNK
        off = i - c * CHUNK
        take = min(CHUNK - off, count - pos)
        rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([spec.seed, c])))
        Tc = rng.uniform(spec.T_range[0], spec.T_range[1], CHUNK)
        a0, a1 = spec.p_atm_range
        if a0 == a1:
            pc = np.full(CHUNK, a0 * P_ATM)
        else:
            pc = P_ATM * np.exp(rng.uniform(math.log(a0), math.log(a1), CHUNK))
        G = rng.gamma(spec.alpha, 1.0, size=(CHUNK, ns))
        G /= G.sum(axis=1, keepdims=True)
        T[pos:pos + take] = Tc[off:off + take]
        p[pos:pos + take] = pc[off:off + take]
        Y[:, pos:pos + take] = G[off:off + take].T
        pos += take
        i += take
    return T, p, Y


_CACHE: Dict[str, Mechanism] = {}


def direct_fits(mech: Mechanism) -> Mechanism:
    """The same mechanism with its transport given by direct polynomial fits in
    ln T of eta_k, lambda_k and 1/D_jk (least squares on 64 log-spaced points of
    300-3000 K of the curves its ln fits describe); name suffixed "_direct"."""
    import dataclasses
    L = np.linspace(math.log(300.0), math.log(3000.0), 64)

    def refit(c, sign):
        return np.polyfit(L, np.exp(sign * np.polyval(c[::-1], L)), 4)[::-1]

    ns = mech.n_species
    eta = np.array([refit(mech.eta_fit[k], 1.0) for k in range(ns)])
    lam = np.array([refit(mech.lam_fit[k], 1.0) for k in range(ns)])
    dif = np.zeros_like(mech.diff_fit)
    for j in range(ns):
        for k in range(j, ns):
            dif[j, k] = dif[k, j] = refit(mech.diff_fit[j, k], -1.0)
    return dataclasses.replace(mech, name=mech.name + "_direct", eta_fit=eta, lam_fit=lam, diff_fit=dif,
                               transport_fit="direct")


def special_rates(mech: Mechanism, seed: int = 7) -> Mechanism:
    """The same mechanism with the special-case mix of Arrhenius parameters that
    the paper counts for its ethanol mechanism (Sec. 2.3.1): about 27 % of the
    rate constants with beta = E = 0 (k = A), 0.6 % with E = 0 and a small integer
    beta (k = A T^beta), and 21 % sharing (beta, E) with another rate constant;
    A is kept.  Drawn from its own seeded stream; name suffixed "_special"."""
    import dataclasses
    rng = np.random.Generator(np.random.PCG64([seed, 2411]))
    rx = [dataclasses.replace(r) for r in mech.reactions]
    slots = [(i, "rate") for i in range(len(rx))] + [(i, "rate_low") for i, r in enumerate(rx) if r.rate_low is not None]
    order = rng.permutation(len(slots))
    n_const, n_int, n_share = round(0.27 * len(slots)), max(1, round(0.006 * len(slots))), round(0.21 * len(slots))
    general = [slots[j] for j in order[n_const + n_int + n_share:]]
    for j in order[:n_const]:
        i, f = slots[j]
        setattr(rx[i], f, (getattr(rx[i], f)[0], 0.0, 0.0))
    for j in order[n_const:n_const + n_int]:
        i, f = slots[j]
        setattr(rx[i], f, (getattr(rx[i], f)[0], float(rng.choice([-1.0, 1.0, 2.0])), 0.0))
    for j in order[n_const + n_int:n_const + n_int + n_share]:
        i, f = slots[j]
        src_i, src_f = general[int(rng.integers(len(general)))]
        a = getattr(rx[src_i], src_f)
        setattr(rx[i], f, (getattr(rx[i], f)[0], a[1], a[2]))
    return dataclasses.replace(mech, name=mech.name + "_special", reactions=rx)


def mechanism(name: str) -> Mechanism:
    """A synthetic mechanism by name; "<name>_direct" is <name> with direct
    transport fits, "<name>_special" with the paper's special-case Arrhenius mix."""
    if name not in _CACHE:
        if name.endswith("_direct"):
            _CACHE[name] = direct_fits(mechanism(name[: -len("_direct")]))
        elif name.endswith("_special"):
            _CACHE[name] = special_rates(mechanism(name[: -len("_special")]))
        else:
            _CACHE[name] = make_mechanism(SPECS[name])
    return _CACHE[name]


def mechanism_file(name: str, directory: str) -> str:
    """Write (once) the named synthetic mechanism into ``directory``."""
    import os
    os.makedirs(directory, exist_ok=True)
    path = os.path.join(directory, f"{name}.kxmech")
    if not os.path.exists(path):
        tmp = path + f".{os.getpid()}.tmp"
        write_mechanism(mechanism(name), tmp)
        os.replace(tmp, path)
    return path


def make_states_torch(ns: int, spec: StateSpec, count: int, seed: int, device="cuda"):
    """A large batch of states drawn directly in device memory with torch's
    seeded generator (same distributions as make_states; a different
    stream of numbers).  For full-size runs whose states the CPU could not
    draw in reasonable time; a sample of them can be copied back for the
    oracle."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    T = torch.empty(count, dtype=torch.float64, device=device).uniform_(spec.T_range[0], spec.T_range[1], generator=g)
    a0, a1 = spec.p_atm_range
    if a0 == a1:
        p = torch.full((count,), a0 * P_ATM, dtype=torch.float64, device=device)
    else:
        u = torch.empty(count, dtype=torch.float64, device=device).uniform_(math.log(a0), math.log(a1), generator=g)
        p = P_ATM * torch.exp(u)
    Y = torch.empty((ns, count), dtype=torch.float64, device=device)
    chunk = 1 << 20
    for s0 in range(0, count, chunk):
        c = min(chunk, count - s0)
        alpha = torch.full((ns, c), spec.alpha, dtype=torch.float64, device=device)
        G = torch._standard_gamma(alpha, generator=g)
        Y[:, s0:s0 + c] = G / G.sum(dim=0, keepdim=True)
    return T, p, Y
