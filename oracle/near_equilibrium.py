"""Near-equilibrium states for the precision study, built with the oracle.

TEST INFRASTRUCTURE ONLY.  For a state, take one of the fastest reactions
(forward rate k_f prod C^nu' within 1e-3 of the largest; the one whose
reverse-to-forward ratio is already closest to 1) and rescale the mass
fraction of one of its
products (bisection on ln Y, Y renormalised) until the reverse-to-forward
ratio R_r/R_f of that reaction equals a target 1 + u, |u| <= 0.01.  Only the
oracle evaluates the rates, so the states depend on nothing in the GPU path.
"""
from __future__ import annotations

import concurrent.futures as cf
from typing import Optional

import numpy as np

from . import Oracle


def _ratio(o: Oracle, T: float, p: float, Y: np.ndarray, i: int) -> float:
    d = o.reaction_detail(T, p, Y)
    return d["Rr"][i] / d["Rf"][i]


def nudge(o: Oracle, reactions, T: float, p: float, Y: np.ndarray, target: float, iters: int = 80) -> Optional[np.ndarray]:
    """Return Y' with R_r/R_f of the dominant forward reaction at `target`
    (relative 1e-12), or None if no product species moves it there."""
    d = o.reaction_detail(T, p, Y)
    # among the fastest reactions (forward rate within 1e-3 of the largest),
    # the one already closest to equilibrium, so that the nudge stays small
    Rf = np.abs(d["Rf"])
    with np.errstate(divide="ignore", invalid="ignore"):
        lr = np.abs(np.log(np.abs(d["Rr"]) / Rf))
    cand = np.nonzero((Rf >= 1e-3 * Rf.max()) & np.isfinite(lr))[0]
    if cand.size == 0:
        return None
    i = int(cand[np.argmin(lr[cand])])
    prods = [k for k, _ in reactions[i].products]
    reacs = {k for k, _ in reactions[i].reactants}
    for s in prods:
        if s in reacs:
            continue

        def with_y(ly):
            Z = Y.copy()
            Z[s] = np.exp(ly)
            return Z / Z.sum()

        lo, hi = np.log(max(Y[s], 1e-300)) - 80.0, np.log(max(Y[s], 1e-300)) + 80.0
        hi = min(hi, np.log(1e3))
        f_lo = _ratio(o, T, p, with_y(lo), i) - target
        f_hi = _ratio(o, T, p, with_y(hi), i) - target
        if not (np.isfinite(f_lo) and np.isfinite(f_hi)) or f_lo * f_hi > 0:
            continue
        for _ in range(iters):
            mid = 0.5 * (lo + hi)
            f = _ratio(o, T, p, with_y(mid), i) - target
            if f == 0 or abs(f) < 1e-12 * target:
                lo = hi = mid
                break
            if (f < 0) == (f_lo < 0):
                lo, f_lo = mid, f
            else:
                hi = mid
        return with_y(0.5 * (lo + hi))
    return None


def near_equilibrium(path: str, reactions, T, p, Y, seed: int = 0, threads: int = 16):
    """Apply `nudge` to every state (columns of Y); states that cannot be
    moved are returned unchanged and flagged False."""
    rng = np.random.default_rng(seed)
    targets = 1.0 + rng.uniform(-0.01, 0.01, T.shape[0])
    out = Y.copy()
    ok = np.zeros(T.shape[0], bool)
    oracles = [Oracle(path) for _ in range(threads)]

    def work(j):
        o = oracles[j % threads]
        for c in range(j, T.shape[0], threads):
            y = nudge(o, reactions, float(T[c]), float(p[c]), np.ascontiguousarray(Y[:, c]), targets[c])
            if y is not None:
                out[:, c] = y
                ok[c] = True

    with cf.ThreadPoolExecutor(threads) as ex:
        list(ex.map(work, range(threads)))
    return out, ok
