"""Hand-built toy mechanisms for the closed-form pins.

Species have constant heat capacity (only a0, a5, a6 of the NASA-7 blocks
are non-zero, the same in both temperature ranges), so that
cp/R = a0, H/(RT) = a0 + a5/T and S/R = a0 ln T + a6 can be worked by hand,
and power-law transport fits ln eta = ln eta0 + s ln T.
"""
from __future__ import annotations

import math
import os
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from paper_2411_02640_gb300.synth import ATOMIC_MASS, Mechanism, Reaction, write_mechanism


def species_block(specs: Sequence[Tuple[str, Dict[str, int], float, float, float]], elements: List[str],
                  eta0: Optional[Sequence[float]] = None, lam0: Optional[Sequence[float]] = None,
                  s_eta: float = 0.7, s_lam: float = 0.8, d0: float = 2e-5, W: Optional[Sequence[float]] = None):
    ns = len(specs)
    comp = np.array([[d.get(e, 0) for e in elements] for _, d, *_ in specs], int)
    if W is None:
        W = np.array([sum(ATOMIC_MASS[e] * n for e, n in d.items()) for _, d, *_ in specs])
    W = np.asarray(W, float)
    nasa_T = np.tile([300.0, 1000.0, 3000.0], (ns, 1))
    lo = np.zeros((ns, 7))
    for k, (_, _, a0, a5, a6) in enumerate(specs):
        lo[k, 0], lo[k, 5], lo[k, 6] = a0, a5, a6
    eta0 = eta0 if eta0 is not None else [1e-5 * (1 + 0.3 * k) for k in range(ns)]
    lam0 = lam0 if lam0 is not None else [0.02 * (1 + 0.2 * k) for k in range(ns)]
    eta = np.array([[math.log(e), s_eta, 0, 0, 0] for e in eta0], float)
    lam = np.array([[math.log(l), s_lam, 0, 0, 0] for l in lam0], float)
    dif = np.zeros((ns, ns, 5))
    for j in range(ns):
        for k in range(ns):
            dif[j, k] = [math.log(d0 * (1 + 0.1 * (j + k))), 1.75, 0, 0, 0]
    names = [n for n, *_ in specs]
    return dict(elements=elements, species=names, composition=comp, W=W, inert=np.zeros(ns, bool),
                nasa_T=nasa_T, nasa_lo=lo, nasa_hi=lo.copy(), eta_fit=eta, lam_fit=lam, diff_fit=dif)


def toy(name: str, reactions: List[Reaction], directory: str, **kw) -> Tuple[Mechanism, str]:
    specs = kw.pop("specs", None) or [
        ("H", {"H": 1}, 2.5, 2.5e4, -0.5),
        ("O", {"O": 1}, 2.5, 3.0e4, 2.0),
        ("HO", {"H": 1, "O": 1}, 3.5, 4.0e3, 1.5),
        ("N2", {"N": 2}, 3.5, -1.0e3, 4.0),
    ]
    blk = species_block(specs, ["H", "O", "N"], **kw)
    mech = Mechanism(name=name, reactions=reactions, **blk)
    path = os.path.join(directory, name + ".kxmech")
    write_mechanism(mech, path)
    return mech, path


def recomb(kind: str, **kw) -> Reaction:
    """H + O (+M) <=> HO."""
    return Reaction(kind=kind, reversible=True, reactants=[(0, 1), (1, 1)], products=[(2, 1)],
                    rate=kw.pop("rate", (1.0e10, 0.5, 1000.0)), **kw)
