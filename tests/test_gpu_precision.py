"""Precision study on the 160-species / 900-reaction synthetic mechanism:
float32-bulk (mixed) production rates against the float64 GPU path over a
full 2^22-state batch, and both against the float64 oracle on a sample that
includes near-equilibrium states (the reverse rate of one of the fastest
reactions within 1 % of its forward rate).  Prints one JSON line of
statistics ("precision_study: {...}")."""
import json
import os

import numpy as np
import pytest

from paper_2411_02640_gb300 import synth
from tests.gpu_common import MECHDIR, mechanism, oracle, to_device, torch_cuda, wdot_error

pytestmark = pytest.mark.gpu

NAME = "large_160_900"
FULL = 1 << 22
SAMPLE = 1 << 13
NEAR = 1024


def test_precision_study():
    torch = torch_cuda()
    mech = mechanism(NAME)
    m = synth.mechanism(NAME)
    W = np.array(mech.W)
    spec = synth.STATE_SPECS[NAME]
    stats = {"mechanism": NAME, "full_states": FULL}
    # ---- full batch: mixed against float64 on the GPU
    T, p, Y = synth.make_states_torch(m.n_species, spec, FULL, seed=spec.seed)
    w64 = mech.production_rates(T, p, Y, precision="fp64")
    w32 = mech.production_rates(T, p, Y, precision="mixed")
    Wt = torch.tensor(W, device="cuda")[:, None]
    num = (Wt * (w32 - w64).abs()).amax(dim=0)
    den = (Wt * w64.abs()).amax(dim=0)
    e = (num / den).cpu().numpy()
    assert np.all(np.isfinite(e))
    stats["mixed_vs_fp64_gpu"] = {"max": float(e.max()), "p99": float(np.quantile(e, 0.99)),
                                  "median": float(np.median(e))}
    # ---- sample of the batch plus near-equilibrium states, against the oracle
    idx = np.linspace(0, FULL - 1, SAMPLE).astype(np.int64)
    Ts, ps, Ys = T[idx].cpu().numpy(), p[idx].cpu().numpy(), Y[:, idx].cpu().numpy()
    del T, p, Y, w64, w32
    from oracle.near_equilibrium import near_equilibrium
    path = synth.mechanism_file(NAME, MECHDIR)
    Yn, ok = near_equilibrium(path, m.reactions, Ts[:NEAR], ps[:NEAR], Ys[:, :NEAR], seed=7,
                              threads=min(16, os.cpu_count() or 1))
    Tn, pn, Yn = Ts[:NEAR][ok], ps[:NEAR][ok], Yn[:, ok]
    stats["near_equilibrium_states"] = int(ok.sum())
    o = oracle(NAME)
    for label, (Ta, pa, Ya) in {"sample": (Ts, ps, Ys), "near_equilibrium": (Tn, pn, Yn)}.items():
        Td, pd, Yd = to_device(torch, Ta, pa, Ya)
        ref = o.production_rates(Ta, pa, Ya)
        e64 = wdot_error(W, mech.production_rates(Td, pd, Yd, precision="fp64").cpu().numpy(), ref)
        e32 = wdot_error(W, mech.production_rates(Td, pd, Yd, precision="mixed").cpu().numpy(), ref)
        qref = o.rates_of_progress(Ta, pa, Ya)
        gross = o.reaction_gross(Ta, pa, Ya)
        q64 = mech.rates_of_progress(Td, pd, Yd, precision="fp64").cpu().numpy()
        q32 = mech.rates_of_progress(Td, pd, Yd, precision="mixed").cpu().numpy()
        r64 = np.abs(q64 - qref) / gross
        r32 = np.abs(q32 - qref) / gross
        stats[label] = {"states": int(Ta.shape[0]),
                        "fp64_wdot": {"max": float(e64.max()), "p99": float(np.quantile(e64, 0.99))},
                        "mixed_wdot": {"max": float(e32.max()), "p99": float(np.quantile(e32, 0.99))},
                        "fp64_rop_vs_gross": {"max": float(r64.max())},
                        "mixed_rop_vs_gross": {"max": float(r32.max()), "p99": float(np.quantile(r32, 0.99))}}
        assert e64.max() <= 1e-10 and r64.max() <= 1e-10
        assert e32.max() <= 2e-4 and np.quantile(e32, 0.99) <= 1e-4 and r32.max() <= 2e-4
        if label == "near_equilibrium":
            # the nudged reaction of each state: error relative to its own (small) net rate
            rel = []
            for c in range(Ta.shape[0]):
                net = np.abs(qref[:, c])
                near = np.nonzero(net < 0.02 * gross[:, c])[0]
                near = near[np.argsort(-gross[near, c])][:1]
                for i in near:
                    rel.append(abs(q32[i, c] - qref[i, c]) / net[i])
            rel = np.array(rel)
            stats["near_equilibrium"]["mixed_rop_vs_net"] = {"reactions": int(rel.size), "max": float(rel.max()),
                                                             "p99": float(np.quantile(rel, 0.99))}
            assert rel.max() <= 5e-3
    print("\nprecision_study: " + json.dumps(stats))
