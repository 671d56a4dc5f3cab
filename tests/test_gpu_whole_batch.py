"""Whole-batch checks of the float64-accurate production rates.

The default KX_FP64 kernel computes in double-float (float32 pairs, float32
exponent range) and accumulates wdot under a per-state power-of-two scale;
the native float64 kernel (rates_arith = 1) is the plain float64 form of the
same method.  Here the two are compared on the device for EVERY state of
the benchmark's 2^20-state 53/325 batch and of a 2^22-state 160/900 batch
(per state: max_k W_k |dwdot_k| / max_k W_k |wdot_k| <= 1e-10), and the
native kernel is itself held to the oracle on both mechanisms, element by
element, at sizes that span many blocks and end in a ragged tail.  Each
comparison prints its max and p99 ("whole_batch: {...}")."""
import json

import numpy as np
import pytest

from paper_2411_02640_gb300 import synth
from tests.gpu_common import mechanism, oracle, to_device, torch_cuda, wdot_error

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _per_state_error(torch, W, w, ref):
    Wt = torch.tensor(W, dtype=torch.float64, device="cuda")[:, None]
    num = (Wt * (w - ref).abs()).amax(dim=0)
    den = (Wt * ref.abs()).amax(dim=0)
    return (num / torch.where(den > 0, den, torch.ones_like(den))).cpu().numpy()


@pytest.mark.parametrize("name,n", [("gri_53_325", 1 << 20), ("large_160_900", 1 << 22)])
def test_default_kernel_against_native_float64_every_state(name, n):
    torch = torch_cuda()
    if name == "gri_53_325":
        import bench
        T, p, Y = (torch.from_numpy(a).cuda() for a in bench.make_inputs(0, n))
    else:
        spec = synth.STATE_SPECS[name]
        T, p, Y = synth.make_states_torch(synth.mechanism(name).n_species, spec, n, seed=spec.seed)
    df = mechanism(name)
    nat = mechanism(name, rates_arith=1)
    W = np.array(df.W)
    w_df = df.production_rates(T, p, Y, precision="fp64")
    w_nat = nat.production_rates(T, p, Y, precision="fp64")
    assert bool(torch.isfinite(w_df).all()) and bool(torch.isfinite(w_nat).all())
    e = _per_state_error(torch, W, w_df, w_nat)
    stats = {"mechanism": name, "states": n, "max": float(e.max()), "p99": float(np.quantile(e, 0.99)),
             "median": float(np.median(e))}
    print("\nwhole_batch: " + json.dumps(stats))
    assert e.shape[0] == n
    assert e.max() <= TOL, stats


@pytest.mark.parametrize("name,n", [("gri_53_325", 1289), ("large_160_900", 777)])
def test_native_float64_rates_against_oracle(name, n):
    """Native float64 production rates and rates of progress against the
    oracle: wdot per state within 1e-10 of max_k |W_k wdot_k|, each rate of
    progress within 1e-10 of its gross scale |c_i| max(|R_f|, |R_r|)."""
    torch = torch_cuda()
    m = synth.mechanism(name)
    T, p, Y = synth.make_states(m.n_species, synth.STATE_SPECS[name], 7, n)
    mech = mechanism(name, rates_arith=1)
    Td, pd, Yd = to_device(torch, T, p, Y, ld=n + 31)
    w = mech.production_rates(Td, pd, Yd, precision="fp64")[:, :n].cpu().numpy()
    q = mech.rates_of_progress(Td, pd, Yd, precision="fp64")[:, :n].cpu().numpy()
    o = oracle(name)
    err = wdot_error(np.array(mech.W), w, o.production_rates(T, p, Y))
    gross = o.reaction_gross(T, p, Y)
    assert np.all(gross > 0)
    rel = np.abs(q - o.rates_of_progress(T, p, Y)) / gross
    print("\nwhole_batch: " + json.dumps({"mechanism": name, "native_vs_oracle_wdot_max": float(err.max()),
                                          "native_vs_oracle_rop_max": float(rel.max())}))
    assert np.all(np.isfinite(w)) and np.all(np.isfinite(q))
    assert err.max() <= TOL
    assert rel.max() <= TOL
