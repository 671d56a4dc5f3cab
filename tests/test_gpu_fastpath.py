"""The float-pair rate kernel's float32 path: a reaction whose rate is below
2^-40 of its state's scale anchor, for every state of a warp, is evaluated in
float32.  A state's results therefore depend, within the float64 bar, on the
states that share its warp: the same states under other warp groupings
(the batch shifted by 1, 13 and 31 states) must agree to 1e-10 of the
per-point scale, and each grouping must meet that bar against the oracle on
a sample.  Cold batches (where nearly every reaction takes the float32 path),
hot batches (where few do) and mixed warps are all covered."""
import numpy as np
import pytest

from paper_2411_02640_gb300 import synth
from tests.gpu_common import mechanism, oracle, to_device, torch_cuda, wdot_error

pytestmark = pytest.mark.gpu

TOL = 1e-10
NAME = "gri_53_325"


def _states(n, seed, T_range=None):
    m = synth.mechanism(NAME)
    T, p, Y = synth.make_states(m.n_species, synth.STATE_SPECS[NAME], seed, n)
    if T_range is not None:
        T = np.random.default_rng(seed).uniform(T_range[0], T_range[1], n)
    return T, p, Y


@pytest.mark.parametrize("kind,T_range", [("mixed", None), ("cold", (300.0, 700.0)), ("hot", (2200.0, 2800.0))])
def test_warp_groupings_agree_within_the_bar(kind, T_range):
    torch = torch_cuda()
    mech = mechanism(NAME, rates_layout=1)      # one thread per state: the kernel with the float32 path
    W = np.array(mech.W)
    n = 4096
    T, p, Y = _states(n, 31 if kind == "mixed" else 57, T_range)
    Td, pd, Yd = to_device(torch, T, p, Y)
    w0 = mech.production_rates(Td, pd, Yd).cpu().numpy()
    Te, pe, Ye = _states(64, 999)               # other states that shift the warp groupings
    differ = 0
    for shift in (1, 13, 31):
        Ts = np.concatenate([Te[:shift], T]); ps = np.concatenate([pe[:shift], p])
        Ys = np.concatenate([Ye[:, :shift], Y], axis=1)
        ws = mech.production_rates(*to_device(torch, Ts, ps, Ys)).cpu().numpy()[:, shift:]
        err = wdot_error(W, ws, w0)
        assert err.max() <= TOL, (shift, err.max())
        differ += int(np.any(ws != w0, axis=0).sum())
    print(f"\nwarp_groupings[{kind}]: states whose bits changed with the grouping: {differ} of {3 * n}")
    # each grouping against the oracle on a sample of states
    idx = np.linspace(0, n - 1, 256).astype(int)
    ref = oracle(NAME).production_rates(T[idx], p[idx], np.ascontiguousarray(Y[:, idx]))
    assert wdot_error(W, w0[:, idx], ref).max() <= TOL


def test_cold_and_hot_states_in_one_warp():
    """Warps whose 32 states alternate between cold and hot: the hot states'
    large rates keep most reactions off the float32 path for the whole warp;
    both kinds of state against the oracle."""
    torch = torch_cuda()
    mech = mechanism(NAME, rates_layout=1)
    W = np.array(mech.W)
    n = 2048
    T, p, Y = _states(n, 77)
    T = np.where(np.arange(n) % 2 == 0, np.random.default_rng(1).uniform(300.0, 600.0, n),
                 np.random.default_rng(2).uniform(2000.0, 2800.0, n))
    w = mech.production_rates(*to_device(torch, T, p, Y)).cpu().numpy()
    idx = np.arange(0, n, 7)
    ref = oracle(NAME).production_rates(T[idx], p[idx], np.ascontiguousarray(Y[:, idx]))
    err = wdot_error(W, w[:, idx], ref)
    assert np.all(np.isfinite(w)) and err.max() <= TOL, err.max()


@pytest.mark.parametrize("negl,bar", [(0, 1e-3), (1, 1e-9)])
def test_per_species_accuracy(negl, bar):
    """Each species against the oracle relative to its own gross rate
    sum_i |nu_ki| max(|R_f,i|, |R_r,i|): every reaction in float pairs
    (rates_negligible 1) keeps ~1e-11 for every species within 1e-40 of the
    state's largest rate; the default path keeps a species that
    only negligible reactions touch to ~1e-4 of itself (float32), while the
    per-point bar (1e-10 of max_k W_k |wdot_k|) holds for both."""
    torch = torch_cuda()
    mech = mechanism(NAME, rates_layout=1, rates_negligible=negl)
    W = np.array(mech.W)
    m = synth.mechanism(NAME)
    n = 1024
    T, p, Y = _states(n, 404)
    w = mech.production_rates(*to_device(torch, T, p, Y)).cpu().numpy()
    o = oracle(NAME)
    ref = o.production_rates(T, p, Y)
    gross = o.reaction_gross(T, p, Y)                      # [nr, n]
    nu = np.zeros((m.n_species, len(m.reactions)))
    for i, r in enumerate(m.reactions):
        for k, c in r.reactants:
            nu[k, i] += c
        for k, c in r.products:
            nu[k, i] += c
    gk = nu @ gross                                        # [ns, n]
    # species within 1e-40 of their state's largest rate (cold states of this mechanism reach rates of
    # 1e190 and more); the running scale's rescales apply their power of two in two exact steps, so
    # sums accumulated before a jump of more than 2^126 keep their value
    mask = gk > 1e-40 * gross.max(axis=0)[None, :]
    rel = np.abs(w - ref)[mask] / gk[mask]
    assert rel.max() <= bar, rel.max()
    assert wdot_error(W, w, ref).max() <= TOL
    print(f"\nper_species[rates_negligible={negl}]: max {rel.max():.2e}, p99 {np.quantile(rel, 0.99):.2e}")
