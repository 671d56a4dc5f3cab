"""Every reaction form the file format carries -- three-body with
efficiencies and with a single collider species, Lindemann, Troe and SRI
falloff, chemically activated falloff, PLOG, irreversible, a coefficient of 3 -- through the
GPU kernels against the oracle (rates of progress, production rates, the
adjoint)."""
import numpy as np
import pytest

from paper_2411_02640_gb300.synth import P_ATM, Reaction
from tests import toys
from tests.gpu_common import CACHE, to_device, torch_cuda, wdot_error

pytestmark = pytest.mark.gpu


def reactions():
    """One reaction of every kind the kernels support (also used by the CPU test of the
    warp-cooperative gather tables)."""
    return [toys.recomb("elementary"), toys.recomb("three_body", efficiencies={3: 2.0, 0: 0.7}),
          toys.recomb("three_body", collider=3, rate=(3e9, -0.5, 200.0)),
          toys.recomb("falloff", rate=(1e9, 0.3, 400.0), rate_low=(1e12, 0.1, 100.0)),
          toys.recomb("falloff", rate=(5e8, 0.0, 800.0), rate_low=(1e13, -1.1, 100.0), troe=(0.5, 100.0, 2000.0, 3000.0),
                      efficiencies={2: 3.0}),
          toys.recomb("falloff", rate=(2e9, 0.2, 300.0), rate_low=(4e12, 0.1, 500.0), sri=(0.5, 200.0, 1000.0, 1.2, 0.1)),
          toys.recomb("chem_act", rate=(1e9, 0.0, 0.0), rate_low=(1e12, 0.1, 100.0), troe=(0.6, 300.0, 2500.0, 4000.0)),
          Reaction(kind="plog", reversible=True, reactants=[(0, 1), (1, 1)], products=[(2, 1)], rate=(0, 0, 0),
                   plog=[(0.1 * P_ATM, 1e9, 0.2, 300.0), (1.0 * P_ATM, 3e9, 0.0, 500.0), (10 * P_ATM, 1e11, -0.3, 900.0)]),
          Reaction(kind="elementary", reversible=False, reactants=[(2, 1)], products=[(0, 1), (1, 1)],
                   rate=(1e13, 0.0, 2e4)),
          # net coefficients of 3 (the float-pair product path of the accumulation, not the exact scaling)
          Reaction(kind="elementary", reversible=True, reactants=[(2, 3)], products=[(0, 3), (1, 3)],
                   rate=(1e8, 0.5, 1000.0))]


def _mechanism(tmp_path_factory):
    d = str(tmp_path_factory.mktemp("kinds"))
    _, path = toys.toy("kinds", reactions(), d)
    return path


@pytest.fixture(scope="module")
def kinds(tmp_path_factory):
    import oracle as ora
    from paper_2411_02640_gb300 import kx
    torch_cuda()
    path = _mechanism(tmp_path_factory)
    return kx.Mechanism(path, cache_dir=CACHE), ora.Oracle(path)


def _states(n, seed=3):
    rng = np.random.default_rng(seed)
    T = rng.uniform(300.0, 2800.0, n)
    p = P_ATM * np.exp(rng.uniform(np.log(0.02), np.log(200.0), n))     # spans every PLOG interval
    Y = rng.gamma(0.5, 1.0, (4, n))
    Y /= Y.sum(axis=0)
    return T, p, Y


def test_rates_of_progress_all_kinds(kinds):
    import torch
    mech, o = kinds
    T, p, Y = _states(2000)
    Td, pd, Yd = to_device(torch, T, p, Y)
    q = mech.rates_of_progress(Td, pd, Yd).cpu().numpy()
    ref = o.rates_of_progress(T, p, Y)
    gross = o.reaction_gross(T, p, Y)
    rel = np.abs(q - ref) / gross
    assert rel.max() <= 1e-10, (rel.max(), np.unravel_index(rel.argmax(), rel.shape))
    w = mech.production_rates(Td, pd, Yd).cpu().numpy()
    assert wdot_error(np.array(mech.W), w, o.production_rates(T, p, Y)).max() <= 1e-10
    qm = mech.rates_of_progress(Td, pd, Yd, precision="mixed").cpu().numpy()
    assert (np.abs(qm - ref) / gross).max() <= 2e-4


@pytest.mark.parametrize("opts", [{"vjp_layout": 1}, {"rates_arith": 1}, {"vjp_layout": 2}])
def test_adjoint_all_kinds(kinds, opts, tmp_path_factory):
    """Every reaction kind: the double-float adjoint (thread per state and warp-cooperative) and
    native float64."""
    import torch
    from paper_2411_02640_gb300 import kx
    mech, o = kinds
    if opts:
        mech = kx.Mechanism(mech.path, cache_dir=CACHE, lazy=1, **opts)
    T, p, Y = _states(200, seed=9)
    v = np.random.default_rng(1).standard_normal((4, 200))
    Td, pd, Yd = to_device(torch, T, p, Y)
    gT, gY = (t.cpu().numpy() for t in mech.production_rates_vjp(Td, pd, Yd, torch.tensor(v, device="cuda")))
    for i in range(200):
        J = o.jacobian(T[i], p[i], Y[:, i])
        ref = v[:, i] @ J
        scale = np.abs(v[:, i]) @ np.abs(J)
        got = np.concatenate([[gT[i]], gY[:, i]])
        assert np.all(np.abs(got - ref) <= 1e-9 * scale.max()), (i, got, ref)
