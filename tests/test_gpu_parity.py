"""GPU kernels against the FP64 oracle, element by element, through the C ABI.

Bars (float64 path): production rates within 1e-10 of the per-point scale
max_k |W_k wdot_k|; every rate of progress within 1e-10 of its own gross
scale |c_i| max(|R_f,i|, |R_r,i|); thermo and transport within 1e-12
relative (h against the size of its terms, since h changes sign).  The
mixed path is held to the error bounds it is documented with.
Sizes span many blocks and end in a ragged tail (n not a multiple of the
block, ld > n).
"""
import math

import numpy as np
import pytest

from paper_2411_02640_gb300 import synth
from tests.gpu_common import mechanism, oracle, to_device, torch_cuda, wdot_error

pytestmark = pytest.mark.gpu

N_SMALL = 4133          # 32 blocks of 128 plus a ragged 37
LD_PAD = 59
CASES = {"h2o2_9_21": N_SMALL, "gri_53_325": 1289}


def _states(name, n, start=0):
    m = synth.mechanism(name)
    return synth.make_states(m.n_species, synth.STATE_SPECS[name], start, n)


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.mark.parametrize("name", list(CASES))
def test_production_rates_fp64(torch, name):
    n = CASES[name]
    T, p, Y = _states(name, n)
    mech = mechanism(name)
    Td, pd, Yd = to_device(torch, T, p, Y, ld=n + LD_PAD)
    w = mech.production_rates(Td, pd, Yd)[:, :n].cpu().numpy()
    w_ref = oracle(name).production_rates(T, p, Y)
    err = wdot_error(np.array(mech.W), w, w_ref)
    assert np.all(np.isfinite(w))
    assert err.max() <= 1e-10, f"max {err.max():.3e}"


@pytest.mark.parametrize("name,arith", [("h2o2_9_21", 0), ("gri_53_325", 0), ("h2o2_9_21", 1)])
def test_negative_mass_fractions_fp64(torch, name, arith):
    """Small negative mass fractions (undershoots of a transport step) are
    evaluated with signed concentrations, as in the oracle: the float-pair
    kernel carries the sign of each concentration product beside its log
    magnitude; the native float64 kernel (arith=1) multiplies linearly."""
    n = CASES[name]
    T, p, Y = _states(name, n, start=301)
    rng = np.random.default_rng(17)
    neg = rng.random(Y.shape) < 0.1
    Y[neg] = -1e-4 * rng.random(int(neg.sum()))
    mech = mechanism(name, **({"rates_arith": arith} if arith else {}))
    Td, pd, Yd = to_device(torch, T, p, Y, ld=n + LD_PAD)
    w = mech.production_rates(Td, pd, Yd)[:, :n].cpu().numpy()
    o = oracle(name)
    err = wdot_error(np.array(mech.W), w, o.production_rates(T, p, Y))
    assert err.max() <= 1e-10, f"max {err.max():.3e}"
    q = mech.rates_of_progress(Td, pd, Yd)[:, :n].cpu().numpy()
    rel = np.abs(q - o.rates_of_progress(T, p, Y)) / o.reaction_gross(T, p, Y)
    assert rel.max() <= 1e-10, f"max {rel.max():.3e}"


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_negative_mass_fractions_in_some_warps(torch, precision):
    """Negative mass fractions in a few scattered states only: most warps of
    32 states have none (the rate kernels' sign-free copy of the reaction
    loops) and the others mix signed and unsigned states (the signed copy);
    both against the oracle."""
    name = "gri_53_325"
    n = CASES[name]
    T, p, Y = _states(name, n, start=907)
    rng = np.random.default_rng(23)
    some = np.arange(0, n, 97)
    for i in some:
        k = rng.choice(Y.shape[0], 3, replace=False)
        Y[k, i] = -1e-4 * rng.random(3)
    mech = mechanism(name)
    Td, pd, Yd = to_device(torch, T, p, Y, ld=n + LD_PAD)
    w = mech.production_rates(Td, pd, Yd, precision=precision)[:, :n].cpu().numpy()
    o = oracle(name)
    err = wdot_error(np.array(mech.W), w, o.production_rates(T, p, Y))
    assert err.max() <= (1e-10 if precision == "fp64" else 2e-4), f"max {err.max():.3e}"
    assert err[some].max() <= (1e-10 if precision == "fp64" else 2e-4)


@pytest.mark.parametrize("name", list(CASES))
def test_rates_of_progress_fp64(torch, name):
    n = CASES[name]
    T, p, Y = _states(name, n, start=11)
    mech = mechanism(name)
    Td, pd, Yd = to_device(torch, T, p, Y, ld=n + LD_PAD)
    q = mech.rates_of_progress(Td, pd, Yd)[:, :n].cpu().numpy()
    o = oracle(name)
    q_ref = o.rates_of_progress(T, p, Y)
    gross = o.reaction_gross(T, p, Y)
    rel = np.abs(q - q_ref) / np.where(gross > 0, gross, 1.0)
    assert np.all(gross > 0)
    assert rel.max() <= 1e-10, f"max {rel.max():.3e} at reaction {np.unravel_index(rel.argmax(), rel.shape)}"


@pytest.mark.parametrize("name", list(CASES))
def test_thermo(torch, name):
    n = CASES[name]
    T, p, Y = _states(name, n, start=5)
    mech = mechanism(name)
    Td, pd, Yd = to_device(torch, T, p, Y, ld=n + LD_PAD)
    cp, h = (t.cpu().numpy() for t in mech.thermo(Td, pd, Yd))
    o = oracle(name)
    cp_ref, h_ref = o.thermo(T, p, Y)
    np.testing.assert_allclose(cp, cp_ref, rtol=1e-12)
    m = synth.mechanism(name)
    for i in range(0, n, 97):
        t = o.species_thermo(T[i])
        scale = np.sum(Y[:, i] * np.abs(t["h_RT"]) * synth.R_U * T[i] / m.W)
        assert abs(h[i] - h_ref[i]) <= 1e-12 * scale
    assert np.max(np.abs(h - h_ref) / (np.abs(h_ref) + 1e-3 * np.abs(h_ref).max())) < 1e-9


@pytest.mark.parametrize("tr_mode", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_transport_fp64(torch, name, tr_mode):
    """tr_mode 0: double-float arithmetic on the float32 pipe; 1: native float64."""
    n = CASES[name]
    T, p, Y = _states(name, n, start=3)
    mech = mechanism(name, tr_mode=tr_mode)
    Td, pd, Yd = to_device(torch, T, p, Y, ld=n + LD_PAD)
    mu, lam, D = (t.cpu().numpy() for t in mech.transport(Td, pd, Yd))
    mu_r, lam_r, D_r = oracle(name).transport(T, p, Y)
    np.testing.assert_allclose(mu, mu_r, rtol=1e-12)
    np.testing.assert_allclose(lam, lam_r, rtol=1e-12)
    np.testing.assert_allclose(D[:, :n], D_r, rtol=1e-12)


@pytest.mark.parametrize("name", ["h2o2_9_21_direct", "gri_53_325_direct"])
@pytest.mark.parametrize("tr_mode", [0, 1])
def test_transport_direct_fits(torch, name, tr_mode):
    """Direct fits (eta, lambda, 1/D_kj as polynomials in ln T, no
    exponentials): float64-accurate kernels (float pairs, tr_mode 0; native
    float64, tr_mode 1) within 1e-12 of the oracle, the mixed kernels within
    their 5e-6 bound."""
    n = CASES[name.replace("_direct", "")]
    T, p, Y = _states(name, n, start=23)
    mech = mechanism(name, **({"tr_mode": 1} if tr_mode else {}))
    Td, pd, Yd = to_device(torch, T, p, Y, ld=n + LD_PAD)
    mu_r, lam_r, D_r = oracle(name).transport(T, p, Y)
    for prec, tol in (("fp64", 1e-12), ("mixed", 5e-6)):
        mu, lam, D = (t.cpu().numpy() for t in mech.transport(Td, pd, Yd, precision=prec))
        np.testing.assert_allclose(mu, mu_r, rtol=tol)
        np.testing.assert_allclose(lam, lam_r, rtol=tol)
        np.testing.assert_allclose(D[:, :n], D_r, rtol=tol)


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_precision_error_bounds(torch, name):
    """Mixed path: production rates within 2e-4 of the per-point scale
    (p99 within 1e-4), rates of progress within 2e-4 of their own gross
    scale, transport within 5e-6 relative.  The float32 logarithms of the
    rates (|ln R| up to ~300) carry ~1e-5 absolute rounding, which is the
    floor of these bounds."""
    n = CASES[name]
    T, p, Y = _states(name, n, start=21)
    mech = mechanism(name)
    Td, pd, Yd = to_device(torch, T, p, Y)
    o = oracle(name)
    w = mech.production_rates(Td, pd, Yd, precision="mixed").cpu().numpy()
    err = wdot_error(np.array(mech.W), w, o.production_rates(T, p, Y))
    print(f"\n{name} mixed wdot: max {err.max():.3e} p99 {np.quantile(err, 0.99):.3e} median {np.median(err):.3e}")
    q = mech.rates_of_progress(Td, pd, Yd, precision="mixed").cpu().numpy()
    gross = o.reaction_gross(T, p, Y)
    rq = np.abs(q - o.rates_of_progress(T, p, Y)) / gross
    print(f"{name} mixed rop: max {rq.max():.3e} p99 {np.quantile(rq, 0.99):.3e}")
    mu, lam, D = (t.cpu().numpy() for t in mech.transport(Td, pd, Yd, precision="mixed"))
    mu_r, lam_r, D_r = o.transport(T, p, Y)
    et = max(np.max(np.abs(mu / mu_r - 1)), np.max(np.abs(lam / lam_r - 1)), np.max(np.abs(D / D_r - 1)))
    print(f"{name} mixed transport: max rel {et:.3e}")
    assert err.max() <= 2e-4 and np.quantile(err, 0.99) <= 1e-4
    assert rq.max() <= 2e-4
    assert et <= 5e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_domain_edges(torch, precision):
    """T <= 0, p <= 0 or non-finite T/p give NaN for that point only; an
    absent species (Y_k = 0) and a pure species are ordinary states; n = 0
    is a no-op."""
    name = "h2o2_9_21"
    mech = mechanism(name)
    T, p, Y = _states(name, 300)
    T[3], T[7], T[11], p[13], T[17] = 0.0, -5.0, np.nan, 0.0, np.inf
    Y[2, 20:40] = 0.0
    Y[:, 50] = 0.0; Y[4, 50] = 1.0
    Td, pd, Yd = to_device(torch, T, p, Y)
    w = mech.production_rates(Td, pd, Yd, precision=precision).cpu().numpy()
    mu, lam, D = (t.cpu().numpy() for t in mech.transport(Td, pd, Yd, precision=precision))
    bad = [3, 7, 11, 13, 17]
    good = np.setdiff1d(np.arange(300), bad)
    assert np.all(np.isnan(w[:, bad])) and np.all(np.isnan(mu[bad])) and np.all(np.isnan(D[:, bad]))
    assert np.all(np.isfinite(w[:, good])) and np.all(np.isfinite(mu[good])) and np.all(np.isfinite(D[:, good]))
    o = oracle(name)
    w_ref = o.production_rates(T[good], p[good], Y[:, good])
    err = wdot_error(np.array(mech.W), w[:, good], w_ref)
    assert err.max() <= (1e-10 if precision == "fp64" else 2e-4)
    mu_r, lam_r, D_r = o.transport(T[good], p[good], Y[:, good])
    tol = 1e-12 if precision == "fp64" else 5e-6
    np.testing.assert_allclose(D[:, good], D_r, rtol=tol)
    np.testing.assert_allclose(mu[good], mu_r, rtol=tol)
    # n = 0
    empty = torch.empty(0, dtype=torch.float64, device="cuda")
    out = mech.production_rates(empty, empty, torch.empty((mech.n_species, 0), dtype=torch.float64, device="cuda"))
    assert out.shape == (mech.n_species, 0)


def test_point_status(torch):
    """kx_last_point_status: the smallest index of a point outside the domain
    over the calls since the last check, -1 once it has been read; a state
    whose sum Y/W is zero is outside the domain of the concentrations and
    mole fractions (rates, transport, adjoint) but not of the thermo call."""
    name = "h2o2_9_21"
    mech = mechanism(name)
    mech.last_point_status()   # clears what earlier tests on this shared handle recorded
    T, p, Y = _states(name, 300)
    Td, pd, Yd = to_device(torch, T, p, Y)
    mech.production_rates(Td, pd, Yd)
    mech.transport(Td, pd, Yd)
    assert mech.last_point_status() == -1
    T2, p2, Y2 = T.copy(), p.copy(), Y.copy()
    T2[211], p2[97] = -1.0, np.nan
    Td, pd, Yd = to_device(torch, T2, p2, Y2)
    mech.thermo(Td, pd, Yd)
    assert mech.last_point_status() == 97
    assert mech.last_point_status() == -1
    mech.production_rates(Td, pd, Yd, precision="mixed")
    mech.diffusion(Td, pd, Yd)
    assert mech.last_point_status() == 97
    Y3 = Y.copy()
    Y3[:, 150] = 0.0
    Td, pd, Yd = to_device(torch, T, p, Y3)
    mech.thermo(Td, pd, Yd)
    assert mech.last_point_status() == -1
    for call in (lambda: mech.production_rates(Td, pd, Yd), lambda: mech.viscosity_conductivity(Td, pd, Yd),
                 lambda: mech.diffusion(Td, pd, Yd, precision="mixed"),
                 lambda: mech.production_rates_vjp(Td, pd, Yd, torch.ones_like(Yd))):
        call()
        assert mech.last_point_status() == 150
    assert mech.last_point_status() == -1


def test_libmath_variant_agrees(torch):
    """The library's own float64 exp/log against CUDA's exp/log: the same
    kernels built both ways agree to 1e-13 relative (transport) and within
    the production-rate bar."""
    name = "gri_53_325"
    a, b = mechanism(name), mechanism(name, libmath=1)
    T, p, Y = _states(name, 2048, start=99)
    Td, pd, Yd = to_device(torch, T, p, Y)
    for fa, fb in zip(a.transport(Td, pd, Yd), b.transport(Td, pd, Yd)):
        np.testing.assert_allclose(fa.cpu().numpy(), fb.cpu().numpy(), rtol=1e-13)
    wa = a.production_rates(Td, pd, Yd).cpu().numpy()
    wb = b.production_rates(Td, pd, Yd).cpu().numpy()
    assert wdot_error(np.array(a.W), wa, wb).max() <= 1e-11
