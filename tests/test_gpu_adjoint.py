"""The adjoint kernel against the oracle's dense Jacobian (forward-mode dual
numbers, independent of the GPU code) and against central finite
differences of the GPU forward kernel."""
import numpy as np
import pytest

from paper_2411_02640_gb300 import synth
from tests.gpu_common import mechanism, oracle, to_device, torch_cuda

pytestmark = pytest.mark.gpu


def _states(name, n, start=0):
    m = synth.mechanism(name)
    return synth.make_states(m.n_species, synth.STATE_SPECS[name], start, n)


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.mark.parametrize("name,n", [("h2o2_9_21", 300), ("gri_53_325", 256)])
def test_vjp_matches_oracle_jacobian(torch, name, n):
    T, p, Y = _states(name, n, start=1000)
    mech = mechanism(name)
    rng = np.random.default_rng(7)
    v = rng.standard_normal((mech.n_species, n))
    Td, pd, Yd = to_device(torch, T, p, Y)
    gT, gY = mech.production_rates_vjp(Td, pd, Yd, torch.tensor(v, device="cuda"))
    gT, gY = gT.cpu().numpy(), gY.cpu().numpy()
    o = oracle(name)
    for i in range(n):
        J = o.jacobian(T[i], p[i], Y[:, i])              # [ns, 1 + ns]
        ref = v[:, i] @ J
        scale = np.abs(v[:, i]) @ np.abs(J)               # size of the terms of each entry
        got = np.concatenate([[gT[i]], gY[:, i]])
        tol = 1e-9 * scale.max()
        assert np.all(np.abs(got - ref) <= tol + 1e-9 * scale), (i, np.max(np.abs(got - ref) / (scale + 1e-300)))


def test_autograd_function_and_finite_differences(torch):
    from paper_2411_02640_gb300.autograd import production_rates
    name = "gri_53_325"
    T, p, Y = _states(name, 64, start=2000)
    mech = mechanism(name)
    Td, pd, Yd = to_device(torch, T, p, Y)
    Td.requires_grad_(True); Yd.requires_grad_(True)
    w = production_rates(mech, Td, pd, Yd)
    v = torch.randn_like(w)
    (w * v).sum().backward()
    gT, gY = Td.grad.clone(), Yd.grad.clone()
    with torch.no_grad():
        h = 1e-6 * Td
        fd_T = ((mech.production_rates(Td + h, pd, Yd) - mech.production_rates(Td - h, pd, Yd)) * v).sum(0) / (2 * h)
        scale = (torch.abs(mech.production_rates(Td, pd, Yd)) * torch.abs(v)).sum(0) / Td
        assert torch.all(torch.abs(fd_T - gT) <= 1e-5 * scale + 1e-5 * torch.abs(gT))
        for j in range(0, mech.n_species, 13):
            hy = 1e-6 * torch.clamp(Yd[j], min=1e-3)
            Yp, Ym = Yd.clone(), Yd.clone()
            Yp[j] += hy; Ym[j] -= hy
            fd = ((mech.production_rates(Td, pd, Yp) - mech.production_rates(Td, pd, Ym)) * v).sum(0) / (2 * hy)
            sc = (torch.abs(mech.production_rates(Td, pd, Yd)) * torch.abs(v)).sum(0) / torch.clamp(Yd[j], min=1e-3)
            assert torch.all(torch.abs(fd - gY[j]) <= 1e-4 * sc + 1e-5 * torch.abs(gY[j])), j


def test_jacobian_assembly_matches_oracle(torch):
    from paper_2411_02640_gb300.autograd import jacobian
    name = "gri_53_325"
    T, p, Y = _states(name, 32, start=3000)
    mech = mechanism(name)
    Td, pd, Yd = to_device(torch, T, p, Y)
    J = jacobian(mech, Td, pd, Yd).cpu().numpy()
    o = oracle(name)
    for i in range(32):
        Jr = o.jacobian(T[i], p[i], Y[:, i])
        sc = np.abs(Jr).max(axis=1, keepdims=True)
        assert np.all(np.abs(J[i] - Jr) <= 1e-9 * sc + 1e-300)
