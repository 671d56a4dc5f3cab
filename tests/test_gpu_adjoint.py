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


@pytest.mark.parametrize("opts", [{"vjp_layout": 1}, {"rates_arith": 1}, {"vjp_layout": 2}])
@pytest.mark.parametrize("name,n", [("h2o2_9_21", 300), ("gri_53_325", 256), ("large_160_900", 64)])
def test_vjp_matches_oracle_jacobian(torch, name, n, opts):
    """vjp_layout 1: the double-float adjoint, one thread per state; rates_arith 1: native
    float64; vjp_layout 2: the warp-cooperative double-float adjoint (the default's choice for
    batches this small)."""
    T, p, Y = _states(name, n, start=1000)
    mech = mechanism(name, **opts)
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


@pytest.mark.parametrize("opts", [{"vjp_layout": 1}, {"vjp_layout": 1, "vjp_form": 1}, {"rates_arith": 1},
                                  {"vjp_layout": 2}])
def test_vjp_absent_and_negative_species(torch, opts):
    """States with species absent (Y_k = 0 exactly, as in a fresh mixture) and
    small negative mass fractions: the derivative with respect to an absent
    species is finite and nonzero (d(k C_A C_B)/dC_A = k C_B); the double-float
    adjoint forms each such term from log-space quantities (the rate's mantissa
    and power of two times 1/|C_k|, or one exponential per entry with
    vjp_form 1; rates below float64 shifted by 2^2016), so it must match the
    oracle's dual-number Jacobian there too; native float64 beside it."""
    name, n = "gri_53_325", 128
    T, p, Y = _states(name, n, start=5000)
    rng = np.random.default_rng(11)
    Y[rng.random(Y.shape) < 0.25] = 0.0
    neg = rng.random(Y.shape) < 0.05
    Y[neg] = -1e-5 * rng.random(int(neg.sum()))
    mech = mechanism(name, **opts)
    v = rng.standard_normal((mech.n_species, n))
    Td, pd, Yd = to_device(torch, T, p, Y)
    gT, gY = mech.production_rates_vjp(Td, pd, Yd, torch.tensor(v, device="cuda"))
    gT, gY = gT.cpu().numpy(), gY.cpu().numpy()
    assert np.all(np.isfinite(gT)) and np.all(np.isfinite(gY))
    o = oracle(name)
    for i in range(n):
        J = o.jacobian(T[i], p[i], Y[:, i])
        ref = v[:, i] @ J
        scale = np.abs(v[:, i]) @ np.abs(J)
        got = np.concatenate([[gT[i]], gY[:, i]])
        assert np.all(np.abs(got - ref) <= 1e-9 * scale.max() + 1e-9 * scale), (i, np.max(np.abs(got - ref) / (scale + 1e-300)))


def test_automatic_adjoint_choice_follows_the_batch_size(torch):
    """Below the crossover the default handle gives exactly the warp-cooperative
    adjoint's results, above it exactly the thread-per-state adjoint's; the
    two agree within the adjoint's bar on both sides."""
    name = "gri_53_325"
    auto, tps, wc = mechanism(name), mechanism(name, vjp_layout=1), mechanism(name, vjp_layout=2)
    ns = auto.n_species
    T, p, Y = synth.make_states_torch(ns, synth.STATE_SPECS[name], 1 << 18, seed=21)
    v = torch.randn((ns, 1 << 18), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    for n, same in ((1 << 12, wc), (1 << 18, tps)):
        args = (T[:n], p[:n], Y[:, :n].contiguous(), v[:, :n].contiguous())
        a = auto.production_rates_vjp(*args)
        b = same.production_rates_vjp(*args)
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]), n
        c = (tps if same is wc else wc).production_rates_vjp(*args)
        for x, y in zip(a, c):
            # per state, relative to its largest entry (gY) or to the batch's largest (gT); measured
            # ~1e-10 between the two kernels and each against native float64
            sc = torch.abs(y).amax(0).clamp_min(1e-300)
            assert torch.all(torch.abs(x - y) <= 1e-8 * sc), n


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


def test_adjoint_throughput_and_jacobian_assembly_timing(torch):
    """The 53/325 adjoint at 2^18 states (random N(0,1) cotangents) and the
    dense Jacobian assembled from 54 adjoint calls against a central
    finite-difference Jacobian (108 production-rate calls) on 2^14 states;
    prints one JSON line ("adjoint_timing: {...}")."""
    import json
    from paper_2411_02640_gb300.autograd import jacobian
    name = "gri_53_325"
    mech = mechanism(name)
    m = synth.mechanism(name)
    ns = mech.n_species
    T, p, Y = synth.make_states_torch(ns, synth.STATE_SPECS[name], 1 << 18, seed=104)
    v = torch.randn((ns, 1 << 18), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    gT, gY = mech.production_rates_vjp(T, p, Y, v)
    w = mech.production_rates(T, p, Y)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    for _ in range(5):
        mech.production_rates_vjp(T, p, Y, v, out=(gT, gY))
    ev[1].record()
    for _ in range(5):
        mech.production_rates(T, p, Y, out=w)
    ev[2].record()
    torch.cuda.synchronize()
    vjp_ms, fwd_ms = ev[0].elapsed_time(ev[1]) / 5, ev[1].elapsed_time(ev[2]) / 5
    nj = 1 << 14
    Tj, pj, Yj = T[:nj].contiguous(), p[:nj].contiguous(), Y[:, :nj].contiguous()
    J = jacobian(mech, Tj, pj, Yj)
    torch.cuda.synchronize()
    ev[0].record()
    J = jacobian(mech, Tj, pj, Yj)
    ev[1].record()
    # central differences, one column per input; the float64-accurate forward path rounds at about
    # 1e-12 of the per-point scale (float pairs), so the step that balances truncation (h^2) against
    # rounding (eps/h) is h ~ eps^(1/3) = 1e-4 relative

    def fd(m):
        Jfd = torch.empty_like(J)
        h = 1e-4 * Tj
        Jfd[:, :, 0] = ((m.production_rates(Tj + h, pj, Yj) - m.production_rates(Tj - h, pj, Yj)) / (2 * h)).t()
        for j in range(ns):
            hy = 1e-4 * torch.clamp(Yj[j], min=1e-3)
            Yp, Ym = Yj.clone(), Yj.clone()
            Yp[j] += hy
            Ym[j] -= hy
            Jfd[:, :, 1 + j] = ((m.production_rates(Tj, pj, Yp) - m.production_rates(Tj, pj, Ym)) / (2 * hy)).t()
        return Jfd
    fd(mech)
    ev[2].record()
    torch.cuda.synchronize()
    jac_ms, fd_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    # the comparison differences the rates with every reaction in float pairs: the default path's
    # float32 evaluation of negligible reactions leaves the rows of species that only such reactions
    # touch at ~1e-4 of themselves, noise that the differences amplify (far inside the per-point bar)
    Jfd = fd(mechanism(name, rates_negligible=1))
    # the two Jacobians agree to the finite-difference truncation level, row-scaled
    sc = J.abs().amax(dim=2, keepdim=True) + 1e-300
    rel = ((J - Jfd).abs() / sc).flatten()
    agree = rel[:: max(1, rel.numel() // (1 << 22))].quantile(0.99).item()
    stats = {"states_vjp": 1 << 18, "vjp_ms": vjp_ms, "vjp_mpoints_s": (1 << 18) / vjp_ms / 1e3,
             "forward_ms": fwd_ms, "states_jacobian": nj, "jacobian_54_vjp_ms": jac_ms, "fd_jacobian_108_fwd_ms": fd_ms,
             "fd_vs_adjoint_p99_row_scaled": agree}
    print("\nadjoint_timing: " + json.dumps(stats))
    assert agree < 1e-3
