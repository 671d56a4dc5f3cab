"""Parity at the benchmark's full size: 2^20 states of the 53-species /
325-reaction workload, drawn by the benchmark's own input generator and run
through the same calls the benchmark times (float64-accurate and mixed
production rates, thermo, viscosity/conductivity and diffusion), so that
every kernel runs its full grid with many states per thread.  A sample of
states spread over the batch, plus the ragged end, is checked against the
oracle state by state; every output must be finite."""
import numpy as np
import pytest

from tests.gpu_common import mechanism, oracle, to_device, torch_cuda, wdot_error

pytestmark = pytest.mark.gpu

N = 1 << 20


def test_benchmark_workload_sampled_against_oracle():
    torch = torch_cuda()
    import bench
    name = bench.MECH
    T, p, Y = bench.make_inputs(0, N)
    mech = mechanism(name)
    Td, pd, Yd = to_device(torch, T, p, Y)
    out = {"w64": mech.production_rates(Td, pd, Yd, precision="fp64"),
           "wmx": mech.production_rates(Td, pd, Yd, precision="mixed")}
    out["cp"], out["h"] = mech.thermo(Td, pd, Yd)
    out["mu"], out["lam"], out["D"] = mech.transport(Td, pd, Yd, precision="fp64")
    out["mu_mx"], out["lam_mx"], out["D_mx"] = mech.transport(Td, pd, Yd, precision="mixed")
    torch.cuda.synchronize()
    for k, v in out.items():
        assert bool(torch.isfinite(v).all()), k
    idx = np.unique(np.concatenate([np.linspace(0, N - 1, 384).astype(np.int64), np.arange(N - 8, N)]))
    Ts, ps, Ys = T[idx], p[idx], np.ascontiguousarray(Y[:, idx])
    got = {k: (v[:, idx] if v.dim() == 2 else v[idx]).cpu().numpy() for k, v in out.items()}
    o = oracle(name)
    W = np.array(mech.W)
    w_ref = o.production_rates(Ts, ps, Ys)
    assert wdot_error(W, got["w64"], w_ref).max() <= 1e-10
    assert wdot_error(W, got["wmx"], w_ref).max() <= 2e-4
    cp_ref, h_ref = o.thermo(Ts, ps, Ys)
    np.testing.assert_allclose(got["cp"], cp_ref, rtol=1e-12)
    from paper_2411_02640_gb300 import synth
    m = synth.mechanism(name)
    for j in range(len(idx)):   # h against the size of its terms, sum_k |Y_k h_k| (h itself crosses zero)
        t = o.species_thermo(Ts[j])
        scale = np.sum(np.abs(Ys[:, j] * t["h_RT"]) * synth.R_U * Ts[j] / m.W)
        assert abs(got["h"][j] - h_ref[j]) <= 1e-12 * scale
    mu_ref, lam_ref, D_ref = o.transport(Ts, ps, Ys)
    for key, ref in (("mu", mu_ref), ("lam", lam_ref), ("D", D_ref)):
        np.testing.assert_allclose(got[key], ref, rtol=1e-12)
        np.testing.assert_allclose(got[key + "_mx"], ref, rtol=5e-6)
