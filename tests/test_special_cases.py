"""The paper's special cases of the forward rate constant (Sec. 2.3.1) on a
workload that has them: "<name>_special" mechanisms carry the ethanol
mechanism's mix (27 % k = A, 0.6 % k = A T^n, 21 % shared (beta, E)).  The
emitter's counts (no compile needed) must show the exponentials saved in the
native float64 kernel and the float-pair ln k arithmetic saved for k = A; the
GPU kernels must keep parity with the oracle on it."""
import numpy as np
import pytest

from paper_2411_02640_gb300 import kx, synth
from tests.gpu_common import mechanism, oracle, to_device, torch_cuda, wdot_error


def test_special_mix_drawn():
    m = synth.mechanism("gri_53_325_special")
    base = synth.mechanism("gri_53_325")
    ks = [a for r in m.reactions for a in [r.rate] + ([r.rate_low] if r.rate_low else [])]
    const = sum(1 for a in ks if a[1] == 0.0 and a[2] == 0.0)
    assert abs(const / len(ks) - 0.27) < 0.01
    assert [r.rate[0] for r in m.reactions] == [r.rate[0] for r in base.reactions]   # A kept
    assert [(r.reactants, r.products) for r in m.reactions] == [(r.reactants, r.products) for r in base.reactions]


def test_emitter_counts_show_the_special_cases(tmp_path):
    counts = {}
    for name in ("gri_53_325", "gri_53_325_special"):
        path = synth.mechanism_file(name, str(tmp_path))
        native = kx.Mechanism(path, compile_only=1, lazy=1, rates_arith=1, cache_dir=str(tmp_path / "c"))
        pair = kx.Mechanism(path, compile_only=1, lazy=1, cache_dir=str(tmp_path / "c"))
        counts[name] = (native.op_counts("wdot_fp64"), pair.op_counts("wdot_fp64"))
    (nb, pb), (ns_, ps) = counts["gri_53_325"], counts["gri_53_325_special"]
    assert ns_["exp64"] <= nb["exp64"] - 100          # k = A, k = A T^n and shared (beta, E) need no exp
    assert ps["fp32"] < pb["fp32"] - 70 * 30          # ln k = ln A: two float-pair fmas saved per k = A (80 here)


@pytest.mark.gpu
@pytest.mark.parametrize("arith,precision", [(0, "fp64"), (1, "fp64"), (0, "mixed")])
def test_special_mix_parity(arith, precision):
    torch = torch_cuda()
    name = "gri_53_325_special"
    n = 1289
    m = synth.mechanism(name)
    T, p, Y = synth.make_states(m.n_species, synth.STATE_SPECS[name], 17, n)
    mech = mechanism(name, **({"rates_arith": 1} if arith else {}))
    Td, pd, Yd = to_device(torch, T, p, Y)
    w = mech.production_rates(Td, pd, Yd, precision=precision).cpu().numpy()
    err = wdot_error(np.array(mech.W), w, oracle(name).production_rates(T, p, Y))
    assert err.max() <= (1e-10 if precision == "fp64" else 2e-4)
