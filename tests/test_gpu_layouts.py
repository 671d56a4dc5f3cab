"""The two float-pair production-rate kernels and the batch-size choice
between them.  rates_layout 1 is one thread per state (species vectors in
local memory); rates_layout 2 is warp-cooperative (the lanes of a warp share
a state: reactions dealt out over the lanes, species vectors and rates in
shared memory, wdot gathered species-major); the default picks the second
below the first's resident capacity.  Both are held to the oracle element
by element (1e-10 of the per-point scale), the automatic choice is checked to reproduce each kernel bit for bit on its
side of the threshold, and the warp-cooperative kernel is run with every
states-per-warp grouping on a ragged batch."""
import numpy as np
import pytest

from paper_2411_02640_gb300 import synth
from tests.gpu_common import mechanism, oracle, to_device, torch_cuda, wdot_error

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.mark.parametrize("layout", [1, 2])
@pytest.mark.parametrize("name,n", [("h2o2_9_21", 4133), ("gri_53_325", 1289), ("large_160_900", 300)])
def test_each_layout_against_oracle(name, n, layout):
    torch = torch_cuda()
    m = synth.mechanism(name)
    T, p, Y = synth.make_states(m.n_species, synth.STATE_SPECS[name], 77, n)
    mech = mechanism(name, rates_layout=layout)
    Td, pd, Yd = to_device(torch, T, p, Y, ld=n + 13)
    w = mech.production_rates(Td, pd, Yd)[:, :n].cpu().numpy()
    err = wdot_error(np.array(mech.W), w, oracle(name).production_rates(T, p, Y))
    assert np.all(np.isfinite(w))
    assert err.max() <= TOL, f"max {err.max():.3e}"


@pytest.mark.parametrize("group", [1, 2, 4, 8, 16, 32])
def test_warp_cooperative_every_group_size(group):
    """States per warp from 1 to 32 on 9/21 with a ragged batch (1000 states:
    not a multiple of any group)."""
    torch = torch_cuda()
    name, n = "h2o2_9_21", 1000
    m = synth.mechanism(name)
    T, p, Y = synth.make_states(m.n_species, synth.STATE_SPECS[name], 5, n)
    mech = mechanism(name, rates_layout=2, rates_group=group)
    Td, pd, Yd = to_device(torch, T, p, Y)
    w = mech.production_rates(Td, pd, Yd).cpu().numpy()
    err = wdot_error(np.array(mech.W), w, oracle(name).production_rates(T, p, Y))
    assert err.max() <= TOL, f"group {group}: max {err.max():.3e}"


def test_automatic_choice_follows_the_batch_size():
    """Below the thread-per-state kernel's resident capacity the default
    handle gives exactly the warp-cooperative kernel's results, above it
    exactly the thread-per-state kernel's; both sides agree within the bar."""
    torch = torch_cuda()
    name = "gri_53_325"
    auto, tps, wc = mechanism(name), mechanism(name, rates_layout=1), mechanism(name, rates_layout=2)
    spec = synth.STATE_SPECS[name]
    T, p, Y = synth.make_states_torch(auto.n_species, spec, 1 << 18, seed=9)
    W = np.array(auto.W)
    for n, same in ((1 << 12, wc), (1 << 18, tps)):
        Ts, ps, Ys = T[:n], p[:n], Y[:, :n].contiguous()
        a = auto.production_rates(Ts, ps, Ys)
        assert torch.equal(a, same.production_rates(Ts, ps, Ys)), n
        other = tps if same is wc else wc
        assert wdot_error(W, a.cpu().numpy(), other.production_rates(Ts, ps, Ys).cpu().numpy()).max() <= TOL


@pytest.mark.parametrize("layout", [1, 2])
def test_absent_and_negative_species_each_layout(layout):
    """Absent species (Y_k = 0, the ln |C_k| floor) and small negative mass
    fractions (signed concentration products) in both kernels, against the
    oracle; a batch below the crossover so that the default would pick the
    warp-cooperative kernel."""
    torch = torch_cuda()
    name, n = "gri_53_325", 777
    m = synth.mechanism(name)
    T, p, Y = synth.make_states(m.n_species, synth.STATE_SPECS[name], 4242, n)
    rng = np.random.default_rng(23)
    Y[rng.random(Y.shape) < 0.3] = 0.0
    neg = rng.random(Y.shape) < 0.05
    Y[neg] = -1e-4 * rng.random(int(neg.sum()))
    mech = mechanism(name, rates_layout=layout)
    Td, pd, Yd = to_device(torch, T, p, Y, ld=n + 5)
    w = mech.production_rates(Td, pd, Yd)[:, :n].cpu().numpy()
    assert np.all(np.isfinite(w))
    err = wdot_error(np.array(mech.W), w, oracle(name).production_rates(T, p, Y))
    assert err.max() <= TOL, f"max {err.max():.3e}"
