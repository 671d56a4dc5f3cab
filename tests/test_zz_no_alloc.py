"""kx_production_rates_noalloc: the float64-accurate production rates with
the rate kernel's per-state species vectors in the library's static device
scratch array instead of local memory, so that a call allocates nothing on
the device.  Checked: the exported symbol and the scratch size in the
header (CPU); on the GPU, results bit-identical to kx_production_rates at
sizes that reuse each thread's scratch many times, parity with the oracle,
unchanged free device memory across calls, and a call replayed from a CUDA
graph."""
import ctypes
import os

import numpy as np
import pytest

from paper_2411_02640_gb300 import kx, synth
from tests.gpu_common import mechanism, oracle, to_device, torch_cuda, wdot_error

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "kx.h")


def test_entry_point_exported_and_declared():
    L = ctypes.CDLL(kx.library_path())
    assert hasattr(L, "kx_production_rates_noalloc")
    text = open(HEADER).read()
    assert "kx_status kx_production_rates_noalloc(" in text
    assert "#define KX_NOALLOC_SCRATCH_BYTES ((size_t)128 << 20)" in text


@pytest.mark.gpu
@pytest.mark.parametrize("name,n", [("h2o2_9_21", 4133), ("gri_53_325", 300_037)])
def test_noalloc_matches_regular_and_oracle(name, n):
    torch = torch_cuda()
    mech = mechanism(name)
    T, p, Y = synth.make_states_torch(mech.n_species, synth.STATE_SPECS[name], n, seed=41)
    w_ref = mech.production_rates(T, p, Y)
    w = torch.full_like(w_ref, float("nan"))
    mech.production_rates_noalloc(T, p, Y, w)
    torch.cuda.synchronize()
    assert torch.equal(w, w_ref)
    # the oracle on a sample spread over the batch, including the ragged end
    idx = np.unique(np.concatenate([np.linspace(0, n - 1, 256).astype(np.int64), np.arange(n - 5, n)]))
    Ts, ps, Ys = T[idx].cpu().numpy(), p[idx].cpu().numpy(), Y[:, idx].cpu().numpy()
    err = wdot_error(np.array(mech.W), w[:, idx].cpu().numpy(), oracle(name).production_rates(Ts, ps, Ys))
    assert err.max() <= 1e-10


@pytest.mark.gpu
def test_noalloc_calls_leave_free_memory_unchanged_and_replay_from_a_graph():
    torch = torch_cuda()
    name = "gri_53_325"
    mech = mechanism(name)
    n = 1 << 18
    T, p, Y = synth.make_states_torch(mech.n_species, synth.STATE_SPECS[name], n, seed=42)
    w_ref = mech.production_rates(T, p, Y)
    w = torch.empty_like(w_ref)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        mech.production_rates_noalloc(T, p, Y, w)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(w, w_ref)
    # captured into a CUDA graph and replayed on new inputs
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    w.zero_()
    with torch.cuda.graph(g, stream=s):
        mech.production_rates_noalloc(T, p, Y, w, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(w, w_ref)
    T2, p2, Y2 = synth.make_states_torch(mech.n_species, synth.STATE_SPECS[name], n, seed=43)
    T.copy_(T2); p.copy_(p2); Y.copy_(Y2)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(w, mech.production_rates(T, p, Y))
