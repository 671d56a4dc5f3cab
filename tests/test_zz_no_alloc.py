"""kx_production_rates_noalloc: production rates for callers that cannot have
device memory allocated while they run (a solver that gives all free device
memory to its own pool at start-up, a time step that must not stall on the
synchronisation an allocation implies).  The call keeps the rate kernel's
per-state species vectors in the library's static device array instead of
local memory.

Checked here: the exported symbol, the declared array size and the kernel's
small per-thread local memory (CPU); on the
GPU, two calls in a row through the C ABI, the second on other states and
fewer of them (so the array still holds the first call's values), each
against kx_production_rates within the production-rate tolerance, one of them
also against the oracle, and free device memory unchanged across the calls.
This file is collected last so that a run stopping at its first failure has
run every other test before it."""
import ctypes
import os

import numpy as np
import pytest

from paper_2411_02640_gb300 import kx, synth
from tests.gpu_common import mechanism, oracle, torch_cuda, wdot_error

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kx.h")
# float64-accurate production rates: max_k W_k |dwdot_k| / max_k W_k |wdot_k| per state
TOL = 1e-10


def test_entry_point_exported_and_declared():
    L = ctypes.CDLL(kx.library_path())
    assert hasattr(L, "kx_production_rates_noalloc")
    text = open(HEADER).read()
    assert "kx_status kx_production_rates_noalloc(" in text
    assert "#define KX_NOALLOC_SCRATCH_BYTES ((size_t)128 << 20)" in text


@pytest.mark.parametrize("name", ["h2o2_9_21", "gri_53_325"])
def test_noalloc_kernel_local_memory_is_small(name):
    """The no-alloc kernel's own per-thread local memory (stack frame: local
    arrays and register spills, from the compiler's report; compiled without a
    GPU) stays within the 1 KB per thread that a CUDA context reserves by
    default (cudaLimitStackSize) and below the regular kernel's, so its launch
    gives the driver no reason to grow the local-memory backing."""
    m = kx.Mechanism(synth.mechanism_file(name, os.path.join(ROOT, ".kxcache", "mech")),
                     cache_dir=os.path.join(ROOT, ".kxcache"), compile_only=1, lazy=1)
    na = m.kernel_info("wdot_fp64_noalloc")["local_bytes"]
    reg = m.kernel_info("wdot_fp64")["local_bytes"]
    assert 0 <= na <= 1024
    assert na <= reg


def _states(mech, name, n, seed):
    return synth.make_states_torch(mech.n_species, synth.STATE_SPECS[name], n, seed=seed)


@pytest.mark.gpu
@pytest.mark.parametrize("name,n1,n2", [("h2o2_9_21", 4133, 1031), ("gri_53_325", 600_037, 300_011)])
def test_two_calls_in_a_row_match_the_regular_entry_point(name, n1, n2):
    torch = torch_cuda()
    mech = mechanism(name)
    W = np.array(mech.W)
    T1, p1, Y1 = _states(mech, name, n1, seed=41)
    T2, p2, Y2 = _states(mech, name, n2, seed=42)
    ref1 = mech.production_rates(T1, p1, Y1)
    ref2 = mech.production_rates(T2, p2, Y2)
    out1 = torch.full_like(ref1, float("nan"))
    out2 = torch.full_like(ref2, float("nan"))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    mech.production_rates_noalloc(T1, p1, Y1, out1)
    mech.production_rates_noalloc(T2, p2, Y2, out2)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for out, ref in ((out1, ref1), (out2, ref2)):
        assert bool(torch.isfinite(out).all())
        err = wdot_error(W, out.cpu().numpy(), ref.cpu().numpy())
        assert err.max() <= TOL
    # the oracle on a sample of the second call, spread over it and its ragged end
    idx = np.unique(np.concatenate([np.linspace(0, n2 - 1, 192).astype(np.int64), np.arange(n2 - 5, n2)]))
    Ts, ps, Ys = T2[idx].cpu().numpy(), p2[idx].cpu().numpy(), Y2[:, idx].cpu().numpy()
    err = wdot_error(W, out2[:, idx].cpu().numpy(), oracle(name).production_rates(Ts, ps, Ys))
    assert err.max() <= TOL
