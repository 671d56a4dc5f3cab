"""kx_evaluate_host: host-resident states in chunks over two streams, the
copies overlapped with the kernels.  Results must be bit-identical to the
device calls on the same states, for a ragged point count over many chunks,
every output selection and both precisions; argument errors are refused."""
import numpy as np
import pytest

from paper_2411_02640_gb300 import synth
from tests.gpu_common import mechanism, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pipeline_matches_device_calls(precision):
    torch = torch_cuda()
    name = "gri_53_325"
    mech = mechanism(name)
    ns, n = mech.n_species, 70_001
    T, p, Y = synth.make_states(ns, synth.STATE_SPECS[name], 5, n)
    Th, ph, Yh = (torch.from_numpy(a).pin_memory() for a in (T, p, Y))
    out = {"wdot": torch.empty((ns, n), dtype=torch.float64).pin_memory(), "cp": torch.empty(n, dtype=torch.float64).pin_memory(),
           "h": torch.empty(n, dtype=torch.float64).pin_memory(), "mu": torch.empty(n, dtype=torch.float64).pin_memory(),
           "lam": torch.empty(n, dtype=torch.float64).pin_memory(), "Dk": torch.empty((ns, n), dtype=torch.float64).pin_memory()}
    ws = torch.empty(2 * 8192 * mech.evaluate_host_bytes_per_state(7), dtype=torch.uint8, device="cuda")
    s = (torch.cuda.Stream(), torch.cuda.Stream())
    mech.evaluate_host(Th, ph, Yh, out, outputs=7, precision=precision, workspace=ws, max_chunk=8192, streams=s)
    torch.cuda.synchronize()
    Td, pd, Yd = (torch.from_numpy(a).cuda() for a in (T, p, Y))
    ref = {"wdot": mech.production_rates(Td, pd, Yd, precision=precision)}
    ref["cp"], ref["h"] = mech.thermo(Td, pd, Yd)
    ref["mu"], ref["lam"], ref["Dk"] = mech.transport(Td, pd, Yd, precision=precision)
    for k, v in ref.items():
        assert torch.equal(out[k], v.cpu()), k


def test_pipeline_output_selection_and_errors():
    torch = torch_cuda()
    from paper_2411_02640_gb300 import kx
    mech = mechanism("h2o2_9_21")
    ns, n = mech.n_species, 3000
    T, p, Y = synth.make_states(ns, synth.STATE_SPECS["h2o2_9_21"], 9, n)
    Th, ph, Yh = (torch.from_numpy(a).pin_memory() for a in (T, p, Y))
    ws = torch.empty(2 * 1024 * mech.evaluate_host_bytes_per_state(2), dtype=torch.uint8, device="cuda")
    out = {"cp": torch.empty(n, dtype=torch.float64).pin_memory(), "h": torch.empty(n, dtype=torch.float64).pin_memory()}
    s = (torch.cuda.Stream(), torch.cuda.Stream())
    mech.evaluate_host(Th, ph, Yh, out, outputs=mech.OUT_THERMO, workspace=ws, streams=s)
    torch.cuda.synchronize()
    cp, h = mech.thermo(*(torch.from_numpy(a).cuda() for a in (T, p, Y)))
    assert torch.equal(out["cp"], cp.cpu()) and torch.equal(out["h"], h.cpu())
    with pytest.raises(kx.KxError):       # production rates selected without a wdot buffer
        mech.evaluate_host(Th, ph, Yh, out, outputs=mech.OUT_WDOT, workspace=ws, streams=s)
    with pytest.raises(kx.KxError):       # workspace too small for two chunks
        mech.evaluate_host(Th, ph, Yh, out, outputs=mech.OUT_THERMO, workspace=ws[:100], streams=s)


def _host_case(torch, mech, name, n, start):
    ns = mech.n_species
    T, p, Y = synth.make_states(ns, synth.STATE_SPECS[name], start, n)
    host = tuple(torch.from_numpy(a).pin_memory() for a in (T, p, Y))
    out = {"wdot": torch.empty((ns, n), dtype=torch.float64).pin_memory(), "cp": torch.empty(n, dtype=torch.float64).pin_memory(),
           "h": torch.empty(n, dtype=torch.float64).pin_memory(), "mu": torch.empty(n, dtype=torch.float64).pin_memory(),
           "lam": torch.empty(n, dtype=torch.float64).pin_memory(), "Dk": torch.empty((ns, n), dtype=torch.float64).pin_memory()}
    return (T, p, Y), host, out


def _check_against_device_calls(torch, mech, states, out):
    Td, pd, Yd = (torch.from_numpy(a).cuda() for a in states)
    ref = {"wdot": mech.production_rates(Td, pd, Yd)}
    ref["cp"], ref["h"] = mech.thermo(Td, pd, Yd)
    ref["mu"], ref["lam"], ref["Dk"] = mech.transport(Td, pd, Yd)
    for k, v in ref.items():
        assert torch.equal(out[k], v.cpu()), k


def test_back_to_back_calls_share_the_workspace():
    """Three calls queued without a synchronisation in between, on one
    workspace and one pair of streams (the library's own streams and events
    are reused from call to call): each call's chunks must wait for the
    previous call's copies out of the same workspace slots."""
    torch = torch_cuda()
    name = "gri_53_325"
    mech = mechanism(name)
    ws = torch.empty(2 * 4096 * mech.evaluate_host_bytes_per_state(7), dtype=torch.uint8, device="cuda")
    s = (torch.cuda.Stream(), torch.cuda.Stream())
    cases = [_host_case(torch, mech, name, n, start) for n, start in ((20_011, 100), (9_001, 50_000), (13_337, 7))]
    for _, host, out in cases:
        mech.evaluate_host(*host, out, outputs=7, workspace=ws, max_chunk=4096, streams=s)
    torch.cuda.synchronize()
    for states, _, out in cases:
        _check_against_device_calls(torch, mech, states, out)


def test_calls_from_two_host_threads():
    """Two host threads call kx_evaluate_host on one handle at the same time,
    each with its own workspace and streams."""
    import threading
    torch = torch_cuda()
    name = "gri_53_325"
    mech = mechanism(name)
    cases = [_host_case(torch, mech, name, n, start) for n, start in ((30_001, 300), (25_013, 90_000))]
    errors = []

    def run(case):
        try:
            _, host, out = case
            ws = torch.empty(2 * 4096 * mech.evaluate_host_bytes_per_state(7), dtype=torch.uint8, device="cuda")
            s = (torch.cuda.Stream(), torch.cuda.Stream())
            for _ in range(2):
                mech.evaluate_host(*host, out, outputs=7, workspace=ws, max_chunk=4096, streams=s)
            for q in s:
                q.synchronize()
        except Exception as e:   # reported on the main thread
            errors.append(e)

    th = [threading.Thread(target=run, args=(c,)) for c in cases]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    torch.cuda.synchronize()
    for states, _, out in cases:
        _check_against_device_calls(torch, mech, states, out)
