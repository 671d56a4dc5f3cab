"""The continuous-batching server: results the same alone and in the mix
(bit for bit for the mixed-precision rates and the transport; within the
float64 bar for the float64-accurate rates, whose kernel depends on the
batch size),
admission under a device-memory budget, rejection of oversize requests,
and agreement with direct library calls."""
import threading

import numpy as np
import pytest

from paper_2411_02640_gb300 import synth
from tests.gpu_common import mechanism, torch_cuda, wdot_error

pytestmark = pytest.mark.gpu

MECHS = ["h2o2_9_21", "gri_53_325"]


def _req(name, n, start, seed):
    m = synth.mechanism(name)
    return synth.make_states(m.n_species, synth.STATE_SPECS[name], start, n)


@pytest.fixture(scope="module")
def server_parts():
    torch_cuda()
    return {name: mechanism(name) for name in MECHS}


def _workload(seed=0, count=24):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        name = MECHS[i % 2]
        n = int(np.exp(rng.uniform(np.log(1000), np.log(60000))))
        out.append((name, _req(name, n, int(rng.integers(0, 1 << 20)), i), "mixed" if rng.random() < 0.7 else "fp64",
                    bool(rng.random() < 0.3)))
    return out


def test_result_identical_alone_and_in_the_mix(server_parts):
    from paper_2411_02640_gb300.serve import Server
    work = _workload()
    # in the mix: submitted together from several "CFD rank" threads
    with Server(server_parts, hbm_budget=2 << 30, streams=4) as srv:
        futs = [None] * len(work)

        def rank(idx):
            for i in idx:
                name, (T, p, Y), prec, tr = work[i]
                futs[i] = srv.submit(name, T, p, Y, precision=prec, transport=tr)

        th = [threading.Thread(target=rank, args=(range(r, len(work), 3),)) for r in range(3)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        mixed = [f.result(timeout=300) for f in futs]
        st = srv.stats()
    assert st["requests"] == len(work)
    assert st["launches"] < len(work)          # some requests were coalesced
    # alone: one request at a time, no coalescing
    with Server(server_parts, hbm_budget=2 << 30, streams=1, coalesce=False) as srv:
        alone = [srv.submit(name, T, p, Y, precision=prec, transport=tr).result(timeout=300)
                 for name, (T, p, Y), prec, tr in work]
    for a, b, (name, _, prec, tr) in zip(mixed, alone, work):
        if prec == "fp64":
            # a request alone may be small enough for the warp-cooperative rate kernel and in the mix
            # part of a batch large enough for the thread-per-state one: the two agree within the
            # float64 bar (1e-10 of the per-point scale), not bit for bit
            W = np.array(server_parts[name].W)
            assert wdot_error(W, a.wdot, b.wdot).max() <= 1e-10, name
        else:
            assert np.array_equal(a.wdot, b.wdot, equal_nan=True), name
        if tr:
            assert np.array_equal(a.mu, b.mu) and np.array_equal(a.lam, b.lam) and np.array_equal(a.Dk, b.Dk)


def test_agrees_with_direct_calls_and_budget(server_parts):
    import torch
    from paper_2411_02640_gb300.serve import Server
    name = "gri_53_325"
    mech = server_parts[name]
    T, p, Y = _req(name, 5000, 123, 0)
    bpp = 8 * (2 + 53 + 53 + 2 + 53)
    # a budget that admits one request at a time: everything still completes
    with Server(server_parts, hbm_budget=int(6000 * bpp), streams=4) as srv:
        futs = [srv.submit(name, T, p, Y, precision="fp64", transport=True) for _ in range(5)]
        res = [f.result(timeout=300) for f in futs]
        big = srv.submit(name, np.ones(100000), np.ones(100000), np.ones((53, 100000)), transport=True)
        with pytest.raises(MemoryError):
            big.result(timeout=10)
    Td, pd, Yd = (torch.tensor(a, device="cuda") for a in (T, p, Y))
    w = mech.production_rates(Td, pd, Yd).cpu().numpy()
    mu, lam, D = (t.cpu().numpy() for t in mech.transport(Td, pd, Yd))
    for r in res:
        assert np.array_equal(r.wdot, w) and np.array_equal(r.mu, mu) and np.array_equal(r.Dk, D)


def test_failure_in_the_loop_fails_the_waiting_requests(server_parts, monkeypatch):
    """A fault injected on the host (a launch that raises) fails every
    waiting request with an error instead of leaving it hanging."""
    from paper_2411_02640_gb300.serve import Server
    srv = Server(server_parts, hbm_budget=1 << 30, streams=2)

    def boom(*a, **k):
        raise RuntimeError("injected launch failure")
    monkeypatch.setattr(srv, "_launch", boom)
    T, p, Y = _req("h2o2_9_21", 2000, 0, 0)
    futs = [srv.submit("h2o2_9_21", T, p, Y) for _ in range(3)]     # queued before the loop starts
    srv.start()
    for f in futs:
        with pytest.raises(RuntimeError, match="injected"):
            f.result(timeout=30)
    with pytest.raises(RuntimeError):
        srv.submit("h2o2_9_21", T, p, Y)
    srv.stop()


def test_caller_owned_outputs(server_parts):
    """Requests that bring their own pinned host buffers get bit-identical
    results written into them, alone and coalesced with requests that do
    not; the Result's arrays are views of the caller's buffers."""
    import torch
    from paper_2411_02640_gb300.serve import Server
    name = "gri_53_325"
    ns = server_parts[name].n_species
    reqs = [_req(name, n, 1000 + 7 * n, 0) for n in (3000, 5000, 7000)]
    outs = []
    for T, p, Y in reqs:
        n = T.shape[0]
        outs.append({"wdot": torch.empty((ns, n), dtype=torch.float64).pin_memory(),
                     "mu": torch.empty(n, dtype=torch.float64).pin_memory(),
                     "lam": torch.empty(n, dtype=torch.float64).pin_memory(),
                     "Dk": torch.empty((ns, n), dtype=torch.float64).pin_memory()})
    with Server(server_parts, hbm_budget=2 << 30, streams=2) as srv:
        # the middle request keeps the server's staging buffers: one coalesced batch mixes both kinds
        futs = [srv.submit(name, T, p, Y, precision="fp64", transport=True, out=(o if i != 1 else None))
                for i, ((T, p, Y), o) in enumerate(zip(reqs, outs))]
        res = [f.result(timeout=300) for f in futs]
    with Server(server_parts, hbm_budget=2 << 30, streams=1, coalesce=False) as srv:
        ref = [srv.submit(name, T, p, Y, precision="fp64", transport=True).result(timeout=300) for T, p, Y in reqs]
    for i, (a, b) in enumerate(zip(res, ref)):
        for k in ("wdot", "mu", "lam", "Dk"):
            assert np.array_equal(getattr(a, k), getattr(b, k)), (i, k)
    assert np.shares_memory(res[0].wdot, outs[0]["wdot"].numpy())
    with Server(server_parts, hbm_budget=2 << 30) as srv:
        T, p, Y = reqs[0]
        with pytest.raises(ValueError):
            srv.submit(name, T, p, Y, transport=True, out={"wdot": outs[0]["wdot"]})   # transport outputs missing
