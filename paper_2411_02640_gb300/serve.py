"""Continuous-batching server for production-rate / transport requests.

CFD ranks (threads or processes of the host code) submit batches of
thermochemical states of any size for any of several device-resident
mechanisms.  A scheduler thread

  * admits pending requests as stream slots and device memory free up
    (admission is capped by a device-memory budget in bytes);
  * coalesces the admitted requests that share (mechanism, precision,
    transport) into one launch over their concatenated states -- the
    kernels are grid-stride loops sized to the resident capacity of the
    GPU, so a coalesced batch is one persistent launch;
  * runs each batch on one of several CUDA streams (copy in, kernels, copy
    out), so batches of different mechanisms overlap on the device while
    new requests keep arriving;
  * completes a request's Future when its batch's event has fired, and
    records its latency (submit to completion).

The mixed-precision rate kernel and the transport kernels run the same
instruction sequence for a state wherever it lands, so those results are
bit-identical alone and in the mix; the float64-accurate production rates
use the warp-cooperative kernel for batches below the thread-per-state
kernel's resident capacity and the thread-per-state kernel above it, and
the latter evaluates a reaction in float32 when it is negligible for every
state of a warp, so a request's result alone and in the mix agree within
the float64 bar (about 1e-11 of the per-point scale), not bit for bit.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import threading
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from .kx import Mechanism, copy_rows


@dataclass(eq=False)
class Request:
    mech: str
    T: object                     # float64 host tensors: T[n], p[n], Y[N_s, n]
    p: object
    Y: object
    precision: str
    transport: bool
    future: cf.Future
    t_submit: float = 0.0
    t_done: float = 0.0
    out: Optional[Dict[str, object]] = None   # caller-owned host outputs (pinned): wdot, mu, lam, Dk

    @property
    def n(self) -> int:
        return int(self.T.shape[0])


@dataclass
class Result:
    wdot: np.ndarray
    mu: Optional[np.ndarray] = None
    lam: Optional[np.ndarray] = None
    Dk: Optional[np.ndarray] = None
    latency_s: float = 0.0


class _PinnedPool:
    """Pinned host staging buffers reused from batch to batch: allocating
    (and pinning) host memory takes far longer than a copy, so it is done
    once per size class (powers of two, at least 1 MiB) and the buffers are
    handed back when their batch's results have been copied out."""

    def __init__(self, torch):
        self.torch = torch
        self.free: Dict[int, List[object]] = collections.defaultdict(list)
        self.lock = threading.Lock()
        self.allocated = 0

    def get(self, nbytes: int):
        cls = max(1 << 20, 1 << (max(1, int(nbytes)) - 1).bit_length())
        with self.lock:
            if self.free[cls]:
                return self.free[cls].pop()
            self.allocated += cls
        return self.torch.empty(cls, dtype=self.torch.uint8, pin_memory=True)

    def put(self, buf) -> None:
        with self.lock:
            self.free[int(buf.numel())].append(buf)


@dataclass(eq=False)
class _Batch:
    key: tuple
    reqs: List[Request]
    stream: object
    event: object
    nbytes: int
    outs: Dict[str, object] = field(default_factory=dict)
    offsets: List[int] = field(default_factory=list)
    staging: List[object] = field(default_factory=list)   # pooled pinned buffers behind outs


class Server:
    """``Server({"name": Mechanism, ...}, hbm_budget=bytes, streams=4,
    coalesce=True, max_batch_points=2**22)``; ``submit`` returns a
    Future[Result].  With ``coalesce=False`` and ``streams=1`` it serves one
    request at a time (the baseline the batching is compared with)."""

    def __init__(self, mechanisms: Dict[str, Mechanism], hbm_budget: int = 16 << 30, streams: int = 4,
                 coalesce: bool = True, max_batch_points: int = 1 << 22, device: int = 0):
        import torch
        self.torch = torch
        self.mechs = mechanisms
        self.budget = int(hbm_budget)
        self.used = 0
        self.coalesce = coalesce
        self.max_batch = int(max_batch_points)
        self.device = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        self.free_streams = collections.deque(self.streams)
        self.pending: "collections.OrderedDict[tuple, collections.deque]" = collections.OrderedDict()
        self.inflight: List[_Batch] = []
        self.lock = threading.Condition()
        self.running = False
        self.thread: Optional[threading.Thread] = None
        self.latencies: List[float] = []
        self.points_done = 0
        self.launches = 0
        self.error: Optional[BaseException] = None
        self.pool = _PinnedPool(torch)
        # results of requests without their own host buffers are copied out of the pooled staging
        # buffers off the scheduling thread
        self.copier = cf.ThreadPoolExecutor(max_workers=2, thread_name_prefix="kx-serve-copy")

    # ---------------------------------------------------------------- API
    def bytes_per_point(self, name: str, transport: bool) -> int:
        ns = self.mechs[name].n_species
        return 8 * ((2 + ns) + ns + ((2 + ns) if transport else 0))

    def submit(self, name: str, T, p, Y, precision: str = "mixed", transport: bool = False,
               out: Optional[Dict[str, object]] = None) -> cf.Future:
        """Queue one request; ``out`` optionally holds the caller's host
        output tensors (float64, pinned for asynchronous copies): ``wdot``
        [N_s, n] and, with transport, ``mu``, ``lam`` [n] and ``Dk`` [N_s, n];
        the results are copied straight into them and the Result holds views
        of them (a CFD rank reuses its buffers from step to step)."""
        if name not in self.mechs:
            raise KeyError(name)
        if self.error is not None:
            raise RuntimeError(f"serving loop failed: {self.error!r}")
        fut: cf.Future = cf.Future()
        torch = self.torch

        def host(a):
            # numpy arrays (any row stride) or CPU tensors; pinned memory makes the copies asynchronous
            t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.asarray(a, np.float64))
            if t.dtype != torch.float64 or t.is_cuda:
                raise TypeError("requests carry float64 host arrays")
            if t.dim() == 2 and t.stride(1) != 1:
                t = t.contiguous()
            return t
        req = Request(name, host(T), host(p), host(Y), precision, bool(transport), fut, time.perf_counter(), out=out)
        if req.Y.dim() != 2 or req.Y.shape[0] != self.mechs[name].n_species or req.Y.shape[1] != req.n:
            raise ValueError("Y must be [N_s, n]")
        if out is not None:
            ns = self.mechs[name].n_species
            want = {"wdot": (ns, req.n)}
            if transport:
                want.update(mu=(req.n,), lam=(req.n,), Dk=(ns, req.n))
            for k, shp in want.items():
                t = out.get(k)
                if not (isinstance(t, torch.Tensor) and t.dtype == torch.float64 and not t.is_cuda and tuple(t.shape) == shp
                        and t.stride(-1) == 1):
                    raise ValueError(f"out[{k!r}] must be a host float64 tensor of shape {shp} with unit column stride")
        if req.n * self.bytes_per_point(name, transport) > self.budget:
            fut.set_exception(MemoryError(f"request of {req.n} states exceeds the device-memory budget"))
            return fut
        with self.lock:
            self.pending.setdefault((name, precision, bool(transport)), collections.deque()).append(req)
            self.lock.notify()
        return fut

    def start(self) -> "Server":
        self.running = True
        self.thread = threading.Thread(target=self._loop, name="kx-serve", daemon=True)
        self.thread.start()
        return self

    def stop(self, timeout: float = 60.0) -> None:
        with self.lock:
            self.running = False
            self.lock.notify()
        if self.thread:
            self.thread.join(timeout)
        self.copier.shutdown(wait=True)

    def __enter__(self):
        return self.start()

    def __exit__(self, *a):
        self.stop()

    def stats(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return {"requests": len(self.latencies), "points": self.points_done, "launches": self.launches,
                "p50_ms": float(np.quantile(lat, 0.5) * 1e3), "p99_ms": float(np.quantile(lat, 0.99) * 1e3)}

    # ---------------------------------------------------------------- scheduler
    def _loop(self) -> None:
        try:
            self._run()
        except BaseException as exc:            # fail every waiting request instead of hanging it
            with self.lock:
                self.running = False
                waiting = [r for q in self.pending.values() for r in q] + [r for b in self.inflight for r in b.reqs]
                self.pending.clear()
                self.inflight = []
            for r in waiting:
                if not r.future.done():
                    r.future.set_exception(RuntimeError(f"serving loop failed: {exc!r}"))
            self.error = exc

    def _run(self) -> None:
        torch = self.torch
        torch.cuda.set_device(self.device)
        while True:
            with self.lock:
                if not self.running and not self.inflight and not any(self.pending.values()):
                    return
                idle = not self._launch_ready()
            self._complete()
            if idle:
                with self.lock:
                    if self.running and not any(self.pending.values()):
                        self.lock.wait(timeout=0.002 if self.inflight else 0.05)
                if self.inflight:
                    time.sleep(0.0002)

    def _launch_ready(self) -> bool:
        """Admit and launch as many batches as streams and memory allow
        (lock held).  Oldest pending request first."""
        launched = False
        while self.free_streams:
            key = self._oldest_key()
            if key is None:
                break
            q = self.pending[key]
            bpp = self.bytes_per_point(key[0], key[2])
            reqs, pts = [], 0
            while q and (not reqs or self.coalesce):
                r = q[0]
                if reqs and pts + r.n > self.max_batch:
                    break
                if self.used + (pts + r.n) * bpp > self.budget:
                    break
                reqs.append(q.popleft())
                pts += r.n
            if not reqs:
                break                       # the oldest request waits for memory
            try:
                self._launch(key, reqs, pts * bpp)
            except BaseException as exc:
                for r in reqs:              # taken off the queue: fail them here
                    if not r.future.done():
                        r.future.set_exception(RuntimeError(f"serving loop failed: {exc!r}"))
                raise
            launched = True
        return launched

    def _oldest_key(self):
        best, t = None, None
        for k, q in self.pending.items():
            if q and (t is None or q[0].t_submit < t):
                best, t = k, q[0].t_submit
        return best

    def _launch(self, key, reqs: List[Request], nbytes: int) -> None:
        torch = self.torch
        name, prec, transport = key
        mech = self.mechs[name]
        ns = mech.n_species
        stream = self.free_streams.popleft()
        self.used += nbytes
        n = sum(r.n for r in reqs)
        with torch.cuda.stream(stream):
            T = torch.empty(n, dtype=torch.float64, device=self.device)
            p = torch.empty_like(T)
            Y = torch.empty((ns, n), dtype=torch.float64, device=self.device)
            offs, o = [], 0
            for r in reqs:
                offs.append(o)
                T[o:o + r.n].copy_(r.T, non_blocking=True)
                p[o:o + r.n].copy_(r.p, non_blocking=True)
                copy_rows(Y[:, o:o + r.n], r.Y, stream=stream)   # one 2-D copy of the species rows
                o += r.n
            w = mech.production_rates(T, p, Y, precision=prec, stream=stream)

            staging = []

            def down(t):
                buf = self.pool.get(t.numel() * 8)
                staging.append(buf)
                h = buf[:t.numel() * 8].view(torch.float64).view(t.shape)
                h.copy_(t, non_blocking=True)
                return h
            dev = {"wdot": w}
            if transport:
                dev["mu"], dev["lam"], dev["Dk"] = mech.transport(T, p, Y, precision=prec, stream=stream)
            # requests that brought their own host buffers get their outputs copied straight into
            # them (one copy per request and output); the others share pinned staging buffers
            outs = {k: down(t) for k, t in dev.items()} if any(r.out is None for r in reqs) else {}
            for r, o in zip(reqs, offs):
                if r.out is None:
                    continue
                for k, t in dev.items():
                    if t.dim() == 2:
                        copy_rows(r.out[k], t[:, o:o + r.n], stream=stream)
                    else:
                        r.out[k].copy_(t[o:o + r.n], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.launches += 1
        self.inflight.append(_Batch(key, reqs, stream, ev, nbytes, outs, offs, staging))

    def _complete(self) -> None:
        done = []
        with self.lock:
            for b in self.inflight:
                if b.event.query():
                    done.append(b)
            if done:
                ids = {id(b) for b in done}
                self.inflight = [b for b in self.inflight if id(b) not in ids]
            for b in done:
                self.used -= b.nbytes
                self.free_streams.append(b.stream)
            if done:
                self.lock.notify()
        for b in done:
            if b.staging:
                self.copier.submit(self._finish, b)
            else:
                self._finish(b)

    def _finish(self, b: _Batch) -> None:
        """Hand each request of a finished batch its Result: views of its own
        host buffers, or copies out of the pooled staging buffers (which then
        go back to the pool)."""
        for r, o in zip(b.reqs, b.offsets):
            if r.out is not None:
                res = Result(wdot=r.out["wdot"].numpy())
                if r.transport:
                    res.mu, res.lam, res.Dk = (r.out[k].numpy() for k in ("mu", "lam", "Dk"))
            else:
                res = Result(wdot=b.outs["wdot"][:, o:o + r.n].numpy().copy())
                if r.transport:
                    res.mu = b.outs["mu"][o:o + r.n].numpy().copy()
                    res.lam = b.outs["lam"][o:o + r.n].numpy().copy()
                    res.Dk = b.outs["Dk"][:, o:o + r.n].numpy().copy()
            now = time.perf_counter()
            r.t_done = now
            res.latency_s = now - r.t_submit
            with self.lock:
                self.latencies.append(res.latency_s)
                self.points_done += r.n
            r.future.set_result(res)
        for buf in b.staging:
            self.pool.put(buf)
        b.staging = []
        b.outs = {}
