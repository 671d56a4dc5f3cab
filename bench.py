"""Benchmark: production rates + thermo + mixture-averaged transport on the
53-species / 325-reaction synthetic mechanism (30 three-body, 29 Troe),
2^20 states per GPU, float64 path (headline) and mixed path beside it.

One step = kx_production_rates + kx_thermo + kx_transport over the whole
batch (every step of the hot path).  Inputs (T, p, Y: 461 MB) and outputs
are larger than the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl kx|reference]

Under torchrun each rank runs its own 2^20 states (weak scaling, no
collective on the data path); rank 0 prints one JSON line.  --impl
reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MECH = "gri_53_325"
POINTS = 1 << 20
E2E_CHUNK = 1 << 19     # states per chunk of the end-to-end host pipeline (measured: 2^19 19.1-19.6 ms per 2^20-state step, 2^18 19.9)
METRIC = "Mpoints/s wdot+thermo+transport (53sp/325rxn)"
CACHE = os.environ.get("KX_CACHE_DIR", os.path.join(ROOT, ".kxcache"))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {}


SMS = 152
PEAKS_RECORD = os.path.join(ROOT, "profiles", "peaks_gb300.json")


def pipe_rates():
    """Per-clock, per-SM rates of the arithmetic pipes: measured by
    `bench.py --peaks` (kx_probe_pipe) and committed as profiles/peaks_gb300.json;
    the nominal unit counts (2 float64 FMA and 128 float32 lanes per clock per
    SM) where no record exists."""
    try:
        with open(PEAKS_RECORD) as f:
            rec = json.load(f)
        return {"dfma": rec["per_clk_per_sm"]["dfma"], "ffma": rec["per_clk_per_sm"]["ffma"],
                "source": f"measured (kx_probe_pipe, {rec.get('when', '?')}, median SM clock "
                          f"{rec.get('sm_mhz_median', '?')} MHz)"}
    except (OSError, KeyError, ValueError):
        return {"dfma": 2.0, "ffma": 128.0, "source": "nominal unit counts"}


PIPE = pipe_rates()


def fp64_peak_gops(sm_max_mhz: float) -> float:
    """float64 pipe: measured FMA per clock per SM x SMs x the maximum SM clock."""
    return PIPE["dfma"] * SMS * sm_max_mhz * 1e6 / 1e9


def fp32_peak_gops(sm_max_mhz: float) -> float:
    """float32 pipe (and instruction issue): measured FMA lanes per clock per SM x SMs x max clock."""
    return PIPE["ffma"] * SMS * sm_max_mhz * 1e6 / 1e9


def kernel_roofline(mech, name, n, ms, sm_max):
    """Roofline of one kernel against the arithmetic pipe that bounds it:
    the emitter's per-point float64 instructions against the float64 pipe, or
    its float32-pipe instructions (double-float kernels: each float-pair
    primitive at its instruction count) against the float32 pipe, whichever
    takes longer at peak."""
    f64 = ops_per_point(mech, name)
    f32 = mech.op_counts(name)["fp32"]
    p64, p32 = fp64_peak_gops(sm_max), fp32_peak_gops(sm_max)
    if f32 / p32 > f64 / p64:
        ach = f32 * n / (ms * 1e-3) / 1e9
        return {"bound": "alu", "kernel": name, "achieved": ach, "peak": p32, "unit": "G fp32-pipe instr/s",
                "frac": ach / p32, "per_point_instr": f32,
                "peak_source": f"152 SMs x {PIPE['ffma']:.1f} float32 FMA lanes/clk x {sm_max:.0f} MHz (float32 "
                               f"pipe and issue; per-clock rate {PIPE['source']}, max SM clock)"}
    ach = f64 * n / (ms * 1e-3) / 1e9
    return {"bound": "alu", "kernel": name, "achieved": ach, "peak": p64, "unit": "G fp64 instr/s",
            "frac": ach / p64, "per_point_instr": f64,
            "peak_source": f"152 SMs x {PIPE['dfma']:.2f} DFMA/clk x {sm_max:.0f} MHz (float64 pipe; per-clock "
                           f"rate {PIPE['source']}, max SM clock)"}


# float64 instructions that one call of each library routine costs in the
# generated kernels (the library's own exp/log; IEEE division).
COST = {"exp64": 5.0, "log64": 9.0, "div64": 9.0}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    def __init__(self, index: int = 0):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for s in self.samples for j in range(4) if s[3 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def shard(rank: int, n: int):
    """The states of one rank under weak scaling: its own contiguous range
    [rank * n, (rank + 1) * n) of the seeded state stream."""
    return rank * n, n


def max_over_ranks(value: float, dist, device) -> float:
    """The slowest rank's time: one all-reduce (max) of a scalar."""
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def make_inputs(rank: int, n: int):
    from paper_2411_02640_gb300 import synth
    m = synth.mechanism(MECH)
    start, count = shard(rank, n)
    return synth.make_states(m.n_species, synth.STATE_SPECS[MECH], start, count)


def cpu_baseline(seconds_target: float = 15.0):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample."""
    import oracle
    from paper_2411_02640_gb300 import synth
    cores = os.cpu_count() or 1
    o = oracle.Oracle(synth.mechanism_file(MECH, os.path.join(CACHE, "mech")), nthreads=cores)
    n = 256 * cores
    T, p, Y = make_inputs(0, n)
    t0 = time.perf_counter()
    o.production_rates(T, p, Y)
    o.thermo(T, p, Y)
    o.transport(T, p, Y)
    dt = time.perf_counter() - t0
    # scale the sample so that it holds about `seconds_target` of wall time
    n2 = int(min(POINTS, max(n, n * seconds_target / max(dt, 1e-3) / 4)))
    T, p, Y = make_inputs(0, n2)
    t0 = time.perf_counter()
    o.production_rates(T, p, Y)
    o.thermo(T, p, Y)
    o.transport(T, p, Y)
    dt = time.perf_counter() - t0
    # one core, on a sample of about a second
    o1 = oracle.Oracle(synth.mechanism_file(MECH, os.path.join(CACHE, "mech")), nthreads=1)
    n1 = max(64, int(n2 / dt / cores))
    T1, p1, Y1 = make_inputs(0, n1)
    t1 = time.perf_counter()
    o1.production_rates(T1, p1, Y1)
    o1.thermo(T1, p1, Y1)
    o1.transport(T1, p1, Y1)
    dt1 = time.perf_counter() - t1
    return {"value": n2 / dt / 1e6, "unit": "Mpoints/s", "cores": cores, "kind": "oracle",
            "sample": f"{n2} states of the 2^20-state workload, one pass of wdot+thermo+transport",
            "one_core": {"value": n1 / dt1 / 1e6, "sample": f"{n1} states"}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2411_02640_gb300 import synth
    cores = os.cpu_count() or 1
    o = oracle.Oracle(synth.mechanism_file(MECH, os.path.join(CACHE, "mech")), nthreads=cores)
    n = 512 * cores
    T, p, Y = make_inputs(0, n)

    def step():
        o.production_rates(T, p, Y)
        o.thermo(T, p, Y)
        o.transport(T, p, Y)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    v = n / dt / 1e6
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "Mpoints/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{MECH} synthetic mechanism, bounded sample of {n} states per step "
                               f"(the GPU arm runs 2^20 per GPU)", "points_per_step": n},
        "cpu_baseline": {"value": v, "unit": "Mpoints/s", "cores": cores, "kind": "oracle",
                         "sample": f"{n} states per step"},
        "e2e": {"value": v, "unit": "Mpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_kx(args):
    import torch
    import torch.distributed as dist

    from paper_2411_02640_gb300 import kx, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    n = args.points
    path = synth.mechanism_file(MECH, os.path.join(CACHE, "mech"))
    # the kernels of the extra blocks compile in background threads while the main step is timed:
    # compile-only handles (NVRTC, host work with no CUDA call) fill the kernel cache, and the
    # handles are loaded onto the device from it after the timed regions (a load into the context
    # while the end-to-end pipeline runs stalled single steps of it by 30-50 ms)
    import concurrent.futures as cf
    extra = {}
    pool = cf.ThreadPoolExecutor(max_workers=3)
    extra_opts = {"native": (MECH, {"rates_arith": 1, "tr_mode": 1}), "c1": ("h2o2_9_21", {}), "large": ("large_160_900", {})}

    def load_extra(key):
        mname, o = extra_opts[key]
        extra[key].result()
        return kx.Mechanism(synth.mechanism_file(mname, os.path.join(CACHE, "mech")), cache_dir=CACHE, **o)
    if rank == 0 and not args.no_extra:
        def compile_only(mname, o):
            kx.Mechanism(synth.mechanism_file(mname, os.path.join(CACHE, "mech")), cache_dir=CACHE, compile_only=1, **o)
        for key, (mname, o) in extra_opts.items():
            extra[key] = pool.submit(compile_only, mname, o)
    mech = kx.Mechanism(path, cache_dir=CACHE, maxrreg=args.maxrreg, rates_mode=args.rates_mode,
                        rates_arith=args.rates_arith, tr_layout=args.tr_layout, block=args.block,
                        diff_mode=args.diff_mode, rates_layout=args.rates_layout, rates_group=args.rates_group)
    ns = mech.n_species
    T, p, Y = make_inputs(rank, n)
    dev = torch.device("cuda", local)
    Td, pd, Yd = (torch.from_numpy(a).to(dev) for a in (T, p, Y))
    w = torch.empty((ns, n), dtype=torch.float64, device=dev)
    cp = torch.empty(n, dtype=torch.float64, device=dev)
    hm = torch.empty_like(cp)
    mu = torch.empty_like(cp)
    lam = torch.empty_like(cp)
    D = torch.empty((ns, n), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    kernels = {"fp64": ("wdot_fp64", "thermo", "visc_fp64", "diff_fp64"),
               "mixed": ("wdot_mixed", "thermo", "visc_mixed", "diff_mixed")}
    NK = 4

    def step(prec, ev=None):
        if ev: ev[0].record(stream)
        mech.production_rates(Td, pd, Yd, out=w, precision=prec)
        if ev: ev[1].record(stream)
        mech.thermo(Td, pd, Yd, out=(cp, hm))
        if ev: ev[2].record(stream)
        mech.viscosity_conductivity(Td, pd, Yd, out=(mu, lam), precision=prec)
        if ev: ev[3].record(stream)
        mech.diffusion(Td, pd, Yd, out=D, precision=prec)
        if ev: ev[4].record(stream)

    def timed(prec, K, W):
        for _ in range(W):
            step(prec)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(NK + 1)] for _ in range(K)]
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(K):
            step(prec, evs[k])
        t1.record(stream)
        barrier()
        total = t0.elapsed_time(t1)
        per = [sum(e[j].elapsed_time(e[j + 1]) for e in evs) / K for j in range(NK)]
        return total, per

    results = {}
    with ClockSampler(local) as clk:
        for prec in ("fp64", "mixed"):
            total, per = timed(prec, args.steps, args.warmup)
            if world > 1:
                total = max_over_ranks(total, dist, dev)
            results[prec] = (total, per)
    clocks = clk.summary()

    # end to end through the public API from pinned host buffers: kx_evaluate_host copies each
    # chunk's inputs in, runs the four kernels and copies every output back, in chunks over two
    # streams so that the copies overlap the arithmetic
    Th, ph, Yh = (torch.from_numpy(a).pin_memory() for a in (T, p, Y))
    hout = {"wdot": torch.empty((ns, n), dtype=torch.float64).pin_memory(),
            "Dk": torch.empty((ns, n), dtype=torch.float64).pin_memory()}
    for k in ("cp", "h", "mu", "lam"):
        hout[k] = torch.empty(n, dtype=torch.float64).pin_memory()
    chunk = min(n, args.e2e_chunk)
    ws = torch.empty(2 * chunk * mech.evaluate_host_bytes_per_state(7), dtype=torch.uint8, device=dev)
    ss = (torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev))

    def e2e_step():
        for q in ss:
            q.wait_stream(stream)
        mech.evaluate_host(Th, ph, Yh, hout, outputs=7, precision="fp64", workspace=ws, max_chunk=chunk, streams=ss)
        for q in ss:
            stream.wait_stream(q)

    # the background compiles of the extra blocks (NVRTC on many host threads) finish first: the
    # end-to-end loop needs its one host thread to keep the copy and launch queues fed
    for f in extra.values():
        f.result()
    for _ in range(args.warmup + 2):   # two more than the device loop: the first host-link steps run slow
        e2e_step()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps - 1)]
    e0.record(stream)
    for j in range(args.steps):
        e2e_step()
        if j < args.steps - 1:
            marks[j].record(stream)
    e1.record(stream)
    barrier()
    e2e_total = e0.elapsed_time(e1)
    edges = [e0] + marks + [e1]
    e2e_times = [a.elapsed_time(b) for a, b in zip(edges[:-1], edges[1:])]
    e2e_steps = sorted(e2e_times)
    if world > 1:
        e2e_total = max_over_ranks(e2e_total, dist, dev)
    e2e_ms = e2e_total / args.steps
    # the link's plain copy rates, for reading the end-to-end number: one large copy each way
    # between the same pinned outputs / inputs and device memory
    big_h, big_d = hout["wdot"], torch.empty(hout["wdot"].shape, dtype=torch.float64, device=dev)
    for _ in range(2):
        big_d.copy_(big_h, non_blocking=True)
        big_h.copy_(big_d, non_blocking=True)
    e0.record(stream); big_d.copy_(big_h, non_blocking=True); e1.record(stream)
    e1.synchronize()
    h2d_gbs = big_h.numel() * 8 / (e0.elapsed_time(e1) * 1e-3) / 1e9
    e0.record(stream); big_h.copy_(big_d, non_blocking=True); e1.record(stream)
    e1.synchronize()
    d2h_gbs = big_h.numel() * 8 / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del big_d

    if rank == 0:
        pk = peaks()
        total, per = results["fp64"]
        ms = total / args.steps
        value = world * n / (ms * 1e-3) / 1e6
        mtotal, mper = results["mixed"]
        mms = mtotal / args.steps
        # roofline of the dominant kernel of each path against its arithmetic pipe
        names = kernels["fp64"]
        dom = int(np.argmax(per))
        sm_max = float(pk.get("sm_max_mhz", 2070.0))
        roof = kernel_roofline(mech, names[dom], n, per[dom], sm_max)
        hbm = float(pk.get("hbm_gbs", 6787.2))

        def step_bound(knames, ms_each):
            """t_bound of the step: per kernel the slowest of its float64 instructions at the
            float64 peak, its float32-pipe instructions at the float32 peak and its algorithmic
            bytes at the measured HBM copy rate; summed over the kernels of the step."""
            tb, parts = 0.0, {}
            byt = {"wdot": 8 * (2 + 2 * ns), "thermo": 8 * (2 + ns + 2), "visc": 8 * (2 + ns + 2),
                   "diff": 8 * (2 + 2 * ns)}
            for kname, ms_k in zip(knames, ms_each):
                c = mech.op_counts(kname)
                t64 = ops_per_point(mech, kname) * n / (fp64_peak_gops(sm_max) * 1e9)
                t32 = c["fp32"] * n / (fp32_peak_gops(sm_max) * 1e9)
                tm = byt[kname.split("_")[0]] * n / (hbm * 1e9)
                t = max(t64, t32, tm)
                tb += t
                parts[kname] = {"t_bound_ms": t * 1e3, "measured_ms": ms_k,
                                "bound": "fp64" if t == t64 else "fp32" if t == t32 else "hbm"}
            return tb * 1e3, parts

        roof["traffic"] = profiled_traffic(mech, names[dom], n)
        roof["algorithmic_bytes"] = 8 * (2 + ns + ns) * n
        mnames = kernels["mixed"]
        mdom = int(np.argmax(mper))
        line = {
            "metric": METRIC, "value": value, "unit": "Mpoints/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32x2" if args.rates_arith != 1 else "f64+f32x2", "data": "synthetic",
            "precision": "float64-accurate: float-pair (double-float, ~2^-47 per operation) arithmetic on the float32 "
                         "pipe" + (" (production rates native float64)" if args.rates_arith == 1 else "") +
                         "; against the FP64 oracle wdot <= 1e-10 of the per-point scale, thermo and transport "
                         "<= 1e-12 relative",
            "config": {"workload": f"{MECH}: synthetic 53 species / 325 reactions (30 three-body, 29 Troe), "
                                   f"2^20 states per GPU, T U[300,2800] K, p log-U[0.5,40] atm, Y Dirichlet(0.2)",
                       "points_per_gpu": n, "step": "production_rates + thermo + transport (viscosity/conductivity and diffusion)",
                       "l2": "inputs (461 MB) and outputs larger than L2; no flush"},
            "kernel_ms": {k: v for k, v in zip(names, per)},
            "grxn_s": value * 1e6 * mech.n_reactions / 1e9,
            "gdof_s": value * 1e6 * (ns + 2) / 1e9,
            "mixed": {"value": world * n / (mms * 1e-3) / 1e6, "unit": "Mpoints/s", "ms_per_step": mms,
                      "kernel_ms": {k: v for k, v in zip(mnames, mper)},
                      "dtype": "f32 + f32x2 (Gibbs sums) + f64 (wdot accumulation)",
                      "error": "wdot <= 2e-4 of the per-point scale max_k|W_k wdot_k| (p99 <= 1e-4); "
                               "transport <= 5e-6 relative; thermo float64-accurate",
                      "roofline": kernel_roofline(mech, mnames[mdom], n, mper[mdom], sm_max),
                      "step_roofline": (lambda tb: {"t_bound_ms": tb[0], "measured_ms": mms, "frac": tb[0] / mms,
                                                    "kernels": tb[1]})(step_bound(mnames, mper))},
            "roofline": roof,
            "step_roofline": (lambda tb: {"t_bound_ms": tb[0], "measured_ms": ms, "frac": tb[0] / ms, "kernels": tb[1],
                                          "definition": "per kernel max(float64 instr / float64 peak, float32-pipe "
                                                        "instr / float32 peak, algorithmic bytes / measured HBM), "
                                                        "summed over the step"})(step_bound(names, per)),
            "e2e": {"value": world * n / (e2e_ms * 1e-3) / 1e6, "unit": "Mpoints/s", "api": "kx_evaluate_host",
                    "chunk": chunk,
                    "step_ms": {"min": e2e_steps[0], "median": e2e_steps[len(e2e_steps) // 2], "max": e2e_steps[-1],
                                "slowest_step": e2e_times.index(e2e_steps[-1])},
                    "h2d_bytes_per_step": 8 * (2 + ns) * n, "d2h_bytes_per_step": 8 * (2 * ns + 4) * n,
                    "link_gbs": {"h2d": h2d_gbs, "d2h": d2h_gbs,
                                 "note": "one pinned copy of the production-rate array each way"}},
            "gpu_launches": NK * args.steps,
            "clocks": clocks,
        }
        if extra:
            # the plain float64 GPU form of the same step: native float64 production rates
            # (rates_arith 1, fully unrolled) and native float64 transport (tr_mode 1); thermo has
            # only its double-float kernel
            nat = load_extra("native")
            nb = step_block(nat, MECH, n, dev, stream, args.steps, args.warmup, "fp64", sm_max, Td, pd, Yd)
            nb["dtype"] = "f64 (thermo f32x2)"
            nb["roofline"] = kernel_roofline(nat, "wdot_fp64", n, nb["kernel_ms"]["wdot_fp64"], sm_max)
            nb["speedup_of_float_pair_step"] = nb["ms_per_step"] / ms
            nb["speedup_of_mixed_step"] = nb["ms_per_step"] / mms
            line["fp64_native"] = nb
            c1 = load_extra("c1")
            cb = {"workload": "h2o2_9_21: synthetic 9 species / 21 reactions (4 three-body, 2 Troe), 4096 states, "
                              "T U[300,2500] K, p = 1 atm, Y Dirichlet(0.5); all outputs"}
            for prec in ("fp64", "mixed"):
                cb[prec] = step_block(c1, "h2o2_9_21", 4096, dev, stream, max(args.steps, 50), args.warmup, prec, sm_max)
            line["c1_h2o2_9_21_4096"] = cb
            line["large_160_900"] = large_block(load_extra("large"), dev, stream, args.steps, args.warmup, sm_max)
            line["adjoint"] = adjoint_block(mech, Td, pd, Yd, stream, args.warmup)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        if world == 1 and not args.no_serve:
            srv = run_serve_suite(args, sweep=False)
            kb = srv["knee"]["batching"]
            line["serving"] = {"p50_ms": kb["p50_ms"], "p99_ms": kb["p99_ms"], "mpoints_s": kb["mpoints_s"],
                               "rate_req_s": kb["rate_req_s"], "saturated_mpoints_s": kb["saturated_mpoints_s"],
                               "knee": "highest Poisson rate (of 32, 128, 512 req/s; 128 requests each) whose "
                                       "achieved throughput is >= 90 % of the offered load",
                               "one_at_a_time": srv["knee"]["one_at_a_time"],
                               "rates": [{k: x[k] for k in ("rate_req_s", "offered_mpoints_s", "mpoints_s", "p50_ms",
                                                             "p99_ms")} for x in srv["batching"]],
                               "workload": "Poisson arrivals, 1e3-2e6 states per request, mechanisms 9/21, 53/325, "
                                           "160/900; 70% mixed, 20% with transport; host (pinned) in and out"}
        print(json.dumps(line), flush=True)
    pool.shutdown(wait=True)
    if world > 1:
        dist.destroy_process_group()


SERVE_MECHS = ("h2o2_9_21", "gri_53_325", "large_160_900")


def serve_pools(points: int):
    """Per mechanism a pool of seeded states (2^20 drawn, tiled to 2x) that
    requests slice; pinned host memory, as CFD ranks would hand over."""
    import torch
    from paper_2411_02640_gb300 import synth
    pools = {}
    for name in SERVE_MECHS:
        m = synth.mechanism(name)
        T, p, Y = synth.make_states(m.n_species, synth.STATE_SPECS[name], 0, points)
        pools[name] = tuple(torch.from_numpy(np.concatenate([a, a], axis=-1)).pin_memory() for a in (T, p, Y))
    return pools


def serve_outputs(mechs):
    """One set of pinned host result buffers, sized for the largest request of
    the largest mechanism, that every request of a sweep writes into (views of
    its leading columns).  Overlapping requests write the same memory: the
    sweep measures throughput and latency only; the identity of each result
    alone and in the mix is checked by the GPU tests."""
    import torch
    ns = max(m.n_species for m in mechs.values())
    nmax = SERVE_MAX_STATES
    return {"wdot": torch.empty((ns, nmax), dtype=torch.float64).pin_memory(),
            "Dk": torch.empty((ns, nmax), dtype=torch.float64).pin_memory(),
            "mu": torch.empty(nmax, dtype=torch.float64).pin_memory(),
            "lam": torch.empty(nmax, dtype=torch.float64).pin_memory()}


SERVE_MAX_STATES = 2_000_000


def serve_run(mechs, pools, outbuf, rate: float, count: int, seed: int, coalesce: bool, streams: int, budget: int):
    """Poisson arrivals at `rate` requests/s; sizes log-uniform 1e3..2e6 states;
    mechanism uniform over the three; 70 % mixed / 30 % float64; 20 % also
    transport.  Returns achieved throughput (all states over the time from the
    first submission to the last completion), offered throughput and latency
    statistics."""
    from paper_2411_02640_gb300.serve import Server
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(count):
        name = SERVE_MECHS[rng.integers(len(SERVE_MECHS))]
        n = int(np.exp(rng.uniform(np.log(1e3), np.log(SERVE_MAX_STATES))))
        off = int(rng.integers(0, pools[name][0].shape[0] - n))
        reqs.append((name, off, n, "mixed" if rng.random() < 0.7 else "fp64", bool(rng.random() < 0.2)))
    gaps = rng.exponential(1.0 / rate, count)
    srv = Server(mechs, hbm_budget=budget, streams=streams, coalesce=coalesce).start()
    futs = []
    t0 = time.perf_counter()
    t_next = t0
    for (name, off, n, prec, tr), gap in zip(reqs, gaps):
        t_next += gap
        d = t_next - time.perf_counter()
        if d > 0:
            time.sleep(d)
        T, p, Y = pools[name]
        ns = mechs[name].n_species
        o = {"wdot": outbuf["wdot"][:ns, :n]}
        if tr:
            o.update(mu=outbuf["mu"][:n], lam=outbuf["lam"][:n], Dk=outbuf["Dk"][:ns, :n])
        futs.append(srv.submit(name, T[off:off + n], p[off:off + n], Y[:, off:off + n], precision=prec, transport=tr,
                               out=o))
    t_sub = time.perf_counter() - t0
    for f in futs:
        f.result(timeout=600)
    t1 = time.perf_counter()
    srv.stop()
    st = srv.stats()
    pts = sum(r[2] for r in reqs)
    return {"rate_req_s": rate, "requests": count, "mpoints_s": pts / (t1 - t0) / 1e6,
            "offered_mpoints_s": pts / max(t_sub, 1e-9) / 1e6, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "launches": st["launches"], "coalesce": coalesce, "streams": streams}


def run_serve_suite(args, sweep=True):
    """Serving at a range of Poisson request rates, continuous batching (4
    streams, coalescing) against one request at a time; the knee is the
    highest rate whose achieved throughput keeps up with the offered load (at
    least 90 % of it), reported with its p50/p99 latency."""
    import torch
    from paper_2411_02640_gb300 import kx, synth
    torch.cuda.set_device(0)
    mechs = {n: kx.Mechanism(synth.mechanism_file(n, os.path.join(CACHE, "mech")), cache_dir=CACHE)
             for n in SERVE_MECHS}
    pools = serve_pools(1 << 20)
    outbuf = serve_outputs(mechs)
    budget = 48 << 30
    # warm every kernel once
    for name, m in mechs.items():
        T, p, Y = (a[..., :4096].contiguous().cuda() for a in pools[name])
        for prec in ("fp64", "mixed"):
            m.production_rates(T, p, Y, precision=prec)
            m.transport(T, p, Y, precision=prec)
    torch.cuda.synchronize()
    rates = [16.0, 64.0, 128.0, 256.0, 512.0, 1024.0] if sweep else [32.0, 128.0, 512.0]
    out = {"budget_bytes": budget, "mechanisms": list(SERVE_MECHS), "batching": [], "one_at_a_time": []}
    for r in rates:
        count = int(min(512, max(64, 2.0 * r))) if sweep else 128
        out["batching"].append(serve_run(mechs, pools, outbuf, r, count, 105, True, 4, budget))
        out["one_at_a_time"].append(serve_run(mechs, pools, outbuf, r, count, 105, False, 1, budget))

    def knee(rows):
        ok = [x for x in rows if x["mpoints_s"] >= 0.9 * x["offered_mpoints_s"]]
        best = max(ok, key=lambda x: x["rate_req_s"]) if ok else min(rows, key=lambda x: x["rate_req_s"])
        return {"rate_req_s": best["rate_req_s"], "mpoints_s": best["mpoints_s"], "p50_ms": best["p50_ms"],
                "p99_ms": best["p99_ms"], "saturated_mpoints_s": max(x["mpoints_s"] for x in rows)}
    out["knee"] = {"batching": knee(out["batching"]), "one_at_a_time": knee(out["one_at_a_time"])}
    return out


def profiled_traffic(mech, name, n):
    """DRAM bytes of one launch from the committed ncu capture of this exact
    kernel (matched by the hash of its emitted source), scaled to n states;
    None when no capture of the current kernel exists."""
    import glob
    for path in glob.glob(os.path.join(ROOT, "profiles", f"traffic_{name}_*.json")):
        with open(path) as f:
            d = json.load(f)
        if d.get("mechanism") == MECH and d.get("source_hash") == mech.source_hash(name):
            return d["bytes_per_state"] * n
    return None


def ops_per_point(mech, name):
    """float64 instructions per point of a kernel: the emitter's count of plain
    float64 operations plus each library routine at its instruction cost."""
    c = mech.op_counts(name)
    return c["fp64"] + COST["exp64"] * c["exp64"] + COST["log64"] * c["log64"] + COST["div64"] * c["div64"]


def run_alternatives(args):
    """Times kx_production_rates on the bench workload in each of its forms: the float-pair
    default, native float64 with k_r in log space (kc_mode 0) and native float64 with the
    paper's per-species exp(-G/RT) products and one division per reaction (kc_mode 1), and the
    mixed kernel; prints one JSON line with times and the emitter's operation counts."""
    import torch
    from paper_2411_02640_gb300 import kx, synth
    torch.cuda.set_device(0)
    n = args.points
    path = synth.mechanism_file(MECH, os.path.join(CACHE, "mech"))
    T, p, Y = make_inputs(0, n)
    Td, pd, Yd = (torch.from_numpy(a).cuda() for a in (T, p, Y))
    forms = {"fp64_float_pair": ({}, "fp64"), "fp64_native_logspace": ({"rates_arith": 1, "kc_mode": 0}, "fp64"),
             "fp64_native_g3": ({"rates_arith": 1, "kc_mode": 1}, "fp64"), "mixed": ({}, "mixed")}
    out = {}
    for label, (opts, prec) in forms.items():
        mech = kx.Mechanism(path, cache_dir=CACHE, lazy=1, **opts)
        kname = "wdot_fp64" if prec == "fp64" else "wdot_mixed"
        w = mech.production_rates(Td, pd, Yd, precision=prec)
        for _ in range(args.warmup):
            mech.production_rates(Td, pd, Yd, out=w, precision=prec)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            mech.production_rates(Td, pd, Yd, out=w, precision=prec)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        out[label] = {"ms": ms, "mpoints_s": n / (ms * 1e-3) / 1e6, "op_counts": mech.op_counts(kname),
                      "registers": mech.kernel_info(kname)["registers"]}
    # transport with the ln fits and with the paper's direct fits (no exponentials)
    tr = {}
    for mname in (MECH, MECH + "_direct"):
        mech = kx.Mechanism(synth.mechanism_file(mname, os.path.join(CACHE, "mech")), cache_dir=CACHE)
        for prec in ("fp64", "mixed"):
            res = mech.transport(Td, pd, Yd, precision=prec)
            for _ in range(args.warmup):
                mech.transport(Td, pd, Yd, out=res, precision=prec)
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            tv = td = 0.0
            for _ in range(args.steps):
                ev[0].record()
                mech.viscosity_conductivity(Td, pd, Yd, out=res[:2], precision=prec)
                ev[1].record()
                mech.diffusion(Td, pd, Yd, out=res[2], precision=prec)
                ev[2].record()
                torch.cuda.synchronize()
                tv += ev[0].elapsed_time(ev[1]); td += ev[1].elapsed_time(ev[2])
            tr[f"{mname}/{prec}"] = {"visc_ms": tv / args.steps, "diff_ms": td / args.steps}
    print(json.dumps({"metric": "production-rate kernel forms", "points": n, "mechanism": MECH, "forms": out,
                      "transport_fits": tr}), flush=True)


def run_peaks(args):
    """Measured per-clock rates of the arithmetic pipes (kx_probe_pipe): float64
    FMA, float32 FMA, the special-function unit's float32 2^x, and CUDA's own
    float64 exp, log and division per call.  Each probe is calibrated to about
    a quarter of a second per launch, timed with CUDA events on its stream
    (best of three after a warm-up) while nvidia-smi samples the SM clock; the
    per-clock rate divides by the median sampled clock.  --write-peaks stores
    the record that the roofline of the default line reads."""
    import torch
    from paper_2411_02640_gb300 import kx
    torch.cuda.set_device(0)
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    blocks, threads = sms * 8, 256
    sink = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    with ClockSampler(0) as clk:
        for op in kx.PROBE_OPS:
            it = 64
            while True:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                nops = kx.probe_pipe(op, it, blocks, threads, sink, stream)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                if ms > 20.0 or it > (1 << 30):
                    break
                it *= 4
            it = max(1, int(it * 250.0 / ms))
            kx.probe_pipe(op, it, blocks, threads, sink, stream)   # warm-up at the final size
            best = None
            for _ in range(3):
                e0.record(stream)
                nops = kx.probe_pipe(op, it, blocks, threads, sink, stream)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            res[op] = {"ops_per_s": nops / (best * 1e-3), "ms": best, "iters": it}
    clocks = clk.summary()
    mhz = clocks.get("sm_mhz") or 2070.0
    per_clk = {op: r["ops_per_s"] / (mhz * 1e6 * sms) for op, r in res.items()}
    rec = {"metric": "arithmetic pipe rates", "gpu": props.name, "sms": sms, "launch": f"{blocks} x {threads}",
           "sm_mhz_median": mhz, "clocks": clocks, "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
           "ops_per_s": {op: r["ops_per_s"] for op, r in res.items()}, "per_clk_per_sm": per_clk,
           "ms": {op: r["ms"] for op, r in res.items()},
           "float64_cost_in_dfma": {op: per_clk["dfma"] / per_clk[op] for op in ("exp64", "log64", "div64")},
           "note": "eight independent chains per thread; exp64/log64/div64 are per call of CUDA's float64 "
                   "routines (log and division chains include one add each)"}
    if args.write_peaks:
        with open(PEAKS_RECORD, "w") as f:
            json.dump(rec, f, indent=1)
    print(json.dumps(rec), flush=True)


def time_calls(fn, K, W, stream):
    """Mean milliseconds of fn() over K calls after W warm-ups, CUDA events on `stream`."""
    import torch
    for _ in range(W):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / K


def step_block(mech, name, n, dev, stream, K, W, prec, sm_max, T=None, p=None, Y=None):
    """Mpoints/s of the whole step (production rates, thermo, viscosity and
    conductivity, diffusion) of one mechanism at n states, with per-kernel
    times and the roofline of the dominant kernel."""
    import torch
    from paper_2411_02640_gb300 import synth
    ns = mech.n_species
    if T is None:
        T, p, Y = (torch.from_numpy(a).to(dev) for a in synth.make_states(ns, synth.STATE_SPECS[name], 0, n))
    w = torch.empty((ns, n), dtype=torch.float64, device=dev)
    cp, hm, mu, lam = (torch.empty(n, dtype=torch.float64, device=dev) for _ in range(4))
    D = torch.empty((ns, n), dtype=torch.float64, device=dev)
    calls = [lambda: mech.production_rates(T, p, Y, out=w, precision=prec),
             lambda: mech.thermo(T, p, Y, out=(cp, hm)),
             lambda: mech.viscosity_conductivity(T, p, Y, out=(mu, lam), precision=prec),
             lambda: mech.diffusion(T, p, Y, out=D, precision=prec)]
    kms = [time_calls(c, K, W, stream) for c in calls]
    total = time_calls(lambda: [c() for c in calls], K, W, stream)
    knames = ("wdot_" + prec, "thermo", "visc_" + prec, "diff_" + prec)
    dom = int(np.argmax(kms))
    return {"value": n / (total * 1e-3) / 1e6, "unit": "Mpoints/s", "ms_per_step": total, "points": n,
            "kernel_ms": dict(zip(knames, kms)),
            "grxn_s": n / (total * 1e-3) * mech.n_reactions / 1e9, "gdof_s": n / (total * 1e-3) * (ns + 2) / 1e9,
            "roofline": kernel_roofline(mech, knames[dom], n, kms[dom], sm_max)}


def run_sweep(args):
    """Point-count sweep (2^10 .. 2^22 states) of the whole step on the 9/21 and
    53/325 mechanisms, float64-accurate and mixed: Mpoints/s, GRXN/s and GDOF/s."""
    import torch
    from paper_2411_02640_gb300 import kx, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    sm_max = float(peaks().get("sm_max_mhz", 2070.0))
    out = {"metric": "point-count sweep", "rows": []}
    for name in ("h2o2_9_21", MECH):
        mech = kx.Mechanism(synth.mechanism_file(name, os.path.join(CACHE, "mech")), cache_dir=CACHE)
        big = synth.make_states_torch(mech.n_species, synth.STATE_SPECS[name], 1 << 22, seed=synth.STATE_SPECS[name].seed)
        for lg in range(10, 23, 2):
            n = 1 << lg
            T, p, Y = big[0][:n], big[1][:n], big[2][:, :n].contiguous()
            K = max(3, min(200, int(2e6 / n)))
            for prec in ("fp64", "mixed"):
                b = step_block(mech, name, n, dev, stream, K, 3, prec, sm_max, T, p, Y)
                out["rows"].append({"mechanism": name, "points": n, "precision": prec, "mpoints_s": b["value"],
                                    "grxn_s": b["grxn_s"], "gdof_s": b["gdof_s"], "ms_per_step": b["ms_per_step"],
                                    "kernel_ms": b["kernel_ms"]})
        del big
    print(json.dumps(out), flush=True)


def run_sweep_adjoint(args):
    """Batch-size sweep of the adjoint (one call of kx_production_rates_vjp,
    N(0,1) cotangents) on 9/21, 53/325 (2^8 .. 2^18 states) and 160/900
    (2^8 .. 2^16): one thread per state (vjp_layout 1), one warp per state
    (vjp_layout 2) and the default choice between them."""
    import torch
    from paper_2411_02640_gb300 import kx, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    out = {"metric": "adjoint batch-size sweep", "unit": "ms per call", "rows": []}
    for name, lmax in (("h2o2_9_21", 18), (MECH, 18), ("large_160_900", 16)):
        path = synth.mechanism_file(name, os.path.join(CACHE, "mech"))
        forms = {"tps": kx.Mechanism(path, cache_dir=CACHE, lazy=1, vjp_layout=1),
                 "wc": kx.Mechanism(path, cache_dir=CACHE, lazy=1, vjp_layout=2),
                 "default": kx.Mechanism(path, cache_dir=CACHE, lazy=1)}
        ns = forms["tps"].n_species
        spec = synth.STATE_SPECS[name]
        T, p, Y = synth.make_states_torch(ns, spec, 1 << lmax, seed=spec.seed)
        v = torch.randn((ns, 1 << lmax), dtype=torch.float64, device="cuda",
                        generator=torch.Generator("cuda").manual_seed(1))
        for lg in range(8, lmax + 1):
            n = 1 << lg
            a = (T[:n], p[:n], Y[:, :n].contiguous(), v[:, :n].contiguous())
            row = {"mechanism": name, "points": n}
            for key, m in forms.items():
                g = m.production_rates_vjp(*a)
                row[key + "_ms"] = time_calls(lambda: m.production_rates_vjp(*a, out=g), max(3, min(200, (1 << 20) // n)),
                                              3, stream)
            row["default_mpoints_s"] = n / (row["default_ms"] * 1e-3) / 1e6
            out["rows"].append(row)
        del T, p, Y, v
    print(json.dumps(out), flush=True)


def adjoint_block(mech, T, p, Y, stream, W):
    """The adjoint v^T d wdot/d(T, Y) of the bench mechanism (kx_production_rates_vjp, N(0,1)
    cotangents) on the first 2^18 and 4096 of the bench states: Mpoints/s of one call, the
    library's choice of kernel by batch size."""
    import torch
    out = {"workload": f"{MECH}: the first n of the bench states, cotangents N(0,1) (seeded)"}
    for n, key, K in ((1 << 18, "n_262144", 10), (4096, "n_4096", 200)):
        a = (T[:n], p[:n], Y[:, :n].contiguous(),
             torch.randn((mech.n_species, n), dtype=torch.float64, device=T.device,
                         generator=torch.Generator(T.device).manual_seed(1)))
        g = mech.production_rates_vjp(*a)
        ms = time_calls(lambda: mech.production_rates_vjp(*a, out=g), K, max(W, 3), stream)
        out[key] = {"ms": ms, "mpoints_s": n / (ms * 1e-3) / 1e6}
    return out


def large_block(mech, dev, stream, K, W, sm_max, n=1 << 22, name="large_160_900"):
    """Production rates of the 160/900 mechanism at 2^22 states (states drawn on
    the device with torch's seeded generator): float64-accurate and mixed
    Mpoints/s, the kernels' rooflines and the mixed path's error against the
    float64-accurate path over every state."""
    import torch
    from paper_2411_02640_gb300 import synth
    spec = synth.STATE_SPECS[name]
    T, p, Y = synth.make_states_torch(mech.n_species, spec, n, seed=spec.seed)
    w64 = torch.empty((mech.n_species, n), dtype=torch.float64, device=dev)
    w32 = torch.empty_like(w64)
    out = {"workload": f"{name}: synthetic 160 species / 900 reactions (72 three-body, 54 Troe), {n} states "
                       "drawn on the device, T U[500,2800] K, p log-U[1,60] atm, Y Dirichlet(0.2)", "points": n}
    for prec, w in (("fp64", w64), ("mixed", w32)):
        ms = time_calls(lambda: mech.production_rates(T, p, Y, out=w, precision=prec), K, W, stream)
        out[prec] = {"mpoints_s": n / (ms * 1e-3) / 1e6, "ms": ms,
                     "grxn_s": n / (ms * 1e-3) * mech.n_reactions / 1e9,
                     "roofline": kernel_roofline(mech, "wdot_" + prec, n, ms, sm_max)}
    Wt = torch.tensor(mech.W, dtype=torch.float64, device=dev)[:, None]
    e = ((Wt * (w32 - w64).abs()).amax(dim=0) / (Wt * w64.abs()).amax(dim=0)).cpu().numpy()
    out["mixed"]["error_vs_fp64_gpu"] = {"max": float(e.max()), "p99": float(np.quantile(e, 0.99)),
                                         "measure": "per state max_k W_k |dwdot_k| / max_k W_k |wdot_k|"}
    return out


def run_profile_rates(args):
    """A short driver for ncu captures of one production-rate kernel: loads
    --mech with the given layout options, draws --points states on the
    device and calls kx_production_rates twice (capture the second launch
    with -s 1 -c 1)."""
    import torch
    from paper_2411_02640_gb300 import kx, synth
    torch.cuda.set_device(0)
    spec = synth.STATE_SPECS[args.mech]
    opts = dict(rates_layout=args.rates_layout, rates_group=args.rates_group, maxrreg=args.maxrreg,
                rates_arith=args.rates_arith, block=args.block, vjp_layout=args.vjp_layout, lazy=1)
    m = kx.Mechanism(synth.mechanism_file(args.mech, os.path.join(CACHE, "mech")), cache_dir=CACHE, **opts)
    T, p, Y = synth.make_states_torch(m.n_species, spec, args.points, seed=spec.seed)
    if args.profile_call == "vjp":
        v = torch.randn((m.n_species, args.points), dtype=torch.float64, device="cuda",
                        generator=torch.Generator("cuda").manual_seed(1))
        gT, w = m.production_rates_vjp(T, p, Y, v)
        m.production_rates_vjp(T, p, Y, v, out=(gT, w))
    else:
        w = m.production_rates(T, p, Y, precision=args.precision)
        m.production_rates(T, p, Y, out=w, precision=args.precision)
    torch.cuda.synchronize()
    print(json.dumps({"profile_rates": args.mech, "call": args.profile_call, "points": args.points, "options": opts,
                      "precision": args.precision, "finite": bool(torch.isfinite(w).all())}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kx", choices=["kx", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--points", type=int, default=POINTS, help="states per GPU (profiling of smaller cases)")
    ap.add_argument("--maxrreg", type=int, default=0, help="register cap for the generated kernels (0: compiler)")
    ap.add_argument("--rates-mode", type=int, default=0, help="0 automatic, 1 unrolled, 2 table-driven rate kernels")
    ap.add_argument("--e2e-chunk", type=int, default=E2E_CHUNK, help="states per chunk of the end-to-end pipeline")
    ap.add_argument("--block", type=int, default=0, help="threads per block of the generated kernels (0: 128)")
    ap.add_argument("--diff-mode", type=int, default=0, help="transport pairs: 0/1 symmetric (default), 2 full matrices")
    ap.add_argument("--tr-layout", type=int, default=0, help="transport species vectors: 1 shared, 2 X local, 3 (default) all local")
    ap.add_argument("--rates-arith", type=int, default=0,
                    help="float64-accurate rates: 0 double-float (default), 1 native float64")
    ap.add_argument("--serve", action="store_true", help="serving sweep (rates x batching vs one at a time) only")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving sample in the default line")
    ap.add_argument("--alternatives", action="store_true",
                    help="time the production-rate kernel in each arithmetic / equilibrium form only")
    ap.add_argument("--peaks", action="store_true", help="measure the arithmetic pipes' per-clock rates only")
    ap.add_argument("--write-peaks", action="store_true", help="with --peaks: store the record the roofline reads")
    ap.add_argument("--sweep", action="store_true", help="point-count sweep of the step on 9/21 and 53/325 only")
    ap.add_argument("--sweep-adjoint", action="store_true", help="batch-size sweep of the adjoint's two kernels only")
    ap.add_argument("--profile-rates", action="store_true",
                    help="two production-rate calls on --mech at --points states (a driver for ncu captures)")
    ap.add_argument("--mech", default=MECH, help="mechanism of --profile-rates")
    ap.add_argument("--profile-call", default="rates", choices=["rates", "vjp"],
                    help="--profile-rates: production rates or their adjoint (random N(0,1) cotangents)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"], help="precision of --profile-rates")
    ap.add_argument("--rates-layout", type=int, default=0,
                    help="float-pair rates: 0 by batch size, 1 thread per state, 2 warp-cooperative")
    ap.add_argument("--rates-group", type=int, default=0, help="warp-cooperative rates: states per warp (0: one)")
    ap.add_argument("--vjp-layout", type=int, default=0,
                    help="adjoint of --profile-call vjp: 0 by batch size, 1 thread per state, 2 warp-cooperative")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the native float64, 9/21 (4096 states) and 160/900 blocks of the default line")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.alternatives:
        run_alternatives(args)
    elif args.peaks:
        run_peaks(args)
    elif args.profile_rates:
        run_profile_rates(args)
    elif args.sweep:
        run_sweep(args)
    elif args.sweep_adjoint:
        run_sweep_adjoint(args)
    elif args.serve:
        print(json.dumps({"metric": "serving", "serving": run_serve_suite(args, sweep=True)}), flush=True)
    else:
        run_kx(args)


if __name__ == "__main__":
    main()
