"""Throughput benchmark: a brick random circuit on one GPU per process.

Default workload (the precision + fusion configuration): the 30-qubit brick
random circuit of depth 40 (U3 on every qubit, then CNOT(i, i+1) on
alternating pairs; the QSB structure of §IV-F), seed 6, complex64 state
(8 GiB) fused into dense 6-qubit blocks on the tensor cores (tcgen05, FP16
hi/lo split products).  The same circuit in complex128 (16 GiB) runs beside
it, fused into 5-qubit blocks on the tensor cores (FP64 operands split into
9-bit integer digits, exact digit products), and both are reported, with
their infidelity measured on the GPU; the other plans of each dtype (tiles,
4- and 5-qubit blocks) are timed as extras.

Metric (§IV-F, Eq. 5 traffic model): effective HBM bandwidth
    2 * 2^n * bytes_per_amplitude * #gates / time
(every logical gate counted as one read + write of the whole vector), and
logical gates per second.  `value` is the whole-job effective GB/s of the
headline dtype (summed over ranks; one independent replica per GPU).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload brick30|brick28|brick26|qft28] [--dtype c64|c128]
                  [--mode auto|fused|tiled|unfused] [--fuse-qubits K]

`--impl reference` times the FP64 CPU oracle (a deliberately plain program)
on the host cores, on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

WORKLOADS = {
    "brick30": dict(n=30, make=lambda: W.brick(30, 40, 6), desc="30-qubit brick random circuit, depth 40, seed 6"),
    "brick28": dict(n=28, make=lambda: W.brick(28, 40, 3), desc="28-qubit brick random circuit, depth 40, seed 3"),
    "qft28": dict(n=28, make=lambda: W.qft(28), desc="28-qubit QFT"),
    "brick26": dict(n=26, make=lambda: W.brick(26, 40, 6), desc="26-qubit brick random circuit, depth 40, seed 6"),
    "brick20": dict(n=20, make=lambda: W.brick(20, 40, 6), desc="20-qubit brick random circuit, depth 40, seed 6"),
    "brick33": dict(n=33, make=lambda: W.brick(33, 20, 7), desc="33-qubit brick random circuit, depth 20, seed 7"),
}

# DRAM bytes (read + write) per launch from one ncu capture on the 26-qubit
# workload (profiles/); per launch traffic grows with the state, so n qubits
# scale it by 2^(n - 26).  Set to None whenever the kernel changes until it
# is re-captured.
TILE_C64_TRAFFIC_26Q = 536.910848e6 + 475.749632e6       # k_tile<0,3,1,1> (its ncu capture at 26 qubits)
BLOCK_C64_TRAFFIC_26Q = {  # the block kernels' ncu captures at 26 qubits
    "k_fused_umma_tma<6,window>": 536.997376e6 + 476.200192e6,
    "k_fused_umma_tma<6,rows>": 537.023232e6 + 476.058368e6,
    "k_fused_umma<6>": 537.065216e6 + 475.915776e6,
}
BLOCK_C128_TRAFFIC_26Q = {  # the complex128 block kernels' ncu captures at 26 qubits (double-float storage)
    "k_fused_c128<5,window>": 1073.883e6 + 1013.351e6,
}
S_BYTES = {"c64": 8, "c128": 16}
# what each dtype's arithmetic is, for the report
ARITHMETIC = {
    "c64": "complex64 storage; FP32 arithmetic (tensor-core blocks: FP16 hi/lo split products, ~2^-22 per product)",
    "c128": ("complex128 in and out (FP64); during a plan, double-float pairs (~2^-46 relative down to 2^-80, "
             "float precision below, zero below 2^-126); tensor-core blocks: each group's values on a 43-bit "
             "fixed-point grid split into five 9-bit integer digits, exact FP16 digit products and exact FP32 level "
             "sums (error ~2^-44 of the group's largest amplitude)"),
}


def metric_name(wl):
    return "effective HBM GB/s (2*2^n*bytes_per_amp per logical gate) & gates/s, %s" % wl["desc"]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for name, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(backend):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample of the same workload)
# ---------------------------------------------------------------------------

_ORACLE_PSI = {}


def oracle_sample(workload, budget_s):
    """Run the oracle over the first gates of the workload circuit until
    ``budget_s`` of wall time is spent; returns (gates_done, seconds, n).
    The state vector is allocated once per size and reused."""
    import oracle
    wl = WORKLOADS[workload]
    n = wl["n"]
    circ = wl["make"]()
    if n not in _ORACLE_PSI:
        _ORACLE_PSI[n] = oracle.zero_state(n)
        oracle.run_circuit(_ORACLE_PSI[n], circ[:1])  # touch the pages before timing
    psi = _ORACLE_PSI[n]
    psi[:] = 0
    psi[0] = 1
    done, t0 = 0, time.perf_counter()
    while done < len(circ) and time.perf_counter() - t0 < budget_s:
        oracle.run_circuit(psi, circ[done:done + 1])
        done += 1
    return done, time.perf_counter() - t0, n


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args):
    world, rank, _ = dist_setup("gloo")
    if rank != 0:
        return 0
    wl = WORKLOADS[args.workload]
    n = wl["n"]
    S = 16  # the oracle computes in FP64 (complex128)
    per_step = []
    gates = 0
    for i in range(args.warmup + args.steps):
        g, t, _ = oracle_sample(args.workload, args.ref_budget)
        if i >= args.warmup:
            per_step.append(t)
            gates += g
    T = sum(per_step)
    gbs = 2.0 * (1 << n) * S * gates / T / 1e9
    line = {
        "impl": "reference", "metric": metric_name(wl),
        "value": gbs, "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * T / len(per_step), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"] + " (oracle, FP64 complex128)", "n": n, "gates_per_step": gates / len(per_step)},
        "gates_per_s": gates / T,
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": f"first gates of the circuit, {args.ref_budget:.0f} s of wall time per step"},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def timed_run(qs, torch, state, plan, steps, warmup, world, device, profile=True):
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        state.set_basis(0)
        state.run(plan)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    step_ms = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        state.set_basis(0)
        if profile:
            step_ms.append(state.run_profiled(plan))
        else:
            state.run(plan)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return allreduce_max(ms, world, device), step_ms


FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x 2 flop x max SM clock


def circuit_flops(circ, n):
    """Algorithmic floating-point operations of a circuit on 2^n amplitudes:
    a dense one-qubit gate costs 4 complex multiplies and 2 complex adds per
    amplitude pair (14 flops per amplitude); a phase or diagonal gate 6 flops
    per amplitude it changes; X-type gates and swaps none."""
    N = float(1 << n)
    f = 0.0
    for g in circ:
        if g.name in ("U3", "H", "RX", "RY", "Y"):
            f += 14 * N
        elif g.name in ("RZ",):
            f += 6 * N
        elif g.name in ("Z", "S", "T", "P"):
            f += 6 * N / 2
        elif g.name in ("CZ", "CP"):
            f += 6 * N / 4
    return f


def box_runs(q, n):
    """Runs of consecutive qubits of one class (the block's, or the others')
    over 0..n-1 once the tile's 7 lowest non-block qubits are taken: the
    dimensions of the TMA view a block's tiles move through (at most 5)."""
    inq = set(q)
    cls = [1 if b in inq else 0 for b in range(n)]
    return 1 + sum(1 for b in range(1, n) if cls[b] != cls[b - 1])


def step_kernel(plan, i, kind):
    """The kernel a plan step launches: block steps are told apart by their
    qubits (at least 128 groups and at most 5 runs of block and other
    qubits: a set starting with the run 0..a-1, a >= 4 for complex64 and 3
    for complex128, runs the rows form of the TMA kernel, reported as "rows"
    for qubits 0..k-1 and "lowrun" otherwise; another set with qubit 0
    outside it or in the run 0, 1 its box form, reported as "window" for
    consecutive qubits and "box" otherwise; other sets gather per thread:
    complex64 k_fused_umma<k>, complex128 k_fused_c128<k,gather>); other
    blocks the SIMT k_dense; other steps keep their kind."""
    if kind != "block":
        return kind
    q = sorted(plan.step_qubits(i))
    k = len(q)
    if not ((plan.dtype == "c128" and k in (4, 5)) or (plan.dtype == "c64" and k >= 4)):
        return "k_dense<%d>" % k
    full = plan.n - k >= 7
    name = "k_fused_c128" if plan.dtype == "c128" else "k_fused_umma_tma"
    a = 0
    while a < k and q[a] == a:
        a += 1
    if full and box_runs(q, plan.n) <= 5:
        if a >= (3 if plan.dtype == "c128" else 4):
            return "%s<%d,%s>" % (name, k, "rows" if a == k else "lowrun")
        if a == 0 or a == 2:
            return "%s<%d,%s>" % (name, k, "window" if q == list(range(q[0], q[0] + k)) else "box")
    return "k_fused_c128<%d,gather>" % k if plan.dtype == "c128" else "k_fused_umma<%d>" % k


def kernel_roofline(plan, step_ms, peak):
    """Per kernel: algorithmic bytes and device time summed over the timed
    steps; the dominant kernel (largest time) gives the roofline object."""
    info = [(step_kernel(plan, i, kind), b) for i, (kind, b) in enumerate(plan.step_info())]
    tot_t, tot_b, cnt = {}, {}, {}
    for ms in step_ms:
        for (kind, b), t in zip(info, ms):
            tot_t[kind] = tot_t.get(kind, 0.0) + t
            tot_b[kind] = tot_b.get(kind, 0.0) + b
            cnt[kind] = cnt.get(kind, 0) + 1
    if not tot_t:
        return None, {}
    dom = max(tot_t, key=tot_t.get)
    achieved = tot_b[dom] / (tot_t[dom] / 1e3) / 1e9
    per_kind = {k: {"launches": cnt[k], "ms": tot_t[k], "share": tot_t[k] / sum(tot_t.values()),
                    "GB/s": tot_b[k] / (tot_t[k] / 1e3) / 1e9} for k in tot_t}
    return {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "bytes_per_launch": tot_b[dom] / cnt[dom],
            "ms_per_launch": tot_t[dom] / cnt[dom], "traffic": None}, per_kind


def unfused_classes(qs, torch, device, n, reps=10):
    """Per-gate-class unfused passes (the RX-per-qubit sweep of §IV-C widened
    to four classes) on every target 0..n-1: algorithmic HBM GB/s per class,
    dtype and target (10 gates per target, device time of the 10 passes);
    the fraction of the measured HBM peak is reported beside the median."""
    out = {}
    targets = list(range(n))
    for dt in ("c64", "c128"):
        s = qs.State(n, dt, device=device)
        # a dense state (a U3 on every qubit): no amplitude is zero, so no
        # arithmetic fast path applies
        s.run(qs.Plan(qs.Circuit(W.brick(n, 1, 4)), n, dt, mode=qs.PLAN_TILED))
        for cls in ("U3", "RZ", "CNOT", "CZ"):
            res = []
            for t in targets:
                circ = W.microbench(n, cls, t, seed=5, reps=reps)
                p = qs.Plan(qs.Circuit(circ), n, dt, mode=qs.PLAN_UNFUSED)
                s.run(p)
                ms = s.run_profiled(p)
                b = sum(x[1] for x in p.step_info())
                res.append(b / (ms.sum() / 1e3) / 1e9)
            out.setdefault(cls, {})[dt] = {"targets": targets, "GBps": [round(x, 1) for x in res],
                                           "min": round(min(res), 1), "median": round(float(np.median(res)), 1),
                                           "argmin": targets[int(np.argmin(res))]}
        del s
    return out


def batch_workload(qs, torch, device, count=512, layers=8, seed=9):
    """512 hardware-efficient-ansatz circuits, n uniform in [10, 20], complex64:
    one batch (graph replay; the autotuner picks the tile shape and from how
    many qubits circuits run as fused tensor-core plans on side streams
    instead of in the persistent launch) vs one tiled plan per circuit
    launched one after another."""
    sizes = W.batch_sizes(count, 10, 20, seed)
    circs = [W.hea(n, layers, 10 + i)[0] for i, n in enumerate(sizes)]
    b = qs.Batch(sizes, circs, dtype="c64", autotune=True)
    b.run(True)
    b.sync()
    st = b.stats()
    reps = 5
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        b.run(True)
    b.sync()
    t_batch = (time.perf_counter() - t0) / reps
    # one by one: each circuit its own plan and launches, same tiles
    plans = [qs.Plan(qs.Circuit(c), n, "c64", mode=qs.PLAN_TILED) for n, c in zip(sizes, circs)]
    views = [qs.State(n, "c64", tensor=b.state(i)) for i, n in enumerate(sizes)]
    for v, p in zip(views, plans):
        v.set_basis(0)
        v.run(p)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for v, p in zip(views, plans):
        v.set_basis(0)
        v.run(p)
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    gates = sum(len(c) for c in circs)
    return {"circuits": count, "n_range": [10, 20], "gates": gates, "passes": st["passes"], "units": st["units"],
            "grid": st["grid"], "graph": st["graph"], "tuned_opts": {"tile_qubits": b.opts.tile_qubits,
                                                                     "slot_qubits": b.opts.slot_qubits,
                                                                     "groups_per_thread": b.opts.groups_per_thread,
                                                                     "fuse_min_qubits": b.opts.fuse_min_qubits},
            "batched_ms": 1e3 * t_batch, "circuits_per_s": count / t_batch,
            "hbm_GBps_batched": st["hbm_bytes"] / t_batch / 1e9,
            "hbm_frac_batched": st["hbm_bytes"] / t_batch / 1e9 / measured_peaks()[0],
            "one_by_one_ms": 1e3 * t_single, "one_by_one_circuits_per_s": count / t_single,
            "speedup_vs_one_by_one": t_single / t_batch}


def adjoint_workload(qs, torch, device, n=20, layers=10, batch=64):
    """Adjoint gradients: 20-qubit hardware-efficient ansatz, 10 layers of RY
    and RZ (400 parameters), CZ ladder, transverse-field Ising observable,
    64 parameter sets in one call."""
    circ, _ = W.hea(n, layers, 11)
    thetas = np.stack([W.hea(n, layers, 11 + b)[1] for b in range(batch)])
    terms = W.tfim(n)
    c = qs.Circuit(circ)
    out = {"n": n, "params": thetas.shape[1], "batch": batch}
    for dt in ("c128", "c64"):
        s = qs.State(n, dt, device=device)
        qs.adjoint_grad(s, c, thetas[:4], terms)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e, g = qs.adjoint_grad(s, c, thetas, terms)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        out[dt] = {"ms_per_gradient": 1e3 * t / batch, "gradients_per_s": batch / t,
                   "energy0": float(e[0]), "grad0_norm": float(np.linalg.norm(g[0]))}
        del s
    return out


def run_ours(args):
    import torch
    world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import paper_2203_16044_gb300 as qs

    wl = WORKLOADS[args.workload]
    n = wl["n"]
    circ = wl["make"]()
    peak, peak_kind = measured_peaks()
    results = {}
    dtypes = [args.dtype] + ([d for d in ("c64", "c128") if d != args.dtype] if args.both else [])
    circuit = qs.Circuit(circ)
    states = {}
    e2e = None
    tune_file = os.path.join(tempfile.gettempdir(), "qs_tune_cache_%d.txt" % os.getpid())
    qs.set_tune_cache(tune_file)
    tuned = {}
    for dt in dtypes:
        state = qs.State(n, dt, device=device)
        if args.mode == "auto":
            # the library's autotuner picks the plan shape (dense-block width
            # k or tile shape) by timing candidates on this state, before the
            # timed region
            t0 = time.perf_counter()
            opts, tms = qs.autotune(circuit, state)
            kw = qs.plan_kwargs(opts)
            plan = qs.Plan(circuit, n, dt, **kw)
            mode_name = {qs.PLAN_FUSED: "fused", qs.PLAN_TILED: "tiled"}.get(opts.mode, str(opts.mode))
            fq = opts.fuse_qubits
            tuned[dt] = {"opts": {k: v for k, v in kw.items() if v}, "tuned_ms": tms,
                         "tuning_s": time.perf_counter() - t0}
        else:
            mode_name, mode, fq = plan_mode(qs, args, dt)
            plan = qs.Plan(circuit, n, dt, mode=mode, fuse_qubits=fq)
        st = plan.stats()
        with ClockSampler(local) as clk:
            ms, step_ms = timed_run(qs, torch, state, plan, args.steps, args.warmup, world, device)
        roof, per_kind = kernel_roofline(plan, step_ms, peak)
        if roof and roof["kernel"] == "tile":
            # tile passes run many gates per HBM pass: FP32-issue bound, not HBM
            flops = circuit_flops(circ, n)
            tile_ms = per_kind["tile"]["ms"] / len(step_ms)
            roof_hbm = dict(roof)
            roof = {"kernel": "tile", "bound": "alu", "traffic": None, "achieved": flops / (tile_ms / 1e3) / 1e12,
                    "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": flops / (tile_ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
                    "flops_per_step": flops, "ms_per_launch": roof_hbm["ms_per_launch"],
                    "hbm": {"achieved": roof_hbm["achieved"], "peak": peak, "unit": "GB/s",
                            "frac": roof_hbm["frac"], "bytes_per_launch": roof_hbm["bytes_per_launch"]}}
            if dt == "c128":
                roof["note"] = "complex128 in double-float: each FP64-equivalent flop costs ~6 FP32-pipe ops"
            elif TILE_C64_TRAFFIC_26Q is not None:
                roof["traffic"] = TILE_C64_TRAFFIC_26Q * 2.0 ** (n - 26)
                roof["traffic_source"] = "ncu dram__bytes_read.sum + dram__bytes_write.sum at 26 qubits, scaled by 2^(n-26)"
        elif roof and roof["kernel"].startswith("k_fused_umma") and dt == "c64":
            roof["tensor"] = ("tcgen05.mma kind::f16, 3 MMAs per K step (FP16 hi/lo split under power-of-two "
                              "scaling), TMEM accumulator; one TMA box per 128-group tile"
                              if roof["kernel"].startswith("k_fused_umma_tma") else
                              "tcgen05.mma kind::tf32, 3 MMAs (3xTF32) per K step, TMEM accumulator")
            if roof["kernel"] in BLOCK_C64_TRAFFIC_26Q:
                roof["traffic"] = BLOCK_C64_TRAFFIC_26Q[roof["kernel"]] * 2.0 ** (n - 26)
                roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of %s "
                                          "at 26 qubits, scaled by 2^(n-26)" % roof["kernel"])
        elif roof and roof["kernel"].startswith("k_fused_c128"):
            roof["tensor"] = ("tcgen05.mma kind::f16 on exact 9-bit integer digits of the FP64 operands: 5 digits "
                              "per value, 19 digit-pair products (levels 0-5) summed per level in TMEM")
            if roof["kernel"] in BLOCK_C128_TRAFFIC_26Q:
                roof["traffic"] = BLOCK_C128_TRAFFIC_26Q[roof["kernel"]] * 2.0 ** (n - 26)
                roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of %s "
                                          "at 26 qubits, scaled by 2^(n-26)" % roof["kernel"])
        S = S_BYTES[dt]
        eff = st["metric_bytes"] / (ms / 1e3) / 1e9
        # launches per step: one per plan step, k_set_one, and for complex128
        # the two storage-layout switches (FP64 <-> double-float)
        extra = 1 + (2 if dt == "c128" else 0)
        results[dt] = {"ms_per_step": ms, "effective_GBps": eff * world, "gates_per_s": st["gates"] / (ms / 1e3) * world,
                       "plan": mode_name + (f" k={fq}" if mode_name == "fused" else ""),
                       "autotune": tuned.get(dt),
                       "arithmetic": ARITHMETIC[dt],
                       "passes": st["passes"], "gates": st["gates"], "hbm_bytes_per_step": st["hbm_bytes"],
                       "hbm_GBps": st["hbm_bytes"] / (ms / 1e3) / 1e9, "roofline": roof, "kernels": per_kind,
                       "clocks": clk.summary(), "bytes_per_amp": S,
                       "gpu_launches": (st["passes"] + extra) * args.steps}
        states[dt] = state
        del plan
        if dt == args.dtype and not args.no_e2e:
            # end to end through the C ABI with host buffers, right after the
            # headline (before the other dtype's runs), with the same plan
            # shape (the autotuner's cached answer is looked up again inside)
            e2e = run_e2e(qs, torch, args, n, circ, dt, device, world)
    # precision: infidelity of the headline run against complex128 on the GPU
    infid = None
    if "c64" in states and "c128" in states:
        infid = fidelity_vs_c128(torch, states["c64"].tensor, states["c128"].tensor)
    extras = {}
    want = set() if args.no_extras else (
        {"plans", "reductions", "measure", "brick33", "c128_unfused", "classes", "c128_config2", "policies", "batch",
         "adjoint"} if args.extras == "all" else set(args.extras.split(",")))
    if "plans" in want:
        extras["c64_plans_%dq" % n] = dtype_plans(qs, torch, device, n, circuit, "c64", states.get("c128"))
        extras["c128_plans_%dq" % n] = dtype_plans(qs, torch, device, n, circuit, "c128", None)
    if "reductions" in want:
        extras["reductions_%dq" % n] = reductions(qs, torch, states, n)
    if "measure" in want and "c64" in states:
        extras["measure_%dq" % n] = measurement(qs, torch, states["c64"], n)
    if "brick33" in want:
        extras["c64_brick33_d20"] = c64_33q(qs, torch, device, args.fuse_qubits)
    if "c128_unfused" in want:
        base = c128_unfused(qs, torch, device, n, circuit)
        base["speedup_of_headline"] = base["ms"] / results[args.dtype]["ms_per_step"]
        extras["c128_unfused_%dq" % n] = base
    if "classes" in want:
        extras["unfused_classes_28q"] = unfused_classes(qs, torch, device, 28)
    if "c128_config2" in want:
        extras["c128_brick_qft_28q"] = c128_config2(qs, torch, device, 28)
    if "policies" in want:
        extras["planner_policies_30q"] = planner_policies(qs, torch, device, 30)
    if "batch" in want:
        extras["batch_512_hea"] = batch_workload(qs, torch, device)
    if "adjoint" in want:
        extras["adjoint_20q_400p"] = adjoint_workload(qs, torch, device)
    head = results[args.dtype]
    line = {
        "metric": metric_name(wl),
        "value": head["effective_GBps"], "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": wl["desc"], "n": n, "gates": head["gates"], "dtype": args.dtype,
                   "plan": head["plan"], "passes": head["passes"], "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (state %.0f MiB, L2 126 MiB)" % (2.0 ** n * S_BYTES[args.dtype] / 2 ** 20)},
        "gates_per_s": head["gates_per_s"],
        "autotune": head["autotune"],
        "hbm_GBps_algorithmic": head["hbm_GBps"],
        "roofline": dict(head["roofline"], peak_source=peak_kind) if head["roofline"] else None,
        "kernels": head["kernels"],
        "clocks": head["clocks"],
        "gpu_launches": head["gpu_launches"],
        "e2e": e2e,
        "precision": infid,
        "other_dtypes": {dt: {k: v for k, v in r.items() if k not in ("kernels",)} for dt, r in results.items()
                         if dt != args.dtype},
        "extras": extras,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        g, t, n_cpu = oracle_sample(args.workload, args.cpu_budget)
        line["cpu_baseline"] = {"value": 2.0 * (1 << n_cpu) * 16 * g / t / 1e9, "unit": "GB/s", "cores": cpu_cores(),
                                "kind": "oracle",
                                "sample": f"first {g} gates of the same circuit at n={n_cpu}, FP64 complex128 "
                                          f"(16 B/amplitude), {t:.1f} s wall",
                                "gates_per_s": g / t}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def plan_mode(qs, args, dt):
    """(name, plan mode, fuse_qubits) for a dtype: `auto` picks the fastest
    measured plan, dense tensor-core blocks for both dtypes (complex128
    blocks have at most 5 qubits)."""
    name = args.mode
    if name == "auto":
        name = "fused"
    mode = {"fused": qs.PLAN_FUSED, "tiled": qs.PLAN_TILED, "unfused": qs.PLAN_UNFUSED}[name]
    fq = args.fuse_qubits if dt == "c64" else min(args.fuse_qubits, 5)
    return name, mode, (fq if name == "fused" else 0)


def fidelity_vs_c128(torch, t64, t128):
    """The complex64 result against the complex128 one, in FP64 on the GPU:
    the stated infidelity 1 - |<a|b>|^2, the normalised form
    1 - |<a|b>|^2 / (<a|a> <b|b>) (which a norm above 1 cannot push below
    the true error) and the complex64 norm's distance from the reference's."""
    a = t64.to(torch.complex128)
    ov = abs(torch.vdot(a, t128).item()) ** 2
    na, nb = torch.vdot(a, a).real.item(), torch.vdot(t128, t128).real.item()
    del a
    return {"infidelity_vs_c128": 1.0 - ov, "infidelity_normalised_vs_c128": 1.0 - ov / (na * nb),
            "norm2_c64": na, "norm2_c128": nb}


def dtype_plans(qs, torch, device, n, circuit, dt, ref128, reps=2):
    """The circuit in one dtype under each plan: tiles (SIMT, many gates per
    pass) and dense 4-, 5- (and for complex64 6-) qubit blocks (tensor
    cores), with the infidelity of each complex64 plan against the complex128
    result when it is at hand."""
    out = {}
    s = qs.State(n, dt, device=device)
    plans = [("tiled", qs.PLAN_TILED, 0), ("fused_k4", qs.PLAN_FUSED, 4), ("fused_k5", qs.PLAN_FUSED, 5)]
    if dt == "c64":
        plans.append(("fused_k6", qs.PLAN_FUSED, 6))
    for name, mode, fq in plans:
        p = qs.Plan(circuit, n, dt, mode=mode, fuse_qubits=fq)
        s.set_basis(0)
        s.run(p)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for _ in range(reps):
            s.set_basis(0)
            e0.record()
            s.run(p)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = p.stats()
        r = {"ms": min(ms), "passes": st["passes"], "effective_GBps": st["metric_bytes"] / (min(ms) / 1e3) / 1e9}
        if ref128 is not None and dt == "c64":
            r.update(fidelity_vs_c128(torch, s.tensor, ref128.tensor))
        out[name] = r
        del p
    del s
    return out


def planner_policies(qs, torch, device, n):
    """The paper's own workloads at n qubits, complex64, under each plan
    policy: per-gate passes; tile passes over the lowest qubits with a swap
    inserted for every remote target (swap insertion, §III-D) or one fused
    bit-pair exchange per routing point (fused-permutation insertion,
    §III-D, Listing 1); tile passes that gather their high qubits in place
    (tile-gather); dense 6-qubit tensor-core blocks.  Reports HBM passes per
    logical gate (and how many are exchanges, with their bytes) and the time
    of one run (after one warm-up)."""
    wls = {"qsb_sets10": W.qsb(n, 22, sets=10), "hadamard_x11": W.hadamard_bench(n),
           "qv_like_d10": W.qv_like(n, 10, 13)}
    out = {}
    s = qs.State(n, "c64", device=device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for wname, circ in wls.items():
        c = qs.Circuit(circ)
        row = {"gates": len(circ)}
        for pname, mode, fq in (("unfused", qs.PLAN_UNFUSED, 0), ("swap_insertion", qs.PLAN_SWAP, 0),
                                ("fused_permutation", qs.PLAN_PERMUTE, 0), ("tile_gather", qs.PLAN_TILED, 0),
                                ("fused_k6", qs.PLAN_FUSED, 6)):
            p = qs.Plan(c, n, "c64", mode=mode, fuse_qubits=fq)
            st = p.stats()
            ex = [b for k, b in p.step_info() if k == "swap"]
            s.set_basis(0)
            s.run(p)
            s.set_basis(0)
            torch.cuda.synchronize()
            e0.record()
            s.run(p)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            row[pname] = {"passes": st["passes"], "passes_per_gate": st["passes"] / len(circ), "ms": ms,
                          "exchange_passes": len(ex), "exchange_bytes": sum(ex),
                          "effective_GBps": st["metric_bytes"] / (ms / 1e3) / 1e9,
                          "hbm_GBps_algorithmic": st["hbm_bytes"] / (ms / 1e3) / 1e9}
            del p
        out[wname] = row
    del s
    return out


def reductions(qs, torch, states, n, reps=5):
    """FP64-accumulated reductions on the headline states (a7): norm, inner
    product with itself, and the TFIM expectation (its X-mask groups share
    tile passes: qs_expect_pauli_passes reads of the state).  Each call
    returns its value to the host, so the host clock around the calls
    includes the device-to-host read; GB/s counts the state bytes each call
    reads, hbm_frac divides that by the measured copy bandwidth."""
    out = {}
    terms = W.tfim(n)
    groups = len({t.xmask for t in terms})
    peak = measured_peaks()[0]
    for dt, s in states.items():
        S = S_BYTES[dt]
        N = float(1 << n)
        passes = qs.expect_pauli_passes(n, dt, terms)
        r = {}
        # the inner product of the state with itself is its norm (the
        # library recognises the same vector): one read, counted once
        for name, fn, nbytes in (("norm2", lambda: s.norm2(), N * S),
                                 ("inner_self", lambda: s.inner(s), N * S),
                                 ("expect_tfim", lambda: s.expect_pauli(terms), passes * N * S)):
            fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                v = fn()
            t = (time.perf_counter() - t0) / reps
            r[name] = {"ms": 1e3 * t, "GBps": nbytes / t / 1e9, "hbm_frac": nbytes / t / 1e9 / peak,
                       "value": v.real if isinstance(v, complex) else v}
        r["tfim_groups"] = groups
        r["tfim_passes"] = passes
        out[dt] = r
    return out


def measurement(qs, torch, s, n, reps=3):
    """Computational-basis measurement on the headline complex64 state after
    the circuit: marginal probabilities of one and of six qubits (one read
    pass per 8 outcomes), 2^20 samples (the chunk-sum pass, the host prefix
    and one scan of up to 1024 amplitudes per sample), and a measurement of
    one qubit with its collapse (a probability pass plus a read-write
    pass), last because it changes the state.  Host clock around each call
    (each returns to the host); GB/s counts the state bytes read and
    written."""
    N = float(1 << n)
    S = 8
    u = np.random.default_rng(9).random(1 << 20)
    out = {}
    for name, fn, nbytes in (("probabilities_1q", lambda: s.probabilities([n - 1]), N * S),
                             ("probabilities_6q", lambda: s.probabilities([0, 5, 10, 15, 20, 25]), N * S),
                             ("sample_1M", lambda: s.sample(u), N * S)):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        t = (time.perf_counter() - t0) / reps
        out[name] = {"ms": 1e3 * t, "GBps": nbytes / t / 1e9}
    out["sample_1M"]["shots_per_s"] = (1 << 20) / (out["sample_1M"]["ms"] / 1e3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    o, p = s.measure(n // 2, 0.3)
    t = time.perf_counter() - t0
    out["measure_collapse"] = {"ms": 1e3 * t, "GBps": 3 * N * S / t / 1e9, "outcome": o, "probability": p,
                               "norm2_after": s.norm2()}
    return out


def c64_33q(qs, torch, device, fq):
    """The 33-qubit complex64 brick circuit of depth 20 (64 GiB state) under
    the fused plan: one warm-up run, one timed run (CUDA events)."""
    wl = WORKLOADS["brick33"]
    n, circ = wl["n"], wl["make"]()
    s = qs.State(n, "c64", device=device)
    p = qs.Plan(qs.Circuit(circ), n, "c64", mode=qs.PLAN_FUSED, fuse_qubits=fq)
    s.run(p)
    torch.cuda.synchronize()
    s.set_basis(0)
    ms = s.run_profiled(p)
    st = p.stats()
    t = float(ms.sum())
    out = {"workload": wl["desc"], "plan": "fused k=%d" % fq, "ms": t, "passes": st["passes"],
           "effective_GBps": st["metric_bytes"] / (t / 1e3) / 1e9, "gates_per_s": st["gates"] / (t / 1e3),
           "hbm_GBps_algorithmic": st["hbm_bytes"] / (t / 1e3) / 1e9,
           "norm2": s.norm2()}
    del s, p
    return out


def c128_config2(qs, torch, device, n=28):
    """The 28-qubit complex128 brick (depth 40, seed 3) and QFT (seeded
    basis state) under the plain per-gate kernels and the 5-qubit
    tensor-core block plan: one warm-up run, one timed run each (CUDA
    events)."""
    out = {}
    s = qs.State(n, "c128", device=device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for wname, circ, x0 in (("brick_d40", W.brick(n, 40, 3), 0), ("qft", W.qft(n), W.basis_index(n, 4))):
        c = qs.Circuit(circ)
        for pname, mode, fq in (("unfused", qs.PLAN_UNFUSED, 0), ("fused_k5", qs.PLAN_FUSED, 5)):
            p = qs.Plan(c, n, "c128", mode=mode, fuse_qubits=fq)
            s.set_basis(x0)
            s.run(p)
            s.set_basis(x0)
            torch.cuda.synchronize()
            e0.record()
            s.run(p)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            st = p.stats()
            out.setdefault(wname, {"gates": len(circ)})[pname] = {
                "ms": ms, "passes": st["passes"], "effective_GBps": st["metric_bytes"] / (ms / 1e3) / 1e9,
                "gates_per_s": len(circ) / (ms / 1e3), "hbm_GBps_algorithmic": st["hbm_bytes"] / (ms / 1e3) / 1e9}
            del p
    del s
    return out


def c128_unfused(qs, torch, device, n, circuit):
    """The plain per-gate complex128 path (one kernel per gate, FP64 layout in
    HBM) on the same circuit: the baseline the fused complex64 path is
    compared with.  One warm-up run, one timed run (CUDA events)."""
    s = qs.State(n, "c128", device=device)
    p = qs.Plan(circuit, n, "c128", mode=qs.PLAN_UNFUSED)
    s.run(p)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.set_basis(0)
    e0.record()
    s.run(p)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = p.stats()
    out = {"ms": ms, "passes": st["passes"], "effective_GBps": st["metric_bytes"] / (ms / 1e3) / 1e9,
           "hbm_GBps_algorithmic": st["hbm_bytes"] / (ms / 1e3) / 1e9}
    del s, p
    return out


def run_e2e(qs, torch, args, n, circ, dt, device, world):
    """Per step: queue the host state's copy to the device (pinned memory,
    qs_copy_from_host_async), build the circuit, look its plan shape up in
    the autotuner's cache (or take the --mode given) and compile it while the
    copy runs, run it (queued behind the copy on the same stream), device ->
    host (pinned); timed on the host around the whole call chain, with the
    time of each phase reported beside it.  The value is the median step
    (the host link is shared with the machine's other GPUs, and single steps
    have measured up to 3x slower transfers); every step's time and phases
    are reported too."""
    tdt = torch.complex64 if dt == "c64" else torch.complex128
    host = torch.zeros(1 << n, dtype=tdt, pin_memory=True)
    host[0] = 1
    state = qs.State(n, dt, device=device)
    S = S_BYTES[dt]
    steps = max(1, min(args.steps + 2, 5))
    gates = len(circ)
    times, phases = [], []
    for i in range(1 + steps):
        torch.cuda.synchronize()
        barrier(world)
        t = [time.perf_counter()]
        state.copy_from_host_async(host.data_ptr())  # returns once queued
        t.append(time.perf_counter())
        c = qs.Circuit(circ)
        if args.mode == "auto":
            opts, _ = qs.autotune(c, state)  # a cache hit: tuned before the timed steps
            p = qs.Plan(c, n, dt, **qs.plan_kwargs(opts))
        else:
            _, mode, fq = plan_mode(qs, args, dt)
            p = qs.Plan(c, n, dt, mode=mode, fuse_qubits=fq)
        t.append(time.perf_counter())
        state.run(p)
        assert qs.lib().qs_copy_to_host(state.handle, ctypes_ptr(host)) == 0  # waits for the run, then copies
        t.append(time.perf_counter())
        if i > 0:
            times.append(t[-1] - t[0])
            phases.append(np.diff(t))
        host.zero_()
        host[0] = 1
    T = allreduce_max(float(np.median(times)), world, device)
    ph = np.median(phases, axis=0) * 1e3
    del state
    return {"value": 2.0 * (1 << n) * S * gates / T / 1e9 * world, "unit": "GB/s",
            "h2d_bytes_per_step": (1 << n) * S, "d2h_bytes_per_step": (1 << n) * S,
            "ms_per_step": 1000 * T, "gates_per_s": gates / T * world, "steps": steps, "statistic": "median",
            "mean_ms_per_step": 1000 * float(np.mean(times)),
            "phases_ms": {"h2d_queue": float(ph[0]), "circuit_and_plan_under_h2d": float(ph[1]),
                          "h2d_rest_run_and_d2h": float(ph[2])},
            "steps_ms": [[round(1e3 * float(v), 2) for v in p] for p in phases]}


def ctypes_ptr(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="brick30", choices=sorted(WORKLOADS))
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--mode", default="auto", choices=["auto", "fused", "tiled", "unfused"])
    ap.add_argument("--fuse-qubits", type=int, default=6, help="block width of the fused plan (4..6)")
    ap.add_argument("--both", type=int, default=1, help="also run the other dtype")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the class sweep, batch and adjoint workloads")
    ap.add_argument("--extras", default="all",
                    help="comma-separated extra workloads to run (plans, reductions, measure, brick33, c128_unfused, "
                         "classes, c128_config2, policies, batch, adjoint), or all")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=8.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
