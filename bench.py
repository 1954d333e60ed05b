"""Benchmark: coupled-field MLUPS of the multirate MRT-LBM on B300.

Workload: the thermosolutal free dendrite with forced convection on a
512 x 512 lattice (phi, U, T on D2Q9 plus D2Q9 flow; update factors
phi 1, U 1, T 2, flow 2; k = 0.15, Le = 10, inlet velocity 0.01 from the left,
outflow right, periodic top/bottom, seed radius 8), FP32 storage and
arithmetic, synthetic seeded inputs.

One step = one schedule period = 2 base steps, in which every field updates
at least once (phase x2, transfer x2, U x2, T x1, flow x1).  Coupled-field
MLUPS = lattice nodes x base steps / s / 1e6.  L2 is flushed (a 512 MiB
buffer written) between timed steps, and each step is timed on the device
with CUDA events on the library's stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only other implementation of
the method here) on the host cores, on a bounded sample of the same workload.
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

import workloads as W  # noqa: E402

N_LATTICE = 512
STEP_BASE = 2          # base steps per bench step (one schedule period)
METRIC = "coupled-field MLUPS"
UNIT = "MLUPS"

# element sizes of the stored populations and of the macroscopic fields per
# storage precision (16-bit storage keeps FP32 macros)
POP_BYTES = {"f64": 8, "f32": 4, "f16dev": 2, "bf16dev": 2}
MACRO_BYTES = {"f64": 8, "f32": 4, "f16dev": 4, "bf16dev": 4}


def algo_bytes(prec="f32", q=9, ori=False):
    """Algorithmic bytes per node of one launch of each update kernel: the
    stored state read and written once (phase: q - 1 populations, 8 on D2Q9
    and 4 on D2Q5; flow: 8 populations; U and T: the 2 first-moment planes),
    each macro read / written once; with grain orientations the phase update
    also reads each node's crystal angle."""
    pb, m = POP_BYTES[prec], MACRO_BYTES[prec]
    pops = 2 * 8 * pb
    moms = 2 * 2 * pb
    return {
        "phase": 2 * (q - 1) * pb + (5 if ori else 4) * m,   # pops R+W, phi^q, U, T (, angle) R, phi^{q+1} W
        "transfer": 6 * m,                      # phi^q, phi^{q+1}, U, T R; U, T W
        "scalar_U": moms + 5 * m,               # j R+W, U R+W, phi R, u R (2)
        "scalar_T": moms + 5 * m,
        "flow": pops + 7 * m,                   # pops, phi R, (rho, ux, uy) R + W
    }


ALGO_BYTES = algo_bytes("f32")


def transport_bytes(tr, u, t, f, has_T=True, has_flow=True, prec="f32"):
    """Algorithmic bytes per node of one fused transport launch: the transfer
    reads phi^q, phi^{q+1}, U, T once; each scheduled scalar reads and writes
    its first moments and writes its macro, the flow its 8 populations and
    macros; a macro whose field does not update in this step is written back
    with the injection."""
    m, pops, moms = MACRO_BYTES[prec], 2 * 8 * POP_BYTES[prec], 2 * 2 * POP_BYTES[prec]
    b = m                                       # phi (current) R
    if tr:
        b += m + m + (m if has_T else 0)        # phi^q, U, T R
        b += (0 if u else m) + (0 if (t or not has_T) else m)   # injected macros carried over
    else:
        b += (m if u else 0) + (m if t else 0)
    if (u or t) and has_flow:
        b += 2 * m                              # u for the scalar equilibria
    if u:
        b += moms + m
    if t:
        b += moms + m
    if f:
        b += pops + 6 * m - (2 * m if (u or t) else 0)   # rho, u R (u shared with the scalars) + W
    return b


def period_bytes(p, prec="f32"):
    """(total transport bytes per node over one schedule period, launches)."""
    from math import gcd
    L = 1
    for N in (p.N_phi, p.N_U, p.N_T, p.N_F):
        L = L * N // gcd(L, N)
    tot, n = 0, 0
    for k in range(2 * L):
        tr = (k + 1) % p.N_phi == 0
        u = p.has_U and (k + 1) % p.N_U == 0
        t = p.has_T and (k + 1) % p.N_T == 0
        f = p.has_flow and (k + 1) % p.N_F == 0
        if tr or u or t or f:
            tot += transport_bytes(tr, u, t, f, p.has_T, p.has_flow, prec)
            n += 1
    return tot, n


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of ncu captures
# per kernel variant ("q<velocities of the phase, U, T lattices>:kind:variant"),
# summarised in profiles/: per launch on the 512^2 workload, and per node on
# 8192^2 (times the nodes a launch processes for the 8192^2 measurement).
# Reported only while the kernel sources hash to TRAFFIC_SOURCE_SHA; after any
# change of the code the traffic is null until re-measured.
TRAFFIC_SOURCE_SHA = "ace4b0757b2c0eb7"
# (transport: the mean of the period's two kinds of launch, transfer + U
# alone and transfer + U + T + flow, like the algorithmic bytes it is set
# against)
TRAFFIC_PER_LAUNCH_512 = {"q5:transport:8": 14232256.0, "q5:transport:16": 14231744.0, "q5:phase:4": 7369088.0,
                          "q5:phase:8": 7366272.0}
# measured directly on an 8192^2 lattice (single-pass counters; the traffic
# of a vector-strip launch does not depend on the data), FP32; the phase
# update with grain angles (":ori")
TRAFFIC_PER_NODE_8192 = {
    "q5:flow:1016": 92.63, "q5:flow:1032": 93.35, "q5:phase:1016:ori": 52.21, "q5:phase:1032:ori": 52.41,
    "q5:scalar_T:1016": 36.04, "q5:scalar_T:1032": 36.54, "q5:scalar_U:1016": 36.03, "q5:scalar_U:1032": 36.58,
    "q5:transfer:1016": 23.80, "q5:transfer:1032": 23.84, "q9:flow:1016": 92.63, "q9:flow:1032": 93.47,
    "q9:phase:1016:ori": 84.72, "q9:phase:1032:ori": 85.0, "q9:scalar_T:1016": 35.95, "q9:scalar_T:1032": 36.32,
    "q9:scalar_U:1016": 35.97, "q9:scalar_U:1032": 36.4, "q9:transfer:1016": 23.80, "q9:transfer:1032": 23.83,
}


def kernel_source_sha():
    """Hash of the CUDA sources with comments and blank space removed: a
    change of the code invalidates the stored traffic, a change of a comment
    does not."""
    import hashlib
    import re
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2609_25670_b300", "csrc")
    for nm in sorted(os.listdir(d)):
        if nm.endswith((".cu", ".cuh")):
            with open(os.path.join(d, nm)) as f:
                src = f.read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            src = re.sub(r"//[^\n]*", "", src)
            src = "\n".join(ln.rstrip() for ln in src.splitlines() if ln.strip())
            h.update(nm.encode() + b"\0" + src.encode())
    return h.hexdigest()[:16]


def lattice_label(p):
    return "phi/U/T/flow on D2Q9" if getattr(p, "q_scalar", 9) != 5 else "phi/U/T on D2Q5, flow on D2Q9"


def workload_label(p, prec="f32"):
    return (f"thermosolutal free dendrite + forced convection, {p.nx}x{p.ny}, {lattice_label(p)}, "
            f"N=({p.N_phi},{p.N_U},{p.N_T},{p.N_F}), {STORAGE_LABEL[prec]}")


STORAGE_LABEL = {"f64": "FP64", "f32": "FP32", "f16dev": "FP32 arithmetic, FP16 deviation storage",
                 "bf16dev": "FP32 arithmetic, BF16 deviation storage"}


def workload(n=None, q=5):
    wl = W.thermosolutal_convection(n=n or N_LATTICE, R=8.0)
    wl.params.q_scalar = q
    return wl


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value, device=None):
    """The maximum of a per-rank number over every rank of the process group
    (the number itself with one rank or no group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(nodes, base_steps_per_step, steps, world, ms_max):
    """Whole-job MLUPS: the node updates of every rank's replica over the
    slowest rank's time (weak scaling: each rank advances its own lattice)."""
    return nodes * base_steps_per_step * steps * world / (ms_max * 1e-3) / 1e6


def gated_steps(torch, stream, flush, advance, steps, reinit=None):
    """`steps` bench steps on `stream`: an L2 flush (untimed), then one
    advance() between two CUDA events.  A bounded sleep kernel queued first
    holds the stream while the host enqueues every step, so the device runs
    the steps back to back from its queue and a pause of the host thread
    (scheduling, the clock sampler's queries) cannot fall inside a timed
    step.  The gate is checked: an event recorded behind the sleep must still
    be pending once the host has enqueued the last step.  If the device got
    there first (a host slower than the gate), the times hold host gaps: the
    state is re-initialised with `reinit` and the steps are timed again
    behind a gate four times longer, at most three attempts in all.
    Returns (the per-step times in ms, whether the gate held)."""
    gate_s = 0.01 + 1e-3 * steps
    for attempt in range(3):
        if attempt and reinit is not None:
            reinit()
            torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        gate = torch.cuda.Event()
        with torch.cuda.stream(stream):
            torch.cuda._sleep(int(min(gate_s, 8.0) * 2.0e9))   # ~gate_s at the 2 GHz SM clock
            gate.record(stream)
        for k in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
                ev[k][0].record(stream)
            advance()
            with torch.cuda.stream(stream):
                ev[k][1].record(stream)
        held = not gate.query()
        torch.cuda.synchronize()
        times = [a.elapsed_time(b) for a, b in ev]
        if held:
            break
        gate_s *= 4.0
    return times, held


def refine_tiles(sim, torch, flush, tiles, steps=24):
    """In-place refinement of the autotuner's choice on an L2-resident
    lattice: lbm_autotune times each kind's variants back to back on the
    live state, where every launch after the first finds the state in L2,
    while a bench step starts from a flushed L2.  Time whole flushed steps
    (graph replays) for the tile heights of the kinds that run every step
    and keep the fastest; the live state is advanced by these steps, which
    leaves the workload unchanged in kind (the timed region follows).
    Returns the refined choices."""
    stream = sim.stream
    kinds = ["phase", "transport"] if sim.fused else ["phase", "transfer", "scalar_U"]
    for kind in kinds:
        best, best_v = None, tiles[kind]
        for v in sorted({4, 8, 16, tiles[kind]}):
            sim.set_tile(kind, v)
            sim.advance(STEP_BASE)                    # capture with this variant
            torch.cuda.synchronize()
            ms = sorted(gated_steps(torch, stream, flush, lambda: sim.advance(STEP_BASE), steps)[0])[steps // 2]
            if best is None or ms < best:
                best, best_v = ms, v
        sim.set_tile(kind, best_v)
        tiles[kind] = best_v
    return tiles


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(target_s: float = 12.0, max_steps: int = 4000, q: int = 5):
    """The FP64 oracle on the host cores, on a bounded sample of the workload:
    the full 512^2 lattice advanced for as many base steps as fit in ~target_s."""
    import oracle
    wl = workload(None, q)
    o = oracle.Oracle(wl.params, wl.fields)
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps and (time.perf_counter() - t0) < target_s:
        o.advance(STEP_BASE)
        steps += STEP_BASE
    dt = time.perf_counter() - t0
    cores = oracle.num_threads()
    # the same oracle on one thread, a shorter sample continuing the run
    oracle.set_threads(1)
    t1, steps1 = time.perf_counter(), 0
    while steps1 < max_steps and (time.perf_counter() - t1) < target_s / 3:
        o.advance(STEP_BASE)
        steps1 += STEP_BASE
    dt1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    o.close()
    nodes = wl.params.nx * wl.params.ny
    return {"value": nodes * steps / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "value_1_thread": nodes * steps1 / dt1 / 1e6,
            "sample": "%d^2 thermosolutal+flow lattice (%s), first %d base steps, FP64 oracle (%.1f s); "
                      "1 thread: the next %d base steps (%.1f s)" % (
                N_LATTICE, lattice_label(wl.params), steps, dt, steps1, dt1)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    wl = workload(None, args.q_scalar)
    o = oracle.Oracle(wl.params, wl.fields)
    for _ in range(args.warmup):
        o.advance(STEP_BASE)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.advance(STEP_BASE)
    dt = time.perf_counter() - t0
    nodes = wl.params.nx * wl.params.ny
    v = nodes * STEP_BASE * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": workload_label(wl.params, args.precision or "f32"),
                       "base_steps_per_step": STEP_BASE},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "%d steps of %d base steps on the full %d^2 lattice" % (
                                 args.steps, STEP_BASE, N_LATTICE)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import paper_2609_25670_b300 as lbm

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = workload(args.lattice, args.q_scalar)
    p = wl.params
    nodes = p.nx * p.ny
    prec = args.precision or "f32"
    if args.orientation is not None:        # one grain turned by this angle (profiling of the angle reads)
        wl.fields["theta"] = np.full((p.ny, p.nx), float(args.orientation))
    sim = lbm.Simulation(p, precision=prec)
    if args.fusion != "auto":
        sim.set_fusion(args.fusion == "on")
    sim.init_fields(wl.fields)
    stream = sim.stream
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    # warm-up, tile autotuning on the live state (leaves it unchanged), graph capture
    for _ in range(max(args.warmup, 3) if args.warmup > 0 else 0):
        sim.advance(STEP_BASE)
    tiles = sim.autotune(reps=10)
    if nodes * 200 < 126 * 2 ** 20 and not args.tile:     # state in L2: refine on flushed steps
        tiles = refine_tiles(sim, torch, flush, tiles)
    for spec in args.tile or []:            # fixed kernel variants (profiling runs)
        kind, v = spec.split("=")
        sim.set_tile(kind, int(v))
        tiles[kind] = int(v)
    sim.advance(STEP_BASE)
    kinds = ["phase", "transfer", "scalar_U", "scalar_T", "flow", "transport"]
    tb, tn = period_bytes(p, prec)
    algo = algo_bytes(prec, args.q_scalar)
    algo["transport"] = tb / max(tn, 1)       # mean over the period's transport launches
    # untimed pre-pass with every kind timed, to find the dominant kernel; the
    # timed region then times only that kind (fewest event nodes in the graph)
    sim.timing_enable(kinds)
    for _ in range(10):
        with torch.cuda.stream(stream):
            flush.fill_(0.0)
        sim.advance(STEP_BASE)
    pre = sim.timing_read(reset=True)
    dom = max(kinds, key=lambda k: pre[k][0])

    def timed_region():
        """args.steps steps (the caller re-initialises the state first, so
        that every timed region covers the first 2 * steps base steps of the
        workload), L2 flushed before each step, CUDA events around each step
        on the library stream; returns (total ms, wall s, whether the gate held)."""
        barrier()
        w0 = time.perf_counter()
        t, held = gated_steps(torch, stream, flush, lambda: sim.advance(STEP_BASE), args.steps,
                              reinit=lambda: sim.init_fields(wl.fields))
        barrier()
        return sum(t), time.perf_counter() - w0, held

    # the timed region: graphs without timing nodes (an event-record node
    # around a launch inside a graph adds several microseconds per launch)
    sim.timing_enable([])
    sim.advance(STEP_BASE)           # recapture without timing nodes, untimed
    sim.init_fields(wl.fields)       # untimed: the timed steps start from the initial state
    launches0 = sim.launch_counts()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms, wall, gate_held = timed_region()
    clk = clocks.stop()
    launches1 = sim.launch_counts()
    gpu_launches = int(sum(launches1[k] - launches0[k] for k in launches1))
    ms_max = max_over_ranks(ms, dev)
    value = job_throughput(nodes, STEP_BASE, args.steps, world, ms_max)
    # the dominant kernel's own launches: a second timed region of the same
    # steps with its CUDA events recorded inside the graphs
    sim.timing_enable([dom])
    sim.advance(STEP_BASE)           # recapture with the dominant kind's timing nodes, untimed
    sim.timing_read(reset=True)
    sim.init_fields(wl.fields)
    ms_instr, _, _ = timed_region()
    ktimes = sim.timing_read(reset=True)
    sim.timing_enable([])
    state_finite = not sim.diagnostics()["nonfinite"]

    # roofline of the dominant kernel (largest share of the timed kernel time)
    dom_ms, dom_n = ktimes[dom]
    avg_s = dom_ms * 1e-3 / max(dom_n, 1)
    peak, peak_kind = measured_peaks()
    achieved = algo[dom] * nodes / avg_s / 1e9
    traffic = None
    if args.lattice in (None, N_LATTICE) and prec == "f32" and TRAFFIC_SOURCE_SHA == kernel_source_sha():
        traffic = TRAFFIC_PER_LAUNCH_512.get("q%d:%s:%d" % (args.q_scalar, dom, tiles[dom]))

    # end to end through the public API with pinned host buffers
    host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in wl.fields.items()}
    host_np = {k: v.numpy() for k, v in host.items()}
    out_phi = torch.empty((p.ny, p.nx), dtype=torch.float64).pin_memory().numpy()
    e2e_steps = 0 if args.no_e2e else max(3, min(args.steps, 50))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sim.init_fields(host_np)
        sim.advance(STEP_BASE)
        sim.field("phi", out=out_phi)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_val = nodes * STEP_BASE * e2e_steps * world / e2e_s / 1e6 if e2e_steps else None
    h2d = 6 * 8 * nodes
    d2h = 8 * nodes

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "f64" else "f32",
            "data": "synthetic (seeded)",
            "config": {"workload": workload_label(p, prec), "storage": prec, "base_steps_per_step": STEP_BASE,
                       "fused_transport": sim.fused, "fusion_choice": args.fusion,
                       "l2": "flushed between steps (512 MiB write)", "parallelism": "replicas" if world > 1 else "1 GPU"},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "algo_bytes_per_node": algo[dom], "avg_launch_us": avg_s * 1e6,
                         "launches_timed": dom_n,
                         "timed_in": "a second timed region of the same steps with the kernel's CUDA events "
                                     "inside the graphs (%.1f us per step there against %.1f without them)" % (
                                         ms_instr * 1e3 / args.steps, ms * 1e3 / args.steps)},
            "kernel_avg_us_prepass": {k: pre[k][0] / max(pre[k][1], 1) * 1e3 for k in kinds},
            "tiles": {k: tiles[k] for k in kinds},
            "gpu_launches": gpu_launches,
            "wall_s_timed_region": wall,
            "gate_held": gate_held,
            "state_finite_after_timed_regions": state_finite,
            "timing": "CUDA events around each step's advance on the library stream; the steps are queued "
                      "behind a bounded sleep kernel (included in wall_s_timed_region, not in value) that is checked "
                      "to outlast the host's enqueueing (re-timed behind a longer one otherwise)",
            "clocks": clk,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps, "calls": "init_fields(host f64 x6) + advance(2) + field(phi -> host)"},
        }
    sim.close()
    del flush
    if rank == 0:
        if not args.no_large and world == 1:
            line["large_lattice"] = large_lattice(args, torch, lbm, local, measured_peaks, args.q_scalar)
        if not args.no_alt_lattice and world == 1:
            alt = 9 if args.q_scalar == 5 else 5
            line["d2q%d" % alt] = lattice_variant(args, torch, lbm, local, dev, 512 * 1024 * 1024, alt)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(q=args.q_scalar)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def lattice_variant(args, torch, lbm, local, dev, flush_bytes, q):
    """The same workloads with the other velocity set of the phase, U and T
    lattices (q = 9: the paper's D2Q9; q = 5: D2Q5; the flow is D2Q9 in
    both): the 512^2 configuration, timed as the main measurement (CUDA
    events on the library stream, L2 flushed between steps, from the
    re-initialised state), and the 8192^2 HBM-bound measurement with its
    dominant-kernel roofline."""
    wl = workload(args.lattice, q)
    p = wl.params
    prec = args.precision or "f32"
    sim = lbm.Simulation(p, precision=prec)
    if args.fusion != "auto":
        sim.set_fusion(args.fusion == "on")
    sim.init_fields(wl.fields)
    stream = sim.stream
    flush = torch.empty(flush_bytes // 4, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 3)):
        sim.advance(STEP_BASE)
    tiles = sim.autotune(reps=10)
    if p.nx * p.ny * 200 < 126 * 2 ** 20:
        tiles = refine_tiles(sim, torch, flush, tiles)
    sim.advance(STEP_BASE)
    steps = min(args.steps, 400)        # within the first 800 base steps (the D2Q9 reading of this
    sim.init_fields(wl.fields)          # workload turns non-finite after ~2 100)
    torch.cuda.synchronize()
    t, held = gated_steps(torch, stream, flush, lambda: sim.advance(STEP_BASE), steps,
                          reinit=lambda: sim.init_fields(wl.fields))
    ms = sum(t)
    fused = sim.fused
    finite = not sim.diagnostics()["nonfinite"]
    sim.close()
    del flush
    nodes = p.nx * p.ny
    out = {"workload": workload_label(p, prec), "value": nodes * STEP_BASE * steps / (ms * 1e-3) / 1e6,
           "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "gate_held": held, "fused_transport": fused,
           "tiles": {k: tiles[k] for k in ("phase", "transfer", "scalar_U", "scalar_T", "flow", "transport")},
           "l2": "flushed between steps (512 MiB write)", "state_finite_after_timed_region": finite}
    if not args.no_large:
        out["large_lattice"] = large_lattice(args, torch, lbm, local, measured_peaks, q)
    return out


_GRAINS = {}


def grain_angles_8192():
    """Voronoi grain angles of the 8192^2 multi-dendrite lattice (one crystal
    angle per seed, drawn in [0, pi/2)); built once per process."""
    if "theta" not in _GRAINS:
        p, pts = W.multi_dendrite_params(8192)
        _GRAINS["theta"] = W.grain_orientation(pts, W.multi_dendrite_angles(len(pts)), 0, 0, 8192, 8192, rows=32)
    return _GRAINS["theta"]


def large_lattice(args, torch, lbm, local, peaks_fn, q=9):
    """The HBM-bound regime: the 8192^2 multi-dendrite workload (thermosolutal
    growth with convection, 32 Poisson-disc seeds, update factors (1, 1, 4,
    2), FP32; about 20 GB of state, so every step streams from HBM).  Seeded
    on the device's own data path (lbm_init_seed), autotuned, then timed over
    whole schedule periods of 4 base steps with CUDA events."""
    p, pts = W.multi_dendrite_params(8192)
    p.q_scalar = q
    prec = args.precision or "f32"
    sim = lbm.Simulation(p, precision=prec)
    sim.set_orientation(grain_angles_8192())          # each grain in its own crystal frame
    sim.init_seed([{"kind": "circle", "x": float(x), "y": float(y), "r": 8.0} for x, y in pts], U0=0.0, T0=-0.55)
    period = 4
    for _ in range(2):
        sim.advance(period)
    tiles = sim.autotune(reps=3)
    sim.advance(period)
    kinds = ["phase", "transfer", "scalar_U", "scalar_T", "flow", "transport"]
    sim.timing_enable(kinds)
    sim.advance(2 * period)
    pre = sim.timing_read(reset=True)
    dom = max(kinds, key=lambda k: pre[k][0])
    steps = 10
    stream = sim.stream

    def timed_periods():
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            e0.record(stream)
        for _ in range(steps):
            sim.advance(period)
        with torch.cuda.stream(stream):
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # timed region without timing nodes in the graphs, then the same periods
    # again with the dominant kind's CUDA events for its launch duration
    sim.timing_enable([])
    sim.advance(period)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    ms = timed_periods()
    clk = clocks.stop()
    sim.timing_enable([dom])
    sim.advance(period)
    sim.timing_read(reset=True)
    timed_periods()
    kt = sim.timing_read(reset=True)
    fused = sim.fused
    sim.close()
    nodes = p.nx * p.ny
    base = steps * period
    ab = algo_bytes(prec, q, ori=True)
    # algorithmic bytes per node per base step of the staged path (the fused
    # path moves fewer); U every step, T every 4th, flow every 2nd
    step_bytes = ab["phase"] + ab["transfer"] + ab["scalar_U"] + ab["scalar_T"] / p.N_T + ab["flow"] / p.N_F
    if fused:
        tb, tn = period_bytes(p, prec)
        step_bytes = ab["phase"] + tb / (2 * period)
    peak, peak_kind = peaks_fn()
    gbs = step_bytes * nodes * base / (ms * 1e-3) / 1e9
    dom_algo = dict(ab)
    tb, tn = period_bytes(p, prec)
    dom_algo["transport"] = tb / max(tn, 1)
    avg_s = kt[dom][0] * 1e-3 / max(kt[dom][1], 1)
    dom_gbs = dom_algo[dom] * nodes / avg_s / 1e9
    traffic, traffic_note = None, None
    key = "q%d:%s:%d%s" % (q, dom, tiles[dom], ":ori" if dom == "phase" else "")
    if prec == "f32" and TRAFFIC_SOURCE_SHA == kernel_source_sha() and key in TRAFFIC_PER_NODE_8192:
        traffic, traffic_note = TRAFFIC_PER_NODE_8192[key] * nodes, "8192^2 capture of this variant"
    return {"workload": "8192x8192 multi-dendrite thermosolutal growth with convection, 32 seeds in grains of "
                        "random crystal orientation, N=(1,1,4,2), "
                        + lattice_label(p) + ", " + STORAGE_LABEL[prec], "storage": prec,
            "value": nodes * base / (ms * 1e-3) / 1e6, "unit": UNIT, "base_steps": base,
            "ms_per_period": ms / steps, "fused_transport": fused,
            "step": {"algo_bytes_per_node_per_base_step": step_bytes, "achieved_GBs": gbs, "peak": peak,
                     "frac": gbs / peak, "peak_kind": peak_kind},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": dom_gbs, "peak": peak, "unit": "GB/s",
                         "frac": dom_gbs / peak, "traffic": traffic, "traffic_note": traffic_note,
                         "algo_bytes_per_node": dom_algo[dom], "avg_launch_us": avg_s * 1e6,
                         "launches_timed": kt[dom][1]},
            "kernel_avg_us_prepass": {k: pre[k][0] / max(pre[k][1], 1) * 1e3 for k in kinds},
            "tiles": {k: tiles[k] for k in kinds}, "clocks": clk, "l2": "inputs larger than L2 (~20 GB state)"}


def run_ensemble(args):
    """Batched ensemble: 64 thermosolutal members of sizes 128..1024 (seeded
    draws of undercooling, Le, update factors, seed radius), 16-bit deviation
    storage with FP32 arithmetic; aggregate MLUPS of the batched launches vs
    the same members advanced one after another.  One step = one common
    schedule period (8 base steps)."""
    import torch
    import paper_2609_25670_b300 as lbm
    ms = W.ensemble_members(count=args.members, seed=4)
    prec = args.precision or "f16dev"
    sim = lbm.Simulation([m.params for m in ms], precision=prec)
    for i, m in enumerate(ms):
        sim.init_fields(m.fields, sim=i)
    period = 8
    nodes = sum(m.params.nx * m.params.ny for m in ms)
    res = {}
    for mode in ("batched", "sequential"):
        sim.set_batching(mode == "batched")
        for _ in range(max(args.warmup, 3)):
            sim.advance(period)
        if mode == "batched":
            sim.autotune(reps=3)
            sim.advance(period)
        torch.cuda.synchronize()
        l0 = sim.launch_counts()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(sim.stream):
            e0.record(sim.stream)
        for _ in range(args.steps):
            sim.advance(period)
        with torch.cuda.stream(sim.stream):
            e1.record(sim.stream)
        torch.cuda.synchronize()
        ms_t = e0.elapsed_time(e1)
        l1 = sim.launch_counts()
        res[mode] = {"value": nodes * period * args.steps / (ms_t * 1e-3) / 1e6, "ms_per_step": ms_t / args.steps,
                     "gpu_launches": int(sum(l1[k] - l0[k] for k in l1))}
    line = {"metric": METRIC + " (ensemble aggregate)", "value": res["batched"]["value"], "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["batched"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "f64" else "f32", "data": "synthetic (seeded)",
            "config": {"workload": "batched ensemble of %d thermosolutal members, sizes 128..1024, seed 4" % len(ms),
                       "storage": prec, "nodes": nodes, "base_steps_per_step": period, "l2": "inputs larger than L2"},
            "gpu_launches": res["batched"]["gpu_launches"], "sequential": res["sequential"],
            "speedup_vs_sequential": res["batched"]["value"] / res["sequential"]["value"]}
    print(json.dumps(line), flush=True)
    sim.close()
    return 0


def run_sweep(args):
    """Update-factor sweeps (Secs. 4.1 and 4.4), measured on the GPU:

    * the thermal free dendrite (128^2, phi + T) with N_T in {1, 2, 4, 8} at
      fixed physics: tip velocity over the last 500 of 2000 base steps and
      MLUPS of the 2000 steps;
    * the Sec. 4.4 directional saline-water case with the evolving
      temperature (Table 1, bottom wall at T_b = -20, 1000 x 1000) for
      Le in {1, 10, 100, 1000} with N_U = Le: MLUPS over two schedule
      periods (at least 2000 base steps), solute drift R_M and the front
      height after them."""
    import torch
    import paper_2609_25670_b300 as lbm
    prec = args.precision or "f32"

    def timed(sim, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with torch.cuda.stream(sim.stream):
            e0.record(sim.stream)
        sim.advance(n)
        with torch.cuda.stream(sim.stream):
            e1.record(sim.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    thermal = []
    for NT in (1, 2, 4, 8):
        wl = W.thermal_free_dendrite(n=128, N_T=NT)
        sim = lbm.Simulation(wl.params, precision=prec)
        sim.init_fields(wl.fields)
        hist = []
        for _ in range(100):
            sim.advance(20)
            hist.append(sim.diagnostics()["tip"].copy())
        sim.init_fields(wl.fields)
        sim.advance(max(args.warmup, 3) * NT)
        ms = timed(sim, 2000)
        sim.close()
        h = np.asarray(hist)
        thermal.append({"N_T": NT, "tau_T": 3.0 * NT * wl.params.kappaL / wl.params.rhoCpL + 0.5,
                        "v_tip": float(((h[-1] - h[-26]) / 500.0).mean()), "tip_2000": float(h[-1].mean()),
                        "mlups": 128 * 128 * 2000 / (ms * 1e-3) / 1e6})
    v1 = thermal[0]["v_tip"]
    for r in thermal:
        r["v_tip_rel_to_NT1"] = r["v_tip"] / v1

    directional = []
    for Le in (1, 10, 100, 1000):
        wl = W.directional_evolving_T(Le=Le)
        sim = lbm.Simulation(wl.params, precision=prec)
        sim.init_fields(wl.fields)
        m0 = sim.diagnostics()["M_C"]
        period = max(1, Le)
        sim.advance(period)
        sim.autotune(reps=3)
        n = 2 * max(1000, period)
        ms = timed(sim, n)
        d = sim.diagnostics()
        sim.close()
        directional.append({"Le": Le, "N_U": Le, "base_steps": n + period,
                            "mlups": wl.params.nx * wl.params.ny * n / (ms * 1e-3) / 1e6,
                            "R_M": (d["M_C"] - m0) / m0, "front_height": float(d["tip"][1]),
                            "nonfinite": int(d["nonfinite"])})
    line = {"metric": METRIC + " (update-factor sweeps)",
            "value": next(r["mlups"] for r in directional if r["Le"] == 100), "unit": UNIT,
            "n_gpus": 1, "steps": 1, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == "f64" else "f32", "data": "synthetic (seeded)",
            "config": {"workload": "Sec. 4.4 directional saline water with evolving T, 1000x1000, Le = 100 "
                                   "(value); thermal dendrite N_T sweep and Le sweep in the details",
                       "storage": prec},
            "thermal_dendrite_NT_sweep": thermal, "directional_Le_sweep": directional}
    print(json.dumps(line), flush=True)
    return 0


def run_configs(args):
    """The workload list's cases at their stated lengths, with the outputs
    each one names (physics results of the CUDA path; parity against the
    oracle is the tests' job):

    * thermal free dendrite, 128^2 periodic, FP64, N_T in {1, 2}, 2000 base
      steps, on the D2Q9 and the D2Q5 phase / temperature lattices: tip
      position history (every 20 steps), tip velocity over the last 500
      steps, enthalpy drift;
    * thermosolutal free dendrite with forced convection, 512^2, 20 000 base
      steps, FP64 and FP32, on D2Q9 and D2Q5: upstream (-x, facing the inlet)
      and downstream (+x) tip velocities over the last 2000 steps, solute
      drift R_M, FP32 against FP64;
    * directional solidification, 1024 x 2048, frozen pulled gradient, Le in
      {1, 10, 100, 1000} (N_U = Le), 200 000 base steps, FP32 storage and
      FP16 deviation storage: front height, R_M, finiteness;
    * large multi-dendrite growth with convection, 8192^2, 50 000 base steps,
      FP32, D2Q5 and D2Q9: R_M and the step-level algorithmic HBM throughput.
    A run whose fields turn non-finite stops there and reports the base step
    of the first diagnostics call that saw it."""
    import torch
    import paper_2609_25670_b300 as lbm

    def timed(sim, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with torch.cuda.stream(sim.stream):
            e0.record(sim.stream)
        sim.advance(n)
        with torch.cuda.stream(sim.stream):
            e1.record(sim.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def history(sim, total, every):
        """Tip history sampled every `every` base steps; stops at the first
        sample that sees a non-finite field (returns its base step, else None)."""
        hist, ms, bad = [], 0.0, None
        for k in range(total // every):
            ms += timed(sim, every)
            d = sim.diagnostics()
            if d["nonfinite"]:
                bad = (k + 1) * every
                break
            hist.append(d["tip"].copy())
        return np.asarray(hist), ms, d, bad

    def chunked(sim, total, chunk):
        """advance in chunks with a finiteness check after each"""
        ms, bad, done = 0.0, None, 0
        while done < total:
            n = min(chunk, total - done)
            ms += timed(sim, n)
            done += n
            d = sim.diagnostics()
            if d["nonfinite"]:
                bad = done
                break
        return ms, d, bad, done

    out = {}
    # 1. thermal free dendrite
    rows = []
    for q in (9, 5):
        for NT in (1, 2):
            wl = W.thermal_free_dendrite(n=128, N_T=NT)
            wl.params.q_scalar = q
            sim = lbm.Simulation(wl.params, precision="f64")
            sim.init_fields(wl.fields)
            d0 = sim.diagnostics()
            h, ms, d, bad = history(sim, 2000, 20)
            sim.close()
            rows.append({"lattice": "D2Q%d" % q, "N_T": NT, "storage": "f64",
                         "v_tip": float(((h[-1] - h[-1 - min(25, len(h) - 1)]) / (20.0 * min(25, len(h) - 1))).mean()),
                         "tip_last": h[-1].tolist(),
                         "H_drift_rel": (d["H"] - d0["H"]) / abs(d0["H"]), "nonfinite_at_base_step": bad,
                         "mlups": 128 * 128 * 20 * len(h) / (ms * 1e-3) / 1e6})
    out["thermal_dendrite_128"] = rows
    # 2. thermosolutal + convection
    rows = []
    for q, prec in ((9, "f64"), (9, "f32"), (5, "f64"), (5, "f32")):
        wl = W.thermosolutal_convection(n=512, R=8.0)
        wl.params.q_scalar = q
        sim = lbm.Simulation(wl.params, precision=prec)
        sim.init_fields(wl.fields)
        m0 = sim.diagnostics()["M_C"]
        sim.autotune(reps=3)                             # on the live state, which it leaves unchanged
        h, ms, d, bad = history(sim, 20000, 200)         # 100 samples, the last at step 20 000
        sim.close()
        m = min(10, len(h) - 1)
        v = (h[-1] - h[-1 - m]) / (m * 200)             # the last 2000 finite base steps (fewer if cut short)
        rows.append({"lattice": "D2Q%d" % q, "storage": prec, "base_steps": 200 * len(h),
                     "v_tip_downstream_+x": float(v[0]), "v_tip_upstream_-x": float(v[2]),
                     "v_tip_+y": float(v[1]), "v_tip_-y": float(v[3]), "tips_last": h[-1].tolist(),
                     "R_M": (d["M_C"] - m0) / m0 if bad is None else None, "nonfinite_at_base_step": bad,
                     "mlups": 512 * 512 * 200 * len(h) / (ms * 1e-3) / 1e6})
    for r in rows:
        ref = next(x for x in rows if x["lattice"] == r["lattice"] and x["storage"] == "f64")
        if r is not ref:
            r["v_tip_rel_diff_vs_f64"] = {k: abs(r[k] - ref[k]) / abs(ref[k])
                                          for k in ("v_tip_downstream_+x", "v_tip_upstream_-x")}
    out["thermosolutal_convection_512"] = rows
    # 3. directional Le sweep
    rows = []
    for Le in (1, 10, 100, 1000):
        wl = W.directional_saline(Le=Le)
        for prec in ("f32", "f16dev"):
            sim = lbm.Simulation(wl.params, precision=prec)
            sim.init_fields(wl.fields)
            m0 = sim.diagnostics()["M_C"]
            period = max(1, Le)
            sim.advance(2 * period)
            sim.autotune(reps=2)
            n = 200000 - 2 * period
            ms, d, bad, done = chunked(sim, n, 20000)
            sim.close()
            rows.append({"Le": Le, "N_U": Le, "storage": prec, "base_steps": 2 * period + done,
                         "front_height": float(d["tip"][1]) if bad is None else None,
                         "R_M": (d["M_C"] - m0) / m0 if bad is None else None, "nonfinite_at_base_step": bad,
                         "mlups": wl.params.nx * wl.params.ny * done / (ms * 1e-3) / 1e6})
    out["directional_1024x2048"] = rows
    # 4. large multi-dendrite
    rows = []
    for q in (5, 9):
        p, pts = W.multi_dendrite_params(8192)
        p.q_scalar = q
        sim = lbm.Simulation(p, precision="f32")
        sim.set_orientation(grain_angles_8192())
        sim.init_seed([{"kind": "circle", "x": float(x), "y": float(y), "r": 8.0} for x, y in pts], U0=0.0,
                      T0=-0.55)
        m0 = sim.diagnostics()["M_C"]
        sim.autotune(reps=3)
        ms, d, bad, done = chunked(sim, 50000, 5000)
        fused = sim.fused
        sim.close()
        ab = algo_bytes("f32", q, ori=True)
        step_bytes = ab["phase"] + ab["transfer"] + ab["scalar_U"] + ab["scalar_T"] / p.N_T + ab["flow"] / p.N_F
        nodes = p.nx * p.ny
        gbs = step_bytes * nodes * done / (ms * 1e-3) / 1e9
        peak, peak_kind = measured_peaks()
        rows.append({"lattice": "D2Q%d" % q, "storage": "f32", "base_steps": done,
                     "R_M": (d["M_C"] - m0) / m0 if bad is None else None, "nonfinite_at_base_step": bad,
                     "fused_transport": fused, "mlups": nodes * done / (ms * 1e-3) / 1e6,
                     "step_algo_GBs": gbs if not fused else None, "peak": peak,
                     "frac": gbs / peak if not fused else None, "peak_kind": peak_kind})
    out["multi_dendrite_8192"] = rows
    line = {"metric": METRIC + " (workload list, full lengths)",
            "value": rows[0]["mlups"], "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded)",
            "config": {"workload": "8192x8192 multi-dendrite, D2Q5 phase/U/T, 50 000 base steps (value); "
                                   "the other cases in the details"},
            "results": out}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="convection512", choices=["convection512", "ensemble", "sweep", "configs"],
                    help="convection512: the reported workload; ensemble: batched-ensemble measurement; "
                         "sweep: update-factor sweeps (thermal dendrite N_T, directional Le)")
    ap.add_argument("--members", type=int, default=64)
    ap.add_argument("--precision", default=None)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end pass (profiling runs)")
    ap.add_argument("--no-large", action="store_true", help="skip the 8192^2 HBM-bound measurement")
    ap.add_argument("--fusion", default="auto", choices=["auto", "on", "off"],
                    help="one fused transport launch per base step (on), one launch per stage (off), "
                         "or the autotuner's choice (auto)")
    ap.add_argument("--tile", action="append", metavar="KIND=V",
                    help="fix a kernel variant after autotuning (profiling runs): V > 0 tile height, V < 0 strip height")
    ap.add_argument("--q-scalar", type=int, default=5, choices=[9, 5],
                    help="velocities of the phase, U and T lattices: 5 (D2Q5, as the workload list states "
                         "them; default) or 9 (the paper's D2Q9)")
    ap.add_argument("--orientation", type=float, default=None,
                    help="crystal angle of the (single) grain of the main workload (profiling runs)")
    ap.add_argument("--no-alt-lattice", action="store_true",
                    help="skip the measurement on the other velocity set")
    ap.add_argument("--lattice", type=int, default=None,
                    help="lattice size override for profiling runs (the reported workload is 512)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "configs":
        return run_configs(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
