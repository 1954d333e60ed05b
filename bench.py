"""Benchmark: coupled-field MLUPS of the multirate MRT-LBM on B300.

Reported workload: large multi-dendrite thermosolutal growth with convection
on an 8192 x 8192 lattice -- phi, U, T on D2Q5 lattices and the D2Q9 flow,
32 seeds of radius 8 placed by seeded dart throwing (Poisson disc), each in a
grain of its own crystal orientation in [0, pi/2) (Voronoi cells), Le = 100,
k = 0.3, inlet velocity 0.005 from the left, outflow right, periodic
top/bottom, update factors (phi 1, U 1, T 4, flow 2) -- with FP32 storage
and arithmetic; the same workload with FP16 deviation storage (FP32
arithmetic) is measured beside it ("mixed_storage"), with its error against
the FP64 path at the same configuration.  Synthetic seeded inputs.

One step = one schedule period = 4 base steps (phase x4, transfer x4, U x4,
T x1, flow x2).  Coupled-field MLUPS = lattice nodes x base steps / s / 1e6.
The state (13.2 GB in FP32, 8.6 GB with FP16 storage) is far larger than L2, so every step streams from
HBM; each step is timed on the device with CUDA events on the library's
stream.  Also reported: the 512 x 512 thermosolutal free dendrite with forced
convection (L2-resident, flushed between steps) and the paper's D2Q9 scalar
lattices at 8192^2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only other implementation of
the method here) on the host cores, on a bounded sample of the same workload
(a window of the 8192^2 lattice around a seed, one schedule period per step).
"""
from __future__ import annotations

import argparse
import json
import math
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

N_LATTICE = 512        # the thermosolutal + convection lattice
STEP_BASE = 2          # its base steps per bench step (one schedule period)
MD_N = 8192            # the multi-dendrite lattice (the reported workload)
MD_PERIOD = 4          # its schedule period: lcm(1, 1, 4, 2) base steps
MD_RESEED_BASE_STEPS = 800   # timed steps restart from the initial state after this many base steps
METRIC = "coupled-field MLUPS"
UNIT = "MLUPS"
KINDS = ["phase", "transfer", "scalar_U", "scalar_T", "flow", "transport"]

# element sizes of the stored populations and of the macroscopic fields per
# storage precision (16-bit storage keeps FP32 macros)
POP_BYTES = {"f64": 8, "f32": 4, "f16dev": 2, "bf16dev": 2}
MACRO_BYTES = {"f64": 8, "f32": 4, "f16dev": 4, "bf16dev": 4}
# the residual plane of the compensated U macro (BF16, read and written by
# each U update) with FP32 arithmetic
U_RESIDUAL_BYTES = {"f64": 0, "f32": 4, "f16dev": 4, "bf16dev": 4}


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
        "scalar_U": moms + 5 * m + U_RESIDUAL_BYTES[prec],   # j R+W, U R+W, phi R, u R (2), residual R+W
        "scalar_T": moms + 5 * m,
        "flow": pops + 7 * m,                   # pops, phi R, (rho, ux, uy) R + W
    }



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
        b += moms + m + U_RESIDUAL_BYTES[prec]
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


def step_bytes_md(p, prec, fused, q):
    """Algorithmic bytes per node per base step of the multi-dendrite
    workload: phase and transfer every step, U every N_U-th, T every N_T-th,
    flow every N_F-th (the fused path: the phase plus the period mean of the
    fused launches)."""
    ab = algo_bytes(prec, q, ori=True)
    if fused:
        tb, _ = period_bytes(p, prec)
        return ab["phase"] / p.N_phi + tb / (2 * MD_PERIOD)
    return ((ab["phase"] + ab["transfer"]) / p.N_phi + ab["scalar_U"] / p.N_U + ab["scalar_T"] / p.N_T
            + ab["flow"] / p.N_F)


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of ncu captures
# per kernel variant, summarised in profiles/.  TRAFFIC_PER_LAUNCH_512: per
# launch on the 512^2 workload ("q<velocities of the phase, U, T lattices>:
# kind:variant"; none recorded).  TRAFFIC_PER_NODE: per node
# ("<storage>:q<velocities>:kind:variant", ":ori" for the phase update with
# grain angles), times the nodes of a launch.  Reported only while the
# time-stepping kernels' sources hash to TRAFFIC_SOURCE_SHA; after any
# change of their code the traffic is null until re-measured.
TRAFFIC_SOURCE_SHA = "faf9e2710514f844"
TRAFFIC_PER_LAUNCH_512 = {}
# one launch per kernel of the 8192^2 multi-dendrite workload (D2Q5 phase,
# U, T; grain angles), single-pass counters (profiles/
# dram_traffic_multidendrite8192_d2q5_f32_f16.md); equal to the algorithmic
# bytes within 1 %.  A 2048^2 capture keeps most of a launch's writes in the
# 126 MB L2 until after the kernel, so it undercounts them.
TRAFFIC_PER_NODE = {
    "f32:q5:flow:1016": 92.75, "f32:q5:phase:1016:ori": 52.43, "f32:q5:phase:1032:ori": 52.97,
    "f32:q5:scalar_T:1016": 36.01, "f32:q5:scalar_U:1016": 40.07, "f32:q5:transfer:1016": 23.84,
    "f16dev:q5:flow:1032": 60.75, "f16dev:q5:phase:1016:ori": 36.13, "f16dev:q5:phase:1032:ori": 36.17,
    "f16dev:q5:scalar_T:1032": 28.11, "f16dev:q5:scalar_U:1032": 32.16, "f16dev:q5:transfer:1016": 23.84,
}


# the sources of the time-stepping kernels (and of their launch geometry:
# strip and tile counts, shared-memory sizes); the initialisation, output
# and diagnostics kernels (lbm_aux.cuh) and the host library never run
# inside a timed region's kernels
TIMED_KERNEL_SOURCES = ("lbm_common.cuh", "lbm_kernels.cuh", "lbm_strip.cuh", "lbm_transport.cuh")


def kernel_source_sha():
    """Hash of the time-stepping kernels' CUDA sources with comments and
    blank space removed: a change of their code invalidates the stored
    traffic, a change of a comment does not."""
    import hashlib
    import re
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2609_25670_b300", "csrc")
    for nm in sorted(os.listdir(d)):
        if nm in TIMED_KERNEL_SOURCES:
            with open(os.path.join(d, nm)) as f:
                src = f.read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            src = re.sub(r"//[^\n]*", "", src)
            src = "\n".join(ln.rstrip() for ln in src.splitlines() if ln.strip())
            h.update(nm.encode() + b"\0" + src.encode())
    return h.hexdigest()[:16]


def lattice_label(p):
    return "phi/U/T/flow on D2Q9" if getattr(p, "q_scalar", 9) != 5 else "phi/U/T on D2Q5, flow on D2Q9"


STORAGE_LABEL = {"f64": "FP64", "f32": "FP32", "f16dev": "FP32 arithmetic, FP16 deviation storage",
                 "bf16dev": "FP32 arithmetic, BF16 deviation storage"}


def workload_label(p, prec="f32"):
    return (f"thermosolutal free dendrite + forced convection, {p.nx}x{p.ny}, {lattice_label(p)}, "
            f"N=({p.N_phi},{p.N_U},{p.N_T},{p.N_F}), {STORAGE_LABEL[prec]}")


def md_label(p, prec="f32"):
    return (f"{p.nx}x{p.ny} multi-dendrite thermosolutal growth with convection, 32 Poisson-disc seeds in "
            f"grains of random crystal orientation, Le=100, k=0.3, u_in=0.005, "
            f"N=({p.N_phi},{p.N_U},{p.N_T},{p.N_F}), {lattice_label(p)}, {STORAGE_LABEL[prec]}")


def workload(n=None, q=5):
    wl = W.thermosolutal_convection(n=n or N_LATTICE, R=8.0)
    wl.params.q_scalar = q
    return wl


def md_workload(n=None, q=5):
    """Parameters and seed centres of the multi-dendrite workload (n x n)."""
    p, pts = W.multi_dendrite_params(n or MD_N)
    p.q_scalar = q
    return p, pts


def md_seeds(pts):
    return [{"kind": "circle", "x": float(x), "y": float(y), "r": 8.0} for x, y in pts]


_GRAINS = {}


def grain_angles(n=MD_N):
    """Voronoi grain angles of the n x n multi-dendrite lattice (one crystal
    angle per seed, drawn in [0, pi/2)); built once per process and size."""
    if n not in _GRAINS:
        p, pts = W.multi_dendrite_params(n)
        _GRAINS[n] = W.grain_orientation(pts, W.multi_dendrite_angles(len(pts)), 0, 0, n, n, rows=32)
    return _GRAINS[n]


def grain_angles_8192():
    return grain_angles(8192)


def md_window(q, w, seed_index=0):
    """A bounded sample of the multi-dendrite workload for the CPU oracle: the
    w x w window of the 8192^2 lattice centred on one seed, with the
    lattice's physics, boundary kinds, grain angles and initial fields read on
    the window.  Returns (params, fields, description)."""
    p, pts = md_workload(MD_N, q)
    cx, cy = pts[seed_index]
    x0 = int(min(max(0, round(cx) - w // 2), MD_N - w))
    y0 = int(min(max(0, round(cy) - w // 2), MD_N - w))
    theta = W.grain_orientation(pts, W.multi_dendrite_angles(len(pts)), x0, y0, w, w)
    fields = W.circle_seeds_window(p, pts, 8.0, x0, y0, w, w, U0=0.0, T0=-0.55)
    fields["theta"] = theta
    p.nx = p.ny = w
    p.tip_cx, p.tip_cy = int(round(cx)) - x0, int(round(cy)) - y0
    return p, fields, "%dx%d window of the 8192^2 lattice at (%d, %d) around seed %d" % (w, w, x0, y0, seed_index)


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
    """`steps` bench steps on `stream`: an L2 flush (untimed, skipped when
    `flush` is None), then one advance() between two CUDA events.  A bounded
    sleep kernel queued first holds the stream while the host enqueues every
    step, so the device runs the steps back to back from its queue and a
    pause of the host thread (scheduling, the clock sampler's queries) cannot
    fall inside a timed step.  The gate is checked: an event recorded behind
    the sleep must still be pending once the host has enqueued the last
    step.  If the device got there first (a host slower than the gate), the
    times hold host gaps: the state is re-initialised with `reinit` and the
    steps are timed again behind a gate four times longer, at most three
    attempts in all.  Returns (the per-step times in ms, whether the gate
    held)."""
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
                if flush is not None:
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


VECTOR_STRIP_HEIGHTS = (8, 16, 32)


def refine_vector_tiles(sim, torch, tiles, period, steps=8):
    """Refinement of the autotuner's choice among the vector-strip heights
    (variants 1000 + H) on a lattice larger than L2: lbm_autotune times a
    kind's launches back to back, each as the only kernel in flight, which
    ranks close variants differently from a bench step where every kind
    follows another.  For each kind that runs a vector strip, time whole
    schedule periods (graph replays, the median of `steps`) for each strip
    height and keep the fastest.  The live state is advanced by these
    periods; the caller re-initialises before its timed region.  Returns the
    refined choices."""
    stream = sim.stream
    kinds = [k for k in KINDS if k != "transport" and tiles.get(k, 0) > 1000]
    for kind in kinds:
        best, best_v = None, tiles[kind]
        for v in sorted({1000 + h for h in VECTOR_STRIP_HEIGHTS} | {tiles[kind]}):
            sim.set_tile(kind, v)
            sim.advance(period)                       # capture with this variant
            torch.cuda.synchronize()
            ms = sorted(gated_steps(torch, stream, None, lambda: sim.advance(period), steps)[0])[steps // 2]
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


def cpu_baseline(target_s: float = 12.0, q: int = 5, w: int = 512):
    """The FP64 oracle on the host cores, on a bounded sample of the
    multi-dendrite workload: a w x w window of the 8192^2 lattice around a
    seed (the lattice's physics and grain angles), advanced for as many
    schedule periods as fit in ~target_s; then the next periods on one
    thread."""
    import oracle
    p, fields, what = md_window(q, w)
    o = oracle.Oracle(p, fields)
    t0 = time.perf_counter()
    steps = 0
    while (time.perf_counter() - t0) < target_s:
        o.advance(MD_PERIOD)
        steps += MD_PERIOD
    dt = time.perf_counter() - t0
    cores = oracle.num_threads()
    oracle.set_threads(1)
    t1, steps1 = time.perf_counter(), 0
    while (time.perf_counter() - t1) < target_s / 3:
        o.advance(MD_PERIOD)
        steps1 += MD_PERIOD
    dt1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    o.close()
    nodes = p.nx * p.ny
    return {"value": nodes * steps / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "value_1_thread": nodes * steps1 / dt1 / 1e6,
            "sample": "%s (%s, FP64 oracle), the first %d base steps (%.1f s); 1 thread: the next %d base "
                      "steps (%.1f s)" % (what, lattice_label(p), steps, dt, steps1, dt1)}


def run_reference(args):
    """The FP64 oracle on the host cores on the reported workload's metric:
    each step one schedule period (4 base steps) of a 256 x 256 window of the
    8192^2 multi-dendrite lattice around a seed."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    p, fields, what = md_window(args.q_scalar, 256)
    o = oracle.Oracle(p, fields)
    for _ in range(args.warmup):
        o.advance(MD_PERIOD)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.advance(MD_PERIOD)
    dt = time.perf_counter() - t0
    nodes = p.nx * p.ny
    v = nodes * MD_PERIOD * args.steps / dt / 1e6
    full, _ = md_workload(MD_N, args.q_scalar)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": md_label(full, args.precision or "f32"), "base_steps_per_step": MD_PERIOD},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "each step: one schedule period (%d base steps) of the %s" % (
                                 MD_PERIOD, what)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def timed_md_steps(torch, sim, steps, reinit, nvtx=False):
    """`steps` schedule periods, each between two CUDA events on the library
    stream; every MD_RESEED_BASE_STEPS base steps (untimed, between events)
    the state restarts from the initial fields, so every timed step lies in
    the workload's first base steps.  nvtx: the first step's launches inside
    an NVTX range "lbm_period" (profiling runs select them by it).  Returns
    per-step milliseconds."""
    chunk = max(1, MD_RESEED_BASE_STEPS // MD_PERIOD)
    times = []
    done = 0
    while done < steps:
        n = min(chunk, steps - done)
        if done:
            reinit()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for k in range(n):
            with torch.cuda.stream(sim.stream):
                ev[k][0].record(sim.stream)
            mark = nvtx and done == 0 and k == 0
            if mark:
                torch.cuda.nvtx.range_push("lbm_period")
            sim.advance(MD_PERIOD)
            if mark:
                torch.cuda.nvtx.range_pop()
            with torch.cuda.stream(sim.stream):
                ev[k][1].record(sim.stream)
        torch.cuda.synchronize()
        times += [a.elapsed_time(b) for a, b in ev]
        done += n
    return times


def measure_md(args, torch, lbm, local, dev, prec, q, world=1, with_e2e=False):
    """One multi-dendrite measurement (n x n, storage `prec`, velocities q of
    the phase, U, T lattices): seeded through lbm_init_seed, autotuned on the
    live state, `args.steps` timed schedule periods from the initial state,
    then the same steps again with the dominant kernel's CUDA events inside
    the graphs for its launch duration; with_e2e adds the end-to-end pass
    through the public API with pinned host buffers."""
    p, pts = md_workload(args.lattice, q)
    nodes = p.nx * p.ny
    sim = lbm.Simulation(p, precision=prec)
    if args.fusion != "auto":
        sim.set_fusion(args.fusion == "on")
    if args.no_graphs:
        sim.set_graphs(False)
    sim.set_orientation(grain_angles(p.nx))          # each grain in its own crystal frame
    seeds = md_seeds(pts)

    def reinit():
        sim.init_seed(seeds, U0=0.0, T0=-0.55)

    reinit()
    for _ in range(max(args.warmup, 3)):
        sim.advance(MD_PERIOD)
    if args.no_autotune:                    # profiling runs: the variants --tile fixes, the defaults otherwise
        tiles = {k: 0 for k in KINDS}
    else:
        tiles = sim.autotune(reps=3)
        tiles = refine_vector_tiles(sim, torch, tiles, MD_PERIOD)
    for spec in args.tile or []:            # fixed kernel variants (profiling runs)
        kind, v = spec.split("=")
        sim.set_tile(kind, int(v))
        tiles[kind] = int(v)
    sim.advance(MD_PERIOD)
    sim.timing_enable(KINDS)                # untimed pre-pass: which kind dominates
    sim.advance(2 * MD_PERIOD)
    pre = sim.timing_read(reset=True)
    dom = max(KINDS, key=lambda k: pre[k][0])
    sim.timing_enable([])
    sim.advance(MD_PERIOD)                  # recapture without timing nodes, untimed
    reinit()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = sim.launch_counts()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    w0 = time.perf_counter()
    times = timed_md_steps(torch, sim, args.steps, reinit, nvtx=args.nvtx)
    wall = time.perf_counter() - w0
    clk = clocks.stop()
    launches1 = sim.launch_counts()
    if world > 1:
        torch.distributed.barrier()
    # launches of the re-seeding between chunks are not inside timed steps
    reseeds = (args.steps - 1) // max(1, MD_RESEED_BASE_STEPS // MD_PERIOD)
    gpu_launches = int(sum(launches1[k] - launches0[k] for k in launches1 if k != "init"))
    ms = sum(times)
    ms_max = max_over_ranks(ms, dev)
    fused = sim.fused
    # the dominant kernel's own launches, timed inside the graphs
    sim.timing_enable([dom])
    sim.advance(MD_PERIOD)
    sim.timing_read(reset=True)
    reinit()
    n_dom = min(args.steps, 50)
    ms_instr = sum(timed_md_steps(torch, sim, n_dom, reinit))
    kt = sim.timing_read(reset=True)
    sim.timing_enable([])
    finite = not sim.diagnostics()["nonfinite"]

    peak, peak_kind = measured_peaks()
    sb = step_bytes_md(p, prec, fused, q)
    gbs = sb * nodes * MD_PERIOD * args.steps / (ms * 1e-3) / 1e9
    dom_algo = algo_bytes(prec, q, ori=True)
    tb, tn = period_bytes(p, prec)
    dom_algo["transport"] = tb / max(tn, 1)
    avg_s = kt[dom][0] * 1e-3 / max(kt[dom][1], 1)
    dom_gbs = dom_algo[dom] * nodes / avg_s / 1e9
    traffic, traffic_note = None, None
    key = "%s:q%d:%s:%d%s" % (prec, q, dom, tiles[dom], ":ori" if dom == "phase" else "")
    if TRAFFIC_SOURCE_SHA == kernel_source_sha() and key in TRAFFIC_PER_NODE:
        traffic = TRAFFIC_PER_NODE[key] * nodes
        traffic_note = "ncu capture of one launch of this variant on the 8192^2 lattice (single-pass counters)"
    out = {
        "workload": md_label(p, prec), "storage": prec, "nodes": nodes,
        "value": job_throughput(nodes, MD_PERIOD, args.steps, world, ms_max), "unit": UNIT,
        "ms_per_step": ms_max / args.steps, "ms_per_step_median": statistics.median(times),
        "base_steps_per_step": MD_PERIOD, "fused_transport": fused, "gpu_launches": gpu_launches,
        "reseeds_between_timed_steps": reseeds, "wall_s_timed_region": wall,
        "step": {"algo_bytes_per_node_per_base_step": sb, "achieved": gbs, "peak": peak, "unit": "GB/s",
                 "frac": gbs / peak, "peak_kind": peak_kind},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": dom_gbs, "peak": peak, "unit": "GB/s",
                     "frac": dom_gbs / peak, "traffic": traffic, "traffic_note": traffic_note,
                     "peak_kind": peak_kind, "algo_bytes_per_node": dom_algo[dom],
                     "avg_launch_us": avg_s * 1e6, "launches_timed": kt[dom][1],
                     "timed_in": "a second timed region of %d steps with the kernel's CUDA events inside the "
                                 "graphs (%.3f ms per step there against %.3f without them)" % (
                                     n_dom, ms_instr / n_dom, ms / args.steps)},
        "kernel_avg_us_prepass": {k: pre[k][0] / max(pre[k][1], 1) * 1e3 for k in KINDS},
        "tiles": {k: tiles[k] for k in KINDS}, "clocks": clk,
        "state_finite_after_timed_regions": finite,
        "l2": "inputs larger than L2 (%.1f GB of device state)" % (sim.device_bytes() / 1e9),
    }
    if with_e2e and not args.no_e2e:
        out["e2e"] = md_e2e(args, torch, sim, p, pts, world)
    sim.close()
    return out


def md_e2e(args, torch, sim, p, pts, world):
    """End to end through the public API with host buffers, each step:
    lbm_init_seed from the host list of the workload's seeds (the fields are
    generated on the device), lbm_advance of one schedule period, lbm_fields
    of phi (the arithmetic type) into one of two device buffers, and that
    buffer's copy into pinned host memory on a second stream, so that step
    k's copy to the host overlaps step k + 1's work on the device (a buffer
    is reused only after its copy has completed).  Host time over the steps,
    from a synchronised device to the completion of the last copy, with a
    barrier under torchrun on both sides."""
    seeds = md_seeds(pts)
    dt_ = torch.float64 if sim.precision == "f64" else torch.float32
    stage = [torch.empty((p.ny, p.nx), dtype=dt_, device="cuda") for _ in range(2)]
    host = [torch.empty((p.ny, p.nx), dtype=dt_).pin_memory() for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    done = [None, None]

    def step(k):
        b = k % 2
        if done[b] is not None:
            done[b].synchronize()                  # the copy out of stage[b] two steps ago has completed
        sim.init_seed(seeds, U0=0.0, T0=-0.55)
        sim.advance(MD_PERIOD)
        sim.field("phi", out=stage[b], as_f64=False)
        copy_stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(copy_stream):
            host[b].copy_(stage[b], non_blocking=True)
            done[b] = torch.cuda.Event()
            done[b].record(copy_stream)

    steps = max(3, min(args.steps, 100))          # the device-timed step count; the last copy is the only one not overlapped
    for k in range(2):                             # untimed (first touch of the pinned pages)
        step(k)
    torch.cuda.synchronize()
    done = [None, None]
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for k in range(steps):
        step(k)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    dt = time.perf_counter() - t0
    dt = max_over_ranks(dt)
    nodes = p.nx * p.ny
    seed_bytes = len(seeds) * 48                  # lbm_seed: kind, reserved, five doubles
    return {"value": nodes * MD_PERIOD * steps * world / dt / 1e6, "unit": UNIT,
            "h2d_bytes_per_step": seed_bytes, "d2h_bytes_per_step": host[0].numel() * host[0].element_size(),
            "steps": steps, "ms_per_step": dt * 1e3 / steps,
            "calls": "lbm_init_seed(%d host seeds; fields generated on the device) + lbm_advance(4) + "
                     "lbm_fields(phi -> device buffer, %s) + its copy to pinned host memory on a second stream "
                     "(overlapping the next step) per step" % (len(seeds), "FP64" if sim.precision == "f64" else "FP32")}


def md_accuracy(args, torch, lbm, dev, q, precs=("f32", "f16dev"), base_steps=1000):
    """Error of the FP32 and 16-bit storage forms against the FP64 path on the
    multi-dendrite configuration (the FP64 path itself matches the oracle
    within 1e-10 in the parity tests): max-abs phi, U, T after `base_steps`
    base steps, and the difference of the relative solute drift
    R_M = (M_C - M_C(0)) / M_C(0).  On the workload's stable variant
    (workloads.stable_variant: N = (2, 2, 4, 2), D_S raised so that every
    relaxation time is >= 0.52): the listed instance's phase relaxation time
    0.515 (tau0 = 800) lets rounding grow into a non-finite field within a
    few thousand base steps, so its FP32-FP64 difference measures that growth
    rather than the storage."""
    p, pts = md_workload(args.lattice, q)
    W.stable_variant(p)
    seeds = md_seeds(pts)
    res = {}
    ref = None
    for prec in ("f64",) + tuple(precs):
        sim = lbm.Simulation(p, precision=prec)
        sim.set_orientation(grain_angles(p.nx))
        sim.init_seed(seeds, U0=0.0, T0=-0.55)
        m0 = sim.diagnostics()["M_C"]
        sim.advance(base_steps)
        d = sim.diagnostics()
        fl = {}
        for k in ("phi", "U", "T"):
            t = torch.empty((p.ny, p.nx), dtype=torch.float64, device=dev)
            sim.field(k, out=t)
            fl[k] = t
        torch.cuda.synchronize()
        sim.close()
        rm = (d["M_C"] - m0) / m0
        if ref is None:
            ref = (fl, rm)
            res["f64"] = {"R_M": rm}
            continue
        res[prec] = {"max_abs_err_vs_f64": {k: float((fl[k] - ref[0][k]).abs().max()) for k in fl},
                     "R_M": rm, "R_M_diff_vs_f64": abs(rm - ref[1])}
        del fl
    del ref
    torch.cuda.empty_cache()
    res["base_steps"] = base_steps
    res["workload"] = "stable variant: N=(%d,%d,%d,%d), D_S/D_L=%.2f" % (p.N_phi, p.N_U, p.N_T, p.N_F, p.DS / p.DL)
    return res


def run_ours(args):
    import torch
    import paper_2609_25670_b300 as lbm

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    prec = args.precision or "f32"
    q = args.q_scalar
    main = measure_md(args, torch, lbm, local, dev, prec, q, world=world, with_e2e=True)
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "f64" else "f32",
            "data": "synthetic (seeded)",
            "config": {"workload": main["workload"], "storage": prec, "base_steps_per_step": MD_PERIOD,
                       "fused_transport": main["fused_transport"], "l2": main["l2"],
                       "parallelism": "replicas" if world > 1 else "1 GPU"},
            "roofline": main["roofline"], "step_roofline": main["step"],
            "gpu_launches": main["gpu_launches"], "clocks": main["clocks"], "e2e": main.get("e2e"),
            "timing": "CUDA events around each step's lbm_advance on the library stream; every %d timed steps "
                      "the state restarts from the initial fields between steps (untimed)" % max(
                          1, MD_RESEED_BASE_STEPS // MD_PERIOD),
            "details": {k: main[k] for k in ("ms_per_step_median", "kernel_avg_us_prepass", "tiles",
                                            "wall_s_timed_region", "state_finite_after_timed_regions",
                                            "reseeds_between_timed_steps", "nodes")},
        }
    if world == 1 and not args.no_extra:
        torch.cuda.empty_cache()
        mixed = measure_md(args, torch, lbm, local, dev, "f16dev", q)
        torch.cuda.empty_cache()
        mixed["speedup_vs_fp32"] = mixed["value"] / main["value"]
        if not args.no_accuracy:
            mixed["accuracy"] = md_accuracy(args, torch, lbm, dev, q)
        line["mixed_storage"] = mixed
        torch.cuda.empty_cache()
        line["d2q%d" % (9 if q == 5 else 5)] = {
            "multi_dendrite": measure_md(args, torch, lbm, local, dev, prec, 9 if q == 5 else 5)}
        torch.cuda.empty_cache()
        line["convection_512"] = measure_convection512(args, torch, lbm, local, dev, q)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(q=q)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def measure_convection512(args, torch, lbm, local, dev, q, print_line=False):
    """The 512^2 thermosolutal free dendrite with forced convection (its
    state fits L2): L2 flushed (512 MiB write) before every step, steps of
    one schedule period (2 base steps) queued behind a checked sleep gate,
    each timed with CUDA events; then the dominant kernel's launch time from
    a second timed region with its events inside the graphs."""
    wl = workload(N_LATTICE if args.workload != "convection512" else args.lattice, q)
    p = wl.params
    nodes = p.nx * p.ny
    prec = args.precision or "f32"
    sim = lbm.Simulation(p, precision=prec)
    if args.fusion != "auto":
        sim.set_fusion(args.fusion == "on")
    sim.init_fields(wl.fields)
    stream = sim.stream
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 3)):
        sim.advance(STEP_BASE)
    tiles = sim.autotune(reps=10)
    if nodes * 200 < 126 * 2 ** 20 and not args.tile:     # state in L2: refine on flushed steps
        tiles = refine_tiles(sim, torch, flush, tiles)
    for spec in args.tile or []:
        kind, v = spec.split("=")
        sim.set_tile(kind, int(v))
        tiles[kind] = int(v)
    sim.advance(STEP_BASE)
    tb, tn = period_bytes(p, prec)
    algo = algo_bytes(prec, q)
    algo["transport"] = tb / max(tn, 1)
    sim.timing_enable(KINDS)
    for _ in range(10):
        with torch.cuda.stream(stream):
            flush.fill_(0.0)
        sim.advance(STEP_BASE)
    pre = sim.timing_read(reset=True)
    dom = max(KINDS, key=lambda k: pre[k][0])
    steps = min(args.steps, 400)        # within the workload's first 800 base steps

    def timed_region():
        torch.cuda.synchronize()
        t, held = gated_steps(torch, stream, flush, lambda: sim.advance(STEP_BASE), steps,
                              reinit=lambda: sim.init_fields(wl.fields))
        return sum(t), held

    sim.timing_enable([])
    sim.advance(STEP_BASE)
    sim.init_fields(wl.fields)
    l0 = sim.launch_counts()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    ms, held = timed_region()
    clk = clocks.stop()
    l1 = sim.launch_counts()
    sim.timing_enable([dom])
    sim.advance(STEP_BASE)
    sim.timing_read(reset=True)
    sim.init_fields(wl.fields)
    ms_instr, _ = timed_region()
    kt = sim.timing_read(reset=True)
    sim.timing_enable([])
    finite = not sim.diagnostics()["nonfinite"]
    fused = sim.fused
    sim.close()
    del flush
    dom_ms, dom_n = kt[dom]
    avg_s = dom_ms * 1e-3 / max(dom_n, 1)
    peak, peak_kind = measured_peaks()
    achieved = algo[dom] * nodes / avg_s / 1e9
    traffic = None
    if prec == "f32" and TRAFFIC_SOURCE_SHA == kernel_source_sha():
        traffic = TRAFFIC_PER_LAUNCH_512.get("q%d:%s:%d" % (q, dom, tiles[dom]))
    return {"workload": workload_label(p, prec), "value": nodes * STEP_BASE * steps / (ms * 1e-3) / 1e6,
            "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "base_steps_per_step": STEP_BASE,
            "gate_held": held, "fused_transport": fused, "gpu_launches": int(sum(l1[k] - l0[k] for k in l1)),
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "algo_bytes_per_node": algo[dom], "avg_launch_us": avg_s * 1e6,
                         "launches_timed": dom_n,
                         "note": "the state (~51 MB) fits L2: the fraction is algorithmic bytes over time, "
                                 "not DRAM throughput"},
            "kernel_avg_us_prepass": {k: pre[k][0] / max(pre[k][1], 1) * 1e3 for k in KINDS},
            "tiles": {k: tiles[k] for k in KINDS}, "clocks": clk,
            "l2": "flushed between steps (512 MiB write)", "state_finite_after_timed_region": finite,
            "timed_in": "%.1f us per step with the dominant kernel's events in the graphs against %.1f without" % (
                ms_instr * 1e3 / steps, ms * 1e3 / steps)}


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
      D2Q5, FP32 and FP16 storage: R_M and the step-level algorithmic HBM
      throughput.
    The 512^2, directional and multi-dendrite cases run both as listed and as
    their stable variant (workloads.stable_variant: update factors and D_S
    chosen so that every relaxation time is >= 0.52, as the paper keeps them
    in range).  A run whose fields turn non-finite stops there and reports
    the base step of the first diagnostics call that saw it."""
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
    # 2. thermosolutal + convection: the listed instance and its stable variant
    def variant_params(p, v):
        if v == "stable":
            W.stable_variant(p)
        return p

    def label(p):
        return "N=(%d,%d,%d,%d), D_S/D_L=%.3g, tau_U=(%.3f liquid, %.3f solid)" % (
            p.N_phi, p.N_U, p.N_T, p.N_F, p.DS / p.DL, W.tau_U(p, -1.0), W.tau_U(p, 1.0))

    rows = []
    for v in ("listed", "stable"):
        for q, prec in ((9, "f64"), (9, "f32"), (5, "f64"), (5, "f32")):
            wl = W.thermosolutal_convection(n=512, R=8.0)
            wl.params.q_scalar = q
            variant_params(wl.params, v)
            sim = lbm.Simulation(wl.params, precision=prec)
            sim.init_fields(wl.fields)
            sim.autotune(reps=3)                             # on the live state, which it leaves unchanged
            h, ms, d, bad = history(sim, 20000, 200)         # 100 samples, the last at step 20 000
            sim.close()
            m = min(10, len(h) - 1)
            v_tip = (h[-1] - h[-1 - m]) / (m * 200)         # the last 2000 finite base steps (fewer if cut short)
            rows.append({"variant": v, "params": label(wl.params), "lattice": "D2Q%d" % q, "storage": prec,
                         "base_steps": 200 * len(h), "v_tip_downstream_+x": float(v_tip[0]),
                         "v_tip_upstream_-x": float(v_tip[2]), "v_tip_+y": float(v_tip[1]),
                         "v_tip_-y": float(v_tip[3]), "tips_last": h[-1].tolist(),
                         "R_M": d["R_M"] if bad is None else None, "nonfinite_at_base_step": bad,
                         "mlups": 512 * 512 * 200 * len(h) / (ms * 1e-3) / 1e6})
    for r in rows:
        ref = next(x for x in rows if x["lattice"] == r["lattice"] and x["variant"] == r["variant"]
                   and x["storage"] == "f64")
        if r is not ref and r["nonfinite_at_base_step"] is None and ref["nonfinite_at_base_step"] is None:
            r["v_tip_rel_diff_vs_f64"] = {k: abs(r[k] - ref[k]) / abs(ref[k])
                                          for k in ("v_tip_downstream_+x", "v_tip_upstream_-x")}
            r["R_M_diff_vs_f64"] = abs(r["R_M"] - ref["R_M"])
    out["thermosolutal_convection_512"] = rows
    # 3. directional Le sweep
    rows = []
    for v in ("listed", "stable"):
        for Le in (1, 10, 100, 1000):
            wl = W.directional_saline(Le=Le)
            variant_params(wl.params, v)
            for prec in ("f32", "f16dev"):
                sim = lbm.Simulation(wl.params, precision=prec)
                sim.init_fields(wl.fields)
                period = max(1, wl.params.N_U)
                sim.advance(2 * period)
                sim.autotune(reps=2)
                n = 200000 - 2 * period
                ms, d, bad, done = chunked(sim, n, 20000)
                sim.close()
                rows.append({"variant": v, "params": label(wl.params), "Le": Le, "storage": prec,
                             "base_steps": 2 * period + done,
                             "front_height": float(d["tip"][1]) if bad is None else None,
                             "R_M": d["R_M"] if bad is None else None, "nonfinite_at_base_step": bad,
                             "mlups": wl.params.nx * wl.params.ny * done / (ms * 1e-3) / 1e6})
    out["directional_1024x2048"] = rows
    # 4. large multi-dendrite (D2Q5 lattices; the listed instance and the stable variant, FP32 and FP16)
    rows = []
    for v, prec in (("listed", "f32"), ("stable", "f32"), ("stable", "f16dev")):
        p, pts = W.multi_dendrite_params(8192)
        p.q_scalar = 5
        variant_params(p, v)
        sim = lbm.Simulation(p, precision=prec)
        sim.set_orientation(grain_angles_8192())
        sim.init_seed([{"kind": "circle", "x": float(x), "y": float(y), "r": 8.0} for x, y in pts], U0=0.0,
                      T0=-0.55)
        sim.autotune(reps=3)
        ms, d, bad, done = chunked(sim, 50000, 5000)
        fused = sim.fused
        sim.close()
        nodes = p.nx * p.ny
        step_bytes = step_bytes_md(p, prec, fused, 5)
        gbs = step_bytes * nodes * done / (ms * 1e-3) / 1e9
        peak, peak_kind = measured_peaks()
        rows.append({"variant": v, "params": label(p), "lattice": "D2Q5", "storage": prec, "base_steps": done,
                     "R_M": d["R_M"] if bad is None else None, "nonfinite_at_base_step": bad,
                     "fused_transport": fused, "mlups": nodes * done / (ms * 1e-3) / 1e6,
                     "step_algo_GBs": gbs, "peak": peak, "frac": gbs / peak, "peak_kind": peak_kind})
    out["multi_dendrite_8192"] = rows
    line = {"metric": METRIC + " (workload list, full lengths)",
            "value": rows[0]["mlups"], "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded)",
            "config": {"workload": "8192x8192 multi-dendrite, D2Q5 phase/U/T, listed instance, FP32, up to 50 000 "
                                   "base steps (value); stable variants and the other cases in the details"},
            "results": out}
    print(json.dumps(line), flush=True)
    return 0


def run_ablation(args):
    """Source-coupling ablation (Sec. 4.4): the directional saline-water case
    with the evolving temperature (1000 x 1000, Table 1, N_U = Le) at
    Le in {1, 10, 100}, instantaneous against accumulated coupling, each
    advanced to `--ablation-steps` base steps (100 000 by default: the paper
    reports the accumulated Le = 100 run non-finite at 0.0532 ms = 26 600
    base steps, the instantaneous ones stable to 1e7).  Every `--ablation-every` base steps: S_phi and J_U (maxima
    since the previous sample), R_M; a run stops at the first sample that
    sees a non-finite field and reports that base step."""
    import torch
    import paper_2609_25670_b300 as lbm
    prec = args.precision or "f32"
    total, every = args.ablation_steps, args.ablation_every
    runs = []
    ms_total, nodes_steps = 0.0, 0
    for Le in (1, 10, 100):
        for coupling in ("instantaneous", "accumulated"):
            wl = W.directional_evolving_T(Le=Le)
            wl.params.accumulated = coupling == "accumulated"
            sim = lbm.Simulation(wl.params, precision=prec)
            sim.init_fields(wl.fields)
            m0 = sim.diagnostics()["M_C"]
            hist, bad, done, ms = [], None, 0, 0.0
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            while done < total:
                n = min(every, total - done)
                with torch.cuda.stream(sim.stream):
                    e0.record(sim.stream)
                sim.advance(n)
                with torch.cuda.stream(sim.stream):
                    e1.record(sim.stream)
                d = sim.diagnostics()
                ms += e0.elapsed_time(e1)
                done += n
                if d["nonfinite"]:
                    bad = done
                    break
                hist.append((done, d["S_phi"], d["J_U"], (d["M_C"] - m0) / m0))
            sim.close()
            ms_total += ms
            nodes_steps += wl.params.nx * wl.params.ny * done
            h = np.asarray(hist) if hist else np.zeros((0, 4))
            js = h[:, 2] if len(h) else np.zeros(1)
            runs.append({"Le": Le, "N_U": Le, "coupling": coupling, "base_steps": done,
                         "nonfinite_at_base_step": bad,
                         "max_S_phi": float(h[:, 1].max()) if len(h) else None,
                         "max_J_U": float(js.max()), "median_J_U": float(np.median(js)),
                         "J_U_pulse_ratio": float(js.max() / max(np.median(js), 1e-300)),
                         "R_M_last": float(h[-1, 3]) if len(h) else None,
                         "mlups": wl.params.nx * wl.params.ny * done / (ms * 1e-3) / 1e6,
                         "history_every_%d" % every: [[int(a), float(b), float(c), float(r)] for a, b, c, r in h]})
    inst100 = next(r for r in runs if r["Le"] == 100 and r["coupling"] == "instantaneous")
    line = {"metric": METRIC + " (source-coupling ablation)", "value": inst100["mlups"], "unit": UNIT,
            "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == "f64" else "f32", "data": "synthetic (seeded)",
            "config": {"workload": "Sec. 4.4 directional saline water with evolving T, 1000x1000, N_U = Le, "
                                   "instantaneous vs accumulated coupling, %d base steps, samples every %d" % (
                                       total, every), "storage": prec},
            "summary": {"%s_Le%d" % (r["coupling"], r["Le"]): {k: r[k] for k in (
                "nonfinite_at_base_step", "max_S_phi", "max_J_U", "J_U_pulse_ratio", "R_M_last")} for r in runs},
            "runs": runs}
    print(json.dumps(line), flush=True)
    return 0


def run_convection512(args):
    """The 512^2 thermosolutal + convection measurement alone (profiling runs:
    --lattice sets its size)."""
    import torch
    import paper_2609_25670_b300 as lbm
    dev = torch.device("cuda", torch.cuda.current_device())
    r = measure_convection512(args, torch, lbm, 0, dev, args.q_scalar)
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": r["steps"],
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if (args.precision or "f32") == "f64" else "f32",
            "data": "synthetic (seeded)", "config": {"workload": r["workload"], "l2": r["l2"]},
            "roofline": r["roofline"], "gpu_launches": r["gpu_launches"], "clocks": r["clocks"], "details": r}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="multidendrite8192",
                    choices=["multidendrite8192", "convection512", "ensemble", "sweep", "configs", "ablation"],
                    help="multidendrite8192: the reported workload (with the FP16 arm, the D2Q9 lattices and "
                         "the 512^2 case as extra keys); convection512: the 512^2 case alone; ensemble: "
                         "batched-ensemble measurement; sweep: update-factor sweeps; configs: the workload list "
                         "at its stated lengths; ablation: the source-coupling ablation")
    ap.add_argument("--members", type=int, default=64)
    ap.add_argument("--ablation-steps", type=int, default=100000)
    ap.add_argument("--ablation-every", type=int, default=200)
    ap.add_argument("--precision", default=None)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end pass (profiling runs)")
    ap.add_argument("--no-extra", action="store_true",
                    help="only the reported measurement (no FP16 arm, other lattice or 512^2 case)")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the FP64 comparison of the FP16 arm")
    ap.add_argument("--fusion", default="auto", choices=["auto", "on", "off"],
                    help="one fused transport launch per base step (on), one launch per stage (off), "
                         "or the autotuner's choice (auto)")
    ap.add_argument("--tile", action="append", metavar="KIND=V",
                    help="fix a kernel variant after autotuning (profiling runs): V > 0 tile height, V < 0 strip "
                         "height, 1000 + H vector strip height")
    ap.add_argument("--q-scalar", type=int, default=5, choices=[9, 5],
                    help="velocities of the phase, U and T lattices: 5 (D2Q5, as the workload list states "
                         "them; default) or 9 (the paper's D2Q9)")
    ap.add_argument("--nvtx", action="store_true",
                    help="profiling runs: the first timed step's launches inside an NVTX range 'lbm_period'")
    ap.add_argument("--no-graphs", action="store_true", help="profiling runs: plain stream launches, no CUDA graphs")
    ap.add_argument("--no-autotune", action="store_true", help="profiling runs: no autotuning (use --tile)")
    ap.add_argument("--lattice", type=int, default=None,
                    help="lattice size override for profiling runs (reported: 8192, or 512 for convection512)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "configs":
        return run_configs(args)
    if args.workload == "ablation":
        return run_ablation(args)
    if args.workload == "convection512":
        return run_convection512(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
