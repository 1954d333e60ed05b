"""Parity at the full sizes of the workload list, in the launch configuration
bench.py times (autotuned kernel variants, graphs, fusion as the autotuner
chooses):

* 512^2 thermosolutal + convection: element by element against the oracle
  (FP64 within 1e-10, FP32 within the linear rounding bound for the steps run);
* 1024 x 2048 directional solidification: element by element, FP64 and the
  16-bit deviation storages;
* the 64-member ensemble, batched: every member element by element (FP64);
* 8192^2 multi-dendrite (too large for the oracle as a whole): sampled
  outputs, element by element against the oracle run on windows of the same
  initial state (exact beyond the method's dependence radius), FP64, FP32
  and FP16 deviation storage.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import active, run_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2609_25670_b300 as lbm  # noqa: E402


def _bench_like(p, fields, steps, precision, warm=4):
    """Warm-up, autotune on the live state, then the rest of the steps."""
    sim = lbm.Simulation(p, precision=precision)
    sim.init_fields(fields)
    sim.advance(warm)
    sim.autotune(reps=2)
    sim.advance(steps - warm)
    out = {k: sim.field(k) for k in active(p)}
    out["diag"] = sim.diagnostics()
    sim.close()
    return out


@pytest.mark.parametrize("q", [9, 5])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 2e-4)])
def test_convection_512_full_size(prec, tol, q):
    """FP32 bound: about 20 roundings per base step, each with relative error
    below 2^-22 (the FP32 reciprocals are the hardware approximation, the
    largest per-operation error of the path), over 40 steps on values of
    order one: 40 * 20 * 2.4e-7 = 1.9e-4.  q: D2Q9 scalar lattices (the
    paper's) or D2Q5 (the five-velocity option)."""
    wl = W.thermosolutal_convection(n=512, R=8.0)
    wl.params.q_scalar = q
    steps = 40
    g = _bench_like(wl.params, wl.fields, steps, prec)
    o = run_oracle(wl.params, wl.fields, steps)
    for k in active(wl.params):
        assert np.abs(g[k] - o[k]).max() < tol, k
    assert abs(g["diag"]["M_C"] - o["diag"]["M_C"]) < (1e-12 if prec == "f64" else 1e-6) * o["diag"]["M_C"]


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f16dev", 3e-4), ("bf16dev", 3e-3)])
def test_directional_1024x2048_full_size(prec, tol):
    """Le = 10 (N_U = 10), frozen pulled temperature; 16-bit bounds: the
    deviation rounding per store (FP16 5e-6, BF16 4e-5) over 30 steps, x2."""
    wl = W.directional_saline(Le=10, nx=1024, ny=2048, y0=100.0, seed=3)
    steps = 30
    g = _bench_like(wl.params, wl.fields, steps, prec)
    o = run_oracle(wl.params, wl.fields, steps)
    for k in active(wl.params):
        assert np.abs(g[k] - o[k]).max() < tol, k


def test_ensemble_64_members_full_size_fp64():
    ms = W.ensemble_members(count=64, seed=4)
    steps = 8
    sim = lbm.Simulation([m.params for m in ms], precision="f64")
    for i, m in enumerate(ms):
        sim.init_fields(m.fields, sim=i)
    sim.advance(4)
    sim.autotune(reps=1)
    sim.advance(steps - 4)
    got = [{k: sim.field(k, sim=i) for k in active(m.params)} for i, m in enumerate(ms)]
    sim.close()
    for i, m in enumerate(ms):
        o = run_oracle(m.params, m.fields, steps)
        for k in active(m.params):
            assert np.abs(got[i][k] - o[k]).max() < 1e-10, (i, k)


def _windows(n, pts, w, m):
    """Sampling windows of an n x n lattice: (x0, y0, compare box) with the
    box in window coordinates.  Three windows centred on seeds (exact beyond
    the margin m on every side) and two on the inlet and outflow columns
    (exact up to the lattice's own boundary on that side)."""
    out = []
    for (cx, cy) in pts[:3]:
        x0 = min(max(int(cx) - w // 2, 1), n - w - 1)
        y0 = min(max(int(cy) - w // 2, 1), n - w - 1)
        out.append((x0, y0, (m, w - m, m, w - m)))
    out.append((0, n // 2 - w // 2, (0, w - m, m, w - m)))
    out.append((n - w, n // 2 - w // 2, (m, w, m, w - m)))
    return out


_ORI = {}


def _full_orientation(pts, ang, n):
    """The Voronoi grain angles of the whole n x n lattice (built once)."""
    if n not in _ORI:
        _ORI[n] = W.grain_orientation(pts, ang, 0, 0, n, n, rows=32)
    return _ORI[n]


@pytest.mark.parametrize("prec,tol,q", [("f64", 1e-10, 9), ("f32", 4e-5, 9), ("f32", 4e-5, 5), ("f16dev", 2e-4, 5)])
def test_multi_dendrite_8192_sampled_windows(prec, tol, q):
    """8192^2 multi-dendrite growth with convection (32 seeds, N = (1, 1, 4,
    2)), too large for the oracle as a whole: seeded through lbm_init_seed,
    autotuned and advanced through the period graphs as bench.py runs it,
    then compared element by element with the oracle run on 160^2 windows
    cut from the same initial state.  After k base steps a node depends only
    on the initial state within 6k nodes (pinned on the oracle by
    test_update_is_local_within_six_nodes_per_base_step), so the window's
    oracle result is the exact full-lattice result beyond that margin.
    FP32 bound: 8 steps x 20 roundings x 2^-22 (the hardware reciprocal) =
    3.8e-5 on values of order one.  q = 5: the same with D2Q5 phase, U and
    T lattices.  FP16 deviation storage (the mixed form the bench measures
    beside FP32): each store rounds deviations of order 1e-2 by up to
    2^-11, ~5e-6 a store, two stores a base step over 8 steps, x2.  Each seed's grain has its own crystal angle (Voronoi cells
    of the seeds, angles drawn in [0, pi/2)); the windows carry the same
    angles."""
    from dataclasses import replace
    n, steps, w = 8192, 8, 160
    m = 6 * steps
    p, pts = W.multi_dendrite_params(n)
    p.q_scalar = q
    ang = W.multi_dendrite_angles(len(pts))
    seeds = [{"kind": "circle", "x": float(x), "y": float(y), "r": 8.0} for x, y in pts]
    sim = lbm.Simulation(p, precision=prec)
    sim.set_orientation(_full_orientation(pts, ang, n))          # the grains' crystal frames
    sim.init_seed(seeds, U0=0.0, T0=-0.55)
    sim.autotune(reps=1)
    sim.advance(steps)
    d = sim.diagnostics()
    assert d["nonfinite"] == 0 and d["base_step"] == steps
    full = {}
    for k in active(p):
        t = torch.empty((n, n), dtype=torch.float64, device="cuda")
        sim.field(k, out=t)
        full[k] = t
    sim.close()
    for (x0, y0, (xa, xb, ya, yb)) in _windows(n, pts, w, m):
        pw = replace(p, nx=w, ny=w, tip_cx=w // 2, tip_cy=w // 2)
        fw = W.circle_seeds_window(p, pts, 8.0, x0, y0, w, w, 0.0, -0.55)
        fw["theta"] = W.grain_orientation(pts, ang, x0, y0, w, w)
        o = run_oracle(pw, fw, steps)
        for k in active(p):
            g = full[k][y0 + ya:y0 + yb, x0 + xa:x0 + xb].cpu().numpy()
            err = np.abs(g - o[k][ya:yb, xa:xb]).max()
            assert err < tol, (prec, x0, y0, k, err)
    del full
    torch.cuda.empty_cache()
