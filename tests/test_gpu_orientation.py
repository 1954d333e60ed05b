"""Grains of different crystal orientation (the multi-dendrite case): Eqs. 2-3
evaluated in each grain's turned crystal frame, through the C ABI, against
the FP64 oracle given the same orientation field, on every phase kernel
variant (shared-memory tiles, vector strips and their frame) and both
velocity sets.  Tolerances as elsewhere: FP64 within 1e-11 for short runs,
FP32 within the linear rounding bound."""
import math

import numpy as np
import pytest

import workloads as W
from gpu_helpers import active, run_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2609_25670_b300 as lbm  # noqa: E402

KINDS = ("phase", "transfer", "scalar_U", "scalar_T", "flow")


def _grains(n=150, m=96, q=9):
    """Four seeds in four grains of different angle, all four fields."""
    wl = W.thermosolutal_convection(n=n, R=6.0)
    p = wl.params
    p.nx, p.ny = n, m
    p.tip_cx, p.tip_cy = n // 2, m // 2
    p.q_scalar = q
    p.eps = 0.05
    pts = np.array([[0.25 * n, 0.3 * m], [0.7 * n, 0.25 * m], [0.3 * n, 0.72 * m], [0.75 * n, 0.7 * m]])
    ang = np.array([0.0, math.pi / 8, math.pi / 4, 1.3])
    f = W.circle_seeds_window(p, pts, 6.0, 0, 0, n, m, 0.0, -0.55)
    f["theta"] = W.grain_orientation(pts, ang, 0, 0, n, m)
    return p, f


@pytest.mark.parametrize("q", [9, 5])
@pytest.mark.parametrize("variant", [4, 8, 16, 1008, 1016, 1032])
def test_grain_frames_every_phase_variant_fp64(variant, q):
    p, f = _grains(n=301 if variant > 1000 else 150, q=q)
    sim = lbm.Simulation(p, precision="f64")
    sim.set_fusion(False)
    for k in KINDS:
        sim.set_tile(k, variant)
    sim.init_fields(f)
    sim.advance(30)
    got = {k: sim.field(k) for k in active(p)}
    sim.close()
    o = run_oracle(p, f, 30)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 1e-11, (variant, q, k)


def test_grain_frames_fused_fp64_and_fp32():
    """The default (autotuned, fused) path; FP32 bound 200 steps x 20
    roundings x 2^-22 = 1e-3 (the grain angles add one FP32 sincos)."""
    p, f = _grains()
    o = run_oracle(p, f, 200)
    for prec, tol in (("f64", 1e-10), ("f32", 1e-3)):
        sim = lbm.Simulation(p, precision=prec)
        sim.init_fields(f)
        sim.advance(4)
        sim.autotune(reps=1)
        sim.advance(196)
        for k in active(p):
            assert np.abs(sim.field(k) - o[k]).max() < tol, (prec, k)
        sim.close()


def test_orientation_can_be_cleared():
    """set_orientation(None) restores the axis-aligned Eq. 2: the same fields
    as a simulation that never had one."""
    p, f = _grains()
    f_plain = {k: v for k, v in f.items() if k != "theta"}
    outs = []
    for turned_then_cleared in (False, True):
        sim = lbm.Simulation(p, precision="f64")
        if turned_then_cleared:
            sim.set_orientation(f["theta"])
            sim.set_orientation(None)
        sim.init_fields(f_plain)
        sim.advance(20)
        outs.append(sim.field("phi"))
        sim.close()
    assert np.array_equal(outs[0], outs[1])
