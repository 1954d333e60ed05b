"""lbm_init_seed generates the initial fields on the device (FP64 arithmetic
per node) from the seed list: compared with the seeded generators of
workloads (numpy, FP64) on lattices with many circles, circles clipped by
the lattice edges, circles wholly off the lattice, a sinusoidal layer
(Eq. 41) and a noisy planar front, for FP64 and FP32 storage, with and
without the flow."""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2609_25670_b300 as lbm  # noqa: E402


def _circles_case(n=700, m=500, count=20, seed=4):
    wl = W.thermosolutal_convection(n=n, R=6.0)
    p = wl.params
    p.nx, p.ny = n, m
    p.tip_cx, p.tip_cy = n // 2, m // 2
    rng = np.random.default_rng(seed)
    pts = np.column_stack([rng.uniform(-5, n + 5, count), rng.uniform(-5, m + 5, count)])   # some off the lattice
    pts[:3] = [[2.0, 3.5], [n - 1.5, m / 2], [n / 3, m - 0.5]]                               # clipped by edges
    return p, pts


@pytest.mark.parametrize("precision,tol", [("f64", 1e-14), ("f32", 1e-7)])
def test_many_circles_match_the_generator(precision, tol):
    p, pts = _circles_case()
    R = 7.5
    want = W.circle_seeds_window(p, pts, R, 0, 0, p.nx, p.ny, U0=0.02, T0=-0.4)
    sim = lbm.Simulation(p, precision=precision)
    sim.init_seed([{"kind": "circle", "x": float(x), "y": float(y), "r": R} for x, y in pts], U0=0.02, T0=-0.4)
    for k in ("phi", "U", "T", "ux", "uy", "rho"):
        assert np.abs(sim.field(k) - want[k]).max() < tol, k
    sim.close()


@pytest.mark.parametrize("precision,tol", [("f64", 1e-14), ("f32", 1e-7)])
def test_seeds_off_the_lattice(precision, tol):
    """A circle whose reach misses the lattice reaches no block; with every
    seed off the lattice no block is seeded and the fields are the liquid
    values alone (phi = -1, u_x = u_in)."""
    p, pts = _circles_case(n=300, m=200, count=4)
    far = np.array([[-500.0, 50.0], [150.0, 900.0], [1e4, -1e4]])
    sim = lbm.Simulation(p, precision=precision)
    for cen in (np.vstack([pts, far]), far):
        sim.init_seed([{"kind": "circle", "x": float(x), "y": float(y), "r": 7.5} for x, y in cen], U0=0.01, T0=-0.3)
        want = W.circle_seeds_window(p, cen, 7.5, 0, 0, p.nx, p.ny, U0=0.01, T0=-0.3)
        for k in ("phi", "U", "T", "ux", "uy", "rho"):
            assert np.abs(sim.field(k) - want[k]).max() < tol, k
    assert np.all(sim.field("phi") == -1.0)
    sim.close()


def test_sinusoid_layer_matches_the_generator():
    wl = W.thermosolutal_convection(n=300, R=6.0)
    p = wl.params
    p.nx, p.ny = 300, 120
    p.tip_cx, p.tip_cy = 150, 30
    p.has_flow = False
    sim = lbm.Simulation(p, precision="f64")
    sim.init_seed([{"kind": "sinusoid", "y": 30.0, "amp": 4.0, "waves": 3.0}], U0=0.0, T0=-0.5)
    want = W.sinusoid_layer(p.nx, p.ny, p.W0, h=30.0, amp=4.0, waves=3.0)
    assert np.abs(sim.field("phi") - want).max() < 1e-14
    sim.close()


def test_noisy_planar_front_and_circle_combined():
    """The largest profile wins node by node; the planar noise is the
    counter-based draw of the node's row-major index."""
    wl = W.thermosolutal_convection(n=256, R=6.0)
    p = wl.params
    p.nx, p.ny = 256, 200
    p.tip_cx, p.tip_cy = 128, 120
    p.has_flow = False
    sim = lbm.Simulation(p, precision="f64")
    sim.init_seed([{"kind": "planar", "y": 50.0, "amp": 0.02}, {"kind": "circle", "x": 128.0, "y": 120.0, "r": 10.0}],
                  U0=0.0, T0=-0.5, rng_seed=9)
    want = np.maximum(W.planar_front(p.nx, p.ny, 50.0, p.W0, noise_amp=0.02, seed=9),
                      W.circle_seed(p.nx, p.ny, 128.0, 120.0, 10.0, p.W0))
    assert np.abs(sim.field("phi") - want).max() < 1e-14
    sim.close()


def test_reinitialisation_resets_the_state():
    """A second lbm_init_seed after stepping gives the same fields as the
    first and restarts the clock and R_M."""
    p, pts = _circles_case(n=300, m=200, count=6)
    seeds = [{"kind": "circle", "x": float(x), "y": float(y), "r": 6.0} for x, y in pts]
    sim = lbm.Simulation(p, precision="f32")
    sim.init_seed(seeds, U0=0.0, T0=-0.55)
    first = sim.field("phi")
    sim.advance(20)
    sim.init_seed(seeds, U0=0.0, T0=-0.55)
    d = sim.diagnostics()
    assert d["base_step"] == 0 and d["R_M"] == 0.0
    assert np.array_equal(sim.field("phi"), first)
    sim.close()
    assert math.isfinite(d["M_C"])
