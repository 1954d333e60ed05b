"""Degenerate lattice sizes: the smallest the library accepts (nx, ny >= 4)
and lattices narrower or shorter than one tile or one vector strip.  Every
node is then a frame node: each kernel path runs through its boundary maps
(mirror ghosts at walls, wraps at periodic sides, the inlet and outflow
columns of the flow a few nodes apart), and the halo of a tile wraps onto
the same few rows and columns more than once.  FP64 GPU path against the
FP64 oracle within 1e-11 after 16 base steps, for every kernel variant,
both velocity sets, wall and periodic sides, and both couplings."""
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
STEPS = 16

# (nx, ny): one node more than the minimum, single-tile and single-row
# shapes, and the smallest lattice with a vector-strip interior (130 x 13
# holds one 120-column strip of 8 rows) inside a one-unit frame
SIZES = [(4, 4), (5, 7), (4, 37), (37, 5), (130, 13)]

# variant -> (fused transport?, per-kind variant)
VARIANTS = {
    "tiles4": (False, {k: 4 for k in KINDS}),
    "tiles16": (False, {k: 16 for k in KINDS}),
    "fused8": (True, {"phase": 8, "transport": 8}),
    "fused16": (True, {"phase": 16, "transport": 4}),
    "warp_strips4": (False, {"phase": 8, "transfer": 8, "scalar_U": -4, "scalar_T": -4, "flow": 8}),
    "warp_strips32": (False, {"phase": 8, "transfer": 8, "scalar_U": -32, "scalar_T": -32, "flow": 8}),
    "vector_strips8": (False, {k: 1008 for k in KINDS}),
    "vector_strips32": (False, {k: 1032 for k in KINDS}),
}


def _state(nx, ny, q, bc, seed):
    """All four fields with random perturbations about a small seed."""
    wl = W.thermosolutal_convection(n=max(nx, ny), R=2.0)
    p = wl.params
    p.nx, p.ny = nx, ny
    p.tip_cx, p.tip_cy = nx // 2, ny // 2
    p.q_scalar = q
    p.eps = 0.05
    p.bc_scalar_x = p.bc_scalar_y = bc
    if bc == W.BC_PERIODIC:
        p.bc_flow_x = W.BC_PERIODIC
    rng = np.random.default_rng(seed)
    phi = W.circle_seed(nx, ny, nx / 2 + 0.3, ny / 2 - 0.2, 0.3 * min(nx, ny), p.W0)
    f = W.base_fields(p, phi, U0=0.0, T0=-0.55)
    f["phi"] = np.clip(phi + 0.05 * rng.standard_normal((ny, nx)), -1.0, 1.0)
    f["U"] = 0.1 * rng.standard_normal((ny, nx)) + 0.05
    f["T"] = -0.55 + 0.05 * rng.standard_normal((ny, nx))
    f["ux"] = 0.01 + 0.002 * rng.standard_normal((ny, nx))
    f["uy"] = 0.002 * rng.standard_normal((ny, nx))
    f["rho"] = 1 + 0.001 * rng.standard_normal((ny, nx))
    return p, f


def _run(p, f, variant):
    fused, tiles = VARIANTS[variant]
    sim = lbm.Simulation(p, precision="f64")
    sim.set_fusion(fused)
    for k, v in tiles.items():
        sim.set_tile(k, v)
    sim.init_fields(f)
    sim.advance(STEPS)
    got = {k: sim.field(k) for k in active(p)}
    diag = sim.diagnostics()
    sim.close()
    return got, diag


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("bc", [W.BC_WALL, W.BC_PERIODIC])
@pytest.mark.parametrize("q", [9, 5])
@pytest.mark.parametrize("size", SIZES, ids=lambda s: "%dx%d" % s)
def test_small_lattice_every_variant_fp64(size, q, bc, variant):
    p, f = _state(*size, q, bc, seed=size[0] * 100 + size[1])
    got, diag = _run(p, f, variant)
    o = run_oracle(p, f, STEPS)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 1e-11, (k, size, q, bc, variant)
    assert abs(diag["M_C"] - o["diag"]["M_C"]) <= 1e-12 * abs(o["diag"]["M_C"])
    assert not diag["nonfinite"]


@pytest.mark.parametrize("variant", ["tiles4", "fused8", "vector_strips8"])
@pytest.mark.parametrize("q", [9, 5])
@pytest.mark.parametrize("size", [(4, 4), (37, 5), (130, 13)], ids=lambda s: "%dx%d" % s)
def test_small_lattice_accumulated_coupling_fp64(size, q, variant):
    """Multirate (1, 3, 2, 2) with the phase-change increments accumulated
    over the solute's three fine steps."""
    p, f = _state(*size, q, W.BC_WALL, seed=7)
    p.N_U = 3
    p.accumulated = True
    got, diag = _run(p, f, variant)
    o = run_oracle(p, f, STEPS)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 1e-11, (k, size, q, variant)
    assert abs(diag["J_U"] - o["diag"]["J_U"]) <= 1e-11 * max(1.0, o["diag"]["J_U"])
