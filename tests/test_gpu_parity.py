"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 runs must match the oracle within 1e-10 max-abs after up to 1000 base
steps; FP32 and 16-bit-storage runs within bounds derived from the rounding
of the arithmetic and storage types: about 20 roundings per base step, each
with relative error 2^-22 (FP32 with the hardware reciprocal), or of the
stored deviations (FP16 2^-11, BF16 2^-8 relative to values of order 1e-2),
accumulated linearly over the steps."""
import math

import numpy as np
import pytest

import workloads as W
from gpu_helpers import active, max_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _check(p, fields, steps, tol, precision="f64", **kw):
    g = run_gpu(p, fields, steps, precision=precision, **kw)
    o = run_oracle(p, fields, steps)
    err = max_err(g, o, active(p))
    assert max(err.values()) <= tol, err
    return g, o, err


# ---------------------------------------------------------------------------
# single field updates, isolated through the schedule (a huge update factor
# keeps a field from firing within the run)
# ---------------------------------------------------------------------------
BIG = 100000


def _random_state(n=70, m=45, seed=0, flow=True, bc=W.BC_WALL):
    wl = W.thermosolutal_convection(n=n, R=8.0)
    p = wl.params
    p.nx, p.ny = n, m
    p.tip_cx, p.tip_cy = n // 2, m // 2
    p.bc_scalar_x = p.bc_scalar_y = bc
    p.has_flow = flow
    p.eps = 0.05
    rng = np.random.default_rng(seed)
    phi = W.circle_seed(n, m, n / 2 + 0.3, m / 2 - 0.2, 12.0, p.W0)
    f = W.base_fields(p, phi, U0=0.0, T0=-0.55)
    f["U"] = 0.1 * rng.standard_normal((m, n)) * (1 - phi ** 2) + 0.05
    f["T"] = -0.55 + 0.05 * rng.standard_normal((m, n))
    if flow:
        f["ux"] = 0.01 + 0.002 * rng.standard_normal((m, n))
        f["uy"] = 0.002 * rng.standard_normal((m, n))
        f["rho"] = 1 + 0.001 * rng.standard_normal((m, n))
    return p, f


@pytest.mark.parametrize("bc", [W.BC_WALL, W.BC_PERIODIC])
@pytest.mark.parametrize("which", ["phase", "U", "T", "flow"])
def test_single_update_fp64(which, bc):
    p, f = _random_state(bc=bc, flow=(which in ("flow", "U")))
    if bc == W.BC_PERIODIC:
        p.bc_flow_x = W.BC_PERIODIC
    p.N_phi = 1 if which == "phase" else BIG
    p.N_U = 1 if which == "U" else BIG
    p.N_T = 1 if which == "T" else BIG
    p.N_F = 1 if which == "flow" else BIG
    _check(p, f, 3, 1e-13)


# ---------------------------------------------------------------------------
# whole runs
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N_T", [1, 2])
def test_thermal_dendrite_fp64_1000_steps(N_T):
    """128^2 periodic thermal dendrite (phi + T), FP64, 1000 base steps:
    max-abs phi, T within 1e-10 of the oracle; exact enthalpy invariant."""
    wl = W.thermal_free_dendrite(n=128, N_T=N_T)
    g, o, err = _check(wl.params, wl.fields, 1000, 1e-10)
    assert abs(g["diag"]["H"] - o["diag"]["H"]) < 1e-9
    assert np.abs(g["diag"]["tip"] - o["diag"]["tip"]).max() < 1e-8


def test_thermosolutal_convection_fp64_ragged():
    """All four fields with inlet/outflow, multirate (1, 1, 2, 2), on a
    ragged 80 x 70 lattice (tiles of 32 x 8 do not divide it)."""
    wl = W.thermosolutal_convection(n=80, R=8.0)
    p = wl.params
    p.ny = 70
    p.tip_cy = 35
    f = W.base_fields(p, W.circle_seed(80, 70, 40, 35, 8.0, p.W0), U0=0.0, T0=-0.55)
    g, o, err = _check(p, f, 300, 1e-10)
    assert abs(g["diag"]["M_C"] - o["diag"]["M_C"]) / o["diag"]["M_C"] < 1e-12


def test_accumulated_coupling_fp64():
    wl = W.thermosolutal_convection(n=64, R=6.0, N=(1, 3, 2, 2))
    wl.params.accumulated = True
    g, o, err = _check(wl.params, wl.fields, 120, 1e-10)
    assert abs(g["diag"]["J_U"] - o["diag"]["J_U"]) <= 1e-10 * max(1.0, o["diag"]["J_U"])


def test_directional_frozen_temperature_fp64():
    wl = W.directional_saline(Le=10, nx=96, ny=160, y0=40.0, seed=3)
    g, o, err = _check(wl.params, wl.fields, 200, 1e-10)


def test_graphs_and_chunking_bitwise_identical():
    wl = W.thermosolutal_convection(n=64, R=6.0)
    a = run_gpu(wl.params, wl.fields, 40, precision="f32", graphs=True)
    b = run_gpu(wl.params, wl.fields, 40, precision="f32", graphs=False, chunks=[3, 5, 1, 31])
    for k in active(wl.params):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("fuse", [True, False])
def test_half_period_graphs_bitwise(fuse):
    """Graph replays of either half of the ping-pong period, entered from any
    phase of the schedule (advance(2) with update factors (1, 1, 2, 2); a
    3-step chunk shifts the phase), give exactly the eager result."""
    import paper_2609_25670_b300 as lbm
    wl = W.thermosolutal_convection(n=64, R=6.0, N=(1, 1, 2, 2))
    chunks = [2] * 7 + [3] + [2] * 6 + [1] + [4] * 3 + [2]
    outs = []
    for graphs in (True, False):
        sim = lbm.Simulation(wl.params, precision="f32")
        sim.set_fusion(fuse)
        sim.set_graphs(graphs)
        sim.init_fields(wl.fields)
        for c in chunks:
            sim.advance(c)
        outs.append({k: sim.field(k) for k in active(wl.params)})
        sim.close()
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k


def test_fp32_thermosolutal_1000_steps():
    """FP32 storage and arithmetic against the FP64 oracle after 1000 steps."""
    wl = W.thermosolutal_convection(n=128, R=8.0)
    g, o, err = _check(wl.params, wl.fields, 1000, 2e-3, precision="f32")
    assert abs(g["diag"]["M_C"] - o["diag"]["M_C"]) / o["diag"]["M_C"] < 1e-5


def test_init_seed_matches_generator():
    import paper_2609_25670_b300 as lbm
    wl = W.thermosolutal_convection(n=96, R=8.0)
    sim = lbm.Simulation(wl.params, precision="f64")
    sim.init_seed([{"kind": "circle", "x": 48, "y": 48, "r": 8.0}], U0=0.0, T0=-0.55)
    for k in ("phi", "U", "T", "ux", "rho"):
        assert np.abs(sim.field(k) - wl.fields[k]).max() < 1e-14, k
    sim.close()
    wd = W.directional_saline(Le=10, nx=64, ny=96, y0=40.0, seed=3)
    sim = lbm.Simulation(wd.params, precision="f64")
    sim.init_seed([{"kind": "planar", "y": 40.0, "amp": 0.01}], U0=0.0, rng_seed=3)
    assert np.abs(sim.field("phi") - wd.fields["phi"]).max() < 1e-14
    sim.close()


UPDATE_KINDS = ("phase", "transfer", "scalar_U", "scalar_T", "flow", "transport")
STRIP_KINDS = ("scalar_U", "scalar_T")
VSTRIP_KINDS = ("phase", "transfer", "scalar_U", "scalar_T", "flow")


@pytest.mark.parametrize("h", [4, 8, 16, 32])
@pytest.mark.parametrize("bc", [W.BC_WALL, W.BC_PERIODIC])
def test_strip_kernels_match_oracle_fp64(h, bc):
    """Warp-strip variants of the U and T updates (strip height h) against
    the oracle: FP64, ragged lattice (strips of 30 columns and h rows do not
    divide it), walls or periodic scalar boundaries, all fields coupled."""
    import paper_2609_25670_b300 as lbm
    p, f = _random_state(n=95, m=75, seed=5, bc=bc)
    if bc == W.BC_PERIODIC:
        p.bc_flow_x = W.BC_PERIODIC
    sim = lbm.Simulation(p, precision="f64")
    sim.set_fusion(False)
    for k in STRIP_KINDS:
        sim.set_tile(k, -h)
    sim.init_fields(f)
    sim.advance(30)
    got = {k: sim.field(k) for k in active(p)}
    sim.close()
    o = run_oracle(p, f, 30)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 1e-11, k


@pytest.mark.parametrize("h", [8, 16, 32])
@pytest.mark.parametrize("bc", [W.BC_WALL, W.BC_PERIODIC])
def test_vector_strip_kernels_match_oracle_fp64(h, bc):
    """Vector strips (four nodes per lane) on the interior of the U, T and
    flow updates, with 1-wide strips (U, T) or shared-memory tiles (flow) on
    the frame around it: FP64 against the oracle on a lattice whose interior
    holds several vector strips and a ragged remainder, inlet / outflow or
    periodic flow boundaries."""
    import paper_2609_25670_b300 as lbm
    p, f = _random_state(n=301, m=90, seed=6, bc=bc)
    if bc == W.BC_PERIODIC:
        p.bc_flow_x = W.BC_PERIODIC
    sim = lbm.Simulation(p, precision="f64")
    sim.set_fusion(False)
    for k in VSTRIP_KINDS:
        sim.set_tile(k, 1000 + h)
    sim.init_fields(f)
    sim.advance(24)
    got = {k: sim.field(k) for k in active(p)}
    sim.close()
    o = run_oracle(p, f, 24)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 1e-11, k


def test_vector_strips_directional_fp64():
    """Vector strips with the frozen, pulled temperature field (directional
    solidification: theta from the base-step clock) against the oracle."""
    import paper_2609_25670_b300 as lbm
    wl = W.directional_saline(Le=10, nx=256, ny=160, y0=40.0, seed=3)
    sim = lbm.Simulation(wl.params, precision="f64")
    for k in VSTRIP_KINDS:
        sim.set_tile(k, 1008)
    sim.init_fields(wl.fields)
    sim.advance(50)
    got = {k: sim.field(k) for k in active(wl.params)}
    sim.close()
    o = run_oracle(wl.params, wl.fields, 50)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 1e-10, k


def test_vector_strips_accumulated_fp64():
    """Coarse-step injection written by the transfer and read by the U / T
    vector strips (Sec. 4.4 ablation)."""
    import paper_2609_25670_b300 as lbm
    wl = W.thermosolutal_convection(n=260, R=6.0, N=(1, 3, 2, 2))
    wl.params.accumulated = True
    sim = lbm.Simulation(wl.params, precision="f64")
    for k in VSTRIP_KINDS:
        sim.set_tile(k, 1016)
    sim.init_fields(wl.fields)
    sim.advance(36)
    got = {k: sim.field(k) for k in active(wl.params)}
    d = sim.diagnostics()
    sim.close()
    o = run_oracle(wl.params, wl.fields, 36)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 1e-10, k
    assert abs(d["J_U"] - o["diag"]["J_U"]) <= 1e-10 * max(1.0, o["diag"]["J_U"])


@pytest.mark.parametrize("prec,tol", [("f32", 1e-5), ("f16dev", 2e-4), ("bf16dev", 2e-3)])
def test_vector_strips_and_tiles_agree(prec, tol):
    """Vector strips and tiles in FP32 arithmetic with each storage type:
    the same arithmetic up to rounding order (16-bit storage rounds the same
    deviations, so the two stay within FP32 rounding of each other)."""
    import paper_2609_25670_b300 as lbm
    wl = W.thermosolutal_convection(n=256, R=8.0)
    outs = []
    for v in (8, 1016):
        sim = lbm.Simulation(wl.params, precision=prec)
        sim.set_fusion(False)
        for k in VSTRIP_KINDS:
            sim.set_tile(k, v)
        sim.init_fields(wl.fields)
        sim.advance(20)
        outs.append({k: sim.field(k) for k in active(wl.params)})
        sim.close()
    for k in outs[0]:
        assert np.abs(outs[0][k] - outs[1][k]).max() < tol, k


def test_strip_and_tile_agree_fp32():
    """Strip and tile variants: the same arithmetic, different rounding order."""
    import paper_2609_25670_b300 as lbm
    wl = W.thermosolutal_convection(n=96, R=8.0)
    outs = []
    for v in (8, -16):
        sim = lbm.Simulation(wl.params, precision="f32")
        sim.set_fusion(False)
        for k in STRIP_KINDS:
            sim.set_tile(k, v)
        sim.init_fields(wl.fields)
        sim.advance(40)
        outs.append({k: sim.field(k) for k in active(wl.params)})
        sim.close()
    for k in outs[0]:
        assert np.abs(outs[0][k] - outs[1][k]).max() < 1e-5, k


@pytest.mark.parametrize("ty", [4, 8, 16])
def test_every_tile_shape_matches_oracle_fp64(ty):
    """Each compiled tile height is a correct implementation on its own:
    FP64, ragged 80 x 70 lattice (edge and interior tiles), all fields."""
    import paper_2609_25670_b300 as lbm
    wl = W.thermosolutal_convection(n=80, R=8.0)
    p = wl.params
    p.ny, p.tip_cy = 70, 35
    f = W.base_fields(p, W.circle_seed(80, 70, 40, 35, 8.0, p.W0), U0=0.0, T0=-0.55)
    sim = lbm.Simulation(p, precision="f64")
    for k in UPDATE_KINDS:
        sim.set_tile(k, ty)
    sim.init_fields(f)
    sim.advance(60)
    got = {k: sim.field(k) for k in active(p)}
    sim.close()
    o = run_oracle(p, f, 60)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 1e-11, k


def test_autotuned_tiles_agree_to_rounding():
    """Different tile shapes (and the interior / edge paths they select) are
    different compilations of the same arithmetic: they agree to
    floating-point contraction rounding; a fixed tile choice is bitwise
    reproducible."""
    import paper_2609_25670_b300 as lbm
    wl = W.thermosolutal_convection(n=96, R=8.0)
    outs = []
    for tune in (False, True, False):
        sim = lbm.Simulation(wl.params, precision="f32")
        sim.init_fields(wl.fields)
        sim.advance(10)
        if tune:
            ch = sim.autotune(reps=2)
            assert set(ch[k] for k in UPDATE_KINDS) <= {4, 8, 16, -4, -8, -16, -32, 1008, 1016, 1032}
        sim.advance(30)
        outs.append({k: sim.field(k) for k in active(wl.params)})
        sim.close()
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[2][k]), k           # same tiles: bitwise
        assert np.abs(outs[0][k] - outs[1][k]).max() < 1e-5, k    # FP32 rounding, 40 steps


@pytest.mark.parametrize("prec,tol", [("f16dev", 5e-3), ("bf16dev", 4e-2)])
def test_deviation_storage_thermosolutal(prec, tol):
    """16-bit storage of the deviations f_i - ref_i with FP32 arithmetic
    against the FP64 oracle after 1000 base steps.  The deviations are at
    most of order 1e-2, so a store rounds with absolute error ~5e-6 (FP16)
    or ~4e-5 (BF16); linear accumulation over 1000 steps gives 5e-3 and
    4e-2."""
    wl = W.thermosolutal_convection(n=128, R=8.0)
    g, o, err = _check(wl.params, wl.fields, 1000, tol, precision=prec)
    assert abs(g["diag"]["M_C"] - o["diag"]["M_C"]) / o["diag"]["M_C"] < 1e-5


def test_unfused_path_fp64():
    """The one-launch-per-stage path (transfer, U, T, flow separately) against
    the oracle, FP64, ragged lattice, all fields, multirate (1, 1, 2, 2)."""
    import paper_2609_25670_b300 as lbm
    wl = W.thermosolutal_convection(n=80, R=8.0)
    p = wl.params
    p.ny, p.tip_cy = 70, 35
    f = W.base_fields(p, W.circle_seed(80, 70, 40, 35, 8.0, p.W0), U0=0.0, T0=-0.55)
    sim = lbm.Simulation(p, precision="f64")
    sim.set_fusion(False)
    sim.init_fields(f)
    sim.advance(120)
    got = {k: sim.field(k) for k in active(p)}
    counts = sim.launch_counts()
    sim.close()
    assert counts["transport"] == 0 and counts["transfer"] > 0
    o = run_oracle(p, f, 120)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 1e-10, k


def test_autotune_fusion_choice():
    """The autotuner picks the fused or staged path unless it was fixed."""
    import paper_2609_25670_b300 as lbm
    wl = W.thermosolutal_convection(n=96, R=8.0)
    for fixed in (None, True, False):
        sim = lbm.Simulation(wl.params, precision="f32")
        if fixed is not None:
            sim.set_fusion(fixed)
        sim.init_fields(wl.fields)
        sim.advance(4)
        sim.autotune(reps=2)
        if fixed is not None:
            assert sim.fused == fixed
        n0 = sim.launch_counts()
        sim.advance(4)
        n = sim.launch_counts()
        assert (n["transport"] > n0["transport"]) == sim.fused
        assert (n["transfer"] > n0["transfer"]) != sim.fused
        sim.close()


def test_fused_and_unfused_agree_fp32():
    """One fused launch per base step vs one launch per stage: the same
    arithmetic in different compilations (contraction rounding only)."""
    import paper_2609_25670_b300 as lbm
    wl = W.thermosolutal_convection(n=96, R=8.0)
    outs = []
    for fuse in (True, False):
        sim = lbm.Simulation(wl.params, precision="f32")
        sim.set_fusion(fuse)
        sim.init_fields(wl.fields)
        sim.advance(40)
        outs.append({k: sim.field(k) for k in active(wl.params)})
        n = sim.launch_counts()
        assert (n["transport"] > 0) == fuse
        sim.close()
    for k in outs[0]:
        assert np.abs(outs[0][k] - outs[1][k]).max() < 1e-5, k


def test_nonfinite_is_detected_and_sticky():
    """Failure detection without a GPU fault: a NaN planted on the host in the
    initial U field spreads through the update; lbm_diagnostics reports it
    (status NONFINITE), lbm_advance then refuses until the simulation is
    initialised again, after which it runs normally."""
    import paper_2609_25670_b300 as lbm
    wl = W.thermosolutal_convection(n=64, R=6.0)
    bad = {k: v.copy() for k, v in wl.fields.items()}
    bad["U"][10, 12] = np.nan
    sim = lbm.Simulation(wl.params, precision="f32")
    sim.init_fields(bad)
    sim.advance(4)
    d = sim.diagnostics()
    assert d["nonfinite"] == 1 and d["status"] == 5
    with pytest.raises(lbm.LbmError):
        sim.advance(1)
    sim.init_fields(wl.fields)
    sim.advance(4)
    d = sim.diagnostics()
    assert d["nonfinite"] == 0 and d["status"] == 0
    sim.close()


@pytest.mark.parametrize("v", [8, 1016])
def test_accumulated_coupling_fp32_long_intervals(v):
    """The accumulated coupling in FP32 with a long coarse interval (N_U = 40:
    forty phase-change increments summed per node before each U update, with
    Kahan compensation) against the FP64 oracle after 400 base steps, within
    the linear FP32 rounding bound of the steps run (400 x 20 x 2^-22 = 2e-3),
    solute mass within 1e-5 relative; tiles and vector strips."""
    import paper_2609_25670_b300 as lbm
    wl = W.thermosolutal_convection(n=260, R=6.0, N=(1, 40, 2, 2))
    wl.params.accumulated = True
    sim = lbm.Simulation(wl.params, precision="f32")
    for k in VSTRIP_KINDS:
        sim.set_tile(k, v)
    sim.init_fields(wl.fields)
    sim.advance(400)
    got = {k: sim.field(k) for k in active(wl.params)}
    d = sim.diagnostics()
    sim.close()
    o = run_oracle(wl.params, wl.fields, 400)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 2e-3, k
    assert abs(d["M_C"] - o["diag"]["M_C"]) < 1e-5 * o["diag"]["M_C"]
