"""The phase update fused with the phase-change transfer (phase variants
2000 + h): one launch collides and streams phi (Eqs. 2-4, 14, 18, 21-26) and
applies the transfer of Eqs. 36-39 to the interior it covers, a second
launch applies the transfer on the frame around it.

Parity with the FP64 oracle on lattices whose interior holds several fused
strips and a ragged remainder (walls and periodic boundaries, D2Q9 and D2Q5,
grain frames, the frozen temperature of directional solidification); the
fused and staged forms in FP32 arithmetic with each storage type agree to
rounding; the solute inventory of the fused FP32 path stays within 1e-8 of
the oracle's; variants that do not apply (accumulated coupling, batched
ensembles) fall back to the staged launches."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import active, run_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_2609_25670_b300 as lbm  # noqa: E402

VSTRIP_KINDS = ("transfer", "scalar_U", "scalar_T", "flow")


def _random_state(n, m, seed, bc, q=9):
    wl = W.thermosolutal_convection(n=n, R=8.0)
    p = wl.params
    p.nx, p.ny = n, m
    p.tip_cx, p.tip_cy = n // 2, m // 2
    p.bc_scalar_x = p.bc_scalar_y = bc
    if bc == W.BC_PERIODIC:
        p.bc_flow_x = W.BC_PERIODIC
    p.eps = 0.05
    p.q_scalar = q
    rng = np.random.default_rng(seed)
    phi = W.circle_seed(n, m, n / 2 + 0.3, m / 2 - 0.2, 14.0, p.W0)
    f = W.base_fields(p, phi, U0=0.0, T0=-0.55)
    f["U"] = 0.1 * rng.standard_normal((m, n)) * (1 - phi ** 2) + 0.05
    f["T"] = -0.55 + 0.05 * rng.standard_normal((m, n))
    f["ux"] = 0.01 + 0.002 * rng.standard_normal((m, n))
    f["uy"] = 0.002 * rng.standard_normal((m, n))
    f["rho"] = 1 + 0.001 * rng.standard_normal((m, n))
    return p, f


def _run(p, f, steps, precision, phase_variant, others=1016):
    sim = lbm.Simulation(p, precision=precision)
    sim.set_fusion(False)
    sim.set_tile("phase", phase_variant)
    for k in VSTRIP_KINDS:
        sim.set_tile(k, others)
    sim.init_fields(f)
    sim.advance(steps)
    out = {k: sim.field(k) for k in active(p)}
    out["diag"] = sim.diagnostics()
    sim.close()
    return out


@pytest.mark.parametrize("h", [16, 32])
@pytest.mark.parametrize("q", [9, 5])
@pytest.mark.parametrize("bc", [W.BC_WALL, W.BC_PERIODIC])
def test_fused_phase_transfer_matches_oracle_fp64(h, q, bc):
    """301 x 110: five fused strips across (28 V = 56 columns apart) with a
    ragged remainder and several strip rows; every field and the S_phi / J_U
    maxima (the transfer's |Delta U|) against the oracle after 24 base
    steps."""
    p, f = _random_state(301, 110, seed=11, bc=bc, q=q)
    g = _run(p, f, 24, "f64", 2000 + h)
    o = run_oracle(p, f, 24)
    for k in active(p):
        assert np.abs(g[k] - o[k]).max() < 1e-11, k
    for k in ("S_phi", "J_U", "M_C"):
        assert abs(g["diag"][k] - o["diag"][k]) <= 1e-10 * max(1.0, abs(o["diag"][k])), k


def test_fused_phase_transfer_grain_frames_fp64():
    """Grains of different crystal orientation (the multi-dendrite workload's
    phase update) on the D2Q5 lattice: four seeds in four grains."""
    n, m = 301, 140
    wl = W.thermosolutal_convection(n=n, R=6.0)
    p = wl.params
    p.nx, p.ny = n, m
    p.tip_cx, p.tip_cy = n // 2, m // 2
    p.q_scalar = 5
    p.eps = 0.05
    pts = np.array([[0.25 * n, 0.3 * m], [0.7 * n, 0.25 * m], [0.3 * n, 0.72 * m], [0.75 * n, 0.7 * m]])
    ang = np.array([0.0, np.pi / 8, np.pi / 4, 1.3])
    f = W.circle_seeds_window(p, pts, 6.0, 0, 0, n, m, 0.0, -0.55)
    f["theta"] = W.grain_orientation(pts, ang, 0, 0, n, m)
    g = _run(p, f, 20, "f64", 2032)
    o = run_oracle(p, f, 20)
    for k in active(p):
        assert np.abs(g[k] - o[k]).max() < 1e-11, k


def test_fused_phase_transfer_directional_fp64():
    """Frozen, pulled temperature (no T field: the fused launch transfers to
    U only) against the oracle."""
    wl = W.directional_saline(Le=10, nx=256, ny=160, y0=40.0, seed=3)
    sim = lbm.Simulation(wl.params, precision="f64")
    sim.set_tile("phase", 2016)
    for k in ("transfer", "scalar_U"):
        sim.set_tile(k, 1008)
    sim.init_fields(wl.fields)
    sim.advance(50)
    got = {k: sim.field(k) for k in active(wl.params)}
    sim.close()
    o = run_oracle(wl.params, wl.fields, 50)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 1e-10, k


def test_fused_phase_transfer_small_lattice_is_all_frame():
    """A lattice too small for a fused strip: the phase tiles and the frame
    transfer cover all of it."""
    p, f = _random_state(60, 28, seed=13, bc=W.BC_WALL, q=9)
    g = _run(p, f, 12, "f64", 2016)
    o = run_oracle(p, f, 12)
    for k in active(p):
        assert np.abs(g[k] - o[k]).max() < 1e-11, k


@pytest.mark.parametrize("prec,tol", [("f32", 1e-5), ("f16dev", 2e-4), ("bf16dev", 2e-3)])
@pytest.mark.parametrize("q", [9, 5])
def test_fused_and_staged_agree(prec, tol, q):
    """FP32 arithmetic with each storage type: the fused launch and the
    staged phase + transfer launches are the same arithmetic up to rounding
    order."""
    wl = W.thermosolutal_convection(n=256, R=8.0)
    wl.params.q_scalar = q
    outs = [_run(wl.params, wl.fields, 20, prec, v) for v in (1016, 2016)]
    for k in active(wl.params):
        assert np.abs(outs[0][k] - outs[1][k]).max() < tol, k


@pytest.mark.parametrize("q", [9, 5])
def test_fused_fp32_solute_drift_within_1e8_of_the_oracle(q):
    """The transfer of Eqs. 36-39 conserves the solute exactly up to
    rounding: with the fused launch the FP32 inventory stays within 1e-8 of
    the oracle's after 1000 base steps (128^2, D_S = 1e-1 D_L)."""
    wl = W.thermosolutal_convection(n=128, R=8.0)
    p = wl.params
    p.q_scalar = q
    p.DS = 1e-1 * p.DL
    o = oracle.Oracle(p, wl.fields)
    m0 = o.diagnostics()["M_C"]
    o.advance(1000)
    r_or = (o.diagnostics()["M_C"] - m0) / m0
    o.close()
    sim = lbm.Simulation(p, precision="f32")
    sim.set_fusion(False)
    sim.set_tile("phase", 2016)
    sim.init_fields(wl.fields)
    sim.advance(1000)
    r = sim.diagnostics()["R_M"]
    sim.close()
    assert abs(r - r_or) < 1e-8, (r, r_or)


def test_fused_variant_falls_back_under_accumulated_coupling():
    """The accumulated coupling (Sec. 4.4 ablation) runs the staged launches
    whatever the phase variant: the result equals the staged variant's
    bitwise and matches the oracle."""
    wl = W.thermosolutal_convection(n=200, R=6.0, N=(1, 3, 2, 2))
    wl.params.accumulated = True
    outs = []
    for v in (1016, 2016):
        sim = lbm.Simulation(wl.params, precision="f64")
        sim.set_tile("phase", v)
        sim.init_fields(wl.fields)
        sim.advance(18)
        outs.append({k: sim.field(k) for k in active(wl.params)})
        sim.close()
    o = run_oracle(wl.params, wl.fields, 18)
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k
        assert np.abs(outs[1][k] - o[k]).max() < 1e-10, k


def test_autotune_considers_the_fused_variant():
    """The autotuner's choice (fused or staged phase) reproduces the oracle
    in FP64 and reports a valid phase variant."""
    wl = W.thermosolutal_convection(n=300, R=8.0)
    sim = lbm.Simulation(wl.params, precision="f64")
    sim.set_fusion(False)
    sim.init_fields(wl.fields)
    tiles = sim.autotune(reps=2)
    assert tiles["phase"] in (4, 8, 16, 1008, 1016, 1032, 2016, 2032)
    sim.advance(10)
    got = {k: sim.field(k) for k in active(wl.params)}
    sim.close()
    o = run_oracle(wl.params, wl.fields, 10)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 1e-11, k


def test_batched_ensemble_ignores_the_fused_variant():
    """A batched ensemble keeps its batched phase launch: members with the
    fused variant set still match the oracle one by one."""
    wls = [W.thermosolutal_convection(n=n, R=6.0) for n in (96, 130)]
    sim = lbm.Simulation([w.params for w in wls], precision="f64")
    sim.set_tile("phase", 2016)
    for i, w in enumerate(wls):
        sim.init_fields(w.fields, sim=i)
    sim.advance(8)
    got = [{k: sim.field(k, sim=i) for k in active(w.params)} for i, w in enumerate(wls)]
    sim.close()
    for i, w in enumerate(wls):
        o = run_oracle(w.params, w.fields, 8)
        for k in active(w.params):
            assert np.abs(got[i][k] - o[k]).max() < 1e-11, (i, k)
