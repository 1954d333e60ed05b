"""The five-velocity option of the scalar lattices (D2Q5 for phi, U and T,
the flow staying D2Q9), through the C ABI, against the FP64 oracle run with
the same option: every kernel variant (shared-memory tiles, warp strips,
vector strips with their frame, the fused transport launch, the batched
ensemble launches), every boundary kind, both couplings and every storage
type.  Tolerances as for D2Q9: FP64 within 1e-10 after up to 1000 base steps
(single updates and short runs 1e-11 to 1e-13); FP32 2e-3 and 16-bit
deviation storage 5e-3 / 4e-2 after 1000 steps (the bounds derived from the
rounding of the arithmetic and storage types)."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import active, max_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2609_25670_b300 as lbm  # noqa: E402

BIG = 100000
KINDS = ("phase", "transfer", "scalar_U", "scalar_T", "flow")


def _q5(p):
    p.q_scalar = 5
    return p


def _check(p, fields, steps, tol, precision="f64", **kw):
    g = run_gpu(p, fields, steps, precision=precision, **kw)
    o = run_oracle(p, fields, steps)
    err = max_err(g, o, active(p))
    assert max(err.values()) <= tol, err
    return g, o, err


def _random_state(n=70, m=45, seed=0, flow=True, bc=W.BC_WALL):
    wl = W.thermosolutal_convection(n=n, R=8.0)
    p = _q5(wl.params)
    p.nx, p.ny = n, m
    p.tip_cx, p.tip_cy = n // 2, m // 2
    p.bc_scalar_x = p.bc_scalar_y = bc
    if bc == W.BC_PERIODIC:
        p.bc_flow_x = W.BC_PERIODIC
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
@pytest.mark.parametrize("which", ["phase", "U", "T"])
def test_single_update_fp64(which, bc):
    """One field updated alone (the others held by huge update factors)."""
    p, f = _random_state(bc=bc, flow=(which == "U"))
    p.N_phi = 1 if which == "phase" else BIG
    p.N_U = 1 if which == "U" else BIG
    p.N_T = 1 if which == "T" else BIG
    p.N_F = BIG
    _check(p, f, 3, 1e-13)


def test_phase_state_is_four_planes():
    """The phase field of a D2Q5 run stores populations 1..4 only: four
    planes instead of eight per ping-pong buffer."""
    wl = W.thermal_free_dendrite(n=128, N_T=1)
    sizes = []
    for q in (9, 5):
        wl.params.q_scalar = q
        sim = lbm.Simulation(wl.params, precision="f32")
        sizes.append(sim.device_bytes())
        sim.close()
    pitch = 128
    assert sizes[0] - sizes[1] == 2 * 4 * pitch * 128 * 4


@pytest.mark.parametrize("N_T", [1, 2])
def test_thermal_dendrite_fp64_1000_steps(N_T):
    """The thermal free dendrite on D2Q5 phase and temperature lattices, as
    the workload list states it: 128^2 periodic, FP64, 1000 base steps,
    within 1e-10 of the oracle; enthalpy and tips."""
    wl = W.thermal_free_dendrite(n=128, N_T=N_T)
    _q5(wl.params)
    g, o, err = _check(wl.params, wl.fields, 1000, 1e-10)
    assert abs(g["diag"]["H"] - o["diag"]["H"]) < 1e-9
    assert np.abs(g["diag"]["tip"] - o["diag"]["tip"]).max() < 1e-8


@pytest.mark.parametrize("fuse", [True, False])
def test_thermosolutal_convection_fp64_ragged(fuse):
    """All four fields (D2Q5 phi, U, T; D2Q9 flow) with inlet / outflow,
    multirate (1, 1, 2, 2), ragged 80 x 70, fused and staged."""
    wl = W.thermosolutal_convection(n=80, R=8.0)
    p = _q5(wl.params)
    p.ny, p.tip_cy = 70, 35
    f = W.base_fields(p, W.circle_seed(80, 70, 40, 35, 8.0, p.W0), U0=0.0, T0=-0.55)
    sim = lbm.Simulation(p, precision="f64")
    sim.set_fusion(fuse)
    sim.init_fields(f)
    sim.advance(300)
    got = {k: sim.field(k) for k in active(p)}
    d = sim.diagnostics()
    sim.close()
    o = run_oracle(p, f, 300)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 1e-10, k
    assert abs(d["M_C"] - o["diag"]["M_C"]) / o["diag"]["M_C"] < 1e-12


@pytest.mark.parametrize("ty", [4, 8, 16])
def test_every_tile_shape_fp64(ty):
    wl = W.thermosolutal_convection(n=80, R=8.0)
    p = _q5(wl.params)
    p.ny, p.tip_cy = 70, 35
    f = W.base_fields(p, W.circle_seed(80, 70, 40, 35, 8.0, p.W0), U0=0.0, T0=-0.55)
    sim = lbm.Simulation(p, precision="f64")
    for k in KINDS + ("transport",):
        sim.set_tile(k, ty)
    sim.init_fields(f)
    sim.advance(60)
    got = {k: sim.field(k) for k in active(p)}
    sim.close()
    o = run_oracle(p, f, 60)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 1e-11, k


@pytest.mark.parametrize("h", [4, 8, 16, 32])
@pytest.mark.parametrize("bc", [W.BC_WALL, W.BC_PERIODIC])
def test_warp_strips_fp64(h, bc):
    p, f = _random_state(n=95, m=75, seed=5, bc=bc)
    sim = lbm.Simulation(p, precision="f64")
    sim.set_fusion(False)
    for k in ("scalar_U", "scalar_T"):
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
def test_vector_strips_fp64(h, bc):
    """Vector strips over the interior and their frame, on a lattice whose
    interior holds several strips and a ragged remainder."""
    p, f = _random_state(n=301, m=90, seed=6, bc=bc)
    sim = lbm.Simulation(p, precision="f64")
    sim.set_fusion(False)
    for k in KINDS:
        sim.set_tile(k, 1000 + h)
    sim.init_fields(f)
    sim.advance(24)
    got = {k: sim.field(k) for k in active(p)}
    sim.close()
    o = run_oracle(p, f, 24)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 1e-11, k


def test_accumulated_coupling_fp64():
    wl = W.thermosolutal_convection(n=260, R=6.0, N=(1, 3, 2, 2))
    p = _q5(wl.params)
    p.accumulated = True
    for v in (8, 1016):
        sim = lbm.Simulation(p, precision="f64")
        for k in KINDS:
            sim.set_tile(k, v)
        sim.init_fields(wl.fields)
        sim.advance(36)
        got = {k: sim.field(k) for k in active(p)}
        d = sim.diagnostics()
        sim.close()
        o = run_oracle(p, wl.fields, 36)
        for k in got:
            assert np.abs(got[k] - o[k]).max() < 1e-10, (v, k)
        assert abs(d["J_U"] - o["diag"]["J_U"]) <= 1e-10 * max(1.0, o["diag"]["J_U"])


def test_directional_frozen_temperature_vector_strips_fp64():
    wl = W.directional_saline(Le=10, nx=256, ny=160, y0=40.0, seed=3)
    p = _q5(wl.params)
    sim = lbm.Simulation(p, precision="f64")
    for k in KINDS:
        sim.set_tile(k, 1008)
    sim.init_fields(wl.fields)
    sim.advance(50)
    got = {k: sim.field(k) for k in active(p)}
    sim.close()
    o = run_oracle(p, wl.fields, 50)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 1e-10, k


@pytest.mark.parametrize("variant", [("tiles", 8), ("strips", -16), ("vstrips", 1016), ("fused", 8)])
def test_dirichlet_bottom_wall_fp64(variant):
    """T held at T_b below row 0 (anti-bounce-back of the one D2Q5 link that
    crosses the wall, with the D2Q5 weight) on every variant that streams T
    across it."""
    kind, v = variant
    wl = W.directional_evolving_T(Le=10, nx=290 if kind == "vstrips" else 97, ny=70)
    p = _q5(wl.params)
    f = dict(wl.fields)
    f["T"] = f["T"] + 0.5 * np.random.default_rng(0).standard_normal(f["T"].shape)
    sim = lbm.Simulation(p, precision="f64")
    sim.set_fusion(kind == "fused")
    if kind == "fused":
        sim.set_tile("transport", v)
    elif kind == "strips":
        sim.set_tile("scalar_T", v)
        sim.set_tile("scalar_U", v)
    else:
        for k in KINDS:
            if kind == "tiles" or k != "flow":
                sim.set_tile(k, v)
    sim.init_fields(f)
    sim.advance(40)
    got = {k: sim.field(k) for k in active(p)}
    sim.close()
    o = run_oracle(p, f, 40)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 1e-10, k


def test_fp32_1000_steps():
    wl = W.thermosolutal_convection(n=128, R=8.0)
    _q5(wl.params)
    g, o, err = _check(wl.params, wl.fields, 1000, 2e-3, precision="f32")
    assert abs(g["diag"]["M_C"] - o["diag"]["M_C"]) / o["diag"]["M_C"] < 1e-5


@pytest.mark.parametrize("prec,tol", [("f16dev", 5e-3), ("bf16dev", 4e-2)])
def test_deviation_storage_1000_steps(prec, tol):
    """Phase deviations f_i - w_i phi with the D2Q5 weights, flow deviations,
    U / T first moments, 16-bit, FP32 arithmetic."""
    wl = W.thermosolutal_convection(n=128, R=8.0)
    _q5(wl.params)
    g, o, err = _check(wl.params, wl.fields, 1000, tol, precision=prec)
    assert abs(g["diag"]["M_C"] - o["diag"]["M_C"]) / o["diag"]["M_C"] < 1e-5


@pytest.mark.parametrize("prec,tol", [("f32", 1e-5), ("f16dev", 2e-4)])
def test_vector_strips_and_tiles_agree(prec, tol):
    wl = W.thermosolutal_convection(n=256, R=8.0)
    _q5(wl.params)
    outs = []
    for v in (8, 1016):
        sim = lbm.Simulation(wl.params, precision=prec)
        sim.set_fusion(False)
        for k in KINDS:
            sim.set_tile(k, v)
        sim.init_fields(wl.fields)
        sim.advance(20)
        outs.append({k: sim.field(k) for k in active(wl.params)})
        sim.close()
    for k in outs[0]:
        assert np.abs(outs[0][k] - outs[1][k]).max() < tol, k


def test_batched_ensemble_equals_members_alone_and_oracle():
    """Batched launches over uneven D2Q5 members equal each member advanced
    alone (bitwise), and FP64 members match the oracle."""
    ms = W.ensemble_members(count=5, seed=11, sizes=(40, 64, 72, 96))
    for m in ms:
        _q5(m.params)
    steps = 24
    for prec in ("f32", "f64"):
        sim = lbm.Simulation([m.params for m in ms], precision=prec)
        for i, m in enumerate(ms):
            sim.init_fields(m.fields, sim=i)
        sim.advance(steps)
        batched = [{k: sim.field(k, sim=i) for k in active(m.params)} for i, m in enumerate(ms)]
        sim.close()
        for i, m in enumerate(ms):
            if prec == "f32":
                one = lbm.Simulation(m.params, precision=prec)
                one.init_fields(m.fields)
                one.advance(steps)
                for k in active(m.params):
                    assert np.array_equal(batched[i][k], one.field(k)), (i, k)
                one.close()
            else:
                o = run_oracle(m.params, m.fields, steps)
                for k in active(m.params):
                    assert np.abs(batched[i][k] - o[k]).max() < 1e-11, (i, k)


def test_ensemble_rejects_mixed_velocity_sets():
    ms = W.ensemble_members(count=2, seed=11, sizes=(40, 64))
    ms[0].params.q_scalar = 5
    with pytest.raises(lbm.LbmError):
        lbm.Simulation([m.params for m in ms], precision="f32")
