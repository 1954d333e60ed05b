"""Body force (Eqs. 27, 30 with the forcing term of Eq. 14) on the GPU against
the FP64 oracle, on every compiled form of the flow update: shared-memory
tiles of each height, the fused transport launch, the vector strips (FP64 and
FP32 arithmetic) and the 16-bit-storage vector strip.

Reading R-force: one flow update moves rho u by dt_F F_b (the forcing term of
Eq. 14 carries dt_F, as the scalar sources do); the oracle's pins fix it
(Newton's law, Guo's stationary moments, body-force Poiseuille)."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import active, run_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2609_25670_b300 as lbm  # noqa: E402


def _forced_state(n, m, NF, flow_bc, seed=11):
    """All four fields coupled around a seed, a body force along both axes
    (strong enough that a wrong sign, factor or dt_F scaling moves u by far
    more than the tolerance within the run)."""
    wl = W.thermosolutal_convection(n=n, R=10.0, N=(1, 1, 2, NF))
    p = wl.params
    p.nx, p.ny = n, m
    p.tip_cx, p.tip_cy = n // 2, m // 2
    p.bc_flow_x, p.bc_flow_y = flow_bc
    p.Fbx, p.Fby = 4.0e-5, -2.5e-5
    p.eps = 0.04
    rng = np.random.default_rng(seed)
    phi = W.circle_seed(n, m, n / 2 + 0.4, m / 2 - 0.3, 12.0, p.W0)
    f = W.base_fields(p, phi, U0=0.0, T0=-0.55)
    f["U"] = 0.1 * rng.standard_normal((m, n)) * (1 - phi ** 2) + 0.05
    f["ux"] = (0.01 if flow_bc[0] == W.BC_INLET_OUTFLOW else 0.0) + 0.002 * rng.standard_normal((m, n))
    f["uy"] = 0.002 * rng.standard_normal((m, n))
    f["rho"] = 1 + 0.001 * rng.standard_normal((m, n))
    return p, f


FLOW_BCS = [(W.BC_INLET_OUTFLOW, W.BC_PERIODIC), (W.BC_PERIODIC, W.BC_WALL)]


def _run(p, f, steps, precision, flow_variant=None, fuse=False):
    sim = lbm.Simulation(p, precision=precision)
    sim.set_fusion(fuse)
    if flow_variant is not None:
        sim.set_tile("transport" if fuse else "flow", flow_variant)
    sim.init_fields(f)
    sim.advance(steps)
    out = {k: sim.field(k) for k in active(p)}
    sim.close()
    return out


@pytest.mark.parametrize("NF", [1, 2])
@pytest.mark.parametrize("flow_bc", FLOW_BCS)
@pytest.mark.parametrize("variant,fuse", [(4, False), (8, False), (16, False), (1008, False), (1016, False),
                                          (1032, False), (4, True), (8, True), (16, True)])
def test_forced_flow_every_variant_fp64(NF, flow_bc, variant, fuse):
    """FP64 with F_b != 0 within 1e-11 of the oracle after 24 base steps on a
    ragged 301 x 90 lattice (several vector strips and a remainder)."""
    p, f = _forced_state(301, 90, NF, flow_bc)
    steps = 24
    got = _run(p, f, steps, "f64", variant, fuse)
    o = run_oracle(p, f, steps)
    for k in got:
        assert np.abs(got[k] - o[k]).max() < 1e-11, k
    # the force did act: without it the velocities would differ by ~ steps F
    assert abs(float(np.mean(o["ux"] - f["ux"]))) > 1e-4 * abs(p.Fbx) * steps


@pytest.mark.parametrize("prec,tol", [("f32", 2e-5), ("f16dev", 5e-4), ("bf16dev", 4e-3)])
@pytest.mark.parametrize("variant", [8, 1016])
def test_forced_flow_reduced_precision(prec, tol, variant):
    """FP32 arithmetic with FP32, FP16 or BF16 storage (the 16-bit kinds run
    the 16-bit vector strip at variant 1016) against the oracle after 24 base
    steps, F_b != 0, N_F = 2.  The force moves u by ~1e-3 over the run, so a
    missing dt_F or a sign error exceeds these bounds by an order of
    magnitude; the bounds are the storage rounding of the short run."""
    p, f = _forced_state(301, 90, 2, FLOW_BCS[0])
    steps = 24
    got = _run(p, f, steps, prec, variant)
    o = run_oracle(p, f, steps)
    for k in ("ux", "uy", "rho"):
        assert np.abs(got[k] - o[k]).max() < tol, (k, np.abs(got[k] - o[k]).max())


def test_body_force_poiseuille_gpu():
    """Body-force Poiseuille flow (liquid everywhere, walls in y, N_F = 2) on
    the vector strips in FP64 after 3000 base steps (steady to ~1e-8): equal
    to the oracle within 1e-12 of u_max, and its bulk curvature is -F/nu."""
    nx, ny, nu, F = 300, 16, 1.0 / 6.0, 1.0e-6
    p = W.Params(nx=nx, ny=ny, has_flow=True, bc_flow_x=W.BC_PERIODIC, bc_flow_y=W.BC_WALL,
                 bc_scalar_x=W.BC_PERIODIC, bc_scalar_y=W.BC_WALL, N_F=2, nu=nu, Fbx=F, W0=1, tau0=1)
    f = W.base_fields(p, -np.ones((ny, nx)))
    got = _run(p, f, 3000, "f64", 1016)
    o = run_oracle(p, f, 3000)
    umax = float(np.abs(o["ux"]).max())
    assert np.abs(got["ux"] - o["ux"]).max() < 1e-10 * umax
    u = got["ux"][:, nx // 2]
    d2 = u[2:] - 2 * u[1:-1] + u[:-2]
    assert np.abs(d2 / (-F / nu) - 1).max() < 1e-6
