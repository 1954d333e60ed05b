"""The bottom wall held at T = T_b (Sec. 4.4: the cold bottom boundary kept
at -20 C), by anti-bounce-back at the half-way wall, through the C ABI on
every kernel variant that streams the temperature across that wall: the
shared-memory tiles, the warp strips, the frame of the vector strips and the
fused transport kernel; element by element against the FP64 oracle."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import active, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2609_25670_b300 as lbm  # noqa: E402

KINDS = ("phase", "transfer", "scalar_U", "scalar_T", "flow")


def _state(nx=97, ny=70, Le=10, seed=0):
    """The Sec. 4.4 case on a small ragged lattice, with a perturbed
    temperature so that heat crosses the bottom wall from the first step."""
    wl = W.directional_evolving_T(Le=Le, nx=nx, ny=ny)
    f = dict(wl.fields)
    rng = np.random.default_rng(seed)
    f["T"] = f["T"] + 0.5 * rng.standard_normal(f["T"].shape)
    return wl.params, f


@pytest.mark.parametrize("variant", [("tiles", 4), ("tiles", 8), ("tiles", 16), ("strips", -8), ("strips", -16),
                                     ("vstrips", 1008), ("vstrips", 1016), ("fused", 4), ("fused", 8),
                                     ("fused", 16)])
def test_dirichlet_wall_every_variant_fp64(variant):
    kind, v = variant
    p, f = _state(nx=290 if kind == "vstrips" else 97)
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
        assert np.abs(got[k] - o[k]).max() < 1e-11 * max(1.0, np.abs(o[k]).max()), (variant, k)


def test_directional_evolving_T_fp64_1000_steps():
    """Sec. 4.4 at Le = 10 (N_U = 10), 1000 base steps, FP64 within 1e-10 of
    the oracle relative to the field's magnitude (T is of order 20)."""
    p, f = _state(nx=128, ny=96, Le=10, seed=1)
    g = run_gpu(p, f, 1000, precision="f64")
    o = run_oracle(p, f, 1000)
    for k in active(p):
        assert np.abs(g[k] - o[k]).max() < 1e-10 * max(1.0, np.abs(o[k]).max()), k
    assert abs(g["diag"]["M_C"] - o["diag"]["M_C"]) < 1e-12 * o["diag"]["M_C"]


def test_directional_evolving_T_fp32_300_steps():
    """FP32 over 300 base steps: 300 steps x 20 roundings x 2^-22 = 1.4e-3 of
    each field's magnitude."""
    p, f = _state(nx=128, ny=96, Le=10, seed=2)
    g = run_gpu(p, f, 300, precision="f32")
    o = run_oracle(p, f, 300)
    for k in active(p):
        scale = max(1.0, np.abs(o[k]).max())
        assert np.abs(g[k] - o[k]).max() < 1.5e-3 * scale, k


def test_dirichlet_needs_T_and_a_bottom_wall():
    p, f = _state()
    p.bc_scalar_y = W.BC_PERIODIC
    with pytest.raises(lbm.LbmError):
        lbm.Simulation(p, precision="f64")
