"""Source-coupling ablation (Sec. 4.4) on the GPU: instantaneous against
accumulated coupling of the phase-change source at N_U = 100 (the Le = 100
directional saline-water case with the evolving temperature, on a smaller
lattice), both against the FP64 oracle, and the direction of the paper's
finding: accumulating the phase-change increments over the coarse solute
step concentrates them into larger jumps of U (J_U) than the immediate
transfer makes."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import active

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_2609_25670_b300 as lbm  # noqa: E402


def _run_pair(p, f, samples, every, precision):
    sim = lbm.Simulation(p, precision=precision)
    sim.init_fields(f)
    o = oracle.Oracle(p, f)
    g_hist, o_hist = [], []
    for _ in range(samples):
        sim.advance(every)
        o.advance(every)
        g_hist.append(sim.diagnostics())
        o_hist.append(o.diagnostics())
    got = {k: sim.field(k) for k in active(p)}
    ref = {k: o.get(k) for k in active(p)}
    sim.close()
    o.close()
    return g_hist, o_hist, got, ref


@pytest.mark.parametrize("precision,tol", [("f64", 1e-10), ("f32", 2e-4)])
def test_accumulated_coupling_concentrates_the_source_at_NU_100(precision, tol):
    """Le = 100 (N_U = 100), 200 x 160 lattice, 300 base steps sampled every
    100: S_phi and J_U of every sample and the fields equal the oracle's
    (FP64 within 1e-10; FP32 within a short-run rounding bound), and the
    accumulated coupling's largest U jump exceeds the instantaneous one by
    more than an order of magnitude, while its phase-change increments S_phi
    stay of the same size."""
    res = {}
    for acc in (False, True):
        wl = W.directional_evolving_T(Le=100, nx=200, ny=160)
        p = wl.params
        p.accumulated = acc
        g, o, got, ref = _run_pair(p, wl.fields, 3, 100, precision)
        for k in got:
            assert np.abs(got[k] - ref[k]).max() < tol, (acc, k, np.abs(got[k] - ref[k]).max())
        for gd, od in zip(g, o):
            for k in ("S_phi", "J_U"):
                assert abs(gd[k] - od[k]) <= tol * max(1.0, abs(od[k])), (acc, k, gd[k], od[k])
        res[acc] = (max(d["S_phi"] for d in o), max(d["J_U"] for d in o))
    (s_inst, j_inst), (s_acc, j_acc) = res[False], res[True]
    assert j_inst == pytest.approx(s_inst, rel=1e-12)        # instantaneous: the jump is the increment
    assert j_acc > 10.0 * j_inst, (j_acc, j_inst)
    assert 0.1 < s_acc / s_inst < 10.0, (s_acc, s_inst)
