"""Update-factor sweep of the thermal free dendrite (Sec. 4.1 with the
temperature update factor N_T varied at fixed physics): the reduced-precision
CUDA path's tip velocity against the FP64 oracle's, within 1 %, at every
N_T of the sweep."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2609_25670_b300 as lbm  # noqa: E402

EVERY, SAMPLES = 20, 100          # tip sampled every 20 base steps, 2000 steps


def _tip_velocity(hist):
    """Mean over the four axis tips of the tip advance over the last 500 base
    steps, per base step (Sec. 4.1's tip histories, central part of the run)."""
    h = np.asarray(hist)
    return float(((h[-1] - h[-26]) / (25 * EVERY)).mean())


def _oracle_history(p, f):
    o = oracle.Oracle(p, f)
    hist = []
    for _ in range(SAMPLES):
        o.advance(EVERY)
        hist.append(o.diagnostics()["tip"].copy())
    o.close()
    return hist


@pytest.mark.parametrize("q", [9, 5])
@pytest.mark.parametrize("N_T", [1, 2, 4])
@pytest.mark.parametrize("prec", ["f32", "f16dev"])
def test_tip_velocity_within_one_percent(prec, N_T, q):
    """q: the phase and temperature lattices on D2Q9 (the paper's) or D2Q5
    (the velocity sets the workload list names for this case)."""
    wl = W.thermal_free_dendrite(n=128, N_T=N_T)
    wl.params.q_scalar = q
    sim = lbm.Simulation(wl.params, precision=prec)
    sim.init_fields(wl.fields)
    hist = []
    for _ in range(SAMPLES):
        sim.advance(EVERY)
        hist.append(sim.diagnostics()["tip"].copy())
    sim.close()
    v_gpu = _tip_velocity(hist)
    v_orc = _tip_velocity(_oracle_history(wl.params, wl.fields))
    assert v_orc > 0.005
    assert abs(v_gpu - v_orc) < 0.01 * v_orc, (prec, N_T, v_gpu, v_orc)
