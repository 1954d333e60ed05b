"""Batched ensemble (one launch per kernel kind over the tiles of all
members): identical to advancing each member alone, and matching the oracle."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import active, run_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2609_25670_b300 as lbm  # noqa: E402


def members(count=6, seed=11):
    # uneven sizes, including ones the 32-wide tiles do not divide
    return W.ensemble_members(count=count, seed=seed, sizes=(40, 64, 72, 96))


def _run_ensemble(ms, steps, precision, batching=True, chunks=None):
    sim = lbm.Simulation([m.params for m in ms], precision=precision)
    if not batching:
        sim.set_batching(False)
    for i, m in enumerate(ms):
        sim.init_fields(m.fields, sim=i)
    for c in (chunks or [steps]):
        sim.advance(c)
    out = [{k: sim.field(k, sim=i) for k in active(m.params)} for i, m in enumerate(ms)]
    diags = [sim.diagnostics(sim=i) for i in range(len(ms))]
    sim.close()
    return out, diags


def test_batched_equals_each_member_alone():
    ms = members()
    steps = 24    # a multiple of the common period (2 * lcm(1, 2, 4) = 8)
    batched, _ = _run_ensemble(ms, steps, "f32")
    sequential, _ = _run_ensemble(ms, steps, "f32", batching=False)
    for i, m in enumerate(ms):
        sim = lbm.Simulation(m.params, precision="f32")
        sim.init_fields(m.fields)
        sim.advance(steps)
        alone = {k: sim.field(k) for k in active(m.params)}
        sim.close()
        for k in alone:
            assert np.array_equal(batched[i][k], alone[k]), (i, k)
            assert np.array_equal(sequential[i][k], alone[k]), (i, k)


def test_batched_unaligned_chunks_equal():
    ms = members(count=4, seed=12)
    a, _ = _run_ensemble(ms, 19, "f32")
    b, _ = _run_ensemble(ms, 19, "f32", chunks=[3, 8, 8])
    for i in range(len(ms)):
        for k in a[i]:
            assert np.array_equal(a[i][k], b[i][k]), (i, k)


def test_batched_fp64_matches_oracle():
    ms = members(count=3, seed=13)
    steps = 40
    got, diags = _run_ensemble(ms, steps, "f64")
    for i, m in enumerate(ms):
        o = run_oracle(m.params, m.fields, steps)
        for k in active(m.params):
            assert np.abs(got[i][k] - o[k]).max() < 1e-10, (i, k)
        assert abs(diags[i]["M_C"] - o["diag"]["M_C"]) < 1e-9 * o["diag"]["M_C"]


def test_autotune_batched_keeps_results():
    ms = W.ensemble_members(count=4, seed=14, sizes=(64, 96, 160, 256))
    sim = lbm.Simulation([m.params for m in ms], precision="f32")
    for i, m in enumerate(ms):
        sim.init_fields(m.fields, sim=i)
    sim.advance(8)
    sim.autotune(reps=2)
    sim.advance(16)
    tuned = [sim.field("phi", sim=i) for i in range(len(ms))]
    sim.close()
    ref, _ = _run_ensemble(ms, 24, "f32")
    for i in range(len(ms)):
        # tile shapes agree to floating-point contraction rounding
        assert np.abs(tuned[i] - ref[i]["phi"]).max() < 1e-5


@pytest.mark.parametrize("v", [-8, -32, 1016])
def test_batched_strips_equal_each_member_alone(v):
    """Warp-strip U / T kernels in the batched launches: bitwise the results
    of each member advanced alone with the same variant."""
    ms = W.ensemble_members(count=4, seed=14, sizes=(64, 96, 160, 256))
    steps = 16
    sim = lbm.Simulation([m.params for m in ms], precision="f32")
    for k in ("scalar_U", "scalar_T"):
        sim.set_tile(k, v)
    for i, m in enumerate(ms):
        sim.init_fields(m.fields, sim=i)
    sim.advance(steps)
    batched = [{k: sim.field(k, sim=i) for k in active(m.params)} for i, m in enumerate(ms)]
    sim.close()
    for i, m in enumerate(ms):
        sim = lbm.Simulation(m.params, precision="f32")
        for k in ("scalar_U", "scalar_T"):
            sim.set_tile(k, v)
        sim.init_fields(m.fields)
        sim.advance(steps)
        for k in active(m.params):
            assert np.array_equal(batched[i][k], sim.field(k)), (i, k)
        sim.close()
