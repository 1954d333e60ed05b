"""Host-side pieces of the inputs and of the measurement, on the CPU: the
stable variants of the listed workloads, the windowed generation of the
multi-dendrite fields, and the byte model the bench's roofline divides by."""
import math
import os
import sys

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _taus(p):
    tau_phi = 3.0 * p.N_phi * p.dt_base * p.W0 * p.W0 / p.tau0 + 0.5
    return tau_phi, W.tau_U(p, -1.0), W.tau_U(p, 1.0)


@pytest.mark.parametrize("make", [
    lambda: W.thermosolutal_convection(512).params,
    lambda: W.directional_saline(Le=1).params,
    lambda: W.directional_saline(Le=100).params,
    lambda: W.multi_dendrite_params(8192)[0],
])
def test_stable_variant_brings_every_relaxation_time_into_range(make):
    """Eq. 24 with D_eff of Eq. 7: after stable_variant every relaxation time
    of phi and U is >= 0.52, with the smallest update factors that do it, and
    the liquid diffusivity, k and the other factors untouched."""
    p = make()
    before = (p.N_T, p.N_F, p.DL, p.k, p.tau0, p.W0)
    listed = (p.N_phi, p.N_U)
    W.stable_variant(p)
    assert (p.N_T, p.N_F, p.DL, p.k, p.tau0, p.W0) == before
    assert p.N_phi >= listed[0] and p.N_U >= listed[1]
    for t in _taus(p):
        assert t >= 0.52 - 1e-12, _taus(p)
    # minimal factors: a raised factor one less would leave tau_phi or tau_U,L below 0.52
    if p.N_phi > listed[0]:
        assert 3.0 * (p.N_phi - 1) * p.W0 ** 2 / p.tau0 + 0.5 < 0.52
    if p.N_U > listed[1]:
        q = W.Params(**p.as_dict())
        q.N_U -= 1
        assert W.tau_U(q, -1.0) < 0.52


def test_stable_variant_of_the_multi_dendrite_case():
    """The 8192^2 listed instance: tau_phi 0.515, tau_U 0.515 / 0.5005 ->
    N = (2, 2, 4, 2), D_S = 0.2 D_L."""
    p = W.multi_dendrite_params(8192)[0]
    assert _taus(p)[0] == pytest.approx(0.515)
    W.stable_variant(p)
    assert (p.N_phi, p.N_U, p.N_T, p.N_F) == (2, 2, 4, 2)
    assert p.DS / p.DL == pytest.approx(0.2)


def test_in_range_workload_is_unchanged():
    p = W.directional_evolving_T(Le=100).params          # tau_U,S = 1.28 with k = 0.001
    d = p.as_dict()
    W.stable_variant(p)
    assert p.as_dict() == d


def test_multi_dendrite_fields_equal_the_full_evaluation():
    p, pts = W.multi_dendrite_params(384)
    a = W.multi_dendrite_fields(p, pts)
    b = W.multi_dendrite(384).fields
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_bench_byte_model():
    """Algorithmic bytes per node of the reported workload (D2Q5 phase, U, T
    with grain angles, D2Q9 flow, N = (1, 1, 4, 2)): 52 + 24 + 40 + 36/4 +
    92/2 = 171 B in FP32, 36 + 24 + 32 + 28/4 + 60/2 = 129 B with FP16
    deviation storage; the stable variant's N_phi = 2 halves phase and
    transfer."""
    sys.path.insert(0, ROOT)
    import bench
    p, _ = bench.md_workload(8192, 5)
    assert bench.step_bytes_md(p, "f32", False, 5) == 171
    assert bench.step_bytes_md(p, "f16dev", False, 5) == 129
    W.stable_variant(p)
    assert bench.step_bytes_md(p, "f32", False, 5) == pytest.approx((52 + 24) / 2 + 40 / 2 + 36 / 4 + 92 / 2)
    ab = bench.algo_bytes("f32", 9, ori=True)
    assert ab == {"phase": 84, "transfer": 24, "scalar_U": 40, "scalar_T": 36, "flow": 92}
    assert bench.algo_bytes("f64", 9)["scalar_U"] == 72          # FP64 keeps no residual plane
