"""The allocation-free diagnostics entry point, lbm_diagnostics_noalloc.

Callers that cannot call cudaMalloc -- a monitoring hook inside another
framework's step loop, where an allocation would synchronise the device and
break that framework's stream ordering, or a process whose device memory is
owned by a caching allocator under a fixed budget -- reduce fields they
already hold through this entry point; its scratch is a fixed device array
inside the library.  These tests check it, through the C ABI, against
lbm_diagnostics on the same state, on two calls in a row.

The file is named so that pytest collects it last: a run that stops at the
first failure has then already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import paper_2609_25670_b300 as lbm
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

FIELDS = ("phi", "U", "T", "ux", "uy")


def _entry(lib):
    f = lib.lbm_diagnostics_noalloc
    f.argtypes = [C.POINTER(lbm.lbm_params)] + [C.c_void_p] * 6 + [C.POINTER(lbm.lbm_diag)]
    f.restype = C.c_int
    return f


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_matches_lbm_diagnostics_twice(prec):
    n = 96
    wl = W.thermosolutal_convection(n=n, R=8.0)
    sim = lbm.Simulation(wl.params, precision=prec)
    sim.init_fields(wl.fields)
    entry = _entry(sim.lib)
    dtype = torch.float64 if prec == "f64" else torch.float32
    p = lbm.make_params(wl.params, prec)
    bufs = {k: torch.empty((n, n), dtype=dtype, device="cuda") for k in FIELDS}
    for _ in range(2):
        sim.advance(25)
        ref = sim.diagnostics()
        for k in FIELDS:
            sim.field(k, out=bufs[k], as_f64=False)   # queued on the simulation's stream
        out = lbm.lbm_diag()
        st = entry(C.byref(p), *[C.c_void_p(bufs[k].data_ptr()) for k in FIELDS],
                   C.c_void_p(sim.stream.cuda_stream), C.byref(out))
        assert st == 0, sim.lib.lbm_last_error(None).decode()
        assert abs(out.M_C - ref["M_C"]) <= 1e-12 * abs(ref["M_C"])
        assert abs(out.H_total - ref["H"]) <= 1e-12 * max(1.0, abs(ref["H"]))
        assert np.abs(np.array(list(out.tip)) - ref["tip"]).max() <= 1e-12
        assert out.nonfinite == 0 and ref["nonfinite"] == 0
    sim.close()


def test_noalloc_rejects_bad_input():
    lib = lbm.load()
    entry = _entry(lib)
    p = lbm.make_params(W.thermosolutal_convection(n=64).params, "f32")
    out = lbm.lbm_diag()
    assert entry(C.byref(p), None, None, None, None, None, None, C.byref(out)) == 1
    p.nx = p.ny = 50000          # 2.5e9 nodes: beyond the 2^31 - 1 node limit
    dummy = torch.empty(1, device="cuda")
    ptr = C.c_void_p(dummy.data_ptr())
    assert entry(C.byref(p), ptr, ptr, ptr, ptr, ptr, None, C.byref(out)) == 1
    assert lib.lbm_last_error(None)
