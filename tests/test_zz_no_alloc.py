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


def _solute_tolerance(prec, p, U, M_C):
    """lbm_diagnostics adds the residual of the compensated U macro (FP32
    arithmetic) to the solute sum; the caller's FP32 U field holds U rounded
    to FP32, at most half a unit in the last place from hi + lo.  So the two
    sums differ by at most (1 - k)/2 * max D(phi) * sum_i ulp(U_i) / 2, with
    D(phi) = (1 + k) - (1 - k) phi <= 2; FP64 keeps no residual."""
    if prec == "f64":
        return 1e-12 * abs(M_C)
    u = U.detach().cpu().numpy().astype(np.float32)
    return 0.5 * (1.0 - p.k) * float(np.sum(np.spacing(np.abs(u)).astype(np.float64))) + 1e-12 * abs(M_C)


@pytest.mark.parametrize("prec,n", [("f32", 96), ("f64", 96), ("f16dev", 96), ("f32", 1024)])
def test_noalloc_matches_lbm_diagnostics_twice(prec, n):
    """Two calls in a row on a state that moves between them; 1024^2 has more
    nodes than the 1184 x 256 threads of the fixed scratch, so each thread
    strides over several of them; f16dev reads the same float fields."""
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
        assert abs(out.M_C - ref["M_C"]) <= _solute_tolerance(prec, wl.params, bufs["U"], ref["M_C"])
        assert abs(out.H_total - ref["H"]) <= 1e-12 * max(1.0, abs(ref["H"]))
        assert np.abs(np.array(list(out.tip)) - ref["tip"]).max() <= 1e-12
        assert out.nonfinite == 0 and ref["nonfinite"] == 0
        assert out.R_M == 0.0 and out.S_phi == 0.0 and out.J_U == 0.0
    sim.close()


def test_noalloc_reports_a_nonfinite_field():
    """A NaN written into the caller's U field on the host side of the test:
    the call returns LBM_E_NONFINITE and still fills out (nonfinite = 1, the
    tips of the finite phase field)."""
    n = 96
    wl = W.thermosolutal_convection(n=n, R=8.0)
    lib = lbm.load()
    entry = _entry(lib)
    p = lbm.make_params(wl.params, "f32")
    bufs = {k: torch.from_numpy(np.ascontiguousarray(wl.fields[k], dtype=np.float32)).cuda() for k in FIELDS}
    bufs["U"][n // 3, n // 5] = float("nan")
    torch.cuda.synchronize()
    out = lbm.lbm_diag()
    st = entry(C.byref(p), *[C.c_void_p(bufs[k].data_ptr()) for k in FIELDS], None, C.byref(out))
    assert st == 5, lib.lbm_last_error(None).decode()
    assert out.nonfinite == 1
    assert np.all(np.isfinite(np.array(list(out.tip)))) and max(out.tip) > 0


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


def test_noalloc_refuses_a_capturing_stream():
    """The call synchronises its stream, which no capture allows: on a stream
    that is being captured it returns LBM_E_INVALID_ARG before any work, and
    the capture can then be ended normally."""
    n = 64
    wl = W.thermosolutal_convection(n=n, R=8.0)
    lib = lbm.load()
    entry = _entry(lib)
    p = lbm.make_params(wl.params, "f32")
    bufs = {k: torch.from_numpy(np.ascontiguousarray(wl.fields[k], dtype=np.float32)).cuda() for k in FIELDS}
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    out = lbm.lbm_diag()
    with torch.cuda.graph(g, stream=s):
        bufs["phi"].mul_(1.0)                     # some captured work
        st = entry(C.byref(p), *[C.c_void_p(bufs[k].data_ptr()) for k in FIELDS], C.c_void_p(s.cuda_stream),
                   C.byref(out))
    assert st == 1
    assert "capture" in lib.lbm_last_error(None).decode()
