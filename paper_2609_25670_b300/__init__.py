"""Python binding of the B300 multirate MRT-LBM library (include/lbm.h).

Argument marshalling only: every step of the lattice Boltzmann path runs in
the CUDA kernels of liblbm.so.  PyTorch supplies device memory (through the
library's allocator callback into torch's caching allocator) and the CUDA
stream.  There is no fallback: if liblbm.so is missing or cannot be loaded,
``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Iterable, List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

PARAMS_VERSION = 3
BC_PERIODIC, BC_WALL, BC_INLET_OUTFLOW = 0, 1, 2
FIELD_U, FIELD_T, FIELD_FROZEN_T, FIELD_FLOW = 1, 2, 4, 8
PRECISIONS = {"f64": 0, "f32": 1, "f16dev": 2, "bf16dev": 3}
COUPLING_INSTANTANEOUS, COUPLING_ACCUMULATED = 0, 1
SEED_CIRCLE, SEED_PLANAR, SEED_SINUSOID = 0, 1, 2
OUT_FIELDS = {"phi": 0, "U": 1, "T": 2, "ux": 3, "uy": 4, "rho": 5, "C": 6, "theta": 7}
KERNEL_KINDS = ["phase", "transfer", "scalar_U", "scalar_T", "flow", "diag", "init", "transport"]
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSTABLE_PARAMS", 3: "OOM", 4: "CUDA", 5: "NONFINITE",
          6: "TIMEOUT", 7: "STATE"}

EXPORTED = ["lbm_create", "lbm_init_seed", "lbm_init_fields", "lbm_advance", "lbm_fields",
            "lbm_diagnostics", "lbm_last_error", "lbm_destroy", "lbm_set_graphs", "lbm_timing_enable",
            "lbm_timing_read", "lbm_launch_counts", "lbm_device_bytes", "lbm_autotune",
            "lbm_diagnostics_noalloc", "lbm_set_batching", "lbm_set_tile", "lbm_set_fusion",
            "lbm_get_fusion", "lbm_set_orientation"]


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class lbm_params(C.Structure):
    _fields_ = [
        ("struct_version", C.c_uint32), ("nx", C.c_int32), ("ny", C.c_int32), ("fields", C.c_uint32),
        ("bc_scalar_x", C.c_int32), ("bc_scalar_y", C.c_int32), ("bc_flow_x", C.c_int32),
        ("bc_flow_y", C.c_int32), ("precision", C.c_uint32), ("coupling", C.c_uint32),
        ("N_phi", C.c_int32), ("N_U", C.c_int32), ("N_T", C.c_int32), ("N_F", C.c_int32),
        ("tip_cx", C.c_int32), ("tip_cy", C.c_int32), ("T_ymin_dirichlet", C.c_int32),
        ("q_scalar", C.c_int32), ("dt_base", C.c_double),
        ("W0", C.c_double), ("tau0", C.c_double), ("eps", C.c_double), ("lam", C.c_double),
        ("Mc", C.c_double), ("k", C.c_double), ("DL", C.c_double), ("DS", C.c_double),
        ("kappaS", C.c_double), ("kappaL", C.c_double), ("rhoCpS", C.c_double), ("rhoCpL", C.c_double),
        ("rhoL_Lh", C.c_double), ("T_shift", C.c_double), ("T_scale", C.c_double),
        ("nu", C.c_double), ("u_in", C.c_double), ("Fbx", C.c_double), ("Fby", C.c_double),
        ("s_e", C.c_double), ("s_eps", C.c_double), ("s_q", C.c_double),
        ("theta_c", C.c_double), ("frozen_G", C.c_double), ("frozen_y0", C.c_double),
        ("frozen_V", C.c_double), ("T_ymin", C.c_double),
    ]


class lbm_seed(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("x", C.c_double), ("y", C.c_double),
                ("r", C.c_double), ("amp", C.c_double), ("waves", C.c_double)]


class lbm_diag(C.Structure):
    _fields_ = [("base_step", C.c_int64), ("M_C", C.c_double), ("H_total", C.c_double),
                ("S_phi", C.c_double), ("J_U", C.c_double), ("tip", C.c_double * 4),
                ("nonfinite", C.c_int32), ("reserved", C.c_int32), ("R_M", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class lbm_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load liblbm.so (raises OSError if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("liblbm.so not found at %s; run paper_2609_25670_b300/build.py" % path)
    lib = C.CDLL(path)
    vp, i32, i64, u32, dp = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.POINTER(C.c_double)
    lib.lbm_create.argtypes = [C.POINTER(lbm_params), i32, C.POINTER(lbm_params), C.POINTER(lbm_allocator), vp,
                               C.POINTER(vp)]
    lib.lbm_init_seed.argtypes = [vp, i32, C.POINTER(lbm_seed), i32, C.c_double, C.c_double, C.c_uint64]
    lib.lbm_init_fields.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, i32]
    lib.lbm_advance.argtypes = [vp, i64]
    lib.lbm_fields.argtypes = [vp, i32, u32, vp, i32, i32]
    lib.lbm_diagnostics.argtypes = [vp, i32, C.POINTER(lbm_diag)]
    lib.lbm_last_error.argtypes = [vp]
    lib.lbm_last_error.restype = C.c_char_p
    lib.lbm_destroy.argtypes = [vp]
    lib.lbm_destroy.restype = None
    lib.lbm_set_graphs.argtypes = [vp, i32]
    lib.lbm_timing_enable.argtypes = [vp, u32]
    lib.lbm_timing_read.argtypes = [vp, dp, C.POINTER(C.c_int64), i32]
    lib.lbm_launch_counts.argtypes = [vp, C.POINTER(C.c_int64)]
    lib.lbm_device_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
    lib.lbm_autotune.argtypes = [vp, i32, C.POINTER(C.c_int32)]
    lib.lbm_set_batching.argtypes = [vp, i32]
    lib.lbm_set_tile.argtypes = [vp, i32, i32]
    lib.lbm_set_fusion.argtypes = [vp, i32]
    lib.lbm_get_fusion.argtypes = [vp, C.POINTER(C.c_int32)]
    lib.lbm_diagnostics_noalloc.argtypes = [C.POINTER(lbm_params)] + [vp] * 6 + [C.POINTER(lbm_diag)]
    lib.lbm_set_orientation.argtypes = [vp, i32, vp, i32]
    for nm in EXPORTED:
        f = getattr(lib, nm)
        if nm not in ("lbm_last_error", "lbm_destroy"):
            f.restype = C.c_int
    _lib = lib
    return lib


def _get(p, name, default=None):
    if isinstance(p, dict):
        return p.get(name, default)
    return getattr(p, name, default)


def make_params(p, precision: str = "f32") -> lbm_params:
    """Fill lbm_params from an object or dict with the workload attribute names
    (nx, ny, has_U, has_T, frozen_T, has_flow, bc_*, accumulated, N_*, ...)."""
    s = lbm_params()
    s.struct_version = PARAMS_VERSION
    s.nx, s.ny = int(_get(p, "nx")), int(_get(p, "ny"))
    f = 0
    if _get(p, "has_U", False): f |= FIELD_U
    if _get(p, "has_T", False): f |= FIELD_T
    if _get(p, "frozen_T", False): f |= FIELD_FROZEN_T
    if _get(p, "has_flow", False): f |= FIELD_FLOW
    s.fields = f
    s.bc_scalar_x = int(_get(p, "bc_scalar_x", BC_WALL))
    s.bc_scalar_y = int(_get(p, "bc_scalar_y", BC_WALL))
    s.bc_flow_x = int(_get(p, "bc_flow_x", BC_PERIODIC))
    s.bc_flow_y = int(_get(p, "bc_flow_y", BC_PERIODIC))
    s.precision = PRECISIONS[precision]
    s.coupling = COUPLING_ACCUMULATED if _get(p, "accumulated", False) else COUPLING_INSTANTANEOUS
    for nm in ("N_phi", "N_U", "N_T", "N_F"):
        setattr(s, nm, int(_get(p, nm, 1)))
    s.tip_cx, s.tip_cy = int(_get(p, "tip_cx", 0)), int(_get(p, "tip_cy", 0))
    s.T_ymin_dirichlet = 1 if _get(p, "T_ymin_dirichlet", False) else 0
    s.q_scalar = int(_get(p, "q_scalar", 9))
    defaults = dict(dt_base=1.0, W0=1.0, tau0=1.0, eps=0.0, lam=0.0, Mc=0.0, k=1.0, DL=0.0, DS=0.0,
                    kappaS=0.0, kappaL=0.0, rhoCpS=1.0, rhoCpL=1.0, rhoL_Lh=1.0, T_shift=0.0, T_scale=1.0,
                    nu=0.1, u_in=0.0, Fbx=0.0, Fby=0.0, s_e=1.2, s_eps=1.4, s_q=1.2, theta_c=0.0,
                    frozen_G=0.0, frozen_y0=0.0, frozen_V=0.0, T_ymin=0.0)
    for nm, dv in defaults.items():
        setattr(s, nm, float(_get(p, nm, dv)))
    return s


def _ptr(a) -> int:
    """Address of a numpy array or a torch tensor (contiguous float64 expected)."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return int(a.data_ptr())


class Simulation:
    """One or more simulations advanced together on the current CUDA device.

    params: an object / dict with the workload attributes (see make_params), or
    a list of them for an ensemble (all with the same precision)."""

    def __init__(self, params, precision: str = "f32", stream=None, torch_allocator: bool = True):
        import torch
        self._torch = torch
        self.lib = load()
        plist = list(params) if isinstance(params, (list, tuple)) else [params]
        self.params = plist
        self._ps = (lbm_params * len(plist))(*[make_params(p, precision) for p in plist])
        self.precision = precision
        self.n_sims = len(plist)
        self.nx = [int(_get(p, "nx")) for p in plist]
        self.ny = [int(_get(p, "ny")) for p in plist]
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self._keep = []
        alloc_ptr = None
        if torch_allocator:
            dev = torch.cuda.current_device()
            tstream = self.stream

            def _alloc(nbytes, _stream, _ctx):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, tstream)
                except Exception:
                    return None

            def _free(ptr, _nbytes, _stream, _ctx):
                torch.cuda.caching_allocator_delete(ptr)

            a = lbm_allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
            self._keep += [a]
            alloc_ptr = C.byref(a)
        h = C.c_void_p()
        st = self.lib.lbm_create(C.byref(self._ps[0]), self.n_sims,
                                 self._ps if self.n_sims > 1 else None, alloc_ptr,
                                 C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != 0:
            raise LbmError(st, self.lib.lbm_last_error(None).decode())
        self.h = h

    # ---- error helper
    def _ck(self, st: int):
        if st != 0:
            raise LbmError(st, self.lib.lbm_last_error(self.h).decode())

    # ---- initialisation
    def set_orientation(self, theta, sim: int = 0):
        """Per-node crystal angle of the grains ((ny, nx) float64 numpy array
        or CUDA tensor), or None for the axis-aligned anisotropy."""
        if theta is None:
            self._ck(self.lib.lbm_set_orientation(self.h, sim, None, 0))
            return
        if isinstance(theta, np.ndarray):
            theta = np.ascontiguousarray(theta, dtype=np.float64)
            dev = 0
        else:
            assert theta.dtype == self._torch.float64 and theta.is_contiguous()
            dev = 1 if theta.is_cuda else 0
            if dev:
                self.stream.wait_stream(self._torch.cuda.current_stream())
        self._ck(self.lib.lbm_set_orientation(self.h, sim, C.c_void_p(_ptr(theta)), dev))

    def init_fields(self, fields: Dict, sim: int = 0):
        """fields: phi, U, T, ux, uy, rho as (ny, nx) float64 host numpy arrays,
        or contiguous float64 CUDA tensors (all of one kind); an optional
        "theta" entry sets the grain orientation first (set_orientation)."""
        if "theta" in fields:
            self.set_orientation(fields["theta"], sim)
        keys = ("phi", "U", "T", "ux", "uy", "rho")
        arrs = []
        dev = 0
        for k in keys:
            a = fields.get(k)
            if a is None:
                arrs.append(None)
                continue
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, dtype=np.float64)
            else:
                dev = 1 if a.is_cuda else 0
                assert a.dtype == self._torch.float64 and a.is_contiguous()
            arrs.append(a)
        ptrs = [C.c_void_p(_ptr(a)) if a is not None else None for a in arrs]
        if dev:     # the tensors were written on torch's current stream
            self.stream.wait_stream(self._torch.cuda.current_stream())
        self._ck(self.lib.lbm_init_fields(self.h, sim, *ptrs, dev))

    def init_seed(self, seeds: Sequence[Dict], U0: float = 0.0, T0: float = 0.0, rng_seed: int = 0, sim: int = 0):
        kinds = {"circle": SEED_CIRCLE, "planar": SEED_PLANAR, "sinusoid": SEED_SINUSOID}
        arr = (lbm_seed * len(seeds))()
        for i, s in enumerate(seeds):
            arr[i].kind = kinds[s["kind"]] if isinstance(s["kind"], str) else int(s["kind"])
            for nm in ("x", "y", "r", "amp", "waves"):
                setattr(arr[i], nm, float(s.get(nm, 0.0)))
        self._ck(self.lib.lbm_init_seed(self.h, sim, arr, len(seeds), float(U0), float(T0), int(rng_seed)))

    # ---- stepping
    def advance(self, n_base_steps: int):
        self._ck(self.lib.lbm_advance(self.h, int(n_base_steps)))

    def set_batching(self, enable: bool):
        """Ensembles: one launch per kernel kind over all members (default) or
        members one after another."""
        self._ck(self.lib.lbm_set_batching(self.h, 1 if enable else 0))

    def set_tile(self, kind: str, ty: int):
        """Fix the tile height of one update kernel kind (4, 8 or 16)."""
        self._ck(self.lib.lbm_set_tile(self.h, KERNEL_KINDS.index(kind), int(ty)))

    def set_fusion(self, enable: bool):
        """One fused launch per base step after the phase update, or one per
        stage (the default until autotune() has timed both); fixes the choice."""
        self._ck(self.lib.lbm_set_fusion(self.h, 1 if enable else 0))

    @property
    def fused(self) -> bool:
        v = C.c_int32(0)
        self._ck(self.lib.lbm_get_fusion(self.h, C.byref(v)))
        return bool(v.value)

    def set_graphs(self, enable: bool):
        self._ck(self.lib.lbm_set_graphs(self.h, 1 if enable else 0))

    # ---- outputs
    def field(self, name: str, sim: int = 0, out=None, as_f64: bool = True):
        """Copy a macroscopic field: into `out` (numpy host array or CUDA tensor)
        if given, else into a new float64 numpy array."""
        which = OUT_FIELDS[name]
        if out is None:
            out = np.empty((self.ny[sim], self.nx[sim]), dtype=np.float64 if as_f64 else
                           (np.float64 if self.precision == "f64" else np.float32))
        dev = 0 if isinstance(out, np.ndarray) else (1 if out.is_cuda else 0)
        if dev:     # ordered after the tensor's last use on torch's current stream
            self.stream.wait_stream(self._torch.cuda.current_stream())
        self._ck(self.lib.lbm_fields(self.h, sim, which, C.c_void_p(_ptr(out)), dev, 1 if as_f64 else 0))
        if dev:     # and its readers after the library's write
            self._torch.cuda.current_stream().wait_stream(self.stream)
        return out

    def diagnostics(self, sim: int = 0, raise_nonfinite: bool = False) -> Dict:
        d = lbm_diag()
        st = self.lib.lbm_diagnostics(self.h, sim, C.byref(d))
        if st != 0 and (st != 5 or raise_nonfinite):
            self._ck(st)
        return {"base_step": d.base_step, "M_C": d.M_C, "R_M": d.R_M, "H": d.H_total, "S_phi": d.S_phi,
                "J_U": d.J_U, "tip": np.array(list(d.tip)), "nonfinite": d.nonfinite, "status": st}

    # ---- measurement hooks
    def timing_enable(self, kinds: Iterable[str]):
        mask = 0
        for k in kinds:
            mask |= 1 << KERNEL_KINDS.index(k)
        self._ck(self.lib.lbm_timing_enable(self.h, mask))

    def timing_read(self, reset: bool = False) -> Dict[str, tuple]:
        ms = (C.c_double * len(KERNEL_KINDS))()
        cnt = (C.c_int64 * len(KERNEL_KINDS))()
        self._ck(self.lib.lbm_timing_read(self.h, ms, cnt, 1 if reset else 0))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_KINDS)}

    def autotune(self, reps: int = 20) -> Dict[str, int]:
        """Pick the fastest compiled tile height per kernel kind on the current state."""
        ch = (C.c_int32 * len(KERNEL_KINDS))()
        self._ck(self.lib.lbm_autotune(self.h, int(reps), ch))
        return {k: ch[i] for i, k in enumerate(KERNEL_KINDS)}

    def launch_counts(self) -> Dict[str, int]:
        cnt = (C.c_int64 * len(KERNEL_KINDS))()
        self._ck(self.lib.lbm_launch_counts(self.h, cnt))
        return {k: cnt[i] for i, k in enumerate(KERNEL_KINDS)}

    def device_bytes(self) -> int:
        b = C.c_size_t()
        self._ck(self.lib.lbm_device_bytes(self.h, C.byref(b)))
        return b.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
