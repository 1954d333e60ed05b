"""FP64 CPU oracle of the multirate MRT-LBM (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. It shares no code with the CUDA path; its only
common input is the ``workloads`` module (parameter sets and seeded initial
fields).

The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64, literal moment-space
products); this file compiles it with gcc and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c into liblbm_oracle.so (gcc, -O2, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
               _SRC, "-o", _LIB, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


class _OrcParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32),
        ("has_U", C.c_int32), ("has_T", C.c_int32), ("frozen_T", C.c_int32), ("has_flow", C.c_int32),
        ("bc_scalar_x", C.c_int32), ("bc_scalar_y", C.c_int32),
        ("bc_flow_x", C.c_int32), ("bc_flow_y", C.c_int32),
        ("accumulated", C.c_int32),
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


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        lib.orc_create.restype = C.c_void_p
        lib.orc_create.argtypes = [C.POINTER(_OrcParams)]
        lib.orc_destroy.argtypes = [C.c_void_p]
        lib.orc_set_fields.argtypes = [C.c_void_p] + [dp] * 6
        lib.orc_advance.argtypes = [C.c_void_p, C.c_int64]
        lib.orc_stage.argtypes = [C.c_void_p, C.c_int]
        lib.orc_get.argtypes = [C.c_void_p, C.c_int, dp]
        lib.orc_diag.argtypes = [C.c_void_p, dp]
        lib.orc_step.restype = C.c_int64
        lib.orc_step.argtypes = [C.c_void_p]
        lib.orc_aniso.argtypes = [C.c_double, C.c_double, C.c_double, dp, dp, dp]
        for nm in ("orc_feq_scalar", "orc_meq_scalar", "orc_feq_phase", "orc_meq_phase",
                   "orc_feq_flow", "orc_meq_flow"):
            getattr(lib, nm).argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, dp]
        lib.orc_matrices.argtypes = [dp, dp, C.POINTER(C.c_int), C.POINTER(C.c_int), dp]
        lib.orc_collide_scalar.argtypes = [dp, dp, C.c_double, C.c_double, dp]
        lib.orc_aniso_frame.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, dp, dp, dp]
        lib.orc_set_orientation.argtypes = [C.c_void_p, C.c_void_p]
        lib.orc_collide_scalar_q.argtypes = [C.c_int, dp, dp, C.c_double, C.c_double, dp]
        lib.orc_matrices5.argtypes = [dp, dp, dp]
        for nm in ("orc_feq_scalar_q", "orc_meq_scalar_q", "orc_feq_phase_q", "orc_meq_phase_q"):
            getattr(lib, nm).argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, dp]
        lib.orc_relaxation_times.argtypes = [C.POINTER(_OrcParams), C.c_double, dp]
        lib.orc_num_threads.restype = C.c_int
        lib.orc_set_threads.argtypes = [C.c_int]
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def to_orc_params(p) -> _OrcParams:
    d = p.as_dict() if hasattr(p, "as_dict") else dict(p)
    o = _OrcParams()
    o.nx, o.ny = int(d["nx"]), int(d["ny"])
    o.has_U, o.has_T = int(bool(d["has_U"])), int(bool(d["has_T"]))
    o.frozen_T, o.has_flow = int(bool(d["frozen_T"])), int(bool(d["has_flow"]))
    o.bc_scalar_x, o.bc_scalar_y = int(d["bc_scalar_x"]), int(d["bc_scalar_y"])
    o.bc_flow_x, o.bc_flow_y = int(d["bc_flow_x"]), int(d["bc_flow_y"])
    o.accumulated = int(bool(d["accumulated"]))
    o.N_phi, o.N_U, o.N_T, o.N_F = int(d["N_phi"]), int(d["N_U"]), int(d["N_T"]), int(d["N_F"])
    o.tip_cx, o.tip_cy = int(d["tip_cx"]), int(d["tip_cy"])
    o.T_ymin_dirichlet = int(bool(d.get("T_ymin_dirichlet", False)))
    o.q_scalar = int(d.get("q_scalar", 9))
    for nm in ("dt_base", "W0", "tau0", "eps", "lam", "Mc", "k", "DL", "DS", "kappaS", "kappaL",
               "rhoCpS", "rhoCpL", "rhoL_Lh", "T_shift", "T_scale", "nu", "u_in", "Fbx", "Fby",
               "s_e", "s_eps", "s_q", "theta_c", "frozen_G", "frozen_y0", "frozen_V"):
        setattr(o, nm, float(d[nm]))
    o.T_ymin = float(d.get("T_ymin", 0.0))
    return o


FIELD_IDS = {"phi": 0, "U": 1, "T": 2, "ux": 3, "uy": 4, "rho": 5, "C": 6, "theta": 7,
             "dU": 8, "dT": 9, "phi_new": 10}


class Oracle:
    """One FP64 simulation. ``fields`` are (ny, nx) float64 arrays."""

    def __init__(self, params, fields: Dict[str, np.ndarray]):
        self._lib = _load()
        self.params = params
        self._p = to_orc_params(params)
        self.nx, self.ny = self._p.nx, self._p.ny
        self._h = self._lib.orc_create(C.byref(self._p))
        self.set_fields(fields)

    def set_fields(self, fields: Dict[str, np.ndarray]):
        """Initial macroscopic fields; an optional "theta" entry is the
        per-node crystal angle of the grains (R-orientation)."""
        th = fields.get("theta")
        if th is not None:
            th = np.ascontiguousarray(th, dtype=np.float64)
            assert th.shape == (self.ny, self.nx)
            self._lib.orc_set_orientation(self._h, th.ctypes.data)
        else:
            self._lib.orc_set_orientation(self._h, None)
        arrs = [np.ascontiguousarray(fields[k], dtype=np.float64) for k in ("phi", "U", "T", "ux", "uy", "rho")]
        for a in arrs:
            assert a.shape == (self.ny, self.nx)
        self._lib.orc_set_fields(self._h, *[_dp(a) for a in arrs])

    def advance(self, n: int):
        self._lib.orc_advance(self._h, int(n))

    def stage(self, which: int):
        self._lib.orc_stage(self._h, int(which))

    @property
    def step(self) -> int:
        return int(self._lib.orc_step(self._h))

    def get(self, which) -> np.ndarray:
        wid = FIELD_IDS[which] if isinstance(which, str) else int(which)
        out = np.empty((self.ny, self.nx), dtype=np.float64)
        self._lib.orc_get(self._h, wid, _dp(out))
        return out

    def pops(self, field: str) -> np.ndarray:
        base = {"phi": 11, "U": 20, "T": 29, "F": 38}[field]
        return np.stack([self.get(base + i) for i in range(9)])

    def diagnostics(self) -> Dict[str, float]:
        out = np.zeros(10)
        self._lib.orc_diag(self._h, _dp(out))
        return {"M_C": out[0], "H": out[1], "S_phi": out[2], "J_U": out[3],
                "tip": out[4:8].copy(), "nonfinite": int(out[8]), "base_step": int(out[9])}

    def close(self):
        if self._h:
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- thin access to the oracle's exported pieces, for the pins ----
def matrices():
    lib = _load()
    M = np.zeros(81)
    Mi = np.zeros(81)
    ex = (C.c_int * 9)()
    ey = (C.c_int * 9)()
    w = np.zeros(9)
    lib.orc_matrices(_dp(M), _dp(Mi), ex, ey, _dp(w))
    return M.reshape(9, 9), Mi.reshape(9, 9), np.array(ex[:]), np.array(ey[:]), w


def matrices5():
    """M, M^-1 and the weights of the five-velocity scalar lattice."""
    lib = _load()
    M = np.zeros(25)
    Mi = np.zeros(25)
    w = np.zeros(5)
    lib.orc_matrices5(_dp(M), _dp(Mi), _dp(w))
    return M.reshape(5, 5), Mi.reshape(5, 5), w


def equilibrium_q(q: int, kind: str, a: float, ux: float, uy: float, c: float):
    """f_eq and m_eq of the scalar ("scalar") or phase ("phase") equilibrium on
    the q-velocity lattice (q = 9 or 5)."""
    lib = _load()
    f = np.zeros(q)
    m = np.zeros(q)
    getattr(lib, "orc_feq_%s_q" % kind)(q, a, ux, uy, c, _dp(f))
    getattr(lib, "orc_meq_%s_q" % kind)(q, a, ux, uy, c, _dp(m))
    return f, m


def collide_scalar_q(q: int, f: np.ndarray, meq: np.ndarray, tau: float, dtQ: float) -> np.ndarray:
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    meq = np.ascontiguousarray(meq, dtype=np.float64)
    out = np.zeros(q)
    lib.orc_collide_scalar_q(int(q), _dp(f), _dp(meq), float(tau), float(dtQ), _dp(out))
    return out


def equilibrium(kind: str, a: float, ux: float, uy: float, c: float):
    lib = _load()
    f = np.zeros(9)
    m = np.zeros(9)
    getattr(lib, "orc_feq_" + kind)(a, ux, uy, c, _dp(f))
    getattr(lib, "orc_meq_" + kind)(a, ux, uy, c, _dp(m))
    return f, m


def aniso(gx: float, gy: float, eps: float):
    lib = _load()
    a, nx, ny = C.c_double(), C.c_double(), C.c_double()
    lib.orc_aniso(gx, gy, eps, C.byref(a), C.byref(nx), C.byref(ny))
    return a.value, nx.value, ny.value


def collide_scalar(f: np.ndarray, meq: np.ndarray, tau: float, dtQ: float) -> np.ndarray:
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    meq = np.ascontiguousarray(meq, dtype=np.float64)
    out = np.zeros(9)
    lib.orc_collide_scalar(_dp(f), _dp(meq), float(tau), float(dtQ), _dp(out))
    return out


def relaxation_times(params, phi: float):
    """[tau_phi (a_s = 1), tau_U, tau_T, tau_F] at the given phi (Eqs. 24, 32)."""
    lib = _load()
    o = to_orc_params(params)
    out = np.zeros(4)
    lib.orc_relaxation_times(C.byref(o), float(phi), _dp(out))
    return out


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_threads(n: int):
    _load().orc_set_threads(int(n))


def aniso_frame(gx: float, gy: float, eps: float, vartheta: float):
    """(a_s, N_x, N_y) of Eqs. 2-3 in the frame of a crystal turned by vartheta."""
    lib = _load()
    a, nx, ny = C.c_double(), C.c_double(), C.c_double()
    lib.orc_aniso_frame(gx, gy, eps, vartheta, C.byref(a), C.byref(nx), C.byref(ny))
    return a.value, nx.value, ny.value
