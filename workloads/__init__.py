"""Seeded synthetic workloads: parameter sets and initial macroscopic fields.

This module is shared by the FP64 oracle and the CUDA path. It holds none of
the lattice Boltzmann arithmetic: it only states the inputs of a run (grid,
boundary kinds, material constants, update factors) and generates the initial
macroscopic fields phi, U, T, u, rho on the host in FP64. Each side then builds
its own distributions from them (f = f_eq of the initial fields).

Parameter sets follow the paper's statement of the problem:
  * circular seed phi = tanh[(R0 - r)/(sqrt(2) W0)]          (Sec. 4.1)
  * lambda = a1 W0 / d0 with a1 = 0.8839                     (Sec. 4.1)
  * thermosolutal constants M_c, k_c, D_L, D_S = 1e-2 D_L    (Sec. 4.3)
  * directional-solidification lattice constants             (Sec. 4.4, Table 1)
and tau0 from the vanishing-kinetics relation tau0 = a2 lambda W0^2 / D with
a2 = 0.6267 (it reproduces the paper's tau0 = 125 of Sec. 4.1 at W0 = 2.5).

Random numbers come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used
as a counter-based generator: the k-th draw of stream s is mix(s + (k+1)*gamma),
u = (mix >> 11) * 2^-53.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Dict, List, Optional, Sequence

import numpy as np

A1 = 0.8839          # Sec. 4.1: lambda = a1 W0 / d0
A2 = 0.6267          # vanishing-kinetics constant: tau0 = a2 lambda W0^2 / D

# boundary kinds (same integer values as the C header's LBM_BC_*)
BC_PERIODIC = 0
BC_WALL = 1
BC_INLET_OUTFLOW = 2

GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


# ---------------------------------------------------------------------------
# SplitMix64, counter form
# ---------------------------------------------------------------------------
def splitmix64(seed: int, n: int) -> np.ndarray:
    """First n outputs of SplitMix64 started at `seed`, as uint64."""
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + k * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from SplitMix64 (53 high bits)."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# ---------------------------------------------------------------------------
# Parameter set
# ---------------------------------------------------------------------------
@dataclass
class Params:
    """Inputs of one simulation (lattice units, dx = 1).

    Field switches: has_U (solute), has_T (evolving temperature), frozen_T
    (prescribed theta(y, t) = theta_c + G (y - y0 - V t), no T populations),
    has_flow (D2Q9 flow).  With neither has_T nor frozen_T, theta = theta_c.
    The temperature variable T maps to the undercooling by
    theta = (T - T_shift) / T_scale (Eq. 5); with T_shift = 0, T_scale = 1 the
    T field is theta itself.
    """
    nx: int
    ny: int
    has_U: bool = False
    has_T: bool = False
    frozen_T: bool = False
    has_flow: bool = False
    bc_scalar_x: int = BC_WALL
    bc_scalar_y: int = BC_WALL
    bc_flow_x: int = BC_PERIODIC
    bc_flow_y: int = BC_PERIODIC
    accumulated: bool = False          # source-coupling ablation (Sec. 4.4)
    N_phi: int = 1
    N_U: int = 1
    N_T: int = 1
    N_F: int = 1
    dt_base: float = 1.0
    # phase field (Eqs. 1-4)
    W0: float = 1.0
    tau0: float = 1.0
    eps: float = 0.0
    lam: float = 0.0
    # solute (Eqs. 5-9)
    Mc: float = 0.0
    k: float = 1.0
    DL: float = 0.0
    DS: float = 0.0
    # temperature (Eqs. 10-12)
    kappaS: float = 0.0
    kappaL: float = 0.0
    rhoCpS: float = 1.0
    rhoCpL: float = 1.0
    rhoL_Lh: float = 1.0
    T_shift: float = 0.0
    T_scale: float = 1.0
    # flow (Eqs. 13, 27-33)
    nu: float = 0.1
    u_in: float = 0.0
    Fbx: float = 0.0
    Fby: float = 0.0
    s_e: float = 1.2
    s_eps: float = 1.4
    s_q: float = 1.2
    # prescribed undercooling
    theta_c: float = 0.0
    frozen_G: float = 0.0
    frozen_y0: float = 0.0
    frozen_V: float = 0.0
    # diagnostics: node the tip crossings are measured from
    tip_cx: int = 0
    tip_cy: int = 0
    # bottom wall held at T = T_ymin (Sec. 4.4) instead of zero flux for T
    T_ymin_dirichlet: bool = False
    T_ymin: float = 0.0
    # velocities of the phi, U, T lattices: 9 (the paper's D2Q9) or 5 (D2Q5)
    q_scalar: int = 9

    def as_dict(self) -> Dict:
        return dict(self.__dict__)


@dataclass
class Workload:
    name: str
    params: Params
    fields: Dict[str, np.ndarray]          # phi, U, T, ux, uy, rho; (ny, nx) float64
    n_base_steps: int
    extra: Dict = field(default_factory=dict)


# ---------------------------------------------------------------------------
# Initial-field generators
# ---------------------------------------------------------------------------
def _grid(nx: int, ny: int):
    y, x = np.mgrid[0:ny, 0:nx]
    return x.astype(np.float64), y.astype(np.float64)


def circle_seed(nx: int, ny: int, cx: float, cy: float, R: float, W0: float) -> np.ndarray:
    """phi = tanh[(R - r)/(sqrt 2 W0)] around (cx, cy) (Sec. 4.1)."""
    x, y = _grid(nx, ny)
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    return np.tanh((R - r) / (math.sqrt(2.0) * W0))


def planar_front(nx: int, ny: int, y0: float, W0: float, noise_amp: float = 0.0,
                 seed: int = 0) -> np.ndarray:
    """Solid below y0: phi = tanh[(y0 - y)/(sqrt 2 W0)], plus uniform noise
    amp*(2u-1) on nodes with |phi| < 0.99, clipped to [-1, 1]. Draw k is node
    k in row-major (y, x) order."""
    x, y = _grid(nx, ny)
    phi = np.tanh((y0 - y) / (math.sqrt(2.0) * W0))
    if noise_amp > 0.0:
        u = uniform01(seed, nx * ny).reshape(ny, nx)
        band = np.abs(phi) < 0.99
        phi = np.where(band, np.clip(phi + noise_amp * (2.0 * u - 1.0), -1.0, 1.0), phi)
    return phi


def sinusoid_layer(nx: int, ny: int, W0: float, h: float = 10.0, amp: float = 1.0,
                   waves: float = 5.0) -> np.ndarray:
    """phi = tanh[(h + amp sin(2 pi waves x / L) - y)/(sqrt 2 W0)] (Eq. 41)."""
    x, y = _grid(nx, ny)
    return np.tanh((h + amp * np.sin(2.0 * math.pi * waves * x / nx) - y) / (math.sqrt(2.0) * W0))


def base_fields(p: Params, phi: np.ndarray, U0: float = 0.0, T0: float = 0.0) -> Dict[str, np.ndarray]:
    """Uniform U, T; flow at rest or u = u_in * f_L with f_L = (1 - phi)/2; rho = 1."""
    ny, nx = phi.shape
    f = {
        "phi": np.ascontiguousarray(phi, dtype=np.float64),
        "U": np.full((ny, nx), float(U0)),
        "T": np.full((ny, nx), float(T0)),
        "ux": np.zeros((ny, nx)),
        "uy": np.zeros((ny, nx)),
        "rho": np.ones((ny, nx)),
    }
    if p.has_flow and p.u_in != 0.0:
        f["ux"] = p.u_in * (1.0 - f["phi"]) / 2.0
    return f


# Lower bound of the solute relaxation time in the solid for the labelled
# "stable solid" variants of the listed workloads: the paper keeps tau_U in
# 0.524 - 0.860 through its choice of update factors (Sec. 4.3, and
# tau_U,L = 0.578 in Sec. 4.4); the listed instances with D_S = 1e-2 D_L put
# the solid side at 0.5005 - 0.508, where the flux moments barely relax.
TAU_U_SOLID_MIN = 0.52


def stable_solid(p: Params, tau_min: float = TAU_U_SOLID_MIN) -> Params:
    """Raise D_S, if needed, so that the solid-side solute relaxation time
    tau_U,S = 3 N_U dt_base D_S / k + 1/2 (Eqs. 7, 24 at phi = 1) is at least
    tau_min; every other parameter unchanged.  Returns p."""
    need = (tau_min - 0.5) * p.k / (3.0 * p.N_U * p.dt_base)
    if p.DS < need:
        p.DS = need
    return p


def stable_variant(p: Params, tau_min: float = TAU_U_SOLID_MIN) -> Params:
    """The labelled variant of a listed workload whose relaxation times all
    lie at or above tau_min, in the way the paper keeps them in range -- by
    the update factors (Sec. 3.3; Secs. 4.3-4.4 choose N_U so that tau_U stays
    in 0.524 - 0.860): N_phi raised to the smallest factor with
    tau_phi = 3 N_phi dt_base W0^2 / tau0 + 1/2 >= tau_min (Eq. 24 at
    a_s = 1), N_U to the smallest with tau_U,L >= tau_min, and then D_S by
    stable_solid.  A workload already in range is returned unchanged.
    Returns p."""
    w = p.W0 * p.W0 / p.tau0
    while 3.0 * p.N_phi * p.dt_base * w + 0.5 < tau_min:
        p.N_phi += 1
    if p.has_U:
        while tau_U(p, -1.0) < tau_min:
            p.N_U += 1
        stable_solid(p, tau_min)
    return p


def tau_U(p: Params, phi: float) -> float:
    """Solute relaxation time of Eq. 24 with D_eff of Eq. 7."""
    D = ((1 + phi) * p.DS + (1 - phi) * p.DL) / ((1 + p.k) - (1 - p.k) * phi)
    return 3.0 * p.N_U * p.dt_base * D + 0.5


def karma_tau0(lam: float, W0: float, D: float) -> float:
    return A2 * lam * W0 * W0 / D


# ---------------------------------------------------------------------------
# The five workloads (lattice units), with a size override for tests
# ---------------------------------------------------------------------------
def thermal_free_dendrite(n: int = 128, N_T: int = 1, R: float = 5.0,
                          n_base_steps: int = 2000) -> Workload:
    """Pure thermal free dendrite, periodic n x n, phi + T (no U, no flow).

    W0 = 1, eps = 0.05, d0 = 0.1385 W0, lambda = a1 W0/d0, alpha = 0.2,
    tau0 = a2 lambda W0^2/alpha (Pe = 0.25 as in Sec. 4.1), L_h/C_p = 1,
    theta0 = -0.55, seed radius R at node (n/2, n/2)."""
    W0 = 1.0
    lam = A1 * W0 / (0.1385 * W0)
    alpha = 0.2
    tau0 = 20.0
    p = Params(nx=n, ny=n, has_T=True, bc_scalar_x=BC_PERIODIC, bc_scalar_y=BC_PERIODIC,
               N_T=N_T, W0=W0, tau0=tau0, eps=0.05, lam=lam,
               kappaS=alpha, kappaL=alpha, rhoCpS=1.0, rhoCpL=1.0, rhoL_Lh=1.0,
               tip_cx=n // 2, tip_cy=n // 2)
    phi = circle_seed(n, n, n // 2, n // 2, R, W0)
    return Workload("thermal_free_dendrite_%d_NT%d" % (n, N_T), p,
                    base_fields(p, phi, U0=0.0, T0=-0.55), n_base_steps)


def thermosolutal_convection(n: int = 512, R: float = 8.0, n_base_steps: int = 20000,
                             N=(1, 1, 2, 2), u_in: float = 0.01) -> Workload:
    """Thermosolutal free dendrite with forced convection, n x n.

    Flow: inlet u_in at x = 0, outflow at x = n-1, periodic in y; scalars
    zero-flux on all sides. W0 = 2, eps = 0.02, lambda = 1.5955 (d0 = 0.554 W0),
    M_c = 0.1, k = 0.15, U0 = 0, theta0 = -0.55, D_L = 0.04, D_S = 1e-2 D_L,
    tau0 = 100, Le = 10 (alpha = 0.4), nu = 0.05, update factors
    (phi, U, T, F) = N, seed radius R at the centre."""
    W0 = 2.0
    lam = A1 * W0 / (0.554 * W0)
    DL = 0.04
    alpha = 10.0 * DL
    p = Params(nx=n, ny=n, has_U=True, has_T=True, has_flow=True,
               bc_scalar_x=BC_WALL, bc_scalar_y=BC_WALL,
               bc_flow_x=BC_INLET_OUTFLOW, bc_flow_y=BC_PERIODIC,
               N_phi=N[0], N_U=N[1], N_T=N[2], N_F=N[3],
               W0=W0, tau0=100.0, eps=0.02, lam=lam,
               Mc=0.1, k=0.15, DL=DL, DS=1e-2 * DL,
               kappaS=alpha, kappaL=alpha, rhoCpS=1.0, rhoCpL=1.0, rhoL_Lh=1.0,
               nu=0.05, u_in=u_in, tip_cx=n // 2, tip_cy=n // 2)
    phi = circle_seed(n, n, n // 2, n // 2, R, W0)
    return Workload("thermosolutal_convection_%d" % n, p,
                    base_fields(p, phi, U0=0.0, T0=-0.55), n_base_steps)


def directional_saline(Le: int = 100, nx: int = 1024, ny: int = 2048, y0: float = 100.0, k: float = 0.15,
                       noise: float = 0.01, seed: int = 3, n_base_steps: int = 200000) -> Workload:
    """Directional solidification with a frozen linear temperature gradient.

    W0 = 2, tau0 = 150, eps = 0.03 (Sec. 4.4 and Table 1); k = 0.15,
    C_inf = 0.03, m_L = -57, Gamma = 0.268, L_h/C_pL = 133.6/1.676, so
    d0 = Gamma/(|m_L|(1-k)C_inf), lambda = a1 W0/d0,
    M_c = |m_L|(1-k)C_inf/(L_h/C_pL). D_L = 0.026/Le, D_S = 1e-2 D_L,
    N_U = Le, N_phi = 1. theta(y, t) = 2e-4 (y - y0 - 0.005 t); planar
    interface at y0 with seeded noise; U = 0 (C/C_inf = 1 in the liquid)."""
    W0 = 2.0
    Cinf, mL, Gamma, LhCp = 0.03, -57.0, 0.268, 133.6 / 1.676
    d0 = Gamma / (abs(mL) * (1.0 - k) * Cinf)
    lam = A1 * W0 / d0
    Mc = abs(mL) * (1.0 - k) * Cinf / LhCp
    DL = 0.026 / Le
    p = Params(nx=nx, ny=ny, has_U=True, frozen_T=True,
               bc_scalar_x=BC_WALL, bc_scalar_y=BC_WALL,
               N_U=int(Le), W0=W0, tau0=150.0, eps=0.03, lam=lam,
               Mc=Mc, k=k, DL=DL, DS=1e-2 * DL,
               frozen_G=2e-4, frozen_y0=y0, frozen_V=0.005,
               tip_cx=nx // 2, tip_cy=0)
    phi = planar_front(nx, ny, y0, W0, noise, seed)
    return Workload("directional_Le%d_%dx%d" % (Le, nx, ny), p,
                    base_fields(p, phi, U0=0.0), n_base_steps)


def directional_evolving_T(Le: int = 100, nx: int = 1000, ny: int = 1000, n_base_steps: int = 10_000_000) -> Workload:
    """Directional thermosolutal solidification of saline water with an
    evolving temperature field (Sec. 4.4, Table 1, Eqs. 41-42).

    Table 1 lattice values: L_h = 133.6, C_pL = 1.676, C_pS = 0.836,
    kappa_L = 0.0437, kappa_S = 0.178 (rho_S = rho_L = 1), k_c = 0.001,
    C_inf = 0.03, m_L = -57, Gamma = 0.268, eps = 0.03; W0 = 2, tau0 = 150.
    d0 = Gamma/(|m_L|(1-k)C_inf), lambda = a1 W0/d0, M_c per Eq. 5, and
    theta = (T - T_m - m_L C_inf)/(L_h/C_pL) with T_m = 0 (Eq. 5).  D_L =
    0.026/Le (Eq. 42 in lattice units), D_S = 1e-2 D_L, N_U = Le,
    N_phi = N_T = 1.  Initial layer phi of Eq. 41 (mean height 10, amplitude
    1, five wavelengths across), T = T_b = -20 everywhere and held at the
    bottom wall, U = 0, no flow; zero flux for phi and U on every wall and
    for T at the top; periodic in x (the Eq. 41 perturbation spans whole
    wavelengths)."""
    W0, k, Cinf, mL, Gamma = 2.0, 0.001, 0.03, -57.0, 0.268
    Lh, CpL, CpS = 133.6, 1.676, 0.836
    d0 = Gamma / (abs(mL) * (1.0 - k) * Cinf)
    lam = A1 * W0 / d0
    Mc = abs(mL) * (1.0 - k) * Cinf / (Lh / CpL)
    DL = 0.026 / Le
    Tb = -20.0
    p = Params(nx=nx, ny=ny, has_U=True, has_T=True,
               bc_scalar_x=BC_PERIODIC, bc_scalar_y=BC_WALL,
               N_U=int(Le), W0=W0, tau0=150.0, eps=0.03, lam=lam,
               Mc=Mc, k=k, DL=DL, DS=1e-2 * DL,
               kappaS=0.178, kappaL=0.0437, rhoCpS=CpS, rhoCpL=CpL, rhoL_Lh=Lh,
               T_shift=0.0 + mL * Cinf, T_scale=Lh / CpL,
               T_ymin_dirichlet=True, T_ymin=Tb,
               tip_cx=nx // 2, tip_cy=0)
    phi = sinusoid_layer(nx, ny, W0, h=10.0, amp=1.0, waves=5.0)
    return Workload("directional_evolving_T_Le%d_%dx%d" % (Le, nx, ny), p,
                    base_fields(p, phi, U0=0.0, T0=Tb), n_base_steps)


def ensemble_members(count: int = 64, seed: int = 4, sizes=(128, 256, 512, 1024),
                     n_base_steps: int = 2000) -> List[Workload]:
    """Batched ensemble of thermosolutal free dendrites (no flow, zero-flux).

    Per member, draws in order from one SplitMix64 stream: size index
    floor(4u), undercooling 0.3 + 0.3u, Le index floor(3u) over {1, 10, 100},
    update-factor pair floor(3u) over (N_T, N_U) in {(1,1), (1,2), (2,4)},
    seed radius 4 + floor(7u). W0 = 2, eps = 0.02, lambda = 1.5955, M_c = 0.1,
    k = 0.15, alpha = 0.2, D_L = 0.2/Le, D_S = 1e-2 D_L, tau0 = 4/D_L."""
    u = uniform01(seed, 5 * count).reshape(count, 5)
    pairs = [(1, 1), (1, 2), (2, 4)]
    Les = [1, 10, 100]
    out = []
    W0 = 2.0
    lam = A1 * W0 / (0.554 * W0)
    for m in range(count):
        n = sizes[min(int(4 * u[m, 0]), len(sizes) - 1)]
        delta = 0.3 + 0.3 * u[m, 1]
        Le = Les[min(int(3 * u[m, 2]), 2)]
        NT, NU = pairs[min(int(3 * u[m, 3]), 2)]
        R = 4 + int(7 * u[m, 4])
        DL = 0.2 / Le
        p = Params(nx=n, ny=n, has_U=True, has_T=True,
                   bc_scalar_x=BC_WALL, bc_scalar_y=BC_WALL,
                   N_U=NU, N_T=NT, W0=W0, tau0=4.0 / DL, eps=0.02, lam=lam,
                   Mc=0.1, k=0.15, DL=DL, DS=1e-2 * DL,
                   kappaS=0.2, kappaL=0.2, rhoCpS=1.0, rhoCpL=1.0, rhoL_Lh=1.0,
                   tip_cx=n // 2, tip_cy=n // 2)
        phi = circle_seed(n, n, n // 2, n // 2, R, W0)
        out.append(Workload("ensemble_%02d_n%d" % (m, n), p,
                            base_fields(p, phi, U0=0.0, T0=-delta), n_base_steps,
                            extra={"Le": Le, "delta": delta, "R": R}))
    return out


def poisson_disc(n_seeds: int, lo: float, hi: float, min_dist: float, seed: int,
                 max_attempts: int = 1_000_000) -> np.ndarray:
    """Dart throwing: accept a uniform point in [lo, hi)^2 if it is at least
    min_dist from every accepted point; stops at n_seeds or max_attempts.
    Draws 2 numbers per attempt from one SplitMix64 stream."""
    pts: List = []
    batch = 4096
    drawn = 0
    while len(pts) < n_seeds and drawn < max_attempts:
        u = uniform01(seed, 2 * (drawn + batch))[2 * drawn:].reshape(-1, 2)
        for a, b in u:
            drawn += 1
            x = lo + (hi - lo) * a
            y = lo + (hi - lo) * b
            if all((x - q[0]) ** 2 + (y - q[1]) ** 2 >= min_dist * min_dist for q in pts):
                pts.append((x, y))
                if len(pts) == n_seeds:
                    break
            if drawn >= max_attempts:
                break
    return np.array(pts, dtype=np.float64).reshape(-1, 2)


def multi_dendrite_params(n: int = 8192, n_seeds: int = 32, min_dist: float = 800.0, seed: int = 5):
    """Parameters and seed centres of multi_dendrite without the host fields
    (for device-side seeding of large lattices)."""
    W0 = 2.0
    lam = A1 * W0 / (0.554 * W0)
    DL = 0.005
    p = Params(nx=n, ny=n, has_U=True, has_T=True, has_flow=True,
               bc_scalar_x=BC_WALL, bc_scalar_y=BC_WALL,
               bc_flow_x=BC_INLET_OUTFLOW, bc_flow_y=BC_PERIODIC,
               N_T=4, N_F=2, W0=W0, tau0=800.0, eps=0.02, lam=lam,
               Mc=0.1, k=0.3, DL=DL, DS=1e-2 * DL,
               kappaS=0.5, kappaL=0.5, rhoCpS=1.0, rhoCpL=1.0, rhoL_Lh=1.0,
               nu=0.05, u_in=0.005, tip_cx=n // 2, tip_cy=n // 2)
    pts = poisson_disc(n_seeds, 64.0, n - 64.0, min_dist * n / 8192.0, seed)
    return p, pts


def multi_dendrite(n: int = 8192, n_seeds: int = 32, min_dist: float = 800.0, seed: int = 5,
                   n_base_steps: int = 50000) -> Workload:
    """Large multi-dendrite thermosolutal growth with convection.

    W0 = 2, eps = 0.02, lambda = 1.5955, M_c = 0.1, k = 0.3, U0 = 0,
    theta0 = -0.55, D_L = 0.005, D_S = 5e-5, alpha = 0.5 (Le = 100),
    tau0 = 800, nu = 0.05, u_in = 0.005, update factors (1, 1, 4, 2),
    seeds of radius 8 placed by dart throwing in [64, n - 64)^2.  Crystal
    orientations theta_g = (pi/2) u are returned in extra['angles'] (the
    per-grain frame is an extension beyond the paper's axis-aligned Eq. 2)."""
    p, pts = multi_dendrite_params(n, n_seeds, min_dist, seed)
    W0 = p.W0
    phi = np.full((n, n), -1.0)
    for (cx, cy) in pts:
        phi = np.maximum(phi, circle_seed(n, n, cx, cy, 8.0, W0))
    angles = multi_dendrite_angles(len(pts), seed)
    return Workload("multi_dendrite_%d" % n, p, base_fields(p, phi, U0=0.0, T0=-0.55),
                    n_base_steps, extra={"seeds": pts, "angles": angles})


def multi_dendrite_fields(p: Params, pts, R: float = 8.0, U0: float = 0.0, T0: float = -0.55) -> Dict[str, np.ndarray]:
    """Initial fields of the whole multi-dendrite lattice (circles of radius R
    at the centres `pts`, Sec. 4.1 profile), built seed by seed on windows:
    beyond r = R + 20 sqrt(2) W0 + 2 the profile tanh[(R - r)/(sqrt 2 W0)]
    rounds to -1 exactly, so the result equals the full-lattice evaluation of
    multi_dendrite() without its cost on large lattices."""
    nx, ny = p.nx, p.ny
    sw = math.sqrt(2.0) * p.W0
    phi = np.full((ny, nx), -1.0)
    reach = abs(R) + 20.0 * sw + 2.0
    for (cx, cy) in np.asarray(pts, dtype=np.float64).reshape(-1, 2):
        xa, xb = int(max(0, math.floor(cx - reach))), int(min(nx, math.ceil(cx + reach) + 1))
        ya, yb = int(max(0, math.floor(cy - reach))), int(min(ny, math.ceil(cy + reach) + 1))
        y, x = np.mgrid[ya:yb, xa:xb]
        r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
        np.maximum(phi[ya:yb, xa:xb], np.tanh((R - r) / sw), out=phi[ya:yb, xa:xb])
    return base_fields(p, phi, U0=U0, T0=T0)


def multi_dendrite_angles(n_seeds: int, seed: int = 5) -> np.ndarray:
    """Crystal angles of the multi-dendrite grains, uniform in [0, pi/2)
    (the draws multi_dendrite returns in extra['angles'])."""
    return 0.5 * math.pi * uniform01(seed + 1, n_seeds)


def grain_orientation(pts, angles, x0: int, y0: int, w: int, h: int, rows: int = 64) -> np.ndarray:
    """Per-node crystal angle of the window [x0, x0 + w) x [y0, y0 + h): the
    angle of the nearest seed centre (Voronoi grains at initialisation; the
    first seed wins a tie).  Evaluated `rows` rows at a time."""
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 2)
    angles = np.asarray(angles, dtype=np.float64)
    out = np.empty((h, w), dtype=np.float64)
    x = np.arange(x0, x0 + w, dtype=np.float64)
    for r0 in range(0, h, rows):
        y = np.arange(y0 + r0, y0 + min(h, r0 + rows), dtype=np.float64)
        d2 = (x[None, :, None] - pts[None, None, :, 0]) ** 2 + (y[:, None, None] - pts[None, None, :, 1]) ** 2
        out[r0:r0 + len(y)] = angles[np.argmin(d2, axis=2)]
    return out


def circle_seeds_window(p: Params, pts, R: float, x0: int, y0: int, w: int, h: int,
                        U0: float = 0.0, T0: float = 0.0) -> Dict[str, np.ndarray]:
    """Initial fields of the window [x0, x0 + w) x [y0, y0 + h) of a lattice
    seeded with circles of radius R at the global centres `pts`:
    phi = max(-1, max_s tanh[(R - r_s)/(sqrt 2 W0)]) (Sec. 4.1), U = U0,
    T = T0, u = u_in (1 - phi)/2 with the flow on, rho = 1.  It is the same
    field a full-lattice generation gives, read on the window, without
    building the full lattice."""
    y, x = np.mgrid[y0:y0 + h, x0:x0 + w]
    x = x.astype(np.float64)
    y = y.astype(np.float64)
    phi = np.full((h, w), -1.0)
    for (cx, cy) in pts:
        r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
        phi = np.maximum(phi, np.tanh((R - r) / (math.sqrt(2.0) * p.W0)))
    return base_fields(p, phi, U0=U0, T0=T0)
