"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every test here runs on the CPU and checks the oracle (oracle/lbm_oracle.c)
against something other than itself: printed values of the paper, closed-form
solutions, exact discrete invariants, symmetries and the structure of the
moment basis.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Moment basis (Eqs. 15-16)
# ---------------------------------------------------------------------------
def test_moment_matrix_is_the_polynomial_basis():
    """Rows of M are the D2Q9 moments 1, e, eps, jx, qx, jy, qy, pxx, pxy
    evaluated on the velocity set (Eq. 15), and M M^T is diagonal with
    (9, 36, 36, 6, 12, 6, 12, 4, 4); M^-1 M = I."""
    M, Mi, ex, ey, w = oracle.matrices()
    e2 = ex ** 2 + ey ** 2
    rows = np.array([
        np.ones(9), -4 + 3 * e2, 4 - 10.5 * e2 + 4.5 * e2 ** 2, ex, (3 * e2 - 5) * ex,
        ey, (3 * e2 - 5) * ey, ex ** 2 - ey ** 2, ex * ey], dtype=float)
    assert np.array_equal(M, rows)
    assert np.allclose(M @ M.T, np.diag([9, 36, 36, 6, 12, 6, 12, 4, 4]), atol=0)
    assert np.abs(Mi @ M - np.eye(9)).max() < 1e-15
    # weights: isotropy sums of the lattice
    assert abs(w.sum() - 1) < 1e-15
    assert abs((w * ex).sum()) < 1e-16 and abs((w * ex * ex).sum() - 1 / 3) < 1e-15
    assert abs((w * ex * ex * ey * ey).sum() - 1 / 9) < 1e-15


@pytest.mark.parametrize("kind", ["scalar", "phase", "flow"])
@pytest.mark.parametrize("c", [1.0, 0.5, 1.0 / 15.0])
def test_equilibrium_moments(kind, c):
    """M f_eq equals the printed equilibrium moments: Eq. 19 -> Eq. 20,
    Eq. 21 -> Eq. 22, Eq. 28 -> Eq. 29."""
    M, *_ = oracle.matrices()
    rng = np.random.default_rng(1)
    for _ in range(20):
        a, ux, uy = rng.uniform(-1, 1), rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1)
        if kind == "flow":
            a = 1 + 0.1 * a
        f, m = oracle.equilibrium(kind, a, ux, uy, c)
        assert np.abs(M @ f - m).max() < 1e-14


def test_scalar_collision_closed_form():
    """With S = diag(1,1,1,s,1,s,1,1,1) (Eq. 23), the literal product of Eq. 14
    equals f_eq + (1 - s)(e_i . j_neq)/6 + dt w_i Q, where j_neq is the first
    moment of f - f_eq (column 3 of M^-1 is e_x/6, column 5 is e_y/6)."""
    M, Mi, ex, ey, w = oracle.matrices()
    rng = np.random.default_rng(2)
    for _ in range(50):
        f = rng.uniform(0, 0.3, 9)
        chi = f.sum()
        ux, uy, c, tau, dtQ = rng.uniform(-.05, .05), rng.uniform(-.05, .05), rng.choice([1, .5, .25]), \
            rng.uniform(0.51, 3), rng.uniform(-1e-3, 1e-3)
        feq, meq = oracle.equilibrium("scalar", chi, ux, uy, c)
        out = oracle.collide_scalar(f, meq, tau, dtQ)
        jn = np.array([(ex * (f - feq)).sum(), (ey * (f - feq)).sum()])
        ref = feq + (1 - 1 / tau) * (ex * jn[0] + ey * jn[1]) / 6 + dtQ * w
        assert np.abs(out - ref).max() < 1e-15


# ---------------------------------------------------------------------------
# Anisotropy (Eqs. 2-3)
# ---------------------------------------------------------------------------
def test_anisotropy_function_and_correction_vector():
    """a_s(n) = 1 + eps cos 4 alpha (trigonometric form of Eq. 2), and
    N = |grad phi|^2 a_s d a_s / d(grad phi) (Eq. 3) checked against a central
    difference of a_s with respect to the gradient components."""
    eps = 0.05
    for alpha in np.linspace(0.01, 2 * math.pi, 37):
        r = 0.3
        gx, gy = -r * math.cos(alpha), -r * math.sin(alpha)   # n = -g/|g| = (cos, sin)
        a, Nx, Ny = oracle.aniso(gx, gy, eps)
        assert abs(a - (1 + eps * math.cos(4 * alpha))) < 1e-14
        h = 1e-6
        dax = (oracle.aniso(gx + h, gy, eps)[0] - oracle.aniso(gx - h, gy, eps)[0]) / (2 * h)
        day = (oracle.aniso(gx, gy + h, eps)[0] - oracle.aniso(gx, gy - h, eps)[0]) / (2 * h)
        assert abs(Nx - r * r * a * dax) < 1e-8
        assert abs(Ny - r * r * a * day) < 1e-8
    assert oracle.aniso(0.0, 0.0, eps) == (1.0, 0.0, 0.0)


# ---------------------------------------------------------------------------
# Printed parameter values (tests/golden/paper_parameters.txt)
# ---------------------------------------------------------------------------
def _golden():
    rows = {}
    for line in open(os.path.join(GOLDEN, "paper_parameters.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, _inp, val, tol, _cite = [s.strip() for s in line.split("|")]
        rows[name] = (float(val), float(tol))
    return rows


def test_printed_relaxation_times_and_constants():
    g = _golden()

    def check(name, value):
        ref, tol = g[name]
        assert abs(value - ref) <= tol * abs(ref), (name, value, ref)

    p = W.Params(nx=4, ny=4, has_flow=True, N_F=1, dt_base=1 / 15, nu=4.62, W0=1, tau0=1)
    check("tau_F_forced_thermal", oracle.relaxation_times(p, -1.0)[3])
    p = W.Params(nx=4, ny=4, has_U=True, N_U=30, DL=0.004, DS=4e-5, k=0.15, W0=1, tau0=1)
    check("tau_U_solid_Le50", oracle.relaxation_times(p, 1.0)[1])
    check("tau_U_liquid_Le50", oracle.relaxation_times(p, -1.0)[1])
    p = W.Params(nx=4, ny=4, has_T=True, N_T=1, kappaS=0.2, kappaL=0.2, W0=1, tau0=1)
    check("tau_T_Le50", oracle.relaxation_times(p, -1.0)[2])
    wl = W.directional_saline(Le=100, nx=8, ny=8)
    p = wl.params
    check("tau_UL_directional", oracle.relaxation_times(p, -1.0)[1])
    check("lambda_thermosolutal", W.thermosolutal_convection(n=8).params.lam)
    wt = W.directional_saline(Le=100, nx=8, ny=8, k=0.001)
    d0 = W.A1 * wt.params.W0 / wt.params.lam
    check("d0_table1", d0)
    check("lambda_table1", wt.params.lam)
    check("Mc_table1", wt.params.Mc)
    # Table 1 diffusivities from conductivities and capacities with rho = 1
    p = W.Params(nx=4, ny=4, has_T=True, N_T=1, kappaS=0.178, kappaL=0.0437, rhoCpS=0.836,
                 rhoCpL=1.676, W0=1, tau0=1)
    check("alpha_L_table1", (oracle.relaxation_times(p, -1.0)[2] - 0.5) / 3)
    check("alpha_S_table1", (oracle.relaxation_times(p, 1.0)[2] - 0.5) / 3)
    lam = W.A1 / 0.1385
    check("tau0_thermal", W.karma_tau0(lam, 2.5, 0.2))
    check("Dtilde_solutal", 0.25 * 50 / 2.5 ** 2)


# ---------------------------------------------------------------------------
# Transport: closed-form solutions
# ---------------------------------------------------------------------------
def _gaussian_run(field, N, steps=400, n=128, s0=5.0, D=1.0 / 6.0):
    if field == "U":
        p = W.Params(nx=n, ny=n, has_U=True, bc_scalar_x=0, bc_scalar_y=0, N_U=N, DL=D, DS=D,
                     k=0.15, W0=1, tau0=1)
    else:
        p = W.Params(nx=n, ny=n, has_T=True, bc_scalar_x=0, bc_scalar_y=0, N_T=N, kappaS=D,
                     kappaL=D, W0=1, tau0=1)
    f = W.base_fields(p, -np.ones((n, n)))
    x, y = np.meshgrid(np.arange(n) - n / 2, np.arange(n) - n / 2)
    r2 = x * x + y * y
    f[field] = 0.1 * np.exp(-r2 / (2 * s0 * s0))
    o = oracle.Oracle(p, f)
    o.advance(steps)
    s2 = s0 * s0 + 2 * D * steps
    ana = 0.1 * s0 * s0 / s2 * np.exp(-r2 / (2 * s2))
    return o, p, ana, x, y, s2


@pytest.mark.parametrize("field", ["U", "T"])
@pytest.mark.parametrize("N,tol", [(1, 1e-4), (2, 5e-3), (4, 1.5e-2)])
def test_gaussian_pulse_decay(field, N, tol):
    """Pure diffusion of a Gaussian pulse (u = 0, phi = -1 everywhere, so the
    phase field and the phase-change sources vanish): A s0^2/(s0^2 + 2Dt)
    exp(-r^2/(2(s0^2 + 2Dt))) with D = (tau - 1/2)/(3 dt_chi) (Eq. 24), for
    update factors 1, 2, 4 at the same physical D (Eq. 34)."""
    o, p, ana, *_ = _gaussian_run(field, N)
    got = o.get(field)
    assert np.linalg.norm(got - ana) / np.linalg.norm(ana) < tol
    assert abs(got.sum() - ana.sum()) / ana.sum() < 1e-3


def test_nonequilibrium_gradient_matches_analytic():
    """Eq. 40 applied to the oracle's populations recovers the gradient of the
    diffusing Gaussian (second-order accurate)."""
    o, p, ana, x, y, s2 = _gaussian_run("U", 1)
    M, Mi, ex, ey, w = oracle.matrices()
    f = o.pops("U")
    U = f.sum(axis=0)
    feq = w[:, None, None] * U[None]
    tau = 3 * 1.0 * p.DL + 0.5
    gx = -3.0 / tau * np.tensordot(ex, f - feq, axes=1)
    gy = -3.0 / tau * np.tensordot(ey, f - feq, axes=1)
    agx, agy = -x / s2 * ana, -y / s2 * ana
    err = math.sqrt(np.sum((gx - agx) ** 2 + (gy - agy) ** 2) / np.sum(agx ** 2 + agy ** 2))
    assert err < 5e-3


@pytest.mark.parametrize("NF,tol", [(1, 4e-3), (2, 1.5e-2)])
def test_taylor_green_decay(NF, tol):
    """Taylor-Green vortex in a periodic liquid (phi = -1, so Eq. 33 reduces to
    plain streaming) decays as exp(-2 nu k^2 t) (Eqs. 27-32)."""
    n, u0, nu, steps = 64, 0.02, 0.02, 400
    kk = 2 * math.pi / n
    p = W.Params(nx=n, ny=n, has_flow=True, bc_flow_x=0, bc_flow_y=0, bc_scalar_x=0, bc_scalar_y=0,
                 N_F=NF, nu=nu, W0=1, tau0=1)
    x, y = np.meshgrid(np.arange(n) + 0.0, np.arange(n) + 0.0)
    f = W.base_fields(p, -np.ones((n, n)))
    f["ux"] = -u0 * np.cos(kk * x) * np.sin(kk * y)
    f["uy"] = u0 * np.sin(kk * x) * np.cos(kk * y)
    f["rho"] = 1 + 3 * (-u0 * u0 / 4 * (np.cos(2 * kk * x) + np.cos(2 * kk * y)))
    o = oracle.Oracle(p, f)
    o.advance(steps)
    dec = math.exp(-2 * nu * kk * kk * steps)
    for k in ("ux", "uy"):
        ana = f[k] * dec
        assert np.linalg.norm(o.get(k) - ana) / np.linalg.norm(ana) < tol


def test_uniform_stream_inlet_outflow_is_steady():
    """A uniform liquid stream u = u_in, rho = 1 is an exact fixed point of the
    flow update with the inlet / outflow columns and periodic sides."""
    p = W.Params(nx=32, ny=16, has_flow=True, bc_flow_x=W.BC_INLET_OUTFLOW, bc_flow_y=0,
                 N_F=2, nu=0.05, u_in=0.01, W0=1, tau0=1)
    f = W.base_fields(p, -np.ones((16, 32)))
    o = oracle.Oracle(p, f)
    o.advance(50)
    assert np.abs(o.get("ux") - 0.01).max() < 1e-15
    assert np.abs(o.get("uy")).max() < 1e-15
    assert np.abs(o.get("rho") - 1).max() < 1e-14


def test_partial_bounce_back_mass_and_solid_reversal():
    """Eq. 33 splits each link pair's outgoing populations between its two
    ends, so total mass is exactly conserved for any phi; with phi = +1 (f_L = 0)
    every population is reflected in place and u flips sign each update."""
    n = 24
    rng = np.random.default_rng(3)
    p = W.Params(nx=n, ny=n, has_flow=True, bc_flow_x=0, bc_flow_y=0, bc_scalar_x=0, bc_scalar_y=0,
                 nu=0.05, W0=1, tau0=1, eps=0.0, lam=0.0)
    phi = np.clip(rng.uniform(-1.2, 1.2, (n, n)), -1, 1)
    f = W.base_fields(p, phi)
    f["ux"] = rng.uniform(-0.02, 0.02, (n, n))
    f["uy"] = rng.uniform(-0.02, 0.02, (n, n))
    f["rho"] = 1 + rng.uniform(-0.01, 0.01, (n, n))
    o = oracle.Oracle(p, f)
    m0 = o.pops("F").sum()
    o.stage(3)
    assert abs(o.pops("F").sum() - m0) / m0 < 1e-14
    fs = dict(f)
    fs["phi"] = np.ones((n, n))
    o2 = oracle.Oracle(p, fs)
    o2.stage(3)
    assert np.abs(o2.get("ux") + f["ux"]).max() < 1e-15
    assert np.abs(o2.get("uy") + f["uy"]).max() < 1e-15


# ---------------------------------------------------------------------------
# Body force (Eqs. 13, 14, 27, 30): Newton's law, Guo's second moments,
# body-force Poiseuille flow.  Reading R-force: the forcing term of Eq. 14
# carries dt_F, so one flow update moves rho u by dt_F F_b.
# ---------------------------------------------------------------------------
E9 = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])


def _liquid_flow_params(nx, ny, NF, nu, Fbx, Fby, bc_y=W.BC_PERIODIC, **kw):
    return W.Params(nx=nx, ny=ny, has_flow=True, bc_flow_x=W.BC_PERIODIC, bc_flow_y=bc_y,
                    bc_scalar_x=W.BC_PERIODIC, bc_scalar_y=bc_y, N_F=NF, nu=nu, Fbx=Fbx, Fby=Fby,
                    W0=1, tau0=1, **kw)


@pytest.mark.parametrize("NF", [1, 2, 3])
def test_uniform_body_force_newton_and_guo_moments(NF):
    """A uniform liquid on a periodic lattice under a constant body force is
    homogeneous, so streaming is the identity and only the collision acts.
    (1) Newton: after K updates (time t = K dt_F) the Eq. 27 velocity is
    u0 + F (t + dt_F/2), exactly, and rho stays 1 (G_0 = 0).
    (2) Guo's forcing (Eq. 30 with (I - S/2), Eq. 14) makes every relaxed
    moment m_k with equilibrium E_k(u) and forcing G_k(u, F) settle at
    E_k(u) - (the part of G_k linear in F)/2 in lattice units, whatever its
    rate s_k: the raw moments then describe the raw momentum exactly.  Derived
    here for the D2Q9 basis polynomials: energy e = -2 + 3u^2 - 3u.F,
    epsilon = 1 - 3u^2 + 3u.F, q_x = -u_x + F_x/2, p_xx - p_yy =
    u_x^2 - u_y^2 - (F_x u_x - F_y u_y), p_xy = u_x u_y - (F_x u_y + F_y u_x)/2,
    with u' = u dt_F and F' = F dt_F^2 (the per-update impulse over c_F).  A
    wrong sign, factor or dt_F scaling in any G_k fails one of them."""
    n, nu = 6, 0.04
    dt = float(NF)
    Fx, Fy = 3.0e-6, -2.0e-6
    p = _liquid_flow_params(n, n, NF, nu, Fx, Fy)
    f = W.base_fields(p, -np.ones((n, n)))
    u0x, u0y = 4.0e-3, -1.5e-3
    f["ux"] = np.full((n, n), u0x)
    f["uy"] = np.full((n, n), u0y)
    o = oracle.Oracle(p, f)
    K = 80                                     # updates; transients decay as |1 - s_k|^K
    o.advance(K * NF)
    t = K * dt
    assert np.abs(o.get("ux") - (u0x + Fx * (t + 0.5 * dt))).max() < 1e-13
    assert np.abs(o.get("uy") - (u0y + Fy * (t + 0.5 * dt))).max() < 1e-13
    assert np.abs(o.get("rho") - 1.0).max() < 1e-14
    fp = o.pops("F")[:, 0, 0]
    o.close()
    ux = (u0x + Fx * (t + 0.5 * dt)) * dt      # lattice units
    uy = (u0y + Fy * (t + 0.5 * dt)) * dt
    fx, fy = Fx * dt * dt, Fy * dt * dt
    ex, ey = E9[:, 0], E9[:, 1]
    e2 = ex * ex + ey * ey
    u2, uF = ux * ux + uy * uy, ux * fx + uy * fy
    got = {
        "e": np.dot(-4 + 3 * e2, fp),
        "eps": np.dot(4 - 10.5 * e2 + 4.5 * e2 * e2, fp),
        "qx": np.dot((-5 + 3 * e2) * ex, fp),
        "qy": np.dot((-5 + 3 * e2) * ey, fp),
        "pxx": np.dot(ex * ex - ey * ey, fp),
        "pxy": np.dot(ex * ey, fp),
    }
    want = {
        "e": -2 + 3 * u2 - 3 * uF,
        "eps": 1 - 3 * u2 + 3 * uF,
        "qx": -ux + fx / 2,
        "qy": -uy + fy / 2,
        "pxx": ux * ux - uy * uy - (fx * ux - fy * uy),
        "pxy": ux * uy - (fx * uy + fy * ux) / 2,
    }
    for k in got:
        assert abs(got[k] - want[k]) < 1e-13, (k, got[k], want[k])   # |u.F| terms ~1e-7


@pytest.mark.parametrize("NF", [1, 2])
def test_body_force_poiseuille(NF):
    """Body-force Poiseuille flow between half-way bounce-back walls (periodic
    in x, liquid phi = -1 so Eq. 33 is plain streaming).  Steady Eq. 13:
    nu u'' + F = 0, so (a) in the bulk the discrete second difference of u is
    -F/nu (the LBM reproduces the parabola exactly there) in base time units
    at every update factor -- the force acts per unit time, not per update;
    (b) u is symmetric about the channel centre, u_y = 0; (c) with the energy
    flux rate s_q set so that (1/s_nu - 1/2)(1/s_q - 1/2) = 3/16 the bounce-back
    wall sits exactly half a link outside the last node, and u equals the
    parabola F/(2 nu) (y + 1/2)(ny - 1/2 - y); (d) with the paper's s_q = 1.2
    the parabola holds up to a uniform wall slip below 1 % of u_max."""
    nx, ny, nu, F = 4, 12, 1.0 / 6.0, 1.0e-6
    dt = float(NF)
    tauF = 3 * dt * nu + 0.5
    y = np.arange(ny)
    ana = F / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    for sq, tol in ((1.0 / (0.5 + (3.0 / 16.0) / (tauF - 0.5)), 1e-8), (1.2, 1e-2)):
        p = _liquid_flow_params(nx, ny, NF, nu, F, 0.0, bc_y=W.BC_WALL, s_q=sq)
        o = oracle.Oracle(p, W.base_fields(p, -np.ones((ny, nx))))
        o.advance(5000)
        u = o.get("ux")
        uy = o.get("uy")
        o.close()
        assert np.abs(u - u[:, :1]).max() < 1e-18             # uniform along x
        u = u[:, 0]
        d2 = u[2:] - 2 * u[1:-1] + u[:-2]
        assert np.abs(d2 / (-F / nu) - 1).max() < 1e-8, (sq, d2)
        assert np.abs(u - u[::-1]).max() < 1e-9 * ana.max()
        assert np.abs(uy).max() < 1e-15
        assert np.abs(u - ana).max() < tol * ana.max(), (sq, np.abs(u - ana).max() / ana.max())


def test_inlet_outflow_columns_with_nonuniform_density():
    """Reading Q9 on a state whose density varies along x, so that the inlet
    column's new density is not its old one: after every flow update the
    inlet column x = 0 carries exactly the inlet velocity (u_x = u_in, u_y = 0)
    at the density of its downstream neighbour x = 1 (zero-gradient density,
    the populations being f_eq(rho(x=1), u_in)); the outflow column copies
    x = L-2 (equal rho, u).  Taking the density from any other column, or
    before streaming, breaks rho(0) == rho(1)."""
    nx, ny = 24, 10
    p = W.Params(nx=nx, ny=ny, has_flow=True, bc_flow_x=W.BC_INLET_OUTFLOW, bc_flow_y=W.BC_PERIODIC,
                 bc_scalar_x=W.BC_WALL, bc_scalar_y=W.BC_PERIODIC, N_F=1, nu=0.05, u_in=0.01,
                 W0=1, tau0=1)
    x, yy = np.meshgrid(np.arange(nx) + 0.0, np.arange(ny) + 0.0)
    f = W.base_fields(p, -np.ones((ny, nx)))
    f["rho"] = 1.0 + 0.02 * np.sin(2 * np.pi * x / nx) + 0.005 * np.cos(2 * np.pi * yy / ny)
    f["ux"] = 0.01 + 0.003 * np.cos(2 * np.pi * yy / ny)
    f["uy"] = 0.002 * np.sin(2 * np.pi * x / nx)
    o = oracle.Oracle(p, f)
    prev0 = f["rho"][:, 0]
    for _ in range(6):
        o.advance(1)
        rho, ux, uy = o.get("rho"), o.get("ux"), o.get("uy")
        assert np.abs(rho[:, 0] - rho[:, 1]).max() < 1e-15
        assert np.abs(rho[:, 0] - prev0).max() > 1e-5          # the inlet density did move
        assert np.abs(ux[:, 0] - 0.01).max() < 1e-16
        assert np.abs(uy[:, 0]).max() < 1e-17
        for a in (rho, ux, uy):
            assert np.array_equal(a[:, -1], a[:, -2])
        assert np.ptp(rho[:, 1]) > 1e-4                        # still non-uniform
        prev0 = rho[:, 0].copy()
    o.close()


# ---------------------------------------------------------------------------
# Phase field: closed forms
# ---------------------------------------------------------------------------
def _front_position(row):
    i = np.where((row[:-1] >= 0) & (row[1:] < 0))[0][-1]
    return i + row[i] / (row[i] - row[i + 1])


def test_stationary_planar_interface():
    """eps = 0, lambda = 0: phi = -tanh(x/(sqrt 2 W0)) solves
    W0^2 phi'' + phi - phi^3 = 0, so it must stay put (Eqs. 1, 4)."""
    W0, n = 2.0, 128
    p = W.Params(nx=n, ny=4, frozen_T=True, bc_scalar_x=1, bc_scalar_y=0, W0=W0, tau0=12.0)
    x = np.arange(n) + 0.0
    phi = np.tile(-np.tanh((x - 64.0) / (math.sqrt(2) * W0)), (4, 1))
    o = oracle.Oracle(p, W.base_fields(p, phi))
    o.advance(1000)
    assert np.abs(o.get("phi") - phi).max() < 1e-3


@pytest.mark.parametrize("eps", [0.0, 0.05])
def test_planar_front_velocity(eps):
    """Travelling-wave solution to first order in lambda theta (solvability):
    v tau0 a_s int phi'^2 = lambda |theta| int (1 - phi^2)^2 dphi gives
    v = (4 sqrt 2 / 5) |lambda theta| W0 / (a_s tau0); along an axis
    a_s = 1 + eps and N = 0.  Pins the phase source scaling (Q_phi/tau0 per
    unit time), tau_phi of Eq. 24 and the a_s^2 weighting of Eq. 26."""
    W0, tau0, lt, n = 2.0, 12.0, -0.02, 256
    p = W.Params(nx=n, ny=4, frozen_T=True, bc_scalar_x=1, bc_scalar_y=0, W0=W0, tau0=tau0,
                 eps=eps, lam=1.0, theta_c=lt)
    x = np.arange(n) + 0.0
    phi = np.tile(-np.tanh((x - 60) / (math.sqrt(2) * W0 * (1 + eps))), (4, 1))
    o = oracle.Oracle(p, W.base_fields(p, phi))
    o.advance(1000)
    a = _front_position(o.get("phi")[0])
    o.advance(3000)
    b = _front_position(o.get("phi")[0])
    v = (b - a) / 3000
    va = 4 * math.sqrt(2) / 5 * abs(lt) * W0 / (tau0 * (1 + eps))
    assert abs(v / va - 1) < 0.03


def _shrink_rates(eps, n=160, R=50.0, W0=2.0, tau0=12.0, t0=40, dt=200):
    p = W.Params(nx=n, ny=n, frozen_T=True, bc_scalar_x=0, bc_scalar_y=0, W0=W0, tau0=tau0, eps=eps)
    c = n // 2
    o = oracle.Oracle(p, W.base_fields(p, W.circle_seed(n, n, c, c, R, W0)))

    def radii():
        ph = o.get("phi")
        ra = _front_position(ph[c, c:])
        rd = _front_position(np.array([ph[c + k, c + k] for k in range(c - 1)])) * math.sqrt(2)
        return ra, rd

    o.advance(t0)
    a = radii()
    o.advance(dt)
    b = radii()
    return (b[0] - a[0]) / dt, (b[1] - a[1]) / dt


@pytest.mark.slow
def test_anisotropic_curvature_flow():
    """Curvature-driven shrinkage (lambda = 0) of a circle: the sharp-interface
    limit of Eq. 1 (W = W0 a_s, tau = tau0 a_s^2) gives
    v_n = -(W0^2/tau0)(a_s + a_s'')/a_s kappa; with a_s = 1 + eps cos 4 alpha the
    axis/diagonal factors are (1 - 15 eps)/(1 + eps) and (1 + 15 eps)/(1 - eps).
    The anisotropy of the rates comes only from the N term of Eq. 3 (without
    it the rate is isotropic), so this pins N's sign and size."""
    a0, d0 = _shrink_rates(0.0)
    a1, d1 = _shrink_rates(0.02)
    assert abs(d0 / a0 - 1) < 0.1
    eps = 0.02
    fa, fd = (1 - 15 * eps) / (1 + eps), (1 + 15 * eps) / (1 - eps)
    assert abs((a1 / a0) / fa - 1) < 0.12
    assert abs((d1 / d0) / fd - 1) < 0.12
    assert 1.5 < d1 / a1 < 2.3


# ---------------------------------------------------------------------------
# Exact invariants of the multirate coupling (Eqs. 36-39)
# ---------------------------------------------------------------------------
def _thermosolutal_small(n=48, bcx=W.BC_WALL, steps=60, flow=True, N=(1, 1, 2, 2)):
    wl = W.thermosolutal_convection(n=n, R=6.0, N=N)
    p = wl.params
    p.bc_scalar_x = bcx
    p.bc_scalar_y = bcx
    p.has_flow = flow
    p.eps = 0.05
    o = oracle.Oracle(p, wl.fields)
    o.advance(steps)
    return o, p


@pytest.mark.parametrize("bc", [W.BC_WALL, W.BC_PERIODIC])
def test_solute_balance_exact_over_phase_step(bc):
    """One phase update plus the immediate transfer leaves sum C/C_inf
    unchanged: with D(phi) = (1+k) - (1-k) phi, Eq. 38 makes
    2 dC/C_inf = -2 (1-k) div J, and the isotropic divergence sums to zero under
    periodic wrap or the mirrored wall ghosts."""
    o, p = _thermosolutal_small(bcx=bc)
    c0 = o.get("C").sum()
    o.stage(0)
    assert abs(o.get("dU")).max() > 1e-6          # the transfer did something
    assert abs(o.get("C").sum() - c0) / c0 < 1e-13


def test_enthalpy_exact_thermal_dendrite_multirate():
    """Equal capacities, L_h/C_p = 1, periodic: sum(T - phi/2) is conserved by
    each phase update + latent-heat transfer (Eq. 38) and by each temperature
    update (Q_T^tr = 0), whatever N_T is."""
    wl = W.thermal_free_dendrite(n=64, N_T=2, R=5.0)
    o = oracle.Oracle(wl.params, wl.fields)
    h0 = (o.get("T") - 0.5 * o.get("phi")).sum()
    o.advance(301)
    h1 = (o.get("T") - 0.5 * o.get("phi")).sum()
    assert abs(h1 - h0) / abs(h0) < 1e-13
    assert o.diagnostics()["tip"][0] > 6.0         # the seed grew


def test_injection_changes_only_the_zeroth_moment():
    """Eq. 39: adding w_i dU to f^U changes sum f by dU and leaves the first
    moment unchanged (sum w_i e_i = 0)."""
    o, p = _thermosolutal_small(steps=1, N=(1, 2, 2, 2))
    M, Mi, ex, ey, w = oracle.matrices()
    f0 = o.pops("U")
    o.stage(0)
    f1 = o.pops("U")
    dU = o.get("dU")
    assert np.abs(f1.sum(0) - f0.sum(0) - dU).max() < 1e-14
    assert np.abs(np.tensordot(ex, f1 - f0, axes=1)).max() < 1e-15
    assert np.abs(np.tensordot(ey, f1 - f0, axes=1)).max() < 1e-15


def test_static_interface_solute_conservation():
    """With a (nearly) static interface the solute equation conserves int C in
    the continuum: (1-k) D(phi) [div(D_eff grad U) + Q_U^tr]
    = (1-k) div(D(phi) D_eff grad U), D(phi) = (1+k) - (1-k) phi.  Without the
    Q_U^tr term of Eq. 8 sum C would change by about
    -sum (1-k)/2 D(phi) Q_U^tr dt (estimated below with central differences);
    the oracle's drift must be a small fraction of that."""
    n, ny, W0, k = 64, 8, 2.0, 0.15
    p = W.Params(nx=n, ny=ny, has_U=True, frozen_T=True, bc_scalar_x=1, bc_scalar_y=0,
                 W0=W0, tau0=12.0, lam=0.0, Mc=0.0, k=k, DL=0.1, DS=0.001)
    x = np.arange(n) + 0.0
    phi = np.tile(-np.tanh((x - 32.0) / (math.sqrt(2) * W0)), (ny, 1))
    f = W.base_fields(p, phi)
    f["U"] = np.tile(0.3 * np.exp(-((x - 36.0) ** 2) / 18.0), (ny, 1))
    o = oracle.Oracle(p, f)
    c0 = o.get("C").sum()
    qtr = 0.0
    for _ in range(400):
        ph, U = o.get("phi")[0], o.get("U")[0]
        Deff = ((1 + ph) * p.DS + (1 - ph) * p.DL) / ((1 + k) - (1 - k) * ph)
        qtr += ny * np.sum(0.5 * (1 - k) ** 2 * Deff * np.gradient(U) * np.gradient(ph))
        o.advance(1)
    drift = o.get("C").sum() - c0
    assert abs(qtr) > 0.5
    assert abs(drift) < 0.1 * abs(qtr)


# ---------------------------------------------------------------------------
# Symmetry and schedule
# ---------------------------------------------------------------------------
@pytest.mark.slow
def test_fourfold_symmetry_thermal_dendrite():
    """Periodic 128^2, seed centred on node (64, 64): the lattice, the
    isotropic stencils and Eq. 2 are invariant under the mirrors about that
    node's axes and diagonal (together they generate the 90-degree rotation),
    so phi must be too (FP64, 1000 steps)."""
    wl = W.thermal_free_dendrite(n=128)
    o = oracle.Oracle(wl.params, wl.fields)
    o.advance(1000)
    phi = o.get("phi")
    c = 64
    idx = (np.arange(128) - c) % 128

    def about_c(a):          # re-index so that node c sits at the origin
        return a[np.ix_(idx, idx)]

    s = about_c(phi)
    assert np.abs(s[:, (-np.arange(128)) % 128] - s).max() < 1e-10
    assert np.abs(s[(-np.arange(128)) % 128, :] - s).max() < 1e-10
    assert np.abs(s.T - s).max() < 1e-10
    assert o.diagnostics()["tip"].std() < 1e-9


def test_accumulated_equals_instantaneous_at_unit_factors():
    """When every field updates every base step, deferring the transfer to
    the next coarse update changes nothing: the same increment is injected
    before the same collision (the paper reports the two as nearly identical
    at N_U = 1, Sec. 4.4)."""
    res = []
    for acc in (False, True):
        wl = W.thermosolutal_convection(n=40, R=6.0, N=(1, 1, 1, 1))
        wl.params.accumulated = acc
        o = oracle.Oracle(wl.params, wl.fields)
        o.advance(30)
        res.append((o.get("phi"), o.get("U"), o.get("T")))
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_tip_diagnostic_on_known_profile():
    """The outermost phi = 0 crossing of tanh[(R - r)/(sqrt 2 W0)] along the
    axes is at distance R, up to the error of linear interpolation between
    nodes (for W0 = 1 and R = 10.3: 10 + 0.2092/0.6671 - 10.3 = 0.0136)."""
    n, R = 64, 10.3
    p = W.Params(nx=n, ny=n, frozen_T=True, bc_scalar_x=0, bc_scalar_y=0, W0=1.0, tau0=1.0,
                 tip_cx=32, tip_cy=32)
    o = oracle.Oracle(p, W.base_fields(p, W.circle_seed(n, n, 32, 32, R, 1.0)))
    tip = o.diagnostics()["tip"]
    assert np.abs(tip - R).max() < 0.015


@pytest.mark.parametrize("steps", [1, 4])
def test_update_is_local_within_six_nodes_per_base_step(steps):
    """The method is an explicit local update (Eqs. 25-26 stream one link;
    the gradients of Eq. 40, the compact stencil of the anti-trapping
    divergence and the phase-field gradient reach one node each; Fig. 1's
    chain phase -> transfer -> U/T/flow adds at most five nodes of reach per
    base step).  So the state at a node after k base steps depends only on
    the initial state within 6k nodes: a run on a window of the lattice
    reproduces the full-lattice run bit for bit at nodes farther than 6k from
    the window's artificial edges, and also up to an edge that is the
    lattice's own boundary.  The full-size GPU parity tests rely on this to
    check sampled outputs of lattices too large for the oracle."""
    from dataclasses import replace
    n = 192
    p, pts = W.multi_dendrite_params(n, n_seeds=3, min_dist=70.0)
    full = W.circle_seeds_window(p, pts, 8.0, 0, 0, n, n, 0.0, -0.55)
    o = oracle.Oracle(p, full)
    o.advance(steps)
    ref = {f: o.get(f) for f in ("phi", "U", "T", "ux", "uy", "rho")}
    o.close()
    m = 6 * steps
    w = 96
    # an interior window around the first seed, and windows on the inlet and
    # outflow columns (their lattice-side edge is exact)
    cx, cy = int(pts[0][0]), int(pts[0][1])
    x0 = min(max(cx - w // 2, 1), n - w - 1)
    y0 = min(max(cy - w // 2, 1), n - w - 1)
    cases = [(x0, y0, (m, w - m, m, w - m)), (0, 40, (0, w - m, m, w - m)), (n - w, 40, (m, w, m, w - m))]
    for (wx, wy, (xa, xb, ya, yb)) in cases:
        pw = replace(p, nx=w, ny=w, tip_cx=w // 2, tip_cy=w // 2)
        o = oracle.Oracle(pw, W.circle_seeds_window(p, pts, 8.0, wx, wy, w, w, 0.0, -0.55))
        o.advance(steps)
        for f, r in ref.items():
            got = o.get(f)[ya:yb, xa:xb]
            assert np.array_equal(got, r[wy + ya:wy + yb, wx + xa:wx + xb]), (wx, wy, f)
        o.close()


@pytest.mark.parametrize("q", [9, 5])
@pytest.mark.parametrize("N_T,alpha", [(1, 0.1), (2, 0.1), (1, 0.026)])
def test_dirichlet_wall_conduction_erf(N_T, alpha, q):
    """A bottom wall held at T_b (Sec. 4.4) conducting into a uniform liquid
    (phi = -1, no phase change, no flow): the semi-infinite solution
    T = T_b + (T0 - T_b) erf((y + 1/2) / (2 sqrt(alpha t))) with the wall half
    a link below row 0.  alpha = 0.026 is Table 1's liquid diffusivity
    (tau = 0.578); N_T = 2 takes the same alpha on the coarse clock.  A wall
    displaced by half a link misses by 2.6-5 %, plain bounce-back never
    reaches T_b.  q = 5: the same on the D2Q5 temperature lattice, whose
    anti-bounce-back carries its own weight (2 w_2 T_b with w_2 = 1/6); the
    D2Q9 weight there would hold the wall at 2/3 of T_b."""
    from scipy.special import erf
    nx, ny, steps, T0, Tb = 4, 300, 1200, 0.5, -1.0
    p = W.Params(nx=nx, ny=ny, has_T=True, bc_scalar_x=W.BC_PERIODIC, bc_scalar_y=W.BC_WALL,
                 N_T=N_T, W0=1.0, tau0=1.0, kappaS=alpha, kappaL=alpha, rhoCpS=1.0, rhoCpL=1.0,
                 T_ymin_dirichlet=True, T_ymin=Tb, tip_cx=2, tip_cy=ny // 2, q_scalar=q)
    o = oracle.Oracle(p, W.base_fields(p, np.full((ny, nx), -1.0), U0=0.0, T0=T0))
    o.advance(steps)
    T = o.get("T")
    y = np.arange(ny)
    exact = Tb + (T0 - Tb) * erf((y + 0.5) / (2.0 * math.sqrt(alpha * steps)))
    assert np.abs(T - exact[:, None])[: ny // 2].max() < 2e-3 * (T0 - Tb)


# ---------------------------------------------------------------------------
# Five-velocity option of the scalar lattices (D2Q5 for phi, U, T; flow D2Q9)
# ---------------------------------------------------------------------------
E5 = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1]])


def test_d2q5_basis_equilibria_and_collision_closed_form():
    """Moment basis (1, e_x, e_y, -4 + 5|e|^2, e_x^2 - e_y^2) is orthogonal
    with M M^T = diag(5, 2, 2, 20, 4); the equilibria of Eqs. 19 and 21 on the
    five velocities (weights 1/3, 1/6) have the moments the oracle relaxes to;
    and the literal product f - M^-1 S (M f - m_eq) + dt w_i Q with
    S = diag(1, 1/tau, 1/tau, 1, 1) equals the closed form
    w_i A + 3 w_i e_i.b + (1 - 1/tau) e_i.(j - b)/2 (A = chi + dt Q, b the
    first moment of f_eq, j that of f): the form the CUDA kernels use."""
    M, Mi, w = oracle.matrices5()
    assert np.array_equal(M @ M.T, np.diag([5.0, 2.0, 2.0, 20.0, 4.0]))
    assert np.abs(M @ Mi - np.eye(5)).max() < 1e-15
    assert np.allclose(w, [1 / 3, 1 / 6, 1 / 6, 1 / 6, 1 / 6], rtol=0, atol=1e-16)
    rng = np.random.default_rng(7)
    for kind in ("scalar", "phase"):
        a, ux, uy, c = 0.7, 0.013, -0.021, 2.0
        f, m = oracle.equilibrium_q(5, kind, a, ux, uy, c)
        assert np.abs(M @ f - m).max() < 1e-15
        assert abs(f.sum() - a) < 1e-15
        b = f @ E5
        exp_b = (a * np.array([ux, uy]) if kind == "scalar" else np.array([ux, uy])) / c
        assert np.abs(b - exp_b).max() < 1e-16
    for _ in range(5):
        fin = 0.2 + 0.05 * rng.standard_normal(5)
        chi, tau, dtQ = fin.sum(), 0.5 + rng.random() * 2, 0.01 * rng.standard_normal()
        feq, meq = oracle.equilibrium_q(5, "scalar", chi, 0.01, -0.02, 1.0)
        lit = oracle.collide_scalar_q(5, fin, meq, tau, dtQ)
        A, b, j = chi + dtQ, feq @ E5, fin @ E5
        closed = w * A + 3 * w * (E5 @ b) + (1 - 1 / tau) * (E5 @ (j - b)) / 2
        assert np.abs(lit - closed).max() < 1e-15


@pytest.mark.parametrize("field", ["U", "T"])
@pytest.mark.parametrize("N,tol", [(1, 1e-3), (2, 5e-3)])
def test_d2q5_gaussian_pulse_decay(field, N, tol):
    """Pure diffusion on the five-velocity lattice: c_s^2 = 1/3 as on D2Q9, so
    D = (tau - 1/2)/(3 dt) (Eq. 24) and the pulse decays as
    A s0^2/(s0^2 + 2Dt) exp(-r^2/(2(s0^2 + 2Dt)))."""
    n, s0, D, steps = 128, 5.0, 1.0 / 6.0, 400
    if field == "U":
        p = W.Params(nx=n, ny=n, has_U=True, bc_scalar_x=0, bc_scalar_y=0, N_U=N, DL=D, DS=D,
                     k=0.15, W0=1, tau0=1, q_scalar=5)
    else:
        p = W.Params(nx=n, ny=n, has_T=True, bc_scalar_x=0, bc_scalar_y=0, N_T=N, kappaS=D,
                     kappaL=D, W0=1, tau0=1, q_scalar=5)
    f = W.base_fields(p, -np.ones((n, n)))
    x, y = np.meshgrid(np.arange(n) - n / 2, np.arange(n) - n / 2)
    r2 = x * x + y * y
    f[field] = 0.1 * np.exp(-r2 / (2 * s0 * s0))
    o = oracle.Oracle(p, f)
    o.advance(steps)
    s2 = s0 * s0 + 2 * D * steps
    ana = 0.1 * s0 * s0 / s2 * np.exp(-r2 / (2 * s2))
    got = o.get(field)
    assert np.linalg.norm(got - ana) / np.linalg.norm(ana) < tol
    assert abs(got.sum() - ana.sum()) / ana.sum() < 1e-3


@pytest.mark.parametrize("eps", [0.0, 0.05])
def test_d2q5_planar_front_velocity(eps):
    """The travelling front of Eq. 1 on the five-velocity phase lattice:
    v = (4 sqrt 2 / 5) |lambda theta| W0 / (a_s tau0) to first order, as on
    D2Q9 (the source, tau_phi and Eq. 26 do not depend on the velocity set)."""
    W0, tau0, lt, n = 2.0, 12.0, -0.02, 256
    p = W.Params(nx=n, ny=4, frozen_T=True, bc_scalar_x=1, bc_scalar_y=0, W0=W0, tau0=tau0,
                 eps=eps, lam=1.0, theta_c=lt, q_scalar=5)
    x = np.arange(n) + 0.0
    phi = np.tile(-np.tanh((x - 60) / (math.sqrt(2) * W0 * (1 + eps))), (4, 1))
    o = oracle.Oracle(p, W.base_fields(p, phi))
    o.advance(1000)
    a = _front_position(o.get("phi")[0])
    o.advance(3000)
    b = _front_position(o.get("phi")[0])
    va = 4 * math.sqrt(2) / 5 * abs(lt) * W0 / (tau0 * (1 + eps))
    assert abs((b - a) / 3000 / va - 1) < 0.03


@pytest.mark.parametrize("bc", [W.BC_WALL, W.BC_PERIODIC])
def test_d2q5_solute_balance_exact_over_phase_step(bc):
    """The transfer (Eqs. 36-39) is lattice-independent apart from the
    injection weights, which sum to one on D2Q5 too: sum C/C_inf is unchanged
    by a phase update plus its transfer."""
    wl = W.thermosolutal_convection(n=48, R=6.0)
    p = wl.params
    p.bc_scalar_x = p.bc_scalar_y = bc
    p.eps, p.q_scalar = 0.05, 5
    o = oracle.Oracle(p, wl.fields)
    o.advance(60)
    c0 = o.get("C").sum()
    o.stage(0)
    assert abs(o.get("dU")).max() > 1e-6
    assert abs(o.get("C").sum() - c0) / c0 < 1e-13


def test_d2q5_fourfold_symmetry_thermal_dendrite():
    """The five velocities are invariant under the mirrors about the axes and
    the diagonal, so a centred seed stays four-fold symmetric (FP64)."""
    wl = W.thermal_free_dendrite(n=96)
    wl.params.q_scalar = 5
    o = oracle.Oracle(wl.params, wl.fields)
    o.advance(400)
    s = np.roll(np.roll(o.get("phi"), -48, 0), -48, 1)
    assert np.abs(s[:, (-np.arange(96)) % 96] - s).max() < 1e-10
    assert np.abs(s[(-np.arange(96)) % 96, :] - s).max() < 1e-10
    assert np.abs(s.T - s).max() < 1e-10


def test_isotropic_growth_without_anisotropy():
    """With the four-fold anisotropy switched off (eps = 0) a circular seed in
    an undercooled melt grows as a circle on the D2Q9 lattices: after 1500
    base steps its radius along an axis and along a diagonal agree within 3 %
    (the isotropy the nine-velocity set gives the phase-field streaming of
    Eq. 26 and the thermal solver).  A dropped diagonal population or a wrong
    diagonal weight breaks it."""
    wl = W.thermal_free_dendrite(n=128, N_T=1)
    p = wl.params
    p.eps = 0.0
    o = oracle.Oracle(p, wl.fields)
    o.advance(1500)
    phi = o.get("phi")
    o.close()
    c = 64

    def radius(dx, dy):
        r = 0.0
        for t in np.arange(0.0, 63.0, 0.25):
            i, j = int(round(c + dy * t)), int(round(c + dx * t))
            if 0 <= i < 128 and 0 <= j < 128 and phi[i, j] > 0:
                r = t * math.hypot(dx, dy)
        return r

    ra, rd = radius(1.0, 0.0), radius(1 / math.sqrt(2), 1 / math.sqrt(2))
    assert ra > 20.0
    assert abs(ra - rd) < 0.03 * ra, (ra, rd)


# ---------------------------------------------------------------------------
# Grains of different crystal orientation (the multi-dendrite case)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("vartheta", [0.0, math.pi / 8, 0.3, math.pi / 4, 1.2])
def test_anisotropy_in_a_turned_crystal_frame(vartheta):
    """a_s of a crystal whose axes are turned by vartheta is
    1 + eps cos 4(alpha - vartheta) (the trigonometric form of Eq. 2 about the
    crystal axes), and N = |grad phi|^2 a_s d a_s / d(grad phi) (Eq. 3) holds
    in the lattice frame: checked against central differences of a_s."""
    eps = 0.05
    for alpha in np.linspace(0.01, 2 * math.pi, 29):
        r = 0.3
        gx, gy = -r * math.cos(alpha), -r * math.sin(alpha)       # n = (cos alpha, sin alpha)
        a, Nx, Ny = oracle.aniso_frame(gx, gy, eps, vartheta)
        assert abs(a - (1 + eps * math.cos(4 * (alpha - vartheta)))) < 1e-14
        h = 1e-6
        dax = (oracle.aniso_frame(gx + h, gy, eps, vartheta)[0] - oracle.aniso_frame(gx - h, gy, eps, vartheta)[0]) / (2 * h)
        day = (oracle.aniso_frame(gx, gy + h, eps, vartheta)[0] - oracle.aniso_frame(gx, gy - h, eps, vartheta)[0]) / (2 * h)
        assert abs(Nx - r * r * a * dax) < 1e-8
        assert abs(Ny - r * r * a * day) < 1e-8


def test_quarter_turned_crystal_equals_the_unturned_one():
    """Eq. 2 has four-fold symmetry, so a grain turned by pi/2 grows exactly
    as an unturned one (up to the rounding of cos(pi/2)); a zero angle field
    is the axis-aligned form bit for bit."""
    wl = W.thermal_free_dendrite(n=64, R=5.0)
    runs = []
    for th in (None, 0.0, 0.5 * math.pi):
        f = dict(wl.fields)
        if th is not None:
            f["theta"] = np.full_like(f["phi"], th)
        o = oracle.Oracle(wl.params, f)
        o.advance(200)
        runs.append(o.get("phi"))
        o.close()
    assert np.array_equal(runs[0], runs[1])
    assert np.abs(runs[0] - runs[2]).max() < 1e-12


def test_turned_crystal_grows_along_its_own_axes():
    """A seed in a grain turned by pi/4 grows its primary arms along the
    diagonals: after 1500 base steps its diagonal and axial radii swap roles
    against the unturned seed's (each within 10 % of the other's, the
    difference being the lattice's own small anisotropy)."""
    wl = W.thermal_free_dendrite(n=128, N_T=1)
    c = 64

    def radii(theta):
        f = dict(wl.fields)
        if theta is not None:
            f["theta"] = np.full_like(f["phi"], theta)
        o = oracle.Oracle(wl.params, f)
        o.advance(1500)
        phi = o.get("phi")
        o.close()

        def radius(dx, dy):
            r = 0.0
            for t in np.arange(0.0, 63.0, 0.25):
                i, j = int(round(c + dy * t)), int(round(c + dx * t))
                if 0 <= i < 128 and 0 <= j < 128 and phi[i, j] > 0:
                    r = t * math.hypot(dx, dy)
            return r
        return radius(1.0, 0.0), radius(1 / math.sqrt(2), 1 / math.sqrt(2))

    a0, d0 = radii(None)
    a1, d1 = radii(math.pi / 4)
    assert a0 > d0 * 1.1 and d1 > a1 * 1.1
    assert abs(d1 - a0) < 0.1 * a0 and abs(a1 - d0) < 0.1 * d0


def test_grain_orientation_is_the_nearest_seed_angle():
    """The Voronoi orientation field of the input generator against brute
    force on a small window."""
    pts = np.array([[10.0, 10.0], [40.0, 12.0], [25.0, 40.0]])
    ang = np.array([0.1, 0.7, 1.3])
    th = W.grain_orientation(pts, ang, 5, 7, 30, 20, rows=3)
    for yy in range(20):
        for xx in range(30):
            d = [(5 + xx - px) ** 2 + (7 + yy - py) ** 2 for px, py in pts]
            assert th[yy, xx] == ang[int(np.argmin(d))]
