/*
 * FP64 CPU oracle of the unified multirate MRT lattice Boltzmann method for
 * thermosolutal dendritic solidification (Liu, Wu, Zhan; Secs. 2-3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header, table or helper with the CUDA path.
 *
 * It is a plain, slow, literal statement of the algorithm:
 *   - every collision is the literal moment-space product of Eq. 14,
 *     m = M f, m* = m - S (m - m_eq) [+ (I - S/2) G_F], f* = M^-1 m*,
 *     with M from Eq. 16 and M^-1 obtained by Gauss-Jordan elimination;
 *   - two full buffers per distribution set; every stage is a separate
 *     loop over all nodes;
 *   - the per-base-step order is the workflow of Fig. 1 (Sec. 3.3): phase
 *     update, phase-change transfer (Eqs. 36-39), concentration update,
 *     temperature update, flow update, each only when scheduled (Eq. 34).
 *
 * Readings of points the paper leaves open:
 *   R-sched  field chi fires at base step n iff (n+1) mod N_chi == 0.
 *   R-gradphi  grad(phi) by the isotropic stencil g_a = 3 sum_i w_i e_ia phi(x+e_i)
 *            (the same stencil as the divergence of J, Sec. 3.3); Eq. 40 is
 *            used for grad U and grad T.
 *   R-ghost  zero-flux walls: scalar ghost = mirror about the half-link wall;
 *            J ghost = mirror with its wall-normal component negated.
 *   R-bb     zero-flux for the distributions: half-way bounce-back; for phi
 *            through the Eq. 26 form with the node's own old value.
 *   R-as2    a_s^2 of Eq. 26 is that of the destination node (from grad phi^q).
 *   R-qphi   phase source per step dt_phi w_i Q_phi / tau0 (Eq. 1 carries
 *            Q_phi beside tau0 d_t phi).
 *   R-zero   |grad phi|^2 <= 1e-12: n = 0, N = 0, a_s = 1.
 *   R-ustar  U* in Eqs. 37-38 is the pre-injection U of this phase step.
 *   R-inlet  inlet column: after streaming f_i = f_eq_i(rho(x=1), u_in);
 *            outflow column: f_i(L-1) = f_i(L-2).
 *   R-frozen prescribed theta(y, t) = theta_c + G (y - y0 - V t) with t the
 *            time at the start of the base step.
 *   R-d2q5   the five-velocity option of the scalar lattices (see WQ5 / MM5).
 *   R-orientation  grains of different crystal orientation (the multi-
 *            dendrite case): Eq. 2 is written for crystal axes along x and y;
 *            a node of a grain turned by vartheta evaluates Eqs. 2-3 on its
 *            gradient turned into the crystal frame and turns N back
 *            (orc_aniso_frame).  Without an orientation field: Eq. 2 as printed.
 *   R-force  the Guo forcing term of Eq. 14 carries the factor dt_F (see
 *            collide_flow), so a flow update moves rho u by dt_F F_b.
 *   R-dirichlet  the cold bottom wall kept at T_b (Sec. 4.4): anti-bounce-back
 *            at the half-way wall below row 0, f_i = -f*_opp(i) + 2 w_i T_b
 *            for the links that enter row 0 from below; phi and U keep zero
 *            flux there.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* D2Q9 lattice, Eq. 15                                               */
/* ------------------------------------------------------------------ */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WQ[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* Five-velocity option for the scalar lattices (phi, U, T); the paper fixes
 * D2Q9 for all four fields, D2Q5 is read as the same scheme on the rest
 * velocity and the four axis links of Eq. 15: weights 1/3 and 1/6 (c_s^2 =
 * 1/3, so Eq. 24 ties tau to the diffusivity as on D2Q9), moments
 * (1, e_x, e_y, -4 + 5|e|^2, e_x^2 - e_y^2) and every moment but the two
 * fluxes relaxed at rate one, as Eq. 23 does on D2Q9. */
static const double WQ5[5] = {1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0};
static const double MM5[5][5] = {
    {1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0},
    {0, 0, 1, 0, -1},
    {-4, 1, 1, 1, 1},
    {0, 1, -1, 1, -1}};
static double MI5[5][5];

/* Transformation matrix of Eq. 16, as printed. */
static const double MM[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

static double MI[9][9];
static int mi_ready = 0;

static int opposite(int i) {
    for (int j = 0; j < 9; ++j)
        if (EX[j] == -EX[i] && EY[j] == -EY[i]) return j;
    return -1;
}

/* Inverse of an n x n matrix (n <= 9) by Gauss-Jordan elimination with
 * partial pivoting; A and out are row-major. */
static void gauss_jordan(int n, const double* A, double* out) {
    double a[9][18];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c) a[r][c] = (c < n) ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(a[r][c]) > fabs(a[p][c])) p = r;
        if (p != c)
            for (int k = 0; k < 2 * n; ++k) { double t = a[c][k]; a[c][k] = a[p][k]; a[p][k] = t; }
        double d = a[c][c];
        for (int k = 0; k < 2 * n; ++k) a[c][k] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double m = a[r][c];
            if (m != 0.0)
                for (int k = 0; k < 2 * n; ++k) a[r][k] -= m * a[c][k];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) out[r * n + c] = a[r][c + n];
}

/* M^-1 of both lattices */
static void build_minv(void) {
    if (mi_ready) return;
    gauss_jordan(9, &MM[0][0], &MI[0][0]);
    gauss_jordan(5, &MM5[0][0], &MI5[0][0]);
    mi_ready = 1;
}

/* weight w_i of the q-velocity scalar lattice (q = 9 or 5, the first five
 * velocities of Eq. 15) */
static double wq_s(int q, int i) { return q == 5 ? WQ5[i] : WQ[i]; }

static void mat_vec(const double A[9][9], const double* v, double* out) {
    for (int r = 0; r < 9; ++r) {
        double s = 0.0;
        for (int c = 0; c < 9; ++c) s += A[r][c] * v[c];
        out[r] = s;
    }
}

/* ------------------------------------------------------------------ */
/* Parameters (own definition; the CUDA path has its own)              */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t nx, ny;
    int32_t has_U, has_T, frozen_T, has_flow;
    int32_t bc_scalar_x, bc_scalar_y; /* 0 periodic, 1 wall */
    int32_t bc_flow_x, bc_flow_y;     /* 0 periodic, 1 wall, 2 inlet/outflow (x) */
    int32_t accumulated;
    int32_t N_phi, N_U, N_T, N_F;
    int32_t tip_cx, tip_cy;
    int32_t T_ymin_dirichlet;  /* 1: T = T_ymin on the wall below row 0 */
    int32_t q_scalar;          /* velocities of the phi, U, T lattices: 9 (0 reads as 9) or 5 */
    double dt_base;
    double W0, tau0, eps, lam;
    double Mc, k, DL, DS;
    double kappaS, kappaL, rhoCpS, rhoCpL, rhoL_Lh, T_shift, T_scale;
    double nu, u_in, Fbx, Fby, s_e, s_eps, s_q;
    double theta_c, frozen_G, frozen_y0, frozen_V;
    double T_ymin;
} orc_params;

typedef struct {
    orc_params p;
    int nn;
    int64_t step;          /* base steps done */
    double *f[4][2];       /* [phi, U, T, F][buffer] -> 9*nn, plane i at i*nn */
    int cur[4];
    double *phi, *phi_new; /* macro phi^q and phi^{q+1} */
    double *U, *T, *ux, *uy, *rho;
    double *post;          /* 9*nn post-collision scratch */
    double *as2;           /* nn */
    double *Jx, *Jy, *dU, *dT;
    double *accU, *accT;   /* accumulated-coupling stores */
    double *ori;           /* crystal angle of each node's grain, or NULL (axis-aligned Eq. 2) */
    double S_phi, J_U;     /* maxima since the last diagnostics read */
} orc_sim;

enum { F_PHI = 0, F_U = 1, F_T = 2, F_F = 3 };

static int qs(const orc_params* p) { return p->q_scalar == 5 ? 5 : 9; }

/* ------------------------------------------------------------------ */
/* Neighbour addressing                                                */
/* ------------------------------------------------------------------ */
static int wrap(int v, int n) { v %= n; return v < 0 ? v + n : v; }

/* scalar-field ghost (R-ghost): periodic wrap or mirror about the wall;
 * *flipx / *flipy report whether the x / y wall was crossed. */
static int scalar_nb(const orc_params* p, int x, int y, int* flipx, int* flipy) {
    int fx = 0, fy = 0;
    if (x < 0 || x >= p->nx) {
        if (p->bc_scalar_x == 0) x = wrap(x, p->nx);
        else { x = (x < 0) ? (-1 - x) : (2 * p->nx - 1 - x); fx = 1; }
    }
    if (y < 0 || y >= p->ny) {
        if (p->bc_scalar_y == 0) y = wrap(y, p->ny);
        else { y = (y < 0) ? (-1 - y) : (2 * p->ny - 1 - y); fy = 1; }
    }
    if (flipx) *flipx = fx;
    if (flipy) *flipy = fy;
    return y * p->nx + x;
}

/* streaming source of direction i into node (x, y); -1 if it lies behind a wall */
static int scalar_src(const orc_params* p, int x, int y, int i) {
    int sx = x - EX[i], sy = y - EY[i];
    if (sx < 0 || sx >= p->nx) { if (p->bc_scalar_x != 0) return -1; sx = wrap(sx, p->nx); }
    if (sy < 0 || sy >= p->ny) { if (p->bc_scalar_y != 0) return -1; sy = wrap(sy, p->ny); }
    return sy * p->nx + sx;
}

static int flow_src(const orc_params* p, int x, int y, int i) {
    int sx = x - EX[i], sy = y - EY[i];
    if (sx < 0 || sx >= p->nx) { if (p->bc_flow_x != 0) return -1; sx = wrap(sx, p->nx); }
    if (sy < 0 || sy >= p->ny) { if (p->bc_flow_y != 0) return -1; sy = wrap(sy, p->ny); }
    return sy * p->nx + sx;
}

/* isotropic gradient (R-gradphi): g_a = 3 sum_{i=1..8} w_i e_ia s(x + e_i) */
static void grad_iso(const orc_params* p, const double* s, int x, int y, double* gx, double* gy) {
    double ax = 0.0, ay = 0.0;
    for (int i = 1; i < 9; ++i) {
        double v = s[scalar_nb(p, x + EX[i], y + EY[i], NULL, NULL)];
        ax += WQ[i] * EX[i] * v;
        ay += WQ[i] * EY[i] * v;
    }
    *gx = 3.0 * ax;
    *gy = 3.0 * ay;
}

/* ------------------------------------------------------------------ */
/* Model functions, Sec. 2                                              */
/* ------------------------------------------------------------------ */
/* Eq. 2 and Eq. 3 with n = -grad phi/|grad phi|; N is |g|^2 a_s d a_s/d g,
 * with d a_s/d g_x = 16 eps g_x g_y^2 (g_x^2 - g_y^2)/|g|^6 (Eq. 2 differentiated). */
void orc_aniso(double gx, double gy, double eps, double* as, double* Nx, double* Ny) {
    double g2 = gx * gx + gy * gy;
    if (g2 <= 1e-12) { *as = 1.0; *Nx = 0.0; *Ny = 0.0; return; }
    double nx = -gx / sqrt(g2), ny = -gy / sqrt(g2);
    double a = 1.0 - 3.0 * eps + 4.0 * eps * (nx * nx * nx * nx + ny * ny * ny * ny);
    double g6 = g2 * g2 * g2;
    double dax = 16.0 * eps * gx * gy * gy * (gx * gx - gy * gy) / g6;
    double day = 16.0 * eps * gy * gx * gx * (gy * gy - gx * gx) / g6;
    *as = a;
    *Nx = g2 * a * dax;
    *Ny = g2 * a * day;
}

/* Eqs. 2-3 in the frame of a crystal whose axes are turned by vartheta
 * (R-orientation): the gradient is taken into the crystal frame,
 * g' = R(-vartheta) g, Eq. 2 and Eq. 3 are evaluated there, and N is turned
 * back, N = R(vartheta) N'.  With vartheta = 0 this is orc_aniso. */
void orc_aniso_frame(double gx, double gy, double eps, double vartheta, double* as, double* Nx, double* Ny) {
    const double c = cos(vartheta), sn = sin(vartheta);
    const double Rm[2][2] = {{c, sn}, {-sn, c}};     /* R(-vartheta) */
    const double gpx = Rm[0][0] * gx + Rm[0][1] * gy, gpy = Rm[1][0] * gx + Rm[1][1] * gy;
    double Npx, Npy;
    orc_aniso(gpx, gpy, eps, as, &Npx, &Npy);
    *Nx = Rm[0][0] * Npx + Rm[1][0] * Npy;             /* R(vartheta) = R(-vartheta)^T */
    *Ny = Rm[0][1] * Npx + Rm[1][1] * Npy;
}

static void aniso_at(const orc_sim* s, int n, double gx, double gy, double* as, double* Nx, double* Ny) {
    if (s->ori) orc_aniso_frame(gx, gy, s->p.eps, s->ori[n], as, Nx, Ny);
    else orc_aniso(gx, gy, s->p.eps, as, Nx, Ny);
}

static double theta_at(const orc_sim* s, int node, int y, double t) {
    const orc_params* p = &s->p;
    if (p->has_T) return (s->T[node] - p->T_shift) / p->T_scale;           /* Eq. 5 */
    if (p->frozen_T) return p->theta_c + p->frozen_G * ((double)y - p->frozen_y0 - p->frozen_V * t);
    return p->theta_c;
}

static double D_eff(const orc_params* p, double phi) {                     /* Eq. 7 */
    return ((1.0 + phi) * p->DS + (1.0 - phi) * p->DL) / ((1.0 + p->k) - (1.0 - p->k) * phi);
}
static double rhoCp_eff(const orc_params* p, double phi) {                 /* Eq. 11 */
    return 0.5 * (1.0 + phi) * p->rhoCpS + 0.5 * (1.0 - phi) * p->rhoCpL;
}
static double kappa_eff(const orc_params* p, double phi) {                 /* Eq. 11 */
    return 0.5 * (1.0 + phi) * p->kappaS + 0.5 * (1.0 - phi) * p->kappaL;
}


/* Relaxation times of Eqs. 24 and 32 at a given phi (a_s = 1 for phi's own):
 * out = [tau_phi, tau_U, tau_T, tau_F]. */
void orc_relaxation_times(const orc_params* p, double phi, double* out) {
    double dphi = p->N_phi * p->dt_base, dU = p->N_U * p->dt_base;
    double dT = p->N_T * p->dt_base, dF = p->N_F * p->dt_base;
    out[0] = 3.0 * dphi * p->W0 * p->W0 / p->tau0 + 0.5;
    out[1] = 3.0 * dU * D_eff(p, phi) + 0.5;
    out[2] = 3.0 * dT * kappa_eff(p, phi) / rhoCp_eff(p, phi) + 0.5;
    out[3] = 3.0 * dF * p->nu + 0.5;
}

/* ------------------------------------------------------------------ */
/* Equilibria (exported for the equilibrium-moment pins)                */
/* ------------------------------------------------------------------ */
/* Eqs. 19-22 on the q-velocity scalar lattice; on D2Q5 the equilibrium
 * moments are those of the same equilibrium, (chi, chi u_x/c, chi u_y/c,
 * -2/3 chi, 0), resp. (phi, v_x/c, v_y/c, -2/3 phi, 0). */
void orc_feq_scalar_q(int q, double chi, double ux, double uy, double c, double* feq) {   /* Eq. 19 */
    for (int i = 0; i < q; ++i) feq[i] = wq_s(q, i) * chi * (1.0 + 3.0 * (EX[i] * ux + EY[i] * uy) / c);
}
void orc_meq_scalar_q(int q, double chi, double ux, double uy, double c, double* m) {     /* Eq. 20 */
    if (q == 5) {
        double v[5] = {chi, ux * chi / c, uy * chi / c, -2.0 / 3.0 * chi, 0.0};
        memcpy(m, v, sizeof v);
        return;
    }
    double v[9] = {chi, -2.0 * chi, chi, ux * chi / c, -ux * chi / c, uy * chi / c, -uy * chi / c, 0.0, 0.0};
    memcpy(m, v, sizeof v);
}
void orc_feq_phase_q(int q, double phi, double vx, double vy, double c, double* feq) {   /* Eq. 21 */
    for (int i = 0; i < q; ++i) feq[i] = wq_s(q, i) * (phi + 3.0 * (EX[i] * vx + EY[i] * vy) / c);
}
void orc_meq_phase_q(int q, double phi, double vx, double vy, double c, double* m) {      /* Eq. 22 */
    if (q == 5) {
        double v[5] = {phi, vx / c, vy / c, -2.0 / 3.0 * phi, 0.0};
        memcpy(m, v, sizeof v);
        return;
    }
    double v[9] = {phi, -2.0 * phi, phi, vx / c, -vx / c, vy / c, -vy / c, 0.0, 0.0};
    memcpy(m, v, sizeof v);
}
void orc_feq_scalar(double chi, double ux, double uy, double c, double* feq) { orc_feq_scalar_q(9, chi, ux, uy, c, feq); }
void orc_meq_scalar(double chi, double ux, double uy, double c, double* m) { orc_meq_scalar_q(9, chi, ux, uy, c, m); }
void orc_feq_phase(double phi, double vx, double vy, double c, double* feq) { orc_feq_phase_q(9, phi, vx, vy, c, feq); }
void orc_meq_phase(double phi, double vx, double vy, double c, double* m) { orc_meq_phase_q(9, phi, vx, vy, c, m); }
void orc_feq_flow(double rho, double ux, double uy, double c, double* feq) {     /* Eq. 28 */
    double u2 = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        feq[i] = WQ[i] * rho * (1.0 + 3.0 * eu / c + 4.5 * eu * eu / (c * c) - 1.5 * u2 / (c * c));
    }
}
void orc_meq_flow(double rho, double ux, double uy, double c, double* m) {       /* Eq. 29 */
    double u2 = (ux * ux + uy * uy) / (c * c);
    double v[9] = {rho, rho * (-2.0 + 3.0 * u2), rho * (1.0 - 3.0 * u2), rho * ux / c, -rho * ux / c,
                   rho * uy / c, -rho * uy / c, rho * (ux * ux - uy * uy) / (c * c), rho * ux * uy / (c * c)};
    memcpy(m, v, sizeof v);
}
static void guo_moments(double Fx, double Fy, double ux, double uy, double c, double* G) { /* Eq. 30 */
    double fu = Fx * ux + Fy * uy;
    G[0] = 0.0;
    G[1] = 6.0 * fu / (c * c);
    G[2] = -6.0 * fu / (c * c);
    G[3] = Fx / c;
    G[4] = -Fx / c;
    G[5] = Fy / c;
    G[6] = -Fy / c;
    G[7] = 2.0 * (Fx * ux - Fy * uy) / (c * c);
    G[8] = (Fy * ux + Fx * uy) / (c * c);
}

void orc_matrices(double* M81, double* Minv81, int* ex, int* ey, double* w) {
    build_minv();
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) { M81[r * 9 + c] = MM[r][c]; Minv81[r * 9 + c] = MI[r][c]; }
    for (int i = 0; i < 9; ++i) { ex[i] = EX[i]; ey[i] = EY[i]; w[i] = WQ[i]; }
}
void orc_matrices5(double* M25, double* Minv25, double* w) {
    build_minv();
    for (int r = 0; r < 5; ++r)
        for (int c = 0; c < 5; ++c) { M25[r * 5 + c] = MM5[r][c]; Minv25[r * 5 + c] = MI5[r][c]; }
    for (int i = 0; i < 5; ++i) w[i] = WQ5[i];
}

/* Scalar collision of Eq. 14 with S of Eq. 23 (literal products):
 * f* = f - M^-1 S (M f - m_eq) + dt w_i Q, on the q-velocity lattice (on
 * D2Q5 S = diag(1, 1/tau, 1/tau, 1, 1)). Exported for the closed-form pins. */
void orc_collide_scalar_q(int q, const double* f, const double* meq, double tau, double dtQ, double* fpost) {
    build_minv();
    if (q == 5) {
        double m[5], d[5];
        const double S[5] = {1, 1.0 / tau, 1.0 / tau, 1, 1};
        for (int r = 0; r < 5; ++r) {
            m[r] = 0.0;
            for (int c = 0; c < 5; ++c) m[r] += MM5[r][c] * f[c];
            d[r] = S[r] * (m[r] - meq[r]);
        }
        for (int i = 0; i < 5; ++i) {
            double corr = 0.0;
            for (int c = 0; c < 5; ++c) corr += MI5[i][c] * d[c];
            fpost[i] = f[i] - corr + dtQ * WQ5[i];
        }
        return;
    }
    double m[9], d[9], corr[9];
    mat_vec(MM, f, m);
    double S[9] = {1, 1, 1, 1.0 / tau, 1, 1.0 / tau, 1, 1, 1};
    for (int k = 0; k < 9; ++k) d[k] = S[k] * (m[k] - meq[k]);
    mat_vec(MI, d, corr);
    for (int i = 0; i < 9; ++i) fpost[i] = f[i] - corr[i] + dtQ * WQ[i];
}
void orc_collide_scalar(const double* f, const double* meq, double tau, double dtQ, double* fpost) {
    orc_collide_scalar_q(9, f, meq, tau, dtQ, fpost);
}

/* Flow collision of Eq. 14 with S of Eq. 31 and Guo forcing (Eq. 30).
 * R-force: the forcing term enters as dt_F M^-1 (I - S/2) G_F, with the same
 * factor dt_F that Eq. 14 gives the scalar sources and Eq. 27 the half-force
 * shift, so that one flow update moves rho u by dt_F F_b (Guo's scheme); the
 * printed G_F alone would move it by F_b per update whatever dt_F is.  At
 * dt_F = 1 the two coincide. */
static void collide_flow(const orc_params* p, const double* f, double c, double dt, double* fpost,
                         double* rho_o, double* ux_o, double* uy_o) {
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) { rho += f[i]; jx += EX[i] * f[i]; jy += EY[i] * f[i]; }
    double ux = (c * jx + 0.5 * dt * p->Fbx) / rho;   /* Eq. 27 */
    double uy = (c * jy + 0.5 * dt * p->Fby) / rho;
    double tauF = 3.0 * dt * p->nu + 0.5;             /* Eq. 32 */
    double S[9] = {0.0, p->s_e, p->s_eps, 0.0, p->s_q, 0.0, p->s_q, 1.0 / tauF, 1.0 / tauF};
    double m[9], meq[9], G[9], mp[9];
    mat_vec(MM, f, m);
    orc_meq_flow(rho, ux, uy, c, meq);
    guo_moments(p->Fbx, p->Fby, ux, uy, c, G);
    for (int k = 0; k < 9; ++k) mp[k] = m[k] - S[k] * (m[k] - meq[k]) + dt * (1.0 - 0.5 * S[k]) * G[k];
    mat_vec(MI, mp, fpost);
    if (rho_o) { *rho_o = rho; *ux_o = ux; *uy_o = uy; }
}

/* ------------------------------------------------------------------ */
/* Simulation object                                                    */
/* ------------------------------------------------------------------ */
orc_sim* orc_create(const orc_params* p) {
    build_minv();
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->p = *p;
    s->nn = p->nx * p->ny;
    size_t n = (size_t)s->nn;
    for (int fld = 0; fld < 4; ++fld)
        for (int b = 0; b < 2; ++b) s->f[fld][b] = (double*)calloc(9 * n, sizeof(double));
    s->phi = calloc(n, 8); s->phi_new = calloc(n, 8);
    s->U = calloc(n, 8); s->T = calloc(n, 8);
    s->ux = calloc(n, 8); s->uy = calloc(n, 8); s->rho = calloc(n, 8);
    s->post = calloc(9 * n, 8); s->as2 = calloc(n, 8);
    s->Jx = calloc(n, 8); s->Jy = calloc(n, 8); s->dU = calloc(n, 8); s->dT = calloc(n, 8);
    s->accU = calloc(n, 8); s->accT = calloc(n, 8);
    return s;
}

void orc_destroy(orc_sim* s) {
    if (!s) return;
    for (int fld = 0; fld < 4; ++fld)
        for (int b = 0; b < 2; ++b) free(s->f[fld][b]);
    free(s->phi); free(s->phi_new); free(s->U); free(s->T); free(s->ux); free(s->uy); free(s->rho);
    free(s->post); free(s->as2); free(s->Jx); free(s->Jy); free(s->dU); free(s->dT);
    free(s->accU); free(s->accT);
    free(s->ori);
    free(s);
}

/* Per-node crystal angle (ny x nx, row-major), or NULL for the axis-aligned
 * form; set it before orc_set_fields, whose phase equilibria use it. */
void orc_set_orientation(orc_sim* s, const double* vartheta) {
    if (!vartheta) { free(s->ori); s->ori = NULL; return; }
    if (!s->ori) s->ori = (double*)malloc((size_t)s->nn * 8);
    memcpy(s->ori, vartheta, (size_t)s->nn * 8);
}

/* Initial distributions f = f_eq of the initial macroscopic fields. For phi
 * the equilibrium carries v_n from the initial gradient. */
void orc_set_fields(orc_sim* s, const double* phi, const double* U, const double* T, const double* ux,
                    const double* uy, const double* rho) {
    const orc_params* p = &s->p;
    int nn = s->nn;
    memcpy(s->phi, phi, nn * 8);
    memcpy(s->U, U, nn * 8);
    memcpy(s->T, T, nn * 8);
    memcpy(s->ux, ux, nn * 8);
    memcpy(s->uy, uy, nn * 8);
    memcpy(s->rho, rho, nn * 8);
    for (int b = 0; b < 4; ++b) s->cur[b] = 0;
    double cphi = 1.0 / (p->N_phi * p->dt_base), cU = 1.0 / (p->N_U * p->dt_base);
    double cT = 1.0 / (p->N_T * p->dt_base), cF = 1.0 / (p->N_F * p->dt_base);
    const int q = qs(p);
    for (int fld = 0; fld < 3; ++fld) memset(s->f[fld][0], 0, 9 * (size_t)nn * 8);
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            int n = y * p->nx + x;
            double feq[9], gx, gy, as, Nx, Ny;
            grad_iso(p, s->phi, x, y, &gx, &gy);
            aniso_at(s, n, gx, gy, &as, &Nx, &Ny);
            orc_feq_phase_q(q, phi[n], -p->W0 * p->W0 * Nx / p->tau0, -p->W0 * p->W0 * Ny / p->tau0, cphi, feq);
            for (int i = 0; i < q; ++i) s->f[F_PHI][0][i * nn + n] = feq[i];
            double vx = p->has_flow ? ux[n] : 0.0, vy = p->has_flow ? uy[n] : 0.0;
            orc_feq_scalar_q(q, U[n], vx, vy, cU, feq);
            for (int i = 0; i < q; ++i) s->f[F_U][0][i * nn + n] = feq[i];
            orc_feq_scalar_q(q, T[n], vx, vy, cT, feq);
            for (int i = 0; i < q; ++i) s->f[F_T][0][i * nn + n] = feq[i];
            orc_feq_flow(rho[n], ux[n], uy[n], cF, feq);
            for (int i = 0; i < 9; ++i) s->f[F_F][0][i * nn + n] = feq[i];
        }
    memset(s->accU, 0, nn * 8);
    memset(s->accT, 0, nn * 8);
    s->step = 0;
    s->S_phi = 0.0;
    s->J_U = 0.0;
}

/* ------------------------------------------------------------------ */
/* Phase-field update: Eqs. 2-4, 14, 21-24, 26, 18                      */
/* ------------------------------------------------------------------ */
static void phase_step(orc_sim* s, double t) {
    const orc_params* p = &s->p;
    int nn = s->nn;
    double dt = p->N_phi * p->dt_base, c = 1.0 / dt;
    double* f = s->f[F_PHI][s->cur[F_PHI]];
    double* fn = s->f[F_PHI][1 - s->cur[F_PHI]];
    const int q = qs(p);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            int n = y * p->nx + x;
            double gx, gy, as, Nx, Ny;
            grad_iso(p, s->phi, x, y, &gx, &gy);
            aniso_at(s, n, gx, gy, &as, &Nx, &Ny);
            double vnx = -p->W0 * p->W0 * Nx / p->tau0, vny = -p->W0 * p->W0 * Ny / p->tau0;
            double tau = 3.0 * dt * as * as * p->W0 * p->W0 / p->tau0 + 0.5;         /* Eq. 24 */
            double ph = s->phi[n];
            double Ustar = p->has_U ? s->U[n] : 0.0;
            double th = theta_at(s, n, y, t);
            double one = 1.0 - ph * ph;
            double Q = ph * one - p->lam * (p->Mc * Ustar + th) * one * one;          /* Eq. 4 */
            double fl[9], meq[9], fp[9];
            for (int i = 0; i < q; ++i) fl[i] = f[i * nn + n];
            orc_meq_phase_q(q, ph, vnx, vny, c, meq);
            orc_collide_scalar_q(q, fl, meq, tau, dt * Q / p->tau0, fp);
            for (int i = 0; i < q; ++i) s->post[i * nn + n] = fp[i];
            s->as2[n] = as * as;
        }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            int n = y * p->nx + x;
            double a2 = s->as2[n], sum = 0.0;
            for (int i = 0; i < q; ++i) {
                int src = scalar_src(p, x, y, i);
                double inc = (src < 0) ? s->post[opposite(i) * nn + n] : s->post[i * nn + src];
                double v = (inc - (1.0 - a2) * f[i * nn + n]) / a2;                /* Eq. 26 */
                fn[i * nn + n] = v;
                sum += v;
            }
            s->phi_new[n] = sum;                                                   /* Eq. 18 */
        }
    s->cur[F_PHI] = 1 - s->cur[F_PHI];
}

/* Phase-change transfer, Eqs. 36-39 */
static void pc_transfer(orc_sim* s) {
    const orc_params* p = &s->p;
    int nn = s->nn;
    double pre = p->W0 / (2.0 * sqrt(2.0));
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            int n = y * p->nx + x;
            double dphi = s->phi_new[n] - s->phi[n];                               /* Eq. 36 */
            double gx, gy;
            grad_iso(p, s->phi_new, x, y, &gx, &gy);
            double g2 = gx * gx + gy * gy, nxv = 0.0, nyv = 0.0;
            if (g2 > 1e-12) { nxv = -gx / sqrt(g2); nyv = -gy / sqrt(g2); }
            double Us = p->has_U ? s->U[n] : 0.0;
            double a = pre * (1.0 + (1.0 - p->k) * Us) * dphi;                     /* Eq. 37 */
            s->Jx[n] = a * nxv;
            s->Jy[n] = a * nyv;
        }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            int n = y * p->nx + x;
            double div = 0.0;
            for (int i = 1; i < 9; ++i) {
                int fx, fy;
                int m = scalar_nb(p, x + EX[i], y + EY[i], &fx, &fy);
                double jx = fx ? -s->Jx[m] : s->Jx[m];
                double jy = fy ? -s->Jy[m] : s->Jy[m];
                div += WQ[i] * (EX[i] * jx + EY[i] * jy);
            }
            div *= 3.0;
            double dphi = s->phi_new[n] - s->phi[n];
            double pn = s->phi_new[n];
            double Us = p->has_U ? s->U[n] : 0.0;
            s->dU[n] = ((1.0 + (1.0 - p->k) * Us) * dphi - 2.0 * div) / ((1.0 + p->k) - (1.0 - p->k) * pn); /* Eq. 38 */
            s->dT[n] = p->rhoL_Lh * dphi / (2.0 * rhoCp_eff(p, pn));
        }
    /* Eq. 39: isotropic injection into the distributions and the macros */
    double smax = 0.0;
    for (int n = 0; n < nn; ++n) {
        if (p->has_U) {
            double a = fabs(s->dU[n]);
            if (a > smax) smax = a;
        }
    }
    if (smax > s->S_phi) s->S_phi = smax;
    if (!p->accumulated) {
        if (smax > s->J_U) s->J_U = smax;
        double* fu = s->f[F_U][s->cur[F_U]];
        double* ft = s->f[F_T][s->cur[F_T]];
        const int q = qs(p);
        for (int n = 0; n < nn; ++n) {
            if (p->has_U) {
                for (int i = 0; i < q; ++i) fu[i * nn + n] += wq_s(q, i) * s->dU[n];
                s->U[n] += s->dU[n];
            }
            if (p->has_T) {
                for (int i = 0; i < q; ++i) ft[i * nn + n] += wq_s(q, i) * s->dT[n];
                s->T[n] += s->dT[n];
            }
        }
    } else {
        for (int n = 0; n < nn; ++n) { s->accU[n] += s->dU[n]; s->accT[n] += s->dT[n]; }
    }
    /* phi^{q+1} becomes the current phase field */
    double* t = s->phi; s->phi = s->phi_new; s->phi_new = t;
}

/* Accumulated coupling: inject the stored sum at the coarse update. */
static void inject_accumulated(orc_sim* s, int fld) {
    const orc_params* p = &s->p;
    int nn = s->nn;
    double* f = s->f[fld][s->cur[fld]];
    double* acc = (fld == F_U) ? s->accU : s->accT;
    double* mac = (fld == F_U) ? s->U : s->T;
    double jmax = 0.0;
    const int q = qs(p);
    for (int n = 0; n < nn; ++n) {
        for (int i = 0; i < q; ++i) f[i * nn + n] += wq_s(q, i) * acc[n];
        mac[n] += acc[n];
        if (fld == F_U && fabs(acc[n]) > jmax) jmax = fabs(acc[n]);
        acc[n] = 0.0;
    }
    if (fld == F_U && jmax > s->J_U) s->J_U = jmax;
}

/* Concentration / temperature update: Eqs. 7-8 / 10-12 (tr parts), 14, 19-20,
 * 23-25, 40, 18. */
static void scalar_step(orc_sim* s, int fld) {
    const orc_params* p = &s->p;
    int nn = s->nn;
    int N = (fld == F_U) ? p->N_U : p->N_T;
    double dt = N * p->dt_base, c = 1.0 / dt;
    if (p->accumulated) inject_accumulated(s, fld);
    double* f = s->f[fld][s->cur[fld]];
    double* fn = s->f[fld][1 - s->cur[fld]];
    double* mac = (fld == F_U) ? s->U : s->T;
    const int q = qs(p);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            int n = y * p->nx + x;
            double fl[9], feq[9], meq[9], fp[9];
            double chi = 0.0;
            for (int i = 0; i < q; ++i) { fl[i] = f[i * nn + n]; chi += fl[i]; }   /* Eq. 18 */
            double ph = s->phi[n];
            double vx = p->has_flow ? s->ux[n] : 0.0, vy = p->has_flow ? s->uy[n] : 0.0;
            double D, coef;
            if (fld == F_U) {
                D = D_eff(p, ph);
                coef = -(1.0 - p->k) * D / ((1.0 + p->k) - (1.0 - p->k) * ph);       /* Eq. 8, tr */
            } else {
                double rc = rhoCp_eff(p, ph);
                D = kappa_eff(p, ph) / rc;
                coef = (p->rhoCpS - p->rhoCpL) / (2.0 * rc) * D;                     /* Eq. 12, tr */
            }
            double tau = 3.0 * dt * D + 0.5;                                          /* Eq. 24 */
            orc_feq_scalar_q(q, chi, vx, vy, c, feq);
            double sx = 0.0, sy = 0.0;
            for (int i = 1; i < q; ++i) { sx += (fl[i] - feq[i]) * EX[i]; sy += (fl[i] - feq[i]) * EY[i]; }
            double gcx = -3.0 / tau * sx, gcy = -3.0 / tau * sy;                      /* Eq. 40 */
            double gpx, gpy;
            grad_iso(p, s->phi, x, y, &gpx, &gpy);
            double Q = coef * (gcx * gpx + gcy * gpy);
            orc_meq_scalar_q(q, chi, vx, vy, c, meq);
            orc_collide_scalar_q(q, fl, meq, tau, dt * Q, fp);
            for (int i = 0; i < q; ++i) s->post[i * nn + n] = fp[i];
        }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            int n = y * p->nx + x;
            double sum = 0.0;
            for (int i = 0; i < q; ++i) {
                int src = scalar_src(p, x, y, i);
                double v;
                if (src >= 0) v = s->post[i * nn + src];                               /* Eq. 25 */
                else if (fld == F_T && p->T_ymin_dirichlet && y - EY[i] < 0)
                    v = -s->post[opposite(i) * nn + n] + 2.0 * wq_s(q, i) * p->T_ymin;  /* R-dirichlet */
                else v = s->post[opposite(i) * nn + n];                                 /* R-bb */
                fn[i * nn + n] = v;
                sum += v;
            }
            mac[n] = sum;                                                            /* Eq. 18 */
        }
    s->cur[fld] = 1 - s->cur[fld];
}

/* Flow update: Eqs. 27-33 */
static void flow_step(orc_sim* s) {
    const orc_params* p = &s->p;
    int nn = s->nn;
    double dt = p->N_F * p->dt_base, c = 1.0 / dt;
    double* f = s->f[F_F][s->cur[F_F]];
    double* fn = s->f[F_F][1 - s->cur[F_F]];
#pragma omp parallel for schedule(static)
    for (int n = 0; n < nn; ++n) {
        double fl[9], fp[9];
        for (int i = 0; i < 9; ++i) fl[i] = f[i * nn + n];
        collide_flow(p, fl, c, dt, fp, NULL, NULL, NULL);
        for (int i = 0; i < 9; ++i) s->post[i * nn + n] = fp[i];
    }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            int n = y * p->nx + x;
            double fLy = 0.5 * (1.0 - s->phi[n]);
            for (int i = 0; i < 9; ++i) {
                int src = flow_src(p, x, y, i);
                int o = opposite(i);
                double v;
                if (src < 0) v = s->post[o * nn + n];
                else {
                    double fLmid = 0.5 * (0.5 * (1.0 - s->phi[src]) + fLy);
                    v = fLmid * s->post[i * nn + src] + (1.0 - fLmid) * s->post[o * nn + n]; /* Eq. 33 */
                }
                fn[i * nn + n] = v;
            }
        }
    if (p->bc_flow_x == 2) {                                                         /* R-inlet */
        int nx = p->nx;
        for (int y = 0; y < p->ny; ++y) {
            int r = y * nx;
            for (int i = 0; i < 9; ++i) fn[i * nn + r + nx - 1] = fn[i * nn + r + nx - 2];
            double rho1 = 0.0;
            for (int i = 0; i < 9; ++i) rho1 += fn[i * nn + r + 1];
            double feq[9];
            orc_feq_flow(rho1, p->u_in, 0.0, c, feq);
            for (int i = 0; i < 9; ++i) fn[i * nn + r] = feq[i];
        }
    }
    for (int n = 0; n < nn; ++n) {                                                  /* Eq. 27 */
        double rho = 0.0, jx = 0.0, jy = 0.0;
        for (int i = 0; i < 9; ++i) { double v = fn[i * nn + n]; rho += v; jx += EX[i] * v; jy += EY[i] * v; }
        s->rho[n] = rho;
        s->ux[n] = (c * jx + 0.5 * dt * p->Fbx) / rho;
        s->uy[n] = (c * jy + 0.5 * dt * p->Fby) / rho;
    }
    s->cur[F_F] = 1 - s->cur[F_F];
}

/* One base step in the workflow order of Fig. 1 (Eq. 34 schedule). */
static void base_step(orc_sim* s) {
    const orc_params* p = &s->p;
    int64_t n = s->step;
    double t = (double)n * p->dt_base;
    if ((n + 1) % p->N_phi == 0) { phase_step(s, t); pc_transfer(s); }
    if (p->has_U && (n + 1) % p->N_U == 0) scalar_step(s, F_U);
    if (p->has_T && (n + 1) % p->N_T == 0) scalar_step(s, F_T);
    if (p->has_flow && (n + 1) % p->N_F == 0) flow_step(s);
    s->step = n + 1;
}

void orc_advance(orc_sim* s, int64_t nsteps) {
    for (int64_t k = 0; k < nsteps; ++k) base_step(s);
}

/* Single stages, for invariant pins: one phase update + transfer, or one
 * scalar / flow update, regardless of the schedule. */
void orc_stage(orc_sim* s, int which) {
    double t = (double)s->step * s->p.dt_base;
    if (which == 0) { phase_step(s, t); pc_transfer(s); }
    else if (which == 1) scalar_step(s, F_U);
    else if (which == 2) scalar_step(s, F_T);
    else if (which == 3) flow_step(s);
    else if (which == 4) phase_step(s, t);   /* phase update only: phi^{q+1} in phi_new */
}

/* which: 0 phi, 1 U, 2 T, 3 ux, 4 uy, 5 rho, 6 C/C_inf, 7 theta, 8 dU, 9 dT,
 * 10 phi^{q+1} (after a which=4 stage), 11..19 f^phi_i, 20..28 f^U_i,
 * 29..37 f^T_i, 38..46 f^F_i */
void orc_get(const orc_sim* s, int which, double* out) {
    const orc_params* p = &s->p;
    int nn = s->nn;
    for (int n = 0; n < nn; ++n) {
        double v = 0.0;
        int y = n / p->nx;
        switch (which) {
            case 0: v = s->phi[n]; break;
            case 1: v = s->U[n]; break;
            case 2: v = s->T[n]; break;
            case 3: v = s->ux[n]; break;
            case 4: v = s->uy[n]; break;
            case 5: v = s->rho[n]; break;
            case 6: v = 0.5 * (1.0 + (1.0 - p->k) * s->U[n]) * ((1.0 + p->k) - (1.0 - p->k) * s->phi[n]); break;
            case 7: v = theta_at(s, n, y, (double)s->step * p->dt_base); break;
            case 8: v = s->dU[n]; break;
            case 9: v = s->dT[n]; break;
            case 10: v = s->phi_new[n]; break;
            default: {
                int k = which - 11, fld = k / 9, i = k % 9;
                if (fld >= 0 && fld < 4) v = s->f[fld][s->cur[fld]][i * nn + n];
            }
        }
        out[n] = v;
    }
}

int64_t orc_step(const orc_sim* s) { return s->step; }

/* tip crossing distance along one axis through (cx, cy); dir 0:+x 1:+y 2:-x 3:-y.
 * Outermost phi = 0 crossing, linear interpolation. */
static double tip_dist(const orc_sim* s, int dir) {
    const orc_params* p = &s->p;
    int cx = p->tip_cx, cy = p->tip_cy;
    int len = (dir == 0) ? p->nx - cx : (dir == 1) ? p->ny - cy : (dir == 2) ? cx + 1 : cy + 1;
#define PHI_AT(k) s->phi[(dir == 0) ? (cy * p->nx + cx + (k)) : (dir == 1) ? ((cy + (k)) * p->nx + cx) \
                       : (dir == 2) ? (cy * p->nx + cx - (k)) : ((cy - (k)) * p->nx + cx)]
    if (PHI_AT(len - 1) >= 0.0) return (double)(len - 1);
    for (int k = len - 2; k >= 0; --k) {
        double a = PHI_AT(k), b = PHI_AT(k + 1);
        if (a >= 0.0 && b < 0.0) return (double)k + a / (a - b);
    }
#undef PHI_AT
    return 0.0;
}

/* out: [M_C, H, S_phi, J_U, tip+x, tip+y, tip-x, tip-y, nonfinite, step]
 * M_C = sum C/C_inf (Eq. 5 inverted); H = sum [(rho Cp)_eff T - rho_L L_h phi/2].
 * S_phi and J_U are maxima since the previous call (then reset). */
void orc_diag(orc_sim* s, double* out) {
    const orc_params* p = &s->p;
    double MC = 0.0, H = 0.0;
    int bad = 0;
    for (int n = 0; n < s->nn; ++n) {
        double ph = s->phi[n];
        if (p->has_U) MC += 0.5 * (1.0 + (1.0 - p->k) * s->U[n]) * ((1.0 + p->k) - (1.0 - p->k) * ph);
        if (p->has_T) H += rhoCp_eff(p, ph) * s->T[n] - 0.5 * p->rhoL_Lh * ph;
        double vals[5] = {ph, s->U[n], s->T[n], s->ux[n], s->uy[n]};
        for (int k = 0; k < 5; ++k) if (!isfinite(vals[k])) bad = 1;
    }
    out[0] = MC;
    out[1] = H;
    out[2] = s->S_phi;
    out[3] = s->J_U;
    for (int d = 0; d < 4; ++d) out[4 + d] = tip_dist(s, d);
    out[8] = bad;
    out[9] = (double)s->step;
    s->S_phi = 0.0;
    s->J_U = 0.0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
