/*
 * lbm.h -- C ABI of the B300 multirate MRT lattice Boltzmann library for
 * thermosolutal dendritic solidification (Liu, Wu, Zhan: "A unified multirate
 * lattice Boltzmann framework for thermosolutal dendritic solidification").
 *
 * The library advances, on one CUDA device, the four coupled D2Q9 distribution
 * sets of the paper -- phase phi, supersaturation U, temperature T and flow F
 * (Sec. 3.1, Eq. 15) -- each at its own update factor N_chi (Eq. 34), with the
 * phase-step transfer of solute rejection and latent heat (Eqs. 36-39).
 *
 * Conventions for every entry point:
 *   - All functions return an lbm_status; none aborts, traps or exits.  After
 *     an error, lbm_last_error(h) returns a one-line description.
 *   - Fields are row-major ny x nx (x fastest), node (x, y) at y*nx + x, in
 *     lattice units (dx = 1).
 *   - The caller owns every pointer it passes (params, seeds, field buffers);
 *     the library copies what it keeps.  The library owns the device state it
 *     allocates (through the lbm_allocator if given, else cudaMalloc).
 *   - Work is queued on the CUDA stream given to lbm_create; calls that return
 *     data to the host (lbm_fields with host dst, lbm_diagnostics) synchronise
 *     that stream.  One handle must not be used from two threads at once.
 *   - Status codes are sticky for LBM_E_NONFINITE: once a diagnostics call has
 *     seen a non-finite value (the failure mode of the paper's accumulated
 *     coupling, Sec. 4.4), lbm_advance refuses with LBM_E_STATE until the
 *     simulation is initialised again.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_PARAMS_VERSION 3u

typedef enum {
    LBM_OK = 0,
    LBM_E_INVALID_ARG = 1,     /* null pointer, bad size, bad enum value          */
    LBM_E_UNSTABLE_PARAMS = 2, /* a relaxation time <= 1/2 (Eqs. 24, 32) etc.     */
    LBM_E_OOM = 3,             /* device allocation failed                         */
    LBM_E_CUDA = 4,            /* a CUDA runtime call failed                       */
    LBM_E_NONFINITE = 5,       /* a macroscopic field holds NaN or Inf             */
    LBM_E_TIMEOUT = 6,         /* a bounded device wait ran out                    */
    LBM_E_STATE = 7            /* call out of order (not initialised, sticky error)*/
} lbm_status;

/* boundary kinds (Sec. 4: zero-flux walls for phi, U, T; periodic or
 * inlet/outflow for the flow) */
enum { LBM_BC_PERIODIC = 0, LBM_BC_WALL = 1, LBM_BC_INLET_OUTFLOW = 2 };

/* lbm_params.fields: phi is always present */
enum {
    LBM_FIELD_U = 1u,        /* solute, Eq. 6                                      */
    LBM_FIELD_T = 2u,        /* temperature, Eq. 10                                */
    LBM_FIELD_FROZEN_T = 4u, /* prescribed theta(y,t) = theta_c + G (y - y0 - V t) */
    LBM_FIELD_FLOW = 8u      /* D2Q9 flow, Eqs. 13, 27-33                          */
};

/* lbm_params.precision: storage of the distributions / arithmetic.  The
 * stored state of a field is: phase and flow, populations 1..8 (population 0
 * follows from the macro); U and T, the first moment (j_x, j_y) of the
 * streamed populations -- with the relaxation matrix of Eq. 23 every other
 * moment of a scalar collision relaxes to equilibrium at rate one, so the
 * macro and j determine the post-collision populations exactly. */
enum {
    LBM_PREC_F64 = 0,      /* FP64 storage and arithmetic                          */
    LBM_PREC_F32 = 1,      /* FP32 storage and arithmetic                          */
    LBM_PREC_F16_DEV = 2,  /* FP16 storage, FP32 arithmetic: phase f_i - w_i phi,
                              flow f_i - w_i rho, U/T j as is                      */
    LBM_PREC_BF16_DEV = 3  /* BF16 storage of the same quantities, FP32 arithmetic */
};

/* lbm_params.coupling (Sec. 4.4 source-coupling ablation) */
enum { LBM_COUPLING_INSTANTANEOUS = 0, LBM_COUPLING_ACCUMULATED = 1 };

/* Inputs of one simulation.  Symbols follow the paper:
 *   Eq. 34:   dt_chi = N_chi dt_base
 *   Eqs. 1-4: W0, tau0, eps (eps_s), lam (lambda)
 *   Eqs. 5-9: Mc, k (k_c), DL, DS
 *   Eqs. 10-12: kappaS, kappaL, rhoCpS, rhoCpL (volumetric heat capacities),
 *             rhoL_Lh (rho_L L_h); theta = (T - T_shift)/T_scale (Eq. 5)
 *   Eqs. 27-33: nu, u_in (inlet velocity), Fbx, Fby (body force), s_e, s_eps, s_q
 *   frozen temperature: theta = theta_c + frozen_G (y - frozen_y0 - frozen_V t);
 *             with neither T nor FROZEN_T, theta = theta_c.
 *   tip_cx, tip_cy: node through which lbm_diagnostics measures the tips.
 *   T_ymin_dirichlet, T_ymin: with T on and bc_scalar_y = WALL, the bottom
 *             wall holds T = T_ymin (Sec. 4.4, the cold bottom boundary kept at
 *             T_b) instead of zero flux, by anti-bounce-back at the half-way
 *             wall; phi and U keep zero flux there.
 *   q_scalar: velocities of the phi, U and T lattices.  0 or 9: D2Q9, the
 *             paper's lattice for all four fields (Sec. 3.1, Eq. 15).  5:
 *             D2Q5, the rest velocity and the four axis links of Eq. 15 with
 *             weights 1/3, 1/6 (c_s^2 = 1/3, so Eq. 24 is unchanged),
 *             moments (1, e_x, e_y, 5|e|^2 - 4, e_x^2 - e_y^2) and every
 *             moment but the two fluxes relaxed at rate one, as Eq. 23 does
 *             on D2Q9; the phase field then stores 4 population planes
 *             instead of 8.  The flow stays D2Q9.  All members of an
 *             ensemble share it (version 3). */
typedef struct {
    uint32_t struct_version; /* = LBM_PARAMS_VERSION */
    int32_t nx, ny;          /* lattice size, >= 4 each */
    uint32_t fields;         /* LBM_FIELD_* bits */
    int32_t bc_scalar_x, bc_scalar_y; /* PERIODIC or WALL, for phi, U, T */
    int32_t bc_flow_x, bc_flow_y;     /* PERIODIC, WALL or (x only) INLET_OUTFLOW */
    uint32_t precision;      /* LBM_PREC_* */
    uint32_t coupling;       /* LBM_COUPLING_* */
    int32_t N_phi, N_U, N_T, N_F; /* update factors, >= 1 */
    int32_t tip_cx, tip_cy;
    int32_t T_ymin_dirichlet;    /* 1: T = T_ymin on the bottom wall (version 2) */
    int32_t q_scalar;            /* 0 / 9: D2Q9 scalar lattices; 5: D2Q5 (version 3) */
    double dt_base;
    double W0, tau0, eps, lam;
    double Mc, k, DL, DS;
    double kappaS, kappaL, rhoCpS, rhoCpL, rhoL_Lh, T_shift, T_scale;
    double nu, u_in, Fbx, Fby, s_e, s_eps, s_q;
    double theta_c, frozen_G, frozen_y0, frozen_V;
    double T_ymin;               /* bottom-wall temperature (version 2) */
} lbm_params;

/* Initial-condition primitives for lbm_init_seed. phi is the maximum over all
 * seeds of their profiles:
 *   CIRCLE:   tanh[(r - |x - (x, y)|)/(sqrt 2 W0)]                 (Sec. 4.1)
 *   PLANAR:   tanh[(y - y_node)/(sqrt 2 W0)] plus noise amp*(2u - 1) on nodes
 *             with |phi| < 0.99, clipped to [-1, 1]; u is the draw of node
 *             n = y*nx + x from SplitMix64 seeded with rng_seed
 *   SINUSOID: tanh[(y + amp sin(2 pi waves x / nx) - y_node)/(sqrt 2 W0)] (Eq. 41) */
enum { LBM_SEED_CIRCLE = 0, LBM_SEED_PLANAR = 1, LBM_SEED_SINUSOID = 2 };
typedef struct {
    int32_t kind;
    int32_t reserved;
    double x, y, r, amp, waves;
} lbm_seed;

/* Diagnostics of one simulation (Sec. 4.1 tip histories, Sec. 4.4 ablation).
 *   M_C     = sum over nodes of C/C_inf = (1 + (1-k) U)((1+k) - (1-k) phi)/2 (Eq. 5), FP64 sum
 *             (FP32 states: each node's term and each thread's partial sum as a
 *             pair of FP32 numbers, ~2^-46 relative; the totals FP64)
 *   H_total = sum of (rho Cp)_eff(phi) T - rho_L L_h phi / 2, FP64 sum (FP32
 *             states: the per-thread partial sums as pairs of FP32 numbers)
 *   S_phi   = max |Delta U_pc| over nodes and phase steps since the previous call
 *   J_U     = max |U_post - U_pre| over the phase-change applications since the
 *             previous call (equals S_phi under instantaneous coupling)
 *   tip[d]  = distance from (tip_cx, tip_cy) of the outermost phi = 0 crossing
 *             along +x, +y, -x, -y (linear interpolation)
 *   nonfinite = 1 if any phi, U, T, ux, uy is NaN or Inf
 *   R_M     = relative solute drift (M_C - M_C(0)) / M_C(0) since the last
 *             lbm_init_seed / lbm_init_fields (Sec. 4.4); 0 from
 *             lbm_diagnostics_noalloc, which keeps no history */
typedef struct {
    int64_t base_step;
    double M_C, H_total, S_phi, J_U;
    double tip[4];
    int32_t nonfinite;
    int32_t reserved;
    double R_M;       /* (M_C - M_C(0)) / M_C(0), M_C(0) of the last initialisation (Sec. 4.4) */
} lbm_diag;

/* Optional device allocator (e.g. a framework's caching allocator).  alloc
 * returns device memory of at least `bytes` usable on `stream`, or NULL;
 * free releases it.  Both may be called from lbm_create / lbm_destroy only. */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* ptr, size_t bytes, void* stream, void* ctx);
    void* ctx;
} lbm_allocator;

typedef struct lbm_sim* lbm_handle;

/* Create n_sims independent simulations on the current CUDA device.
 * p: parameters of every simulation when per_sim is NULL; otherwise per_sim
 * holds n_sims parameter sets and p only selects precision (all members must
 * share it).  a: NULL for cudaMalloc.  cuda_stream: a cudaStream_t (NULL =
 * legacy default stream).  Validates every field (versions, sizes >= 4,
 * N_chi >= 1, tau_chi > 1/2 in both phases, nonzero denominators).
 * Errors: INVALID_ARG, UNSTABLE_PARAMS, OOM, CUDA.  On error *out = NULL. */
lbm_status lbm_create(const lbm_params* p, int32_t n_sims, const lbm_params* per_sim,
                      const lbm_allocator* a, void* cuda_stream, lbm_handle* out);

/* Initialise simulation `sim` from seed primitives (generated on the device,
 * FP64 arithmetic per node, then stored in the arithmetic type): phi from
 * the seeds (the largest of their profiles), U = U0, T = T0, rho = 1,
 * u = u_in (1 - phi)/2 along x when the flow is on; then every distribution
 * is set to the equilibrium of these fields (for phi with v_n from the
 * initial gradient, Eqs. 19, 21, 28).  Resets the base-step clock and the
 * sticky error.  Returns once the seed list has been read (the caller may
 * reuse it); the generation and initialisation kernels run on, ordered on
 * the stream before any later call's work. */
lbm_status lbm_init_seed(lbm_handle h, int32_t sim, const lbm_seed* seeds, int32_t n_seeds,
                         double U0, double T0, uint64_t rng_seed);

/* Initialise simulation `sim` from caller fields, each ny x nx FP64: phi, U,
 * T, ux, uy, rho (U / T / ux, uy, rho are ignored when that field is off, and
 * may then be NULL).  src_is_device: 1 if the pointers are device memory.
 * Then as lbm_init_seed.  Returns once the source buffers have been read (the
 * caller may then reuse or free them); the conversion and initialisation run
 * on, ordered on the stream before any later call's work. */
lbm_status lbm_init_fields(lbm_handle h, int32_t sim, const double* phi, const double* U,
                           const double* T, const double* ux, const double* uy,
                           const double* rho, int32_t src_is_device);

/* Advance every simulation by n_base_steps ticks of the global clock (Eq. 34;
 * field chi updates at base step n iff (n+1) mod N_chi == 0, in the order
 * phase -> transfer -> U -> T -> flow of Fig. 1).  Asynchronous: returns once
 * the work is queued (as captured CUDA graphs of one schedule period when
 * graphs are enabled).  Errors: STATE (not initialised / sticky), CUDA. */
lbm_status lbm_advance(lbm_handle h, int64_t n_base_steps);

/* Copy a macroscopic field of simulation `sim` into dst (ny x nx).
 * which: 0 phi, 1 U, 2 T, 3 ux, 4 uy, 5 rho, 6 C/C_inf, 7 theta.
 * as_f64 = 1: dst holds doubles; 0: dst holds the arithmetic type (double for
 * F64, float otherwise).  dst_is_device: 1 for a device pointer (copy queued
 * on the stream), 0 for host memory (synchronises).  Fields that are off read
 * as zeros (U, T), theta_c-based theta, or rest (ux, uy = 0, rho = 1). */
lbm_status lbm_fields(lbm_handle h, int32_t sim, uint32_t which, void* dst, int32_t dst_is_device,
                      int32_t as_f64);

/* Reduce the diagnostics of simulation `sim` on the device (FP64 totals,
 * deterministic order) and return them; resets the S_phi / J_U maxima.
 * Synchronises the stream.  Returns NONFINITE (and sets the sticky state)
 * when a non-finite value is present; *out is filled in either case. */
lbm_status lbm_diagnostics(lbm_handle h, int32_t sim, lbm_diag* out);

/* One-line description of the last error on h (or of the last failed
 * lbm_create when h is NULL).  Owned by the library; valid until the next call. */
const char* lbm_last_error(lbm_handle h);

/* Free every device buffer and graph of h.  NULL is a no-op. */
void lbm_destroy(lbm_handle h);

/* ---- runtime controls and measurement hooks (no counterpart in the paper) ---- */

/* enable = 1 (default): lbm_advance replays CUDA graphs captured per schedule
 * period; 0: plain stream launches.  Results are identical. */
lbm_status lbm_set_graphs(lbm_handle h, int32_t enable);

/* Batched ensemble (default on when n_sims >= 2): while the members are in
 * lockstep, each base step runs one launch per kernel kind whose blocks cover
 * the tiles of every member that updates that field in that step (members keep
 * their own parameters, sizes and update factors); the launches of one common
 * schedule period are one CUDA graph.  enable = 0 advances the members one
 * after another with their own graphs (the results are identical).
 * Errors: INVALID_ARG (fewer than two members, or a common period over 4096
 * base steps). */
lbm_status lbm_set_batching(lbm_handle h, int32_t enable);

/* enable = 1: under instantaneous coupling, everything a base step does
 * after the phase update -- the phase-change transfer (Eqs. 36-39) and the
 * scheduled U, T and flow updates -- runs as one fused launch per base step
 * (LBM_K_TRANSPORT) that recomputes the transfer on the halo it needs instead
 * of storing the injected U, T.  0: one launch per stage (the default until
 * lbm_autotune has timed both).  The two agree to floating-point contraction
 * rounding.  An explicit call fixes the choice: lbm_autotune no longer
 * changes it.  Recaptures graphs. */
lbm_status lbm_set_fusion(lbm_handle h, int32_t enable);

/* *enabled receives 1 when base steps run the fused transport launch. */
lbm_status lbm_get_fusion(lbm_handle h, int32_t* enabled);

/* Grain orientation of simulation `sim` (the multi-dendrite case draws a
 * crystal angle per seed; Eq. 2 is written for crystal axes along x and y).
 * theta: ny x nx FP64, the angle of the crystal axes of the grain each node
 * belongs to; Eqs. 2-3 are then evaluated on the phase gradient turned into
 * that frame, g' = R(-theta) g, and N is turned back, N = R(theta) N'.
 * NULL restores the axis-aligned Eq. 2 of the paper (the default).
 * src_is_device: 1 if theta is device memory.  The field is kept (in the
 * arithmetic type, allocated on first use through the handle's allocator)
 * until replaced; it applies from the next update, and to the initial phase
 * equilibria of a later lbm_init_seed / lbm_init_fields, so set it before
 * them.  Synchronises the stream.  Errors: INVALID_ARG, OOM, CUDA. */
lbm_status lbm_set_orientation(lbm_handle h, int32_t sim, const double* theta, int32_t src_is_device);

/* Kernel kinds for timing and launch counts. */
enum { LBM_K_PHASE = 0, LBM_K_TRANSFER = 1, LBM_K_SCALAR_U = 2, LBM_K_SCALAR_T = 3,
       LBM_K_FLOW = 4, LBM_K_DIAG = 5, LBM_K_INIT = 6,
       LBM_K_TRANSPORT = 7,   /* fused transfer + U + T + flow of one base step */
       LBM_K_COUNT = 8 };

/* Time every launch of the kernel kinds in kind_mask (bit k = kind k) with
 * CUDA events on the library's stream, inside graphs as event-record nodes
 * that each replay points at fresh events.  No host wait is added to
 * lbm_advance: the times are read by lbm_timing_read and lbm_diagnostics
 * (which synchronise the stream), or when more than 4096 timed launches are
 * queued.  kind_mask = 0 turns timing off.  Recaptures graphs. */
lbm_status lbm_timing_enable(lbm_handle h, uint32_t kind_mask);

/* Per kind: accumulated milliseconds and number of timed launches since the
 * last reset; reset = 1 clears them. ms and count hold LBM_K_COUNT entries. */
lbm_status lbm_timing_read(lbm_handle h, double* ms, int64_t* count, int32_t reset);

/* Autotuner: for every update kernel kind of every simulation, time each
 * compiled tile shape (32 x 4, 32 x 8, 32 x 16 threads) over `reps` launches on
 * the current state and keep the fastest.  The update kernels read one
 * ping-pong buffer and write the other, so the repeated launches leave the
 * simulation unchanged (the S_phi / J_U maxima are cleared).  Unless
 * lbm_set_fusion was called, it also times one half schedule period both as
 * fused transport launches and as one launch per stage (from the per-launch
 * times, each transport stage combination the schedule uses timed once) and
 * keeps the faster.  chosen (nullable) receives LBM_K_COUNT tile heights of
 * simulation 0.  Recaptures graphs.
 * Errors: STATE (not initialised), CUDA. */
lbm_status lbm_autotune(lbm_handle h, int32_t reps, int32_t* chosen);

/* Fix the tile height (4, 8 or 16 rows of 32 nodes) of one update kernel kind
 * (LBM_K_PHASE .. LBM_K_FLOW) for every simulation and for the batched
 * launches.  Different tile shapes are different compilations of the same
 * arithmetic and agree to floating-point contraction rounding; a fixed
 * choice makes runs bitwise reproducible.  Recaptures graphs.
 * Errors: INVALID_ARG. */
lbm_status lbm_set_tile(lbm_handle h, int32_t kind, int32_t ty);

/* Number of kernel launches the library has issued (graph replays count
 * their kernel nodes), per kind; counts hold LBM_K_COUNT entries. */
lbm_status lbm_launch_counts(lbm_handle h, int64_t* counts);

/* Bytes of device memory held by h. */
lbm_status lbm_device_bytes(lbm_handle h, size_t* bytes);

/* Diagnostics of caller-held fields, allocating nothing.  The paper has no
 * counterpart: this is a service for callers that cannot call cudaMalloc --
 * e.g. a monitoring hook inside another framework's step loop, where an
 * allocation would synchronise the device and break that framework's stream
 * ordering, or a process whose device memory is owned by a caching allocator
 * under a fixed budget.  It reduces the same quantities as lbm_diagnostics
 * (M_C, H_total, tips, nonfinite; S_phi = J_U = 0 and base_step = 0, since it
 * keeps no history) over fields the caller passes, without a handle.
 *   p:      parameters of the fields (nx, ny, fields bits, k, heat
 *           capacities, rhoL_Lh, tip_cx / tip_cy are used; validated as in
 *           lbm_create); p->precision selects the element type: double for
 *           LBM_PREC_F64, float otherwise.
 *   phi, U, T, ux, uy: device pointers, dense ny x nx row-major in that type
 *           (as lbm_fields writes them with as_f64 = 0); U / T / ux, uy may be
 *           NULL when that field is off.
 *   cuda_stream: stream the reduction runs on (NULL = legacy default);
 *           the call synchronises it.   out: host struct, filled on return.
 * Scratch: a fixed file-scope device array of about 28 KB (partial sums of at
 * most 1184 blocks plus result slots), held by every GPU that loads the
 * library until the process exits.  Lattices of more than 2^31 - 1 nodes are
 * rejected with LBM_E_INVALID_ARG.  Every call looks up the array's device
 * address (cudaGetSymbolAddress) with the current device.  The call
 * synchronises its stream and copies the results to the host, so it may
 * never run while a capture into a CUDA graph is active: on a capturing
 * stream it returns LBM_E_INVALID_ARG; in the global capture mode it would
 * also invalidate captures on other streams, so do not call it then.  Calls
 * share the array and it keeps the last call's contents: calls that overlap
 * on the GPU race.  With FP32 arithmetic lbm_diagnostics adds the residual of
 * the compensated U macro to the solute sum, which the caller's FP32 U field
 * does not hold: the two M_C agree to the rounding of U to FP32.
 * Errors: INVALID_ARG, UNSTABLE_PARAMS (as lbm_create), CUDA, NONFINITE
 * (out is filled).  Errors are reported by lbm_last_error(NULL). */
lbm_status lbm_diagnostics_noalloc(const lbm_params* p, const void* phi, const void* U, const void* T,
                                   const void* ux, const void* uy, void* cuda_stream, lbm_diag* out);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
