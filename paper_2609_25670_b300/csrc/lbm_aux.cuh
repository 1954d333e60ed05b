// Auxiliary kernels: initial distributions, FP64 staging, output fields,
// diagnostics reductions, the base-step clock.
#pragma once
#include "lbm_common.cuh"

namespace lbmk {

// ---------------------------------------------------------------------------
// Initial distributions f = f_eq of the macroscopic fields (Eqs. 19, 21, 28);
// for U and T their first moments, the stored state of those fields.  Q: the
// velocities of the phase lattice (9, or 5 for D2Q5: populations 1..4 only).
// seeded: the fields come from seed primitives, so U = U0, T = T0, u_y = 0
// and rho = 1 on every node and only phi and u_x are read.  (The kernel is
// bound by instruction issue: interior nodes read their 3 x 3 neighbourhood
// at fixed offsets, and only the lattice's edge nodes map ghosts; eight
// blocks of 256 threads stay resident, as with one ghost map per neighbour.)
// ---------------------------------------------------------------------------
template <typename R, typename ST, bool DEV, int Q>
__global__ void __launch_bounds__(256, 8) k_init(const KP<R> P, const R* __restrict__ phi, const R* __restrict__ Um,
                       const R* __restrict__ Tm, const R* __restrict__ uxm, const R* __restrict__ uym,
                       const R* __restrict__ rhom, ST* __restrict__ fphi, ST* __restrict__ fU, ST* __restrict__ fT,
                       ST* __restrict__ fF, int seeded, R U0, R T0) {
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (gx >= P.nx || gy >= P.ny) return;
    const size_t node = (size_t)gy * P.pitch + gx;
    // gradient with the same ghost rule as the update kernels
    R s[3][3];
    if (gx > 0 && gx < P.nx - 1 && gy > 0 && gy < P.ny - 1) {
        const R* c = phi + node;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) s[dy + 1][dx + 1] = c[(ptrdiff_t)dy * P.pitch + dx];
    } else {
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx)
                s[dy + 1][dx + 1] =
                    phi[(size_t)scalar_map(gy + dy, P.ny, P.bsy) * P.pitch + scalar_map(gx + dx, P.nx, P.bsx)];
    }
    const R gxv = (s[1][2] - s[1][0]) * (R(1) / R(3)) + (s[2][2] - s[2][0] + s[0][2] - s[0][0]) * (R(1) / R(12));
    const R gyv = (s[2][1] - s[0][1]) * (R(1) / R(3)) + (s[2][2] + s[2][0] - s[0][2] - s[0][0]) * (R(1) / R(12));
    R as, Nx, Ny;
    if (P.ori) aniso_frame(gxv, gyv, P.eps, P.ori[node], as, Nx, Ny);     // grain frame
    else aniso(gxv, gyv, P.eps, as, Nx, Ny);
    const R bx = -P.dtp * P.W0sq_tau0 * Nx, by = -P.dtp * P.W0sq_tau0 * Ny;
    const R ph = s[1][1];
    R vx = R(0), vy = R(0), rho = R(1);
    if (P.has_flow) {
        vx = uxm[node];
        if (!seeded) { vy = uym[node]; rho = rhom[node]; }
    }
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const R w = Q == 5 ? wqq<R, 5>(i) : wq<R>(i), ex = (R)c_ex[i], ey = (R)c_ey[i];
        const R dp = R(3) * w * (ex * bx + ey * by);                                   // Eq. 21 minus w_i phi
        fphi[(size_t)(i - 1) * P.plane + node] = Cvt<ST>::st(DEV ? dp : w * ph + dp);
    }
    // U, T: the first moment of f_eq of Eq. 19, sum_i e_i 3 w_i chi dt (e_i . u)
    // = dt chi u (sum_i w_i e_i e_i = I / 3 on D2Q9 and on D2Q5)
    if (P.has_U) {
        const R U = seeded ? U0 : Um[node];
        fU[node] = Cvt<ST>::st(P.dtU * U * vx);
        fU[(size_t)P.plane + node] = Cvt<ST>::st(P.dtU * U * vy);
        if constexpr (Compensated<R>::value) {          // residual of the compensated macro
            using Lo = typename LoOf<ST>::T;
            reinterpret_cast<Lo*>(fU + 2 * (size_t)P.plane)[node] = Cvt<Lo>::st(R(0));
        }
    }
    if (P.has_T) {
        const R T = seeded ? T0 : Tm[node];
        fT[node] = Cvt<ST>::st(P.dtT * T * vx);
        fT[(size_t)P.plane + node] = Cvt<ST>::st(P.dtT * T * vy);
    }
    if (P.has_flow) {
        R fe[9];
        feq_flow<R>(rho, vx, vy, P.cF, fe);                                                // Eq. 28
#pragma unroll
        for (int i = 1; i < 9; ++i)
            fF[(size_t)(i - 1) * P.plane + node] = Cvt<ST>::st(DEV ? fe[i] - wq<R>(i) * rho : fe[i]);
    }
}

// Initial fields from seed primitives, FP64 arithmetic per node: phi is the
// largest of the seeds' tanh profiles (-1 where none reaches; a circle
// reaches the box of r + 20 sqrt(2) W0 + 2 nodes around its centre, beyond
// which tanh rounds to -1), a planar front with amp > 0 adds uniform noise of
// amplitude amp in its diffuse layer (|phi| < 0.99) from a counter-based
// SplitMix64 draw per node; U = U0, T = T0, rho = 1, u_y = 0 and
// u_x = u_in (1 - phi) / 2 when the flow is on.
struct SeedDev {
    int kind;                      // 0 circle, 1 planar, 2 sinusoid
    int xa, xb, ya, yb;            // a circle's reach: the nodes [xa, xb) x [ya, yb)
    double x, y, r, amp, waves;
};
__host__ __device__ inline unsigned long long splitmix64(unsigned long long seed, unsigned long long k) {
    unsigned long long z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;    // SplitMix64 (Steele, Lea, Flood 2014)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// a seed-field block: SEED_BX x SEED_BY threads over SEED_BX columns and
// SEED_BY * SEED_ROWS rows
constexpr int SEED_BX = 32, SEED_BY = 8, SEED_ROWS = 8;
constexpr int SEED_BH = SEED_BY * SEED_ROWS;

// The values of a node that no seed reaches, on every node: phi = -1, U = U0,
// T = T0, u_x = u_in (the FP64 profile at phi = -1, rounded on the host),
// u_y = 0, rho = 1.  k_seed_fields then rewrites the blocks that seeds
// reach.  (The FP64 profile code sizes that kernel's registers, three blocks
// per SM, which would leave this store stream at half the bandwidth.)
template <typename R>
__global__ void __launch_bounds__(SEED_BX * SEED_BY)
k_seed_fill(int nx, int ny, int pitch, R U0, R T0, R ux_liquid, R* __restrict__ phi, R* __restrict__ U,
            R* __restrict__ T, R* __restrict__ ux, R* __restrict__ uy, R* __restrict__ rho) {
    const int x = blockIdx.x * SEED_BX + threadIdx.x;
    if (x >= nx) return;
#pragma unroll
    for (int g = 0; g < SEED_ROWS; ++g) {
        const int y = blockIdx.y * SEED_BH + g * SEED_BY + threadIdx.y;
        if (y >= ny) break;
        const size_t o = (size_t)y * pitch + x;
        phi[o] = R(-1);
        if (U) U[o] = U0;
        if (T) T[o] = T0;
        if (ux) { ux[o] = ux_liquid; uy[o] = R(0); rho[o] = R(1); }
    }
}

// blocks: the block indices (by * nbx + bx) to run, one per CUDA block, or
// null for the whole grid (blockIdx.x, blockIdx.y).  A block first lists the
// seeds that can reach its region (64 at a time).
template <typename R>
__global__ void __launch_bounds__(SEED_BX * SEED_BY)
k_seed_fields(int nx, int ny, int pitch, const SeedDev* __restrict__ seeds, int n_seeds,
              const int* __restrict__ blocks, int nbx, double sw, unsigned long long rng_seed, double U0, double T0,
              double u_in, R* __restrict__ phi, R* __restrict__ U, R* __restrict__ T, R* __restrict__ ux,
              R* __restrict__ uy, R* __restrict__ rho) {
    __shared__ int list[64];
    __shared__ int cnt;
    int bxi = blockIdx.x, byi = blockIdx.y;
    if (blocks) { const int b = blocks[blockIdx.x]; bxi = b % nbx; byi = b / nbx; }
    const int x = bxi * SEED_BX + threadIdx.x;
    const int t = threadIdx.y * SEED_BX + threadIdx.x;
    const int bx0 = bxi * SEED_BX, by0 = byi * SEED_BH;
    const int bx1 = bx0 + SEED_BX, by1 = by0 + SEED_BH;
    double p[SEED_ROWS];
#pragma unroll
    for (int g = 0; g < SEED_ROWS; ++g) p[g] = -1.0;
    for (int base = 0; base < n_seeds; base += 64) {
        if (t == 0) cnt = 0;
        __syncthreads();
        if (t < 64 && base + t < n_seeds) {
            const SeedDev& q = seeds[base + t];
            if (q.kind != 0 || (q.xa < bx1 && q.xb > bx0 && q.ya < by1 && q.yb > by0)) list[atomicAdd(&cnt, 1)] = base + t;
        }
        __syncthreads();
        const int c = cnt;
        for (int j = 0; x < nx && j < c; ++j) {   // the largest profile: the order of the list does not matter
            const SeedDev sd = seeds[list[j]];
#pragma unroll
            for (int g = 0; g < SEED_ROWS; ++g) {
                const int y = by0 + g * SEED_BY + threadIdx.y;
                if (y >= ny) break;
                double v;
                if (sd.kind == 0) {
                    if (x < sd.xa || x >= sd.xb || y < sd.ya || y >= sd.yb) continue;
                    const double dx = x - sd.x, dy = y - sd.y;
                    v = tanh((sd.r - sqrt(dx * dx + dy * dy)) / sw);
                } else if (sd.kind == 1) {
                    v = tanh((sd.y - y) / sw);
                    if (sd.amp > 0.0 && fabs(v) < 0.99) {
                        const double u = (double)(splitmix64(rng_seed, (size_t)y * nx + x) >> 11) * 0x1.0p-53;
                        v = fmin(1.0, fmax(-1.0, v + sd.amp * (2.0 * u - 1.0)));
                    }
                } else {
                    const double pi = 3.14159265358979323846;
                    v = tanh((sd.y + sd.amp * sin(2.0 * pi * sd.waves * x / nx) - y) / sw);
                }
                p[g] = fmax(p[g], v);
            }
        }
        __syncthreads();                          // before the list is refilled
    }
    if (x >= nx) return;
#pragma unroll
    for (int g = 0; g < SEED_ROWS; ++g) {
        const int y = by0 + g * SEED_BY + threadIdx.y;
        if (y >= ny) break;
        const size_t o = (size_t)y * pitch + x;
        phi[o] = (R)p[g];
        if (U) U[o] = (R)U0;
        if (T) T[o] = (R)T0;
        if (ux) {
            ux[o] = (R)(u_in * 0.5 * (1.0 - p[g]));
            uy[o] = R(0);
            rho[o] = R(1);
        }
    }
}

// FP64 staging -> arithmetic type, with a pitch
template <typename R>
__global__ void k_from_f64(const double* __restrict__ src, R* __restrict__ dst, int nx, int ny, int pitch) {
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (gx < nx && gy < ny) dst[(size_t)gy * pitch + gx] = (R)src[(size_t)gy * nx + gx];
}

// derived output fields into a dense ny x nx buffer of type O
// which: 0 phi 1 U 2 T 3 ux 4 uy 5 rho 6 C/C_inf 7 theta.  ulo: the residual
// plane of the compensated U macro (lo_kind 1: float, 2: BF16; 0: none),
// added to U in U and C/C_inf.  A block of blockDim.x x blockDim.y threads
// covers OUT_ROWS groups of blockDim.y rows: with one node per thread the
// launch of a one-load, one-store copy ran at the rate blocks are started.
constexpr int OUT_ROWS = 8;
template <typename R, typename O>
__global__ void k_out(const KP<R> P, int which, const R* __restrict__ phi, const R* __restrict__ Um,
                      const R* __restrict__ Tm, const R* __restrict__ uxm, const R* __restrict__ uym,
                      const R* __restrict__ rhom, const void* __restrict__ ulo, int lo_kind,
                      O* __restrict__ dst, const long long* __restrict__ clock) {
    const int gx = blockIdx.x * blockDim.x + threadIdx.x;
    if (gx >= P.nx) return;
    // every row's value first, then the stores: the loads of the OUT_ROWS rows
    // are in flight together
    O vals[OUT_ROWS];
#pragma unroll
    for (int g = 0; g < OUT_ROWS; ++g) {
        const int gy = (blockIdx.y * OUT_ROWS + g) * blockDim.y + threadIdx.y;
        vals[g] = O(0);
        if (gy >= P.ny) continue;
        const size_t node = (size_t)gy * P.pitch + gx;
        auto u_total = [&]() -> O {     // U and the residual of its compensated macro (read only when asked for)
            O Uo = (O)(P.has_U ? Um[node] : R(0));
            if (P.has_U && lo_kind == 1) Uo += (O)static_cast<const float*>(ulo)[node];
            if (P.has_U && lo_kind == 2) Uo += (O)__bfloat162float(static_cast<const __nv_bfloat16*>(ulo)[node]);
            return Uo;
        };
        switch (which) {
            case 0: vals[g] = (O)phi[node]; break;
            case 1: vals[g] = u_total(); break;
            case 2: vals[g] = (O)(P.has_T ? Tm[node] : R(0)); break;
            case 3: vals[g] = (O)(P.has_flow ? uxm[node] : R(0)); break;
            case 4: vals[g] = (O)(P.has_flow ? uym[node] : R(0)); break;
            case 5: vals[g] = (O)(P.has_flow ? rhom[node] : R(1)); break;
            case 6: {
                const O Uo = u_total();
                vals[g] = O(0.5) * (O(1) + (O(1) - (O)P.k) * Uo) * ((O(1) + (O)P.k) - (O(1) - (O)P.k) * (O)phi[node]);
                break;
            }
            case 7: {
                R v;
                if (P.has_T) v = (Tm[node] - P.T_shift) * P.inv_T_scale;
                else if (P.frozen_T) v = theta_frozen(P, gy, (R)(*clock) * P.dt_base);
                else v = P.theta_c;
                vals[g] = (O)v;
                break;
            }
        }
    }
#pragma unroll
    for (int g = 0; g < OUT_ROWS; ++g) {
        const int gy = (blockIdx.y * OUT_ROWS + g) * blockDim.y + threadIdx.y;
        if (gy < P.ny) dst[(size_t)gy * P.nx + gx] = vals[g];
    }
}

// ---------------------------------------------------------------------------
// Diagnostics: deterministic FP64 reductions (warp shuffle -> block -> grid)
// ---------------------------------------------------------------------------
// part[b*3 + 0] = sum C/C_inf, [1] = sum H, [2] = non-finite count, for block b
// Ulo: the residual plane of the compensated U macro (type Lo, pitch layout),
// added to U in the solute sum, or null.  Block b sums rows b, b + gridDim.x,
// ... (threads across each row), so the order is fixed for a given lattice.
// FP64 arithmetic is a small fraction of the FP32 rate on this GPU: with an
// FP32 state the solute term (the conservation diagnostic, Eq. 39) is formed
// from the stored macro values in double-float arithmetic (a value held as
// the unevaluated sum of two FP32 numbers: Dekker's product via a fused
// multiply-add, Knuth's TwoSum; about 2^-46 relative per term) and summed
// per thread the same way, the residual plane's part (~1e-8 of the rest) in
// FP32; the enthalpy term is formed in FP32 and summed in double-float; the
// non-finite test runs on the stored values.  Each thread's sums become FP64
// once, and the warp, block and grid sums are FP64.  An FP64 state takes FP64
// throughout.
struct DFloat { float h, l; };                 // h + l, |l| <= ulp(h) / 2 after renormalising
__device__ __forceinline__ void df_add(DFloat& s, float h, float l) {
    float t, e;
    two_sum(s.h, h, t, e);
    s.h = t;
    s.l = add_rn(s.l, add_rn(e, l));
}
// a b + c as (hi, lo): hi = fl(a b), lo = c + (a b - hi) rounded once
__device__ __forceinline__ void df_mul(float a, float b, float& hi, float& lo) {
    hi = __fmul_rn(a, b);
    lo = __fmaf_rn(a, b, -hi);
}
// solute_only: the solute sum alone (T, u_x, u_y are not read; the enthalpy
// and non-finite slots are zero), each thread's order unchanged, so M_C is
// the same to the last bit.
template <typename R, typename Lo = R>
__global__ void __launch_bounds__(256)
k_diag_partial(const KP<R> P, const R* __restrict__ phi, const R* __restrict__ Um, const R* __restrict__ Tm,
               const R* __restrict__ uxm, const R* __restrict__ uym, double* __restrict__ part,
               const Lo* __restrict__ Ulo = nullptr, int solute_only = 0) {
    __shared__ double s[3][8];
    // mc: twice the solute sum of the stored macros (the factor 1/2 of C is
    // applied once at the end: exact); mlo: the residual plane's part,
    // (1 - k) lo ((1 + k) - (1 - k) phi), a term ~1e-8 of the rest, in the
    // arithmetic type
    double mc = 0.0, h = 0.0, bad = 0.0;
    R mlo = R(0);
    const double omk = 1.0 - (double)P.k, opk = 1.0 + (double)P.k;
    const R omkR = R(1) - P.k, opkR = R(1) + P.k;
    // FP32 state: 1 - k and 1 + k as double-float pairs, the sums as pairs
    const float omk_h = (float)omk, omk_l = (float)(omk - (double)omk_h);
    const float opk_h = (float)opk, opk_l = (float)(opk - (double)opk_h);
    DFloat smc{0.f, 0.f}, sh{0.f, 0.f};
    for (int y = blockIdx.x; y < P.ny; y += gridDim.x) {
        const size_t row = (size_t)y * P.pitch;
        for (int x = threadIdx.x; x < P.nx; x += blockDim.x) {
            const size_t node = row + x;
            const R ph = phi[node];
            const R U = P.has_U ? Um[node] : R(0);
            const bool full = !solute_only;
            const R T = P.has_T && full ? Tm[node] : R(0);
            const R vx = P.has_flow && full ? uxm[node] : R(0), vy = P.has_flow && full ? uym[node] : R(0);
            if (P.has_U) {
                if constexpr (sizeof(R) == 8) {
                    mc += fma(omk, (double)U, 1.0) * fma(-omk, (double)ph, opk);
                } else {
                    // A = 1 + (1 - k) U and B = (1 + k) - (1 - k) phi as pairs, then A B
                    float pa, ea, pb, eb, ah, at, bh, bt, mh, ml;
                    df_mul(omk_h, (float)U, pa, ea);
                    ea = __fmaf_rn(omk_l, (float)U, ea);
                    two_sum(1.0f, pa, ah, at);
                    const float al = add_rn(at, ea);
                    df_mul(omk_h, (float)ph, pb, eb);
                    eb = __fmaf_rn(omk_l, (float)ph, eb);
                    two_sum(opk_h, -pb, bh, bt);
                    const float bl = sub_rn(add_rn(bt, opk_l), eb);
                    df_mul(ah, bh, mh, ml);
                    ml = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, ml));
                    df_add(smc, mh, ml);
                }
                if (Ulo) mlo += omkR * (R)Cvt<Lo>::ld(Ulo[node]) * (opkR - omkR * ph);
            }
            if (P.has_T && full) {
                const R ht = (R(0.5) * (R(1) + ph) * P.cS + R(0.5) * (R(1) - ph) * P.cL) * T - R(0.5) * P.rhoL_Lh * ph;
                if constexpr (sizeof(R) == 8) h += ht;
                else df_add(sh, (float)ht, 0.f);
            }
            if (full && (!isfinite(ph) || !isfinite(U) || !isfinite(T) || !isfinite(vx) || !isfinite(vy))) bad += 1.0;
        }
    }
    if constexpr (sizeof(R) == 4) {
        mc = (double)smc.h + (double)smc.l;
        h = (double)sh.h + (double)sh.l;
    }
    mc = 0.5 * (mc + (double)mlo);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mc += __shfl_xor_sync(0xffffffffu, mc, o);
        h += __shfl_xor_sync(0xffffffffu, h, o);
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s[0][w] = mc; s[1][w] = h; s[2][w] = bad; }
    __syncthreads();
    if (threadIdx.x < 3) {
        double a = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += s[threadIdx.x][i];
        part[blockIdx.x * 3 + threadIdx.x] = a;
    }
}

// out[0..2] = totals of the partials (fixed order), out[3..6] tips,
// out[7] = S_phi, out[8] = J_U; the maxima slots are then cleared.  One block
// of DIAG_FINAL_THREADS: warp 0 sums the partials, and four warps scan each
// tip direction.  sums_only: out[0..2] and the maxima only (tips not scanned).
constexpr int DIAG_FINAL_THREADS = 512;
template <typename R>
__global__ void __launch_bounds__(DIAG_FINAL_THREADS)
k_diag_final(const KP<R> P, const double* __restrict__ part, int nblocks, const R* __restrict__ phi, int cx, int cy,
             unsigned long long* __restrict__ smax, double* __restrict__ out, int sums_only = 0) {
    __shared__ int sbest[DIAG_FINAL_THREADS / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        double a[3] = {0.0, 0.0, 0.0};
        for (int b = lane; b < nblocks; b += 32)
            for (int j = 0; j < 3; ++j) a[j] += part[b * 3 + j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            for (int j = 0; j < 3; ++j) a[j] += __shfl_xor_sync(0xffffffffu, a[j], o);
        if (lane == 0) {
            out[0] = a[0];
            out[1] = a[1];
            out[2] = a[2];
            out[7] = __longlong_as_double((long long)smax[0]);
            out[8] = __longlong_as_double((long long)smax[1]);
        }
    }
    if (!sums_only) {          // uniform over the block: its barriers are reached by every thread
        // tips: warps 4d .. 4d + 3 scan direction d (+x, +y, -x, -y) for the
        // outermost crossing
        const int d = warp >> 2, sub = warp & 3;
        const int len = (d == 0) ? P.nx - cx : (d == 1) ? P.ny - cy : (d == 2) ? cx + 1 : cy + 1;
        auto at = [&](int k) -> double {
            const int x = (d == 0) ? cx + k : (d == 2) ? cx - k : cx;
            const int y = (d == 1) ? cy + k : (d == 3) ? cy - k : cy;
            return (double)phi[(size_t)y * P.pitch + x];
        };
        int best = -1;
#pragma unroll 4
        for (int k = 32 * sub + lane; k < len - 1; k += 128)
            if (at(k) >= 0.0 && at(k + 1) < 0.0) best = max(best, k);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (lane == 0) sbest[warp] = best;
        __syncthreads();
        if (sub == 0 && lane == 0) {
            best = max(max(sbest[warp], sbest[warp + 1]), max(sbest[warp + 2], sbest[warp + 3]));
            double r = 0.0;
            if (len > 0 && at(len - 1) >= 0.0) r = (double)(len - 1);
            else if (best >= 0) { const double a = at(best), b = at(best + 1); r = (double)best + a / (a - b); }
            out[3 + d] = r;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) { smax[0] = 0ull; smax[1] = 0ull; }
}

__global__ void k_set_clock(long long* clock, long long v) { *clock = v; }
__global__ void k_tick(long long* clock, long long d) { *clock += d; }

}  // namespace lbmk
