// Device kernels of the multirate MRT-LBM (Liu, Wu, Zhan, Secs. 3.1-3.3).
//
// One thread per lattice node, 32 x TY tiles. Every field update is one
// fused pass: the block loads phi on its tile plus a 2-node ghost ring into
// shared memory, collides every node of the tile plus a 1-node ring into
// shared memory (recomputing the ring's collisions instead of exchanging
// them), then each thread pulls its nine post-collision populations and
// writes the streamed result.
//
// Storage (per field, per ping-pong buffer): populations 1..8 as planes of
// `pitch * ny` elements of type ST; population 0 is never stored.  It follows
// from the node's zeroth moment, which the macroscopic arrays carry:
//   phase: f_0 = phi - sum_{i>0} f_i          (Eq. 18)
//   flow:  f_0 = rho - sum_{i>0} f_i          (Eq. 27)
//   U, T:  f_0 is not needed at all; the collision uses only the zeroth
//          moment (the macro) and the first moment (Eq. 23 relaxes every
//          other moment to equilibrium).
// With DEV = true the planes hold deviations h_i = f_i - ref_i in 16 bits:
//   phase ref_i = w_i phi, U/T ref_i = w_i chi (cancels in the first moment),
//   flow ref_i = f_eq_i(rho, u) of Eq. 28.
//
// The U and T macros include every phase-change increment already injected
// (Eq. 39).  The injection adds w_i Delta to the populations, which changes
// the zeroth moment by Delta and leaves every first moment unchanged
// (sum w_i e_i = 0); since the collision reads only those two moments, the
// population-side add is carried exactly by the macro alone.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbmk {

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_INLET_OUTFLOW = 2 };

// D2Q9 velocity set and weights (Eq. 15)
__device__ __constant__ int c_ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ __constant__ int c_ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__device__ __constant__ int c_opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

template <typename R> struct Wt {
    static constexpr R w0 = R(4) / R(9), w1 = R(1) / R(9), w2 = R(1) / R(36);
};
template <typename R> __device__ __forceinline__ R wq(int i) {
    return i == 0 ? Wt<R>::w0 : (i < 5 ? Wt<R>::w1 : Wt<R>::w2);
}

// Coefficients derived on the host in FP64, then rounded to R.
template <typename R> struct KP {
    int nx, ny, pitch;
    long long plane;       // elements per population plane
    int bsx, bsy, bfx, bfy; // scalar / flow boundary kinds
    int has_U, has_T, frozen_T, has_flow, accumulated;
    // phase (Eqs. 2-4, 21-24)
    R dtp, W0sq_tau0, inv_tau0, eps, lam, Mc;
    // transfer (Eqs. 37-38)
    R k, at_pre, rhoL_Lh;
    // solute (Eqs. 7-8)
    R dtU, DS, DL;
    // thermal (Eqs. 11-12)
    R dtT, kS, kL, cS, cL, T_shift, inv_T_scale;
    // flow (Eqs. 27-32)
    R dtF, cF, Fbx, Fby, se, seps, sq, snu, u_in;
    // prescribed undercooling
    R theta_c, fG, fy0, fV, dt_base;
};

// ---------------------------------------------------------------------------
// storage conversion
// ---------------------------------------------------------------------------
template <typename ST> struct Cvt;
template <> struct Cvt<double> {
    static __device__ __forceinline__ double ld(double v) { return v; }
    template <typename R> static __device__ __forceinline__ double st(R v) { return (double)v; }
};
template <> struct Cvt<float> {
    static __device__ __forceinline__ float ld(float v) { return v; }
    template <typename R> static __device__ __forceinline__ float st(R v) { return (float)v; }
};
template <> struct Cvt<__half> {
    static __device__ __forceinline__ float ld(__half v) { return __half2float(v); }
    template <typename R> static __device__ __forceinline__ __half st(R v) { return __float2half_rn((float)v); }
};
template <> struct Cvt<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(__nv_bfloat16 v) { return __bfloat162float(v); }
    template <typename R> static __device__ __forceinline__ __nv_bfloat16 st(R v) { return __float2bfloat16_rn((float)v); }
};

// ---------------------------------------------------------------------------
// boundary index maps
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrap_idx(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}
// scalar ghost (zero-flux wall = mirror about the half-link wall; periodic wrap)
__device__ __forceinline__ int scalar_map(int v, int n, int bc) {
    if (v >= 0 && v < n) return v;
    if (bc == BC_PERIODIC) return wrap_idx(v, n);
    v = (v < 0) ? (-1 - v) : (2 * n - 1 - v);
    return min(max(v, 0), n - 1);
}
// a node that collides: inside the domain, or a periodic image
__device__ __forceinline__ bool resolve(int& v, int n, int bc) {
    if (v >= 0 && v < n) return true;
    if (bc != BC_PERIODIC) return false;
    v = wrap_idx(v, n);
    return true;
}
__device__ __forceinline__ bool outside(int v, int n) { return v < 0 || v >= n; }

// isotropic gradient g_a = 3 sum_i w_i e_ia s(x + e_i) on a shared tile
template <typename R, int GX>
__device__ __forceinline__ void iso_grad(const R (*s)[GX], int cx, int cy, R& gx, R& gy) {
    const R E = s[cy][cx + 1], Wv = s[cy][cx - 1], N = s[cy + 1][cx], S = s[cy - 1][cx];
    const R NE = s[cy + 1][cx + 1], NW = s[cy + 1][cx - 1], SE = s[cy - 1][cx + 1], SW = s[cy - 1][cx - 1];
    gx = (E - Wv) * (R(1) / R(3)) + (NE - NW + SE - SW) * (R(1) / R(12));
    gy = (N - S) * (R(1) / R(3)) + (NE + NW - SE - SW) * (R(1) / R(12));
}

// Eq. 2 and Eq. 3 (N = 16 eps a_s g_x g_y^2 (g_x^2 - g_y^2)/|g|^4, y by symmetry)
template <typename R>
__device__ __forceinline__ void aniso(R gx, R gy, R eps, R& as, R& Nx, R& Ny) {
    const R gx2 = gx * gx, gy2 = gy * gy, g2 = gx2 + gy2;
    if (g2 <= R(1e-12)) { as = R(1); Nx = R(0); Ny = R(0); return; }
    const R inv = R(1) / g2, inv2 = inv * inv;
    as = R(1) - R(3) * eps + R(4) * eps * (gx2 * gx2 + gy2 * gy2) * inv2;
    const R t = R(16) * eps * as * inv2;
    Nx = t * gx * gy2 * (gx2 - gy2);
    Ny = t * gy * gx2 * (gy2 - gx2);
}

// f*_i = w_i A + 3 w_i (e_i . b) + (e_i . c): the scalar collision of Eq. 14
// with S of Eq. 23 in closed form (columns 3 and 5 of M^-1 are e_x/6, e_y/6),
// A = chi + dt Q, b = j_eq = first moment of f_eq, c = (1 - s) j_neq / 6.
template <typename R, int HY, int HX>
__device__ __forceinline__ void put_scalar_post(R (*sp)[HY][HX], int ly, int lx, R A, R bx, R by, R cx, R cy) {
    const R w1 = Wt<R>::w1, w2 = Wt<R>::w2;
    const R a1 = w1 * A, a2 = w2 * A, b1x = R(3) * w1 * bx, b1y = R(3) * w1 * by;
    const R b2x = R(3) * w2 * bx, b2y = R(3) * w2 * by;
    sp[0][ly][lx] = Wt<R>::w0 * A;
    sp[1][ly][lx] = a1 + b1x + cx;
    sp[2][ly][lx] = a1 + b1y + cy;
    sp[3][ly][lx] = a1 - b1x - cx;
    sp[4][ly][lx] = a1 - b1y - cy;
    sp[5][ly][lx] = a2 + (b2x + b2y) + (cx + cy);
    sp[6][ly][lx] = a2 + (b2y - b2x) + (cy - cx);
    sp[7][ly][lx] = a2 - (b2x + b2y) - (cx + cy);
    sp[8][ly][lx] = a2 + (b2x - b2y) + (cx - cy);
}

template <typename R> __device__ __forceinline__ R theta_frozen(const KP<R>& P, int y, R t) {
    return P.theta_c + P.fG * ((R)y - P.fy0 - P.fV * t);
}

// ---------------------------------------------------------------------------
// Work items of a tile.  Every update kernel collides the tile plus a 1-node
// ring: item A of thread (tx, ty) is its own node (halo position tx+1, ty+1);
// item B of threads tid < NR is one of the NR = 2(TX+2) + 2 TY ring positions.
// All global loads of both items are issued before the first barrier, so a
// block pays one memory round trip before it computes.
// ---------------------------------------------------------------------------
template <int TY>
__device__ __forceinline__ void ring_pos(int t, int& lx, int& ly) {
    constexpr int HX = 34;
    if (t < HX) { lx = t; ly = 0; }
    else if (t < 2 * HX) { lx = t - HX; ly = TY + 1; }
    else if (t < 2 * HX + TY) { lx = 0; ly = t - 2 * HX + 1; }
    else { lx = HX - 1; ly = t - 2 * HX - TY + 1; }
}

// resolve both coordinates (each is always evaluated)
__device__ __forceinline__ bool resolve_xy(int& x, int& y, int nx, int ny, int bcx, int bcy) {
    const bool a = resolve(x, nx, bcx);
    const bool b = resolve(y, ny, bcy);
    return a && b;
}

// phi on the tile plus a 2-node ghost ring (scalar boundary rule)
template <typename R, int TY>
__device__ __forceinline__ void load_phi_ring2(const KP<R>& P, const R* __restrict__ phi, R (*s)[36], int x0, int y0,
                                               int tid) {
    constexpr int GX = 36, GY = TY + 4, NT = 32 * TY;
    R v[(GX * GY + NT - 1) / NT];
#pragma unroll
    for (int k = 0; k < (GX * GY + NT - 1) / NT; ++k) {
        const int p = tid + k * NT;
        if (p < GX * GY) {
            const int lx = p % GX, ly = p / GX;
            const int gx = scalar_map(x0 - 2 + lx, P.nx, P.bsx), gy = scalar_map(y0 - 2 + ly, P.ny, P.bsy);
            v[k] = phi[(size_t)gy * P.pitch + gx];
        }
    }
#pragma unroll
    for (int k = 0; k < (GX * GY + NT - 1) / NT; ++k) {
        const int p = tid + k * NT;
        if (p < GX * GY) s[p / GX][p % GX] = v[k];
    }
}

template <typename R, typename ST>
__device__ __forceinline__ void load8(const ST* __restrict__ f, size_t node, long long plane, R* v) {
#pragma unroll
    for (int i = 1; i < 9; ++i) v[i] = (R)Cvt<ST>::ld(f[(size_t)(i - 1) * plane + node]);
}
template <typename R> __device__ __forceinline__ R mom_x(const R* v) { return v[1] - v[3] + v[5] - v[6] - v[7] + v[8]; }
template <typename R> __device__ __forceinline__ R mom_y(const R* v) { return v[2] - v[4] + v[5] + v[6] - v[7] - v[8]; }

// ---------------------------------------------------------------------------
// Phase-field update (Eqs. 2-4, 14, 21-24, 26, 18)
// ---------------------------------------------------------------------------
// collision of the phase populations at halo position (lx, ly); returns a_s^2
template <typename R, int TY>
__device__ __forceinline__ R phase_collide(const KP<R>& P, const R (*sphi)[36], R (*sp)[TY + 2][34], int lx, int ly,
                                           int gy, R jx, R jy, R Us, R Tv, R tnow) {
    const R c = sphi[ly + 1][lx + 1];
    R gxv, gyv, as, Nx, Ny;
    iso_grad<R, 36>(sphi, lx + 1, ly + 1, gxv, gyv);
    aniso(gxv, gyv, P.eps, as, Nx, Ny);
    const R a2 = as * as;
    const R s = R(1) / (R(3) * P.dtp * a2 * P.W0sq_tau0 + R(0.5));              // Eq. 24
    R th;
    if (P.has_T) th = (Tv - P.T_shift) * P.inv_T_scale;                          // Eq. 5
    else if (P.frozen_T) th = theta_frozen(P, gy, tnow);
    else th = P.theta_c;
    const R one = R(1) - c * c;
    const R Q = c * one - P.lam * (P.Mc * Us + th) * one * one;                   // Eq. 4
    const R bx = -P.dtp * P.W0sq_tau0 * Nx, by = -P.dtp * P.W0sq_tau0 * Ny;      // dt v_n (Eqs. 21-22)
    const R k6 = (R(1) - s) * (R(1) / R(6));
    put_scalar_post<R, TY + 2, 34>(sp, ly, lx, c + P.dtp * Q * P.inv_tau0, bx, by, k6 * (jx - bx), k6 * (jy - by));
    return a2;
}

template <typename R, typename ST, bool DEV, int TY>
__global__ void __launch_bounds__(32 * TY)
k_phase(const KP<R> P, const ST* __restrict__ fin, ST* __restrict__ fout, const R* __restrict__ phi,
        R* __restrict__ phin, const R* __restrict__ Um, const R* __restrict__ Tm,
        const long long* __restrict__ clock, long long step_off) {
    constexpr int TX = 32, HX = TX + 2, HY = TY + 2, GY = TY + 4, NR = 2 * HX + 2 * TY;
    static_assert(NR <= 32 * TY, "ring larger than the block");
    __shared__ R sphi[GY][36];
    __shared__ R spost[9][HY][HX];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    int ax = x0 + tx, ay = y0 + ty;
    const bool own = ax < P.nx && ay < P.ny;
    const bool va = resolve_xy(ax, ay, P.nx, P.ny, P.bsx, P.bsy);
    int blx = 0, bly = 0, bx = 0, by = 0;
    bool vb = false;
    if (tid < NR) {
        ring_pos<TY>(tid, blx, bly);
        bx = x0 - 1 + blx;
        by = y0 - 1 + bly;
        vb = resolve_xy(bx, by, P.nx, P.ny, P.bsx, P.bsy);
    }
    const size_t na = (size_t)ay * P.pitch + ax, nb = (size_t)by * P.pitch + bx;
    R fa[9], fb[9];
    R Ua = R(0), Ta = R(0), Ub = R(0), Tb = R(0);
    if (va) {
        load8<R, ST>(fin, na, P.plane, fa);
        if (P.has_U) Ua = Um[na];
        if (P.has_T) Ta = Tm[na];
    }
    if (vb) {
        load8<R, ST>(fin, nb, P.plane, fb);
        if (P.has_U) Ub = Um[nb];
        if (P.has_T) Tb = Tm[nb];
    }
    load_phi_ring2<R, TY>(P, phi, sphi, x0, y0, tid);
    R tnow = R(0);
    if (P.frozen_T) tnow = (R)((clock ? *clock : 0ll) + step_off) * P.dt_base;
    __syncthreads();
    R a2own = R(1);
    if (va) a2own = phase_collide<R, TY>(P, sphi, spost, tx + 1, ty + 1, ay, mom_x(fa), mom_y(fa), Ua, Ta, tnow);
    if (vb) phase_collide<R, TY>(P, sphi, spost, blx, bly, by, mom_x(fb), mom_y(fb), Ub, Tb, tnow);
    __syncthreads();
    if (!own) return;
    const R c = sphi[ty + 2][tx + 2];
    const R inva2 = R(1) / a2own;
    R s8 = R(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        if (DEV) fa[i] += wq<R>(i) * c;          // decode h_i = f_i - w_i phi
        s8 += fa[i];
    }
    fa[0] = c - s8;                              // population 0 from the zeroth moment
    const int gx = x0 + tx, gy = y0 + ty;
    R fn[9], sum = R(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int sx = gx - c_ex[i], sy = gy - c_ey[i];
        const bool wall = (P.bsx != BC_PERIODIC && outside(sx, P.nx)) || (P.bsy != BC_PERIODIC && outside(sy, P.ny));
        const R inc = wall ? spost[c_opp[i]][ty + 1][tx + 1] : spost[i][ty + 1 - c_ey[i]][tx + 1 - c_ex[i]];
        fn[i] = fa[i] + (inc - fa[i]) * inva2;                                   // Eq. 26
        sum += fn[i];
    }
    const size_t node = (size_t)gy * P.pitch + gx;
    phin[node] = sum;                                                            // Eq. 18
#pragma unroll
    for (int i = 1; i < 9; ++i)
        fout[(size_t)(i - 1) * P.plane + node] = Cvt<ST>::st(DEV ? fn[i] - wq<R>(i) * sum : fn[i]);
}

// ---------------------------------------------------------------------------
// Phase-change transfer (Eqs. 36-39)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void atomic_max_pos(unsigned long long* slot, double v) {
    if (v > 0.0) atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}

// map a halo position to the node whose J fills it: periodic wrap, or the
// mirrored node with the wall-normal flips; (cx, cy) = its shared-tile position
__device__ __forceinline__ bool j_source(int& g, int n, int bc, int base, int& c, bool& flip) {
    flip = false;
    if (g >= 0 && g < n) return true;
    if (bc == BC_PERIODIC) { g = wrap_idx(g, n); return true; }
    g = (g < 0) ? (-1 - g) : (2 * n - 1 - g);
    flip = true;
    c = g - base;
    return g >= 0 && g < n;
}

template <typename R, int TY>
__global__ void __launch_bounds__(32 * TY)
k_transfer(const KP<R> P, const R* __restrict__ phio, const R* __restrict__ phin, const R* __restrict__ Uin,
           R* __restrict__ Uout, const R* __restrict__ Tin, R* __restrict__ Tout, R* __restrict__ accU,
           R* __restrict__ accT, int acc_reset_U, int acc_reset_T, unsigned long long* __restrict__ smax) {
    constexpr int TX = 32, HX = TX + 2, HY = TY + 2, GX = 36, GY = TY + 4, NT = 32 * TY, NR = 2 * HX + 2 * TY;
    __shared__ R spn[GY][GX];
    __shared__ R sJx[HY][HX], sJy[HY][HX];
    __shared__ double sred[NT / 32];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    // item A: own halo position; item B: a ring position
    int alx = tx + 1, aly = ty + 1, blx = 0, bly = 0;
    if (tid < NR) ring_pos<TY>(tid, blx, bly);
    int ax = x0 - 1 + alx, ay = y0 - 1 + aly, bx = x0 - 1 + blx, by = y0 - 1 + bly;
    int acx = alx + 1, acy = aly + 1, bcx = blx + 1, bcy = bly + 1;
    bool afx, afy, bfx = false, bfy = false;
    const bool va = j_source(ax, P.nx, P.bsx, x0 - 2, acx, afx) & j_source(ay, P.ny, P.bsy, y0 - 2, acy, afy) &&
                    acx >= 1 && acx <= GX - 2 && acy >= 1 && acy <= GY - 2;
    bool vb = false;
    if (tid < NR)
        vb = j_source(bx, P.nx, P.bsx, x0 - 2, bcx, bfx) & j_source(by, P.ny, P.bsy, y0 - 2, bcy, bfy) &&
             bcx >= 1 && bcx <= GX - 2 && bcy >= 1 && bcy <= GY - 2;
    const size_t na = (size_t)ay * P.pitch + ax, nb = (size_t)by * P.pitch + bx;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool own = gx < P.nx && gy < P.ny;
    const size_t node = (size_t)gy * P.pitch + gx;
    R poa = R(0), Usa = R(0), pob = R(0), Usb = R(0), Town = R(0), accUo = R(0), accTo = R(0);
    if (va) { poa = phio[na]; if (P.has_U) Usa = Uin[na]; }
    if (vb) { pob = phio[nb]; if (P.has_U) Usb = Uin[nb]; }
    if (own) {
        if (P.has_T) Town = Tin[node];
        if (P.accumulated) {
            if (P.has_U && !acc_reset_U) accUo = accU[node];
            if (P.has_T && !acc_reset_T) accTo = accT[node];
        }
    }
    load_phi_ring2<R, TY>(P, phin, spn, x0, y0, tid);
    __syncthreads();
    const R pre = P.at_pre;
    auto jfill = [&](bool v, int lx, int ly, int cx, int cy, bool fx, bool fy, R po, R Us) {
        R jx = R(0), jy = R(0);
        if (v) {
            R gxv, gyv;
            iso_grad<R, GX>(spn, cx, cy, gxv, gyv);
            const R g2 = gxv * gxv + gyv * gyv;
            R nxv = R(0), nyv = R(0);
            if (g2 > R(1e-12)) {
                const R ig = R(1) / sqrt(g2);
                nxv = -gxv * ig;
                nyv = -gyv * ig;
            }
            const R a = pre * (R(1) + (R(1) - P.k) * Us) * (spn[cy][cx] - po);     // Eqs. 36-37
            jx = fx ? -a * nxv : a * nxv;
            jy = fy ? -a * nyv : a * nyv;
        }
        sJx[ly][lx] = jx;
        sJy[ly][lx] = jy;
    };
    jfill(va, alx, aly, acx, acy, afx, afy, poa, Usa);
    if (tid < NR) jfill(vb, blx, bly, bcx, bcy, bfx, bfy, pob, Usb);
    __syncthreads();
    double mydu = 0.0;
    if (own) {
        const int hx = tx + 1, hy = ty + 1;
        const R div = (sJx[hy][hx + 1] - sJx[hy][hx - 1] + sJy[hy + 1][hx] - sJy[hy - 1][hx]) * (R(1) / R(3)) +
                      ((sJx[hy + 1][hx + 1] + sJy[hy + 1][hx + 1]) + (sJy[hy + 1][hx - 1] - sJx[hy + 1][hx - 1]) -
                       (sJx[hy - 1][hx - 1] + sJy[hy - 1][hx - 1]) + (sJx[hy - 1][hx + 1] - sJy[hy - 1][hx + 1])) *
                          (R(1) / R(12));
        const R pn = spn[ty + 2][tx + 2];
        const R dphi = pn - poa;                      // item A of an own node is the node itself
        if (P.has_U) {
            const R Us = Usa;
            const R dU = ((R(1) + (R(1) - P.k) * Us) * dphi - R(2) * div) /
                         ((R(1) + P.k) - (R(1) - P.k) * pn);                       // Eq. 38
            mydu = fabs((double)dU);
            if (!P.accumulated) Uout[node] = Us + dU;                               // Eq. 39
            else accU[node] = accUo + dU;
        }
        if (P.has_T) {
            const R rc = R(0.5) * (R(1) + pn) * P.cS + R(0.5) * (R(1) - pn) * P.cL;
            const R dT = P.rhoL_Lh * dphi / (R(2) * rc);                            // Eq. 38
            if (!P.accumulated) Tout[node] = Town + dT;
            else accT[node] = accTo + dT;
        }
    }
    // block maximum of |Delta U_pc| -> S_phi (and J_U when instantaneous)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mydu = fmax(mydu, __shfl_xor_sync(0xffffffffu, mydu, o));
    if ((tid & 31) == 0) sred[tid >> 5] = mydu;
    __syncthreads();
    if (tid == 0 && P.has_U) {
        double m = 0.0;
        for (int w = 0; w < NT / 32; ++w) m = fmax(m, sred[w]);
        atomic_max_pos(&smax[0], m);
        if (!P.accumulated) atomic_max_pos(&smax[1], m);
    }
}

// ---------------------------------------------------------------------------
// Concentration / temperature update (Eqs. 7-8, 10-12 tr parts; 14, 19-20,
// 23-25, 40, 18).  FIELD 0 = U, 1 = T.
// ---------------------------------------------------------------------------
template <typename R, int TY, int FIELD>
__device__ __forceinline__ void scalar_collide(const KP<R>& P, const R (*sphi)[36], R (*sp)[TY + 2][34], int lx,
                                               int ly, R chi, R jx, R jy, R vx, R vy) {
    const R dt = FIELD == 0 ? P.dtU : P.dtT;
    const R ph = sphi[ly + 1][lx + 1];
    R D, coef;
    if (FIELD == 0) {
        const R den = (R(1) + P.k) - (R(1) - P.k) * ph;
        D = ((R(1) + ph) * P.DS + (R(1) - ph) * P.DL) / den;                      // Eq. 7
        coef = -(R(1) - P.k) * D / den;                                           // Eq. 8, tr
    } else {
        const R rc = R(0.5) * (R(1) + ph) * P.cS + R(0.5) * (R(1) - ph) * P.cL;
        D = (R(0.5) * (R(1) + ph) * P.kS + R(0.5) * (R(1) - ph) * P.kL) / rc;     // Eq. 11
        coef = (P.cS - P.cL) / (R(2) * rc) * D;                                   // Eq. 12, tr
    }
    const R s = R(1) / (R(3) * dt * D + R(0.5));                                  // Eq. 24
    const R bx = dt * chi * vx, by = dt * chi * vy;                                // Eqs. 19-20
    const R jnx = jx - bx, jny = jy - by;
    R gpx, gpy;
    iso_grad<R, 36>(sphi, lx + 1, ly + 1, gpx, gpy);
    const R Q = coef * (R(-3) * s) * (jnx * gpx + jny * gpy);                       // Eq. 40 in Eq. 8 / 12
    const R k6 = (R(1) - s) * (R(1) / R(6));
    put_scalar_post<R, TY + 2, 34>(sp, ly, lx, chi + dt * Q, bx, by, k6 * jnx, k6 * jny);
}

template <typename R, typename ST, bool DEV, int TY, int FIELD>
__global__ void __launch_bounds__(32 * TY)
k_scalar(const KP<R> P, const ST* __restrict__ fin, ST* __restrict__ fout, const R* __restrict__ mac_in,
         R* __restrict__ mac_out, const R* __restrict__ acc, const R* __restrict__ phi, const R* __restrict__ ux,
         const R* __restrict__ uy, unsigned long long* __restrict__ smax) {
    constexpr int TX = 32, HX = TX + 2, HY = TY + 2, GY = TY + 4, NT = 32 * TY, NR = 2 * HX + 2 * TY;
    __shared__ R sphi[GY][36];
    __shared__ R spost[9][HY][HX];
    __shared__ double sred[NT / 32];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    int ax = x0 + tx, ay = y0 + ty;
    const bool va = resolve_xy(ax, ay, P.nx, P.ny, P.bsx, P.bsy);
    int blx = 0, bly = 0, bx = 0, by = 0;
    bool vb = false;
    if (tid < NR) {
        ring_pos<TY>(tid, blx, bly);
        bx = x0 - 1 + blx;
        by = y0 - 1 + bly;
        vb = resolve_xy(bx, by, P.nx, P.ny, P.bsx, P.bsy);
    }
    const size_t na = (size_t)ay * P.pitch + ax, nb = (size_t)by * P.pitch + bx;
    R fa[9], fb[9];
    R ca = R(0), cb = R(0), uxa = R(0), uya = R(0), uxb = R(0), uyb = R(0), acca = R(0);
    if (va) {
        load8<R, ST>(fin, na, P.plane, fa);
        ca = mac_in[na];
        if (P.accumulated) { acca = acc[na]; ca += acca; }   // coarse-step injection (Sec. 4.4 ablation)
        if (P.has_flow) { uxa = ux[na]; uya = uy[na]; }
    }
    if (vb) {
        load8<R, ST>(fin, nb, P.plane, fb);
        cb = mac_in[nb];
        if (P.accumulated) cb += acc[nb];
        if (P.has_flow) { uxb = ux[nb]; uyb = uy[nb]; }
    }
    load_phi_ring2<R, TY>(P, phi, sphi, x0, y0, tid);
    __syncthreads();
    if (va) scalar_collide<R, TY, FIELD>(P, sphi, spost, tx + 1, ty + 1, ca, mom_x(fa), mom_y(fa), uxa, uya);
    if (vb) scalar_collide<R, TY, FIELD>(P, sphi, spost, blx, bly, cb, mom_x(fb), mom_y(fb), uxb, uyb);
    __syncthreads();
    const int gx = x0 + tx, gy = y0 + ty;
    double myj = 0.0;
    if (gx < P.nx && gy < P.ny) {
        const size_t node = (size_t)gy * P.pitch + gx;
        R fn[9], sum = R(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sx = gx - c_ex[i], sy = gy - c_ey[i];
            const bool wall = (P.bsx != BC_PERIODIC && outside(sx, P.nx)) || (P.bsy != BC_PERIODIC && outside(sy, P.ny));
            fn[i] = wall ? spost[c_opp[i]][ty + 1][tx + 1] : spost[i][ty + 1 - c_ey[i]][tx + 1 - c_ex[i]]; // Eq. 25
            sum += fn[i];
        }
        mac_out[node] = sum;                                                      // Eq. 18
#pragma unroll
        for (int i = 1; i < 9; ++i)
            fout[(size_t)(i - 1) * P.plane + node] = Cvt<ST>::st(DEV ? fn[i] - wq<R>(i) * sum : fn[i]);
        if (FIELD == 0 && P.accumulated) myj = fabs((double)acca);
    }
    if (FIELD == 0 && P.accumulated) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) myj = fmax(myj, __shfl_xor_sync(0xffffffffu, myj, o));
        if ((tid & 31) == 0) sred[tid >> 5] = myj;
        __syncthreads();
        if (tid == 0) {
            double m = 0.0;
            for (int w = 0; w < NT / 32; ++w) m = fmax(m, sred[w]);
            atomic_max_pos(&smax[1], m);
        }
    }
}

// ---------------------------------------------------------------------------
// Flow update (Eqs. 27-33) with the inlet / outflow columns
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void feq_flow(R rho, R ux, R uy, R c, R* f) {               // Eq. 28
    const R ic = R(1) / c, u2 = (ux * ux + uy * uy) * ic * ic;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const R eu = ((R)c_ex[i] * ux + (R)c_ey[i] * uy) * ic;
        f[i] = wq<R>(i) * rho * (R(1) + R(3) * eu + R(4.5) * eu * eu - R(1.5) * u2);
    }
}

// MRT collision of Eq. 14 with S of Eq. 31 and Guo forcing (Eq. 30); f holds
// populations 1..8 (decoded) on entry, rho and u the macros written with them
template <typename R, int TY>
__device__ __forceinline__ void flow_collide(const KP<R>& P, R (*sp)[TY + 2][34], int lx, int ly, R* f, R rho) {
    const R c = P.cF, dt = P.dtF;
    R s8 = R(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) s8 += f[i];
    f[0] = rho - s8;
    const R jx = mom_x(f), jy = mom_y(f);
    const R ux = (c * jx + R(0.5) * dt * P.Fbx) / rho, uy = (c * jy + R(0.5) * dt * P.Fby) / rho; // Eq. 27
    const R ic = R(1) / c, ic2 = ic * ic, u2 = (ux * ux + uy * uy) * ic2;
    // non-conserved moments of f (rows 1, 2, 4, 6, 7, 8 of M, Eq. 16)
    const R sa = f[1] + f[2] + f[3] + f[4], sd = f[5] + f[6] + f[7] + f[8];
    const R m1 = R(-4) * f[0] - sa + R(2) * sd;
    const R m2 = R(4) * f[0] - R(2) * sa + sd;
    const R m4 = R(-2) * f[1] + R(2) * f[3] + f[5] - f[6] - f[7] + f[8];
    const R m6 = R(-2) * f[2] + R(2) * f[4] + f[5] + f[6] - f[7] - f[8];
    const R m7 = f[1] - f[2] + f[3] - f[4];
    const R m8 = f[5] - f[6] + f[7] - f[8];
    // Eq. 29 equilibria, Eq. 30 Guo moments, Eq. 31 rates; dm_k scaled by the
    // diagonal of M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
    const R fu = (P.Fbx * ux + P.Fby * uy) * ic2;
    const R G1 = R(6) * fu, G3 = P.Fbx * ic, G5 = P.Fby * ic;
    const R G7 = R(2) * (P.Fbx * ux - P.Fby * uy) * ic2, G8 = (P.Fby * ux + P.Fbx * uy) * ic2;
    const R d1 = (-P.se * (m1 - rho * (R(-2) + R(3) * u2)) + (R(1) - R(0.5) * P.se) * G1) * (R(1) / R(36));
    const R d2 = (-P.seps * (m2 - rho * (R(1) - R(3) * u2)) - (R(1) - R(0.5) * P.seps) * G1) * (R(1) / R(36));
    const R d3 = G3 * (R(1) / R(6));
    const R d4 = (-P.sq * (m4 + rho * ux * ic) - (R(1) - R(0.5) * P.sq) * G3) * (R(1) / R(12));
    const R d5 = G5 * (R(1) / R(6));
    const R d6 = (-P.sq * (m6 + rho * uy * ic) - (R(1) - R(0.5) * P.sq) * G5) * (R(1) / R(12));
    const R d7 = (-P.snu * (m7 - rho * (ux * ux - uy * uy) * ic2) + (R(1) - R(0.5) * P.snu) * G7) * (R(1) / R(4));
    const R d8 = (-P.snu * (m8 - rho * ux * uy * ic2) + (R(1) - R(0.5) * P.snu) * G8) * (R(1) / R(4));
    const R axis = -d1 - R(2) * d2, diag = R(2) * d1 + d2;
    sp[0][ly][lx] = f[0] - R(4) * d1 + R(4) * d2;
    sp[1][ly][lx] = f[1] + axis + d3 - R(2) * d4 + d7;
    sp[2][ly][lx] = f[2] + axis + d5 - R(2) * d6 - d7;
    sp[3][ly][lx] = f[3] + axis - d3 + R(2) * d4 + d7;
    sp[4][ly][lx] = f[4] + axis - d5 + R(2) * d6 - d7;
    sp[5][ly][lx] = f[5] + diag + d3 + d4 + d5 + d6 + d8;
    sp[6][ly][lx] = f[6] + diag - d3 - d4 + d5 + d6 - d8;
    sp[7][ly][lx] = f[7] + diag - d3 - d4 - d5 - d6 + d8;
    sp[8][ly][lx] = f[8] + diag + d3 + d4 - d5 - d6 - d8;
}

template <typename R, typename ST, bool DEV, int TY>
__global__ void __launch_bounds__(32 * TY)
k_flow(const KP<R> P, const ST* __restrict__ fin, ST* __restrict__ fout, const R* __restrict__ phi,
       const R* __restrict__ ux_in, const R* __restrict__ uy_in, const R* __restrict__ rho_in,
       R* __restrict__ ux_out, R* __restrict__ uy_out, R* __restrict__ rho_out) {
    constexpr int TX = 32, HX = TX + 2, HY = TY + 2, NR = 2 * HX + 2 * TY;
    __shared__ R sfl[HY][HX];
    __shared__ R spost[9][HY][HX];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const R c = P.cF, dt = P.dtF;
    int ax = x0 + tx, ay = y0 + ty;
    const bool va = resolve_xy(ax, ay, P.nx, P.ny, P.bfx, P.bfy);
    int blx = 0, bly = 0, bx = 0, by = 0;
    bool vb = false;
    if (tid < NR) {
        ring_pos<TY>(tid, blx, bly);
        bx = x0 - 1 + blx;
        by = y0 - 1 + bly;
        vb = resolve_xy(bx, by, P.nx, P.ny, P.bfx, P.bfy);
    }
    const size_t na = (size_t)ay * P.pitch + ax, nb = (size_t)by * P.pitch + bx;
    R fa[9], fb[9];
    R ra = R(1), rb = R(1), uxa = R(0), uya = R(0), uxb = R(0), uyb = R(0), pa = R(0), pb = R(0);
    if (va) {
        load8<R, ST>(fin, na, P.plane, fa);
        ra = rho_in[na]; uxa = ux_in[na]; uya = uy_in[na]; pa = phi[na];
    }
    if (vb) {
        load8<R, ST>(fin, nb, P.plane, fb);
        rb = rho_in[nb]; uxb = ux_in[nb]; uyb = uy_in[nb]; pb = phi[nb];
    }
    if (DEV) {     // h_i = f_i - f_eq_i(rho, u) of the writer's macros
        R ref[9];
        if (va) { feq_flow<R>(ra, uxa, uya, c, ref);
#pragma unroll
            for (int i = 1; i < 9; ++i) fa[i] += ref[i]; }
        if (vb) { feq_flow<R>(rb, uxb, uyb, c, ref);
#pragma unroll
            for (int i = 1; i < 9; ++i) fb[i] += ref[i]; }
    }
    if (va) {
        sfl[ty + 1][tx + 1] = R(0.5) * (R(1) - pa);                                  // f_L = (1 - phi)/2
        flow_collide<R, TY>(P, spost, tx + 1, ty + 1, fa, ra);
    }
    if (vb) {
        sfl[bly][blx] = R(0.5) * (R(1) - pb);
        flow_collide<R, TY>(P, spost, blx, bly, fb, rb);
    }
    __syncthreads();
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx >= P.nx || gy >= P.ny) return;
    const size_t node = (size_t)gy * P.pitch + gx;
    // streamed value of direction i into the node at shared position (hx, hy),
    // global (gxn, gyn), with the weighted partial bounce-back of Eq. 33
    auto pulled = [&](int i, int hx, int hy, int gxn, int gyn) -> R {
        const int sx = gxn - c_ex[i], sy = gyn - c_ey[i];
        const int o = c_opp[i];
        const bool blocked = (P.bfx != BC_PERIODIC && outside(sx, P.nx)) || (P.bfy != BC_PERIODIC && outside(sy, P.ny));
        if (blocked) return spost[o][hy][hx];
        const R fLm = R(0.5) * (sfl[hy - c_ey[i]][hx - c_ex[i]] + sfl[hy][hx]);
        return fLm * spost[i][hy - c_ey[i]][hx - c_ex[i]] + (R(1) - fLm) * spost[o][hy][hx];
    };
    R fn[9];
    const int hx = tx + 1, hy = ty + 1;
    if (P.bfx == BC_INLET_OUTFLOW && gx == P.nx - 1) {
#pragma unroll
        for (int i = 0; i < 9; ++i) fn[i] = pulled(i, hx - 1, hy, gx - 1, gy);      // f(L-1) = f(L-2)
    } else if (P.bfx == BC_INLET_OUTFLOW && gx == 0) {
        R rho1 = R(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) rho1 += pulled(i, hx + 1, hy, gx + 1, gy);
        feq_flow<R>(rho1, P.u_in, R(0), c, fn);                                     // f = f_eq(rho(1), u_in)
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) fn[i] = pulled(i, hx, hy, gx, gy);
    }
    R rho = R(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) rho += fn[i];
    const R jx = mom_x(fn), jy = mom_y(fn);
    const R ux = (c * jx + R(0.5) * dt * P.Fbx) / rho, uy = (c * jy + R(0.5) * dt * P.Fby) / rho;
    rho_out[node] = rho;
    ux_out[node] = ux;
    uy_out[node] = uy;
    if (DEV) {
        R ref[9];
        feq_flow<R>(rho, ux, uy, c, ref);
#pragma unroll
        for (int i = 1; i < 9; ++i) fout[(size_t)(i - 1) * P.plane + node] = Cvt<ST>::st(fn[i] - ref[i]);
    } else {
#pragma unroll
        for (int i = 1; i < 9; ++i) fout[(size_t)(i - 1) * P.plane + node] = Cvt<ST>::st(fn[i]);
    }
}
// ---------------------------------------------------------------------------
// Initial distributions f = f_eq of the macroscopic fields (Eqs. 19, 21, 28)
// ---------------------------------------------------------------------------
template <typename R, typename ST, bool DEV>
__global__ void k_init(const KP<R> P, const R* __restrict__ phi, const R* __restrict__ Um, const R* __restrict__ Tm,
                       const R* __restrict__ uxm, const R* __restrict__ uym, const R* __restrict__ rhom,
                       ST* __restrict__ fphi, ST* __restrict__ fU, ST* __restrict__ fT, ST* __restrict__ fF) {
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (gx >= P.nx || gy >= P.ny) return;
    const size_t node = (size_t)gy * P.pitch + gx;
    // gradient with the same ghost rule as the update kernels
    R s[3][3];
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx)
            s[dy + 1][dx + 1] = phi[(size_t)scalar_map(gy + dy, P.ny, P.bsy) * P.pitch + scalar_map(gx + dx, P.nx, P.bsx)];
    const R gxv = (s[1][2] - s[1][0]) * (R(1) / R(3)) + (s[2][2] - s[2][0] + s[0][2] - s[0][0]) * (R(1) / R(12));
    const R gyv = (s[2][1] - s[0][1]) * (R(1) / R(3)) + (s[2][2] + s[2][0] - s[0][2] - s[0][0]) * (R(1) / R(12));
    R as, Nx, Ny;
    aniso(gxv, gyv, P.eps, as, Nx, Ny);
    const R bx = -P.dtp * P.W0sq_tau0 * Nx, by = -P.dtp * P.W0sq_tau0 * Ny;
    const R ph = s[1][1];
    R vx = R(0), vy = R(0);
    if (P.has_flow) { vx = uxm[node]; vy = uym[node]; }
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const R w = wq<R>(i), ex = (R)c_ex[i], ey = (R)c_ey[i];
        const R dp = R(3) * w * (ex * bx + ey * by);                                   // Eq. 21 minus w_i phi
        fphi[(size_t)(i - 1) * P.plane + node] = Cvt<ST>::st(DEV ? dp : w * ph + dp);
        if (P.has_U) {
            const R U = Um[node], d = R(3) * w * U * P.dtU * (ex * vx + ey * vy);       // Eq. 19
            fU[(size_t)(i - 1) * P.plane + node] = Cvt<ST>::st(DEV ? d : w * U + d);
        }
        if (P.has_T) {
            const R T = Tm[node], d = R(3) * w * T * P.dtT * (ex * vx + ey * vy);
            fT[(size_t)(i - 1) * P.plane + node] = Cvt<ST>::st(DEV ? d : w * T + d);
        }
    }
    if (P.has_flow) {
        R fe[9];
        feq_flow<R>(rhom[node], uxm[node], uym[node], P.cF, fe);                          // Eq. 28
#pragma unroll
        for (int i = 1; i < 9; ++i) fF[(size_t)(i - 1) * P.plane + node] = Cvt<ST>::st(DEV ? R(0) : fe[i]);
    }
}

// FP64 staging -> arithmetic type, with a pitch
template <typename R>
__global__ void k_from_f64(const double* __restrict__ src, R* __restrict__ dst, int nx, int ny, int pitch) {
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (gx < nx && gy < ny) dst[(size_t)gy * pitch + gx] = (R)src[(size_t)gy * nx + gx];
}

// derived output fields into a dense ny x nx buffer of type O
// which: 0 phi 1 U 2 T 3 ux 4 uy 5 rho 6 C/C_inf 7 theta
template <typename R, typename O>
__global__ void k_out(const KP<R> P, int which, const R* __restrict__ phi, const R* __restrict__ Um,
                      const R* __restrict__ Tm, const R* __restrict__ uxm, const R* __restrict__ uym,
                      const R* __restrict__ rhom, const R* __restrict__ accU, const R* __restrict__ accT,
                      O* __restrict__ dst, const long long* __restrict__ clock) {
    const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (gx >= P.nx || gy >= P.ny) return;
    const size_t node = (size_t)gy * P.pitch + gx;
    R v = R(0);
    const R U = P.has_U ? Um[node] : R(0);
    switch (which) {
        case 0: v = phi[node]; break;
        case 1: v = U; break;
        case 2: v = P.has_T ? Tm[node] : R(0); break;
        case 3: v = P.has_flow ? uxm[node] : R(0); break;
        case 4: v = P.has_flow ? uym[node] : R(0); break;
        case 5: v = P.has_flow ? rhom[node] : R(1); break;
        case 6: v = R(0.5) * (R(1) + (R(1) - P.k) * U) * ((R(1) + P.k) - (R(1) - P.k) * phi[node]); break;
        case 7:
            if (P.has_T) v = (Tm[node] - P.T_shift) * P.inv_T_scale;
            else if (P.frozen_T) v = theta_frozen(P, gy, (R)(*clock) * P.dt_base);
            else v = P.theta_c;
            break;
    }
    (void)accU; (void)accT;
    dst[(size_t)gy * P.nx + gx] = (O)v;
}

// ---------------------------------------------------------------------------
// Diagnostics: deterministic FP64 reductions (warp shuffle -> block -> grid)
// ---------------------------------------------------------------------------
// part[b*3 + 0] = sum C/C_inf, [1] = sum H, [2] = non-finite count, for block b
template <typename R>
__global__ void __launch_bounds__(256)
k_diag_partial(const KP<R> P, const R* __restrict__ phi, const R* __restrict__ Um, const R* __restrict__ Tm,
               const R* __restrict__ uxm, const R* __restrict__ uym, double* __restrict__ part) {
    __shared__ double s[3][8];
    double mc = 0.0, h = 0.0, bad = 0.0;
    const long long nn = (long long)P.nx * P.ny;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < nn; n += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(n / P.nx), x = (int)(n - (long long)y * P.nx);
        const size_t node = (size_t)y * P.pitch + x;
        const double ph = (double)phi[node];
        const double U = P.has_U ? (double)Um[node] : 0.0;
        const double T = P.has_T ? (double)Tm[node] : 0.0;
        const double vx = P.has_flow ? (double)uxm[node] : 0.0, vy = P.has_flow ? (double)uym[node] : 0.0;
        const double k = (double)P.k;
        if (P.has_U) mc += 0.5 * (1.0 + (1.0 - k) * U) * ((1.0 + k) - (1.0 - k) * ph);
        if (P.has_T)
            h += (0.5 * (1.0 + ph) * (double)P.cS + 0.5 * (1.0 - ph) * (double)P.cL) * T - 0.5 * (double)P.rhoL_Lh * ph;
        if (!isfinite(ph) || !isfinite(U) || !isfinite(T) || !isfinite(vx) || !isfinite(vy)) bad += 1.0;
    }
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
// out[7] = S_phi, out[8] = J_U; the maxima slots are then cleared.
template <typename R>
__global__ void __launch_bounds__(128)
k_diag_final(const KP<R> P, const double* __restrict__ part, int nblocks, const R* __restrict__ phi, int cx, int cy,
             unsigned long long* __restrict__ smax, double* __restrict__ out) {
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
    // tips: warp d scans direction d (+x, +y, -x, -y) for the outermost crossing
    const int d = warp;
    const int len = (d == 0) ? P.nx - cx : (d == 1) ? P.ny - cy : (d == 2) ? cx + 1 : cy + 1;
    auto at = [&](int k) -> double {
        const int x = (d == 0) ? cx + k : (d == 2) ? cx - k : cx;
        const int y = (d == 1) ? cy + k : (d == 3) ? cy - k : cy;
        return (double)phi[(size_t)y * P.pitch + x];
    };
    int best = -1;
    for (int k = lane; k < len - 1; k += 32)
        if (at(k) >= 0.0 && at(k + 1) < 0.0) best = max(best, k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) {
        double r = 0.0;
        if (len > 0 && at(len - 1) >= 0.0) r = (double)(len - 1);
        else if (best >= 0) { const double a = at(best), b = at(best + 1); r = (double)best + a / (a - b); }
        out[3 + d] = r;
    }
    __syncthreads();
    if (threadIdx.x == 0) { smax[0] = 0ull; smax[1] = 0ull; }
}

__global__ void k_set_clock(long long* clock, long long v) { *clock = v; }
__global__ void k_tick(long long* clock, long long d) { *clock += d; }

}  // namespace lbmk
