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

// first moment of stored populations 1..8 (deviation references cancel for U, T)
template <typename R, typename ST>
__device__ __forceinline__ void first_moment(const ST* __restrict__ f, size_t node, long long plane, R& jx, R& jy) {
    R v[9];
#pragma unroll
    for (int i = 1; i < 9; ++i) v[i] = (R)Cvt<ST>::ld(f[(size_t)(i - 1) * plane + node]);
    jx = v[1] - v[3] + v[5] - v[6] - v[7] + v[8];
    jy = v[2] - v[4] + v[5] + v[6] - v[7] - v[8];
}

// phase populations 1..8 (+ f_0 from phi); DEV: h_i = f_i - w_i phi
template <typename R, typename ST, bool DEV>
__device__ __forceinline__ void load_phase(const ST* __restrict__ f, size_t node, long long plane, R phi, R* v) {
    R s = R(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        R h = (R)Cvt<ST>::ld(f[(size_t)(i - 1) * plane + node]);
        v[i] = DEV ? (wq<R>(i) * phi + h) : h;
        s += v[i];
    }
    v[0] = phi - s;
}

template <typename R> __device__ __forceinline__ R theta_frozen(const KP<R>& P, int y, R t) {
    return P.theta_c + P.fG * ((R)y - P.fy0 - P.fV * t);
}

// ---------------------------------------------------------------------------
// Phase-field update (Eqs. 2-4, 14, 21-24, 26, 18)
// ---------------------------------------------------------------------------
template <typename R, typename ST, bool DEV, int TY>
__global__ void __launch_bounds__(32 * TY)
k_phase(const KP<R> P, const ST* __restrict__ fin, ST* __restrict__ fout, const R* __restrict__ phi,
        R* __restrict__ phin, const R* __restrict__ Um, const R* __restrict__ Tm,
        const long long* __restrict__ clock, long long step_off) {
    constexpr int TX = 32, HX = TX + 2, HY = TY + 2, GX = TX + 4, GY = TY + 4, NT = 32 * TY;
    __shared__ R sphi[GY][GX];
    __shared__ R spost[9][HY][HX];
    __shared__ R sas2[TY][TX];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.y * TX + threadIdx.x;

    for (int p = tid; p < GX * GY; p += NT) {
        const int lx = p % GX, ly = p / GX;
        const int gx = scalar_map(x0 - 2 + lx, P.nx, P.bsx), gy = scalar_map(y0 - 2 + ly, P.ny, P.bsy);
        sphi[ly][lx] = phi[(size_t)gy * P.pitch + gx];
    }
    R tnow = R(0);
    if (P.frozen_T) tnow = (R)((clock ? *clock : 0ll) + step_off) * P.dt_base;
    __syncthreads();

    for (int p = tid; p < HX * HY; p += NT) {
        const int lx = p % HX, ly = p / HX;
        int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
        if (!resolve(gx, P.nx, P.bsx) || !resolve(gy, P.ny, P.bsy)) continue;
        const size_t node = (size_t)gy * P.pitch + gx;
        const R c = sphi[ly + 1][lx + 1];
        R gxv, gyv, as, Nx, Ny;
        iso_grad<R, GX>(sphi, lx + 1, ly + 1, gxv, gyv);
        aniso(gxv, gyv, P.eps, as, Nx, Ny);
        const R a2 = as * as;
        const R s = R(1) / (R(3) * P.dtp * a2 * P.W0sq_tau0 + R(0.5));          // Eq. 24
        const R Us = P.has_U ? Um[node] : R(0);
        R th;
        if (P.has_T) th = (Tm[node] - P.T_shift) * P.inv_T_scale;                // Eq. 5
        else if (P.frozen_T) th = theta_frozen(P, gy, tnow);
        else th = P.theta_c;
        const R one = R(1) - c * c;
        const R Q = c * one - P.lam * (P.Mc * Us + th) * one * one;               // Eq. 4
        R jx, jy;
        first_moment<R, ST>(fin, node, P.plane, jx, jy);                        // DEV refs cancel
        const R bx = -P.dtp * P.W0sq_tau0 * Nx, by = -P.dtp * P.W0sq_tau0 * Ny;  // dt v_n (Eqs. 21-22)
        const R k6 = (R(1) - s) * (R(1) / R(6));
        put_scalar_post<R, HY, HX>(spost, ly, lx, c + P.dtp * Q * P.inv_tau0, bx, by, k6 * (jx - bx), k6 * (jy - by));
        if (lx >= 1 && lx <= TX && ly >= 1 && ly <= TY) sas2[ly - 1][lx - 1] = a2;
    }
    __syncthreads();

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx >= P.nx || gy >= P.ny) return;
    const size_t node = (size_t)gy * P.pitch + gx;
    const R c = sphi[ty + 2][tx + 2];
    const R inva2 = R(1) / sas2[ty][tx];
    R fo[9], fn[9];
    load_phase<R, ST, DEV>(fin, node, P.plane, c, fo);
    R sum = R(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int sx = gx - c_ex[i], sy = gy - c_ey[i];
        const bool wall = (P.bsx != BC_PERIODIC && outside(sx, P.nx)) || (P.bsy != BC_PERIODIC && outside(sy, P.ny));
        const R inc = wall ? spost[c_opp[i]][ty + 1][tx + 1] : spost[i][ty + 1 - c_ey[i]][tx + 1 - c_ex[i]];
        fn[i] = fo[i] + (inc - fo[i]) * inva2;                                  // Eq. 26
        sum += fn[i];
    }
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

template <typename R, int TY>
__global__ void __launch_bounds__(32 * TY)
k_transfer(const KP<R> P, const R* __restrict__ phio, const R* __restrict__ phin, const R* __restrict__ Uin,
           R* __restrict__ Uout, const R* __restrict__ Tin, R* __restrict__ Tout, R* __restrict__ accU,
           R* __restrict__ accT, int acc_reset_U, int acc_reset_T, unsigned long long* __restrict__ smax) {
    constexpr int TX = 32, HX = TX + 2, HY = TY + 2, GX = TX + 4, GY = TY + 4, NT = 32 * TY;
    __shared__ R spn[GY][GX];
    __shared__ R sJx[HY][HX], sJy[HY][HX];
    __shared__ double sred[NT / 32];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.y * TX + threadIdx.x;
    for (int p = tid; p < GX * GY; p += NT) {
        const int lx = p % GX, ly = p / GX;
        const int gx = scalar_map(x0 - 2 + lx, P.nx, P.bsx), gy = scalar_map(y0 - 2 + ly, P.ny, P.bsy);
        spn[ly][lx] = phin[(size_t)gy * P.pitch + gx];
    }
    __syncthreads();
    const R pre = P.at_pre;
    for (int p = tid; p < HX * HY; p += NT) {
        const int lx = p % HX, ly = p / HX;
        int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
        // the node whose J fills this slot, its shared-tile position, and the
        // wall-normal sign flips of a mirrored ghost
        int cx = lx + 1, cy = ly + 1;
        bool fx = false, fy = false;
        if (outside(gx, P.nx)) {
            if (P.bsx == BC_PERIODIC) gx = wrap_idx(gx, P.nx);
            else { gx = (gx < 0) ? (-1 - gx) : (2 * P.nx - 1 - gx); fx = true; cx = gx - (x0 - 2); }
        }
        if (outside(gy, P.ny)) {
            if (P.bsy == BC_PERIODIC) gy = wrap_idx(gy, P.ny);
            else { gy = (gy < 0) ? (-1 - gy) : (2 * P.ny - 1 - gy); fy = true; cy = gy - (y0 - 2); }
        }
        if (gx < 0 || gx >= P.nx || gy < 0 || gy >= P.ny || cx < 1 || cx > GX - 2 || cy < 1 || cy > GY - 2) {
            sJx[ly][lx] = R(0);   // only reached by slots no valid node reads
            sJy[ly][lx] = R(0);
            continue;
        }
        const size_t node = (size_t)gy * P.pitch + gx;
        R gxv, gyv;
        iso_grad<R, GX>(spn, cx, cy, gxv, gyv);
        const R g2 = gxv * gxv + gyv * gyv;
        R nxv = R(0), nyv = R(0);
        if (g2 > R(1e-12)) {
            const R ig = R(1) / sqrt(g2);
            nxv = -gxv * ig;
            nyv = -gyv * ig;
        }
        const R dphi = spn[cy][cx] - phio[node];                                // Eq. 36
        const R Us = P.has_U ? Uin[node] : R(0);
        const R a = pre * (R(1) + (R(1) - P.k) * Us) * dphi;                    // Eq. 37
        sJx[ly][lx] = fx ? -a * nxv : a * nxv;
        sJy[ly][lx] = fy ? -a * nyv : a * nyv;
    }
    __syncthreads();

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int gx = x0 + tx, gy = y0 + ty;
    double mydu = 0.0;
    if (gx < P.nx && gy < P.ny) {
        const size_t node = (size_t)gy * P.pitch + gx;
        const int hx = tx + 1, hy = ty + 1;
        const R div = (sJx[hy][hx + 1] - sJx[hy][hx - 1] + sJy[hy + 1][hx] - sJy[hy - 1][hx]) * (R(1) / R(3)) +
                      ((sJx[hy + 1][hx + 1] + sJy[hy + 1][hx + 1]) + (sJy[hy + 1][hx - 1] - sJx[hy + 1][hx - 1]) -
                       (sJx[hy - 1][hx - 1] + sJy[hy - 1][hx - 1]) + (sJx[hy - 1][hx + 1] - sJy[hy - 1][hx + 1])) *
                          (R(1) / R(12));
        const R pn = spn[ty + 2][tx + 2];
        const R dphi = pn - phio[node];
        if (P.has_U) {
            const R Us = Uin[node];
            const R dU = ((R(1) + (R(1) - P.k) * Us) * dphi - R(2) * div) /
                         ((R(1) + P.k) - (R(1) - P.k) * pn);                       // Eq. 38
            mydu = fabs((double)dU);
            if (!P.accumulated) Uout[node] = Us + dU;                               // Eq. 39
            else accU[node] = (acc_reset_U ? R(0) : accU[node]) + dU;
        }
        if (P.has_T) {
            const R rc = R(0.5) * (R(1) + pn) * P.cS + R(0.5) * (R(1) - pn) * P.cL;
            const R dT = P.rhoL_Lh * dphi / (R(2) * rc);                            // Eq. 38
            if (!P.accumulated) Tout[node] = Tin[node] + dT;
            else accT[node] = (acc_reset_T ? R(0) : accT[node]) + dT;
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
template <typename R, typename ST, bool DEV, int TY, int FIELD>
__global__ void __launch_bounds__(32 * TY)
k_scalar(const KP<R> P, const ST* __restrict__ fin, ST* __restrict__ fout, const R* __restrict__ mac_in,
         R* __restrict__ mac_out, const R* __restrict__ acc, const R* __restrict__ phi, const R* __restrict__ ux,
         const R* __restrict__ uy, unsigned long long* __restrict__ smax) {
    constexpr int TX = 32, HX = TX + 2, HY = TY + 2, GX = TX + 4, GY = TY + 4, NT = 32 * TY;
    __shared__ R sphi[GY][GX];
    __shared__ R spost[9][HY][HX];
    __shared__ double sred[NT / 32];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const R dt = FIELD == 0 ? P.dtU : P.dtT;
    for (int p = tid; p < GX * GY; p += NT) {
        const int lx = p % GX, ly = p / GX;
        const int gx = scalar_map(x0 - 2 + lx, P.nx, P.bsx), gy = scalar_map(y0 - 2 + ly, P.ny, P.bsy);
        sphi[ly][lx] = phi[(size_t)gy * P.pitch + gx];
    }
    __syncthreads();
    for (int p = tid; p < HX * HY; p += NT) {
        const int lx = p % HX, ly = p / HX;
        int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
        if (!resolve(gx, P.nx, P.bsx) || !resolve(gy, P.ny, P.bsy)) continue;
        const size_t node = (size_t)gy * P.pitch + gx;
        R chi = mac_in[node];
        if (P.accumulated) chi += acc[node];                     // coarse-step injection (Sec. 4.4 ablation)
        const R ph = sphi[ly + 1][lx + 1];
        R D, coef;
        if (FIELD == 0) {
            const R den = (R(1) + P.k) - (R(1) - P.k) * ph;
            D = ((R(1) + ph) * P.DS + (R(1) - ph) * P.DL) / den;                  // Eq. 7
            coef = -(R(1) - P.k) * D / den;                                       // Eq. 8, tr
        } else {
            const R rc = R(0.5) * (R(1) + ph) * P.cS + R(0.5) * (R(1) - ph) * P.cL;
            D = (R(0.5) * (R(1) + ph) * P.kS + R(0.5) * (R(1) - ph) * P.kL) / rc; // Eq. 11
            coef = (P.cS - P.cL) / (R(2) * rc) * D;                               // Eq. 12, tr
        }
        const R s = R(1) / (R(3) * dt * D + R(0.5));                              // Eq. 24
        R vx = R(0), vy = R(0);
        if (P.has_flow) { vx = ux[node]; vy = uy[node]; }
        R jx, jy;
        first_moment<R, ST>(fin, node, P.plane, jx, jy);
        const R bx = dt * chi * vx, by = dt * chi * vy;                            // Eqs. 19-20
        const R jnx = jx - bx, jny = jy - by;
        R gpx, gpy;
        iso_grad<R, GX>(sphi, lx + 1, ly + 1, gpx, gpy);
        const R Q = coef * (R(-3) * s) * (jnx * gpx + jny * gpy);                   // Eq. 40 in Eq. 8 / 12
        const R k6 = (R(1) - s) * (R(1) / R(6));
        put_scalar_post<R, HY, HX>(spost, ly, lx, chi + dt * Q, bx, by, k6 * jnx, k6 * jny);
    }
    __syncthreads();
    const int tx = threadIdx.x, ty = threadIdx.y;
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
        if (FIELD == 0 && P.accumulated) myj = fabs((double)acc[node]);
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

template <typename R, typename ST, bool DEV, int TY>
__global__ void __launch_bounds__(32 * TY)
k_flow(const KP<R> P, const ST* __restrict__ fin, ST* __restrict__ fout, const R* __restrict__ phi,
       const R* __restrict__ ux_in, const R* __restrict__ uy_in, const R* __restrict__ rho_in,
       R* __restrict__ ux_out, R* __restrict__ uy_out, R* __restrict__ rho_out) {
    constexpr int TX = 32, HX = TX + 2, HY = TY + 2, NT = 32 * TY;
    __shared__ R sfl[HY][HX];
    __shared__ R spost[9][HY][HX];
    __shared__ R srho[HY][HX], sux[HY][HX], suy[HY][HX];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const R c = P.cF, dt = P.dtF;
    // pass 1: the halo's liquid fractions and the macros written together with
    // the input populations (they decode population 0 and the deviations)
    for (int p = tid; p < HX * HY; p += NT) {
        const int lx = p % HX, ly = p / HX;
        int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
        if (!resolve(gx, P.nx, P.bfx) || !resolve(gy, P.ny, P.bfy)) continue;
        const size_t node = (size_t)gy * P.pitch + gx;
        sfl[ly][lx] = R(0.5) * (R(1) - phi[node]);                                // f_L = (1 - phi)/2
        srho[ly][lx] = rho_in[node];
        sux[ly][lx] = ux_in[node];
        suy[ly][lx] = uy_in[node];
    }
    __syncthreads();
    const R Mi0 = R(1) / R(9), Mi1 = R(1) / R(36), Mi3 = R(1) / R(6), Mi4 = R(1) / R(12), Mi7 = R(1) / R(4);
    for (int p = tid; p < HX * HY; p += NT) {
        const int lx = p % HX, ly = p / HX;
        int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
        if (!resolve(gx, P.nx, P.bfx) || !resolve(gy, P.ny, P.bfy)) continue;
        const size_t node = (size_t)gy * P.pitch + gx;
        const R rho = srho[ly][lx];
        R f[9];
        if (DEV) {
            R ref[9];
            feq_flow<R>(rho, sux[ly][lx], suy[ly][lx], c, ref);
            R s = R(0);
#pragma unroll
            for (int i = 1; i < 9; ++i) { f[i] = ref[i] + (R)Cvt<ST>::ld(fin[(size_t)(i - 1) * P.plane + node]); s += f[i]; }
            f[0] = rho - s;
        } else {
            R s = R(0);
#pragma unroll
            for (int i = 1; i < 9; ++i) { f[i] = (R)Cvt<ST>::ld(fin[(size_t)(i - 1) * P.plane + node]); s += f[i]; }
            f[0] = rho - s;
        }
        const R jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
        const R jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
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
        // Eq. 29 equilibria, Eq. 30 Guo moments, Eq. 31 rates
        const R fu = (P.Fbx * ux + P.Fby * uy) * ic2;
        const R G1 = R(6) * fu, G3 = P.Fbx * ic, G5 = P.Fby * ic;
        const R G7 = R(2) * (P.Fbx * ux - P.Fby * uy) * ic2, G8 = (P.Fby * ux + P.Fbx * uy) * ic2;
        const R d1 = (-P.se * (m1 - rho * (R(-2) + R(3) * u2)) + (R(1) - R(0.5) * P.se) * G1) * Mi1;
        const R d2 = (-P.seps * (m2 - rho * (R(1) - R(3) * u2)) - (R(1) - R(0.5) * P.seps) * G1) * Mi1;
        const R d3 = G3 * Mi3;
        const R d4 = (-P.sq * (m4 + rho * ux * ic) - (R(1) - R(0.5) * P.sq) * G3) * Mi4;
        const R d5 = G5 * Mi3;
        const R d6 = (-P.sq * (m6 + rho * uy * ic) - (R(1) - R(0.5) * P.sq) * G5) * Mi4;
        const R d7 = (-P.snu * (m7 - rho * (ux * ux - uy * uy) * ic2) + (R(1) - R(0.5) * P.snu) * G7) * Mi7;
        const R d8 = (-P.snu * (m8 - rho * ux * uy * ic2) + (R(1) - R(0.5) * P.snu) * G8) * Mi7;
        (void)Mi0;
        // f* = f + M^-1 dm, with M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
        const R axis = -d1 - R(2) * d2, diag = R(2) * d1 + d2;
        spost[0][ly][lx] = f[0] - R(4) * d1 + R(4) * d2;
        spost[1][ly][lx] = f[1] + axis + d3 - R(2) * d4 + d7;
        spost[2][ly][lx] = f[2] + axis + d5 - R(2) * d6 - d7;
        spost[3][ly][lx] = f[3] + axis - d3 + R(2) * d4 + d7;
        spost[4][ly][lx] = f[4] + axis - d5 + R(2) * d6 - d7;
        spost[5][ly][lx] = f[5] + diag + d3 + d4 + d5 + d6 + d8;
        spost[6][ly][lx] = f[6] + diag - d3 - d4 + d5 + d6 - d8;
        spost[7][ly][lx] = f[7] + diag - d3 - d4 - d5 - d6 + d8;
        spost[8][ly][lx] = f[8] + diag + d3 + d4 - d5 - d6 - d8;
    }
    __syncthreads();
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx >= P.nx || gy >= P.ny) return;
    const size_t node = (size_t)gy * P.pitch + gx;
    // streamed value of direction i into the node at shared position (hx, hy),
    // global (nx_, ny_), with the weighted partial bounce-back of Eq. 33
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
    R rho = R(0), jx, jy;
#pragma unroll
    for (int i = 0; i < 9; ++i) rho += fn[i];
    jx = fn[1] - fn[3] + fn[5] - fn[6] - fn[7] + fn[8];
    jy = fn[2] - fn[4] + fn[5] + fn[6] - fn[7] - fn[8];
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
