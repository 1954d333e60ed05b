// Shared device definitions of the multirate MRT-LBM kernels (Liu, Wu, Zhan,
// Secs. 2-3): lattice constants, the coefficient block, storage conversions,
// boundary index maps and the per-node pieces of the collision operators.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <type_traits>

namespace lbmk {

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_INLET_OUTFLOW = 2 };

// D2Q9 velocity set and weights (Eq. 15); the constexpr copies let fully
// unrolled loops resolve directions at compile time
__device__ __constant__ int c_ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ __constant__ int c_ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__device__ __constant__ int c_opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
__host__ __device__ constexpr int ex_of(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0; }
__host__ __device__ constexpr int ey_of(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0; }
__host__ __device__ constexpr int opp_of(int i) { return i == 0 ? 0 : (i < 5 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5); }

template <typename R> struct Wt {
    static constexpr R w0 = R(4) / R(9), w1 = R(1) / R(9), w2 = R(1) / R(36);
};
template <typename R> __host__ __device__ constexpr R wq(int i) {
    return i == 0 ? Wt<R>::w0 : (i < 5 ? Wt<R>::w1 : Wt<R>::w2);
}

// Velocity set of the phase, U and T lattices: Q = 9 (D2Q9, the paper's
// choice for all four fields, Sec. 3.1) or Q = 5 (D2Q5: the rest velocity
// and the four axis links 1..4 of Eq. 15, weights 1/3 and 1/6, the same
// c_s^2 = 1/3, so Eq. 24 ties tau to the diffusivity as on D2Q9).  On D2Q5
// the populations 5..8 do not exist; the kernels treat them as zeros known
// at compile time.
template <typename R, int Q> __host__ __device__ constexpr R wqq(int i) {
    return Q == 9 ? wq<R>(i) : (i == 0 ? R(1) / R(3) : (i < 5 ? R(1) / R(6) : R(0)));
}
// Factor of the first-moment columns of M^-1: e_i / 6 on D2Q9 (columns 3
// and 5 of Eq. 16's inverse), e_i / 2 on D2Q5 (sum_i e_ix^2 = 2 there).
template <typename R, int Q> __host__ __device__ constexpr R kneq() { return Q == 9 ? R(1) / R(6) : R(1) / R(2); }

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
    // bottom wall held at T = T_ymin (anti-bounce-back) instead of zero flux
    int T_dir_ym;
    R T_ymin;
    // crystal angle of each node's grain (pitch layout), or null: Eq. 2 axis-aligned
    const R* ori;
};

// Reciprocal.  FP32: the hardware approximation (PTX rcp.approx.ftz.f32,
// relative error below 2^-22 ~ 1 ulp) -- every reciprocal here is of a
// quantity of order one, and the FP32 path is judged against the FP64 oracle
// with tolerances far above one ulp per step.  FP64: IEEE division, for the
// parity builds.
__device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
// 1/sqrt(x): the CUDA single-precision rsqrtf (within 2 ulp) for FP32, exact
// division of a correctly rounded sqrt for FP64
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }

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
// resolve both coordinates (each is always evaluated)
__device__ __forceinline__ bool resolve_xy(int& x, int& y, int nx, int ny, int bcx, int bcy) {
    const bool a = resolve(x, nx, bcx);
    const bool b = resolve(y, ny, bcy);
    return a && b;
}

// output nodes a kernel path leaves to another one (empty when x0 == x1)
struct Rect {
    int x0, x1, y0, y1;
    __host__ __device__ __forceinline__ bool in(int x, int y) const { return x >= x0 && x < x1 && y >= y0 && y < y1; }
};

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
    const R inv = rcp(g2), inv2 = inv * inv;
    as = R(1) - R(3) * eps + R(4) * eps * (gx2 * gx2 + gy2 * gy2) * inv2;
    const R t = R(16) * eps * as * inv2;
    Nx = t * gx * gy2 * (gx2 - gy2);
    Ny = t * gy * gx2 * (gy2 - gx2);
}

// Kahan-compensated accumulation (the accumulated coupling's phase-change
// sums over the fine steps between two coarse updates): sum s with the
// compensation c of the low-order part lost so far, increment x
template <typename R> __device__ __forceinline__ void kahan_add(R& s, R& c, R x) {
    const R y = x - c;
    const R t = s + y;
    c = (t - s) - y;
    s = t;
}

// sin and cos of one angle: the CUDA fast single-precision intrinsic for
// FP32 (an angle of order one, absolute error ~2^-21), the double-precision
// library routine for FP64
__device__ __forceinline__ void sincos_r(float x, float& s, float& c) { __sincosf(x, &s, &c); }
__device__ __forceinline__ void sincos_r(double x, double& s, double& c) { sincos(x, &s, &c); }

// Eqs. 2-3 for a grain whose crystal axes are turned by vt (grains of
// different orientation): the gradient taken into the crystal frame,
// g' = R(-vt) g, the anisotropy evaluated there, N turned back, N = R(vt) N'
template <typename R>
__device__ __forceinline__ void aniso_frame(R gx, R gy, R eps, R vt, R& as, R& Nx, R& Ny) {
    R s, c;
    sincos_r(vt, s, c);
    R Npx, Npy;
    aniso(c * gx + s * gy, c * gy - s * gx, eps, as, Npx, Npy);
    Nx = c * Npx - s * Npy;
    Ny = s * Npx + c * Npy;
}

// Additions and products in round-to-nearest that the compiler may not
// contract into fused multiply-adds, and the error-free sum of two numbers
// (Knuth's TwoSum: s = fl(a + b) and e with a + b = s + e exactly).
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
template <typename R> __device__ __forceinline__ void two_sum(R a, R b, R& s, R& e) {
    s = add_rn(a, b);
    const R bv = sub_rn(s, a);
    e = add_rn(sub_rn(a, sub_rn(s, bv)), sub_rn(b, bv));
}

// f*_i = w_i A + 3 w_i (e_i . b) + (e_i . c): the scalar collision of Eq. 14
// with S of Eq. 23 in closed form (columns 3 and 5 of M^-1 are e_x/6, e_y/6;
// on D2Q5 e_x/2, e_y/2), A = chi + dt Q, b = j_eq = first moment of f_eq,
// c = (1 - s) j_neq kneq<Q>.  On D2Q5 only populations 0..4 are written.
// The rest population is A minus the moving ones' weight shares, so the nine
// sum to A up to unbiased rounding: the weights rounded to FP32 sum to
// 1 + 7.5e-9 (D2Q9) or 1 + 3.0e-8 (D2Q5), and w_0 A would scale the zeroth
// moment by that every update -- a drift of the conserved solute sum.
template <typename R, int Q> __device__ __forceinline__ R rest_share(R A, R a1, R a2) {
    return Q == 9 ? sub_rn(A, mul_rn(R(4), add_rn(a1, a2))) : sub_rn(A, mul_rn(R(4), a1));
}
// Change of a node's zeroth moment by its streamed populations fn[0..Q-1]
// (Eq. 18) when its own collision took the zeroth moment chi:
// sum_i (fn_i - r_i), with r_i the populations of chi at rest (w_i chi; the
// rest population as the remainder, as rest_share builds it), so that
// chi + streamed_increment = sum_i fn_i in exact arithmetic (sum_i r_i = chi).
// In FP32 the roundings of w_i A in the neighbours' post-collision values and
// of w_i chi here cancel wherever the field is smooth, and a node of a
// uniform region keeps its value exactly; a plain Q-term sum of values of
// order chi carries the correlated roundings of neighbouring nodes into the
// stored macro as a drift.
template <typename R, int Q> __device__ __forceinline__ R streamed_increment(R chi, const R* fn) {
    // rounded products (mul_rn): a contraction of w_i chi into the
    // subtractions below would leave the rounding errors of w_i chi -- the
    // same at every node of a uniform region -- in the increment
    const R r1 = mul_rn(wqq<R, Q>(1), chi), r2 = mul_rn(Wt<R>::w2, chi);
    R d = (fn[0] - rest_share<R, Q>(chi, r1, r2)) + ((fn[1] - r1) + (fn[3] - r1)) + ((fn[2] - r1) + (fn[4] - r1));
    if constexpr (Q == 9) d += ((fn[5] - r2) + (fn[7] - r2)) + ((fn[6] - r2) + (fn[8] - r2));
    return d;
}

// Compensated solute macro.  With FP32 arithmetic the U macro is stored as
// hi (the macro plane, what every other kernel reads) plus a residual lo in
// a third plane of the U state, so that increments far below the last bit of
// hi -- the transport-related source of Eq. 8 and the slow exchange of a
// smooth field are mostly such -- accumulate instead of being rounded away
// update after update (which drifts the solute inventory).  lo is stored in
// BF16 (the plane's first half with FP32 storage): it keeps FP32's exponent
// range -- the residuals lie far below FP16's smallest normal -- and its 8
// bits leave a loss below 2^-9 of hi's last bit per update.  FP64 stores no
// residual.
template <typename ST> struct LoOf { using T = __nv_bfloat16; };
template <typename R> struct Compensated { static constexpr bool value = sizeof(R) == 4; };
// hi + lo + d as a new (hi, lo): hi takes the rounded sum, lo its exact error
// (the error of lo + d itself lies far below lo's last bit)
template <typename R> __device__ __forceinline__ void comp_add(R hi, R lo, R d, R& hi_out, R& lo_out) {
    two_sum(hi, add_rn(lo, d), hi_out, lo_out);
}
// a / b for the phase-change increment of Eq. 38, whose product with the
// denominator must return the numerator for the exact solute balance of the
// transfer.  FP32: the quotient from the hardware reciprocal, q = a rcp(b),
// then one correction by its residual, q + (a - q b) rcp(b) (Newton's step on
// the quotient, Markstein's residual form): the residual is exact in a fused
// multiply-add, so the result is within one unit in the last place and
// carries no systematic part of the reciprocal's error.  FP64: IEEE division.
__device__ __forceinline__ float div_rn(float a, float b) {
    const float r = rcp(b), q = a * r;
    return fmaf(fmaf(-q, b, a), r, q);
}
__device__ __forceinline__ double div_rn(double a, double b) { return a / b; }

template <typename R, int HY, int HX, int Q = 9>
__device__ __forceinline__ void put_scalar_post(R (*sp)[HY][HX], int ly, int lx, R A, R bx, R by, R cx, R cy) {
    const R w1 = wqq<R, Q>(1), w2 = Wt<R>::w2;
    const R a1 = mul_rn(w1, A), a2 = mul_rn(w2, A), b1x = R(3) * w1 * bx, b1y = R(3) * w1 * by;
    const R b2x = R(3) * w2 * bx, b2y = R(3) * w2 * by;
    sp[0][ly][lx] = rest_share<R, Q>(A, a1, a2);
    sp[1][ly][lx] = a1 + b1x + cx;
    sp[2][ly][lx] = a1 + b1y + cy;
    sp[3][ly][lx] = a1 - b1x - cx;
    sp[4][ly][lx] = a1 - b1y - cy;
    if constexpr (Q == 9) {
        sp[5][ly][lx] = a2 + (b2x + b2y) + (cx + cy);
        sp[6][ly][lx] = a2 + (b2y - b2x) + (cy - cx);
        sp[7][ly][lx] = a2 - (b2x + b2y) - (cx + cy);
        sp[8][ly][lx] = a2 + (b2x - b2y) + (cx - cy);
    }
}

template <typename R> __device__ __forceinline__ R theta_frozen(const KP<R>& P, int y, R t) {
    return P.theta_c + P.fG * ((R)y - P.fy0 - P.fV * t);
}

template <typename R>
__device__ __forceinline__ void feq_flow(R rho, R ux, R uy, R c, R* f) {               // Eq. 28
    const R ic = rcp(c), u2 = (ux * ux + uy * uy) * ic * ic;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const R eu = ((R)ex_of(i) * ux + (R)ey_of(i) * uy) * ic;
        f[i] = wq<R>(i) * rho * (R(1) + R(3) * eu + R(4.5) * eu * eu - R(1.5) * u2);
    }
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long* slot, double v) {
    if (v > 0.0) atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}

}  // namespace lbmk
