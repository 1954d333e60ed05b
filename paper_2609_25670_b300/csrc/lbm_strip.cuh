// Warp-strip update kernels of the multirate MRT-LBM (Liu, Wu, Zhan, Secs.
// 3.1-3.3): register-blocked alternative to the shared-memory tiles.
//
// A warp owns a strip of SW = 30 output columns and H output rows.  Lane l
// sits on column 30 s - 1 + l: lanes 1..30 are the strip's columns, lanes 0
// and 31 its left and right neighbours, whose collisions feed the streaming
// of the edge columns.  The warp walks down the strip one row at a time:
// it collides row r (every lane), shifts the post-collision populations that
// move along x one lane with warp shuffles, and completes row r - 1, whose
// nine incoming populations now sit in registers (row r - 2 for e_y = +1,
// row r - 1 for e_y = 0, row r for e_y = -1).  The loads of row r + 1 are
// issued before row r is computed.  There is no shared memory and no block
// barrier; a strip recomputes H + 2 collision rows for H output rows and
// 32 collision columns for 30 output columns.
//
// Isotropic phi gradients (Eq. 40 context, Q2 reading) are formed from the
// column sums A(c) = phi(c, r)/3 + (phi(c, r-1) + phi(c, r+1))/12 and
// B(c) = phi(c, r+1) - phi(c, r-1):  g_x = A(c+1) - A(c-1),
// g_y = B(c)/3 + (B(c-1) + B(c+1))/12, the same nine-point stencil as the
// tile kernels.  Lanes 0 and 31 also load the phi column beyond them.
#pragma once
#include <cuda_pipeline_primitives.h>
#include <stdint.h>
#include <type_traits>
#include "lbm_common.cuh"
#include "lbm_kernels.cuh"

namespace lbmk {

constexpr int SW = 30;     // output columns per strip
constexpr int NWS = 4;     // warps (strips) per block

template <typename R> __device__ __forceinline__ R from_left(R v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <typename R> __device__ __forceinline__ R from_right(R v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// strips whose collisions, phi stencils and outputs all lie inside the
// lattice with a margin: no index maps, no walls
template <int H>
__device__ __forceinline__ bool strip_interior(int sx, int y0, int nx, int ny) {
    return SW * sx - 2 >= 0 && SW * sx + SW + 1 <= nx - 1 && y0 - 2 >= 0 && y0 + H + 1 <= ny - 1;
}

// isotropic gradient at the lane's column from the phi window (rows r-1, r,
// r+1) of the lane's own column (c*) and of the extra column (e*)
template <typename R>
__device__ __forceinline__ void strip_grad(int lane, R cm, R c0, R cp, R em, R e0, R ep, R& gx, R& gy) {
    const R A = c0 * (R(1) / R(3)) + (cm + cp) * (R(1) / R(12)), B = cp - cm;
    const R Ae = e0 * (R(1) / R(3)) + (em + ep) * (R(1) / R(12)), Be = ep - em;
    R Al = from_left(A), Ar = from_right(A), Bl = from_left(B), Br = from_right(B);
    if (lane == 0) { Al = Ae; Bl = Be; }
    if (lane == 31) { Ar = Ae; Br = Be; }
    gx = Ar - Al;
    gy = B * (R(1) / R(3)) + (Bl + Br) * (R(1) / R(12));
}

// post-collision populations of the scalar collision (Eq. 14 with S of
// Eq. 23 in closed form): p_i = w_i A + 3 w_i (e_i . b) + (e_i . c), on the
// Q-velocity lattice (on D2Q5, p_5..p_8 are compile-time zeros); the rest
// population takes the remainder of A (rest_share), so the zeroth moment
// carries no bias from the rounded weights
template <typename R, int Q = 9>
__device__ __forceinline__ void scalar_post9(R A, R bx, R by, R cx, R cy, R* p) {
    const R w1 = wqq<R, Q>(1), w2 = Wt<R>::w2;
    const R a1 = mul_rn(w1, A), a2 = mul_rn(w2, A), b1x = R(3) * w1 * bx, b1y = R(3) * w1 * by;
    const R b2x = R(3) * w2 * bx, b2y = R(3) * w2 * by;
    p[0] = rest_share<R, Q>(A, a1, a2);
    p[1] = a1 + b1x + cx;
    p[2] = a1 + b1y + cy;
    p[3] = a1 - b1x - cx;
    p[4] = a1 - b1y - cy;
    if constexpr (Q == 9) {
        p[5] = a2 + (b2x + b2y) + (cx + cy);
        p[6] = a2 + (b2y - b2x) + (cy - cx);
        p[7] = a2 - (b2x + b2y) - (cx + cy);
        p[8] = a2 + (b2x - b2y) + (cx - cy);
    } else {
        p[5] = p[6] = p[7] = p[8] = R(0);
    }
}
// a diagonal population moved one lane: on D2Q5 there is none to move
template <int Q, typename R> __device__ __forceinline__ R diag_from_left(R v) { return Q == 9 ? from_left(v) : R(0); }
template <int Q, typename R> __device__ __forceinline__ R diag_from_right(R v) { return Q == 9 ? from_right(v) : R(0); }

// U (FIELD 0) or T (FIELD 1) collision at one node: chi the zeroth moment
// (with every injection), (jx, jy) the first moment, (vx, vy) the advecting
// velocity, ph and (gpx, gpy) phi and its gradient (Eqs. 7-8, 10-12, 19-20,
// 24, 40)
// (returns the rounding error of chi + dt Q, as scalar_collide does)
template <typename R, int FIELD, int Q = 9>
__device__ __forceinline__ R scalar_collide9(const KP<R>& P, R ph, R gpx, R gpy, R chi, R jx, R jy, R vx, R vy,
                                             R* p) {
    const R dt = FIELD == 0 ? P.dtU : P.dtT;
    R D, coef;
    if (FIELD == 0) {
        const R iden = rcp((R(1) + P.k) - (R(1) - P.k) * ph);
        D = ((R(1) + ph) * P.DS + (R(1) - ph) * P.DL) * iden;                     // Eq. 7
        coef = -(R(1) - P.k) * D * iden;                                          // Eq. 8, tr
    } else {
        const R irc = rcp(R(0.5) * (R(1) + ph) * P.cS + R(0.5) * (R(1) - ph) * P.cL);
        D = (R(0.5) * (R(1) + ph) * P.kS + R(0.5) * (R(1) - ph) * P.kL) * irc;     // Eq. 11
        coef = R(0.5) * (P.cS - P.cL) * irc * D;                                  // Eq. 12, tr
    }
    const R s = rcp(R(3) * dt * D + R(0.5));                                      // Eq. 24
    const R bx = dt * chi * vx, by = dt * chi * vy;                                // Eqs. 19-20
    const R jnx = jx - bx, jny = jy - by;
    const R Qs = coef * (R(-3) * s) * (jnx * gpx + jny * gpy);                      // Eq. 40 in Eq. 8 / 12
    const R k6 = (R(1) - s) * kneq<R, Q>();
    R A, Ae;
    two_sum(chi, dt * Qs, A, Ae);
    scalar_post9<R, Q>(A, bx, by, k6 * jnx, k6 * jny, p);
    return Ae;
}

// ---------------------------------------------------------------------------
// Row pipeline.  Each lane copies the words its next rows need from global
// to a per-warp shared ring of D row slots with asynchronous copies
// (cp.async through the pipeline primitives), D - 1 rows ahead of the row it
// computes, so the loads in flight do not depend on the registers free.  A
// slot holds NA arrays x 32 lanes of 4-byte words (8-byte for FP64).  A lane
// only reads words it copied itself, so completion of its own copy group is
// the only ordering needed.  16-bit populations are copied as the aligned
// 4-byte word that holds them.  Slots of nodes that do not collide are
// zero-filled.
// ---------------------------------------------------------------------------
template <typename R> using Word = typename std::conditional<sizeof(R) == 8, unsigned long long, unsigned>::type;
template <typename R> struct Pipe { static constexpr int D = sizeof(R) == 8 ? 2 : 4; };

template <typename R, typename T>
__device__ __forceinline__ void fetch_word(Word<R>* dst, const T* a, int idx, bool v) {
    const void* src = a;
    if (v) {
        if constexpr (sizeof(T) >= sizeof(Word<R>)) src = a + idx;
        else src = (const void*)((uintptr_t)(a + idx) & ~(uintptr_t)(sizeof(Word<R>) - 1));
    }
    __pipeline_memcpy_async(dst, src, sizeof(Word<R>), v ? 0 : sizeof(Word<R>));
}
// value of type R from a copied word: the element itself, or the 16-bit half
// selected by the element index parity `odd`
template <typename R, typename T>
__device__ __forceinline__ R word_value(Word<R> w, bool odd) {
    if constexpr (sizeof(T) == sizeof(Word<R>)) {
        T t;
        memcpy(&t, &w, sizeof(T));
        return (R)Cvt<T>::ld(t);
    } else {
        const unsigned short b = (unsigned short)(odd ? (w >> 16) : (w & 0xffffu));
        T t;
        memcpy(&t, &b, sizeof(T));
        return (R)Cvt<T>::ld(t);
    }
}

// slot arrays of the scalar rows: the first moments (j_x, j_y), the macro,
// the accumulator, the velocity, phi of the next row in the lane's and the
// extra column
enum { SA_JX = 0, SA_JY = 1, SA_CHI = 2, SA_ACC = 3, SA_VX = 4, SA_VY = 5, SA_PC = 6, SA_PE = 7, SA_N = 8 };

template <typename R, typename ST, bool IN>
__device__ __forceinline__ void scalar_row_fetch(const KP<R>& P, const ST* __restrict__ fin,
                                                 const R* __restrict__ mac_in, const R* __restrict__ acc,
                                                 const R* __restrict__ phi, const R* __restrict__ ux,
                                                 const R* __restrict__ uy, int cx, bool colv, int px, int ex, int r,
                                                 Word<R>* slot, int lane) {
    const int pl = (int)P.plane;
    int cy = r;
    const bool v = IN || (colv && resolve(cy, P.ny, P.bsy));
    const int node = v ? cy * P.pitch + cx : 0;
    fetch_word<R>(slot + SA_JX * 32 + lane, fin, node, v);
    fetch_word<R>(slot + SA_JY * 32 + lane, fin + pl, node, v);
    fetch_word<R>(slot + SA_CHI * 32 + lane, mac_in, node, v);
    if (P.accumulated) fetch_word<R>(slot + SA_ACC * 32 + lane, acc, node, v);
    if (P.has_flow) {
        fetch_word<R>(slot + SA_VX * 32 + lane, ux, node, v);
        fetch_word<R>(slot + SA_VY * 32 + lane, uy, node, v);
    }
    const int py = IN ? r + 1 : scalar_map(r + 1, P.ny, P.bsy);
    fetch_word<R>(slot + SA_PC * 32 + lane, phi, py * P.pitch + px, true);
    fetch_word<R>(slot + SA_PE * 32 + lane, phi, py * P.pitch + ex, true);
}

template <typename R, typename ST, bool DEV, int H, int FIELD, bool IN, int Q>
__device__ __forceinline__ void scalar_strip(const KP<R>& P, const ST* __restrict__ fin, ST* __restrict__ fout,
                                             const R* __restrict__ mac_in, R* __restrict__ mac_out,
                                             const R* __restrict__ acc, const R* __restrict__ phi,
                                             const R* __restrict__ ux, const R* __restrict__ uy,
                                             unsigned long long* __restrict__ smax, int sx, int y0, Rect skip,
                                             Word<R>* __restrict__ ring) {
    constexpr int D = Pipe<R>::D, NR = H + 2, SLOT = SA_N * 32;
    const int lane = threadIdx.x & 31, pl = (int)P.plane;
    const int gx = SW * sx - 1 + lane;
    int cx = gx;
    const bool colv = IN || resolve(cx, P.nx, P.bsx);
    int px = gx, ex = gx + (lane == 0 ? -1 : (lane == 31 ? 1 : 0));
    if (!IN) {
        px = scalar_map(px, P.nx, P.bsx);
        ex = scalar_map(ex, P.nx, P.bsx);
    }
    const bool odd = (cx & 1) != 0;               // 16-bit word half of this lane's node (pitch and planes even)
    const bool outl = lane >= 1 && lane <= SW && (IN || gx < P.nx);
    // walls beside this column (sources at x - 1 / x + 1 outside)
    const bool wxm = !IN && P.bsx != BC_PERIODIC && gx == 0;
    const bool wxp = !IN && P.bsx != BC_PERIODIC && gx == P.nx - 1;
    // pipeline prologue: collision rows y0-1 .. y0+D-3
#pragma unroll
    for (int d = 0; d < D - 1; ++d) {
        if (d < NR) scalar_row_fetch<R, ST, IN>(P, fin, mac_in, acc, phi, ux, uy, cx, colv, px, ex, y0 - 1 + d,
                                                ring + d * SLOT, lane);
        __pipeline_commit();
    }
    // phi window of the lane's column and of the extra column
    R cm, c0, em, e0;
    {
        const int ya = IN ? y0 - 2 : scalar_map(y0 - 2, P.ny, P.bsy);
        const int yb = IN ? y0 - 1 : scalar_map(y0 - 1, P.ny, P.bsy);
        cm = phi[ya * P.pitch + px]; em = phi[ya * P.pitch + ex];
        c0 = phi[yb * P.pitch + px]; e0 = phi[yb * P.pitch + ex];
    }
    // carried post-collision values: row r-1 (q0, q1s, q3s; q2, q5s, q6s) and
    // row r-2 (z2, z5s, z6s); own unshifted row r-1 for walls (o[])
    R q0 = R(0), q1 = R(0), q3 = R(0), q2 = R(0), q5 = R(0), q6 = R(0), z2 = R(0), z5 = R(0), z6 = R(0);
    R cq = R(0), aq = R(0);                        // row r-1: zeroth moment that entered its collision, source rounding
    R o[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) o[i] = R(0);
    R myj = R(0);
#pragma unroll 1
    for (int k = 0; k < NR; ++k) {
        const int r = y0 - 1 + k;
        if (k + D - 1 < NR)
            scalar_row_fetch<R, ST, IN>(P, fin, mac_in, acc, phi, ux, uy, cx, colv, px, ex, r + D - 1,
                                        ring + ((k + D - 1) % D) * SLOT, lane);
        __pipeline_commit();
        __pipeline_wait_prior(D - 1);             // this lane's copies of row r have landed
        const Word<R>* sl = ring + (k % D) * SLOT + lane;
        const R jx = word_value<R, ST>(sl[SA_JX * 32], odd), jy = word_value<R, ST>(sl[SA_JY * 32], odd);
        R chi = word_value<R, R>(sl[SA_CHI * 32], false), vx = R(0), vy = R(0), accv = R(0);
        if (P.accumulated) { accv = word_value<R, R>(sl[SA_ACC * 32], false); chi += accv; }  // Sec. 4.4 ablation
        if (P.has_flow) { vx = word_value<R, R>(sl[SA_VX * 32], false); vy = word_value<R, R>(sl[SA_VY * 32], false); }
        const R pc = word_value<R, R>(sl[SA_PC * 32], false), pe = word_value<R, R>(sl[SA_PE * 32], false);
        R gpx, gpy;
        strip_grad<R>(lane, cm, c0, pc, em, e0, pe, gpx, gpy);
        R p[9];
        const R ae = scalar_collide9<R, FIELD, Q>(P, c0, gpx, gpy, chi, jx, jy, vx, vy, p);
        const R s1 = from_left(p[1]), s3 = from_right(p[3]), s5 = diag_from_left<Q>(p[5]);
        const R s6 = diag_from_right<Q>(p[6]), s7 = diag_from_right<Q>(p[7]), s8 = diag_from_left<Q>(p[8]);
        const int y = r - 1;                       // row completed in this iteration
        if (FIELD == 0 && P.accumulated && outl && r >= y0 && r < y0 + H && r < P.ny && !skip.in(gx, r))
            myj = fmax(myj, fabs(accv));
        if (k >= 2 && outl && (IN || y < P.ny) && !skip.in(gx, y)) {
            R fn[9];
            fn[0] = q0; fn[1] = q1; fn[3] = q3;    // e_y = 0: row y
            fn[2] = z2; fn[5] = z5; fn[6] = z6;    // e_y = +1: row y - 1
            fn[4] = p[4]; fn[7] = s7; fn[8] = s8;  // e_y = -1: row y + 1
            if (!IN) {                              // bounce-back from own node at walls (Eq. 25 with Q8)
                const bool wym = P.bsy != BC_PERIODIC && y == 0, wyp = P.bsy != BC_PERIODIC && y == P.ny - 1;
                if (wxm) fn[1] = o[3];
                if (wxp) fn[3] = o[1];
                if (wym) fn[2] = o[4];
                if (wyp) fn[4] = o[2];
                if (wxm || wym) fn[5] = o[7];
                if (wxp || wym) fn[6] = o[8];
                if (wxp || wyp) fn[7] = o[5];
                if (wxm || wyp) fn[8] = o[6];
                if (FIELD == 1 && wym && P.T_dir_ym) {      // bottom wall at T_ymin: anti-bounce-back
                    fn[2] = R(2) * wqq<R, Q>(2) * P.T_ymin - o[4];
                    if (Q == 9) {
                        fn[5] = R(2) * Wt<R>::w2 * P.T_ymin - o[7];
                        fn[6] = R(2) * Wt<R>::w2 * P.T_ymin - o[8];
                    }
                }
            }
            const int node = y * P.pitch + gx;
            store_zeroth<R, ST, FIELD>(fin, fout, (size_t)pl, (size_t)node, cq,
                                       streamed_increment<R, Q>(cq, fn) + aq, mac_out);  // Eq. 18
            store_j<R, ST>(fout, node, pl, fn);
        }
        z2 = q2; z5 = q5; z6 = q6;
        q0 = p[0]; q1 = s1; q3 = s3; q2 = p[2]; q5 = s5; q6 = s6;
        cq = chi;
        aq = ae;
        if (!IN) {
#pragma unroll
            for (int i = 0; i < 9; ++i) o[i] = p[i];
        }
        cm = c0; c0 = pc; em = e0; e0 = pe;
    }
    if (FIELD == 0 && P.accumulated) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) myj = fmax(myj, __shfl_xor_sync(0xffffffffu, myj, d));
        if (lane == 0) atomic_max_pos(&smax[1], (double)myj);
    }
}

template <typename R, typename ST, bool DEV, int H, int FIELD, int Q>
__device__ __forceinline__ void scalar_strip_block(const KP<R>& P, const ST* fin, ST* fout, const R* mac_in,
                                                   R* mac_out, const R* acc, const R* phi, const R* ux, const R* uy,
                                                   unsigned long long* smax, int bx, int by) {
    constexpr int RING = Pipe<R>::D * SA_N * 32;
    __shared__ Word<R> ring[NWS * RING];
    const int w = threadIdx.x >> 5;
    const int sx = bx * NWS + w, y0 = by * H;
    if (sx * SW >= P.nx) return;                   // whole warp: past the last strip
    const Rect none{0, 0, 0, 0};
    if (strip_interior<H>(sx, y0, P.nx, P.ny))
        scalar_strip<R, ST, DEV, H, FIELD, true, Q>(P, fin, fout, mac_in, mac_out, acc, phi, ux, uy, smax, sx, y0,
                                                     none, ring + w * RING);
    else
        scalar_strip<R, ST, DEV, H, FIELD, false, Q>(P, fin, fout, mac_in, mac_out, acc, phi, ux, uy, smax, sx, y0,
                                                      none, ring + w * RING);
}

// ---------------------------------------------------------------------------
// Vector strips: VW = 4 consecutive nodes per lane, so every population
// plane and macroscopic array moves as one 16-byte (FP32) word per lane and
// row -- 512 contiguous bytes per warp -- and the x-shifts of the streaming
// and of the phi stencil need one shuffle per direction for four nodes.
// Lane l holds columns 120 s + 4 l .. +3; lanes 1..30 are the strip's 120
// output columns, lanes 0 and 31 its neighbours.  The 16-bit flow strip and
// the 16-bit D2Q5 phase strip, bound by instruction issue and live state,
// take two nodes per lane instead (60 output columns).  Vector strips cover only
// the interior rectangle [VX0, x1) x [VY0, y1) of a lattice (no index maps,
// no walls, rows padded to 32 elements so every vector is aligned); the 1-wide
// strips of the same launch complete the frame around it.
// ---------------------------------------------------------------------------
constexpr int VW = 4;              // nodes per lane
constexpr int VSW = 30 * VW;       // output columns per vector strip
constexpr int VX0 = VW;            // first interior column (strip 0 starts at column 0)
constexpr int VY0 = 2;             // first interior row

struct VGeo {
    int nxv, nyv;                  // vector strips across / down
    Rect in;                       // the interior they cover
};
// V: nodes per lane (VW, or two for the 16-bit flow and 16-bit D2Q5 phase
// strips): strip s covers columns 30 V s .. 30 V s + 32 V - 1 and writes the
// middle 30 V of them
__host__ __device__ inline VGeo vgeo(int nx, int ny, int H, int V = VW) {
    VGeo g;
    g.nxv = nx >= 32 * V ? (nx - 32 * V) / (30 * V) + 1 : 0;        // columns 120 s .. 120 s + 127 inside (V = 4)
    g.nyv = ny - 4 - H >= 0 ? (ny - 4 - H) / H + 1 : 0;            // rows y0 - 2 .. y0 + H + 1 inside
    if (!g.nxv || !g.nyv) g.nxv = g.nyv = 0;
    g.in = Rect{V, V + 30 * V * g.nxv, VY0, VY0 + H * g.nyv};
    return g;
}

// The frame: the units (strips or tiles) of a uw x uh grid over the lattice
// that are not wholly inside the interior rectangle, numbered row by row.
struct Frame {
    int nu, nv;            // units across / down
    int xa, xb, ya, yb;    // the units wholly inside: [xa, xb) x [ya, yb)
    __host__ __device__ int count() const { return nu * nv - (xb - xa) * (yb - ya); }
    // unit f -> (u, v)
    __host__ __device__ void unit(int f, int& u, int& v) const {
        const int top = ya * nu, w = nu - (xb - xa), mid = (yb - ya) * w;
        if (f < top) { v = f / nu; u = f % nu; return; }
        f -= top;
        if (f < mid) {
            v = ya + f / w;
            const int c = f % w;
            u = c < xa ? c : c + (xb - xa);
            return;
        }
        f -= mid;
        v = yb + f / nu;
        u = f % nu;
    }
};
__host__ __device__ inline Frame frame_of(const Rect& in, int nx, int ny, int uw, int uh) {
    Frame f;
    f.nu = (nx + uw - 1) / uw;
    f.nv = (ny + uh - 1) / uh;
    f.xa = (in.x0 + uw - 1) / uw; f.xb = in.x1 / uw;
    f.ya = (in.y0 + uh - 1) / uh; f.yb = in.y1 / uh;
    if (f.xb <= f.xa || f.yb <= f.ya) f.xa = f.xb = f.ya = f.yb = 0;
    return f;
}

template <typename T, int N> struct alignas(sizeof(T) * N) VecN { T v[N]; };
// fused multiply-add in the arithmetic type
__device__ __forceinline__ float fmaf_r(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaf_r(double a, double b, double c) { return fma(a, b, c); }
template <typename T> using Vec4 = VecN<T, VW>;

// a lane's N stored values to and from the arithmetic type; 16-bit types
// convert two at a time (one paired conversion instruction each)
template <typename ST, typename R, int N = VW> __device__ __forceinline__ VecN<ST, N> pack4(const R* v) {
    VecN<ST, N> o;
    if constexpr (std::is_same<ST, __half>::value) {
        __half2* h = reinterpret_cast<__half2*>(o.v);
#pragma unroll
        for (int k = 0; k < N / 2; ++k) h[k] = __floats2half2_rn((float)v[2 * k], (float)v[2 * k + 1]);
    } else if constexpr (std::is_same<ST, __nv_bfloat16>::value) {
        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(o.v);
#pragma unroll
        for (int k = 0; k < N / 2; ++k) h[k] = __floats2bfloat162_rn((float)v[2 * k], (float)v[2 * k + 1]);
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) o.v[k] = Cvt<ST>::st(v[k]);
    }
    return o;
}
template <typename ST, typename R, int N = VW> __device__ __forceinline__ void unpack4(const VecN<ST, N>& in, R* v) {
    if constexpr (std::is_same<ST, __half>::value) {
        const __half2* h = reinterpret_cast<const __half2*>(in.v);
#pragma unroll
        for (int k = 0; k < N / 2; ++k) {
            const float2 a = __half22float2(h[k]);
            v[2 * k] = (R)a.x; v[2 * k + 1] = (R)a.y;
        }
    } else if constexpr (std::is_same<ST, __nv_bfloat16>::value) {
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(in.v);
#pragma unroll
        for (int k = 0; k < N / 2; ++k) {
            const float2 a = __bfloat1622float2(h[k]);
            v[2 * k] = (R)a.x; v[2 * k + 1] = (R)a.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) v[k] = (R)Cvt<ST>::ld(in.v[k]);
    }
}

// asynchronous copy of one lane's vector (N elements of T) into shared memory
template <typename T, int N = VW>
__device__ __forceinline__ void fetch_vec(unsigned char* dst, const T* src) {
    constexpr int B = (int)sizeof(T) * N, C = B < 16 ? B : 16;
#pragma unroll
    for (int o = 0; o < B; o += C) __pipeline_memcpy_async(dst + o, (const unsigned char*)src + o, C);
}
template <typename T, int N = VW> __device__ __forceinline__ VecN<T, N> sread(const unsigned char* p) {
    return *reinterpret_cast<const VecN<T, N>*>(p);
}

enum { VA_JX = 0, VA_JY = 1, VA_CHI = 2, VA_ACC = 3, VA_VX = 4, VA_VY = 5, VA_PHI = 6, VA_LO = 7, VA_N = 8 };
// per-warp ring of row slots, each holding NA arrays of one 16-byte (FP32)
// entry per lane
template <typename R, int NA, int DD = 0> struct VRingN {
    static constexpr int EB = VW * (int)sizeof(R);     // bytes of one lane's entry
    static constexpr int SLOT = NA * 32 * EB;          // one row
    static constexpr int D = DD ? DD : sizeof(R) == 8 ? 2 : 4;   // rows in the ring (D - 1 in flight)
    static constexpr int BYTES = D * SLOT;
};
// scalar strips; with 16-bit storage a ring of three rows (two in flight), so
// that eight blocks (16 warps) fit on an SM
template <typename R, typename ST = R> using VRing = VRingN<R, VA_N, sizeof(ST) == 2 ? 3 : 0>;
constexpr int VNW = 2;     // warps per block of the vector-strip launches

// One vector strip.  UP = false walks rows y0-1 .. y0+H downwards and
// completes row r-1 after colliding row r; UP = true walks y0+H .. y0-1
// upwards and completes row r+1.  Neighbouring strip rows walk in opposite
// directions, so the halo rows two strips share are read close in time (and
// served by L2 the second time).
template <typename R, typename ST, bool DEV, int H, int FIELD, bool UP, int Q>
__device__ __forceinline__ void scalar_vstrip(const KP<R>& P, const ST* __restrict__ fin, ST* __restrict__ fout,
                                              const R* __restrict__ mac_in, R* __restrict__ mac_out,
                                              const R* __restrict__ acc, const R* __restrict__ phi,
                                              const R* __restrict__ ux, const R* __restrict__ uy,
                                              unsigned long long* __restrict__ smax, int s, int y0,
                                              unsigned char* __restrict__ ring) {
    using RG = VRing<R, ST>;
    constexpr int EB = RG::EB, NR = H + 2, D = RG::D, DIR = UP ? -1 : 1;
    const int lane = threadIdx.x & 31, pl = (int)P.plane, pitch = P.pitch;
    const int c0 = VSW * s + VW * lane;
    const bool outl = lane >= 1 && lane <= 30;
    const int rfirst = UP ? y0 + H : y0 - 1;    // first collision row
    unsigned char* const mine = ring + lane * EB;
    constexpr bool COMP = FIELD == 0 && Compensated<R>::value;
    using Lo = typename LoOf<ST>::T;
    auto fetch_row = [&](int r, unsigned char* slot) {      // collision row r, phi row r + DIR
        const int base = r * pitch + c0;
        fetch_vec<ST>(slot + VA_JX * 32 * EB, fin + base);
        fetch_vec<ST>(slot + VA_JY * 32 * EB, fin + (size_t)pl + base);
        fetch_vec<R>(slot + VA_CHI * 32 * EB, mac_in + base);
        if constexpr (COMP) fetch_vec<Lo>(slot + VA_LO * 32 * EB, reinterpret_cast<const Lo*>(fin + 2 * (size_t)pl) + base);
        if (P.accumulated) fetch_vec<R>(slot + VA_ACC * 32 * EB, acc + base);
        if (P.has_flow) {
            fetch_vec<R>(slot + VA_VX * 32 * EB, ux + base);
            fetch_vec<R>(slot + VA_VY * 32 * EB, uy + base);
        }
        fetch_vec<R>(slot + VA_PHI * 32 * EB, phi + base + DIR * pitch);
    };
#pragma unroll
    for (int d = 0; d < D - 1; ++d) {
        fetch_row(rfirst + DIR * d, mine + d * RG::SLOT);
        __pipeline_commit();
    }
    // phi window: the collision row (p0) and the row behind the walk (pb)
    Vec4<R> pb = *reinterpret_cast<const Vec4<R>*>(phi + (rfirst - DIR) * pitch + c0);
    Vec4<R> p0 = *reinterpret_cast<const Vec4<R>*>(phi + rfirst * pitch + c0);
    // carried post-collision values per node: row r - DIR (q0, q1s, q3s and
    // the three populations that move against the walk, qa*), row r - 2 DIR
    // (za*).  Walking down the latter are e_y = +1 (2, 5, 6); walking up,
    // e_y = -1 (4, 7, 8).
    R q0[VW], q1[VW], q3[VW], qa[VW], qb[VW], qc[VW], za[VW], zb[VW], zc[VW];
    // row r - DIR: the zeroth moments that entered its collision, their source
    // rounding errors and (U, FP32 arithmetic) the residuals of the
    // compensated macro
    R cqv[VW], aqv[VW], lqv[VW];
#pragma unroll
    for (int k = 0; k < VW; ++k)
        q0[k] = q1[k] = q3[k] = qa[k] = qb[k] = qc[k] = za[k] = zb[k] = zc[k] = cqv[k] = aqv[k] = lqv[k] = R(0);
    R myj = R(0);
#pragma unroll 1
    for (int it = 0; it < NR; ++it) {
        const int r = rfirst + DIR * it;
        if (it + D - 1 < NR) fetch_row(r + DIR * (D - 1), mine + ((it + D - 1) % D) * RG::SLOT);
        __pipeline_commit();
        __pipeline_wait_prior(D - 1);              // this lane's copies of row r have landed
        const unsigned char* sl = mine + (it % D) * RG::SLOT;
        // first moments of the streamed populations
        R jx[VW], jy[VW];
        unpack4<ST, R>(sread<ST>(sl + VA_JX * 32 * EB), jx);
        unpack4<ST, R>(sread<ST>(sl + VA_JY * 32 * EB), jy);
        Vec4<R> chi = sread<R>(sl + VA_CHI * 32 * EB), accv{}, vx{}, vy{};
        if (P.accumulated) {
            accv = sread<R>(sl + VA_ACC * 32 * EB);
#pragma unroll
            for (int k = 0; k < VW; ++k) chi.v[k] += accv.v[k];                // Sec. 4.4 ablation
        }
        if (P.has_flow) { vx = sread<R>(sl + VA_VX * 32 * EB); vy = sread<R>(sl + VA_VY * 32 * EB); }
        const Vec4<R> pf = sread<R>(sl + VA_PHI * 32 * EB);   // phi row r + DIR
        // phi rows r-1, r, r+1
        const Vec4<R>& pm = UP ? pf : pb;
        const Vec4<R>& pp = UP ? pb : pf;
        // phi gradients of the four nodes (column sums, one shuffle each side)
        R A[VW + 2], B[VW + 2];
#pragma unroll
        for (int k = 0; k < VW; ++k) {
            A[k + 1] = p0.v[k] * (R(1) / R(3)) + (pm.v[k] + pp.v[k]) * (R(1) / R(12));
            B[k + 1] = pp.v[k] - pm.v[k];
        }
        A[0] = from_left(A[VW]); B[0] = from_left(B[VW]);
        A[VW + 1] = from_right(A[1]); B[VW + 1] = from_right(B[1]);
        R p[VW][9], ae[VW], lo_r[VW];
        if constexpr (COMP) unpack4<Lo, R>(sread<Lo>(sl + VA_LO * 32 * EB), lo_r);   // residuals of row r
#pragma unroll
        for (int k = 0; k < VW; ++k) {
            const R gpx = A[k + 2] - A[k], gpy = B[k + 1] * (R(1) / R(3)) + (B[k] + B[k + 2]) * (R(1) / R(12));
            ae[k] = scalar_collide9<R, FIELD, Q>(P, p0.v[k], gpx, gpy, chi.v[k], jx[k], jy[k], vx.v[k], vy.v[k], p[k]);
        }
        // x-shifts: e_x = +1 (1, 5, 8) from the node on the left, e_x = -1 (3, 6, 7) from the right
        R s1[VW], s5[VW], s8[VW], s3[VW], s6[VW], s7[VW];
        s1[0] = from_left(p[VW - 1][1]); s5[0] = diag_from_left<Q>(p[VW - 1][5]); s8[0] = diag_from_left<Q>(p[VW - 1][8]);
        s3[VW - 1] = from_right(p[0][3]); s6[VW - 1] = diag_from_right<Q>(p[0][6]); s7[VW - 1] = diag_from_right<Q>(p[0][7]);
#pragma unroll
        for (int k = 1; k < VW; ++k) { s1[k] = p[k - 1][1]; s5[k] = p[k - 1][5]; s8[k] = p[k - 1][8]; }
#pragma unroll
        for (int k = 0; k < VW - 1; ++k) { s3[k] = p[k + 1][3]; s6[k] = p[k + 1][6]; s7[k] = p[k + 1][7]; }
        if (FIELD == 0 && P.accumulated && outl && r >= y0 && r < y0 + H)
#pragma unroll
            for (int k = 0; k < VW; ++k) myj = fmax(myj, fabs(accv.v[k]));
        if (it >= 2 && outl) {                     // complete row r - DIR
            const int node = (r - DIR) * pitch + c0;
            Vec4<R> sum, lnew;
            R fn[9][VW];
#pragma unroll
            for (int k = 0; k < VW; ++k) {
                fn[0][k] = q0[k]; fn[1][k] = q1[k]; fn[3][k] = q3[k];
                if (!UP) {                         // 2, 5, 6 from the row above; 4, 7, 8 from row r
                    fn[2][k] = za[k]; fn[5][k] = zb[k]; fn[6][k] = zc[k];
                    fn[4][k] = p[k][4]; fn[7][k] = s7[k]; fn[8][k] = s8[k];
                } else {                           // 4, 7, 8 from the row below; 2, 5, 6 from row r
                    fn[4][k] = za[k]; fn[7][k] = zb[k]; fn[8][k] = zc[k];
                    fn[2][k] = p[k][2]; fn[5][k] = s5[k]; fn[6][k] = s6[k];
                }
                R f9[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) f9[i] = fn[i][k];
                const R d = streamed_increment<R, Q>(cqv[k], f9) + aqv[k];
                if constexpr (COMP) comp_add(cqv[k], lqv[k], d, sum.v[k], lnew.v[k]);
                else sum.v[k] = cqv[k] + d;
            }
            *reinterpret_cast<Vec4<R>*>(mac_out + node) = sum;                    // Eq. 18
            if constexpr (COMP) {
                *reinterpret_cast<Vec4<Lo>*>(reinterpret_cast<Lo*>(fout + 2 * (size_t)pl) + node) =
                    pack4<Lo, R>(lnew.v);
            }
            R ox[VW], oy[VW];
#pragma unroll
            for (int k = 0; k < VW; ++k) {
                ox[k] = fn[1][k] - fn[3][k] + fn[5][k] - fn[6][k] - fn[7][k] + fn[8][k];
                oy[k] = fn[2][k] - fn[4][k] + fn[5][k] + fn[6][k] - fn[7][k] - fn[8][k];
            }
            *reinterpret_cast<Vec4<ST>*>(fout + node) = pack4<ST, R>(ox);
            *reinterpret_cast<Vec4<ST>*>(fout + (size_t)pl + node) = pack4<ST, R>(oy);
        }
#pragma unroll
        for (int k = 0; k < VW; ++k) {
            za[k] = qa[k]; zb[k] = qb[k]; zc[k] = qc[k];
            q0[k] = p[k][0]; q1[k] = s1[k]; q3[k] = s3[k];
            if (!UP) { qa[k] = p[k][2]; qb[k] = s5[k]; qc[k] = s6[k]; }
            else { qa[k] = p[k][4]; qb[k] = s7[k]; qc[k] = s8[k]; }
            cqv[k] = chi.v[k];
            aqv[k] = ae[k];
            if constexpr (COMP) lqv[k] = lo_r[k];
        }
        pb = p0;
        p0 = pf;
    }
    if (FIELD == 0 && P.accumulated) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) myj = fmax(myj, __shfl_xor_sync(0xffffffffu, myj, d));
        if (lane == 0) atomic_max_pos(&smax[1], (double)myj);
    }
}

// One launch: blocks [0, nvb) run vector strips over the interior, the rest
// run the 1-wide strips of the whole lattice, skipping those whose outputs
// all lie in the interior.
template <typename R, typename ST = R> struct VSRing {
    static constexpr int V1 = Pipe<R>::D * SA_N * 32 * (int)sizeof(Word<R>);
    static constexpr int BYTES = VRing<R, ST>::BYTES > V1 ? VRing<R, ST>::BYTES : V1;   // per warp
};
__host__ __device__ inline int vs_vector_blocks(const VGeo& g) { return (g.nxv * g.nyv + VNW - 1) / VNW; }
__host__ __device__ inline int vs_blocks(int nx, int ny, int H) {
    const VGeo g = vgeo(nx, ny, H);
    return vs_vector_blocks(g) + (frame_of(g.in, nx, ny, SW, H).count() + VNW - 1) / VNW;
}

template <typename R, typename ST, bool DEV, int H, int FIELD, int Q>
__device__ __forceinline__ void scalar_vs_block(const KP<R>& P, const ST* fin, ST* fout, const R* mac_in, R* mac_out,
                                                const R* acc, const R* phi, const R* ux, const R* uy,
                                                unsigned long long* smax, int b) {
    extern __shared__ __align__(128) unsigned char ring[];    // VNW * VSRing<R, ST>::BYTES, dynamic
    const int w = threadIdx.x >> 5;
    unsigned char* mine = ring + w * VSRing<R, ST>::BYTES;
    const VGeo g = vgeo(P.nx, P.ny, H);
    const int nvb = vs_vector_blocks(g);
    if (b < nvb) {
        const int vs = b * VNW + w;
        if (vs >= g.nxv * g.nyv) return;           // whole warp
        const int sy = vs / g.nxv;
        if (sy & 1)
            scalar_vstrip<R, ST, DEV, H, FIELD, true, Q>(P, fin, fout, mac_in, mac_out, acc, phi, ux, uy, smax,
                                                         vs % g.nxv, VY0 + H * sy, mine);
        else
            scalar_vstrip<R, ST, DEV, H, FIELD, false, Q>(P, fin, fout, mac_in, mac_out, acc, phi, ux, uy, smax,
                                                          vs % g.nxv, VY0 + H * sy, mine);
        return;
    }
    b -= nvb;
    const Rect& in = g.in;
    const Frame fr = frame_of(in, P.nx, P.ny, SW, H);
    const int f = b * VNW + w;
    if (f >= fr.count()) return;                   // whole warp
    int sx, t;
    fr.unit(f, sx, t);
    const int y0 = t * H;
    Word<R>* r1 = reinterpret_cast<Word<R>*>(mine);
    if (strip_interior<H>(sx, y0, P.nx, P.ny))
        scalar_strip<R, ST, DEV, H, FIELD, true, Q>(P, fin, fout, mac_in, mac_out, acc, phi, ux, uy, smax, sx, y0, in, r1);
    else
        scalar_strip<R, ST, DEV, H, FIELD, false, Q>(P, fin, fout, mac_in, mac_out, acc, phi, ux, uy, smax, sx, y0, in, r1);
}

// ---------------------------------------------------------------------------
// Flow vector strips (Eqs. 27-33 in the interior).  Streaming with the
// partial bounce-back of Eq. 33: the population of direction i entering x
// from s = x - e_i is  fLm p_i(s) + (1 - fLm) p_opp(i)(x),  fLm = (f_L(s) +
// f_L(x)) / 2, f_L = (1 - phi)/2, evaluated as p_opp + fLm (p_i - p_opp)
// with the halves f_L / 2 carried, so that each link costs an add, a
// subtraction and a fused multiply-add.  A completed row needs its own nine
// post-collision values and f_L, and (p_i, f_L) of its sources in the rows
// on either side; both are carried in registers as the warp walks.
// ---------------------------------------------------------------------------
enum { FA_RHO = 8, FA_UX = 9, FA_UY = 10, FA_PHI = 11, FA_N = 12 };
// flow strips: 8 populations, rho, u, phi.  With 16-bit populations the
// strip is bound by its instructions and its live state (the nine
// post-collision values of a row and the source values of two rows, per
// node), not by DRAM: it takes two nodes per lane instead of four, which
// halves that state per thread and lets more warps share an SM, and a ring
// of three rows
template <typename ST> constexpr int flow_nodes_per_lane() { return sizeof(ST) == 2 ? 2 : VW; }
template <typename R, typename ST> struct FRing {
    static constexpr int V = flow_nodes_per_lane<ST>();
    static constexpr int EB = V * (int)sizeof(R);            // bytes of one lane's entry
    static constexpr int SLOT = FA_N * 32 * EB;              // one row
    static constexpr int D = sizeof(ST) == 2 ? 3 : sizeof(R) == 8 ? 2 : 4;
    static constexpr int BYTES = D * SLOT;
};

template <typename R, typename ST, bool DEV, int H, bool UP>
__device__ __forceinline__ void flow_vstrip(const KP<R>& P, const ST* __restrict__ fin, ST* __restrict__ fout,
                                            const R* __restrict__ phi, const R* __restrict__ ux_in,
                                            const R* __restrict__ uy_in, const R* __restrict__ rho_in,
                                            R* __restrict__ ux_out, R* __restrict__ uy_out, R* __restrict__ rho_out,
                                            int s, int y0, unsigned char* __restrict__ ring) {
    using RG = FRing<R, ST>;
    constexpr int V = RG::V;                   // nodes per lane
    constexpr int EB = RG::EB, NR = H + 2, D = RG::D, DIR = UP ? -1 : 1;
    // directions whose source lies in the row behind the walk (far) and in
    // the row just collided (near): axis, from the left (e_x = +1), from the right
    constexpr int FAX = UP ? 4 : 2, FL = UP ? 8 : 5, FR = UP ? 7 : 6;
    constexpr int NAX = UP ? 2 : 4, NL = UP ? 5 : 8, NRt = UP ? 6 : 7;
    const int lane = threadIdx.x & 31, pl = (int)P.plane, pitch = P.pitch;
    const R c = P.cF, dt = P.dtF;
    const int c0 = 30 * V * s + V * lane;
    const bool outl = lane >= 1 && lane <= 30;
    const int rfirst = UP ? y0 + H : y0 - 1;
    unsigned char* const mine = ring + lane * EB;
    auto fetch_row = [&](int r, unsigned char* slot) {
        const int base = r * pitch + c0;
#pragma unroll
        for (int i = 1; i < 9; ++i) fetch_vec<ST, V>(slot + (i - 1) * 32 * EB, fin + (size_t)(i - 1) * pl + base);
        fetch_vec<R, V>(slot + FA_RHO * 32 * EB, rho_in + base);
        fetch_vec<R, V>(slot + FA_UX * 32 * EB, ux_in + base);
        fetch_vec<R, V>(slot + FA_UY * 32 * EB, uy_in + base);
        fetch_vec<R, V>(slot + FA_PHI * 32 * EB, phi + base);
    };
#pragma unroll
    for (int d = 0; d < D - 1; ++d) {
        fetch_row(rfirst + DIR * d, mine + d * RG::SLOT);
        __pipeline_commit();
    }
    // row y (the next to complete): own post o, f_L own / left / right, the
    // shifted post values of directions 1, 3 and of the far pair
    R o[9][V], fy[V], fyl[V], fyr[V], q1[V], q3[V], qa[V], qb[V];
    // far row: axis post, shifted pair, f_L own / left / right
    R zx[V], zl[V], zr[V], zf[V], zfl[V], zfr[V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
#pragma unroll
        for (int i = 0; i < 9; ++i) o[i][k] = R(0);
        fy[k] = fyl[k] = fyr[k] = q1[k] = q3[k] = qa[k] = qb[k] = R(0);
        zx[k] = zl[k] = zr[k] = zf[k] = zfl[k] = zfr[k] = R(0);
    }
#pragma unroll 1
    for (int it = 0; it < NR; ++it) {
        const int r = rfirst + DIR * it;
        if (it + D - 1 < NR) fetch_row(r + DIR * (D - 1), mine + ((it + D - 1) % D) * RG::SLOT);
        __pipeline_commit();
        __pipeline_wait_prior(D - 1);
        const unsigned char* sl = mine + (it % D) * RG::SLOT;
        const VecN<R, V> rho = sread<R, V>(sl + FA_RHO * 32 * EB), vx = sread<R, V>(sl + FA_UX * 32 * EB);
        const VecN<R, V> vy = sread<R, V>(sl + FA_UY * 32 * EB), ph = sread<R, V>(sl + FA_PHI * 32 * EB);
        R p[V][9], fl[V], fr[9][V];
#pragma unroll
        for (int i = 1; i < 9; ++i) unpack4<ST, R, V>(sread<ST, V>(sl + (i - 1) * 32 * EB), fr[i]);
#pragma unroll
        for (int k = 0; k < V; ++k) {
            R f[9];
#pragma unroll
            for (int i = 1; i < 9; ++i) f[i] = fr[i][k];
            if (DEV)       // h_i = f_i - w_i rho of the writer's density
#pragma unroll
                for (int i = 1; i < 9; ++i) f[i] += wq<R>(i) * rho.v[k];
            flow_post9<R>(P, f, rho.v[k], p[k]);
            fl[k] = R(0.25) * (R(1) - ph.v[k]);                                      // f_L / 2 = (1 - phi)/4
        }
        // x-shifts of the post values and of f_L
        R s1[V], s5[V], s8[V], s3[V], s6[V], s7[V], fll[V], flr[V];
        s1[0] = from_left(p[V - 1][1]); s5[0] = from_left(p[V - 1][5]); s8[0] = from_left(p[V - 1][8]);
        fll[0] = from_left(fl[V - 1]);
        s3[V - 1] = from_right(p[0][3]); s6[V - 1] = from_right(p[0][6]); s7[V - 1] = from_right(p[0][7]);
        flr[V - 1] = from_right(fl[0]);
#pragma unroll
        for (int k = 1; k < V; ++k) { s1[k] = p[k - 1][1]; s5[k] = p[k - 1][5]; s8[k] = p[k - 1][8]; fll[k] = fl[k - 1]; }
#pragma unroll
        for (int k = 0; k < V - 1; ++k) { s3[k] = p[k + 1][3]; s6[k] = p[k + 1][6]; s7[k] = p[k + 1][7]; flr[k] = fl[k + 1]; }
        R(&sNL)[V] = UP ? s5 : s8;            // near pair, shifted
        R(&sNR)[V] = UP ? s6 : s7;
        if (it >= 2 && outl) {                 // complete row r - DIR
            const int node = (r - DIR) * pitch + c0;
            VecN<R, V> vrho, vux, vuy;
            R fn[9][V];
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const R f0 = fy[k];
                auto pull = [&](int i, R src, R fls) -> R {
                    const R fLm = fls + f0;                  // the mean f_L of the link (halves carried)
                    const R ob = o[opp_of(i)][k];
                    return fmaf_r(fLm, src - ob, ob);
                };
                fn[0][k] = pull(0, o[0][k], f0);
                fn[1][k] = pull(1, q1[k], fyl[k]);
                fn[3][k] = pull(3, q3[k], fyr[k]);
                fn[FAX][k] = pull(FAX, zx[k], zf[k]);
                fn[FL][k] = pull(FL, zl[k], zfl[k]);
                fn[FR][k] = pull(FR, zr[k], zfr[k]);
                fn[NAX][k] = pull(NAX, p[k][NAX], fl[k]);
                fn[NL][k] = pull(NL, sNL[k], fll[k]);
                fn[NRt][k] = pull(NRt, sNR[k], flr[k]);
                R rr = R(0);
#pragma unroll
                for (int i = 0; i < 9; ++i) rr += fn[i][k];
                R g[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) g[i] = fn[i][k];
                const R jx = mom_x(g), jy = mom_y(g);
                const R irho = rcp(rr);
                vrho.v[k] = rr;
                vux.v[k] = (c * jx + R(0.5) * dt * P.Fbx) * irho;                   // Eq. 27
                vuy.v[k] = (c * jy + R(0.5) * dt * P.Fby) * irho;
            }
            *reinterpret_cast<VecN<R, V>*>(rho_out + node) = vrho;
            *reinterpret_cast<VecN<R, V>*>(ux_out + node) = vux;
            *reinterpret_cast<VecN<R, V>*>(uy_out + node) = vuy;
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                R ev[V];
#pragma unroll
                for (int k = 0; k < V; ++k) ev[k] = DEV ? fn[i][k] - wq<R>(i) * vrho.v[k] : fn[i][k];
                *reinterpret_cast<VecN<ST, V>*>(fout + (size_t)(i - 1) * pl + node) = pack4<ST, R, V>(ev);
            }
        }
        // roll: row y becomes the far row, row r becomes row y
#pragma unroll
        for (int k = 0; k < V; ++k) {
            zx[k] = o[FAX][k]; zl[k] = qa[k]; zr[k] = qb[k]; zf[k] = fy[k]; zfl[k] = fyl[k]; zfr[k] = fyr[k];
#pragma unroll
            for (int i = 0; i < 9; ++i) o[i][k] = p[k][i];
            fy[k] = fl[k]; fyl[k] = fll[k]; fyr[k] = flr[k];
            q1[k] = s1[k]; q3[k] = s3[k];
            qa[k] = UP ? s8[k] : s5[k];
            qb[k] = UP ? s7[k] : s6[k];
        }
    }
}

// One launch of blocks of 32 x 4 threads: blocks [0, nvb) run 4 vector strips
// each over the interior, the rest run the 32 x 4 shared-memory tiles of the
// whole lattice (every boundary kind), skipping tiles wholly inside the
// interior and leaving its nodes to the strips.
constexpr int FVW = 4;     // warps per block of the flow vector launch (= tile height of its frame)
template <typename R, typename ST> struct FVSmem {
    static constexpr int STRIPS = FVW * FRing<R, ST>::BYTES;
    static constexpr int TILE = (int)sizeof(FlowSmem<R, FVW>);
    static constexpr int BYTES = STRIPS > TILE ? STRIPS : TILE;
};
__host__ __device__ inline int fvs_vector_blocks(const VGeo& g) { return (g.nxv * g.nyv + FVW - 1) / FVW; }
// blocks of one flow vector launch; V: nodes per lane of its strips
__host__ __device__ inline int fvs_blocks(int nx, int ny, int H, int V = VW) {
    const VGeo g = vgeo(nx, ny, H, V);
    return fvs_vector_blocks(g) + frame_of(g.in, nx, ny, 32, FVW).count();
}

template <typename R, typename ST, bool DEV, int H>
__device__ __forceinline__ void flow_vs_block(const KP<R>& P, const ST* fin, ST* fout, const R* phi, const R* ux_in,
                                              const R* uy_in, const R* rho_in, R* ux_out, R* uy_out, R* rho_out,
                                              int b) {
    extern __shared__ __align__(128) unsigned char fsm[];   // FVSmem<R, ST>::BYTES, dynamic
    const VGeo g = vgeo(P.nx, P.ny, H, flow_nodes_per_lane<ST>());
    const int nvb = fvs_vector_blocks(g);
    if (b < nvb) {
        const int w = threadIdx.y;
        const int vs = b * FVW + w;
        if (vs >= g.nxv * g.nyv) return;           // whole warp (no block barrier on this path)
        const int sy = vs / g.nxv;
        unsigned char* mine = fsm + w * FRing<R, ST>::BYTES;
        if (sy & 1)
            flow_vstrip<R, ST, DEV, H, true>(P, fin, fout, phi, ux_in, uy_in, rho_in, ux_out, uy_out, rho_out,
                                             vs % g.nxv, VY0 + H * sy, mine);
        else
            flow_vstrip<R, ST, DEV, H, false>(P, fin, fout, phi, ux_in, uy_in, rho_in, ux_out, uy_out, rho_out,
                                              vs % g.nxv, VY0 + H * sy, mine);
        return;
    }
    b -= nvb;
    const Rect& in = g.in;
    int u, v;
    frame_of(in, P.nx, P.ny, 32, FVW).unit(b, u, v);
    const int x0 = u * 32, y0 = v * FVW;
    flow_block<R, ST, DEV, FVW>(*reinterpret_cast<FlowSmem<R, FVW>*>(fsm), P, fin, fout, phi, ux_in, uy_in, rho_in,
                                ux_out, uy_out, rho_out, x0, y0, in);
}

// ---------------------------------------------------------------------------
// Phase-change transfer vector strips (Eqs. 36-39 in the interior).  Row r
// forms J = -a grad(phi^{q+1}) / |grad(phi^{q+1})| with a = W0/(2 sqrt 2)
// (1 + (1-k) U*) (phi^{q+1} - phi^q) at its nodes; row r - DIR, whose J
// neighbours are then all known, gets div J (nine-point isotropic stencil
// as column sums) and the increments Delta U, Delta T.
// ---------------------------------------------------------------------------
enum { TA_PN = 0, TA_PO = 1, TA_U = 2, TA_T = 3, TA_AU = 4, TA_AT = 5, TA_N = 6 };
template <typename R> struct TRing {
    static constexpr int EB = VW * (int)sizeof(R);
    static constexpr int SLOT = TA_N * 32 * EB;
    static constexpr int D = 4;
    static constexpr int BYTES = D * SLOT;
};

template <typename R, int H, bool UP, bool ACC>
__device__ __forceinline__ void transfer_vstrip(const KP<R>& P, const R* __restrict__ phio,
                                                const R* __restrict__ phin, const R* __restrict__ Uin,
                                                R* __restrict__ Uout, const R* __restrict__ Tin, R* __restrict__ Tout,
                                                R* __restrict__ accU, R* __restrict__ accT, int acc_reset_U,
                                                int acc_reset_T, unsigned long long* __restrict__ smax, int s, int y0,
                                                unsigned char* __restrict__ ring) {
    using RG = TRing<R>;
    constexpr int EB = RG::EB, NR = H + 2, D = RG::D, DIR = UP ? -1 : 1;
    const int lane = threadIdx.x & 31, pitch = P.pitch;
    const int c0 = VSW * s + VW * lane;
    const bool outl = lane >= 1 && lane <= 30;
    const int rfirst = UP ? y0 + H : y0 - 1;
    const bool ldU = P.has_U, ldT = P.has_T;      // ACC: the accumulated coupling (P.accumulated)
    const bool ldAU = ACC && P.has_U && !acc_reset_U, ldAT = ACC && P.has_T && !acc_reset_T;
    unsigned char* const mine = ring + lane * EB;
    auto fetch_row = [&](int r, unsigned char* slot) {      // phi^{q+1} of row r + DIR; the rest of row r
        const int base = r * pitch + c0;
        fetch_vec<R>(slot + TA_PN * 32 * EB, phin + base + DIR * pitch);
        fetch_vec<R>(slot + TA_PO * 32 * EB, phio + base);
        if (ldU) fetch_vec<R>(slot + TA_U * 32 * EB, Uin + base);
        if (ldT) fetch_vec<R>(slot + TA_T * 32 * EB, Tin + base);
        if (ldAU) fetch_vec<R>(slot + TA_AU * 32 * EB, accU + base);
        if (ldAT) fetch_vec<R>(slot + TA_AT * 32 * EB, accT + base);
    };
#pragma unroll
    for (int d = 0; d < D - 1; ++d) {
        fetch_row(rfirst + DIR * d, mine + d * RG::SLOT);
        __pipeline_commit();
    }
    Vec4<R> pb = *reinterpret_cast<const Vec4<R>*>(phin + (rfirst - DIR) * pitch + c0);
    Vec4<R> p0 = *reinterpret_cast<const Vec4<R>*>(phin + rfirst * pitch + c0);
    const R pre = P.at_pre, omk = R(1) - P.k;
    // row y = r - DIR: its J, phi^{q+1}, phi^q, U*, T, accumulators; row y - DIR: J
    R jxy[VW], jyy[VW], jxz[VW], jyz[VW], pny[VW], poy[VW], Uy[VW], Ty[VW], aUy[VW], aTy[VW];
#pragma unroll
    for (int k = 0; k < VW; ++k)
        jxy[k] = jyy[k] = jxz[k] = jyz[k] = pny[k] = poy[k] = Uy[k] = Ty[k] = aUy[k] = aTy[k] = R(0);
    R mydu = R(0);
#pragma unroll 1
    for (int it = 0; it < NR; ++it) {
        const int r = rfirst + DIR * it;
        if (it + D - 1 < NR) fetch_row(r + DIR * (D - 1), mine + ((it + D - 1) % D) * RG::SLOT);
        __pipeline_commit();
        __pipeline_wait_prior(D - 1);
        const unsigned char* sl = mine + (it % D) * RG::SLOT;
        const Vec4<R> pf = sread<R>(sl + TA_PN * 32 * EB), po = sread<R>(sl + TA_PO * 32 * EB);
        Vec4<R> Us{}, Tv{}, aU{}, aT{};
        if (ldU) Us = sread<R>(sl + TA_U * 32 * EB);
        if (ldT) Tv = sread<R>(sl + TA_T * 32 * EB);
        if (ldAU) aU = sread<R>(sl + TA_AU * 32 * EB);
        if (ldAT) aT = sread<R>(sl + TA_AT * 32 * EB);
        const Vec4<R>& pm = UP ? pf : pb;          // phi^{q+1} rows r-1, r+1
        const Vec4<R>& pp = UP ? pb : pf;
        // grad phi^{q+1} at row r (column sums) and J there (Eqs. 36-37)
        R A[VW + 2], B[VW + 2];
#pragma unroll
        for (int k = 0; k < VW; ++k) {
            A[k + 1] = p0.v[k] * (R(1) / R(3)) + (pm.v[k] + pp.v[k]) * (R(1) / R(12));
            B[k + 1] = pp.v[k] - pm.v[k];
        }
        A[0] = from_left(A[VW]); B[0] = from_left(B[VW]);
        A[VW + 1] = from_right(A[1]); B[VW + 1] = from_right(B[1]);
        R jx[VW], jy[VW];
#pragma unroll
        for (int k = 0; k < VW; ++k) {
            const R gxv = A[k + 2] - A[k], gyv = B[k + 1] * (R(1) / R(3)) + (B[k] + B[k + 2]) * (R(1) / R(12));
            const R g2 = gxv * gxv + gyv * gyv;
            jx[k] = R(0);
            jy[k] = R(0);
            if (g2 > R(1e-12)) {
                const R a = pre * (R(1) + omk * Us.v[k]) * (p0.v[k] - po.v[k]) * rsq(g2);
                jx[k] = -a * gxv;                  // n = -grad phi / |grad phi|
                jy[k] = -a * gyv;
            }
        }
        if (it >= 2) {
            // div J at row y: column sums over rows y-1, y, y+1
            const R(&jxm)[VW] = UP ? jx : jxz;
            const R(&jxp)[VW] = UP ? jxz : jx;
            const R(&jym)[VW] = UP ? jy : jyz;
            const R(&jyp)[VW] = UP ? jyz : jy;
            R Sx[VW + 2], Dy[VW + 2];
#pragma unroll
            for (int k = 0; k < VW; ++k) {
                Sx[k + 1] = jxy[k] * (R(1) / R(3)) + (jxm[k] + jxp[k]) * (R(1) / R(12));
                Dy[k + 1] = jyp[k] - jym[k];
            }
            Sx[0] = from_left(Sx[VW]); Dy[0] = from_left(Dy[VW]);
            Sx[VW + 1] = from_right(Sx[1]); Dy[VW + 1] = from_right(Dy[1]);
            if (outl) {
                const int node = (r - DIR) * pitch + c0;
                Vec4<R> oU, oT, cU{}, cT{};       // Kahan compensations (second plane of the accumulators)
                if constexpr (ACC) {
                    if (ldAU) cU = *reinterpret_cast<const Vec4<R>*>(accU + P.plane + node);
                    if (ldAT) cT = *reinterpret_cast<const Vec4<R>*>(accT + P.plane + node);
                }
#pragma unroll
                for (int k = 0; k < VW; ++k) {
                    const R div = Sx[k + 2] - Sx[k] + Dy[k + 1] * (R(1) / R(3)) + (Dy[k] + Dy[k + 2]) * (R(1) / R(12));
                    const R dphi = pny[k] - poy[k];
                    if (ldU) {
                        const R dU = div_rn((R(1) + omk * Uy[k]) * dphi - R(2) * div, (R(1) + P.k) - omk * pny[k]);  // Eq. 38
                        mydu = fmax(mydu, fabs(dU));
                        if constexpr (ACC) {
                            oU.v[k] = aUy[k];
                            kahan_add(oU.v[k], cU.v[k], dU);
                        } else {
                            oU.v[k] = Uy[k] + dU;                                            // Eq. 39
                        }
                    }
                    if (ldT) {
                        const R rc = R(0.5) * (R(1) + pny[k]) * P.cS + R(0.5) * (R(1) - pny[k]) * P.cL;
                        const R dT = P.rhoL_Lh * dphi * rcp(R(2) * rc);                       // Eq. 38
                        if constexpr (ACC) {
                            oT.v[k] = aTy[k];
                            kahan_add(oT.v[k], cT.v[k], dT);
                        } else {
                            oT.v[k] = Ty[k] + dT;
                        }
                    }
                }
                if (ldU) *reinterpret_cast<Vec4<R>*>((ACC ? accU : Uout) + node) = oU;
                if (ldT) *reinterpret_cast<Vec4<R>*>((ACC ? accT : Tout) + node) = oT;
                if constexpr (ACC) {
                    if (ldU) *reinterpret_cast<Vec4<R>*>(accU + P.plane + node) = cU;
                    if (ldT) *reinterpret_cast<Vec4<R>*>(accT + P.plane + node) = cT;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < VW; ++k) {
            jxz[k] = jxy[k]; jyz[k] = jyy[k]; jxy[k] = jx[k]; jyy[k] = jy[k];
            pny[k] = p0.v[k]; poy[k] = po.v[k]; Uy[k] = Us.v[k]; Ty[k] = Tv.v[k]; aUy[k] = aU.v[k]; aTy[k] = aT.v[k];
        }
        pb = p0;
        p0 = pf;
    }
    if (P.has_U) {           // warp maximum of |Delta U_pc| -> S_phi (and J_U when instantaneous)
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) mydu = fmax(mydu, __shfl_xor_sync(0xffffffffu, mydu, d));
        if (lane == 0) {
            atomic_max_pos(&smax[0], (double)mydu);
            if (!ACC) atomic_max_pos(&smax[1], (double)mydu);
        }
    }
}

constexpr int TVW = 4;     // warps per block of the transfer vector launch (= tile height of its frame)
template <typename R> struct TVSmem {
    static constexpr int STRIPS = TVW * TRing<R>::BYTES;
    static constexpr int TILE = (int)sizeof(TransferSmem<R, TVW>);
    static constexpr int BYTES = STRIPS > TILE ? STRIPS : TILE;
};
__host__ __device__ inline int tvs_vector_blocks(const VGeo& g) { return (g.nxv * g.nyv + TVW - 1) / TVW; }
__host__ __device__ inline int tvs_blocks(int nx, int ny, int H) {
    const VGeo g = vgeo(nx, ny, H);
    return tvs_vector_blocks(g) + frame_of(g.in, nx, ny, 32, TVW).count();
}

template <typename R, int H>
__device__ __forceinline__ void transfer_vs_block(const KP<R>& P, const R* phio, const R* phin, const R* Uin, R* Uout,
                                                  const R* Tin, R* Tout, R* accU, R* accT, int ru, int rt,
                                                  unsigned long long* smax, int b) {
    extern __shared__ __align__(128) unsigned char tsm[];   // TVSmem<R>::BYTES, dynamic
    const VGeo g = vgeo(P.nx, P.ny, H);
    const int nvb = tvs_vector_blocks(g);
    if (b < nvb) {
        const int w = threadIdx.y;
        const int vs = b * TVW + w;
        if (vs >= g.nxv * g.nyv) return;           // whole warp (no block barrier on this path)
        const int sy = vs / g.nxv;
        unsigned char* mine = tsm + w * TRing<R>::BYTES;
        // the accumulated coupling (Kahan sums) and the instantaneous one as
        // separate instantiations: the latter keeps none of the former's code
        if (P.accumulated) {
            if (sy & 1)
                transfer_vstrip<R, H, true, true>(P, phio, phin, Uin, Uout, Tin, Tout, accU, accT, ru, rt, smax,
                                                  vs % g.nxv, VY0 + H * sy, mine);
            else
                transfer_vstrip<R, H, false, true>(P, phio, phin, Uin, Uout, Tin, Tout, accU, accT, ru, rt, smax,
                                                   vs % g.nxv, VY0 + H * sy, mine);
        } else if (sy & 1)
            transfer_vstrip<R, H, true, false>(P, phio, phin, Uin, Uout, Tin, Tout, accU, accT, ru, rt, smax,
                                               vs % g.nxv, VY0 + H * sy, mine);
        else
            transfer_vstrip<R, H, false, false>(P, phio, phin, Uin, Uout, Tin, Tout, accU, accT, ru, rt, smax,
                                                vs % g.nxv, VY0 + H * sy, mine);
        return;
    }
    b -= nvb;
    const Rect& in = g.in;
    int u, v;
    frame_of(in, P.nx, P.ny, 32, TVW).unit(b, u, v);
    const int x0 = u * 32, y0 = v * TVW;
    transfer_block<R, TVW>(*reinterpret_cast<TransferSmem<R, TVW>*>(tsm), P, phio, phin, Uin, Uout, Tin, Tout, accU,
                           accT, ru, rt, smax, x0, y0, in);
}

// ---------------------------------------------------------------------------
// Phase-field vector strips (Eqs. 2-4, 14, 21-24, 26, 18 in the interior).
// The anisotropic streaming of Eq. 26 blends the incoming post-collision
// value with the destination's own pre-collision population,
// f_i <- f_i + (p_i(x - e_i) - f_i) / a_s^2(x), so a completed row also needs
// its own loaded populations and a_s^2, carried from its collision.
// ---------------------------------------------------------------------------
// ring arrays of a phase row: populations 1..Q-1, then phi, U, T and the
// grain angle
template <int Q> struct PA {
    static constexpr int PHI = Q - 1, U = Q, T = Q + 1, ORI = Q + 2, N = Q + 3;
};
// 16-bit D2Q5 populations: the strip is bound by its instructions and its
// live state (the row's own pre-collision populations, a_s^2 and the source
// values of two rows, per node), like the 16-bit flow strip; it takes two
// nodes per lane instead of four and a ring of three rows
template <int Q, typename ST> constexpr int phase_nodes_per_lane() { return (sizeof(ST) == 2 && Q == 5) ? 2 : VW; }
template <typename R, int Q = 9, typename ST = R> struct PRing {
    static constexpr int V = phase_nodes_per_lane<Q, ST>();
    static constexpr int EB = V * (int)sizeof(R);            // bytes of one lane's entry
    static constexpr int SLOT = PA<Q>::N * 32 * EB;          // one row
    // three rows on D2Q5 with 16-bit or FP32 storage (four blocks per SM fit
    // the ring), two in FP64, four on D2Q9
    static constexpr int D = (sizeof(ST) <= 4 && Q == 5) ? 3 : sizeof(R) == 8 ? 2 : 4;
    static constexpr int BYTES = D * SLOT;
};

template <typename R, typename ST, bool DEV, int H, bool UP, int Q>
__device__ __forceinline__ void phase_vstrip(const KP<R>& P, const ST* __restrict__ fin, ST* __restrict__ fout,
                                             const R* __restrict__ phi, R* __restrict__ phin,
                                             const R* __restrict__ Um, const R* __restrict__ Tm, R tnow, int s,
                                             int y0, unsigned char* __restrict__ ring) {
    using RG = PRing<R, Q, ST>;
    constexpr int V = RG::V;                   // nodes per lane
    constexpr int PA_PHI = PA<Q>::PHI, PA_U = PA<Q>::U, PA_T = PA<Q>::T, PA_ORI = PA<Q>::ORI;
    constexpr int EB = RG::EB, NR = H + 2, D = RG::D, DIR = UP ? -1 : 1;
    constexpr int FAX = UP ? 4 : 2, FL = UP ? 8 : 5, FR = UP ? 7 : 6;     // far row: axis, from left, from right
    constexpr int NAX = UP ? 2 : 4, NL = UP ? 5 : 8, NRt = UP ? 6 : 7;    // near row (just collided)
    const int lane = threadIdx.x & 31, pl = (int)P.plane, pitch = P.pitch;
    const int c0 = 30 * V * s + V * lane;
    const bool outl = lane >= 1 && lane <= 30;
    const int rfirst = UP ? y0 + H : y0 - 1;
    unsigned char* const mine = ring + lane * EB;
    auto fetch_row = [&](int r, unsigned char* slot) {      // populations, U, T of row r; phi of row r + DIR
        const int base = r * pitch + c0;
#pragma unroll
        for (int i = 1; i < Q; ++i) fetch_vec<ST, V>(slot + (i - 1) * 32 * EB, fin + (size_t)(i - 1) * pl + base);
        fetch_vec<R, V>(slot + PA_PHI * 32 * EB, phi + base + DIR * pitch);
        if (P.has_U) fetch_vec<R, V>(slot + PA_U * 32 * EB, Um + base);
        if (P.has_T) fetch_vec<R, V>(slot + PA_T * 32 * EB, Tm + base);
        if (P.ori) fetch_vec<R, V>(slot + PA_ORI * 32 * EB, P.ori + base);
    };
#pragma unroll
    for (int d = 0; d < D - 1; ++d) {
        fetch_row(rfirst + DIR * d, mine + d * RG::SLOT);
        __pipeline_commit();
    }
    VecN<R, V> pb = *reinterpret_cast<const VecN<R, V>*>(phi + (rfirst - DIR) * pitch + c0);
    VecN<R, V> p0 = *reinterpret_cast<const VecN<R, V>*>(phi + rfirst * pitch + c0);
    // row y: own loaded populations (raw), phi, a_s^2, post values q0, q1s,
    // q3s and its far triple; far row: za, zb, zc
    R fy[9][V], cy[V], ay[V], q0[V], q1[V], q3[V], qa[V], qb[V], qc[V], za[V], zb[V], zc[V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
#pragma unroll
        for (int i = 1; i < 9; ++i) fy[i][k] = R(0);
        cy[k] = R(0); ay[k] = R(1);
        q0[k] = q1[k] = q3[k] = qa[k] = qb[k] = qc[k] = za[k] = zb[k] = zc[k] = R(0);
    }
    // rows two at a time with 16-bit D2Q5 populations (an instruction-bound
    // strip: the unrolled loop renames the rolled row state instead of
    // copying it); one at a time otherwise, where the larger body cost more
    // than the copies
#pragma unroll (sizeof(ST) == 2 && Q == 5 ? 2 : 1)
    for (int it = 0; it < NR; ++it) {
        const int r = rfirst + DIR * it;
        if (it + D - 1 < NR) fetch_row(r + DIR * (D - 1), mine + ((it + D - 1) % D) * RG::SLOT);
        __pipeline_commit();
        __pipeline_wait_prior(D - 1);
        const unsigned char* sl = mine + (it % D) * RG::SLOT;
        R f[9][V];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            if (i >= Q) {                          // D2Q5: no diagonal populations
#pragma unroll
                for (int k = 0; k < V; ++k) f[i][k] = R(0);
                continue;
            }
            unpack4<ST, R, V>(sread<ST, V>(sl + (i - 1) * 32 * EB), f[i]);
        }
        const VecN<R, V> pf = sread<R, V>(sl + PA_PHI * 32 * EB);
        VecN<R, V> Us{}, Tv{}, Ov{};
        if (P.has_U) Us = sread<R, V>(sl + PA_U * 32 * EB);
        if (P.has_T) Tv = sread<R, V>(sl + PA_T * 32 * EB);
        if (P.ori) Ov = sread<R, V>(sl + PA_ORI * 32 * EB);
        const VecN<R, V>& pm = UP ? pf : pb;
        const VecN<R, V>& pp = UP ? pb : pf;
        R A[V + 2], B[V + 2];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            A[k + 1] = p0.v[k] * (R(1) / R(3)) + (pm.v[k] + pp.v[k]) * (R(1) / R(12));
            B[k + 1] = pp.v[k] - pm.v[k];
        }
        A[0] = from_left(A[V]); B[0] = from_left(B[V]);
        A[V + 1] = from_right(A[1]); B[V + 1] = from_right(B[1]);
        R p[V][9], a2[V];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const R gxv = A[k + 2] - A[k], gyv = B[k + 1] * (R(1) / R(3)) + (B[k] + B[k + 2]) * (R(1) / R(12));
            const R c = p0.v[k];
            R as, Nx, Ny;
            if (P.ori) aniso_frame(gxv, gyv, P.eps, Ov.v[k], as, Nx, Ny);    // grain frame
            else aniso(gxv, gyv, P.eps, as, Nx, Ny);
            a2[k] = as * as;
            const R sv = rcp(R(3) * P.dtp * a2[k] * P.W0sq_tau0 + R(0.5));                // Eq. 24
            R th;
            if (P.has_T) th = (Tv.v[k] - P.T_shift) * P.inv_T_scale;                    // Eq. 5
            else if (P.frozen_T) th = theta_frozen(P, r, tnow);
            else th = P.theta_c;
            const R one = R(1) - c * c;
            const R Qs = c * one - P.lam * (P.Mc * Us.v[k] + th) * one * one;             // Eq. 4
            const R bx = -P.dtp * P.W0sq_tau0 * Nx, by = -P.dtp * P.W0sq_tau0 * Ny;     // dt v_n (Eqs. 21-22)
            const R k6 = (R(1) - sv) * kneq<R, Q>();
            const R jx = f[1][k] - f[3][k] + f[5][k] - f[6][k] - f[7][k] + f[8][k];
            const R jy = f[2][k] - f[4][k] + f[5][k] + f[6][k] - f[7][k] - f[8][k];
            scalar_post9<R, Q>(c + P.dtp * Qs * P.inv_tau0, bx, by, k6 * (jx - bx), k6 * (jy - by), p[k]);
        }
        R s1[V], s5[V], s8[V], s3[V], s6[V], s7[V];
        s1[0] = from_left(p[V - 1][1]); s5[0] = diag_from_left<Q>(p[V - 1][5]); s8[0] = diag_from_left<Q>(p[V - 1][8]);
        s3[V - 1] = from_right(p[0][3]); s6[V - 1] = diag_from_right<Q>(p[0][6]); s7[V - 1] = diag_from_right<Q>(p[0][7]);
#pragma unroll
        for (int k = 1; k < V; ++k) { s1[k] = p[k - 1][1]; s5[k] = p[k - 1][5]; s8[k] = p[k - 1][8]; }
#pragma unroll
        for (int k = 0; k < V - 1; ++k) { s3[k] = p[k + 1][3]; s6[k] = p[k + 1][6]; s7[k] = p[k + 1][7]; }
        R(&sNL)[V] = UP ? s5 : s8;
        R(&sNR)[V] = UP ? s6 : s7;
        if (it >= 2 && outl) {                     // complete row y = r - DIR (Eq. 26, Eq. 18)
            const int node = (r - DIR) * pitch + c0;
            VecN<R, V> sum;
            R fn[9][V];
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const R c = cy[k];
                R fa[9], s8v = R(0);
#pragma unroll
                for (int i = 1; i < 9; ++i) {
                    fa[i] = fy[i][k];
                    if (DEV && i < Q) fa[i] += wqq<R, Q>(i) * c;                     // decode h_i = f_i - w_i phi
                    s8v += fa[i];
                }
                fa[0] = c - s8v;                                                     // population 0 from phi
                R inc[9];
                inc[0] = q0[k]; inc[1] = q1[k]; inc[3] = q3[k];
                inc[FAX] = za[k]; inc[FL] = zb[k]; inc[FR] = zc[k];
                inc[NAX] = p[k][NAX]; inc[NL] = sNL[k]; inc[NRt] = sNR[k];
                const R inva2 = rcp(ay[k]);
                R t = R(0);
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    fn[i][k] = fa[i] + (inc[i] - fa[i]) * inva2;                     // Eq. 26
                    t += fn[i][k];
                }
                sum.v[k] = t;
            }
            *reinterpret_cast<VecN<R, V>*>(phin + node) = sum;
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                R ev[V];
#pragma unroll
                for (int k = 0; k < V; ++k) ev[k] = DEV ? fn[i][k] - wqq<R, Q>(i) * sum.v[k] : fn[i][k];
                const VecN<ST, V> o = pack4<ST, R, V>(ev);
                *reinterpret_cast<VecN<ST, V>*>(fout + (size_t)(i - 1) * pl + node) = o;
            }
        }
#pragma unroll
        for (int k = 0; k < V; ++k) {
            za[k] = qa[k]; zb[k] = qb[k]; zc[k] = qc[k];
            q0[k] = p[k][0]; q1[k] = s1[k]; q3[k] = s3[k];
            qa[k] = p[k][FAX]; qb[k] = UP ? s8[k] : s5[k]; qc[k] = UP ? s7[k] : s6[k];
#pragma unroll
            for (int i = 1; i < 9; ++i) fy[i][k] = f[i][k];
            cy[k] = p0.v[k];
            ay[k] = a2[k];
        }
        pb = p0;
        p0 = pf;
    }
}

constexpr int PVW = 4;     // warps per block of the phase vector launch (= tile height of its frame)
template <typename R, int Q = 9, typename ST = R> struct PVSmem {
    static constexpr int STRIPS = PVW * PRing<R, Q, ST>::BYTES;
    static constexpr int TILE = (int)sizeof(PhaseSmem<R, PVW, Q>);
    static constexpr int BYTES = STRIPS > TILE ? STRIPS : TILE;
};
__host__ __device__ inline int pvs_blocks(int nx, int ny, int H, int V = VW) {
    const VGeo g = vgeo(nx, ny, H, V);
    return (g.nxv * g.nyv + PVW - 1) / PVW + frame_of(g.in, nx, ny, 32, PVW).count();
}

template <typename R, typename ST, bool DEV, int H, int Q>
__device__ __forceinline__ void phase_vs_block(const KP<R>& P, const ST* fin, ST* fout, const R* phi, R* phin,
                                               const R* Um, const R* Tm, const long long* clock, long long off,
                                               int b) {
    extern __shared__ __align__(128) unsigned char psm[];   // PVSmem<R, Q, ST>::BYTES, dynamic
    const VGeo g = vgeo(P.nx, P.ny, H, phase_nodes_per_lane<Q, ST>());
    const int nvb = (g.nxv * g.nyv + PVW - 1) / PVW;
    if (b < nvb) {
        const int w = threadIdx.y;
        const int vs = b * PVW + w;
        if (vs >= g.nxv * g.nyv) return;           // whole warp (no block barrier on this path)
        R tnow = R(0);
        if (P.frozen_T) tnow = (R)((clock ? *clock : 0ll) + off) * P.dt_base;
        const int sy = vs / g.nxv;
        unsigned char* mine = psm + w * PRing<R, Q, ST>::BYTES;
        if (sy & 1)
            phase_vstrip<R, ST, DEV, H, true, Q>(P, fin, fout, phi, phin, Um, Tm, tnow, vs % g.nxv, VY0 + H * sy,
                                                 mine);
        else
            phase_vstrip<R, ST, DEV, H, false, Q>(P, fin, fout, phi, phin, Um, Tm, tnow, vs % g.nxv, VY0 + H * sy,
                                                  mine);
        return;
    }
    b -= nvb;
    int u, v;
    frame_of(g.in, P.nx, P.ny, 32, PVW).unit(b, u, v);
    phase_block<R, ST, DEV, PVW, Q>(*reinterpret_cast<PhaseSmem<R, PVW, Q>*>(psm), P, fin, fout, phi, phin, Um, Tm, clock,
                                 off, u * 32, v * PVW, g.in);
}

}  // namespace lbmk

// ---------------------------------------------------------------------------
// Launch wrappers.  Single simulation: block (bx, by) holds strips
// bx*NWS .. bx*NWS+NWS-1 of strip row by.  Batched ensemble: block b belongs
// to the last job whose first block is <= b (job tables of lbm_kernels.cuh).
// ---------------------------------------------------------------------------

namespace lbmk {

template <typename J>
__device__ __forceinline__ const J& job_block(const J* __restrict__ jobs, int njobs, int b, int& bx, int& by) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].tile0 <= b) lo = mid;
        else hi = mid - 1;
    }
    const J& j = jobs[lo];
    const int t = b - j.tile0;
    bx = t % j.tiles_x;
    by = t / j.tiles_x;
    return j;
}

template <typename R, typename ST, bool DEV, int H, int FIELD, int Q>
__global__ void __launch_bounds__(32 * NWS)
k_scalar_strip(const KP<R>* __restrict__ P, const ST* __restrict__ fin, ST* __restrict__ fout,
               const R* __restrict__ mac_in, R* __restrict__ mac_out, const R* __restrict__ acc,
               const R* __restrict__ phi, const R* __restrict__ ux, const R* __restrict__ uy,
               unsigned long long* __restrict__ smax) {
    scalar_strip_block<R, ST, DEV, H, FIELD, Q>(*P, fin, fout, mac_in, mac_out, acc, phi, ux, uy, smax, blockIdx.x,
                                             blockIdx.y);
}
template <typename R, typename ST, bool DEV, int H, int FIELD, int Q>
__global__ void __launch_bounds__(32 * VNW)
k_scalar_vs(const KP<R>* __restrict__ P, const ST* __restrict__ fin, ST* __restrict__ fout,
            const R* __restrict__ mac_in, R* __restrict__ mac_out, const R* __restrict__ acc,
            const R* __restrict__ phi, const R* __restrict__ ux, const R* __restrict__ uy,
            unsigned long long* __restrict__ smax) {
    scalar_vs_block<R, ST, DEV, H, FIELD, Q>(*P, fin, fout, mac_in, mac_out, acc, phi, ux, uy, smax, blockIdx.x);
}
// The same with 16-bit storage, compiled for the blocks per SM its three-row
// ring allows (eight) where the registers fit, D2Q5; six on D2Q9, whose U
// strip needs more than 128 registers, and for the batched form (its job
// lookup adds registers).  Without a stated minimum the register
// allocator had kept the 16-bit D2Q5 T strip at 96 registers with spills
// inside its row loop.
template <int Q, bool BATCH> constexpr int scalar16_min_blocks() { return Q == 5 && !BATCH ? 8 : 6; }
template <typename R, typename ST, bool DEV, int H, int FIELD, int Q>
__global__ void __launch_bounds__(32 * VNW, scalar16_min_blocks<Q, false>())
k_scalar_vs16(const KP<R>* __restrict__ P, const ST* __restrict__ fin, ST* __restrict__ fout,
              const R* __restrict__ mac_in, R* __restrict__ mac_out, const R* __restrict__ acc,
              const R* __restrict__ phi, const R* __restrict__ ux, const R* __restrict__ uy,
              unsigned long long* __restrict__ smax) {
    scalar_vs_block<R, ST, DEV, H, FIELD, Q>(*P, fin, fout, mac_in, mac_out, acc, phi, ux, uy, smax, blockIdx.x);
}
template <typename R, typename ST, bool DEV, int H, int FIELD, int Q>
constexpr auto scalar_vs_kernel() {
    if constexpr (sizeof(ST) == 2) return &k_scalar_vs16<R, ST, DEV, H, FIELD, Q>;
    else return &k_scalar_vs<R, ST, DEV, H, FIELD, Q>;
}
template <typename R, typename ST, bool DEV, int H, int FIELD, int Q>
__global__ void __launch_bounds__(32 * VNW) k_scalar_vs_batch(const ScalarJob<R, ST>* __restrict__ jobs, int njobs) {
    int bx, by;
    const ScalarJob<R, ST>& j = job_block(jobs, njobs, blockIdx.x, bx, by);
    scalar_vs_block<R, ST, DEV, H, FIELD, Q>(*j.P, j.fin, j.fout, j.mac_in, j.mac_out, j.acc, j.phi, j.ux, j.uy, j.smax,
                                          by * j.tiles_x + bx);
}
template <typename R, typename ST, bool DEV, int H, int FIELD, int Q>
__global__ void __launch_bounds__(32 * VNW, scalar16_min_blocks<Q, true>()) k_scalar_vs16_batch(const ScalarJob<R, ST>* __restrict__ jobs, int njobs) {
    int bx, by;
    const ScalarJob<R, ST>& j = job_block(jobs, njobs, blockIdx.x, bx, by);
    scalar_vs_block<R, ST, DEV, H, FIELD, Q>(*j.P, j.fin, j.fout, j.mac_in, j.mac_out, j.acc, j.phi, j.ux, j.uy, j.smax,
                                          by * j.tiles_x + bx);
}
template <typename R, typename ST, bool DEV, int H, int FIELD, int Q>
constexpr auto scalar_vs_batch_kernel() {
    if constexpr (sizeof(ST) == 2) return &k_scalar_vs16_batch<R, ST, DEV, H, FIELD, Q>;
    else return &k_scalar_vs_batch<R, ST, DEV, H, FIELD, Q>;
}
template <typename R, typename ST, bool DEV, int H, int Q>
__global__ void __launch_bounds__(32 * PVW)
k_phase_vs(const KP<R>* __restrict__ P, const ST* __restrict__ fin, ST* __restrict__ fout, const R* __restrict__ phi,
           R* __restrict__ phin, const R* __restrict__ Um, const R* __restrict__ Tm,
           const long long* __restrict__ clock, long long step_off) {
    phase_vs_block<R, ST, DEV, H, Q>(*P, fin, fout, phi, phin, Um, Tm, clock, step_off, blockIdx.x);
}
// the same with 16-bit D2Q5 populations (two nodes per lane), five blocks (20 warps) per SM
template <typename R, typename ST, bool DEV, int H, int Q>
__global__ void __launch_bounds__(32 * PVW, 5)
k_phase_vs16(const KP<R>* __restrict__ P, const ST* __restrict__ fin, ST* __restrict__ fout, const R* __restrict__ phi,
             R* __restrict__ phin, const R* __restrict__ Um, const R* __restrict__ Tm,
             const long long* __restrict__ clock, long long step_off) {
    phase_vs_block<R, ST, DEV, H, Q>(*P, fin, fout, phi, phin, Um, Tm, clock, step_off, blockIdx.x);
}
// the same with FP32 D2Q5 populations, four blocks (16 warps) per SM: the
// three-row ring and 128 registers (146 unbounded, three blocks)
template <typename R, typename ST, bool DEV, int H, int Q>
__global__ void __launch_bounds__(32 * PVW, 4)
k_phase_vs32(const KP<R>* __restrict__ P, const ST* __restrict__ fin, ST* __restrict__ fout, const R* __restrict__ phi,
             R* __restrict__ phin, const R* __restrict__ Um, const R* __restrict__ Tm,
             const long long* __restrict__ clock, long long step_off) {
    phase_vs_block<R, ST, DEV, H, Q>(*P, fin, fout, phi, phin, Um, Tm, clock, step_off, blockIdx.x);
}
template <typename R, typename ST, bool DEV, int H, int Q>
constexpr auto phase_vs_kernel() {
    if constexpr (sizeof(ST) == 2 && Q == 5) return &k_phase_vs16<R, ST, DEV, H, Q>;
    else if constexpr (sizeof(ST) == 4 && Q == 5) return &k_phase_vs32<R, ST, DEV, H, Q>;
    else return &k_phase_vs<R, ST, DEV, H, Q>;
}
template <typename R, typename ST, bool DEV, int H, int Q>
__global__ void __launch_bounds__(32 * PVW) k_phase_vs_batch(const PhaseJob<R, ST>* __restrict__ jobs, int njobs) {
    int bx, by;
    const PhaseJob<R, ST>& j = job_block(jobs, njobs, blockIdx.x, bx, by);
    phase_vs_block<R, ST, DEV, H, Q>(*j.P, j.fin, j.fout, j.phi, j.phin, j.Um, j.Tm, j.clock, j.off,
                                  by * j.tiles_x + bx);
}
template <typename R, int H>
__global__ void __launch_bounds__(32 * TVW)
k_transfer_vs(const KP<R>* __restrict__ P, const R* __restrict__ phio, const R* __restrict__ phin,
              const R* __restrict__ Uin, R* __restrict__ Uout, const R* __restrict__ Tin, R* __restrict__ Tout,
              R* __restrict__ accU, R* __restrict__ accT, int acc_reset_U, int acc_reset_T,
              unsigned long long* __restrict__ smax) {
    transfer_vs_block<R, H>(*P, phio, phin, Uin, Uout, Tin, Tout, accU, accT, acc_reset_U, acc_reset_T, smax,
                            blockIdx.x);
}
template <typename R, int H>
__global__ void __launch_bounds__(32 * TVW) k_transfer_vs_batch(const TransferJob<R>* __restrict__ jobs, int njobs) {
    int bx, by;
    const TransferJob<R>& j = job_block(jobs, njobs, blockIdx.x, bx, by);
    transfer_vs_block<R, H>(*j.P, j.phio, j.phin, j.Uin, j.Uout, j.Tin, j.Tout, j.accU, j.accT, j.acc_reset_U,
                            j.acc_reset_T, j.smax, by * j.tiles_x + bx);
}
template <typename R, typename ST, bool DEV, int H>
__global__ void __launch_bounds__(32 * FVW)
k_flow_vs(const KP<R>* __restrict__ P, const ST* __restrict__ fin, ST* __restrict__ fout, const R* __restrict__ phi,
          const R* __restrict__ ux_in, const R* __restrict__ uy_in, const R* __restrict__ rho_in,
          R* __restrict__ ux_out, R* __restrict__ uy_out, R* __restrict__ rho_out) {
    flow_vs_block<R, ST, DEV, H>(*P, fin, fout, phi, ux_in, uy_in, rho_in, ux_out, uy_out, rho_out, blockIdx.x);
}
// the same with 16-bit populations, two nodes per lane and five blocks
// (20 warps) per SM: 96 registers and the three-row ring
template <typename R, typename ST, bool DEV, int H>
__global__ void __launch_bounds__(32 * FVW, 5)
k_flow_vs16(const KP<R>* __restrict__ P, const ST* __restrict__ fin, ST* __restrict__ fout, const R* __restrict__ phi,
            const R* __restrict__ ux_in, const R* __restrict__ uy_in, const R* __restrict__ rho_in,
            R* __restrict__ ux_out, R* __restrict__ uy_out, R* __restrict__ rho_out) {
    flow_vs_block<R, ST, DEV, H>(*P, fin, fout, phi, ux_in, uy_in, rho_in, ux_out, uy_out, rho_out, blockIdx.x);
}
template <typename R, typename ST, bool DEV, int H>
constexpr auto flow_vs_kernel() {
    if constexpr (sizeof(ST) == 2) return &k_flow_vs16<R, ST, DEV, H>;
    else return &k_flow_vs<R, ST, DEV, H>;
}
template <typename R, typename ST, bool DEV, int H>
__global__ void __launch_bounds__(32 * FVW) k_flow_vs_batch(const FlowJob<R, ST>* __restrict__ jobs, int njobs) {
    int bx, by;
    const FlowJob<R, ST>& j = job_block(jobs, njobs, blockIdx.x, bx, by);
    flow_vs_block<R, ST, DEV, H>(*j.P, j.fin, j.fout, j.phi, j.ux_in, j.uy_in, j.rho_in, j.ux_out, j.uy_out,
                                 j.rho_out, by * j.tiles_x + bx);
}
template <typename R, typename ST, bool DEV, int H, int FIELD, int Q>
__global__ void __launch_bounds__(32 * NWS) k_scalar_strip_batch(const ScalarJob<R, ST>* __restrict__ jobs, int njobs) {
    int bx, by;
    const ScalarJob<R, ST>& j = job_block(jobs, njobs, blockIdx.x, bx, by);
    scalar_strip_block<R, ST, DEV, H, FIELD, Q>(*j.P, j.fin, j.fout, j.mac_in, j.mac_out, j.acc, j.phi, j.ux, j.uy,
                                             j.smax, bx, by);
}

}  // namespace lbmk
