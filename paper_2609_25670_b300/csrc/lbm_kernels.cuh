// Update kernels of the multirate MRT-LBM (Liu, Wu, Zhan, Secs. 3.1-3.3).
//
// One thread per lattice node, 32 x TY tiles. Every field update is one
// fused pass: the block stages phi on its tile plus a 2-node ghost ring in
// shared memory, collides every node of the tile plus a 1-node ring into
// shared memory (recomputing the ring's collisions instead of exchanging
// them), then each thread pulls its nine post-collision populations and
// writes the streamed result.  All global loads of a block are issued before
// its first barrier.  Tiles whose ghost ring lies inside the lattice take a
// compile-time "interior" path without boundary maps or wall tests.
//
// Velocity sets: the flow is D2Q9; the phase, U and T lattices are D2Q9
// (Q = 9, the paper's choice) or D2Q5 (Q = 5, rest velocity and axis links;
// a template parameter of every phase, U, T and fused-transport kernel, with
// the diagonal populations 5..8 compile-time zeros).
//
// Storage (per field, per ping-pong buffer), planes of `pitch * ny` elements
// of type ST:
//   phase: populations 1..Q-1; flow: populations 1..8; population 0 is never
//          stored, it follows
//          from the node's zeroth moment, which the macroscopic arrays carry:
//          phase f_0 = phi - sum_{i>0} f_i (Eq. 18), flow f_0 = rho -
//          sum_{i>0} f_i (Eq. 27).
//   U, T:  the first moment (j_x, j_y) of the streamed populations, two
//          planes.  The collision uses only the zeroth moment (the macro) and
//          the first moment: Eq. 23 relaxes every other moment to equilibrium
//          at rate one, so nothing else of the populations survives a
//          collision (load_j / store_j).
// With DEV = true the phase and flow planes hold deviations h_i = f_i - ref_i
// in 16 bits: phase ref_i = w_i phi, flow ref_i = w_i rho (the zeroth-order
// part of Eq. 28; the deviation is of order 3 w_i |u| + |f_neq|, one FMA to
// decode or encode).
// The U, T first moments are stored in ST as they are (the first moment of
// w_i chi is zero, so j is already the deviation).
//
// The U and T macros include every phase-change increment already injected
// (Eq. 39).  The injection adds w_i Delta to the populations, which changes
// the zeroth moment by Delta and leaves every first moment unchanged
// (sum w_i e_i = 0); since the collision reads only those two moments, the
// population-side add is carried exactly by the macro alone.
#pragma once
#include "lbm_common.cuh"

namespace lbmk {

// ---------------------------------------------------------------------------
// Work items of a tile: item A of thread (tx, ty) is its own node (halo
// position tx+1, ty+1); item B of threads tid < NR is one of the
// NR = 2(TX+2) + 2 TY positions of the 1-node ring.
// ---------------------------------------------------------------------------
template <int TY>
__device__ __forceinline__ void ring_pos(int t, int& lx, int& ly) {
    constexpr int HX = 34;
    if (t < HX) { lx = t; ly = 0; }
    else if (t < 2 * HX) { lx = t - HX; ly = TY + 1; }
    else if (t < 2 * HX + TY) { lx = 0; ly = t - 2 * HX + 1; }
    else { lx = HX - 1; ly = t - 2 * HX - TY + 1; }
}

// tile + 2-ring inside the lattice (phi stencils need no ghosts)
template <int TY>
__device__ __forceinline__ bool interior2(int x0, int y0, int nx, int ny) {
    return x0 >= 2 && x0 + 34 <= nx && y0 >= 2 && y0 + TY + 2 <= ny;
}

// phi on the tile plus a 2-node ghost ring (scalar boundary rule)
template <typename R, int TY, bool IN>
__device__ __forceinline__ void load_phi_ring2(const KP<R>& P, const R* __restrict__ phi, R (*s)[36], int x0, int y0,
                                               int tid) {
    constexpr int GX = 36, GY = TY + 4, NT = 32 * TY, K = (GX * GY + NT - 1) / NT;
    R v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int p = tid + k * NT;
        if (p < GX * GY) {
            int gx = x0 - 2 + p % GX, gy = y0 - 2 + p / GX;
            if (!IN) {
                gx = scalar_map(gx, P.nx, P.bsx);
                gy = scalar_map(gy, P.ny, P.bsy);
            }
            v[k] = phi[gy * P.pitch + gx];
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int p = tid + k * NT;
        if (p < GX * GY) s[p / GX][p % GX] = v[k];
    }
}

template <typename R, typename ST>
__device__ __forceinline__ void load8(const ST* __restrict__ f, int node, int plane, R* v) {
#pragma unroll
    for (int i = 1; i < 9; ++i) v[i] = (R)Cvt<ST>::ld(f[node + (i - 1) * plane]);
}
// populations 1..Q-1 of a Q-velocity lattice; on D2Q5 populations 5..8 are zero
template <typename R, typename ST, int Q>
__device__ __forceinline__ void loadQ(const ST* __restrict__ f, int node, int plane, R* v) {
#pragma unroll
    for (int i = 1; i < 9; ++i) v[i] = i < Q ? (R)Cvt<ST>::ld(f[node + (i - 1) * plane]) : R(0);
}
template <typename R> __device__ __forceinline__ R mom_x(const R* v) { return v[1] - v[3] + v[5] - v[6] - v[7] + v[8]; }
template <typename R> __device__ __forceinline__ R mom_y(const R* v) { return v[2] - v[4] + v[5] + v[6] - v[7] - v[8]; }

// Stored state of a scalar field (U or T) besides its zeroth moment (the
// macro): the first moment j = sum_i e_i f_i of the streamed populations, two
// planes.  With S of Eq. 23 every moment of the scalar collision except the
// fluxes m3, m5 relaxes to its equilibrium at rate one, so the post-collision
// populations of a node are a function of (chi, j_x, j_y) and of phi, grad phi
// and u there alone (the closed form of put_scalar_post): the eight
// populations never need to be stored.  The injection of Eq. 39 changes only
// the zeroth moment (sum_i w_i e_i = 0) and is carried by the macro.
template <typename R, typename ST>
__device__ __forceinline__ void load_j(const ST* __restrict__ f, int node, int plane, R& jx, R& jy) {
    jx = (R)Cvt<ST>::ld(f[node]);
    jy = (R)Cvt<ST>::ld(f[node + plane]);
}
template <typename R, typename ST>
__device__ __forceinline__ void store_j(ST* __restrict__ f, int node, int plane, const R* fn) {
    f[node] = Cvt<ST>::st(mom_x(fn));
    f[node + plane] = Cvt<ST>::st(mom_y(fn));
}

// walls around an own node: a population of direction i comes from behind a
// wall when its source node gx - e_ix (gy - e_iy) lies outside a WALL side
struct Walls {
    bool xm, xp, ym, yp;
    __device__ __forceinline__ bool hit(int i) const {
        return (ex_of(i) > 0 && xm) || (ex_of(i) < 0 && xp) || (ey_of(i) > 0 && ym) || (ey_of(i) < 0 && yp);
    }
};
template <bool IN>
__device__ __forceinline__ Walls walls_of(int gx, int gy, int nx, int ny, int bcx, int bcy) {
    Walls w{false, false, false, false};
    if (!IN) {
        w.xm = bcx != BC_PERIODIC && gx == 0;
        w.xp = bcx != BC_PERIODIC && gx == nx - 1;
        w.ym = bcy != BC_PERIODIC && gy == 0;
        w.yp = bcy != BC_PERIODIC && gy == ny - 1;
    }
    return w;
}

// ---------------------------------------------------------------------------
// Phase-field update (Eqs. 2-4, 14, 21-24, 26, 18)
// ---------------------------------------------------------------------------
template <typename R, int TY, int Q = 9> struct PhaseSmem {
    R phi[TY + 4][36];
    R post[Q][TY + 2][34];
};

// collision of the phase populations at halo position (lx, ly); returns a_s^2
template <typename R, int TY, int Q>
__device__ __forceinline__ R phase_collide(const KP<R>& P, const R (*sphi)[36], R (*sp)[TY + 2][34], int lx, int ly,
                                           int gy, R jx, R jy, R Us, R Tv, R tnow, R ori) {
    const R c = sphi[ly + 1][lx + 1];
    R gxv, gyv, as, Nx, Ny;
    iso_grad<R, 36>(sphi, lx + 1, ly + 1, gxv, gyv);
    if (P.ori) aniso_frame(gxv, gyv, P.eps, ori, as, Nx, Ny);     // grain frame
    else aniso(gxv, gyv, P.eps, as, Nx, Ny);
    const R a2 = as * as;
    const R s = rcp(R(3) * P.dtp * a2 * P.W0sq_tau0 + R(0.5));                   // Eq. 24
    R th;
    if (P.has_T) th = (Tv - P.T_shift) * P.inv_T_scale;                          // Eq. 5
    else if (P.frozen_T) th = theta_frozen(P, gy, tnow);
    else th = P.theta_c;
    const R one = R(1) - c * c;
    const R Qs = c * one - P.lam * (P.Mc * Us + th) * one * one;                  // Eq. 4
    const R bx = -P.dtp * P.W0sq_tau0 * Nx, by = -P.dtp * P.W0sq_tau0 * Ny;      // dt v_n (Eqs. 21-22)
    const R k6 = (R(1) - s) * kneq<R, Q>();
    put_scalar_post<R, TY + 2, 34, Q>(sp, ly, lx, c + P.dtp * Qs * P.inv_tau0, bx, by, k6 * (jx - bx), k6 * (jy - by));
    return a2;
}

template <typename R, typename ST, bool DEV, int TY, bool IN, int Q>
__device__ __forceinline__ void phase_tile(PhaseSmem<R, TY, Q>& sm, const KP<R>& P, const ST* __restrict__ fin,
                                           ST* __restrict__ fout, const R* __restrict__ phi, R* __restrict__ phin,
                                           const R* __restrict__ Um, const R* __restrict__ Tm, R tnow, int x0,
                                           int y0, Rect skip) {
    constexpr int TX = 32, HX = TX + 2, NR = 2 * HX + 2 * TY;
    static_assert(NR <= 32 * TY, "ring larger than the block");
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int pl = (int)P.plane;
    int ax = x0 + tx, ay = y0 + ty;
    const bool own = IN || (ax < P.nx && ay < P.ny);
    const bool va = IN || resolve_xy(ax, ay, P.nx, P.ny, P.bsx, P.bsy);
    int blx = 0, bly = 0, bx = 0, by = 0;
    bool vb = false;
    if (tid < NR) {
        ring_pos<TY>(tid, blx, bly);
        bx = x0 - 1 + blx;
        by = y0 - 1 + bly;
        vb = IN || resolve_xy(bx, by, P.nx, P.ny, P.bsx, P.bsy);
    }
    const int na = ay * P.pitch + ax, nb = by * P.pitch + bx;
    R fa[9], fb[9];
    R Ua = R(0), Ta = R(0), Ub = R(0), Tb = R(0);
    if (va) {
        loadQ<R, ST, Q>(fin, na, pl, fa);
        if (P.has_U) Ua = Um[na];
        if (P.has_T) Ta = Tm[na];
    }
    if (vb) {
        loadQ<R, ST, Q>(fin, nb, pl, fb);
        if (P.has_U) Ub = Um[nb];
        if (P.has_T) Tb = Tm[nb];
    }
    R Oa = R(0), Ob = R(0);                      // grain angles
    if (P.ori) {
        if (va) Oa = P.ori[na];
        if (vb) Ob = P.ori[nb];
    }
    load_phi_ring2<R, TY, IN>(P, phi, sm.phi, x0, y0, tid);
    __syncthreads();
    R a2own = R(1);
    if (va) a2own = phase_collide<R, TY, Q>(P, sm.phi, sm.post, tx + 1, ty + 1, ay, mom_x(fa), mom_y(fa), Ua, Ta, tnow, Oa);
    if (vb) phase_collide<R, TY, Q>(P, sm.phi, sm.post, blx, bly, by, mom_x(fb), mom_y(fb), Ub, Tb, tnow, Ob);
    __syncthreads();
    if (!own) return;
    const int gx = x0 + tx, gy = y0 + ty;
    if (skip.in(gx, gy)) return;                  // written by the vector strips of the same launch
    const R c = sm.phi[ty + 2][tx + 2];
    const R inva2 = rcp(a2own);
    R s8 = R(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (DEV) fa[i] += wqq<R, Q>(i) * c;      // decode h_i = f_i - w_i phi
        s8 += fa[i];
    }
    fa[0] = c - s8;                              // population 0 from the zeroth moment
    const Walls w = walls_of<IN>(gx, gy, P.nx, P.ny, P.bsx, P.bsy);
    R fn[9], sum = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const R inc = w.hit(i) ? sm.post[opp_of(i)][ty + 1][tx + 1] : sm.post[i][ty + 1 - ey_of(i)][tx + 1 - ex_of(i)];
        fn[i] = fa[i] + (inc - fa[i]) * inva2;                                   // Eq. 26
        sum += fn[i];
    }
    const int node = gy * P.pitch + gx;
    phin[node] = sum;                                                            // Eq. 18
#pragma unroll
    for (int i = 1; i < Q; ++i) fout[node + (i - 1) * pl] = Cvt<ST>::st(DEV ? fn[i] - wqq<R, Q>(i) * sum : fn[i]);
}

template <typename R, typename ST, bool DEV, int TY, int Q>
__device__ __forceinline__ void phase_block(PhaseSmem<R, TY, Q>& sm, const KP<R>& P, const ST* fin, ST* fout,
                                            const R* phi, R* phin, const R* Um, const R* Tm,
                                            const long long* clock, long long off, int x0, int y0,
                                            Rect skip = Rect{0, 0, 0, 0}) {
    R tnow = R(0);
    if (P.frozen_T) tnow = (R)((clock ? *clock : 0ll) + off) * P.dt_base;
    if (interior2<TY>(x0, y0, P.nx, P.ny))
        phase_tile<R, ST, DEV, TY, true, Q>(sm, P, fin, fout, phi, phin, Um, Tm, tnow, x0, y0, skip);
    else phase_tile<R, ST, DEV, TY, false, Q>(sm, P, fin, fout, phi, phin, Um, Tm, tnow, x0, y0, skip);
}

// ---------------------------------------------------------------------------
// Phase-change transfer (Eqs. 36-39)
// ---------------------------------------------------------------------------
template <typename R, int TY> struct TransferSmem {
    R pn[TY + 4][36];
    R Jx[TY + 2][34], Jy[TY + 2][34];
    R red[TY];
};

// map a halo position to the node whose J fills it: periodic wrap, or the
// mirrored node with the wall-normal flips; c = its shared-tile position
__device__ __forceinline__ bool j_source(int& g, int n, int bc, int base, int& c, bool& flip) {
    flip = false;
    if (g >= 0 && g < n) return true;
    if (bc == BC_PERIODIC) { g = wrap_idx(g, n); return true; }
    g = (g < 0) ? (-1 - g) : (2 * n - 1 - g);
    flip = true;
    c = g - base;
    return g >= 0 && g < n;
}

template <typename R, int TY, bool IN>
__device__ __forceinline__ void transfer_tile(TransferSmem<R, TY>& sm, const KP<R>& P, const R* __restrict__ phio,
                                              const R* __restrict__ phin, const R* __restrict__ Uin,
                                              R* __restrict__ Uout, const R* __restrict__ Tin, R* __restrict__ Tout,
                                              R* __restrict__ accU, R* __restrict__ accT, int acc_reset_U,
                                              int acc_reset_T, unsigned long long* __restrict__ smax, int x0, int y0,
                                              Rect skip) {
    constexpr int TX = 32, HX = TX + 2, GX = 36, GY = TY + 4, NT = 32 * TY, NR = 2 * HX + 2 * TY;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    // item A: own halo position; item B: a ring position
    int alx = tx + 1, aly = ty + 1, blx = 0, bly = 0;
    if (tid < NR) ring_pos<TY>(tid, blx, bly);
    int ax = x0 - 1 + alx, ay = y0 - 1 + aly, bx = x0 - 1 + blx, by = y0 - 1 + bly;
    int acx = alx + 1, acy = aly + 1, bcx = blx + 1, bcy = bly + 1;
    bool afx = false, afy = false, bfx = false, bfy = false;
    bool va = true, vb = tid < NR;
    if (!IN) {
        va = j_source(ax, P.nx, P.bsx, x0 - 2, acx, afx) & j_source(ay, P.ny, P.bsy, y0 - 2, acy, afy) &&
             acx >= 1 && acx <= GX - 2 && acy >= 1 && acy <= GY - 2;
        if (tid < NR)
            vb = j_source(bx, P.nx, P.bsx, x0 - 2, bcx, bfx) & j_source(by, P.ny, P.bsy, y0 - 2, bcy, bfy) &&
                 bcx >= 1 && bcx <= GX - 2 && bcy >= 1 && bcy <= GY - 2;
    }
    const int na = ay * P.pitch + ax, nb = by * P.pitch + bx;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool own = (IN || (gx < P.nx && gy < P.ny)) && !skip.in(gx, gy);
    const int node = gy * P.pitch + gx;
    R poa = R(0), Usa = R(0), pob = R(0), Usb = R(0), Town = R(0), accUo = R(0), accTo = R(0);
    R cUo = R(0), cTo = R(0);                     // Kahan compensations of the accumulators (second plane)
    if (va) { poa = phio[na]; if (P.has_U) Usa = Uin[na]; }
    if (vb) { pob = phio[nb]; if (P.has_U) Usb = Uin[nb]; }
    if (own) {
        if (P.has_T) Town = Tin[node];
        if (P.accumulated) {
            if (P.has_U && !acc_reset_U) { accUo = accU[node]; cUo = accU[node + P.plane]; }
            if (P.has_T && !acc_reset_T) { accTo = accT[node]; cTo = accT[node + P.plane]; }
        }
    }
    load_phi_ring2<R, TY, IN>(P, phin, sm.pn, x0, y0, tid);
    __syncthreads();
    const R pre = P.at_pre, omk = R(1) - P.k;
    auto jfill = [&](bool v, int lx, int ly, int cx, int cy, bool fx, bool fy, R po, R Us) {
        R jx = R(0), jy = R(0);
        if (v) {
            R gxv, gyv;
            iso_grad<R, GX>(sm.pn, cx, cy, gxv, gyv);
            const R g2 = gxv * gxv + gyv * gyv;
            if (g2 > R(1e-12)) {
                const R a = pre * (R(1) + omk * Us) * (sm.pn[cy][cx] - po) * rsq(g2);   // Eqs. 36-37
                jx = fx ? a * gxv : -a * gxv;       // n = -grad phi / |grad phi|
                jy = fy ? a * gyv : -a * gyv;
            }
        }
        sm.Jx[ly][lx] = jx;
        sm.Jy[ly][lx] = jy;
    };
    jfill(va, alx, aly, acx, acy, afx, afy, poa, Usa);
    if (tid < NR) jfill(vb, blx, bly, bcx, bcy, bfx, bfy, pob, Usb);
    __syncthreads();
    R mydu = R(0);
    if (own) {
        const int hx = tx + 1, hy = ty + 1;
        const R div = (sm.Jx[hy][hx + 1] - sm.Jx[hy][hx - 1] + sm.Jy[hy + 1][hx] - sm.Jy[hy - 1][hx]) * (R(1) / R(3)) +
                      ((sm.Jx[hy + 1][hx + 1] + sm.Jy[hy + 1][hx + 1]) + (sm.Jy[hy + 1][hx - 1] - sm.Jx[hy + 1][hx - 1]) -
                       (sm.Jx[hy - 1][hx - 1] + sm.Jy[hy - 1][hx - 1]) + (sm.Jx[hy - 1][hx + 1] - sm.Jy[hy - 1][hx + 1])) *
                          (R(1) / R(12));
        const R pn = sm.pn[ty + 2][tx + 2];
        const R dphi = pn - poa;                      // item A of an own node is the node itself
        if (P.has_U) {
            const R dU = div_rn((R(1) + omk * Usa) * dphi - R(2) * div, (R(1) + P.k) - omk * pn);   // Eq. 38
            mydu = fabs(dU);
            if (!P.accumulated) Uout[node] = Usa + dU;                                // Eq. 39
            else {
                kahan_add(accUo, cUo, dU);
                accU[node] = accUo;
                accU[node + P.plane] = cUo;
            }
        }
        if (P.has_T) {
            const R rc = R(0.5) * (R(1) + pn) * P.cS + R(0.5) * (R(1) - pn) * P.cL;
            const R dT = P.rhoL_Lh * dphi * rcp(R(2) * rc);                           // Eq. 38
            if (!P.accumulated) Tout[node] = Town + dT;
            else {
                kahan_add(accTo, cTo, dT);
                accT[node] = accTo;
                accT[node + P.plane] = cTo;
            }
        }
    }
    // block maximum of |Delta U_pc| -> S_phi (and J_U when instantaneous)
    if (P.has_U) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mydu = fmax(mydu, __shfl_xor_sync(0xffffffffu, mydu, o));
        if ((tid & 31) == 0) sm.red[tid >> 5] = mydu;
        __syncthreads();
        if (tid == 0) {
            R m = R(0);
            for (int w = 0; w < NT / 32; ++w) m = fmax(m, sm.red[w]);
            atomic_max_pos(&smax[0], (double)m);
            if (!P.accumulated) atomic_max_pos(&smax[1], (double)m);
        }
    }
}

template <typename R, int TY>
__device__ __forceinline__ void transfer_block(TransferSmem<R, TY>& sm, const KP<R>& P, const R* phio, const R* phin,
                                               const R* Uin, R* Uout, const R* Tin, R* Tout, R* accU, R* accT,
                                               int ru, int rt, unsigned long long* smax, int x0, int y0,
                                               Rect skip = Rect{0, 0, 0, 0}) {
    if (interior2<TY>(x0, y0, P.nx, P.ny))
        transfer_tile<R, TY, true>(sm, P, phio, phin, Uin, Uout, Tin, Tout, accU, accT, ru, rt, smax, x0, y0, skip);
    else transfer_tile<R, TY, false>(sm, P, phio, phin, Uin, Uout, Tin, Tout, accU, accT, ru, rt, smax, x0, y0, skip);
}

// ---------------------------------------------------------------------------
// Concentration / temperature update (Eqs. 7-8, 10-12 tr parts; 14, 19-20,
// 23-25, 40, 18).  FIELD 0 = U, 1 = T.
// ---------------------------------------------------------------------------
template <typename R, int TY, int Q = 9> struct ScalarSmem {
    R phi[TY + 4][36];
    R post[Q][TY + 2][34];
    R red[TY];
};

// sphi: the phase field on a tile of width GXW whose ring is OFF + 1 nodes
// wide, so halo position (lx, ly) of the 1-ring sits at (lx + OFF, ly + OFF)
// Returns the rounding error of A = chi + dt Q (error-free sum): the part of
// the source the post-collision populations could not carry, which the node
// adds to its own zeroth moment when it completes its update.
template <typename R, int TY, int FIELD, int GXW = 36, int OFF = 1, int Q = 9>
__device__ __forceinline__ R scalar_collide(const KP<R>& P, const R (*sphi)[GXW], R (*sp)[TY + 2][34], int lx,
                                            int ly, R chi, R jx, R jy, R vx, R vy) {
    const R dt = FIELD == 0 ? P.dtU : P.dtT;
    const R ph = sphi[ly + OFF][lx + OFF];
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
    R gpx, gpy;
    iso_grad<R, GXW>(sphi, lx + OFF, ly + OFF, gpx, gpy);
    const R Qs = coef * (R(-3) * s) * (jnx * gpx + jny * gpy);                      // Eq. 40 in Eq. 8 / 12
    const R k6 = (R(1) - s) * kneq<R, Q>();
    R A, Ae;
    two_sum(chi, dt * Qs, A, Ae);
    put_scalar_post<R, TY + 2, 34, Q>(sp, ly, lx, A, bx, by, k6 * jnx, k6 * jny);
    return Ae;
}

// The node's new zeroth moment chi + d (d: streamed_increment plus the
// source's rounding error) into mac_out; for U with FP32 arithmetic as the
// compensated pair (hi in mac_out, lo in the third plane of the U state,
// read from fin's and written to fout's).
template <typename R, typename ST, int FIELD>
__device__ __forceinline__ void store_zeroth(const ST* __restrict__ fin, ST* __restrict__ fout, size_t plane,
                                             size_t node, R chi, R d, R* __restrict__ mac_out) {
    if constexpr (FIELD == 0 && Compensated<R>::value) {
        using Lo = typename LoOf<ST>::T;
        const Lo* lin = reinterpret_cast<const Lo*>(fin + 2 * plane);
        Lo* lout = reinterpret_cast<Lo*>(fout + 2 * plane);
        R hi, lo;
        comp_add(chi, (R)Cvt<Lo>::ld(lin[node]), d, hi, lo);
        mac_out[node] = hi;
        lout[node] = Cvt<Lo>::st(lo);
    } else {
        mac_out[node] = chi + d;
    }
}

template <typename R, typename ST, bool DEV, int TY, int FIELD, bool IN, int Q>
__device__ __forceinline__ void scalar_tile(ScalarSmem<R, TY, Q>& sm, const KP<R>& P, const ST* __restrict__ fin,
                                            ST* __restrict__ fout, const R* __restrict__ mac_in,
                                            R* __restrict__ mac_out, const R* __restrict__ acc,
                                            const R* __restrict__ phi, const R* __restrict__ ux,
                                            const R* __restrict__ uy, unsigned long long* __restrict__ smax, int x0,
                                            int y0) {
    constexpr int TX = 32, HX = TX + 2, NT = 32 * TY, NR = 2 * HX + 2 * TY;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int pl = (int)P.plane;
    int ax = x0 + tx, ay = y0 + ty;
    const bool va = IN || resolve_xy(ax, ay, P.nx, P.ny, P.bsx, P.bsy);
    int blx = 0, bly = 0, bx = 0, by = 0;
    bool vb = false;
    if (tid < NR) {
        ring_pos<TY>(tid, blx, bly);
        bx = x0 - 1 + blx;
        by = y0 - 1 + bly;
        vb = IN || resolve_xy(bx, by, P.nx, P.ny, P.bsx, P.bsy);
    }
    const int na = ay * P.pitch + ax, nb = by * P.pitch + bx;
    R jax = R(0), jay = R(0), jbx = R(0), jby = R(0);
    R ca = R(0), cb = R(0), uxa = R(0), uya = R(0), uxb = R(0), uyb = R(0), acca = R(0);
    if (va) {
        load_j<R, ST>(fin, na, pl, jax, jay);
        ca = mac_in[na];
        if (P.accumulated) { acca = acc[na]; ca += acca; }   // coarse-step injection (Sec. 4.4 ablation)
        if (P.has_flow) { uxa = ux[na]; uya = uy[na]; }
    }
    if (vb) {
        load_j<R, ST>(fin, nb, pl, jbx, jby);
        cb = mac_in[nb];
        if (P.accumulated) cb += acc[nb];
        if (P.has_flow) { uxb = ux[nb]; uyb = uy[nb]; }
    }
    load_phi_ring2<R, TY, IN>(P, phi, sm.phi, x0, y0, tid);
    __syncthreads();
    R aea = R(0);
    if (va) aea = scalar_collide<R, TY, FIELD, 36, 1, Q>(P, sm.phi, sm.post, tx + 1, ty + 1, ca, jax, jay, uxa, uya);
    if (vb) scalar_collide<R, TY, FIELD, 36, 1, Q>(P, sm.phi, sm.post, blx, bly, cb, jbx, jby, uxb, uyb);
    __syncthreads();
    const int gx = x0 + tx, gy = y0 + ty;
    R myj = R(0);
    if (IN || (gx < P.nx && gy < P.ny)) {
        const int node = gy * P.pitch + gx;
        const Walls w = walls_of<IN>(gx, gy, P.nx, P.ny, P.bsx, P.bsy);
        R fn[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (i >= Q) { fn[i] = R(0); continue; }                                   // D2Q5: no diagonals
            fn[i] = w.hit(i) ? sm.post[opp_of(i)][ty + 1][tx + 1] : sm.post[i][ty + 1 - ey_of(i)][tx + 1 - ex_of(i)]; // Eq. 25
            if (FIELD == 1 && !IN && ey_of(i) > 0 && w.ym && P.T_dir_ym)              // bottom wall at T_ymin
                fn[i] = R(2) * wqq<R, Q>(i) * P.T_ymin - sm.post[opp_of(i)][ty + 1][tx + 1];
        }
        store_zeroth<R, ST, FIELD>(fin, fout, (size_t)pl, (size_t)node, ca,
                                   streamed_increment<R, Q>(ca, fn) + aea, mac_out);     // Eq. 18
        store_j<R, ST>(fout, node, pl, fn);
        if (FIELD == 0 && P.accumulated) myj = fabs(acca);
    }
    if (FIELD == 0 && P.accumulated) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) myj = fmax(myj, __shfl_xor_sync(0xffffffffu, myj, o));
        if ((tid & 31) == 0) sm.red[tid >> 5] = myj;
        __syncthreads();
        if (tid == 0) {
            R m = R(0);
            for (int w = 0; w < NT / 32; ++w) m = fmax(m, sm.red[w]);
            atomic_max_pos(&smax[1], (double)m);
        }
    }
}

template <typename R, typename ST, bool DEV, int TY, int FIELD, int Q>
__device__ __forceinline__ void scalar_block(ScalarSmem<R, TY, Q>& sm, const KP<R>& P, const ST* fin, ST* fout,
                                             const R* mac_in, R* mac_out, const R* acc, const R* phi, const R* ux,
                                             const R* uy, unsigned long long* smax, int x0, int y0) {
    if (interior2<TY>(x0, y0, P.nx, P.ny))
        scalar_tile<R, ST, DEV, TY, FIELD, true, Q>(sm, P, fin, fout, mac_in, mac_out, acc, phi, ux, uy, smax, x0, y0);
    else scalar_tile<R, ST, DEV, TY, FIELD, false, Q>(sm, P, fin, fout, mac_in, mac_out, acc, phi, ux, uy, smax, x0, y0);
}

// ---------------------------------------------------------------------------
// Flow update (Eqs. 27-33) with the inlet / outflow columns
// ---------------------------------------------------------------------------
template <typename R, int TY> struct FlowSmem {
    R fl[TY + 2][34];
    R post[9][TY + 2][34];
};

// MRT collision of Eq. 14 with S of Eq. 31 and Guo forcing (Eq. 30); f holds
// populations 1..8 (decoded) on entry, rho the macro written with them; the
// nine post-collision populations go to p.  The forcing term carries the
// factor dt_F that Eq. 14 gives the scalar sources and Eq. 27 the half-force
// shift: one update moves rho u by the impulse dt_F F_b (Guo's scheme; the
// printed G_F alone would move it by F_b whatever dt_F is).
template <typename R>
__device__ __forceinline__ void flow_post9(const KP<R>& P, R* f, R rho, R* p) {
    const R c = P.cF, dt = P.dtF;
    const R Ix = dt * P.Fbx, Iy = dt * P.Fby;                          // impulse per update
    R s8 = R(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) s8 += f[i];
    f[0] = rho - s8;
    const R jx = mom_x(f), jy = mom_y(f);
    const R irho = rcp(rho);
    const R ux = (c * jx + R(0.5) * Ix) * irho, uy = (c * jy + R(0.5) * Iy) * irho;     // Eq. 27
    const R ic = dt, ic2 = ic * ic, u2 = (ux * ux + uy * uy) * ic2;    // 1/c_F = dt_F
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
    const R fu = (Ix * ux + Iy * uy) * ic2;
    const R G1 = R(6) * fu, G3 = Ix * ic, G5 = Iy * ic;
    const R G7 = R(2) * (Ix * ux - Iy * uy) * ic2, G8 = (Iy * ux + Ix * uy) * ic2;
    const R d1 = (-P.se * (m1 - rho * (R(-2) + R(3) * u2)) + (R(1) - R(0.5) * P.se) * G1) * (R(1) / R(36));
    const R d2 = (-P.seps * (m2 - rho * (R(1) - R(3) * u2)) - (R(1) - R(0.5) * P.seps) * G1) * (R(1) / R(36));
    const R d3 = G3 * (R(1) / R(6));
    const R d4 = (-P.sq * (m4 + rho * ux * ic) - (R(1) - R(0.5) * P.sq) * G3) * (R(1) / R(12));
    const R d5 = G5 * (R(1) / R(6));
    const R d6 = (-P.sq * (m6 + rho * uy * ic) - (R(1) - R(0.5) * P.sq) * G5) * (R(1) / R(12));
    const R d7 = (-P.snu * (m7 - rho * (ux * ux - uy * uy) * ic2) + (R(1) - R(0.5) * P.snu) * G7) * (R(1) / R(4));
    const R d8 = (-P.snu * (m8 - rho * ux * uy * ic2) + (R(1) - R(0.5) * P.snu) * G8) * (R(1) / R(4));
    const R axis = -d1 - R(2) * d2, diag = R(2) * d1 + d2;
    p[0] = f[0] - R(4) * d1 + R(4) * d2;
    p[1] = f[1] + axis + d3 - R(2) * d4 + d7;
    p[2] = f[2] + axis + d5 - R(2) * d6 - d7;
    p[3] = f[3] + axis - d3 + R(2) * d4 + d7;
    p[4] = f[4] + axis - d5 + R(2) * d6 - d7;
    p[5] = f[5] + diag + d3 + d4 + d5 + d6 + d8;
    p[6] = f[6] + diag - d3 - d4 + d5 + d6 - d8;
    p[7] = f[7] + diag - d3 - d4 - d5 - d6 + d8;
    p[8] = f[8] + diag + d3 + d4 - d5 - d6 - d8;
}
template <typename R, int TY>
__device__ __forceinline__ void flow_collide(const KP<R>& P, R (*sp)[TY + 2][34], int lx, int ly, R* f, R rho) {
    R p[9];
    flow_post9<R>(P, f, rho, p);
#pragma unroll
    for (int i = 0; i < 9; ++i) sp[i][ly][lx] = p[i];
}

template <typename R, typename ST, bool DEV, int TY, bool IN>
__device__ __forceinline__ void flow_tile(FlowSmem<R, TY>& sm, const KP<R>& P, const ST* __restrict__ fin,
                                          ST* __restrict__ fout, const R* __restrict__ phi,
                                          const R* __restrict__ ux_in, const R* __restrict__ uy_in,
                                          const R* __restrict__ rho_in, R* __restrict__ ux_out,
                                          R* __restrict__ uy_out, R* __restrict__ rho_out, int x0, int y0,
                                          Rect skip) {
    constexpr int TX = 32, HX = TX + 2, NR = 2 * HX + 2 * TY;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int pl = (int)P.plane;
    const R c = P.cF, dt = P.dtF;
    int ax = x0 + tx, ay = y0 + ty;
    const bool va = IN || resolve_xy(ax, ay, P.nx, P.ny, P.bfx, P.bfy);
    int blx = 0, bly = 0, bx = 0, by = 0;
    bool vb = false;
    if (tid < NR) {
        ring_pos<TY>(tid, blx, bly);
        bx = x0 - 1 + blx;
        by = y0 - 1 + bly;
        vb = IN || resolve_xy(bx, by, P.nx, P.ny, P.bfx, P.bfy);
    }
    const int na = ay * P.pitch + ax, nb = by * P.pitch + bx;
    R fa[9], fb[9];
    R ra = R(1), rb = R(1), uxa = R(0), uya = R(0), uxb = R(0), uyb = R(0), pa = R(0), pb = R(0);
    if (va) {
        load8<R, ST>(fin, na, pl, fa);
        ra = rho_in[na]; uxa = ux_in[na]; uya = uy_in[na]; pa = phi[na];
    }
    if (vb) {
        load8<R, ST>(fin, nb, pl, fb);
        rb = rho_in[nb]; uxb = ux_in[nb]; uyb = uy_in[nb]; pb = phi[nb];
    }
    if (DEV) {     // h_i = f_i - w_i rho of the writer's density
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            if (va) fa[i] += wq<R>(i) * ra;
            if (vb) fb[i] += wq<R>(i) * rb;
        }
    }
    if (va) {
        sm.fl[ty + 1][tx + 1] = R(0.5) * (R(1) - pa);                               // f_L = (1 - phi)/2
        flow_collide<R, TY>(P, sm.post, tx + 1, ty + 1, fa, ra);
    }
    if (vb) {
        sm.fl[bly][blx] = R(0.5) * (R(1) - pb);
        flow_collide<R, TY>(P, sm.post, blx, bly, fb, rb);
    }
    __syncthreads();
    const int gx = x0 + tx, gy = y0 + ty;
    if (!IN && (gx >= P.nx || gy >= P.ny)) return;
    if (skip.in(gx, gy)) return;                  // written by the vector strips of the same launch
    const int node = gy * P.pitch + gx;
    // streamed value of direction i into the node at shared position (hx, hy),
    // global (gxn, gyn), with the weighted partial bounce-back of Eq. 33
    auto pulled = [&](int i, int hx, int hy, int gxn, int gyn) -> R {
        const int o = opp_of(i);
        if (!IN) {
            const int sx = gxn - ex_of(i), sy = gyn - ey_of(i);
            const bool blocked = (P.bfx != BC_PERIODIC && outside(sx, P.nx)) || (P.bfy != BC_PERIODIC && outside(sy, P.ny));
            if (blocked) return sm.post[o][hy][hx];
        }
        const R fLm = R(0.5) * (sm.fl[hy - ey_of(i)][hx - ex_of(i)] + sm.fl[hy][hx]);
        return fLm * sm.post[i][hy - ey_of(i)][hx - ex_of(i)] + (R(1) - fLm) * sm.post[o][hy][hx];
    };
    R fn[9];
    const int hx = tx + 1, hy = ty + 1;
    if (!IN && P.bfx == BC_INLET_OUTFLOW && gx == P.nx - 1) {
#pragma unroll
        for (int i = 0; i < 9; ++i) fn[i] = pulled(i, hx - 1, hy, gx - 1, gy);      // f(L-1) = f(L-2)
    } else if (!IN && P.bfx == BC_INLET_OUTFLOW && gx == 0) {
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
    const R irho = rcp(rho);
    const R ux = (c * jx + R(0.5) * dt * P.Fbx) * irho, uy = (c * jy + R(0.5) * dt * P.Fby) * irho;
    rho_out[node] = rho;
    ux_out[node] = ux;
    uy_out[node] = uy;
    if (DEV) {
#pragma unroll
        for (int i = 1; i < 9; ++i) fout[node + (i - 1) * pl] = Cvt<ST>::st(fn[i] - wq<R>(i) * rho);
    } else {
#pragma unroll
        for (int i = 1; i < 9; ++i) fout[node + (i - 1) * pl] = Cvt<ST>::st(fn[i]);
    }
}

template <typename R, typename ST, bool DEV, int TY>
__device__ __forceinline__ void flow_block(FlowSmem<R, TY>& sm, const KP<R>& P, const ST* fin, ST* fout, const R* phi,
                                           const R* ux_in, const R* uy_in, const R* rho_in, R* ux_out, R* uy_out,
                                           R* rho_out, int x0, int y0, Rect skip = Rect{0, 0, 0, 0}) {
    // interior: tile + 1-ring inside the lattice, away from the inlet / outflow columns
    if (x0 >= 1 && x0 + 33 <= P.nx && y0 >= 1 && y0 + TY + 1 <= P.ny)
        flow_tile<R, ST, DEV, TY, true>(sm, P, fin, fout, phi, ux_in, uy_in, rho_in, ux_out, uy_out, rho_out, x0, y0,
                                        skip);
    else
        flow_tile<R, ST, DEV, TY, false>(sm, P, fin, fout, phi, ux_in, uy_in, rho_in, ux_out, uy_out, rho_out, x0,
                                         y0, skip);
}

// ---------------------------------------------------------------------------
// Launch wrappers.  Single simulation: block (bx, by) is tile (bx, by).
// Batched ensemble: one launch covers the tiles of several simulations
// ("jobs"); block b belongs to the last job whose first tile is <= b.
// ---------------------------------------------------------------------------
template <typename R, typename ST> struct PhaseJob {
    const KP<R>* P;     // the member's coefficient block in device memory
    const ST* fin; ST* fout; const R* phi; R* phin; const R* Um; const R* Tm;
    const long long* clock; long long off;
    int tiles_x, tile0;
};
template <typename R> struct TransferJob {
    const KP<R>* P;     // the member's coefficient block in device memory
    const R* phio; const R* phin; const R* Uin; R* Uout; const R* Tin; R* Tout; R* accU; R* accT;
    int acc_reset_U, acc_reset_T; unsigned long long* smax;
    int tiles_x, tile0;
};
template <typename R, typename ST> struct ScalarJob {
    const KP<R>* P;     // the member's coefficient block in device memory
    const ST* fin; ST* fout; const R* mac_in; R* mac_out; const R* acc; const R* phi; const R* ux; const R* uy;
    unsigned long long* smax;
    int tiles_x, tile0;
};
template <typename R, typename ST> struct FlowJob {
    const KP<R>* P;     // the member's coefficient block in device memory
    const ST* fin; ST* fout; const R* phi; const R* ux_in; const R* uy_in; const R* rho_in;
    R* ux_out; R* uy_out; R* rho_out;
    int tiles_x, tile0;
};

template <typename J>
__device__ __forceinline__ const J& job_of_block(const J* __restrict__ jobs, int njobs, int b, int& x0, int& y0,
                                                 int ty) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].tile0 <= b) lo = mid;
        else hi = mid - 1;
    }
    const J& j = jobs[lo];
    const int t = b - j.tile0;
    x0 = (t % j.tiles_x) * 32;
    y0 = (t / j.tiles_x) * ty;
    return j;
}

template <typename R, typename ST, bool DEV, int TY, int Q>
__global__ void __launch_bounds__(32 * TY)
k_phase(const KP<R>* __restrict__ P, const ST* __restrict__ fin, ST* __restrict__ fout, const R* __restrict__ phi,
        R* __restrict__ phin, const R* __restrict__ Um, const R* __restrict__ Tm,
        const long long* __restrict__ clock, long long step_off) {
    __shared__ PhaseSmem<R, TY, Q> sm;
    phase_block<R, ST, DEV, TY, Q>(sm, *P, fin, fout, phi, phin, Um, Tm, clock, step_off, blockIdx.x * 32, blockIdx.y * TY);
}
template <typename R, typename ST, bool DEV, int TY, int Q>
__global__ void __launch_bounds__(32 * TY) k_phase_batch(const PhaseJob<R, ST>* __restrict__ jobs, int njobs) {
    __shared__ PhaseSmem<R, TY, Q> sm;
    int x0, y0;
    const PhaseJob<R, ST>& j = job_of_block(jobs, njobs, blockIdx.x, x0, y0, TY);
    phase_block<R, ST, DEV, TY, Q>(sm, *j.P,j.fin, j.fout, j.phi, j.phin, j.Um, j.Tm, j.clock, j.off, x0, y0);
}

template <typename R, int TY>
__global__ void __launch_bounds__(32 * TY)
k_transfer(const KP<R>* __restrict__ P, const R* __restrict__ phio, const R* __restrict__ phin,
           const R* __restrict__ Uin, R* __restrict__ Uout, const R* __restrict__ Tin, R* __restrict__ Tout,
           R* __restrict__ accU, R* __restrict__ accT, int acc_reset_U, int acc_reset_T,
           unsigned long long* __restrict__ smax) {
    __shared__ TransferSmem<R, TY> sm;
    transfer_block<R, TY>(sm, *P,phio, phin, Uin, Uout, Tin, Tout, accU, accT, acc_reset_U, acc_reset_T, smax,
                          blockIdx.x * 32, blockIdx.y * TY);
}
template <typename R, int TY>
__global__ void __launch_bounds__(32 * TY) k_transfer_batch(const TransferJob<R>* __restrict__ jobs, int njobs) {
    __shared__ TransferSmem<R, TY> sm;
    int x0, y0;
    const TransferJob<R>& j = job_of_block(jobs, njobs, blockIdx.x, x0, y0, TY);
    transfer_block<R, TY>(sm, *j.P,j.phio, j.phin, j.Uin, j.Uout, j.Tin, j.Tout, j.accU, j.accT, j.acc_reset_U,
                          j.acc_reset_T, j.smax, x0, y0);
}

template <typename R, typename ST, bool DEV, int TY, int FIELD, int Q>
__global__ void __launch_bounds__(32 * TY)
k_scalar(const KP<R>* __restrict__ P, const ST* __restrict__ fin, ST* __restrict__ fout,
         const R* __restrict__ mac_in, R* __restrict__ mac_out, const R* __restrict__ acc, const R* __restrict__ phi,
         const R* __restrict__ ux, const R* __restrict__ uy, unsigned long long* __restrict__ smax) {
    __shared__ ScalarSmem<R, TY, Q> sm;
    scalar_block<R, ST, DEV, TY, FIELD, Q>(sm, *P,fin, fout, mac_in, mac_out, acc, phi, ux, uy, smax, blockIdx.x * 32,
                                        blockIdx.y * TY);
}
template <typename R, typename ST, bool DEV, int TY, int FIELD, int Q>
__global__ void __launch_bounds__(32 * TY) k_scalar_batch(const ScalarJob<R, ST>* __restrict__ jobs, int njobs) {
    __shared__ ScalarSmem<R, TY, Q> sm;
    int x0, y0;
    const ScalarJob<R, ST>& j = job_of_block(jobs, njobs, blockIdx.x, x0, y0, TY);
    scalar_block<R, ST, DEV, TY, FIELD, Q>(sm, *j.P,j.fin, j.fout, j.mac_in, j.mac_out, j.acc, j.phi, j.ux, j.uy,
                                        j.smax, x0, y0);
}

template <typename R, typename ST, bool DEV, int TY>
__global__ void __launch_bounds__(32 * TY)
k_flow(const KP<R>* __restrict__ P, const ST* __restrict__ fin, ST* __restrict__ fout, const R* __restrict__ phi,
       const R* __restrict__ ux_in, const R* __restrict__ uy_in, const R* __restrict__ rho_in,
       R* __restrict__ ux_out, R* __restrict__ uy_out, R* __restrict__ rho_out) {
    __shared__ FlowSmem<R, TY> sm;
    flow_block<R, ST, DEV, TY>(sm, *P,fin, fout, phi, ux_in, uy_in, rho_in, ux_out, uy_out, rho_out, blockIdx.x * 32,
                               blockIdx.y * TY);
}
template <typename R, typename ST, bool DEV, int TY>
__global__ void __launch_bounds__(32 * TY) k_flow_batch(const FlowJob<R, ST>* __restrict__ jobs, int njobs) {
    __shared__ FlowSmem<R, TY> sm;
    int x0, y0;
    const FlowJob<R, ST>& j = job_of_block(jobs, njobs, blockIdx.x, x0, y0, TY);
    flow_block<R, ST, DEV, TY>(sm, *j.P,j.fin, j.fout, j.phi, j.ux_in, j.uy_in, j.rho_in, j.ux_out, j.uy_out,
                               j.rho_out, x0, y0);
}

}  // namespace lbmk
