// Fused transport update: one launch per base step for everything that
// follows the phase update -- the phase-change transfer (Eqs. 36-39) and
// the U, T and flow collide-stream updates that are scheduled in that step
// (Eq. 34, workflow of Fig. 1).
//
// A tile needs the injected U*, T* (= U + Delta U_pc, T + Delta T_pc) on its
// 1-node ring for the scalar collisions there; Delta U_pc needs div J on
// that ring, i.e. J on a 2-node ring, i.e. grad phi^{q+1} there, i.e. phi^{q+1}
// on a 3-node ring.  Each block recomputes that halo work instead of
// exchanging it, so the injected macros never make a round trip through
// memory: the transfer and the field updates of a base step read the
// pre-injection U, T once and write only the final state.  Instantaneous
// coupling only (the accumulated ablation uses the separate kernels).
#pragma once
#include "lbm_kernels.cuh"
#include "lbm_strip.cuh"

namespace lbmk {

template <typename R, typename ST> struct TransportJob {
    const KP<R>* P;
    int do_tr, do_U, do_T, do_F;
    const R* phio;                 // phi^q (transfer only)
    const R* phi;                  // the current phase field (phi^{q+1} after a phase update)
    const R* Uin; R* Uout;         // U macro: pre-injection in, final out
    const R* Tin; R* Tout;
    const ST* fUin; ST* fUout;     // first moments (j_x, j_y) of U, two planes
    const ST* fTin; ST* fTout;     // first moments of T
    const ST* fFin; ST* fFout;
    const R* ux_in; const R* uy_in; const R* rho_in;   // flow state before this step's flow update
    R* ux_out; R* uy_out; R* rho_out;
    unsigned long long* smax;
    int tiles_x, tile0;
};

// Words the later stages read, copied asynchronously into shared memory by
// the prologue so that their global latency overlaps the transfer and the U
// update: the T first moments, the flow populations 1..8 and rho.
// Each thread copies and later reads only its own entries (own node: item A,
// a ring node: item B).
enum { PF_TJX = 0, PF_TJY = 1, PF_F = 2, PF_RHO = 10, PF_N = 11 };

template <typename R, int TY> struct TransportSmem {
    static constexpr int NRB = 2 * 34 + 2 * TY;   // ring items
    R phi[TY + 6][38];                 // phase field on the tile + 3-ring
    R Jx[TY + 4][36], Jy[TY + 4][36];  // J on the 2-ring
    R dphi[TY + 4][36];                // Delta phi on the 2-ring
    R Us[TY + 4][36];                  // pre-injection U on the 2-ring
    R Ui[TY + 2][34], Ti[TY + 2][34];  // injected U*, T* on the 1-ring
    R fl[TY + 2][34];                  // liquid fraction on the 1-ring (flow)
    R post[9][TY + 2][34];
    R red[TY];
    Word<R> pa[PF_N][32 * TY];         // prefetched words of item A
    Word<R> pb[PF_N][NRB];             // prefetched words of item B
};

template <int TY>
__device__ __forceinline__ bool interior3(int x0, int y0, int nx, int ny) {
    return x0 >= 3 && x0 + 35 <= nx && y0 >= 3 && y0 + TY + 3 <= ny;
}

// phase field on the tile plus a 3-node ghost ring (scalar boundary rule)
template <typename R, int TY, bool IN>
__device__ __forceinline__ void load_phi_ring3(const KP<R>& P, const R* __restrict__ phi, R (*s)[38], int x0, int y0,
                                               int tid) {
    constexpr int GX = 38, GY = TY + 6, NT = 32 * TY, K = (GX * GY + NT - 1) / NT;
    R v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int p = tid + k * NT;
        if (p < GX * GY) {
            int gx = x0 - 3 + p % GX, gy = y0 - 3 + p / GX;
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

template <typename R, typename ST, bool DEV, int TY, bool IN, int Q>
__device__ __forceinline__ void transport_tile(TransportSmem<R, TY>& sm, const KP<R>& P,
                                               const TransportJob<R, ST>& A, int x0, int y0) {
    constexpr int TX = 32, HX = 34, NT = 32 * TY, NR = 2 * HX + 2 * TY;
    constexpr int R2 = 36 * (TY + 4), K2 = (R2 + NT - 1) / NT;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int pl = (int)P.plane;
    const R omk = R(1) - P.k;
    // 1-ring items (scalar boundaries): A = own node, B = a ring node
    int ax = x0 + tx, ay = y0 + ty;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool own = IN || (gx < P.nx && gy < P.ny);
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

    // ---- prologue: every load that does not depend on shared data
    R po[K2], us[K2];
    int cxs[K2], cys[K2];
    bool fxs[K2], fys[K2], v2[K2];
    if (A.do_tr) {
#pragma unroll
        for (int k = 0; k < K2; ++k) {
            const int p = tid + k * NT;
            v2[k] = false;
            po[k] = us[k] = R(0);
            if (p < R2) {
                int sx = x0 - 2 + p % 36, sy = y0 - 2 + p / 36;
                cxs[k] = p % 36 + 1;
                cys[k] = p / 36 + 1;
                fxs[k] = fys[k] = false;
                bool ok = true;
                if (!IN) {
                    const bool a = j_source(sx, P.nx, P.bsx, x0 - 3, cxs[k], fxs[k]);
                    const bool b = j_source(sy, P.ny, P.bsy, y0 - 3, cys[k], fys[k]);
                    ok = a && b && cxs[k] >= 1 && cxs[k] <= 36 && cys[k] >= 1 && cys[k] <= TY + 4;
                }
                v2[k] = ok;
                if (ok) {
                    const int node = sy * P.pitch + sx;
                    po[k] = A.phio[node];
                    if (P.has_U) us[k] = A.Uin[node];
                }
            }
        }
    }
    R Ta = R(0), Tb = R(0), Ua0 = R(0), Ub0 = R(0);
    if (P.has_T) {
        if (va) Ta = A.Tin[na];
        if (vb) Tb = A.Tin[nb];
    }
    if (!A.do_tr && P.has_U) {
        if (va) Ua0 = A.Uin[na];
        if (vb) Ub0 = A.Uin[nb];
    }
    R jax = R(0), jay = R(0), jbx = R(0), jby = R(0);     // first moments of U (then T)
    if (A.do_U) {
        if (va) load_j<R, ST>(A.fUin, na, pl, jax, jay);
        if (vb) load_j<R, ST>(A.fUin, nb, pl, jbx, jby);
    }
    R uxa = R(0), uya = R(0), uxb = R(0), uyb = R(0);
    if (P.has_flow && (A.do_U || A.do_T)) {
        if (va) { uxa = A.ux_in[na]; uya = A.uy_in[na]; }
        if (vb) { uxb = A.ux_in[nb]; uyb = A.uy_in[nb]; }
    }
    // flow items: the same positions under the flow's own boundary rule
    // (evaluated here for the prefetch and again in the flow stage, so that
    // no index stays live across the stages in between)
    auto flow_item = [&](int lx, int ly, int& fx, int& fy) -> bool {
        fx = x0 - 1 + lx;
        fy = y0 - 1 + ly;
        return IN || resolve_xy(fx, fy, P.nx, P.ny, P.bfx, P.bfy);
    };
    // asynchronous prefetch of the T and flow stages' words
    if (A.do_T) {
        fetch_word<R>(&sm.pa[PF_TJX][tid], A.fTin, na, va);
        fetch_word<R>(&sm.pa[PF_TJY][tid], A.fTin + pl, na, va);
        if (tid < NR) {
            fetch_word<R>(&sm.pb[PF_TJX][tid], A.fTin, nb, vb);
            fetch_word<R>(&sm.pb[PF_TJY][tid], A.fTin + pl, nb, vb);
        }
    }
    if (A.do_F) {
        int fxa, fya, fxb = 0, fyb = 0;
        const bool fva = flow_item(tx + 1, ty + 1, fxa, fya);
        const bool fvb = tid < NR && flow_item(blx, bly, fxb, fyb);
        const int fna = fya * P.pitch + fxa, fnb = fyb * P.pitch + fxb;
#pragma unroll
        for (int i = 1; i < 9; ++i) fetch_word<R>(&sm.pa[PF_F + i - 1][tid], A.fFin + (size_t)(i - 1) * pl, fna, fva);
        fetch_word<R>(&sm.pa[PF_RHO][tid], A.rho_in, fna, fva);
        if (tid < NR) {
#pragma unroll
            for (int i = 1; i < 9; ++i)
                fetch_word<R>(&sm.pb[PF_F + i - 1][tid], A.fFin + (size_t)(i - 1) * pl, fnb, fvb);
            fetch_word<R>(&sm.pb[PF_RHO][tid], A.rho_in, fnb, fvb);
        }
    }
    __pipeline_commit();
    load_phi_ring3<R, TY, IN>(P, A.phi, sm.phi, x0, y0, tid);
    __syncthreads();

    // ---- J^q on the 2-ring (Eqs. 36-37)
    if (A.do_tr) {
        const R pre = P.at_pre;
#pragma unroll
        for (int k = 0; k < K2; ++k) {
            const int p = tid + k * NT;
            if (p < R2) {
                R jx = R(0), jy = R(0), dph = R(0);
                if (v2[k]) {
                    R gxv, gyv;
                    iso_grad<R, 38>(sm.phi, cxs[k], cys[k], gxv, gyv);
                    dph = sm.phi[cys[k]][cxs[k]] - po[k];
                    const R g2 = gxv * gxv + gyv * gyv;
                    if (g2 > R(1e-12)) {
                        const R a = pre * (R(1) + omk * us[k]) * dph * rsq(g2);
                        jx = fxs[k] ? a * gxv : -a * gxv;    // n = -grad phi / |grad phi|
                        jy = fys[k] ? a * gyv : -a * gyv;
                    }
                }
                sm.Jx[p / 36][p % 36] = jx;
                sm.Jy[p / 36][p % 36] = jy;
                sm.dphi[p / 36][p % 36] = dph;
                sm.Us[p / 36][p % 36] = us[k];
            }
        }
        __syncthreads();
    }

    // ---- injected U*, T* on the 1-ring (Eqs. 38-39); S_phi over the tile
    R mydu = R(0);
    auto inject = [&](bool v, int lx, int ly, R Tn, R U0, R& Uo, R& To) -> R {
        R Ui = U0, Ti = Tn, adu = R(0);
        if (v && A.do_tr) {
            const int hx = lx + 1, hy = ly + 1;      // 2-ring coordinates
            const R div = (sm.Jx[hy][hx + 1] - sm.Jx[hy][hx - 1] + sm.Jy[hy + 1][hx] - sm.Jy[hy - 1][hx]) * (R(1) / R(3)) +
                          ((sm.Jx[hy + 1][hx + 1] + sm.Jy[hy + 1][hx + 1]) + (sm.Jy[hy + 1][hx - 1] - sm.Jx[hy + 1][hx - 1]) -
                           (sm.Jx[hy - 1][hx - 1] + sm.Jy[hy - 1][hx - 1]) + (sm.Jx[hy - 1][hx + 1] - sm.Jy[hy - 1][hx + 1])) *
                              (R(1) / R(12));
            const R pn = sm.phi[ly + 2][lx + 2];
            const R dph = sm.dphi[hy][hx];
            if (P.has_U) {
                const R Us = sm.Us[hy][hx];
                const R dU = div_rn((R(1) + omk * Us) * dph - R(2) * div, (R(1) + P.k) - omk * pn);   // Eq. 38
                Ui = Us + dU;                                                                      // Eq. 39
                adu = fabs(dU);
            }
            if (P.has_T) {
                const R rc = R(0.5) * (R(1) + pn) * P.cS + R(0.5) * (R(1) - pn) * P.cL;
                Ti = Tn + P.rhoL_Lh * dph * rcp(R(2) * rc);                                        // Eq. 38
            }
        }
        Uo = Ui;
        To = Ti;
        return adu;
    };
    R Uia, Tia, Uib = R(0), Tib = R(0);
    mydu = inject(va, tx + 1, ty + 1, Ta, Ua0, Uia, Tia);
    if (tid < NR) inject(vb, blx, bly, Tb, Ub0, Uib, Tib);
    sm.Ui[ty + 1][tx + 1] = Uia;
    sm.Ti[ty + 1][tx + 1] = Tia;
    if (tid < NR) {
        sm.Ui[bly][blx] = Uib;
        sm.Ti[bly][blx] = Tib;
    }
    if (own) {
        const int node = gy * P.pitch + gx;
        if (P.has_U && !A.do_U) A.Uout[node] = Uia;     // fields not updated this step keep the injection
        if (P.has_T && !A.do_T) A.Tout[node] = Tia;
    } else {
        mydu = R(0);
    }
    if (A.do_tr && P.has_U) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mydu = fmax(mydu, __shfl_xor_sync(0xffffffffu, mydu, o));
        if ((tid & 31) == 0) sm.red[tid >> 5] = mydu;
    }
    __syncthreads();
    if (A.do_tr && P.has_U && tid == 0) {
        R m = R(0);
        for (int w = 0; w < NT / 32; ++w) m = fmax(m, sm.red[w]);
        atomic_max_pos(&A.smax[0], (double)m);
        atomic_max_pos(&A.smax[1], (double)m);
    }
    const Walls ws = walls_of<IN>(gx, gy, P.nx, P.ny, P.bsx, P.bsy);

    // ---- scalar updates (Eqs. 7-8, 10-12 tr parts; 14, 19-20, 23-25, 40)
    auto scalar_stream = [&](const ST* __restrict__ fin, ST* __restrict__ fout, R* __restrict__ mac_out, bool dir_ym,
                             R chi, R ae, auto field) {
        if (!own) return;
        const int node = gy * P.pitch + gx;
        R fn[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (i >= Q) { fn[i] = R(0); continue; }                                 // D2Q5: no diagonals
            fn[i] = ws.hit(i) ? sm.post[opp_of(i)][ty + 1][tx + 1] : sm.post[i][ty + 1 - ey_of(i)][tx + 1 - ex_of(i)];
            if (!IN && dir_ym && ey_of(i) > 0 && ws.ym)                            // bottom wall at T_ymin
                fn[i] = R(2) * wqq<R, Q>(i) * P.T_ymin - sm.post[opp_of(i)][ty + 1][tx + 1];
        }
        store_zeroth<R, ST, decltype(field)::value>(fin, fout, (size_t)pl, (size_t)node, chi,
                                                     streamed_increment<R, Q>(chi, fn) + ae, mac_out);   // Eq. 18
        store_j<R, ST>(fout, node, pl, fn);
    };
    if (A.do_U) {
        R aea = R(0);
        if (va) aea = scalar_collide<R, TY, 0, 38, 2, Q>(P, sm.phi, sm.post, tx + 1, ty + 1, Uia, jax, jay, uxa, uya);
        if (vb) scalar_collide<R, TY, 0, 38, 2, Q>(P, sm.phi, sm.post, blx, bly, Uib, jbx, jby, uxb, uyb);
        __syncthreads();
        scalar_stream(A.fUin, A.fUout, A.Uout, false, Uia, aea, std::integral_constant<int, 0>{});
        __syncthreads();
    }
    if (A.do_T) {
        __pipeline_wait_prior(0);                   // this thread's prefetched words have landed
        if (va) {
            jax = word_value<R, ST>(sm.pa[PF_TJX][tid], (na & 1) != 0);
            jay = word_value<R, ST>(sm.pa[PF_TJY][tid], (na & 1) != 0);
        }
        if (vb) {
            jbx = word_value<R, ST>(sm.pb[PF_TJX][tid], (nb & 1) != 0);
            jby = word_value<R, ST>(sm.pb[PF_TJY][tid], (nb & 1) != 0);
        }
        R aea = R(0);
        if (va) aea = scalar_collide<R, TY, 1, 38, 2, Q>(P, sm.phi, sm.post, tx + 1, ty + 1, Tia, jax, jay, uxa, uya);
        if (vb) scalar_collide<R, TY, 1, 38, 2, Q>(P, sm.phi, sm.post, blx, bly, Tib, jbx, jby, uxb, uyb);
        __syncthreads();
        scalar_stream(A.fTin, A.fTout, A.Tout, P.T_dir_ym != 0, Tia, aea, std::integral_constant<int, 1>{});
        __syncthreads();
    }

    // ---- flow update (Eqs. 27-33), flow boundaries
    if (A.do_F) {
        const R c = P.cF, dt = P.dtF;
        int fxa, fya, fxb = 0, fyb = 0;
        const bool fva = flow_item(tx + 1, ty + 1, fxa, fya);
        const bool fvb = tid < NR && flow_item(blx, bly, fxb, fyb);
        const int fna = fya * P.pitch + fxa, fnb = fyb * P.pitch + fxb;
        __pipeline_wait_prior(0);                   // this thread's prefetched words have landed
        R fa[9], fb[9];
        R ra = R(1), rb = R(1);
        if (fva) {
#pragma unroll
            for (int i = 1; i < 9; ++i) fa[i] = word_value<R, ST>(sm.pa[PF_F + i - 1][tid], (fna & 1) != 0);
            ra = word_value<R, R>(sm.pa[PF_RHO][tid], false);
        }
        if (fvb) {
#pragma unroll
            for (int i = 1; i < 9; ++i) fb[i] = word_value<R, ST>(sm.pb[PF_F + i - 1][tid], (fnb & 1) != 0);
            rb = word_value<R, R>(sm.pb[PF_RHO][tid], false);
        }
        if (DEV) {     // h_i = f_i - w_i rho of the writer's density
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                if (fva) fa[i] += wq<R>(i) * ra;
                if (fvb) fb[i] += wq<R>(i) * rb;
            }
        }
        // liquid fraction of the 1-ring positions: from the staged phase field
        // where the position lies inside the lattice, else (a periodic image
        // under the flow's own boundary rule) from the node it wraps to
        if (fva) {
            const bool inside = IN || (fxa == x0 + tx && fya == y0 + ty);
            sm.fl[ty + 1][tx + 1] = R(0.5) * (R(1) - (inside ? sm.phi[ty + 3][tx + 3] : A.phi[fna]));
            flow_collide<R, TY>(P, sm.post, tx + 1, ty + 1, fa, ra);
        }
        if (fvb) {
            const bool inside = IN || (fxb == x0 - 1 + blx && fyb == y0 - 1 + bly);
            sm.fl[bly][blx] = R(0.5) * (R(1) - (inside ? sm.phi[bly + 2][blx + 2] : A.phi[fnb]));
            flow_collide<R, TY>(P, sm.post, blx, bly, fb, rb);
        }
        __syncthreads();
        if (own) {
            const int node = gy * P.pitch + gx;
            auto pulled = [&](int i, int hx, int hy, int gxn, int gyn) -> R {
                const int o = opp_of(i);
                if (!IN) {
                    const int sx = gxn - ex_of(i), sy = gyn - ey_of(i);
                    const bool blocked = (P.bfx != BC_PERIODIC && outside(sx, P.nx)) ||
                                         (P.bfy != BC_PERIODIC && outside(sy, P.ny));
                    if (blocked) return sm.post[o][hy][hx];
                }
                const R fLm = R(0.5) * (sm.fl[hy - ey_of(i)][hx - ex_of(i)] + sm.fl[hy][hx]);
                return fLm * sm.post[i][hy - ey_of(i)][hx - ex_of(i)] + (R(1) - fLm) * sm.post[o][hy][hx];
            };
            R fn[9];
            const int hx = tx + 1, hy = ty + 1;
            if (!IN && P.bfx == BC_INLET_OUTFLOW && gx == P.nx - 1) {
#pragma unroll
                for (int i = 0; i < 9; ++i) fn[i] = pulled(i, hx - 1, hy, gx - 1, gy);   // f(L-1) = f(L-2)
            } else if (!IN && P.bfx == BC_INLET_OUTFLOW && gx == 0) {
                R rho1 = R(0);
#pragma unroll
                for (int i = 0; i < 9; ++i) rho1 += pulled(i, hx + 1, hy, gx + 1, gy);
                feq_flow<R>(rho1, P.u_in, R(0), c, fn);                                  // f = f_eq(rho(1), u_in)
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i) fn[i] = pulled(i, hx, hy, gx, gy);
            }
            R rho = R(0);
#pragma unroll
            for (int i = 0; i < 9; ++i) rho += fn[i];
            const R irho = rcp(rho);
            const R ux = (c * mom_x(fn) + R(0.5) * dt * P.Fbx) * irho, uy = (c * mom_y(fn) + R(0.5) * dt * P.Fby) * irho;
            A.rho_out[node] = rho;
            A.ux_out[node] = ux;
            A.uy_out[node] = uy;
            if (DEV) {
#pragma unroll
                for (int i = 1; i < 9; ++i) A.fFout[node + (i - 1) * pl] = Cvt<ST>::st(fn[i] - wq<R>(i) * rho);
            } else {
#pragma unroll
                for (int i = 1; i < 9; ++i) A.fFout[node + (i - 1) * pl] = Cvt<ST>::st(fn[i]);
            }
        }
    }
}

// FP32: at least 1024 resident threads per SM (64 registers a thread), the
// occupancy the tile's latency hiding needs; FP64 (parity runs) unconstrained
template <typename R, int TY> struct TransportOcc { static constexpr int MIN_BLOCKS = sizeof(R) == 4 ? 32 / TY : 1; };

template <typename R, typename ST, bool DEV, int TY, int Q>
__global__ void __launch_bounds__(32 * TY, (TransportOcc<R, TY>::MIN_BLOCKS))
k_transport_batch(const TransportJob<R, ST>* __restrict__ jobs, int njobs) {
    extern __shared__ __align__(16) unsigned char transport_smem[];
    TransportSmem<R, TY>& sm = *reinterpret_cast<TransportSmem<R, TY>*>(transport_smem);
    int x0, y0;
    const TransportJob<R, ST>& j = job_of_block(jobs, njobs, blockIdx.x, x0, y0, TY);
    const KP<R>& P = *j.P;
    if (interior3<TY>(x0, y0, P.nx, P.ny)) transport_tile<R, ST, DEV, TY, true, Q>(sm, P, j, x0, y0);
    else transport_tile<R, ST, DEV, TY, false, Q>(sm, P, j, x0, y0);
}

}  // namespace lbmk
