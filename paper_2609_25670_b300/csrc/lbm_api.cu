// Host runtime of the B300 multirate MRT-LBM: the C ABI of include/lbm.h,
// device-state ownership, the multirate schedule (Eq. 34, workflow of
// Fig. 1), CUDA-graph capture of one schedule period, kernel timing hooks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_aux.cuh"
#include "lbm_kernels.cuh"
#include "lbm_strip.cuh"
#include "lbm_transport.cuh"

using namespace lbmk;

namespace {

constexpr int TX = 32;
constexpr int kMaxGraphPeriod = 4096;

thread_local std::string g_create_error;

enum { FP = 0, FU = 1, FT = 2, FF = 3 };

// an instantiated graph with the kernels it launches per replay and the
// event pairs of its timed launches
// Host-side buffer selectors of one simulation: which half of every
// ping-pong pair is current, and the accumulation-reset flags.
struct Parity {
    int cur_pop[4] = {0, 0, 0, 0};
    int cur_phi = 0, cur_U = 0, cur_T = 0;
    bool acc_reset_U = true, acc_reset_T = true;
};

struct GraphRec {
    cudaGraphExec_t exec = nullptr;
    int kernels[LBM_K_COUNT] = {};
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> events;
    cudaGraph_t graph = nullptr;         // kept while timing nodes exist
    std::vector<std::pair<cudaGraphNode_t, cudaGraphNode_t>> nodes;   // event record nodes of `events`
    std::vector<Parity> post;            // each simulation's selectors after a replay
};

struct SimState {
    lbm_params p{};
    int nx = 0, ny = 0, pitch = 0;
    size_t nn = 0;        // pitch * ny
    void* pops[4][2] = {};   // phase, flow: 8 population planes; U, T: 2 first-moment planes (U with FP32
                             // arithmetic: a third, the residual of its compensated macro)
    int cur_pop[4] = {0, 0, 0, 0};
    void* phi[2] = {};
    int cur_phi = 0;
    void* U[2] = {};
    int cur_U = 0;
    void* T[2] = {};
    int cur_T = 0;
    void* ux[2] = {};
    void* uy[2] = {};
    void* rho[2] = {};
    void* accU = nullptr;
    void* accT = nullptr;
    void* ori_buf = nullptr;             // grain angles in the arithmetic type (allocated on first use)
    void* ori = nullptr;                 // ori_buf when an orientation field is set, else null
    bool acc_reset_U = true, acc_reset_T = true;
    unsigned long long* smax = nullptr;  // [S_phi, J_U] as double bits
    long long* clock = nullptr;          // base step at the start of a graph replay
    void* dkp = nullptr;                 // device copy of the coefficient block KP<R>
    double* part = nullptr;              // diagnostics partial sums
    double* dout = nullptr;              // diagnostics results (9 doubles)
    int diag_blocks = 0;
    int64_t step = 0;
    bool initialized = false;
    bool sticky = false;
    bool has_U = false, has_T = false, frozen_T = false, has_flow = false, accumulated = false;
    int period = 2;                      // 2 * lcm of the update factors: every parity returns
    int half = 1;                        // lcm of the update factors: one captured graph
    GraphRec g[2];                       // the two halves of the period
    int tile[LBM_K_COUNT] = {8, 8, 8, 8, 8, 8, 8, 8};   // tile height per kernel kind (autotuned)
    void* tjobs = nullptr;               // transport jobs: one per base step of the period + an eager slot
    size_t tjob_bytes = 0;               // bytes of one transport job in this precision
    int teager = 0;                      // index of the eager slot
};

Parity get_parity(const SimState& s) {
    Parity q;
    for (int k = 0; k < 4; ++k) q.cur_pop[k] = s.cur_pop[k];
    q.cur_phi = s.cur_phi;
    q.cur_U = s.cur_U;
    q.cur_T = s.cur_T;
    q.acc_reset_U = s.acc_reset_U;
    q.acc_reset_T = s.acc_reset_T;
    return q;
}

void set_parity(SimState& s, const Parity& q) {
    for (int k = 0; k < 4; ++k) s.cur_pop[k] = q.cur_pop[k];
    s.cur_phi = q.cur_phi;
    s.cur_U = q.cur_U;
    s.cur_T = q.cur_T;
    s.acc_reset_U = q.acc_reset_U;
    s.acc_reset_T = q.acc_reset_T;
}

struct TimedEvent {
    int kind;
    cudaEvent_t a, b;
};

}  // namespace

struct lbm_sim {
    std::vector<SimState> sims;
    uint32_t precision = LBM_PREC_F32;
    int q = 9;                           // velocities of the phase, U and T lattices (9 or 5)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    lbm_allocator alloc{};
    bool has_alloc = false;
    std::vector<std::pair<void*, size_t>> blocks;
    size_t bytes = 0;
    bool graphs = true;
    bool fuse = false;                   // fused transport launch (instantaneous coupling)
    bool fuse_auto = true;               // the autotuner may switch `fuse` (until set explicitly)
    bool cap_single = false;             // recording the transport jobs of a single simulation's period
    int cap_tcount = 0;                  // transport launches captured so far in that period
    uint32_t timing_mask = 0;
    double timing_ms[LBM_K_COUNT] = {};
    int64_t timing_n[LBM_K_COUNT] = {};
    int64_t launches[LBM_K_COUNT] = {};
    std::vector<TimedEvent> pending;     // eager-mode timed launches
    std::vector<cudaEvent_t> event_pool;
    bool capturing = false;
    int* cap_kernels = nullptr;          // kernel counts of the graph being captured
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>>* cap_events = nullptr;
    // batched ensemble: one launch per kernel kind covers every member's tiles
    bool batching = false;
    bool recording = false;              // launch_kind appends a job instead of launching
    int batch_tile[LBM_K_COUNT] = {8, 8, 8, 8, 8, 8, 8, 8};
    std::vector<unsigned char> rec[LBM_K_COUNT];
    int rec_jobs[LBM_K_COUNT] = {};
    int rec_tiles[LBM_K_COUNT] = {};
    int64_t half_all = 1;                // lcm of the members' halves: one captured graph
    void* job_buf = nullptr;             // device job tables: one region per half
    size_t job_buf_bytes = 0;
    GraphRec bg[2];                      // the two halves of the common period
    double* staging = nullptr;           // FP64 upload / download staging (lazy)
    size_t staging_bytes = 0;
    void* seed_dev = nullptr;            // device copy of the last seed list and its block list (lbm_init_seed)
    size_t seed_bytes = 0;
    std::string err;
};

namespace {

lbm_status fail(lbm_sim* h, lbm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_create_error = buf;
    return s;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return fail(h, LBM_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// planes of the stored U state: (j_x, j_y), plus the residual of the
// compensated macro with FP32 arithmetic (Compensated in lbm_common.cuh)
int u_planes(uint32_t precision) { return precision == LBM_PREC_F64 ? 2 : 3; }
// the residual plane (BF16) of the current U state, or null
const __nv_bfloat16* u_residual(const lbm_sim* h, const SimState& s) {
    if (!s.has_U || h->precision == LBM_PREC_F64) return nullptr;
    const size_t esz = h->precision == LBM_PREC_F32 ? sizeof(float) : 2;    // element size of the U state
    return (const __nv_bfloat16*)((const char*)s.pops[FU][s.cur_pop[FU]] + 2 * s.nn * esz);
}

lbm_status dev_alloc(lbm_sim* h, size_t bytes, void** out) {
    *out = nullptr;
    if (bytes == 0) return LBM_OK;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (h->has_alloc) {
        p = h->alloc.alloc(bytes, (void*)h->stream, h->alloc.ctx);
        if (!p) return fail(h, LBM_E_OOM, "allocator callback returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(h, LBM_E_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
        }
    }
    h->blocks.push_back({p, bytes});
    h->bytes += bytes;
    *out = p;
    // zero once: row padding and unused halves never hold stale non-finite bits
    cudaError_t e = cudaMemsetAsync(p, 0, bytes, h->stream);
    if (e != cudaSuccess) return fail(h, LBM_E_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    return LBM_OK;
}

// Host -> device upload of a coefficient block or job table, ordered on the
// handle's stream.  The stream is non-blocking (a caller's stream, e.g. from
// PyTorch's pool), so a plain cudaMemcpy on the legacy stream would not wait
// for work queued there: it could land before a pending cudaMemsetAsync of the
// same allocation (which then wipes it), or overwrite a job table that a
// queued launch still reads.  Synchronising afterwards lets the caller reuse
// the host buffer at once.
lbm_status upload_sync(lbm_sim* h, void* dst, const void* src, size_t bytes) {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

void free_all(lbm_sim* h) {
    for (auto& b : h->blocks) {
        if (h->has_alloc) h->alloc.free(b.first, b.second, (void*)h->stream, h->alloc.ctx);
        else cudaFree(b.first);
    }
    h->blocks.clear();
    h->bytes = 0;
    h->staging = nullptr;
    h->staging_bytes = 0;
    h->seed_dev = nullptr;
    h->seed_bytes = 0;
}

size_t real_size(uint32_t prec) { return prec == LBM_PREC_F64 ? 8 : 4; }
size_t store_size(uint32_t prec) { return prec == LBM_PREC_F64 ? 8 : prec == LBM_PREC_F32 ? 4 : 2; }

int64_t gcd64(int64_t a, int64_t b) { return b == 0 ? a : gcd64(b, a % b); }
int64_t lcm64(int64_t a, int64_t b) { return a / gcd64(a, b) * b; }

lbm_status validate(const lbm_params* p, std::string& why) {
    char buf[256];
    auto bad = [&](const char* m) { why = m; return LBM_E_INVALID_ARG; };
    if (p->struct_version != LBM_PARAMS_VERSION) return bad("struct_version != LBM_PARAMS_VERSION");
    if (p->nx < 4 || p->ny < 4) return bad("nx and ny must be >= 4");
    // the update kernels address population planes with 32-bit offsets
    if ((((int64_t)p->nx + 31) / 32 * 32) * p->ny * 8 >= (int64_t)1 << 31)
        return bad("nx * ny must be below 2^28 nodes (rows padded to 32)");
    if (p->fields & ~(uint32_t)(LBM_FIELD_U | LBM_FIELD_T | LBM_FIELD_FROZEN_T | LBM_FIELD_FLOW)) return bad("unknown fields bit");
    if ((p->fields & LBM_FIELD_T) && (p->fields & LBM_FIELD_FROZEN_T)) return bad("T and FROZEN_T are exclusive");
    if (p->bc_scalar_x < 0 || p->bc_scalar_x > 1 || p->bc_scalar_y < 0 || p->bc_scalar_y > 1)
        return bad("scalar boundaries must be PERIODIC or WALL");
    if (p->bc_flow_x < 0 || p->bc_flow_x > 2 || p->bc_flow_y < 0 || p->bc_flow_y > 1)
        return bad("flow boundary x must be PERIODIC, WALL or INLET_OUTFLOW; y PERIODIC or WALL");
    if (p->bc_flow_x == LBM_BC_INLET_OUTFLOW && (p->nx % TX) == 1)
        return bad("INLET_OUTFLOW needs nx % 32 != 1");
    if (p->T_ymin_dirichlet && (!(p->fields & LBM_FIELD_T) || p->bc_scalar_y != LBM_BC_WALL))
        return bad("T_ymin_dirichlet needs the T field and bc_scalar_y = WALL");
    if (p->precision > LBM_PREC_BF16_DEV) return bad("unknown precision");
    if (p->q_scalar != 0 && p->q_scalar != 9 && p->q_scalar != 5) return bad("q_scalar must be 0, 9 or 5");
    if (p->coupling > LBM_COUPLING_ACCUMULATED) return bad("unknown coupling");
    if (p->N_phi < 1 || p->N_U < 1 || p->N_T < 1 || p->N_F < 1) return bad("update factors must be >= 1");
    if (!(p->dt_base > 0.0)) return bad("dt_base must be > 0");
    if (!(p->W0 > 0.0) || !(p->tau0 > 0.0)) return bad("W0 and tau0 must be > 0");
    if (p->tip_cx < 0 || p->tip_cx >= p->nx || p->tip_cy < 0 || p->tip_cy >= p->ny) return bad("tip centre outside the lattice");
    const double dtp = p->N_phi * p->dt_base;
    const double amin = 1.0 - 3.0 * std::fabs(p->eps);
    if (!(amin > 0.0)) return bad("1 - 3 eps must be > 0 (a_s > 0)");
    if (3.0 * dtp * amin * amin * p->W0 * p->W0 / p->tau0 <= 0.0) return bad("tau_phi <= 1/2");
    if (p->fields & LBM_FIELD_U) {
        if (!(p->k > 0.0 && p->k <= 1.0)) return bad("k must be in (0, 1]");
        double dS = p->DS / p->k, dL = p->DL;          // D_eff at phi = +1, -1 (Eq. 7)
        if (!(3.0 * p->N_U * p->dt_base * std::min(dS, dL) > 0.0)) {
            snprintf(buf, sizeof buf, "tau_U <= 1/2 (D_S/k = %g, D_L = %g)", dS, dL);
            why = buf;
            return LBM_E_UNSTABLE_PARAMS;
        }
    }
    if (p->fields & LBM_FIELD_T) {
        if (!(p->rhoCpS > 0.0 && p->rhoCpL > 0.0)) return bad("heat capacities must be > 0");
        if (!(p->T_scale != 0.0)) return bad("T_scale must be nonzero");
        double aS = p->kappaS / p->rhoCpS, aL = p->kappaL / p->rhoCpL;
        if (!(std::min(aS, aL) > 0.0)) { why = "tau_T <= 1/2 (alpha <= 0)"; return LBM_E_UNSTABLE_PARAMS; }
    }
    if (p->fields & LBM_FIELD_FLOW) {
        if (!(p->nu > 0.0)) { why = "tau_F <= 1/2 (nu <= 0)"; return LBM_E_UNSTABLE_PARAMS; }
    }
    return LBM_OK;
}

template <typename R> KP<R> make_kp(const SimState& s) {
    const lbm_params& p = s.p;
    KP<R> k{};
    k.nx = s.nx; k.ny = s.ny; k.pitch = s.pitch; k.plane = (long long)s.nn;
    k.bsx = p.bc_scalar_x; k.bsy = p.bc_scalar_y; k.bfx = p.bc_flow_x; k.bfy = p.bc_flow_y;
    k.has_U = s.has_U; k.has_T = s.has_T; k.frozen_T = s.frozen_T; k.has_flow = s.has_flow;
    k.accumulated = s.accumulated;
    const double dtp = p.N_phi * p.dt_base, dtU = p.N_U * p.dt_base, dtT = p.N_T * p.dt_base, dtF = p.N_F * p.dt_base;
    k.dtp = (R)dtp; k.W0sq_tau0 = (R)(p.W0 * p.W0 / p.tau0); k.inv_tau0 = (R)(1.0 / p.tau0);
    k.eps = (R)p.eps; k.lam = (R)p.lam; k.Mc = (R)p.Mc;
    k.k = (R)p.k; k.at_pre = (R)(p.W0 / (2.0 * std::sqrt(2.0))); k.rhoL_Lh = (R)p.rhoL_Lh;
    k.dtU = (R)dtU; k.DS = (R)p.DS; k.DL = (R)p.DL;
    k.dtT = (R)dtT; k.kS = (R)p.kappaS; k.kL = (R)p.kappaL; k.cS = (R)p.rhoCpS; k.cL = (R)p.rhoCpL;
    k.T_shift = (R)p.T_shift; k.inv_T_scale = (R)(1.0 / p.T_scale);
    k.dtF = (R)dtF; k.cF = (R)(1.0 / dtF); k.Fbx = (R)p.Fbx; k.Fby = (R)p.Fby;
    k.se = (R)p.s_e; k.seps = (R)p.s_eps; k.sq = (R)p.s_q; k.snu = (R)(1.0 / (3.0 * dtF * p.nu + 0.5));
    k.u_in = (R)p.u_in;
    k.theta_c = (R)p.theta_c; k.fG = (R)p.frozen_G; k.fy0 = (R)p.frozen_y0; k.fV = (R)p.frozen_V;
    k.dt_base = (R)p.dt_base;
    k.T_dir_ym = s.has_T && p.T_ymin_dirichlet;
    k.T_ymin = (R)p.T_ymin;
    k.ori = (const R*)s.ori;
    return k;
}

// ---------------------------------------------------------------------------
// launch helpers (timing + launch counts)
// ---------------------------------------------------------------------------
cudaEvent_t pool_get(lbm_sim* h) {
    if (!h->event_pool.empty()) {
        cudaEvent_t e = h->event_pool.back();
        h->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct LaunchScope {
    lbm_sim* h;
    int kind;
    cudaEvent_t a = nullptr, b = nullptr;
    LaunchScope(lbm_sim* h_, int kind_) : h(h_), kind(kind_) {
        if (h->timing_mask & (1u << kind)) {
            if (h->capturing) {
                cudaEventCreate(&a);
                cudaEventCreate(&b);
                cudaEventRecordWithFlags(a, h->stream, cudaEventRecordExternal);
            } else {
                a = pool_get(h);
                b = pool_get(h);
                cudaEventRecord(a, h->stream);
            }
        }
    }
    ~LaunchScope() {
        if (h->capturing) h->cap_kernels[kind]++;
        else h->launches[kind]++;
        if (a) {
            if (h->capturing) {
                cudaEventRecordWithFlags(b, h->stream, cudaEventRecordExternal);
                h->cap_events->push_back({kind, {a, b}});
            } else {
                cudaEventRecord(b, h->stream);
                h->pending.push_back({kind, a, b});
            }
        }
    }
};

lbm_status collect_pending(lbm_sim* h) {
    if (h->pending.empty()) return LBM_OK;
    CK(cudaStreamSynchronize(h->stream));
    for (auto& t : h->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            h->timing_ms[t.kind] += ms;
            h->timing_n[t.kind]++;
        }
        h->event_pool.push_back(t.a);
        h->event_pool.push_back(t.b);
    }
    h->pending.clear();
    return LBM_OK;
}

// Launch one update kernel of `kind` for the current ping-pong parities
// (the caller flips them).  Reads buffer `cur`, writes buffer `1 - cur`: a
// repeated launch recomputes the same output, which the autotuner relies on.
template <int TYV>
inline dim3 grid_of(const SimState& s) { return dim3((s.nx + TX - 1) / TX, (s.ny + TYV - 1) / TYV); }

// Kernel variants of an update kind: v in {4, 8, 16} is a 32 x v
// shared-memory tile (blocks of 32 x v threads), v < 0 a warp strip of
// height -v (blocks of NWS strips, 32 NWS threads), v = VS + h vector strips
// of height h over the interior with 1-wide strips on the frame (one 1-D
// launch).  Blocks of one launch over an nx x ny lattice:
constexpr int VS = 1000;
// fv: nodes per lane of the flow or phase vector strips (nodes_per_lane_of:
// 2 for the 16-bit flow and the 16-bit D2Q5 phase, else VW)
inline void blocks_of(int kind, int v, int nx, int ny, int& bx, int& by, int fv = VW) {
    if (v > VS) {
        bx = kind == LBM_K_FLOW       ? fvs_blocks(nx, ny, v - VS, fv)
             : kind == LBM_K_TRANSFER ? tvs_blocks(nx, ny, v - VS)
             : kind == LBM_K_PHASE    ? pvs_blocks(nx, ny, v - VS, fv)
                                      : vs_blocks(nx, ny, v - VS);
        by = 1;
    } else if (v > 0) {
        bx = (nx + TX - 1) / TX;
        by = (ny + v - 1) / v;
    } else {
        const int strips = (nx + SW - 1) / SW;
        bx = (strips + NWS - 1) / NWS;
        by = (ny - v - 1) / (-v);
    }
}
inline dim3 grid_v(const SimState& s, int kind, int v, int fv = VW) {
    int bx, by;
    blocks_of(kind, v, s.nx, s.ny, bx, by, fv);
    return dim3(bx, by);
}
inline int nodes_per_lane_of(int kind, uint32_t precision, int q) {
    const bool st16 = precision == LBM_PREC_F16_DEV || precision == LBM_PREC_BF16_DEV;
    if (kind == LBM_K_FLOW) return st16 ? flow_nodes_per_lane<__half>() : flow_nodes_per_lane<float>();
    if (kind == LBM_K_PHASE)
        return q == 5 ? (st16 ? phase_nodes_per_lane<5, __half>() : phase_nodes_per_lane<5, float>())
                      : (st16 ? phase_nodes_per_lane<9, __half>() : phase_nodes_per_lane<9, float>());
    return VW;
}
inline bool has_strips(int kind) { return kind == LBM_K_SCALAR_U || kind == LBM_K_SCALAR_T; }
inline bool has_vstrips(int kind) {
    return has_strips(kind) || kind == LBM_K_FLOW || kind == LBM_K_TRANSFER || kind == LBM_K_PHASE;
}
inline bool valid_variant(int kind, int v) {
    return v == 4 || v == 8 || v == 16 ||
           (has_strips(kind) && (v == -4 || v == -8 || v == -16 || v == -32)) ||
           (has_vstrips(kind) && (v == VS + 8 || v == VS + 16 || v == VS + 32));
}

// Update-kernel launch on the handle's stream, with dynamic shared memory
// (opted in above the 48 KB default when a kernel needs more).
template <typename... KArgs, typename... Args>
inline void launch_ex_smem(lbm_sim* h, void (*kern)(KArgs...), dim3 g, dim3 b, size_t smem, Args... args) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = h->stream;
    cfg.attrs = nullptr;
    cfg.numAttrs = 0;
    cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
inline void launch_ex(lbm_sim* h, void (*kern)(KArgs...), dim3 g, dim3 b, Args... args) {
    launch_ex_smem(h, kern, g, b, 0, args...);
}

#define LBM_TY_SWITCH(sel, BODY)                       \
    switch (sel) {                                     \
        case 4: { constexpr int TYV = 4; BODY; } break;   \
        case 16: { constexpr int TYV = 16; BODY; } break; \
        default: { constexpr int TYV = 8; BODY; } break;  \
    }
#define LBM_VS_SWITCH(sel, BODY)                            \
    switch (sel) {                                          \
        case VS + 8: { constexpr int HV = 8; BODY; } break;    \
        case VS + 32: { constexpr int HV = 32; BODY; } break;  \
        default: { constexpr int HV = 16; BODY; } break;       \
    }
#define LBM_STRIP_SWITCH(sel, BODY)                      \
    switch (sel) {                                       \
        case -4: { constexpr int HV = 4; BODY; } break;     \
        case -8: { constexpr int HV = 8; BODY; } break;     \
        case -32: { constexpr int HV = 32; BODY; } break;   \
        default: { constexpr int HV = 16; BODY; } break;    \
    }

// Batched ensemble: instead of launching, append this member's job (the same
// arguments a single launch would get) to the table of `kind`.
template <typename J>
void push_job(lbm_sim* h, int kind, J& j, const SimState& s) {
    int bx, by;
    blocks_of(kind, h->batch_tile[kind], s.nx, s.ny, bx, by, nodes_per_lane_of(kind, h->precision, h->q));
    j.tiles_x = bx;
    j.tile0 = h->rec_tiles[kind];
    h->rec_tiles[kind] += bx * by;
    const unsigned char* b = (const unsigned char*)&j;
    h->rec[kind].insert(h->rec[kind].end(), b, b + sizeof(J));
    h->rec_jobs[kind]++;
}

template <typename R, typename ST, bool DEV>
void record_job(lbm_sim* h, SimState& s, int kind, const long long* clock, long long off) {
    const R* phi_now = (const R*)s.phi[s.cur_phi];
    const R* uxc = s.has_flow ? (const R*)s.ux[s.cur_pop[FF]] : nullptr;
    const R* uyc = s.has_flow ? (const R*)s.uy[s.cur_pop[FF]] : nullptr;
    switch (kind) {
        case LBM_K_PHASE: {
            PhaseJob<R, ST> j{(const KP<R>*)s.dkp,(const ST*)s.pops[FP][s.cur_pop[FP]], (ST*)s.pops[FP][1 - s.cur_pop[FP]],
                              phi_now, (R*)s.phi[1 - s.cur_phi], s.has_U ? (const R*)s.U[s.cur_U] : nullptr,
                              s.has_T ? (const R*)s.T[s.cur_T] : nullptr, clock, off, 0, 0};
            push_job(h, kind, j, s);
            break;
        }
        case LBM_K_TRANSFER: {
            TransferJob<R> j{(const KP<R>*)s.dkp,(const R*)s.phi[1 - s.cur_phi], phi_now,
                             s.has_U ? (const R*)s.U[s.cur_U] : nullptr, s.has_U ? (R*)s.U[1 - s.cur_U] : nullptr,
                             s.has_T ? (const R*)s.T[s.cur_T] : nullptr, s.has_T ? (R*)s.T[1 - s.cur_T] : nullptr,
                             (R*)s.accU, (R*)s.accT, s.acc_reset_U ? 1 : 0, s.acc_reset_T ? 1 : 0, s.smax, 0, 0};
            push_job(h, kind, j, s);
            break;
        }
        case LBM_K_SCALAR_U:
        case LBM_K_SCALAR_T: {
            const int f = kind == LBM_K_SCALAR_U ? FU : FT;
            void* const* mac = kind == LBM_K_SCALAR_U ? s.U : s.T;
            const int cm = kind == LBM_K_SCALAR_U ? s.cur_U : s.cur_T;
            ScalarJob<R, ST> j{(const KP<R>*)s.dkp,(const ST*)s.pops[f][s.cur_pop[f]], (ST*)s.pops[f][1 - s.cur_pop[f]],
                               (const R*)mac[cm], (R*)mac[1 - cm],
                               (const R*)(kind == LBM_K_SCALAR_U ? s.accU : s.accT), phi_now, uxc, uyc, s.smax, 0, 0};
            push_job(h, kind, j, s);
            break;
        }
        case LBM_K_FLOW: {
            const int c = s.cur_pop[FF];
            FlowJob<R, ST> j{(const KP<R>*)s.dkp,(const ST*)s.pops[FF][c], (ST*)s.pops[FF][1 - c], phi_now,
                             (const R*)s.ux[c], (const R*)s.uy[c], (const R*)s.rho[c], (R*)s.ux[1 - c],
                             (R*)s.uy[1 - c], (R*)s.rho[1 - c], 0, 0};
            push_job(h, kind, j, s);
            break;
        }
        default: break;
    }
}

template <typename R, typename ST, bool DEV, int Q>
void launch_batch(lbm_sim* h, int kind, int tysel, const void* jobs, int njobs, int tiles) {
    LaunchScope ls(h, kind);
    const dim3 g(tiles);
    switch (kind) {
        case LBM_K_PHASE:
            if (tysel > VS)
                LBM_VS_SWITCH(tysel, (launch_ex_smem(h, k_phase_vs_batch<R, ST, DEV, HV, Q>, g, dim3(32, PVW),
                                                     (size_t)PVSmem<R, Q, ST>::BYTES, (const PhaseJob<R, ST>*)jobs, njobs)))
            else
                LBM_TY_SWITCH(tysel, (launch_ex(h, k_phase_batch<R, ST, DEV, TYV, Q>, g, dim3(TX, TYV),
                                                (const PhaseJob<R, ST>*)jobs, njobs)))
            break;
        case LBM_K_TRANSFER:
            if (tysel > VS)
                LBM_VS_SWITCH(tysel, (launch_ex_smem(h, k_transfer_vs_batch<R, HV>, g, dim3(32, TVW),
                                                     (size_t)TVSmem<R>::BYTES, (const TransferJob<R>*)jobs, njobs)))
            else
                LBM_TY_SWITCH(tysel, (launch_ex(h, k_transfer_batch<R, TYV>, g, dim3(TX, TYV),
                                                (const TransferJob<R>*)jobs, njobs)))
            break;
        case LBM_K_SCALAR_U:
            if (tysel > VS)
                LBM_VS_SWITCH(tysel, (launch_ex_smem(h, scalar_vs_batch_kernel<R, ST, DEV, HV, 0, Q>(), g, dim3(32 * VNW),
                                                     (size_t)VNW * VSRing<R, ST>::BYTES, (const ScalarJob<R, ST>*)jobs,
                                                     njobs)))
            else if (tysel < 0)
                LBM_STRIP_SWITCH(tysel, (launch_ex(h, k_scalar_strip_batch<R, ST, DEV, HV, 0, Q>, g, dim3(32 * NWS),
                                                   (const ScalarJob<R, ST>*)jobs, njobs)))
            else
                LBM_TY_SWITCH(tysel, (launch_ex(h, k_scalar_batch<R, ST, DEV, TYV, 0, Q>, g, dim3(TX, TYV),
                                                (const ScalarJob<R, ST>*)jobs, njobs)))
            break;
        case LBM_K_SCALAR_T:
            if (tysel > VS)
                LBM_VS_SWITCH(tysel, (launch_ex_smem(h, scalar_vs_batch_kernel<R, ST, DEV, HV, 1, Q>(), g, dim3(32 * VNW),
                                                     (size_t)VNW * VSRing<R, ST>::BYTES, (const ScalarJob<R, ST>*)jobs,
                                                     njobs)))
            else if (tysel < 0)
                LBM_STRIP_SWITCH(tysel, (launch_ex(h, k_scalar_strip_batch<R, ST, DEV, HV, 1, Q>, g, dim3(32 * NWS),
                                                   (const ScalarJob<R, ST>*)jobs, njobs)))
            else
                LBM_TY_SWITCH(tysel, (launch_ex(h, k_scalar_batch<R, ST, DEV, TYV, 1, Q>, g, dim3(TX, TYV),
                                                (const ScalarJob<R, ST>*)jobs, njobs)))
            break;
        case LBM_K_FLOW:
            if (tysel > VS)
                LBM_VS_SWITCH(tysel, (launch_ex_smem(h, k_flow_vs_batch<R, ST, DEV, HV>, g, dim3(32, FVW),
                                                     (size_t)FVSmem<R, ST>::BYTES, (const FlowJob<R, ST>*)jobs, njobs)))
            else
                LBM_TY_SWITCH(tysel, (launch_ex(h, k_flow_batch<R, ST, DEV, TYV>, g, dim3(TX, TYV),
                                                (const FlowJob<R, ST>*)jobs, njobs)))
            break;
        case LBM_K_TRANSPORT:
            LBM_TY_SWITCH(tysel, (launch_ex_smem(h, k_transport_batch<R, ST, DEV, TYV, Q>, g, dim3(TX, TYV),
                                                 sizeof(TransportSmem<R, TYV>), (const TransportJob<R, ST>*)jobs,
                                                 njobs)));
            break;
        default: break;
    }
}

template <int Q>
void launch_batch_q(lbm_sim* h, int kind, int tysel, const void* jobs, int njobs, int tiles) {
    switch (h->precision) {
        case LBM_PREC_F64: launch_batch<double, double, false, Q>(h, kind, tysel, jobs, njobs, tiles); break;
        case LBM_PREC_F32: launch_batch<float, float, false, Q>(h, kind, tysel, jobs, njobs, tiles); break;
        case LBM_PREC_F16_DEV: launch_batch<float, __half, true, Q>(h, kind, tysel, jobs, njobs, tiles); break;
        default: launch_batch<float, __nv_bfloat16, true, Q>(h, kind, tysel, jobs, njobs, tiles); break;
    }
}
void launch_batch_any(lbm_sim* h, int kind, int tysel, const void* jobs, int njobs, int tiles) {
    if (h->q == 5) launch_batch_q<5>(h, kind, tysel, jobs, njobs, tiles);
    else launch_batch_q<9>(h, kind, tysel, jobs, njobs, tiles);
}

template <typename R, typename ST, bool DEV, int Q>
void launch_kind(lbm_sim* h, SimState& s, int kind, int tysel, const long long* clock, long long off) {
    if (h->recording) {
        record_job<R, ST, DEV>(h, s, kind, clock, off);
        return;
    }
    // the coefficients are read from the simulation's device copy, as the
    // batched launches do: one code path, identical arithmetic
    const KP<R>* P = (const KP<R>*)s.dkp;
    LaunchScope ls(h, kind);
    const R* phi_now = (const R*)s.phi[s.cur_phi];
    const R* uxc = s.has_flow ? (const R*)s.ux[s.cur_pop[FF]] : nullptr;
    const R* uyc = s.has_flow ? (const R*)s.uy[s.cur_pop[FF]] : nullptr;
    const R* null_r = nullptr;
    R* null_w = nullptr;
    switch (kind) {
        case LBM_K_PHASE:
            if (tysel > VS)
                LBM_VS_SWITCH(tysel, (launch_ex_smem(h, phase_vs_kernel<R, ST, DEV, HV, Q>(),
                    grid_v(s, kind, tysel, phase_nodes_per_lane<Q, ST>()),
                    dim3(32, PVW), (size_t)PVSmem<R, Q, ST>::BYTES, P, (const ST*)s.pops[FP][s.cur_pop[FP]],
                    (ST*)s.pops[FP][1 - s.cur_pop[FP]], phi_now, (R*)s.phi[1 - s.cur_phi],
                    s.has_U ? (const R*)s.U[s.cur_U] : null_r, s.has_T ? (const R*)s.T[s.cur_T] : null_r, clock, off)))
            else
                LBM_TY_SWITCH(tysel, (launch_ex(h, k_phase<R, ST, DEV, TYV, Q>, grid_of<TYV>(s), dim3(TX, TYV),
                    P, (const ST*)s.pops[FP][s.cur_pop[FP]], (ST*)s.pops[FP][1 - s.cur_pop[FP]], phi_now,
                    (R*)s.phi[1 - s.cur_phi], s.has_U ? (const R*)s.U[s.cur_U] : null_r,
                    s.has_T ? (const R*)s.T[s.cur_T] : null_r, clock, off)))
            break;
        case LBM_K_TRANSFER:   // phi^q = phi[1 - cur], phi^{q+1} = phi[cur] (after the phase flip)
            if (tysel > VS)
                LBM_VS_SWITCH(tysel, (launch_ex_smem(h, k_transfer_vs<R, HV>, grid_v(s, kind, tysel), dim3(32, TVW),
                    (size_t)TVSmem<R>::BYTES, P, (const R*)s.phi[1 - s.cur_phi], phi_now,
                    s.has_U ? (const R*)s.U[s.cur_U] : null_r, s.has_U ? (R*)s.U[1 - s.cur_U] : null_w,
                    s.has_T ? (const R*)s.T[s.cur_T] : null_r, s.has_T ? (R*)s.T[1 - s.cur_T] : null_w, (R*)s.accU,
                    (R*)s.accT, s.acc_reset_U ? 1 : 0, s.acc_reset_T ? 1 : 0, s.smax)))
            else
                LBM_TY_SWITCH(tysel, (launch_ex(h, k_transfer<R, TYV>, grid_of<TYV>(s), dim3(TX, TYV),
                    P, (const R*)s.phi[1 - s.cur_phi], phi_now, s.has_U ? (const R*)s.U[s.cur_U] : null_r,
                    s.has_U ? (R*)s.U[1 - s.cur_U] : null_w, s.has_T ? (const R*)s.T[s.cur_T] : null_r,
                    s.has_T ? (R*)s.T[1 - s.cur_T] : null_w, (R*)s.accU, (R*)s.accT, s.acc_reset_U ? 1 : 0,
                    s.acc_reset_T ? 1 : 0, s.smax)))
            break;
        case LBM_K_SCALAR_U:
        case LBM_K_SCALAR_T: {
            const bool isU = kind == LBM_K_SCALAR_U;
            const int f = isU ? FU : FT;
            const ST* fin = (const ST*)s.pops[f][s.cur_pop[f]];
            ST* fout = (ST*)s.pops[f][1 - s.cur_pop[f]];
            void* const* mac = isU ? s.U : s.T;
            const int cm = isU ? s.cur_U : s.cur_T;
            const R* acc = (const R*)(isU ? s.accU : s.accT);
            if (tysel > VS) {
                const size_t sm = (size_t)VNW * VSRing<R, ST>::BYTES;
                if (isU)
                    LBM_VS_SWITCH(tysel, (launch_ex_smem(h, scalar_vs_kernel<R, ST, DEV, HV, 0, Q>(), grid_v(s, kind, tysel),
                        dim3(32 * VNW), sm, P, fin, fout, (const R*)mac[cm], (R*)mac[1 - cm], acc, phi_now, uxc, uyc,
                        s.smax)))
                else
                    LBM_VS_SWITCH(tysel, (launch_ex_smem(h, scalar_vs_kernel<R, ST, DEV, HV, 1, Q>(), grid_v(s, kind, tysel),
                        dim3(32 * VNW), sm, P, fin, fout, (const R*)mac[cm], (R*)mac[1 - cm], acc, phi_now, uxc, uyc,
                        s.smax)))
            } else if (tysel < 0) {
                if (isU)
                    LBM_STRIP_SWITCH(tysel, (launch_ex(h, k_scalar_strip<R, ST, DEV, HV, 0, Q>, grid_v(s, kind, tysel),
                        dim3(32 * NWS), P, fin, fout, (const R*)mac[cm], (R*)mac[1 - cm], acc, phi_now, uxc, uyc,
                        s.smax)))
                else
                    LBM_STRIP_SWITCH(tysel, (launch_ex(h, k_scalar_strip<R, ST, DEV, HV, 1, Q>, grid_v(s, kind, tysel),
                        dim3(32 * NWS), P, fin, fout, (const R*)mac[cm], (R*)mac[1 - cm], acc, phi_now, uxc, uyc,
                        s.smax)))
            } else if (isU) {
                LBM_TY_SWITCH(tysel, (launch_ex(h, k_scalar<R, ST, DEV, TYV, 0, Q>, grid_of<TYV>(s), dim3(TX, TYV),
                    P, fin, fout, (const R*)mac[cm], (R*)mac[1 - cm], acc, phi_now, uxc, uyc, s.smax)));
            } else {
                LBM_TY_SWITCH(tysel, (launch_ex(h, k_scalar<R, ST, DEV, TYV, 1, Q>, grid_of<TYV>(s), dim3(TX, TYV),
                    P, fin, fout, (const R*)mac[cm], (R*)mac[1 - cm], acc, phi_now, uxc, uyc, s.smax)));
            }
            break;
        }
        case LBM_K_FLOW: {
            const int c = s.cur_pop[FF];
            if (tysel > VS)
                LBM_VS_SWITCH(tysel, (launch_ex_smem(h, flow_vs_kernel<R, ST, DEV, HV>(),
                    grid_v(s, kind, tysel, flow_nodes_per_lane<ST>()),
                    dim3(32, FVW), (size_t)FVSmem<R, ST>::BYTES, P, (const ST*)s.pops[FF][c], (ST*)s.pops[FF][1 - c],
                    phi_now, (const R*)s.ux[c], (const R*)s.uy[c], (const R*)s.rho[c], (R*)s.ux[1 - c],
                    (R*)s.uy[1 - c], (R*)s.rho[1 - c])))
            else
                LBM_TY_SWITCH(tysel, (launch_ex(h, k_flow<R, ST, DEV, TYV>, grid_of<TYV>(s), dim3(TX, TYV),
                    P, (const ST*)s.pops[FF][c], (ST*)s.pops[FF][1 - c], phi_now, (const R*)s.ux[c],
                    (const R*)s.uy[c], (const R*)s.rho[c], (R*)s.ux[1 - c], (R*)s.uy[1 - c], (R*)s.rho[1 - c])))
            break;
        }
        default: break;
    }
}

template <int Q>
void launch_q(lbm_sim* h, SimState& s, int kind, int tysel, const long long* clock, long long off) {
    switch (h->precision) {
        case LBM_PREC_F64: launch_kind<double, double, false, Q>(h, s, kind, tysel, clock, off); break;
        case LBM_PREC_F32: launch_kind<float, float, false, Q>(h, s, kind, tysel, clock, off); break;
        case LBM_PREC_F16_DEV: launch_kind<float, __half, true, Q>(h, s, kind, tysel, clock, off); break;
        default: launch_kind<float, __nv_bfloat16, true, Q>(h, s, kind, tysel, clock, off); break;
    }
}
void launch_any(lbm_sim* h, SimState& s, int kind, int tysel, const long long* clock, long long off) {
    if (h->q == 5) launch_q<5>(h, s, kind, tysel, clock, off);
    else launch_q<9>(h, s, kind, tysel, clock, off);
}

// The update sequence of one base step (Eq. 34 schedule, workflow of Fig. 1).
// ---------------------------------------------------------------------------
// fused transport (transfer + U + T + flow of one base step)
// ---------------------------------------------------------------------------
template <typename R, typename ST>
TransportJob<R, ST> make_transport_job(const SimState& s, bool tr, bool u, bool t, bool f) {
    TransportJob<R, ST> j{};
    j.P = (const KP<R>*)s.dkp;
    j.do_tr = tr; j.do_U = u; j.do_T = t; j.do_F = f;
    j.phio = (const R*)s.phi[1 - s.cur_phi];
    j.phi = (const R*)s.phi[s.cur_phi];
    if (s.has_U) {
        j.Uin = (const R*)s.U[s.cur_U];
        j.Uout = (R*)s.U[1 - s.cur_U];
        j.fUin = (const ST*)s.pops[FU][s.cur_pop[FU]];
        j.fUout = (ST*)s.pops[FU][1 - s.cur_pop[FU]];
    }
    if (s.has_T) {
        j.Tin = (const R*)s.T[s.cur_T];
        j.Tout = (R*)s.T[1 - s.cur_T];
        j.fTin = (const ST*)s.pops[FT][s.cur_pop[FT]];
        j.fTout = (ST*)s.pops[FT][1 - s.cur_pop[FT]];
    }
    if (s.has_flow) {
        const int c = s.cur_pop[FF];
        j.fFin = (const ST*)s.pops[FF][c];
        j.fFout = (ST*)s.pops[FF][1 - c];
        j.ux_in = (const R*)s.ux[c]; j.uy_in = (const R*)s.uy[c]; j.rho_in = (const R*)s.rho[c];
        j.ux_out = (R*)s.ux[1 - c]; j.uy_out = (R*)s.uy[1 - c]; j.rho_out = (R*)s.rho[1 - c];
    }
    j.smax = s.smax;
    return j;
}

template <typename R, typename ST, bool DEV, int TYV>
size_t transport_smem() { return sizeof(TransportSmem<R, TYV>); }

template <typename R, typename ST, bool DEV>
void launch_transport_jobs(lbm_sim* h, int tysel, const void* jobs, int njobs, int tiles) {
    LaunchScope ls(h, LBM_K_TRANSPORT);
    if (h->q == 5) {
        LBM_TY_SWITCH(tysel, (launch_ex_smem(h, k_transport_batch<R, ST, DEV, TYV, 5>, dim3(tiles), dim3(TX, TYV),
                                              transport_smem<R, ST, DEV, TYV>(),
                                              (const TransportJob<R, ST>*)jobs, njobs)));
        return;
    }
    LBM_TY_SWITCH(tysel, (launch_ex_smem(h, k_transport_batch<R, ST, DEV, TYV, 9>, dim3(tiles), dim3(TX, TYV),
                                          transport_smem<R, ST, DEV, TYV>(),
                                          (const TransportJob<R, ST>*)jobs, njobs)));
}

// One simulation's transport launch: recorded (batched ensembles, or the
// job-table pass of a single-simulation capture), replayed from the table
// uploaded before a capture, or staged through the eager slot.
template <typename R, typename ST, bool DEV>
void transport_one(lbm_sim* h, SimState& s, bool tr, bool u, bool t, bool f) {
    TransportJob<R, ST> j = make_transport_job<R, ST>(s, tr, u, t, f);
    if (h->recording && !h->cap_single) {
        push_job(h, LBM_K_TRANSPORT, j, s);
        return;
    }
    const int tyv = s.tile[LBM_K_TRANSPORT];
    j.tiles_x = (s.nx + TX - 1) / TX;
    j.tile0 = 0;
    const int tiles = j.tiles_x * ((s.ny + tyv - 1) / tyv);
    if (h->recording) {       // single-simulation job-table pass
        const unsigned char* b = (const unsigned char*)&j;
        h->rec[LBM_K_TRANSPORT].insert(h->rec[LBM_K_TRANSPORT].end(), b, b + sizeof j);
        h->rec_jobs[LBM_K_TRANSPORT]++;
        return;
    }
    TransportJob<R, ST>* slot;
    if (h->capturing) slot = (TransportJob<R, ST>*)s.tjobs + h->cap_tcount++;
    else {
        slot = (TransportJob<R, ST>*)s.tjobs + s.teager;
        cudaMemcpyAsync(slot, &j, sizeof j, cudaMemcpyHostToDevice, h->stream);
    }
    launch_transport_jobs<R, ST, DEV>(h, tyv, slot, 1, tiles);
}

void transport_any(lbm_sim* h, SimState& s, bool tr, bool u, bool t, bool f) {
    switch (h->precision) {
        case LBM_PREC_F64: transport_one<double, double, false>(h, s, tr, u, t, f); break;
        case LBM_PREC_F32: transport_one<float, float, false>(h, s, tr, u, t, f); break;
        case LBM_PREC_F16_DEV: transport_one<float, __half, true>(h, s, tr, u, t, f); break;
        default: transport_one<float, __nv_bfloat16, true>(h, s, tr, u, t, f); break;
    }
}

void enqueue_base_step(lbm_sim* h, SimState& s, int64_t n, const long long* clock, long long off) {
    const lbm_params& p = s.p;
    if (h->fuse && !s.accumulated) {
        const bool ph = (n + 1) % p.N_phi == 0;
        const bool u = s.has_U && (n + 1) % p.N_U == 0;
        const bool t = s.has_T && (n + 1) % p.N_T == 0;
        const bool f = s.has_flow && (n + 1) % p.N_F == 0;
        if (ph) {
            launch_any(h, s, LBM_K_PHASE, s.tile[LBM_K_PHASE], clock, off);
            s.cur_pop[FP] ^= 1;
            s.cur_phi ^= 1;                  // phi[cur] = phi^{q+1}
        }
        if (ph || u || t || f) {
            transport_any(h, s, ph, u, t, f);
            if (s.has_U && (ph || u)) s.cur_U ^= 1;
            if (s.has_T && (ph || t)) s.cur_T ^= 1;
            if (u) s.cur_pop[FU] ^= 1;
            if (t) s.cur_pop[FT] ^= 1;
            if (f) s.cur_pop[FF] ^= 1;
        }
        return;
    }
    if ((n + 1) % p.N_phi == 0) {
        launch_any(h, s, LBM_K_PHASE, s.tile[LBM_K_PHASE], clock, off);
        s.cur_pop[FP] ^= 1;
        s.cur_phi ^= 1;                      // phi[cur] = phi^{q+1}
        launch_any(h, s, LBM_K_TRANSFER, s.tile[LBM_K_TRANSFER], clock, off);
        if (!s.accumulated) {
            if (s.has_U) s.cur_U ^= 1;
            if (s.has_T) s.cur_T ^= 1;
        } else {
            s.acc_reset_U = false;
            s.acc_reset_T = false;
        }
    }
    if (s.has_U && (n + 1) % p.N_U == 0) {
        launch_any(h, s, LBM_K_SCALAR_U, s.tile[LBM_K_SCALAR_U], clock, off);
        s.cur_pop[FU] ^= 1;
        s.cur_U ^= 1;
        s.acc_reset_U = true;
    }
    if (s.has_T && (n + 1) % p.N_T == 0) {
        launch_any(h, s, LBM_K_SCALAR_T, s.tile[LBM_K_SCALAR_T], clock, off);
        s.cur_pop[FT] ^= 1;
        s.cur_T ^= 1;
        s.acc_reset_T = true;
    }
    if (s.has_flow && (n + 1) % p.N_F == 0) {
        launch_any(h, s, LBM_K_FLOW, s.tile[LBM_K_FLOW], clock, off);
        s.cur_pop[FF] ^= 1;
    }
}

void drop_rec(GraphRec& r) {
    if (r.exec) cudaGraphExecDestroy(r.exec);
    r.exec = nullptr;
    for (auto& e : r.events) {
        cudaEventDestroy(e.second.first);
        cudaEventDestroy(e.second.second);
    }
    r.events.clear();
    if (r.graph) cudaGraphDestroy(r.graph);
    r.graph = nullptr;
    r.nodes.clear();
    std::fill(std::begin(r.kernels), std::end(r.kernels), 0);
    r.post.clear();
}

void drop_graph(SimState& s) {
    drop_rec(s.g[0]);
    drop_rec(s.g[1]);
}

lbm_status end_capture(lbm_sim* h, GraphRec& r) {
    h->capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess) return fail(h, LBM_E_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&r.exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        r.exec = nullptr;
        return fail(h, LBM_E_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
    if (r.events.empty()) {
        cudaGraphDestroy(g);
        return LBM_OK;
    }
    // timing nodes: find the event record node of each captured event, so
    // that every replay can record into fresh events without a host wait
    r.graph = g;
    size_t n = 0;
    CK(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> all(n);
    CK(cudaGraphGetNodes(g, all.data(), &n));
    std::map<cudaEvent_t, cudaGraphNode_t> of;
    for (cudaGraphNode_t nd : all) {
        cudaGraphNodeType t;
        CK(cudaGraphNodeGetType(nd, &t));
        if (t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev = nullptr;
        CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
        of[ev] = nd;
    }
    for (auto& ev : r.events) {
        auto a = of.find(ev.second.first), b = of.find(ev.second.second);
        if (a == of.end() || b == of.end()) return fail(h, LBM_E_CUDA, "timing node missing from the captured graph");
        r.nodes.push_back({a->second, b->second});
    }
    return LBM_OK;
}

// Point the timing nodes of `r` at fresh pool events for the next replay and
// queue them; the elapsed times are read when the pending list is collected.
lbm_status arm_graph_events(lbm_sim* h, GraphRec& r) {
    for (size_t i = 0; i < r.events.size(); ++i) {
        cudaEvent_t a = pool_get(h), b = pool_get(h);
        CK(cudaGraphExecEventRecordNodeSetEvent(r.exec, r.nodes[i].first, a));
        CK(cudaGraphExecEventRecordNodeSetEvent(r.exec, r.nodes[i].second, b));
        h->pending.push_back({r.events[i].first, a, b});
    }
    return LBM_OK;
}

// Capture half `which` of the schedule period: s.half = lcm(N_chi) base steps
// starting at a step n with n mod 2*half == which*half.  Every ping-pong
// parity depends only on n mod 2*half, so the two halves replay forever.
void clear_records(lbm_sim* h);

lbm_status capture_graph(lbm_sim* h, SimState& s, int which) {
    drop_rec(s.g[which]);
    // pass 1: this half's transport jobs (their buffer pointers depend on the
    // parities of each base step), uploaded to the simulation's job table
    clear_records(h);
    const Parity pre = get_parity(s);
    h->recording = true;
    h->cap_single = true;
    for (int k = 0; k < s.half; ++k) enqueue_base_step(h, s, s.step + k, s.frozen_T ? s.clock : nullptr, k);
    h->recording = false;
    h->cap_single = false;
    set_parity(s, pre);
    if (!h->rec[LBM_K_TRANSPORT].empty())
    {
        lbm_status st = upload_sync(h, (unsigned char*)s.tjobs + (size_t)which * s.half * s.tjob_bytes,
                                    h->rec[LBM_K_TRANSPORT].data(), h->rec[LBM_K_TRANSPORT].size());
        if (st) return st;
    }
    clear_records(h);
    // pass 2: capture
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    h->cap_tcount = which * s.half;
    h->cap_kernels = s.g[which].kernels;
    h->cap_events = &s.g[which].events;
    for (int k = 0; k < s.half; ++k) enqueue_base_step(h, s, s.step + k, s.frozen_T ? s.clock : nullptr, k);
    if (s.frozen_T) k_tick<<<1, 1, 0, h->stream>>>(s.clock, s.half);
    s.g[which].post.assign(1, get_parity(s));
    set_parity(s, pre);                  // the replay applies the post state
    return end_capture(h, s.g[which]);
}

void drop_batch_graph(lbm_sim* h) {
    drop_rec(h->bg[0]);
    drop_rec(h->bg[1]);
}

void clear_records(lbm_sim* h) {
    for (int k = 0; k < LBM_K_COUNT; ++k) {
        h->rec[k].clear();
        h->rec_jobs[k] = 0;
        h->rec_tiles[k] = 0;
    }
}

// Capture half `which` of the common period of a batched ensemble (half_all =
// lcm of the members' halves; every member's parities depend only on the step
// mod 2 * half_all): per base step, one launch per kernel kind over the tiles
// of every member that fires (members are independent, so the per-member
// order phase -> transfer -> U -> T -> flow is kept by the order of the
// launches).  The job tables of each half live in their own half of job_buf.
lbm_status capture_batch(lbm_sim* h, int which) {
    drop_rec(h->bg[which]);
    struct Seg { int kind; size_t off; int njobs, tiles; };
    std::vector<std::vector<Seg>> steps((size_t)h->half_all);
    std::vector<unsigned char> all;
    std::vector<Parity> pre;
    for (auto& s : h->sims) pre.push_back(get_parity(s));
    static const int order[6] = {LBM_K_PHASE, LBM_K_TRANSFER, LBM_K_TRANSPORT, LBM_K_SCALAR_U, LBM_K_SCALAR_T,
                                 LBM_K_FLOW};
    for (int64_t k = 0; k < h->half_all; ++k) {
        clear_records(h);
        h->recording = true;
        for (auto& s : h->sims) enqueue_base_step(h, s, s.step + k, s.frozen_T ? s.clock : nullptr, k);
        h->recording = false;
        for (int kind : order) {
            if (!h->rec_jobs[kind]) continue;
            size_t off = (all.size() + 255) & ~size_t(255);
            all.resize(off);
            all.insert(all.end(), h->rec[kind].begin(), h->rec[kind].end());
            steps[k].push_back({kind, off, h->rec_jobs[kind], h->rec_tiles[kind]});
        }
    }
    clear_records(h);
    h->bg[which].post.clear();
    for (size_t i = 0; i < h->sims.size(); ++i) {
        h->bg[which].post.push_back(get_parity(h->sims[i]));
        set_parity(h->sims[i], pre[i]);  // the replay applies the post state
    }
    const size_t region = h->job_buf_bytes / 2;
    if (all.size() > region)
        return fail(h, LBM_E_STATE, "job tables of %zu bytes exceed the %zu reserved", all.size(), region);
    unsigned char* base = (unsigned char*)h->job_buf + (size_t)which * region;
    {
        lbm_status st = upload_sync(h, base, all.data(), all.size());
        if (st) return st;
    }
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    h->cap_kernels = h->bg[which].kernels;
    h->cap_events = &h->bg[which].events;
    for (int64_t k = 0; k < h->half_all; ++k)
        for (const Seg& sg : steps[k])
            launch_batch_any(h, sg.kind, h->batch_tile[sg.kind], base + sg.off, sg.njobs, sg.tiles);
    for (auto& s : h->sims)
        if (s.frozen_T) k_tick<<<1, 1, 0, h->stream>>>(s.clock, h->half_all);
    return end_capture(h, h->bg[which]);
}

lbm_status batch_replay(lbm_sim* h, int which) {
    if (!h->bg[which].events.empty()) {
        lbm_status st = arm_graph_events(h, h->bg[which]);
        if (st) return st;
    }
    CK(cudaGraphLaunch(h->bg[which].exec, h->stream));
    for (int k = 0; k < LBM_K_COUNT; ++k) h->launches[k] += h->bg[which].kernels[k];
    for (size_t i = 0; i < h->sims.size(); ++i) {
        h->sims[i].step += h->half_all;
        set_parity(h->sims[i], h->bg[which].post[i]);
    }
    return LBM_OK;
}

lbm_status graph_replay(lbm_sim* h, SimState& s, int which) {
    if (!s.g[which].events.empty()) {
        lbm_status st = arm_graph_events(h, s.g[which]);
        if (st) return st;
    }
    CK(cudaGraphLaunch(s.g[which].exec, h->stream));
    for (int k = 0; k < LBM_K_COUNT; ++k) h->launches[k] += s.g[which].kernels[k];
    s.step += s.half;
    set_parity(s, s.g[which].post[0]);
    return LBM_OK;
}

template <typename R> void enqueue_diag(lbm_sim* h, SimState& s, bool solute_only = false);

// seeded: the macroscopic fields come from lbm_init_seed (U = U0, T = T0,
// u_y = 0, rho = 1 everywhere)
template <typename R>
lbm_status finish_init(lbm_sim* h, SimState& s, bool seeded = false, double U0 = 0.0, double T0 = 0.0);

template <typename R>
lbm_status upload_and_init(lbm_sim* h, SimState& s, const double* src[6], int src_dev) {
    const size_t n = (size_t)s.nx * s.ny;
    const size_t need = n * sizeof(double);
    void* dst[6] = {s.phi[0], s.U[0], s.T[0], s.ux[0], s.uy[0], s.rho[0]};
    int nf = 0;
    for (int f = 0; f < 6; ++f) nf += (dst[f] && src[f]) ? 1 : 0;
    // one staging slot per field when they fit in 256 MiB: the copies then
    // run back to back instead of each waiting for the previous conversion
    const bool slots = (size_t)nf * need <= ((size_t)256 << 20);
    const size_t want = slots ? (size_t)nf * need : need;
    if (h->staging_bytes < want) {
        void* p = nullptr;
        lbm_status st = dev_alloc(h, want, &p);
        if (st) return st;
        h->staging = (double*)p;
        h->staging_bytes = want;
    }
    const dim3 blk(32, 8), grd((s.nx + 31) / 32, (s.ny + 7) / 8);
    const cudaMemcpyKind kind = src_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int f = 0, k = 0; f < 6; ++f) {
        if (!dst[f] || !src[f]) continue;
        double* slot = h->staging + (slots ? (size_t)k++ * n : 0);
        CK(cudaMemcpyAsync(slot, src[f], need, kind, h->stream));
        if (!slots) k_from_f64<R><<<grd, blk, 0, h->stream>>>(slot, (R*)dst[f], s.nx, s.ny, s.pitch);
    }
    // the caller may reuse its buffers once they have been read
    cudaEvent_t copied = pool_get(h);
    CK(cudaEventRecord(copied, h->stream));
    if (slots)
        for (int f = 0, k = 0; f < 6; ++f)
            if (dst[f] && src[f])
                k_from_f64<R><<<grd, blk, 0, h->stream>>>(h->staging + (size_t)k++ * n, (R*)dst[f], s.nx, s.ny, s.pitch);
    lbm_status st = finish_init<R>(h, s);
    CK(cudaEventSynchronize(copied));
    h->event_pool.push_back(copied);
    return st;
}

// Everything after the macroscopic fields of buffer 0 are in place: the
// equilibrium populations, cleared accumulators and maxima, the reference
// solute inventory M_C(0), the clock.
// the initial distributions of buffer 0 (k_init), for the phase lattice's
// velocity count
template <typename R, typename ST, bool DEV>
void launch_init(lbm_sim* h, SimState& s, bool seeded, double U0, double T0) {
    const dim3 blk(32, 8), grd((s.nx + 31) / 32, (s.ny + 7) / 8);
    const auto kern = h->q == 5 ? &k_init<R, ST, DEV, 5> : &k_init<R, ST, DEV, 9>;
    kern<<<grd, blk, 0, h->stream>>>(make_kp<R>(s), (const R*)s.phi[0], (const R*)s.U[0], (const R*)s.T[0],
                                     (const R*)s.ux[0], (const R*)s.uy[0], (const R*)s.rho[0], (ST*)s.pops[FP][0],
                                     (ST*)s.pops[FU][0], (ST*)s.pops[FT][0], (ST*)s.pops[FF][0], (int)seeded, (R)U0,
                                     (R)T0);
}

template <typename R>
lbm_status finish_init(lbm_sim* h, SimState& s, bool seeded, double U0, double T0) {
    s.cur_phi = s.cur_U = s.cur_T = 0;
    for (int f = 0; f < 4; ++f) s.cur_pop[f] = 0;
    {
        LaunchScope ls(h, LBM_K_INIT);
        switch (h->precision) {
            case LBM_PREC_F64:
            case LBM_PREC_F32: launch_init<R, R, false>(h, s, seeded, U0, T0); break;
            case LBM_PREC_F16_DEV: launch_init<float, __half, true>(h, s, seeded, U0, T0); break;
            default: launch_init<float, __nv_bfloat16, true>(h, s, seeded, U0, T0);
        }
    }
    CK(cudaGetLastError());
    const size_t rs = sizeof(R);
    if (s.accU) CK(cudaMemsetAsync(s.accU, 0, 2 * s.nn * rs, h->stream));
    if (s.accT) CK(cudaMemsetAsync(s.accT, 0, 2 * s.nn * rs, h->stream));
    CK(cudaMemsetAsync(s.smax, 0, 2 * sizeof(unsigned long long), h->stream));
    if (s.clock) CK(cudaMemsetAsync(s.clock, 0, sizeof(long long), h->stream));
    {   // solute inventory of the initial state: the reference M_C(0) of R_M (Sec. 4.4)
        LaunchScope ls(h, LBM_K_INIT);
        enqueue_diag<R>(h, s, true);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(s.dout + 9, s.dout, sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    s.acc_reset_U = s.acc_reset_T = true;
    s.step = 0;
    s.initialized = true;
    s.sticky = false;
    return LBM_OK;
}

// n_listed: the number of seed-field blocks in the block list that follows
// the seeds in h->seed_dev (the lattice is first filled with the values no
// seed reaches), or -1 to run every block.
template <typename R>
lbm_status seed_and_init(lbm_sim* h, SimState& s, int n_seeds, int n_listed, double U0, double T0,
                         uint64_t rng_seed) {
    const dim3 blk(SEED_BX, SEED_BY), grd((s.nx + SEED_BX - 1) / SEED_BX, (s.ny + SEED_BH - 1) / SEED_BH);
    R* const phi = (R*)s.phi[0];
    R* const U = s.has_U ? (R*)s.U[0] : nullptr;
    R* const T = s.has_T ? (R*)s.T[0] : nullptr;
    R* const ux = s.has_flow ? (R*)s.ux[0] : nullptr;
    R* const uy = s.has_flow ? (R*)s.uy[0] : nullptr;
    R* const rho = s.has_flow ? (R*)s.rho[0] : nullptr;
    const SeedDev* sd = (const SeedDev*)h->seed_dev;
    const double sw = std::sqrt(2.0) * s.p.W0;
    if (n_listed < 0) {
        k_seed_fields<R><<<grd, blk, 0, h->stream>>>(s.nx, s.ny, s.pitch, sd, n_seeds, nullptr, (int)grd.x, sw,
                                                     (unsigned long long)rng_seed, U0, T0, s.p.u_in, phi, U, T,
                                                     ux, uy, rho);
    } else {
        const R ux_liquid = (R)(s.p.u_in * 0.5 * (1.0 - (-1.0)));      // the profile's u_x at phi = -1
        k_seed_fill<R><<<grd, blk, 0, h->stream>>>(s.nx, s.ny, s.pitch, (R)U0, (R)T0, ux_liquid, phi, U, T, ux,
                                                   uy, rho);
        if (n_listed > 0)
            k_seed_fields<R><<<n_listed, blk, 0, h->stream>>>(s.nx, s.ny, s.pitch, sd, n_seeds,
                                                              (const int*)(sd + n_seeds), (int)grd.x, sw,
                                                              (unsigned long long)rng_seed, U0, T0, s.p.u_in, phi,
                                                              U, T, ux, uy, rho);
    }
    CK(cudaGetLastError());
    return finish_init<R>(h, s, true, U0, T0);
}


lbm_status init_common(lbm_sim* h, int32_t sim, const double* src[6], int src_dev) {
    SimState& s = h->sims[sim];
    // a captured period graph stays valid: it was captured at a step where every
    // ping-pong parity has its initial value, which initialisation restores
    return h->precision == LBM_PREC_F64 ? upload_and_init<double>(h, s, src, src_dev)
                                        : upload_and_init<float>(h, s, src, src_dev);
}


template <typename R>
lbm_status read_field(lbm_sim* h, SimState& s, uint32_t which, void* dst, int dst_dev, int as_f64) {
    const KP<R> P = make_kp<R>(s);
    const dim3 blk(32, 8), grd((s.nx + 31) / 32, (s.ny + 8 * OUT_ROWS - 1) / (8 * OUT_ROWS));
    const size_t n = (size_t)s.nx * s.ny;
    const size_t esz = as_f64 ? sizeof(double) : sizeof(R);
    void* out = dst;
    if (!dst_dev) {
        if (h->staging_bytes < n * sizeof(double)) {
            void* p = nullptr;
            lbm_status st = dev_alloc(h, n * sizeof(double), &p);
            if (st) return st;
            h->staging = (double*)p;
            h->staging_bytes = n * sizeof(double);
        }
        out = h->staging;
    }
    // clock holds the base step of the last graph replay start; keep it exact here
    if (s.clock) k_set_clock<<<1, 1, 0, h->stream>>>(s.clock, (long long)s.step);
    const int fc = s.cur_pop[FF];
    // U carries the residual of its compensated macro (FP32 arithmetic)
    const void* ulo = u_residual(h, s);
    const int lo_kind = ulo ? 2 : 0;
    if (as_f64)
        k_out<R, double><<<grd, blk, 0, h->stream>>>(P, (int)which, (const R*)s.phi[s.cur_phi],
                                                     s.has_U ? (const R*)s.U[s.cur_U] : nullptr,
                                                     s.has_T ? (const R*)s.T[s.cur_T] : nullptr, (const R*)s.ux[fc],
                                                     (const R*)s.uy[fc], (const R*)s.rho[fc], ulo, lo_kind,
                                                     (double*)out, s.clock);
    else
        k_out<R, R><<<grd, blk, 0, h->stream>>>(P, (int)which, (const R*)s.phi[s.cur_phi],
                                                s.has_U ? (const R*)s.U[s.cur_U] : nullptr,
                                                s.has_T ? (const R*)s.T[s.cur_T] : nullptr, (const R*)s.ux[fc],
                                                (const R*)s.uy[fc], (const R*)s.rho[fc], ulo, lo_kind, (R*)out,
                                                s.clock);
    CK(cudaGetLastError());
    if (!dst_dev) {
        CK(cudaMemcpyAsync(dst, out, n * esz, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    return LBM_OK;
}

// The diagnostics reductions of simulation s into s.dout[0..8] (asynchronous).
// solute_only: dout[0] (M_C, bit for bit the value of the full reduction) and
// the cleared maxima only; the other slots are left as they were.
template <typename R>
void enqueue_diag(lbm_sim* h, SimState& s, bool solute_only) {
    const KP<R> P = make_kp<R>(s);
    {
        const int fc = s.cur_pop[FF];
        const R* Um = s.has_U ? (const R*)s.U[s.cur_U] : nullptr;
        const R* Tm = s.has_T ? (const R*)s.T[s.cur_T] : nullptr;
        const int so = solute_only ? 1 : 0;
        // the solute sum includes the residual plane of the compensated U macro
        if constexpr (sizeof(R) == 4) {
            if (s.has_U)
                k_diag_partial<R, __nv_bfloat16><<<s.diag_blocks, 256, 0, h->stream>>>(
                    P, (const R*)s.phi[s.cur_phi], Um, Tm, (const R*)s.ux[fc], (const R*)s.uy[fc], s.part,
                    u_residual(h, s), so);
            else
                k_diag_partial<R, R><<<s.diag_blocks, 256, 0, h->stream>>>(
                    P, (const R*)s.phi[s.cur_phi], Um, Tm, (const R*)s.ux[fc], (const R*)s.uy[fc], s.part, nullptr,
                    so);
        } else {
            k_diag_partial<R, R><<<s.diag_blocks, 256, 0, h->stream>>>(
                P, (const R*)s.phi[s.cur_phi], Um, Tm, (const R*)s.ux[fc], (const R*)s.uy[fc], s.part, nullptr, so);
        }
        k_diag_final<R><<<1, DIAG_FINAL_THREADS, 0, h->stream>>>(P, s.part, s.diag_blocks, (const R*)s.phi[s.cur_phi],
                                                                 s.p.tip_cx, s.p.tip_cy, s.smax, s.dout, so);
    }
}

template <typename R>
lbm_status run_diag(lbm_sim* h, SimState& s, lbm_diag* out) {
    {
        LaunchScope ls(h, LBM_K_DIAG);
        enqueue_diag<R>(h, s);
    }
    CK(cudaGetLastError());
    double r[10];       // [9]: the solute inventory of the last initialisation
    CK(cudaMemcpyAsync(r, s.dout, sizeof r, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    out->base_step = s.step;
    out->M_C = r[0];
    out->R_M = r[9] != 0.0 ? (r[0] - r[9]) / r[9] : 0.0;
    out->H_total = r[1];
    out->nonfinite = r[2] > 0.0 ? 1 : 0;
    for (int d = 0; d < 4; ++d) out->tip[d] = r[3 + d];
    out->S_phi = r[7];
    out->J_U = r[8];
    out->reserved = 0;
    if (out->nonfinite) {
        s.sticky = true;
        return fail(h, LBM_E_NONFINITE, "non-finite value in the macroscopic fields at base step %lld", (long long)s.step);
    }
    return LBM_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

lbm_status lbm_create(const lbm_params* p, int32_t n_sims, const lbm_params* per_sim, const lbm_allocator* a,
                      void* cuda_stream, lbm_handle* out) {
    lbm_sim* h = nullptr;
    if (!out) return fail(nullptr, LBM_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!p) return fail(nullptr, LBM_E_INVALID_ARG, "params is NULL");
    if (n_sims < 1) return fail(nullptr, LBM_E_INVALID_ARG, "n_sims must be >= 1");
    if (a && (!a->alloc || !a->free)) return fail(nullptr, LBM_E_INVALID_ARG, "allocator needs alloc and free");
    std::vector<lbm_params> ps(n_sims);
    for (int i = 0; i < n_sims; ++i) {
        ps[i] = per_sim ? per_sim[i] : *p;
        std::string why;
        lbm_status st = validate(&ps[i], why);
        if (st) return fail(nullptr, st, "sim %d: %s", i, why.c_str());
        if (ps[i].precision != p->precision) return fail(nullptr, LBM_E_INVALID_ARG, "sim %d: precision differs", i);
        if ((ps[i].q_scalar == 5) != (p->q_scalar == 5))
            return fail(nullptr, LBM_E_INVALID_ARG, "sim %d: q_scalar differs", i);
    }
    h = new lbm_sim();
    h->precision = p->precision;
    h->q = p->q_scalar == 5 ? 5 : 9;
    if (a) { h->alloc = *a; h->has_alloc = true; }
    if (cuda_stream) h->stream = (cudaStream_t)cuda_stream;
    else {
        cudaError_t e = cudaStreamCreate(&h->stream);
        if (e != cudaSuccess) {
            delete h;
            return fail(nullptr, LBM_E_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        }
        h->own_stream = true;
    }
    h->sims.resize(n_sims);
    const size_t rs = real_size(h->precision), ss = store_size(h->precision);
    for (int i = 0; i < n_sims; ++i) {
        SimState& s = h->sims[i];
        s.p = ps[i];
        s.nx = s.p.nx;
        s.ny = s.p.ny;
        s.pitch = (s.nx + 31) / 32 * 32;     // rows start on 128-byte (FP32) boundaries: vector access
        s.nn = (size_t)s.pitch * s.ny;
        s.has_U = (s.p.fields & LBM_FIELD_U) != 0;
        s.has_T = (s.p.fields & LBM_FIELD_T) != 0;
        s.frozen_T = (s.p.fields & LBM_FIELD_FROZEN_T) != 0;
        s.has_flow = (s.p.fields & LBM_FIELD_FLOW) != 0;
        s.accumulated = s.p.coupling == LBM_COUPLING_ACCUMULATED;
        int64_t L = lcm64(lcm64(s.p.N_phi, s.has_U ? s.p.N_U : 1), lcm64(s.has_T ? s.p.N_T : 1, s.has_flow ? s.p.N_F : 1));
        s.half = (int)std::min<int64_t>(L, (int64_t)1 << 29);
        s.period = 2 * s.half;
        const bool present[4] = {true, s.has_U, s.has_T, s.has_flow};
        lbm_status st = LBM_OK;
        for (int f = 0; f < 4 && !st; ++f)
            for (int b = 0; b < 2 && !st; ++b)
                if (present[f])
                    st = dev_alloc(h, (f == FU ? u_planes(h->precision) : f == FT ? 2 : f == FP ? h->q - 1 : 8) * s.nn * ss,
                                   &s.pops[f][b]);
        for (int b = 0; b < 2 && !st; ++b) st = dev_alloc(h, s.nn * rs, &s.phi[b]);
        for (int b = 0; b < 2 && !st; ++b) if (s.has_U) st = dev_alloc(h, s.nn * rs, &s.U[b]);
        for (int b = 0; b < 2 && !st; ++b) if (s.has_T) st = dev_alloc(h, s.nn * rs, &s.T[b]);
        for (int b = 0; b < 2 && !st; ++b)
            if (s.has_flow) {
                st = dev_alloc(h, s.nn * rs, &s.ux[b]);
                if (!st) st = dev_alloc(h, s.nn * rs, &s.uy[b]);
                if (!st) st = dev_alloc(h, s.nn * rs, &s.rho[b]);
            }
        // accumulated coupling: the sums and their Kahan compensations, two planes each
        if (!st && s.accumulated && s.has_U) st = dev_alloc(h, 2 * s.nn * rs, &s.accU);
        if (!st && s.accumulated && s.has_T) st = dev_alloc(h, 2 * s.nn * rs, &s.accT);
        if (!st) st = dev_alloc(h, 2 * sizeof(unsigned long long), (void**)&s.smax);
        if (!st && s.frozen_T) st = dev_alloc(h, sizeof(long long), (void**)&s.clock);
        s.diag_blocks = (int)std::min<size_t>(1184, (s.nn + 255) / 256);
        if (!st) st = dev_alloc(h, 3 * sizeof(double) * s.diag_blocks, (void**)&s.part);
        if (!st) st = dev_alloc(h, 16 * sizeof(double), (void**)&s.dout);
        if (!st) st = dev_alloc(h, sizeof(KP<double>), &s.dkp);
        s.teager = s.half <= kMaxGraphPeriod ? s.period : 0;
        s.tjob_bytes = h->precision == LBM_PREC_F64 ? sizeof(TransportJob<double, double>)
                       : h->precision == LBM_PREC_F32 ? sizeof(TransportJob<float, float>)
                                                      : sizeof(TransportJob<float, __half>);
        if (!st) st = dev_alloc(h, (size_t)(s.teager + 1) * s.tjob_bytes, &s.tjobs);
        if (!st) {
            // after the zeroing memsets queued on the stream (see upload_sync)
            if (h->precision == LBM_PREC_F64) {
                const KP<double> k = make_kp<double>(s);
                st = upload_sync(h, s.dkp, &k, sizeof k);
            } else {
                const KP<float> k = make_kp<float>(s);
                st = upload_sync(h, s.dkp, &k, sizeof k);
            }
        }
        if (st) {
            std::string m = h->err;
            free_all(h);
            if (h->own_stream) cudaStreamDestroy(h->stream);
            delete h;
            return fail(nullptr, st, "%s", m.c_str());
        }
    }
    if (n_sims > 1) {
        // batched ensemble: common period and room for one period of job tables
        int64_t P = 1;
        for (auto& s : h->sims) P = std::min<int64_t>(lcm64(P, s.half), (int64_t)1 << 40);
        h->half_all = P;
        h->batching = P <= kMaxGraphPeriod;
        if (h->batching) {
            const size_t per = std::max(std::max(std::max(sizeof(PhaseJob<double, double>), sizeof(TransferJob<double>)),
                                                 std::max(sizeof(ScalarJob<double, double>), sizeof(FlowJob<double, double>))),
                                        sizeof(TransportJob<double, double>));
            // two halves x P base steps x 6 kinds x (members' jobs + alignment)
            h->job_buf_bytes = 2 * (size_t)P * 6 * ((size_t)n_sims * per + 256);
            lbm_status st = dev_alloc(h, h->job_buf_bytes, &h->job_buf);
            if (st) {
                std::string m = h->err;
                free_all(h);
                if (h->own_stream) cudaStreamDestroy(h->stream);
                delete h;
                return fail(nullptr, st, "%s", m.c_str());
            }
        }
    }
    *out = h;
    return LBM_OK;
}

lbm_status lbm_init_fields(lbm_handle h, int32_t sim, const double* phi, const double* U, const double* T,
                           const double* ux, const double* uy, const double* rho, int32_t src_is_device) {
    if (!h) return fail(nullptr, LBM_E_INVALID_ARG, "handle is NULL");
    if (sim < 0 || sim >= (int)h->sims.size()) return fail(h, LBM_E_INVALID_ARG, "sim index %d out of range", sim);
    SimState& s = h->sims[sim];
    if (!phi) return fail(h, LBM_E_INVALID_ARG, "phi is NULL");
    if (s.has_U && !U) return fail(h, LBM_E_INVALID_ARG, "U is NULL but the solute field is on");
    if (s.has_T && !T) return fail(h, LBM_E_INVALID_ARG, "T is NULL but the temperature field is on");
    if (s.has_flow && (!ux || !uy || !rho)) return fail(h, LBM_E_INVALID_ARG, "ux, uy, rho needed with the flow field on");
    const double* src[6] = {phi, s.has_U ? U : nullptr, s.has_T ? T : nullptr, s.has_flow ? ux : nullptr,
                            s.has_flow ? uy : nullptr, s.has_flow ? rho : nullptr};
    return init_common(h, sim, src, src_is_device);
}

lbm_status lbm_init_seed(lbm_handle h, int32_t sim, const lbm_seed* seeds, int32_t n_seeds, double U0, double T0,
                         uint64_t rng_seed) {
    if (!h) return fail(nullptr, LBM_E_INVALID_ARG, "handle is NULL");
    if (sim < 0 || sim >= (int)h->sims.size()) return fail(h, LBM_E_INVALID_ARG, "sim index %d out of range", sim);
    if (n_seeds < 1 || !seeds) return fail(h, LBM_E_INVALID_ARG, "need at least one seed");
    SimState& s = h->sims[sim];
    std::vector<SeedDev> sd(n_seeds);
    const double sw = std::sqrt(2.0) * s.p.W0;
    for (int k = 0; k < n_seeds; ++k) {
        const lbm_seed& q = seeds[k];
        if (q.kind < LBM_SEED_CIRCLE || q.kind > LBM_SEED_SINUSOID)
            return fail(h, LBM_E_INVALID_ARG, "seed %d: unknown kind %d", k, q.kind);
        SeedDev d{q.kind == LBM_SEED_CIRCLE ? 0 : q.kind == LBM_SEED_PLANAR ? 1 : 2, 0, s.nx, 0, s.ny,
                  q.x, q.y, q.r, q.amp, q.waves};
        if (q.kind == LBM_SEED_CIRCLE) {       // beyond this box tanh rounds to -1, which phi starts from
            const double reach = std::fabs(q.r) + 20.0 * sw + 2.0;
            d.xa = (int)std::max(0.0, std::floor(q.x - reach));
            d.xb = (int)std::min((double)s.nx, std::ceil(q.x + reach) + 1.0);
            d.ya = (int)std::max(0.0, std::floor(q.y - reach));
            d.yb = (int)std::min((double)s.ny, std::ceil(q.y + reach) + 1.0);
        }
        sd[k] = d;
    }
    // the seed-field blocks that a circle's box reaches (every block when a
    // planar or sinusoidal seed is present: n_listed = -1)
    const int nbx = (s.nx + SEED_BX - 1) / SEED_BX, nby = (s.ny + SEED_BH - 1) / SEED_BH;
    bool everywhere = false;
    std::vector<unsigned char> mark((size_t)nbx * nby, 0);
    for (const SeedDev& d : sd) {
        if (d.kind != 0) { everywhere = true; break; }
        if (d.xb <= d.xa || d.yb <= d.ya) continue;
        for (int by = d.ya / SEED_BH; by <= (d.yb - 1) / SEED_BH; ++by)
            for (int bx = d.xa / SEED_BX; bx <= (d.xb - 1) / SEED_BX; ++bx) mark[(size_t)by * nbx + bx] = 1;
    }
    std::vector<int> listed;
    if (!everywhere)
        for (size_t b = 0; b < mark.size(); ++b)
            if (mark[b]) listed.push_back((int)b);
    const size_t sbytes = (size_t)n_seeds * sizeof(SeedDev), lbytes = listed.size() * sizeof(int);
    if (h->seed_bytes < sbytes + lbytes) {
        void* p = nullptr;
        lbm_status st = dev_alloc(h, sbytes + lbytes, &p);
        if (st) return st;
        h->seed_dev = p;
        h->seed_bytes = sbytes + lbytes;
    }
    std::vector<unsigned char> up(sbytes + lbytes);
    std::memcpy(up.data(), sd.data(), sbytes);
    if (lbytes) std::memcpy(up.data() + sbytes, listed.data(), lbytes);
    // from pageable memory: returns once the bytes are staged, so up may go
    CK(cudaMemcpyAsync(h->seed_dev, up.data(), sbytes + lbytes, cudaMemcpyHostToDevice, h->stream));
    const int n_listed = everywhere ? -1 : (int)listed.size();
    return h->precision == LBM_PREC_F64 ? seed_and_init<double>(h, s, n_seeds, n_listed, U0, T0, rng_seed)
                                        : seed_and_init<float>(h, s, n_seeds, n_listed, U0, T0, rng_seed);
}

lbm_status lbm_advance(lbm_handle h, int64_t n_base_steps) {
    if (!h) return fail(nullptr, LBM_E_INVALID_ARG, "handle is NULL");
    if (n_base_steps < 0) return fail(h, LBM_E_INVALID_ARG, "n_base_steps < 0");
    for (auto& s : h->sims) {
        if (!s.initialized) return fail(h, LBM_E_STATE, "simulation not initialised");
        if (s.sticky) return fail(h, LBM_E_STATE, "a non-finite value was seen; initialise again");
    }
    if (h->batching && h->graphs && h->half_all <= kMaxGraphPeriod) {
        // batched ensemble: members in lockstep replay one graph per half of
        // the common ping-pong period
        int64_t left = n_base_steps;
        bool clock_set = false;
        const int64_t H = h->half_all;
        while (left > 0) {
            bool aligned = true;
            for (auto& s : h->sims) aligned = aligned && s.step == h->sims[0].step;
            if (!aligned) break;
            if (h->sims[0].step % H == 0 && left >= H) {
                const int which = (int)((h->sims[0].step / H) % 2);
                if (!h->bg[which].exec) {
                    lbm_status st = capture_batch(h, which);
                    if (st) return st;
                }
                if (!clock_set)
                    for (auto& s : h->sims)
                        if (s.frozen_T) k_set_clock<<<1, 1, 0, h->stream>>>(s.clock, (long long)s.step);
                clock_set = true;
                lbm_status st = batch_replay(h, which);
                if (st) return st;
                left -= H;
            } else {
                for (auto& s : h->sims) {
                    enqueue_base_step(h, s, s.step, nullptr, (long long)s.step);
                    s.step += 1;
                }
                left -= 1;
                clock_set = false;
            }
        }
        n_base_steps = left;   // members out of lockstep continue one by one below
    }
    for (auto& s : h->sims) {
        int64_t left = n_base_steps;
        bool clock_set = false;
        while (left > 0) {
            const bool use_graph = h->graphs && s.half <= kMaxGraphPeriod && (s.step % s.half) == 0 && left >= s.half;
            if (use_graph) {
                const int which = (int)((s.step / s.half) % 2);
                if (!s.g[which].exec) {
                    lbm_status st = capture_graph(h, s, which);
                    if (st) return st;
                }
                if (s.frozen_T && !clock_set) {
                    k_set_clock<<<1, 1, 0, h->stream>>>(s.clock, (long long)s.step);
                    clock_set = true;
                }
                lbm_status st = graph_replay(h, s, which);
                if (st) return st;
                left -= s.half;
            } else {
                enqueue_base_step(h, s, s.step, nullptr, (long long)s.step);
                s.step += 1;
                left -= 1;
                clock_set = false;
            }
        }
    }
    CK(cudaGetLastError());
    // timed launches are read without a host wait until many are queued
    return h->pending.size() > 4096 ? collect_pending(h) : LBM_OK;
}

lbm_status lbm_fields(lbm_handle h, int32_t sim, uint32_t which, void* dst, int32_t dst_is_device, int32_t as_f64) {
    if (!h) return fail(nullptr, LBM_E_INVALID_ARG, "handle is NULL");
    if (sim < 0 || sim >= (int)h->sims.size()) return fail(h, LBM_E_INVALID_ARG, "sim index %d out of range", sim);
    if (which > 7) return fail(h, LBM_E_INVALID_ARG, "unknown field %u", which);
    if (!dst) return fail(h, LBM_E_INVALID_ARG, "dst is NULL");
    SimState& s = h->sims[sim];
    if (!s.initialized) return fail(h, LBM_E_STATE, "simulation not initialised");
    return h->precision == LBM_PREC_F64 ? read_field<double>(h, s, which, dst, dst_is_device, as_f64)
                                        : read_field<float>(h, s, which, dst, dst_is_device, as_f64);
}

lbm_status lbm_diagnostics(lbm_handle h, int32_t sim, lbm_diag* out) {
    if (!h) return fail(nullptr, LBM_E_INVALID_ARG, "handle is NULL");
    if (sim < 0 || sim >= (int)h->sims.size()) return fail(h, LBM_E_INVALID_ARG, "sim index %d out of range", sim);
    if (!out) return fail(h, LBM_E_INVALID_ARG, "out is NULL");
    SimState& s = h->sims[sim];
    if (!s.initialized) return fail(h, LBM_E_STATE, "simulation not initialised");
    lbm_status st = h->precision == LBM_PREC_F64 ? run_diag<double>(h, s, out) : run_diag<float>(h, s, out);
    if (st == LBM_OK || st == LBM_E_NONFINITE) {
        lbm_status c = collect_pending(h);
        if (c) return c;
    }
    return st;
}

const char* lbm_last_error(lbm_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

void lbm_destroy(lbm_handle h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (auto& s : h->sims) drop_graph(s);
    drop_batch_graph(h);
    for (auto& t : h->pending) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    for (auto e : h->event_pool) cudaEventDestroy(e);
    free_all(h);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
}

lbm_status lbm_set_graphs(lbm_handle h, int32_t enable) {
    if (!h) return fail(nullptr, LBM_E_INVALID_ARG, "handle is NULL");
    h->graphs = enable != 0;
    return LBM_OK;
}

lbm_status lbm_timing_enable(lbm_handle h, uint32_t kind_mask) {
    if (!h) return fail(nullptr, LBM_E_INVALID_ARG, "handle is NULL");
    if (kind_mask >> LBM_K_COUNT) return fail(h, LBM_E_INVALID_ARG, "unknown kernel kind bit");
    h->timing_mask = kind_mask;
    for (auto& s : h->sims) drop_graph(s);
    drop_batch_graph(h);
    return LBM_OK;
}

lbm_status lbm_set_tile(lbm_handle h, int32_t kind, int32_t ty) {
    if (!h) return fail(nullptr, LBM_E_INVALID_ARG, "handle is NULL");
    if (kind < 0 || (kind > LBM_K_FLOW && kind != LBM_K_TRANSPORT))
        return fail(h, LBM_E_INVALID_ARG, "kind %d is not an update kernel", kind);
    if (!valid_variant(kind, ty))
        return fail(h, LBM_E_INVALID_ARG, "variant %d is not a tile height in {4, 8, 16}%s", ty,
                    has_strips(kind) ? ", a strip height in {-4, -8, -16, -32} or 1000 + a vector strip height in "
                                       "{8, 16, 32}" : has_vstrips(kind) ? " or 1000 + a vector strip height in {8, 16, 32}"
                                                                         : "");
    for (auto& s : h->sims) {
        s.tile[kind] = ty;
        drop_graph(s);
    }
    h->batch_tile[kind] = ty;
    drop_batch_graph(h);
    return LBM_OK;
}

lbm_status lbm_set_fusion(lbm_handle h, int32_t enable) {
    if (!h) return fail(nullptr, LBM_E_INVALID_ARG, "handle is NULL");
    h->fuse = enable != 0;
    h->fuse_auto = false;
    for (auto& s : h->sims) drop_graph(s);
    drop_batch_graph(h);
    return LBM_OK;
}

lbm_status lbm_set_batching(lbm_handle h, int32_t enable) {
    if (!h) return fail(nullptr, LBM_E_INVALID_ARG, "handle is NULL");
    if (enable && (h->sims.size() < 2 || !h->job_buf))
        return fail(h, LBM_E_INVALID_ARG, "batching needs >= 2 simulations with a common period <= %d", kMaxGraphPeriod);
    h->batching = enable != 0;
    drop_batch_graph(h);
    return LBM_OK;
}

lbm_status lbm_timing_read(lbm_handle h, double* ms, int64_t* count, int32_t reset) {
    if (!h) return fail(nullptr, LBM_E_INVALID_ARG, "handle is NULL");
    lbm_status st = collect_pending(h);
    if (st) return st;
    for (int k = 0; k < LBM_K_COUNT; ++k) {
        if (ms) ms[k] = h->timing_ms[k];
        if (count) count[k] = h->timing_n[k];
        if (reset) { h->timing_ms[k] = 0.0; h->timing_n[k] = 0; }
    }
    return LBM_OK;
}

lbm_status lbm_get_fusion(lbm_handle h, int32_t* enabled) {
    if (!h) return fail(nullptr, LBM_E_INVALID_ARG, "handle is NULL");
    if (!enabled) return fail(h, LBM_E_INVALID_ARG, "enabled is NULL");
    *enabled = h->fuse ? 1 : 0;
    return LBM_OK;
}

lbm_status lbm_autotune(lbm_handle h, int32_t reps, int32_t* chosen) {
    if (!h) return fail(nullptr, LBM_E_INVALID_ARG, "handle is NULL");
    if (reps < 1) return fail(h, LBM_E_INVALID_ARG, "reps must be >= 1");
    static const int variants[10] = {4, 8, 16, -4, -8, -16, -32, VS + 8, VS + 16, VS + 32};
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    const uint32_t mask = h->timing_mask;
    h->timing_mask = 0;
    double cost_fused = 0.0, cost_staged = 0.0;   // per half period, summed over the simulations
    bool choose = false;
    for (auto& s : h->sims) {
        if (!s.initialized) { cudaEventDestroy(a); cudaEventDestroy(b); h->timing_mask = mask;
                              return fail(h, LBM_E_STATE, "simulation not initialised"); }
        const bool can_fuse = !s.accumulated;
        const bool pick = h->fuse_auto && can_fuse;   // time both paths and choose
        const bool fused = h->fuse && can_fuse;
        const bool staged = pick || !fused;
        const bool present[LBM_K_COUNT] = {true, !s.accumulated && staged, s.has_U && staged, s.has_T && staged,
                                           s.has_flow && staged, false, false, can_fuse && (pick || fused)};
        // one launch of `kind` with tile height v on the current state; the
        // transport launch runs the stages in `combo` (bit 0 transfer, 1 U,
        // 2 T, 3 flow), every stage the simulation has by default
        const int all_stages = 1 | (s.has_U ? 2 : 0) | (s.has_T ? 4 : 0) | (s.has_flow ? 8 : 0);
        auto tune_launch = [&](int kind, int v, int combo) {
            if (kind == LBM_K_TRANSPORT) {
                const int keep = s.tile[kind];
                s.tile[kind] = v;
                transport_any(h, s, combo & 1, (combo & 2) != 0, (combo & 4) != 0, (combo & 8) != 0);
                s.tile[kind] = keep;
            } else {
                launch_any(h, s, kind, v, s.clock, 0);
            }
        };
        auto time_launch = [&](int kind, int v, int combo, float* ms) -> lbm_status {
            tune_launch(kind, v, combo);       // warm the variant
            CK(cudaEventRecord(a, h->stream));
            for (int r = 0; r < reps; ++r) tune_launch(kind, v, combo);
            CK(cudaEventRecord(b, h->stream));
            CK(cudaEventSynchronize(b));
            CK(cudaEventElapsedTime(ms, a, b));
            *ms /= (float)reps;
            return LBM_OK;
        };
        double best_ms[LBM_K_COUNT] = {};
        for (int kind = 0; kind < LBM_K_COUNT; ++kind) {
            if (!present[kind]) continue;
            float best = 1e30f;
            int bestv = s.tile[kind];
            for (int v : variants) {
                if (!valid_variant(kind, v)) continue;
                float ms = 0.f;
                lbm_status st = time_launch(kind, v, all_stages, &ms);
                if (st) return st;
                if (ms < best) { best = ms; bestv = v; }
            }
            s.tile[kind] = bestv;
            best_ms[kind] = best;
        }
        if (pick) {
            // cost of one half period (lcm of the update factors) both ways
            choose = true;
            const lbm_params& q = s.p;
            double combo_ms[16];
            for (double& c : combo_ms) c = -1.0;
            const int steps = std::min(s.half, kMaxGraphPeriod);
            for (int k = 0; k < steps; ++k) {
                const bool ph = (k + 1) % q.N_phi == 0;
                const bool u = s.has_U && (k + 1) % q.N_U == 0;
                const bool t = s.has_T && (k + 1) % q.N_T == 0;
                const bool f = s.has_flow && (k + 1) % q.N_F == 0;
                const double base = ph ? best_ms[LBM_K_PHASE] : 0.0;
                cost_staged += base + (ph ? best_ms[LBM_K_TRANSFER] : 0.0) + (u ? best_ms[LBM_K_SCALAR_U] : 0.0) +
                               (t ? best_ms[LBM_K_SCALAR_T] : 0.0) + (f ? best_ms[LBM_K_FLOW] : 0.0);
                const int combo = (ph ? 1 : 0) | (u ? 2 : 0) | (t ? 4 : 0) | (f ? 8 : 0);
                if (combo && combo_ms[combo] < 0.0) {
                    float ms = 0.f;
                    lbm_status st = time_launch(LBM_K_TRANSPORT, s.tile[LBM_K_TRANSPORT], combo, &ms);
                    if (st) return st;
                    combo_ms[combo] = ms;
                }
                cost_fused += base + (combo ? combo_ms[combo] : 0.0);
            }
        }
        drop_graph(s);
    }
    if (choose) h->fuse = cost_fused < cost_staged;
    if (h->batching) {
        // the batched launches: one job per member that has the field, at the
        // current parities (idempotent like the single launches)
        bool any_acc = false;
        for (auto& s : h->sims) any_acc = any_acc || s.accumulated;
        drop_batch_graph(h);
        const bool fused = h->fuse && !any_acc;
        for (int kind = 0; kind < LBM_K_COUNT; ++kind) {
            if (kind == LBM_K_DIAG || kind == LBM_K_INIT) continue;
            if (fused != (kind == LBM_K_TRANSPORT) && kind != LBM_K_PHASE) continue;
            if (kind == LBM_K_TRANSFER && any_acc) continue;
            float best = 1e30f;
            int bestv = h->batch_tile[kind];
            for (int v : variants) {
                if (!valid_variant(kind, v)) continue;
                h->batch_tile[kind] = v;
                clear_records(h);
                h->recording = true;
                for (auto& s : h->sims) {
                    const bool has = kind == LBM_K_PHASE || kind == LBM_K_TRANSFER ||
                                     (kind == LBM_K_SCALAR_U && s.has_U) || (kind == LBM_K_SCALAR_T && s.has_T) ||
                                     (kind == LBM_K_FLOW && s.has_flow);
                    if (kind == LBM_K_TRANSPORT) transport_any(h, s, true, s.has_U, s.has_T, s.has_flow);
                    else if (has) launch_any(h, s, kind, v, s.clock, 0);
                }
                h->recording = false;
                if (!h->rec_jobs[kind]) break;
                {
                    lbm_status st = upload_sync(h, h->job_buf, h->rec[kind].data(), h->rec[kind].size());
                    if (st) return st;
                }
                launch_batch_any(h, kind, v, h->job_buf, h->rec_jobs[kind], h->rec_tiles[kind]);
                CK(cudaEventRecord(a, h->stream));
                for (int r = 0; r < reps; ++r)
                    launch_batch_any(h, kind, v, h->job_buf, h->rec_jobs[kind], h->rec_tiles[kind]);
                CK(cudaEventRecord(b, h->stream));
                CK(cudaEventSynchronize(b));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, a, b));
                if (ms < best) { best = ms; bestv = v; }
            }
            h->batch_tile[kind] = bestv;
        }
        clear_records(h);
    }
    for (auto& s : h->sims) CK(cudaMemsetAsync(s.smax, 0, 2 * sizeof(unsigned long long), h->stream));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    h->timing_mask = mask;
    if (chosen)
        for (int k = 0; k < LBM_K_COUNT; ++k) chosen[k] = h->sims[0].tile[k];
    return LBM_OK;
}

lbm_status lbm_launch_counts(lbm_handle h, int64_t* counts) {
    if (!h || !counts) return fail(h, LBM_E_INVALID_ARG, "NULL argument");
    for (int k = 0; k < LBM_K_COUNT; ++k) counts[k] = h->launches[k];
    return LBM_OK;
}

lbm_status lbm_set_orientation(lbm_handle h, int32_t sim, const double* theta, int32_t src_is_device) {
    if (!h) return fail(nullptr, LBM_E_INVALID_ARG, "handle is NULL");
    if (sim < 0 || sim >= (int)h->sims.size()) return fail(h, LBM_E_INVALID_ARG, "sim index %d out of range", sim);
    SimState& s = h->sims[sim];
    const size_t rs = real_size(h->precision);
    if (!theta) {
        s.ori = nullptr;
    } else {
        if (!s.ori_buf) {
            lbm_status st = dev_alloc(h, s.nn * rs, &s.ori_buf);
            if (st) return st;
        }
        const size_t n = (size_t)s.nx * s.ny, need = n * sizeof(double);
        if (h->staging_bytes < need) {
            void* p = nullptr;
            lbm_status st = dev_alloc(h, need, &p);
            if (st) return st;
            h->staging = (double*)p;
            h->staging_bytes = need;
        }
        CK(cudaMemcpyAsync(h->staging, theta, need, src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           h->stream));
        const dim3 blk(32, 8), grd((s.nx + 31) / 32, (s.ny + 7) / 8);
        if (h->precision == LBM_PREC_F64)
            k_from_f64<double><<<grd, blk, 0, h->stream>>>(h->staging, (double*)s.ori_buf, s.nx, s.ny, s.pitch);
        else
            k_from_f64<float><<<grd, blk, 0, h->stream>>>(h->staging, (float*)s.ori_buf, s.nx, s.ny, s.pitch);
        CK(cudaGetLastError());
        s.ori = s.ori_buf;
    }
    // the coefficient block carries the pointer; kernels read it at every launch
    if (h->precision == LBM_PREC_F64) {
        const KP<double> k = make_kp<double>(s);
        return upload_sync(h, s.dkp, &k, sizeof k);
    }
    const KP<float> k = make_kp<float>(s);
    return upload_sync(h, s.dkp, &k, sizeof k);
}

lbm_status lbm_device_bytes(lbm_handle h, size_t* bytes) {
    if (!h || !bytes) return fail(h, LBM_E_INVALID_ARG, "NULL argument");
    *bytes = h->bytes;
    return LBM_OK;
}

}  // extern "C"

// ===========================================================================
// Diagnostics without allocation.
//
// Some callers cannot call cudaMalloc: a monitoring hook that runs inside
// another framework's step loop (where cudaMalloc would synchronise the device
// and break that framework's stream ordering), or a process whose device
// memory is owned by a caching allocator under a fixed budget.  For them,
// lbm_diagnostics_noalloc reduces fields they already hold in their own
// device buffers, with the reduction's scratch in the file-scope array below
// instead of memory from the allocator or cudaMalloc.
//
// The array is a fixed kNoAllocBlocks x 3 partial sums plus 16 result / flag
// slots (about 28 KB); every GPU that loads this library keeps it until the
// process exits.  All calls share it and it keeps the last call's contents:
// the two maxima slots are cleared on every call (the partials and results
// are fully overwritten), and calls whose work overlaps on the GPU (two
// streams, or two host threads) race on it.
// ===========================================================================
namespace {

constexpr int kNoAllocBlocks = 1184;                 // 8 blocks per SM on 148 SMs
constexpr int kNoAllocSlots = 3 * kNoAllocBlocks + 16;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocSlots];

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// with the device current -- on every call: a lookup costs far less than the
// reduction, and no address survives a device reset (which unloads the
// module and places the array anew when it is loaded again).
cudaError_t noalloc_scratch(double** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = (double*)p;
    return cudaSuccess;
}

template <typename R>
lbm_status noalloc_diag(const SimState& s, const void* phi, const void* U, const void* T, const void* ux,
                        const void* uy, cudaStream_t st, double* scratch, lbm_diag* out) {
    lbm_sim* h = nullptr;   // errors are reported through lbm_last_error(NULL)
    const KP<R> P = make_kp<R>(s);
    const int blocks = (int)std::min<size_t>(kNoAllocBlocks, (s.nn + 255) / 256);
    double* part = scratch;
    unsigned long long* smax = (unsigned long long*)(scratch + 3 * kNoAllocBlocks);
    double* res = scratch + 3 * kNoAllocBlocks + 2;
    CK(cudaMemsetAsync(smax, 0, 2 * sizeof(unsigned long long), st));   // the maxima must start at zero
    k_diag_partial<R><<<blocks, 256, 0, st>>>(P, (const R*)phi, (const R*)U, (const R*)T, (const R*)ux,
                                              (const R*)uy, part);
    k_diag_final<R><<<1, DIAG_FINAL_THREADS, 0, st>>>(P, part, blocks, (const R*)phi, s.p.tip_cx, s.p.tip_cy, smax, res);
    CK(cudaGetLastError());
    double r[9];
    CK(cudaMemcpyAsync(r, res, sizeof r, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out->base_step = 0;
    out->M_C = r[0];
    out->H_total = r[1];
    out->nonfinite = r[2] > 0.0 ? 1 : 0;
    for (int d = 0; d < 4; ++d) out->tip[d] = r[3 + d];
    out->S_phi = 0.0;
    out->J_U = 0.0;
    out->reserved = 0;
    out->R_M = 0.0;
    return out->nonfinite ? fail(nullptr, LBM_E_NONFINITE, "non-finite value in the fields") : LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_diagnostics_noalloc(const lbm_params* p, const void* phi, const void* U, const void* T,
                                              const void* ux, const void* uy, void* cuda_stream, lbm_diag* out) {
    lbm_sim* h = nullptr;
    if (!p || !phi || !out) return fail(nullptr, LBM_E_INVALID_ARG, "params, phi and out must not be NULL");
    std::string why;
    lbm_status st = validate(p, why);
    if (st) return fail(nullptr, st, "%s", why.c_str());
    if ((int64_t)p->nx * p->ny > (int64_t)INT32_MAX)
        return fail(nullptr, LBM_E_INVALID_ARG, "lattice of %lld nodes exceeds the 2^31 - 1 node limit",
                    (long long)p->nx * p->ny);
    SimState s;   // host-side description only: no device memory
    s.p = *p;
    s.nx = p->nx;
    s.ny = p->ny;
    s.pitch = p->nx;
    s.nn = (size_t)p->nx * p->ny;
    s.has_U = (p->fields & LBM_FIELD_U) != 0;
    s.has_T = (p->fields & LBM_FIELD_T) != 0;
    s.frozen_T = (p->fields & LBM_FIELD_FROZEN_T) != 0;
    s.has_flow = (p->fields & LBM_FIELD_FLOW) != 0;
    if ((s.has_U && !U) || (s.has_T && !T) || (s.has_flow && (!ux || !uy)))
        return fail(nullptr, LBM_E_INVALID_ARG, "a field that is switched on was passed as NULL");
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    // the call synchronises its stream and copies to the host: never inside a capture
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(stream, &cap));
    if (cap != cudaStreamCaptureStatusNone)
        return fail(nullptr, LBM_E_INVALID_ARG, "the stream is being captured into a CUDA graph; this call "
                                                "synchronises its stream and may not run during a capture");
    double* scratch = nullptr;
    CK(noalloc_scratch(&scratch));
    return p->precision == LBM_PREC_F64 ? noalloc_diag<double>(s, phi, U, T, ux, uy, stream, scratch, out)
                                        : noalloc_diag<float>(s, phi, U, T, ux, uy, stream, scratch, out);
}
