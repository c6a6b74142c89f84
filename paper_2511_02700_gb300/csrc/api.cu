// C ABI of pide2d (include/pide2d.h): workspace layout, argument checks,
// the precomputation and the time loop of Algorithm 1.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/pide2d.h"
#include "common.cuh"
#include "internal.h"

using namespace pide;

namespace {

constexpr double kPi = 3.14159265358979323846;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Gauss-Legendre nodes/weights on [-1, 1]: Newton's method on P_n with the
// three-term recurrence, w_i = 2 / ((1 - x_i^2) P_n'(x_i)^2).
void gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// quadrature orders of the device precompute
constexpr int kGlNear = 10, kGlFar = 6, kGlEdge = 32, kGlPay = 16, kGlVfar = 4;
constexpr double kTanhSinhStep = 0.125;
constexpr int kGlTotal = 2 * (kGlNear + kGlFar + kGlEdge + kGlPay + kGlVfar);

enum Region {
    R_V0, R_V1, R_V2, R_V3, R_V4, R_BV, R_BY, R_W, R_X, R_OUT,   // 10 state-sized fields
    R_RES, R_DLT,                                                 // R fields
    R_S, R_WH, R_WHI, R_E, R_TWR, R_TWD,
    R_E1D, R_E2D, R_E1F, R_E2F, R_E1L, R_E2L, R_SIN2D, R_SIN2R,
    R_OMEGA, R_PART, R_PARAMS, R_MOMENT, R_GL, R_RESID, R_CTL,
    R_COUNT
};

struct Layout {
    Geometry g;
    int prec;
    size_t off[R_COUNT];
    size_t size[R_COUNT];
    size_t total;
};

template <typename R>
void fill_layout(int N, Layout& L) {
    Geometry& g = L.g;
    g.N = N;
    g.P = 2 * N;
    g.rows = g.P + 2;
    g.ng = spectrum_groups<R>(g.P);
    g.nge = N / rgroup<R>();
    g.ldS = round_up(N + 1, 32);
    g.ldR = round_up(N + 1, 32);
    g.eoff = N / 2 + 3;
    const size_t fieldS = (size_t)(N + 1) * g.ldS * 8;
    const size_t fieldR = (size_t)(N + 1) * g.ldR * sizeof(R);
    for (int i = R_V0; i <= R_OUT; ++i) L.size[i] = fieldS;
    L.size[R_RES] = L.size[R_DLT] = fieldR;
    L.size[R_S] = (size_t)g.ng * g.rows * cgroup_bytes<R>();
    L.size[R_WH] = L.size[R_WHI] = (size_t)g.ng * g.P * cgroup_bytes<R>();
    L.size[R_E] = (size_t)g.nge * N * rgroup_bytes<R>();
    L.size[R_TWR] = (size_t)tw_entries(g.P) * 2 * sizeof(R);   // base table + stage tables
    L.size[R_TWD] = (size_t)tw_entries(g.P) * 16;
    const size_t tl = (size_t)(2 * N + 7);
    L.size[R_E1D] = L.size[R_E2D] = tl * 8;
    L.size[R_E1F] = L.size[R_E2F] = tl * 4;
    L.size[R_E1L] = L.size[R_E2L] = tl * 4;
    L.size[R_SIN2D] = (size_t)(N + 1) * 8;
    L.size[R_SIN2R] = (size_t)(N + 1) * sizeof(R);
    L.size[R_OMEGA] = (size_t)N * N * 8;
    L.size[R_PART] = (size_t)((N * N + 255) / 256) * 3 * 8;
    L.size[R_PARAMS] = 16 * 8;
    L.size[R_MOMENT] = moment_doubles() * 8;
    L.size[R_GL] = (size_t)(kGlTotal + kKtabMax) * 8;     // quadrature nodes, then the K_nu table
    L.size[R_RESID] = 16;
    L.size[R_CTL] = sizeof(FpCtl);
    size_t o = 0;
    for (int i = 0; i < R_COUNT; ++i) {
        L.off[i] = o;
        o += align256(L.size[i]);
    }
    L.total = o;
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

std::string check_grid(const pide2d_grid* g) {
    if (!g) return "grid is NULL";
    if (!is_pow2(g->n) || g->n < 8 || g->n > 4096) return "grid.n must be a power of two in [8, 4096]";
    if (g->n_z != 0 && g->n_z != g->n / 2) return "grid.n_z must be 0 or n/2";
    if (!(g->half_width > 0.0) || !std::isfinite(g->half_width)) return "grid.half_width must be positive";
    if (!std::isfinite(g->s_center[0]) || !std::isfinite(g->s_center[1])) return "grid.s_center must be finite";
    if (g->sl_order != 0 && g->sl_order != 1 && g->sl_order != 3) return "grid.sl_order must be 0, 1 or 3";
    if (g->precision != PIDE2D_FP64 && g->precision != PIDE2D_FP32_BULK) return "grid.precision invalid";
    return "";
}

bool layout_for(const pide2d_grid* g, Layout& L) {
    L.prec = g->precision;
    if (g->precision == PIDE2D_FP64) fill_layout<double>(g->n, L);
    else fill_layout<float>(g->n, L);
    return true;
}

thread_local std::string g_create_error;

}  // namespace

namespace pide {
// error channel of the handle-free entry points (read by pide2d_last_error(NULL))
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace pide

struct pide2d {
    pide2d_grid grid;
    pide2d_model model;
    pide2d_contract contract;
    double theta, dt, tol;
    int kmax, damping, n_steps, sl_order, host_loop;
    Layout L;
    cudaStream_t stream;
    char* ws;
    double h, s_lo1, s_lo2;
    double par[9];
    int steps_done;
    std::vector<int> hist, freel;
    int bv, by;
    pide2d_stats stats;
    std::string err;
    bool broken;
    // device-side fixed-point loop: instantiated loop graphs keyed by their kernel arguments
    struct LoopGraph { std::string key; cudaGraph_t graph; cudaGraphExec_t exec; };
    std::vector<LoopGraph> graphs;
    cudaStream_t cap = nullptr;    // private stream used only to record graphs
    int graph_builds = 0;
    bool ctl_dirty = false;        // device loop ran since the last read of FpCtl
    bool last_step_device = false;
    FpCtl ctl{};                   // host copy of the device statistics
    int nonconv_seen = 0;
    // adjoint tape (pide2d_record / pide2d_adjoint)
    struct Tape {
        char* base = nullptr;
        size_t bytes = 0;
        int interval = 0, ndirs = 0, nckpt = 0, seg_slots = 0;
        size_t off_ckpt = 0, off_seg = 0, off_final = 0, off_adj = 0, off_spec = 0, off_scr = 0, off_acc = 0;
        std::vector<int> ckpt_cnt;
    } tape;
    bool seg_record = false;       // replay of a tape segment: keep every theta step's V and B_w V
    bool force_host_loop = false;
    bool group_nonconv = false;    // a theta step of the multi-job loop stopped without converging
    int seg_slot = 0;
    struct StepMeta { double theta, ht, tau_prev, tau; };
    std::vector<StepMeta> seg_meta;
    // tracing
    bool prof = false;
    struct Rec { int cls; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;

    template <typename T> T* at(int region) const { return reinterpret_cast<T*>(ws + L.off[region]); }
    void* field(int i) const { return ws + L.off[R_V0 + i]; }
};

#define PIDE_CUDA(call)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            H->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
            H->broken = true;                                                             \
            return PIDE2D_ERR_CUDA;                                                       \
        }                                                                                 \
    } while (0)

namespace {

cudaError_t prof_event(pide2d* H, cudaEvent_t* e) {
    if (!H->pool.empty()) {
        *e = H->pool.back();
        H->pool.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(e);
}

// launch `call` bracketed by events of class `cls` when tracing is on
#define PIDE_LAUNCH(cls, call)                                                            \
    do {                                                                                  \
        if (H->prof) {                                                                    \
            pide2d::Rec r_{cls, nullptr, nullptr};                                        \
            PIDE_CUDA(prof_event(H, &r_.a));                                              \
            PIDE_CUDA(prof_event(H, &r_.b));                                              \
            PIDE_CUDA(cudaEventRecord(r_.a, H->stream));                                  \
            PIDE_CUDA(call);                                                              \
            PIDE_CUDA(cudaEventRecord(r_.b, H->stream));                                  \
            H->recs.push_back(r_);                                                        \
        } else {                                                                          \
            PIDE_CUDA(call);                                                              \
        }                                                                                 \
    } while (0)

}  // namespace

// ---------------------------------------------------------------------------
// adjoint tape: checkpoints of the time loop every `interval` time steps
// (history fields and B_w V), a segment buffer for the replay of one
// interval (V and B_w V after every theta step), the adjoint fields, the
// weight spectra of the adjoint and of the parameter directions, scratch
// for the finite differences of the precompute, and the FP64 accumulators.
// ---------------------------------------------------------------------------
namespace {
enum AdjField { A_LAM, A_MU, A_BMU, A_NU, A_XI, A_PEND, A_COUNT };
constexpr int kAdjAcc = 6;        // <xi,V>, <xi,dxx V>, <xi,dxy V>, <xi,dyy V>, shift 1, shift 2
constexpr size_t kMomentBytes = (moment_doubles() * 8 + 255) / 256 * 256;   // moment buffer, 256-aligned

struct TapeLayout {
    size_t ckpt, seg, fin, adj, spec, dw, specx, cacc, cfield, scr, acc, total;
    size_t field, spec1, omega, part, rows, nparts;
    int nckpt, seg_slots;
};

TapeLayout tape_layout(const Layout& L, int n_steps, int interval, int ndirs) {
    TapeLayout t{};
    const int N = L.g.N;
    t.field = align256(L.size[R_V0]);
    t.spec1 = align256(L.size[R_WH]);
    t.omega = align256((size_t)N * N * 8);
    t.part = align256(L.size[R_PART]);
    t.rows = align256((size_t)spectrum_groups<double>(L.g.P) * L.g.P * cgroup_bytes<double>());
    t.nparts = align256((size_t)adjoint_dot_blocks(N) * 4 * 8);
    t.nckpt = (n_steps + interval - 1) / interval;
    t.seg_slots = interval + 3;                       // the damped first step has four theta steps
    size_t o = 0;
    t.ckpt = o;  o += (size_t)t.nckpt * 5 * t.field;  // hist (up to 4) + B_w V per checkpoint
    t.seg = o;   o += (size_t)t.seg_slots * 2 * t.field;
    t.fin = o;   o += 5 * t.field;                    // the final state, put back after the adjoint
    t.adj = o;   o += (size_t)A_COUNT * t.field;
    t.spec = o;  o += 2 * t.spec1;                    // flipped Wh, Whi
    t.dw = o;    o += (size_t)ndirs * t.omega;         // the weights' derivative along each direction
    t.specx = o; o += align256(L.size[R_S]);           // spectrum rows of the adjoint field xi
    t.cacc = o;  o += align256((size_t)(L.g.P / 2 + 1) * L.g.P * 16);   // FP64 sum of conj(xi^) V^
    t.cfield = o; o += t.omega;                        // its inverse: the correlation at the N x N lags
    t.scr = o;   o += 3 * t.omega + t.part + kMomentBytes + 2 * 256 + t.rows + t.nparts;
    t.acc = o;   o += align256((size_t)(kAdjAcc + ndirs) * 8);
    t.total = o;
    return t;
}
}  // namespace

static void* tape_ckpt(pide2d* H, const TapeLayout& t, int k, int slot) {
    return H->tape.base + t.ckpt + ((size_t)k * 5 + slot) * t.field;
}
static void* tape_seg(pide2d* H, const TapeLayout& t, int slot, int which) {
    return H->tape.base + t.seg + ((size_t)slot * 2 + which) * t.field;
}

static pide2d_status save_checkpoint(pide2d* H, int k) {
    const TapeLayout t = tape_layout(H->L, H->n_steps, H->tape.interval, H->tape.ndirs);
    const size_t fb = H->L.size[R_V0];
    for (size_t i = 0; i < H->hist.size(); ++i)
        PIDE_CUDA(cudaMemcpyAsync(tape_ckpt(H, t, k, (int)i), H->field(H->hist[i]), fb, cudaMemcpyDeviceToDevice,
                                  H->stream));
    PIDE_CUDA(cudaMemcpyAsync(tape_ckpt(H, t, k, 4), H->field(H->bv), fb, cudaMemcpyDeviceToDevice, H->stream));
    H->tape.ckpt_cnt[k] = (int)H->hist.size();
    return PIDE2D_OK;
}

// the time-loop state at the start of time step k * interval + 1
static pide2d_status restore_checkpoint(pide2d* H, int k) {
    const TapeLayout t = tape_layout(H->L, H->n_steps, H->tape.interval, H->tape.ndirs);
    const size_t fb = H->L.size[R_V0];
    const int cnt = H->tape.ckpt_cnt[k];
    for (int i = 0; i < cnt; ++i)
        PIDE_CUDA(cudaMemcpyAsync(H->field(i), tape_ckpt(H, t, k, i), fb, cudaMemcpyDeviceToDevice, H->stream));
    PIDE_CUDA(cudaMemcpyAsync(H->field(5), tape_ckpt(H, t, k, 4), fb, cudaMemcpyDeviceToDevice, H->stream));
    H->hist.clear();
    for (int i = 0; i < cnt; ++i) H->hist.push_back(i);
    H->freel.clear();
    for (int i = 4; i >= cnt; --i) H->freel.push_back(i);
    H->bv = 5;
    H->by = 6;
    H->steps_done = k * H->tape.interval;
    return PIDE2D_OK;
}

// during a segment replay: V^s (field `res`) and B_w V^s (now in field bv)
template <typename R>
static pide2d_status record_theta_step(pide2d* H, int res, double theta, double ht, double tau_prev, double tau) {
    const TapeLayout t = tape_layout(H->L, H->n_steps, H->tape.interval, H->tape.ndirs);
    if (H->seg_slot >= t.seg_slots) {
        H->err = "tape segment overflow";
        return PIDE2D_ERR_STATE;
    }
    const size_t fb = H->L.size[R_V0];
    PIDE_CUDA(cudaMemcpyAsync(tape_seg(H, t, H->seg_slot, 0), H->field(res), fb, cudaMemcpyDeviceToDevice, H->stream));
    PIDE_CUDA(cudaMemcpyAsync(tape_seg(H, t, H->seg_slot, 1), H->field(H->bv), fb, cudaMemcpyDeviceToDevice,
                              H->stream));
    H->seg_meta.push_back({theta, ht, tau_prev, tau});
    H->seg_slot++;
    return PIDE2D_OK;
}

// ---------------------------------------------------------------------------
// the fixed-point loop of one theta step as a CUDA graph:
//   reset(FpCtl.k, FpCtl.conv) -> while(cond) { col_solve, dst_row, check, col, inv } -> tally
// k_fp_check clears the condition at convergence, at kmax or on a non-finite
// residual, so every launch of the graph ends.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kMaxLoopGraphs = 24;

template <typename R>
cudaError_t record_loop_graph(pide2d* H, cudaGraph_t g, const ColSolveArgs<R>& da, const DstRowArgs<R>& ra,
                              const ColArgs<R>& ca, const InvArgs<R>& ia, const char** where) {
    cudaStream_t cs = H->cap;
    FpCtl* ctl = H->at<FpCtl>(R_CTL);
    cudaError_t e = cudaSuccess;
#define PIDE_GTRY(call)              \
    do {                             \
        e = (call);                  \
        if (e != cudaSuccess) {      \
            *where = #call;          \
            return e;                \
        }                            \
    } while (0)
    cudaGraphConditionalHandle hnd;
    PIDE_GTRY(cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault));
    cudaMemsetParams mp{};
    mp.dst = ctl;                  // FpCtl.k and FpCtl.conv
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = 2;
    mp.height = 1;
    cudaGraphNode_t reset = nullptr, loop = nullptr;
    PIDE_GTRY(cudaGraphAddMemsetNode(&reset, g, nullptr, 0, &mp));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hnd;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    PIDE_GTRY(cudaGraphAddNode(&loop, g, &reset, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];

    // body: one iteration of the increment form of eq. 3.24
    PIDE_GTRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    auto iteration = [&]() -> cudaError_t {
        cudaError_t x;
        if ((x = launch_col_solve<R>(da, cs)) != cudaSuccess) return x;
        if ((x = cudaMemsetAsync(H->at<void>(R_RESID), 0, 16, cs)) != cudaSuccess) return x;
        if ((x = launch_dst_row<R>(ra, cs)) != cudaSuccess) return x;
        if ((x = launch_fp_check<R>(H->at<void>(R_RESID), ctl, H->tol, H->kmax, (unsigned long long)hnd, cs)) !=
            cudaSuccess)
            return x;
        if ((x = launch_col<R>(ca, cs)) != cudaSuccess) return x;
        return launch_row_inverse<R>(ia, cs);
    };
    e = iteration();
    cudaGraph_t got = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &got);
    if (e != cudaSuccess) { *where = "loop body launches"; return e; }
    if (e2 != cudaSuccess) { *where = "cudaStreamEndCapture(body)"; return e2; }

    // after the loop: fold the step's count into the statistics
    PIDE_GTRY(cudaStreamBeginCaptureToGraph(cs, g, &loop, nullptr, 1, cudaStreamCaptureModeRelaxed));
    e = launch_fp_tally(ctl, cs);
    const cudaError_t e3 = cudaStreamEndCapture(cs, &got);
    if (e != cudaSuccess) { *where = "launch_fp_tally"; return e; }
    if (e3 != cudaSuccess) { *where = "cudaStreamEndCapture"; return e3; }
#undef PIDE_GTRY
    return cudaSuccess;
}

}  // namespace

template <typename R>
static pide2d_status loop_graph(pide2d* H, const ColSolveArgs<R>& da, const DstRowArgs<R>& ra, const ColArgs<R>& ca,
                                const InvArgs<R>& ia, cudaGraphExec_t* exec) {
    std::string key;
    key.append(reinterpret_cast<const char*>(&da), sizeof da);
    key.append(reinterpret_cast<const char*>(&ra), sizeof ra);
    key.append(reinterpret_cast<const char*>(&ca), sizeof ca);
    key.append(reinterpret_cast<const char*>(&ia), sizeof ia);
    for (const auto& e : H->graphs)
        if (e.key == key) {
            *exec = e.exec;
            return PIDE2D_OK;
        }
    if (!H->cap) PIDE_CUDA(cudaStreamCreateWithFlags(&H->cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    PIDE_CUDA(cudaGraphCreate(&g, 0));
    const char* where = "";
    cudaError_t e = record_loop_graph<R>(H, g, da, ra, ca, ia, &where);
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&ex, g, 0);
        where = "cudaGraphInstantiate";
    }
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        H->err = std::string("fixed-point loop graph: ") + where + ": " + cudaGetErrorString(e);
        H->broken = true;
        return PIDE2D_ERR_CUDA;
    }
    if (H->graphs.size() >= kMaxLoopGraphs) {
        // the oldest entry may still be queued on the stream: wait before freeing it
        PIDE_CUDA(cudaStreamSynchronize(H->stream));
        cudaGraphExecDestroy(H->graphs.front().exec);
        cudaGraphDestroy(H->graphs.front().graph);
        H->graphs.erase(H->graphs.begin());
    }
    H->graphs.push_back({std::move(key), g, ex});
    H->graph_builds++;
    *exec = ex;
    return PIDE2D_OK;
}

// read the device loop statistics (synchronises the stream)
static pide2d_status read_ctl(pide2d* H) {
    if (!H->ctl_dirty) return PIDE2D_OK;
    PIDE_CUDA(cudaMemcpyAsync(&H->ctl, H->at<FpCtl>(R_CTL), sizeof(FpCtl), cudaMemcpyDeviceToHost, H->stream));
    PIDE_CUDA(cudaStreamSynchronize(H->stream));
    H->ctl_dirty = false;
    return PIDE2D_OK;
}

// host-loop statistics combined with those of the device loop
static pide2d_stats combined_stats(const pide2d* H) {
    pide2d_stats s = H->stats;
    const double nn = (double)H->grid.n * H->grid.n;
    s.steps_done = H->steps_done;
    s.fp_iters_total += H->ctl.total;
    if (H->ctl.max_step > s.fp_iters_max) s.fp_iters_max = H->ctl.max_step;
    s.cell_iters += nn * (double)(H->ctl.total + H->ctl.substeps);
    if (H->last_step_device) s.last_resid = H->ctl.step_resid;
    return s;
}

// NOT_CONVERGED if a device-loop theta step stopped without meeting eq. 3.25 since the last check
static pide2d_status check_device_convergence(pide2d* H) {
    if (H->ctl.nonconv > H->nonconv_seen) {
        char buf[200];
        std::snprintf(buf, sizeof buf,
                      "fixed-point iteration not converged in %d theta step(s) (kmax %d, last resid %.3e, tol %.3e)",
                      H->ctl.nonconv - H->nonconv_seen, H->kmax, H->ctl.last_resid, H->tol);
        H->err = buf;
        H->nonconv_seen = H->ctl.nonconv;
        return PIDE2D_ERR_NOT_CONVERGED;
    }
    return PIDE2D_OK;
}

// Lagrange weights of the departure stencil for a shift of q cells (eq. 3.22):
// first tap offset o, weights w and their derivatives dw/dq.
static void sl_stencil(int order, double q, int* o, double w[4], double dw[4]) {
    const int fl = (int)std::floor(q);
    const double f = q - fl;
    if (order == 1) {
        *o = fl;
        w[0] = 1.0 - f;
        w[1] = f;
        w[2] = w[3] = 0.0;
        dw[0] = -1.0;
        dw[1] = 1.0;
        dw[2] = dw[3] = 0.0;
    } else {
        *o = fl - 1;
        w[0] = -f * (f - 1.0) * (f - 2.0) / 6.0;
        w[1] = (f + 1.0) * (f - 1.0) * (f - 2.0) / 2.0;
        w[2] = -(f + 1.0) * f * (f - 2.0) / 2.0;
        w[3] = (f + 1.0) * f * (f - 1.0) / 6.0;
        dw[0] = -(3.0 * f * f - 6.0 * f + 2.0) / 6.0;
        dw[1] = (3.0 * f * f - 4.0 * f - 1.0) / 2.0;
        dw[2] = -(3.0 * f * f - 2.0 * f - 2.0) / 2.0;
        dw[3] = (3.0 * f * f - 1.0) / 6.0;
    }
}

// one implicit solve of eq. 3.24 by the fixed-point iteration (3.24)-(3.25),
// in increment form with the DST-I preconditioner:
//   (1 + h_t theta r_w) Y - h_t theta D Y - h_t theta B Y = W  (+ the far-field terms)
// Y holds the start Y^{0} (its boundary ring is part of the input); on return
// Y holds the solution and BY = B Y.  far = 0 solves with a zero far field
// (halo and ring) and takes the weight spectra Wh/Whi as given, which is how
// the transposed system of the adjoint is solved.
template <typename R>
struct SolveSpec {
    St<R>* Y;
    St<R>* BY;
    const St<R>* W;
    int far;
    double Kd;
    // difference sweep: when Vprev is set, the first sweep transforms
    // Y^{0} - Vprev with the halo g(tau) - g(tau_prev) and B_w Y^{0} =
    // BVprev + that sweep (BVprev = B_w Vprev with the halo at tau_prev)
    const St<R>* Vprev;
    const St<R>* BVprev;
    double Kd_prev;
    const void* Wh;
    const void* Whi;
    double theta, ht;
    int step_end;
    bool device_loop;
};

// kernel arguments of one implicit solve (see fixed_point_solve): the full
// sweep of Y^{0} (fa, caf, iaf) and the iteration body (da, ra, cai, iai).
// Blocks that key the loop graphs are zeroed bytewise.
template <typename R>
struct SolveArgs {
    FwdArgs<R> fa;
    ColArgs<R> caf, cai;
    InvArgs<R> iaf, iai;
    ColSolveArgs<R> da;
    DstRowArgs<R> ra;
};

template <typename R>
static void build_solve_args(pide2d* H, const SolveSpec<R>& sp, SolveArgs<R>* out) {
    const Geometry g = H->L.g;
    const int N = g.N;
    const double hg = H->h;
    const double htt = sp.ht * sp.theta;
    const double rw = H->par[1], a11 = H->par[4], a12 = H->par[5], a22 = H->par[6];
    const R d11 = (R)(0.5 * a11 / (hg * hg)), d22 = (R)(0.5 * a22 / (hg * hg)), d12 = (R)(0.25 * a12 / (hg * hg));
    const void* tw = H->at<void>(R_TWR);
    std::memset(out, 0, sizeof *out);
    FwdArgs<R>& fa = out->fa;
    fa.g = g;
    fa.mode = sp.far ? FWD_FULL : FWD_FULL0;
    const bool diff = sp.far && sp.Vprev && sp.BVprev;
    if (diff) {
        fa.mode = FWD_DIFF;
        fa.Yref = sp.Vprev;
        fa.Kd_prev = (R)sp.Kd_prev;
        fa.dKd = (R)(sp.Kd - sp.Kd_prev);
    }
    fa.Y = sp.Y;
    fa.D = H->at<R>(R_DLT);
    fa.E1 = (const R*)(sizeof(R) == 4 ? (const void*)H->at<float>(R_E1F) : (const void*)H->at<double>(R_E1D));
    fa.E2 = (const R*)(sizeof(R) == 4 ? (const void*)H->at<float>(R_E2F) : (const void*)H->at<double>(R_E2D));
    fa.Kd = (R)sp.Kd;
    fa.payoff = H->contract.payoff;
    fa.S = H->at<void>(R_S);
    fa.pair0 = 0;
    fa.npairs = N + 1;
    fa.tw = tw;
    ColArgs<R>& ca = out->caf;
    ca.g = g;
    ca.mode = COL_FULL;
    ca.S = H->at<void>(R_S);
    ca.Wh = sp.Wh;
    ca.rlo = 0;
    ca.rhi = g.P + 2;
    ca.tw = tw;
    if (sp.far && H->contract.payoff == PIDE2D_PUT_AVG) {
        // halo rows above the domain where the put's far field vanishes for every
        // staged s1, i.e. (e^{s1,min} + e^{s2}) / 2 >= K e^{-r tau}: their transforms
        // are zero, so the row pass stops before them and the column pass treats
        // them as zero (a relative margin of 1e-6 covers the FP32 evaluation)
        // (for the difference sweep both g(tau) and g(tau_prev) vanish there)
        const double kz = diff ? std::max(sp.Kd, sp.Kd_prev) : sp.Kd;
        const double e1min = std::exp(H->s_lo1 + (-N / 2 - 1) * hg);
        int m2z = 3 * N / 2 + 1;
        for (int m2 = N; m2 <= 3 * N / 2; ++m2) {
            if (0.5 * (e1min + std::exp(H->s_lo2 + m2 * hg)) >= kz * (1.0 + 1e-6)) {
                m2z = m2;
                break;
            }
        }
        const int rho_z = m2z + N / 2 + 1;          // first zero row of the staged layout
        fa.npairs = (rho_z + 1) / 2;
        ca.rhi = 2 * fa.npairs;                     // rows written by the row pass
    }
    InvArgs<R>& ia = out->iaf;
    ia.g = g;
    ia.mode = INV_FULL;
    ia.do_resid = 1;
    ia.S = H->at<void>(R_S);
    ia.BY = sp.BY;
    ia.Y = sp.Y;
    ia.W = sp.W;
    ia.r = H->at<R>(R_RES);
    ia.D = H->at<R>(R_DLT);
    ia.htt = (R)htt;
    ia.cid = (R)(1.0 + htt * rw);
    ia.d11 = d11;
    ia.d22 = d22;
    ia.d12 = d12;
    ia.rw = (R)rw;
    ia.rw_lo = (R)(rw - (double)(R)rw);
    ia.BV = diff ? sp.BVprev : nullptr;
    ia.E = H->at<R>(R_E);
    ia.tw = tw;
    ColSolveArgs<R>& da = out->da;
    da.g = g;
    da.E = H->at<R>(R_E);
    da.sin2 = H->at<R>(R_SIN2R);
    da.rc0 = (R)(1.0 + htt * rw);
    da.rc1 = (R)(2.0 * htt * a11 / (hg * hg));
    da.rc2 = (R)(2.0 * htt * a22 / (hg * hg));
    da.rscale = (R)(2.0 / N);
    DstRowArgs<R>& ra = out->ra;
    ra.g = g;
    ra.E = H->at<R>(R_E);
    ra.Y = sp.Y;
    ra.D = H->at<R>(R_DLT);
    ra.resid = H->at<void>(R_RESID);
    ra.S = H->at<void>(R_S);
    ra.tw = tw;
    std::memcpy(&out->cai, &ca, sizeof ca);     // bytewise: padding stays zero for the graph keys
    out->cai.mode = COL_INCR;
    out->cai.Wh = sp.Whi;
    out->cai.rlo = N / 2 + 2;
    out->cai.rhi = N / 2 + N + 2;
    std::memcpy(&out->iai, &ia, sizeof ia);
    out->iai.mode = INV_INCR;
    out->iai.BV = nullptr;          // the increment pass does not read it (and it must not key the loop graphs)
}

template <typename R>
static pide2d_status fixed_point_solve(pide2d* H, const SolveSpec<R>& sp, int* iters_out, double* resid_out,
                                       bool* conv_out) {
    *conv_out = false;
    SolveArgs<R> A;
    build_solve_args<R>(H, sp, &A);
    St<R>* Y = sp.Y;
    St<R>* BY = sp.BY;
    // B_w Y^{0} by a full sweep and the first residual
    PIDE_LAUNCH(PIDE2D_KERNEL_ROW_FORWARD_FULL, launch_row_forward<R>(A.fa, H->stream));
    PIDE_LAUNCH(PIDE2D_KERNEL_COL_FULL, launch_col<R>(A.caf, H->stream));
    PIDE_LAUNCH(PIDE2D_KERNEL_ROW_INVERSE_FULL, launch_row_inverse<R>(A.iaf, H->stream));
    ColSolveArgs<R>& da = A.da;
    DstRowArgs<R>& ra = A.ra;
    ColArgs<R>& ca = A.cai;
    InvArgs<R>& ia = A.iai;

    if (sp.device_loop) {
        // the iteration loop runs on the device (graph while-node); the step's
        // fields Y and B_w Y are passed through FpCtl, so the graph depends on
        // h_t and theta only; statistics are kept in FpCtl
        FpCtl* ctl = H->at<FpCtl>(R_CTL);
        ia.do_resid = 1;
        ia.conv_flag = &ctl->conv;
        ia.BY = nullptr;
        ia.BYind = reinterpret_cast<St<R>* const*>(&ctl->BY);
        ra.Y = nullptr;
        ra.Yind = reinterpret_cast<St<R>* const*>(&ctl->Y);
        cudaGraphExec_t ex = nullptr;
        const pide2d_status gs = loop_graph<R>(H, da, ra, ca, ia, &ex);
        if (gs != PIDE2D_OK) return gs;
        PIDE_CUDA(launch_fp_setup(ctl, Y, BY, sp.step_end, H->stream));
        PIDE_CUDA(cudaGraphLaunch(ex, H->stream));
        H->ctl_dirty = true;
        *iters_out = 0;
        *resid_out = 0.0;
        *conv_out = true;      // reported through FpCtl
        return PIDE2D_OK;
    }

    int k = 0;
    double resid = 0.0;
    bool conv = false;
    for (k = 1; k <= H->kmax; ++k) {
        PIDE_LAUNCH(PIDE2D_KERNEL_COL_SOLVE, launch_col_solve<R>(da, H->stream));
        PIDE_CUDA(cudaMemsetAsync(H->at<void>(R_RESID), 0, 16, H->stream));
        PIDE_LAUNCH(PIDE2D_KERNEL_DST_ROW, launch_dst_row<R>(ra, H->stream));
        double rhost = 0.0;
        PIDE_CUDA(cudaMemcpyAsync(&rhost, H->at<void>(R_RESID), sizeof(double), cudaMemcpyDeviceToHost, H->stream));
        PIDE_CUDA(cudaStreamSynchronize(H->stream));
        resid = rhost;
        conv = resid < H->tol;
        if (!std::isfinite(resid)) break;
        // B_w of the increment keeps B_w Y^{k} current (needed for the next W);
        // its row pass ran inside k_dst_row
        PIDE_LAUNCH(PIDE2D_KERNEL_COL_INCR, launch_col<R>(ca, H->stream));
        ia.do_resid = conv ? 0 : 1;
        PIDE_LAUNCH(PIDE2D_KERNEL_ROW_INVERSE_INCR, launch_row_inverse<R>(ia, H->stream));
        if (conv) break;
    }
    if (!conv) k = H->kmax;
    *iters_out = k;
    *resid_out = resid;
    *conv_out = conv;
    return PIDE2D_OK;
}

// ---------------------------------------------------------------------------
// one theta step (eq. 3.23): W and Y^{n,0} (Algorithm 1 steps 2-3), then the
// implicit solve
// ---------------------------------------------------------------------------
// arguments of one theta step (eq. 3.23): W and Y^{n,0} (Algorithm 1 steps 2-3)
// into pa, the implicit solve into sp
template <typename R>
static pide2d_status build_theta_step(pide2d* H, const int* list, int cnt, double theta, double ht, double tau_prev,
                                      double tau, int res, int step_end, PrepArgs<R>* pa_out, SolveSpec<R>* sp_out) {
    const Geometry g = H->L.g;
    const int N = g.N;
    const double hg = H->h;
    const double htm = ht * (1.0 - theta);
    const double rw = H->par[1], a11 = H->par[4], a12 = H->par[5], a22 = H->par[6];
    const R d11 = (R)(0.5 * a11 / (hg * hg)), d22 = (R)(0.5 * a22 / (hg * hg)), d12 = (R)(0.25 * a12 / (hg * hg));
    const double Kd_prev = H->contract.strike * std::exp(-H->model.r * tau_prev);
    const double Kd_now = H->contract.strike * std::exp(-H->model.r * tau);
    St<R>* Y = (St<R>*)H->field(res);
    St<R>* W = H->at<St<R>>(R_W);
    St<R>* BV = (St<R>*)H->field(H->bv);
    St<R>* BY = (St<R>*)H->field(H->by);

    PrepArgs<R>& pa = *pa_out;
    std::memset(&pa, 0, sizeof pa);
    pa.g = g;
    for (int i = 0; i < 4; ++i) pa.V[i] = (const St<R>*)H->field(list[i < cnt ? i : 0]);
    pa.hcount = cnt;
    pa.BV = BV;
    pa.W = W;
    pa.Y = Y;
    pa.cz = H->at<R>(R_RES);   // the residual field is free until the first sweep of the step
    pa.htm = (R)htm;
    pa.rw = (R)rw;
    pa.rw_lo = (R)(rw - (double)(R)rw);
    pa.d11 = d11;
    pa.d22 = d22;
    pa.d12 = d12;
    const double q[2] = {H->par[7] * ht / hg, H->par[8] * ht / hg};
    // the departure stencil and the far-field tables reach N/4 cells at most
    if (!(std::fabs(q[0]) <= N / 4) || !(std::fabs(q[1]) <= N / 4)) {
        H->err = "semi-Lagrangian shift exceeds N/4 cells: time step too large";
        return PIDE2D_ERR_ARG;
    }
    double w[2][4], dw[2][4];
    sl_stencil(H->sl_order, q[0], &pa.o1, w[0], dw[0]);
    sl_stencil(H->sl_order, q[1], &pa.o2, w[1], dw[1]);
    pa.nt = H->sl_order == 1 ? 2 : 4;
    for (int i = 0; i < 4; ++i) {
        pa.w1[i] = (R)w[0][i];
        pa.w2[i] = (R)w[1][i];
    }
    pa.E1d = H->at<double>(R_E1D);
    pa.E2d = H->at<double>(R_E2D);
    pa.E1h = H->at<float>(R_E1F);
    pa.E2h = H->at<float>(R_E2F);
    pa.E1l = H->at<float>(R_E1L);
    pa.E2l = H->at<float>(R_E2L);
    pa.Kd_prev = Kd_prev;
    pa.Kd_now = Kd_now;
    pa.Kdp_h = (float)Kd_prev;
    pa.Kdp_l = (float)(Kd_prev - (double)pa.Kdp_h);
    pa.Kdn_h = (float)Kd_now;
    pa.Kdn_l = (float)(Kd_now - (double)pa.Kdn_h);
    pa.payoff = H->contract.payoff;

    SolveSpec<R>& sp = *sp_out;
    sp = SolveSpec<R>{};
    sp.Y = Y;
    sp.BY = BY;
    sp.W = W;
    sp.far = 1;
    sp.Kd = Kd_now;
    sp.Vprev = pa.V[0];             // V^{n-1}, whose B_w V (with the halo at tau_prev) is BV
    sp.BVprev = BV;
    sp.Kd_prev = Kd_prev;
    sp.Wh = H->at<void>(R_WH);
    sp.Whi = H->at<void>(R_WHI);
    sp.theta = theta;
    sp.ht = ht;
    sp.step_end = step_end;
    sp.device_loop = !H->host_loop && !H->prof && !H->force_host_loop;
    return PIDE2D_OK;
}

template <typename R>
static pide2d_status theta_step(pide2d* H, const int* list, int cnt, double theta, double ht, double tau_prev,
                                double tau, int res, int step_end, int* iters_out, double* resid_out) {
    const int N = H->L.g.N;
    PrepArgs<R> pa;
    SolveSpec<R> sp;
    {
        const pide2d_status bs = build_theta_step<R>(H, list, cnt, theta, ht, tau_prev, tau, res, step_end, &pa, &sp);
        if (bs != PIDE2D_OK) return bs;
    }
    PIDE_LAUNCH(PIDE2D_KERNEL_PREP, launch_prep<R>(pa, H->stream));
    int k = 0;
    double resid = 0.0;
    bool conv = false;
    const pide2d_status s = fixed_point_solve<R>(H, sp, &k, &resid, &conv);
    if (s != PIDE2D_OK) return s;
    std::swap(H->bv, H->by);
    if (H->seg_record) {
        const pide2d_status rs = record_theta_step<R>(H, res, theta, ht, tau_prev, tau);
        if (rs != PIDE2D_OK) return rs;
    }
    *iters_out = k;
    *resid_out = resid;
    if (sp.device_loop) return PIDE2D_OK;
    H->stats.cell_iters += (double)N * N * (k + 1);
    if (!conv) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "fixed-point iteration not converged after %d iterations (resid %.3e, tol %.3e)",
                      H->kmax, resid, H->tol);
        H->err = buf;
        return PIDE2D_ERR_NOT_CONVERGED;
    }
    return PIDE2D_OK;
}

template <typename R>
static pide2d_status do_step(pide2d* H, int* iters, double* resid) {
    pide2d_status st = PIDE2D_OK;
    if (H->tape.base && !H->seg_record && H->steps_done % H->tape.interval == 0) {
        const pide2d_status cs = save_checkpoint(H, H->steps_done / H->tape.interval);
        if (cs != PIDE2D_OK) return cs;
    }
    int k = 0;
    double r = 0.0;
    int ktot = 0;
    const double dt = H->dt;
    if (H->steps_done == 0 && H->damping) {
        const int v0 = H->hist[0];
        int cur = v0;
        for (int j = 0; j < 4; ++j) {
            const int res = H->freel.back();
            H->freel.pop_back();
            const int list[1] = {cur};
            const pide2d_status s = theta_step<R>(H, list, 1, 1.0, dt / 4.0, j * (dt / 4.0), (j + 1) * (dt / 4.0),
                                                  res, j == 3 ? 1 : 0, &k, &r);
            if (s == PIDE2D_ERR_CUDA || s == PIDE2D_ERR_ARG) return s;
            if (s != PIDE2D_OK) st = s;
            if (cur != v0) H->freel.push_back(cur);
            cur = res;
            ktot += k;
        }
        H->hist.assign({cur, v0});
    } else {
        const int res = H->freel.back();
        H->freel.pop_back();
        const int cnt = (int)H->hist.size() < 4 ? (int)H->hist.size() : 4;
        const int n = H->steps_done + 1;
        const pide2d_status s = theta_step<R>(H, H->hist.data(), cnt, H->theta, dt, (n - 1) * dt, n * dt, res, 1,
                                              &k, &r);
        if (s == PIDE2D_ERR_CUDA || s == PIDE2D_ERR_ARG) return s;
        if (s != PIDE2D_OK) st = s;
        H->hist.insert(H->hist.begin(), res);
        if (H->hist.size() > 4) {
            H->freel.push_back(H->hist.back());
            H->hist.pop_back();
        }
        ktot = k;
    }
    H->steps_done++;
    H->stats.steps_done = H->steps_done;
    H->last_step_device = !H->host_loop && !H->prof && !H->force_host_loop;
    if (H->last_step_device) return st;   // counts are on the device (FpCtl)
    H->stats.fp_iters_total += ktot;
    if (ktot > H->stats.fp_iters_max) H->stats.fp_iters_max = ktot;
    H->stats.last_resid = r;
    if (iters) *iters = ktot;
    if (resid) *resid = r;
    return st;
}

// Gauss-Legendre nodes and weights of the device precompute, in the order
// the kernels expect: near, far, edge, payoff, very far
static std::vector<double> quadrature_nodes() {
    std::vector<double> gl(kGlTotal);
    double* p = gl.data();
    gauss_legendre(kGlNear, p, p + kGlNear);
    gauss_legendre(kGlFar, p + 2 * kGlNear, p + 2 * kGlNear + kGlFar);
    gauss_legendre(kGlEdge, p + 2 * (kGlNear + kGlFar), p + 2 * (kGlNear + kGlFar) + kGlEdge);
    gauss_legendre(kGlPay, p + 2 * (kGlNear + kGlFar + kGlEdge), p + 2 * (kGlNear + kGlFar + kGlEdge) + kGlPay);
    double* pv = p + 2 * (kGlNear + kGlFar + kGlEdge + kGlPay);
    gauss_legendre(kGlVfar, pv, pv + kGlVfar);
    return gl;
}

// the precompute on a z-lattice of N x N cells of width hz (N_z = N/2)
static cudaError_t precompute_core(int N, double hz, double* dgl, const pide2d_model& m, double* omega,
                                   double* part, double* moment, double* params, cudaStream_t s) {
    // Levy density constants (Sec. 4)
    const double r11 = m.rho[0], r12 = m.rho[1], r22 = m.rho[2];
    const double det = r11 * r22 - r12 * r12;
    LevyParams L{};
    L.alpha = m.alpha;
    L.nu = 1.0 + m.alpha;
    L.Ri11 = r22 / det;
    L.Ri12 = -r12 / det;
    L.Ri22 = r11 / det;
    L.b1 = L.Ri11 * m.eta[0] + L.Ri12 * m.eta[1];
    L.b2 = L.Ri12 * m.eta[0] + L.Ri22 * m.eta[1];
    const double eta_rho2 = m.eta[0] * L.b1 + m.eta[1] * L.b2;
    L.c1 = std::sqrt(eta_rho2 + 2.0 * m.lambda);
    L.logpref = std::log(m.delta / kPi) + L.nu * std::log(L.c1) - 0.5 * std::log(det);
    L.pref0 = m.delta / (kPi * std::sqrt(det));
    L.gamma_nu = std::tgamma(L.nu);
    // ln(e^x K_nu(x)) from a table over every x = c1 |z|_{rho^-1} that a quadrature
    // node can take: from 1e-8 (below it the R_I moment uses the x -> 0 limit of
    // x^nu K_nu) up to the lattice corner
    {
        const double tr = 0.5 * (L.Ri11 + L.Ri22);
        const double dd = std::sqrt(0.25 * (L.Ri11 - L.Ri22) * (L.Ri11 - L.Ri22) + L.Ri12 * L.Ri12);
        const double x_lo = 1e-8;
        const double x_hi = 1.1 * L.c1 * std::sqrt(tr + dd) * std::sqrt(2.0) * (N / 2 + 1) * hz;
        double du = 0.01;
        const double span = std::log(x_hi / x_lo);
        int n = (int)std::ceil(span / du) + 14;
        if (n > kKtabMax) {
            du = span / (kKtabMax - 14);
            n = kKtabMax;
        }
        // nodes on the lattice du Z: models with the same nu (the perturbed ones of
        // the adjoint's central differences) read the same interpolant of x
        const double u0 = du * std::floor(std::log(x_lo) / du - 5.0);
        double* tab = dgl + kGlTotal;
        const cudaError_t te = launch_ktab(L.nu, u0, du, n, tab, s);
        if (te != cudaSuccess) return te;
        L.ktab = tab;
        L.ku0 = u0;
        L.kidu = 1.0 / du;
        L.kn = n;
    }

    WeightJob j{};
    j.N = N;
    j.h = hz;
    j.M2 = (int)std::ceil(std::sqrt(0.1) * (N / 2) - 0.5);
    j.gl_near_x = dgl;
    j.gl_near_w = dgl + kGlNear;
    j.n_near = kGlNear;
    j.gl_far_x = dgl + 2 * kGlNear;
    j.gl_far_w = dgl + 2 * kGlNear + kGlFar;
    j.n_far = kGlFar;
    j.gl_vfar_x = dgl + 2 * (kGlNear + kGlFar + kGlEdge + kGlPay);
    j.gl_vfar_w = j.gl_vfar_x + kGlVfar;
    j.n_vfar = kGlVfar;
    int nblocks = 0;
    cudaError_t e = launch_weights(L, j, omega, part, &nblocks, s);
    if (e != cudaSuccess) return e;
    const double* edge = dgl + 2 * (kGlNear + kGlFar);
    e = launch_moment(L, 2.0 * hz, edge, edge + kGlEdge, kGlEdge, kTanhSinhStep, moment, s);
    if (e != cudaSuccess) return e;
    return launch_finalize(part, nblocks, moment, m.r, m.sigma_cov, params, s);
}

// weights w (eq. 3.5), the R_I moment (eq. 3.3) and the rates (eq. 3.6) of a
// model, into the given device buffers (params: the 9 values of pide2d_get_weights)
static pide2d_status run_precompute(pide2d* H, const pide2d_model& m, double* omega, double* part, double* moment,
                                    double* params) {
    PIDE_CUDA(precompute_core(H->L.g.N, H->h, H->at<double>(R_GL), m, omega, part, moment, params, H->stream));
    return PIDE2D_OK;
}

// conj(fft2(Omega zero-padded))/P^2 (eq. 3.13) of an N x N weight array: FP64
// row spectra in `rows` ((P/2+1) x P x 16 bytes of scratch), then the FP64
// column FFTs write Wh (and Whi, the increment-sweep variant, unless NULL)
template <typename R>
static pide2d_status weight_spectrum(pide2d* H, const double* omega, void* Wh, void* Whi, void* rows) {
    const Geometry g = H->L.g;
    Geometry gd = g;
    gd.rows = g.P;
    gd.ng = spectrum_groups<double>(g.P);
    FwdArgs<double> wa{};
    wa.g = gd;
    wa.mode = FWD_WEIGHTS;
    wa.omega = omega;
    wa.S = rows;
    wa.pair0 = 0;
    wa.npairs = g.N / 2;
    wa.tw = H->at<void>(R_TWD);
    PIDE_CUDA(launch_row_forward<double>(wa, H->stream));
    PIDE_CUDA(launch_weights_col<R>(gd, rows, Wh, Whi, H->at<void>(R_TWD), H->stream));
    return PIDE2D_OK;
}

// B_w V^0 of an FP32-bulk handle, computed in FP64.  Every later sweep of the
// time loop transforms a difference (Y^{n,0} - V^{n-1}, or an increment), so
// B_w V carries the rounding of this first sweep through the whole solve.
// The FP64 spectra are staged in the state-field region, which holds nothing
// else yet (V^0 is in field 0; the result goes to field bv at the end):
//   R_OUT (field 9)   V^0 in FP64, then B_w V^0 at the interior nodes
//   fields 1..8       FP64 row spectra of Omega, then the FP64 spectrum of V^0,
//                     and the FP64 weight spectrum conj(w^)/P^2 after them
// Each state field holds >= 8 (N+1)^2 bytes, so fields 1..8 hold the
// 32 (N+1)^2 + 32 N (N+1) bytes needed.  The staging is cleared afterwards.
static pide2d_status bv0_fp64(pide2d* H) {
    const Geometry g = H->L.g;
    const int N = g.N;
    cudaStream_t s = H->stream;
    Geometry gd = g;
    gd.ng = spectrum_groups<double>(g.P);
    gd.nge = N / rgroup<double>();
    const size_t rows_b = (size_t)gd.ng * g.P * cgroup_bytes<double>();
    const size_t spec_b = (size_t)gd.ng * gd.rows * cgroup_bytes<double>();
    const size_t wh_off = align256(std::max(rows_b, spec_b));
    const size_t wh_b = (size_t)gd.ng * g.P * cgroup_bytes<double>();
    const size_t avail = H->L.off[R_OUT] - H->L.off[R_V1];
    if (wh_off + wh_b > avail) {
        H->err = "internal: FP64 staging of B_w V^0 does not fit";
        return PIDE2D_ERR_STATE;
    }
    char* base = (char*)H->field(1);
    void* S64 = base;
    void* Wh64 = base + wh_off;
    double* V64 = H->at<double>(R_OUT);
    const void* twd = H->at<void>(R_TWD);
    // conj(w^)/P^2 in FP64 (eq. 3.13), as weight_spectrum with an FP64 output
    Geometry gw = gd;
    gw.rows = g.P;
    FwdArgs<double> wa{};
    wa.g = gw;
    wa.mode = FWD_WEIGHTS;
    wa.omega = H->at<double>(R_OMEGA);
    wa.S = S64;
    wa.pair0 = 0;
    wa.npairs = N / 2;
    wa.tw = twd;
    PIDE_CUDA(launch_row_forward<double>(wa, s));
    PIDE_CUDA(launch_weights_col<double>(gw, S64, Wh64, nullptr, twd, s));
    // V^0 in FP64 (the values field 0 holds as double-float pairs)
    const double* dgl = H->at<double>(R_GL);
    const double* glp = dgl + 2 * (kGlNear + kGlFar + kGlEdge);
    PIDE_CUDA(launch_payoff<double>(gd, H->at<double>(R_E1D), H->at<double>(R_E2D), H->s_lo1, H->s_lo2, H->h,
                                    H->contract.strike, H->contract.payoff, glp, glp + kGlPay, kGlPay, V64, s));
    // the state V^0 is the same FP64 payoff split into (hi, lo)
    PIDE_CUDA(launch_state_from_double<float>(g, V64, g.ldS, (St<float>*)H->field(0), s));
    FwdArgs<double> fa{};
    fa.g = gd;
    fa.mode = FWD_FULL;
    fa.Y = V64;
    fa.E1 = H->at<double>(R_E1D);
    fa.E2 = H->at<double>(R_E2D);
    fa.Kd = H->contract.strike;
    fa.payoff = H->contract.payoff;
    fa.S = S64;
    fa.pair0 = 0;
    fa.npairs = N + 1;
    fa.tw = twd;
    PIDE_CUDA(launch_row_forward<double>(fa, s));
    ColArgs<double> ca{};
    ca.g = gd;
    ca.mode = COL_FULL;
    ca.S = S64;
    ca.Wh = Wh64;
    ca.rlo = 0;
    ca.rhi = g.P + 2;
    ca.tw = twd;
    PIDE_CUDA(launch_col<double>(ca, s));
    InvArgs<double> ia{};
    ia.g = gd;
    ia.mode = INV_OUT;
    ia.do_resid = 0;
    ia.S = S64;
    ia.out = V64;                  // the interior nodes of V^0 are read before this pass
    ia.tw = twd;
    PIDE_CUDA(launch_row_inverse<double>(ia, s));
    PIDE_CUDA(launch_state_from_double<float>(g, V64, g.ldS, (St<float>*)H->field(H->bv), s));
    PIDE_CUDA(cudaMemsetAsync(H->field(1), 0, H->L.off[R_BV] - H->L.off[R_V1], s));
    PIDE_CUDA(cudaMemsetAsync(H->field(6), 0, H->L.off[R_RES] - H->L.off[R_BY], s));
    return PIDE2D_OK;
}

template <typename R>
static pide2d_status do_create(pide2d* H) {
    const Geometry g = H->L.g;
    const int N = g.N;
    cudaStream_t s = H->stream;
    // quadrature nodes
    const std::vector<double> gl = quadrature_nodes();
    double* dgl = H->at<double>(R_GL);
    PIDE_CUDA(cudaMemsetAsync(H->ws, 0, H->L.total, s));
    PIDE_CUDA(cudaMemcpyAsync(dgl, gl.data(), gl.size() * 8, cudaMemcpyHostToDevice, s));

    // tables
    PIDE_CUDA(launch_tables(N, H->s_lo1, H->s_lo2, H->h, H->at<double>(R_E1D), H->at<double>(R_E2D),
                            H->at<float>(R_E1F), H->at<float>(R_E2F), H->at<float>(R_E1L), H->at<float>(R_E2L),
                            H->at<double>(R_SIN2D), s));
    PIDE_CUDA(launch_twiddles<R>(g.P, H->at<void>(R_TWR), s));
    PIDE_CUDA(launch_twiddles<double>(g.P, H->at<void>(R_TWD), s));

    // weights, R_I moment and rates (eqs. 3.3, 3.5, 3.6), then
    // omega-hat = conj(fft2(Omega padded))/P^2 (eq. 3.13) with the FP64 row
    // spectra in the (not yet used) state-field region
    {
        const pide2d_status ps = run_precompute(H, H->model, H->at<double>(R_OMEGA), H->at<double>(R_PART),
                                                H->at<double>(R_MOMENT), H->at<double>(R_PARAMS));
        if (ps != PIDE2D_OK) return ps;
    }
    {
        const pide2d_status ws = weight_spectrum<R>(H, H->at<double>(R_OMEGA), H->at<void>(R_WH),
                                                    H->at<void>(R_WHI), H->field(0));
        if (ws != PIDE2D_OK) return ws;
    }
    PIDE_CUDA(cudaMemsetAsync(H->field(0), 0, H->L.off[R_RES] - H->L.off[R_V0], s));
    PIDE_CUDA(cudaMemsetAsync(H->at<void>(R_CTL), 0, sizeof(FpCtl), s));

    PIDE_CUDA(cudaMemcpyAsync(H->par, H->at<double>(R_PARAMS), 9 * 8, cudaMemcpyDeviceToHost, s));
    // sin^2 table in the transform precision
    PIDE_CUDA(cudaStreamSynchronize(s));
    {
        std::vector<R> s2(N + 1);
        std::vector<double> s2d(N + 1);
        PIDE_CUDA(cudaMemcpyAsync(s2d.data(), H->at<double>(R_SIN2D), (N + 1) * 8, cudaMemcpyDeviceToHost, s));
        PIDE_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i <= N; ++i) s2[i] = (R)s2d[i];
        PIDE_CUDA(cudaMemcpyAsync(H->at<R>(R_SIN2R), s2.data(), (N + 1) * sizeof(R), cudaMemcpyHostToDevice, s));
        PIDE_CUDA(cudaStreamSynchronize(s));
    }
    for (int i = 0; i < 9; ++i) {
        if (!std::isfinite(H->par[i])) {
            H->err = "precomputed rates are not finite";
            return PIDE2D_ERR_ARG;
        }
    }

    // V^0 (eq. 3.18) and B_w V^0
    H->hist.assign({0});
    H->freel.assign({4, 3, 2, 1});
    H->bv = 5;
    H->by = 6;
    if constexpr (sizeof(R) == 4) {
        // V^0 and B_w V^0 from the FP64 payoff and an FP64 sweep
        const pide2d_status bs = bv0_fp64(H);
        if (bs != PIDE2D_OK) return bs;
        PIDE_CUDA(cudaStreamSynchronize(s));
        return PIDE2D_OK;
    }
    const double* glp = dgl + 2 * (kGlNear + kGlFar + kGlEdge);
    PIDE_CUDA(launch_payoff<R>(g, H->at<double>(R_E1D), H->at<double>(R_E2D), H->s_lo1, H->s_lo2, H->h,
                               H->contract.strike, H->contract.payoff, glp, glp + kGlPay, kGlPay,
                               (St<R>*)H->field(0), s));
    FwdArgs<R> fa{};
    fa.g = g;
    fa.mode = FWD_FULL;
    fa.Y = (const St<R>*)H->field(0);
    fa.E1 = (const R*)(sizeof(R) == 4 ? (const void*)H->at<float>(R_E1F) : (const void*)H->at<double>(R_E1D));
    fa.E2 = (const R*)(sizeof(R) == 4 ? (const void*)H->at<float>(R_E2F) : (const void*)H->at<double>(R_E2D));
    fa.Kd = (R)H->contract.strike;
    fa.payoff = H->contract.payoff;
    fa.S = H->at<void>(R_S);
    fa.pair0 = 0;
    fa.npairs = N + 1;
    fa.tw = H->at<void>(R_TWR);
    PIDE_CUDA(launch_row_forward<R>(fa, s));
    ColArgs<R> ca{};
    ca.g = g;
    ca.mode = COL_FULL;
    ca.S = H->at<void>(R_S);
    ca.Wh = H->at<void>(R_WH);
    ca.rlo = 0;
    ca.rhi = g.P + 2;
    ca.tw = H->at<void>(R_TWR);
    PIDE_CUDA(launch_col<R>(ca, s));
    InvArgs<R> ia{};
    ia.g = g;
    ia.mode = INV_FULL;
    ia.do_resid = 0;
    ia.S = H->at<void>(R_S);
    ia.BY = (St<R>*)H->field(H->bv);
    ia.tw = H->at<void>(R_TWR);
    PIDE_CUDA(launch_row_inverse<R>(ia, s));
    PIDE_CUDA(cudaStreamSynchronize(s));
    return PIDE2D_OK;
}

template <typename R>
static pide2d_status do_apply_jump(pide2d* H, const double* U, double tau, int far, double* out) {
    const Geometry g = H->L.g;
    const int N = g.N;
    cudaStream_t s = H->stream;
    double* OUT = H->at<double>(R_OUT);
    St<R>* X = H->at<St<R>>(R_X);
    PIDE_CUDA(cudaMemcpy2DAsync(OUT, (size_t)g.ldS * 8, U, (size_t)(N + 1) * 8, (size_t)(N + 1) * 8, N + 1,
                                cudaMemcpyDefault, s));
    PIDE_CUDA(launch_state_from_double<R>(g, OUT, g.ldS, X, s));
    const double Kd = H->contract.strike * std::exp(-H->model.r * tau);
    FwdArgs<R> fa{};
    fa.g = g;
    fa.mode = far ? FWD_FULL : FWD_FULL0;
    fa.Y = X;
    fa.E1 = (const R*)(sizeof(R) == 4 ? (const void*)H->at<float>(R_E1F) : (const void*)H->at<double>(R_E1D));
    fa.E2 = (const R*)(sizeof(R) == 4 ? (const void*)H->at<float>(R_E2F) : (const void*)H->at<double>(R_E2D));
    fa.Kd = (R)Kd;
    fa.payoff = H->contract.payoff;
    fa.S = H->at<void>(R_S);
    fa.pair0 = 0;
    fa.npairs = N + 1;
    fa.tw = H->at<void>(R_TWR);
    PIDE_CUDA(launch_row_forward<R>(fa, s));
    ColArgs<R> ca{};
    ca.g = g;
    ca.mode = COL_FULL;
    ca.S = H->at<void>(R_S);
    ca.Wh = H->at<void>(R_WH);
    ca.rlo = 0;
    ca.rhi = g.P + 2;
    ca.tw = H->at<void>(R_TWR);
    PIDE_CUDA(launch_col<R>(ca, s));
    InvArgs<R> ia{};
    ia.g = g;
    ia.mode = INV_OUT;
    ia.do_resid = 0;
    ia.S = H->at<void>(R_S);
    ia.out = OUT;
    ia.tw = H->at<void>(R_TWR);
    PIDE_CUDA(launch_row_inverse<R>(ia, s));
    // interior block only
    PIDE_CUDA(cudaMemcpy2DAsync(out + (N + 1) + 1, (size_t)(N + 1) * 8, OUT + g.ldS + 1, (size_t)g.ldS * 8,
                                (size_t)(N - 1) * 8, N - 1, cudaMemcpyDefault, s));
    PIDE_CUDA(cudaStreamSynchronize(s));
    return PIDE2D_OK;
}

// One iteration of the increment loop on a caller residual (pide2d_iteration_probe):
// the DST solve of the non-mixed operator, the increment's B_w sweep and the
// eq. 3.25 quantity, through the kernels and launch shapes of the time loop.
// Scratch: R_OUT (the residual in FP64), R_X (Y, from zero), R_W (B_w Y, from
// zero); W is rebuilt at the start of every theta step, so a probe between
// steps does not disturb the time loop.
template <typename R>
static pide2d_status do_iteration_probe(pide2d* H, const double* r, double ht, double theta, double* delta_out,
                                        double* bdelta_out, double* stop_out) {
    const Geometry g = H->L.g;
    const int N = g.N;
    cudaStream_t s = H->stream;
    double* OUT = H->at<double>(R_OUT);
    St<R>* Y = H->at<St<R>>(R_X);
    St<R>* BY = H->at<St<R>>(R_W);
    PIDE_CUDA(cudaMemcpy2DAsync(OUT, (size_t)g.ldS * 8, r, (size_t)(N + 1) * 8, (size_t)(N + 1) * 8, N + 1,
                                cudaMemcpyDefault, s));
    PIDE_CUDA(launch_row_dst<R>(g, OUT, H->at<R>(R_E), H->at<void>(R_TWR), s));
    PIDE_CUDA(cudaMemsetAsync(Y, 0, H->L.size[R_X], s));
    PIDE_CUDA(cudaMemsetAsync(BY, 0, H->L.size[R_W], s));
    SolveSpec<R> sp{};
    sp.Y = Y;
    sp.BY = BY;
    sp.W = BY;
    sp.far = 0;
    sp.Kd = 0.0;
    sp.Wh = H->at<void>(R_WH);
    sp.Whi = H->at<void>(R_WHI);
    sp.theta = theta;
    sp.ht = ht;
    sp.step_end = 0;
    sp.device_loop = false;
    SolveArgs<R> A;
    build_solve_args<R>(H, sp, &A);
    PIDE_CUDA(launch_col_solve<R>(A.da, s));
    PIDE_CUDA(cudaMemsetAsync(H->at<void>(R_RESID), 0, 16, s));
    PIDE_CUDA(launch_dst_row<R>(A.ra, s));
    PIDE_CUDA(launch_col<R>(A.cai, s));
    A.iai.do_resid = 1;
    PIDE_CUDA(launch_row_inverse<R>(A.iai, s));
    // Y = 0 + delta exactly, B_w Y = 0 + B_w delta exactly
    const size_t ldo = (size_t)(N + 1) * 8;
    if (delta_out) {
        PIDE_CUDA(launch_state_to_double<R>(g, Y, OUT, g.ldS, s));
        PIDE_CUDA(cudaMemcpy2DAsync(delta_out + (N + 1) + 1, ldo, OUT + g.ldS + 1, (size_t)g.ldS * 8,
                                    (size_t)(N - 1) * 8, N - 1, cudaMemcpyDefault, s));
    }
    if (bdelta_out) {
        PIDE_CUDA(launch_state_to_double<R>(g, BY, OUT, g.ldS, s));
        PIDE_CUDA(cudaMemcpy2DAsync(bdelta_out + (N + 1) + 1, ldo, OUT + g.ldS + 1, (size_t)g.ldS * 8,
                                    (size_t)(N - 1) * 8, N - 1, cudaMemcpyDefault, s));
    }
    double stop = 0.0;
    PIDE_CUDA(cudaMemcpyAsync(&stop, H->at<void>(R_RESID), 8, cudaMemcpyDeviceToHost, s));
    PIDE_CUDA(cudaStreamSynchronize(s));
    if (stop_out) *stop_out = stop;
    return PIDE2D_OK;
}

template <typename R>
static pide2d_status do_get_values(pide2d* H, double* dst) {
    const Geometry g = H->L.g;
    const int N = g.N;
    double* OUT = H->at<double>(R_OUT);
    PIDE_CUDA(launch_state_to_double<R>(g, (const St<R>*)H->field(H->hist[0]), OUT, g.ldS, H->stream));
    PIDE_CUDA(cudaMemcpy2DAsync(dst, (size_t)(N + 1) * 8, OUT, (size_t)g.ldS * 8, (size_t)(N + 1) * 8, N + 1,
                                cudaMemcpyDefault, H->stream));
    PIDE_CUDA(cudaStreamSynchronize(H->stream));
    return PIDE2D_OK;
}

template <typename R>
static pide2d_status do_greeks(pide2d* H, double* const* outs) {
    const Geometry g = H->L.g;
    const int N = g.N;
    double* OUT = H->at<double>(R_OUT);
    for (int k = 0; k < 5; ++k) {
        if (!outs[k]) continue;
        PIDE_CUDA(launch_greeks<R>(g, (const St<R>*)H->field(H->hist[0]), H->at<double>(R_E1D),
                                   H->at<double>(R_E2D), H->h, k, OUT, g.ldS, H->stream));
        PIDE_CUDA(cudaMemcpy2DAsync(outs[k] + (N + 1) + 1, (size_t)(N + 1) * 8, OUT + g.ldS + 1, (size_t)g.ldS * 8,
                                    (size_t)(N - 1) * 8, N - 1, cudaMemcpyDefault, H->stream));
        PIDE_CUDA(cudaStreamSynchronize(H->stream));
    }
    return PIDE2D_OK;
}

template <typename R>
static pide2d_status do_price(pide2d* H, double* price) {
    const Geometry g = H->L.g;
    const int N = g.N;
    St<R> v;
    const St<R>* V = (const St<R>*)H->field(H->hist[0]);
    PIDE_CUDA(cudaMemcpyAsync(&v, V + (size_t)(N / 2) * g.ldS + N / 2, sizeof(v), cudaMemcpyDeviceToHost, H->stream));
    PIDE_CUDA(cudaStreamSynchronize(H->stream));
    if constexpr (sizeof(R) == 4) *price = (double)v.x + (double)v.y;
    else *price = v;
    return PIDE2D_OK;
}

template <typename R> St<R> st_host_one();
template <> float2 st_host_one<float>() { return make_float2(1.f, 0.f); }
template <> double st_host_one<double>() { return 1.0; }

// ---------------------------------------------------------------------------
// multi-job time loop: K handles of one geometry advanced in lockstep, every
// kernel launched once for all of them (grid dimension y / z = job)
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kArgAlign = 256;
size_t arr_bytes(size_t each, int K) { return align256(each * (size_t)K); }

template <typename R>
struct GroupLayout {
    size_t pa, fa, caf, iaf, da, ra, cai, iai, chk, conv, kconv, kcount, nonconv, last, active, iter, it_total,
        it_step, it_max, step, step_end, blobs, blob_bytes, total;
    GroupLayout(int K, int T) {
        size_t o = 0;
        pa = o;      o += arr_bytes(sizeof(PrepArgs<R>), K);
        fa = o;      o += arr_bytes(sizeof(FwdArgs<R>), K);
        caf = o;     o += arr_bytes(sizeof(ColArgs<R>), K);
        iaf = o;     o += arr_bytes(sizeof(InvArgs<R>), K);
        da = o;      o += arr_bytes(sizeof(ColSolveArgs<R>), K);
        ra = o;      o += arr_bytes(sizeof(DstRowArgs<R>), K);
        cai = o;     o += arr_bytes(sizeof(ColArgs<R>), K);
        iai = o;     o += arr_bytes(sizeof(InvArgs<R>), K);
        blob_bytes = o;                  // the argument arrays of one theta step (a multiple of 256)
        chk = o;     o += arr_bytes(sizeof(JobCheck), K);
        conv = o;    o += arr_bytes(4, K);
        kconv = o;   o += arr_bytes(4, K);
        kcount = o;  o += arr_bytes(4, K);
        nonconv = o; o += arr_bytes(4, K);
        last = o;    o += arr_bytes(8, K);
        active = o;  o += kArgAlign;
        iter = o;    o += kArgAlign;
        it_total = o; o += arr_bytes(4, K);
        it_step = o; o += arr_bytes(4, K);
        it_max = o;  o += arr_bytes(4, K);
        step = o;    o += kArgAlign;
        step_end = o; o += arr_bytes(4, T);
        blobs = o;   o += blob_bytes * (size_t)T;
        total = o;
    }
};

// the theta steps of a time loop of n_steps steps (the damped first step has four)
int theta_steps(int n_steps, bool damping) { return n_steps + (damping ? 3 : 0); }
}  // namespace

namespace pide {
size_t group_scratch_bytes(int K, int n_steps) {
    const int T = theta_steps(n_steps, true);
    return std::max(GroupLayout<float>(K, T).total, GroupLayout<double>(K, T).total);
}

}  // namespace pide

// The multi-job time loop of a chunk of K fresh handles of one geometry:
//  1. on the host, the argument arrays of every theta step of every job, by
//     the bookkeeping do_step performs (the field rotation does not depend on
//     device results), uploaded as one blob per theta step;
//  2. one CUDA graph for the whole loop: an outer while-node over the theta
//     steps -- k_step_select copies the step's blob into the argument arrays,
//     then W and Y^{n,0} (prep), the difference sweep, the reset of the
//     per-job stopping state, an inner while-node over the fixed-point
//     iterations (column solve, row DST with the eq. 3.25 maxima, the per-job
//     check that ends the inner loop when no job iterates any more, column
//     pass and inverse row pass of the jobs still iterating) and
//     k_step_tally, which folds the counts into per-job statistics and ends
//     the outer loop after the last theta step;
//  3. one launch, one synchronisation, the statistics back to the handles.
template <typename R>
static pide2d_status group_solve(pide2d* const* hs, int K, char* scratch, int upb, std::string* err) {
    pide2d* H0 = hs[0];
    cudaStream_t s = H0->stream;
    auto fail = [&](pide2d* H, pide2d_status st) {
        *err = H->err;
        return st;
    };
    for (int j = 0; j < K; ++j)
        if (hs[j]->steps_done != 0) {
            hs[j]->err = "multi-job loop: handle already stepped";
            return fail(hs[j], PIDE2D_ERR_STATE);
        }
    const bool damped0 = H0->damping != 0;
    const int T = theta_steps(H0->n_steps, damped0);
    const GroupLayout<R> L(K, T);
    std::vector<JobCheck> chk(K);
    int kmax_all = 0;
    for (int j = 0; j < K; ++j) {
        chk[j].resid = hs[j]->at<void>(R_RESID);
        chk[j].tol = hs[j]->tol;
        chk[j].kmax = hs[j]->kmax;
        chk[j].pad = 0;
        kmax_all = std::max(kmax_all, hs[j]->kmax);
    }

    // 1. every theta step's argument arrays
    std::vector<char> blobs(L.blob_bytes * (size_t)T, 0);
    std::vector<int> step_end(T, 0);
    PrepArgs<R> pa0{};
    SolveArgs<R> A0{};
    std::vector<int> cur(K), v0(K);
    int t = 0;
    while (H0->steps_done < H0->n_steps) {
        const bool damped = H0->steps_done == 0 && H0->damping;
        const int nsub = damped ? 4 : 1;
        for (int j = 0; j < K; ++j) cur[j] = v0[j] = hs[j]->hist[0];
        for (int sub = 0; sub < nsub; ++sub, ++t) {
            if (t >= T) {
                H0->err = "multi-job loop: theta step count";
                return fail(H0, PIDE2D_ERR_STATE);
            }
            char* blob = blobs.data() + L.blob_bytes * (size_t)t;
            step_end[t] = (!damped || sub == 3) ? 1 : 0;
            for (int j = 0; j < K; ++j) {
                pide2d* H = hs[j];
                if (H->damping != H0->damping || H->n_steps != H0->n_steps) {
                    H->err = "multi-job loop: jobs differ in damping or step count";
                    return fail(H, PIDE2D_ERR_ARG);
                }
                int list[4];
                int cnt;
                double theta, ht, tau_prev, tau;
                const int res = H->freel.back();
                H->freel.pop_back();
                if (damped) {
                    const double q = H->dt / 4.0;
                    list[0] = cur[j];
                    cnt = 1;
                    theta = 1.0;
                    ht = q;
                    tau_prev = sub * q;
                    tau = (sub + 1) * q;
                } else {
                    const int n = H->steps_done + 1;
                    cnt = (int)H->hist.size() < 4 ? (int)H->hist.size() : 4;
                    for (int i = 0; i < cnt; ++i) list[i] = H->hist[i];
                    theta = H->theta;
                    ht = H->dt;
                    tau_prev = (n - 1) * H->dt;
                    tau = n * H->dt;
                }
                PrepArgs<R> pa;
                SolveSpec<R> sp;
                const pide2d_status bs =
                    build_theta_step<R>(H, list, cnt, theta, ht, tau_prev, tau, res, step_end[t], &pa, &sp);
                if (bs != PIDE2D_OK) return fail(H, bs);
                SolveArgs<R> A;
                build_solve_args<R>(H, sp, &A);
                A.iai.conv_flag = nullptr;
                std::memcpy(blob + L.pa + j * sizeof pa, &pa, sizeof pa);
                std::memcpy(blob + L.fa + j * sizeof A.fa, &A.fa, sizeof A.fa);
                std::memcpy(blob + L.caf + j * sizeof A.caf, &A.caf, sizeof A.caf);
                std::memcpy(blob + L.iaf + j * sizeof A.iaf, &A.iaf, sizeof A.iaf);
                std::memcpy(blob + L.da + j * sizeof A.da, &A.da, sizeof A.da);
                std::memcpy(blob + L.ra + j * sizeof A.ra, &A.ra, sizeof A.ra);
                std::memcpy(blob + L.cai + j * sizeof A.cai, &A.cai, sizeof A.cai);
                std::memcpy(blob + L.iai + j * sizeof A.iai, &A.iai, sizeof A.iai);
                if (t == 0 && j == 0) {
                    pa0 = pa;
                    A0 = A;
                }
                // bookkeeping of theta_step / do_step
                std::swap(H->bv, H->by);
                if (damped) {
                    if (cur[j] != v0[j]) H->freel.push_back(cur[j]);
                    cur[j] = res;
                } else {
                    H->hist.insert(H->hist.begin(), res);
                    if (H->hist.size() > 4) {
                        H->freel.push_back(H->hist.back());
                        H->hist.pop_back();
                    }
                }
            }
        }
        for (int j = 0; j < K; ++j) {
            pide2d* Hj = hs[j];
            if (damped) Hj->hist.assign({cur[j], v0[j]});
            Hj->steps_done++;
            Hj->stats.steps_done = Hj->steps_done;
            Hj->last_step_device = false;
        }
    }
    const int Tused = t;
    // the row pass of the full sweep covers every job's row range at every step
    A0.fa.npairs = H0->L.g.N + 1;

    JobsState st{};
    st.conv = reinterpret_cast<int*>(scratch + L.conv);
    st.kconv = reinterpret_cast<int*>(scratch + L.kconv);
    st.kcount = reinterpret_cast<int*>(scratch + L.kcount);
    st.nonconv = reinterpret_cast<int*>(scratch + L.nonconv);
    st.last = reinterpret_cast<double*>(scratch + L.last);
    st.active = reinterpret_cast<int*>(scratch + L.active);
    st.iter = reinterpret_cast<int*>(scratch + L.iter);
    st.it_total = reinterpret_cast<int*>(scratch + L.it_total);
    st.it_step = reinterpret_cast<int*>(scratch + L.it_step);
    st.it_max = reinterpret_cast<int*>(scratch + L.it_max);
    st.step = reinterpret_cast<int*>(scratch + L.step);
    const JobCheck* dchk = reinterpret_cast<const JobCheck*>(scratch + L.chk);
    {
        pide2d* H = H0;
        PIDE_CUDA(cudaMemcpyAsync(scratch + L.chk, chk.data(), sizeof(JobCheck) * K, cudaMemcpyHostToDevice, s));
        PIDE_CUDA(cudaMemcpyAsync(scratch + L.step_end, step_end.data(), 4 * (size_t)Tused, cudaMemcpyHostToDevice, s));
        PIDE_CUDA(cudaMemcpyAsync(scratch + L.blobs, blobs.data(), L.blob_bytes * (size_t)Tused,
                                  cudaMemcpyHostToDevice, s));
        // per-job stopping state and statistics, the iteration and step counters
        PIDE_CUDA(cudaMemsetAsync(scratch + L.conv, 0, L.step_end - L.conv, s));
    }

    // 2. the graph of the whole loop
    pide2d* H = H0;
    if (!H->cap) PIDE_CUDA(cudaStreamCreateWithFlags(&H->cap, cudaStreamNonBlocking));
    cudaStream_t cs = H->cap;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    PIDE_CUDA(cudaGraphCreate(&g, 0));
    const char* where = "";
    cudaError_t e = cudaSuccess;
#define PIDE_GTRY(call)          \
    do {                         \
        e = (call);              \
        if (e != cudaSuccess) {  \
            where = #call;       \
            goto graph_done;     \
        }                        \
    } while (0)
    {
        auto arr = [&](size_t off) { return scratch + off; };
        cudaGraphConditionalHandle hout, hin;
        PIDE_GTRY(cudaGraphConditionalHandleCreate(&hout, g, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cpo{};
        cpo.type = cudaGraphNodeTypeConditional;
        cpo.conditional.handle = hout;
        cpo.conditional.type = cudaGraphCondTypeWhile;
        cpo.conditional.size = 1;
        cudaGraphNode_t outer = nullptr;
        PIDE_GTRY(cudaGraphAddNode(&outer, g, nullptr, nullptr, 0, &cpo));
        cudaGraph_t body_o = cpo.conditional.phGraph_out[0];
        PIDE_GTRY(cudaGraphConditionalHandleCreate(&hin, body_o, 1, cudaGraphCondAssignDefault));
        // the theta step's prologue
        PIDE_GTRY(cudaStreamBeginCaptureToGraph(cs, body_o, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        {
            cudaError_t x = launch_step_select(arr(L.blobs), L.blob_bytes, st, scratch, cs);
            const JobsCtl all{st.conv, st.kconv, st.iter, 0};
            if (x == cudaSuccess) x = launch_prep_jobs<R>(pa0, (const PrepArgs<R>*)arr(L.pa), K, true, cs);
            if (x == cudaSuccess) x = launch_row_forward_jobs<R>(A0.fa, (const FwdArgs<R>*)arr(L.fa), K, all, upb, cs);
            if (x == cudaSuccess) x = launch_col_jobs<R>(A0.caf, (const ColArgs<R>*)arr(L.caf), K, all, upb, cs);
            if (x == cudaSuccess) x = launch_row_inverse_jobs<R>(A0.iaf, (const InvArgs<R>*)arr(L.iaf), K, all, upb, cs);
            if (x == cudaSuccess) x = launch_jobs_reset<R>(K, dchk, st, (unsigned long long)hin, cs);
            cudaGraph_t got = nullptr;
            const cudaError_t x2 = cudaStreamEndCapture(cs, &got);
            if (x != cudaSuccess) { e = x; where = "theta-step prologue launches"; goto graph_done; }
            if (x2 != cudaSuccess) { e = x2; where = "cudaStreamEndCapture(prologue)"; goto graph_done; }
        }
        {
            // the prologue is a chain: its last node has no dependents
            size_t nn = 0;
            PIDE_GTRY(cudaGraphGetNodes(body_o, nullptr, &nn));
            std::vector<cudaGraphNode_t> nodes(nn);
            PIDE_GTRY(cudaGraphGetNodes(body_o, nodes.data(), &nn));
            std::vector<cudaGraphNode_t> leaves;
            for (auto nd : nodes) {
                size_t nd_out = 0;
                PIDE_GTRY(cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &nd_out));
                if (nd_out == 0) leaves.push_back(nd);
            }
            cudaGraphNodeParams cpi{};
            cpi.type = cudaGraphNodeTypeConditional;
            cpi.conditional.handle = hin;
            cpi.conditional.type = cudaGraphCondTypeWhile;
            cpi.conditional.size = 1;
            cudaGraphNode_t inner = nullptr;
            PIDE_GTRY(cudaGraphAddNode(&inner, body_o, leaves.data(), nullptr, leaves.size(), &cpi));
            cudaGraph_t body_i = cpi.conditional.phGraph_out[0];
            // one fixed-point iteration of every job still iterating
            PIDE_GTRY(cudaStreamBeginCaptureToGraph(cs, body_i, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
            {
                const JobsCtl head{st.conv, st.kconv, st.iter, 1};
                const JobsCtl tail{st.conv, st.kconv, st.iter, 2};
                cudaError_t x = launch_col_solve_jobs<R>(A0.da, (const ColSolveArgs<R>*)arr(L.da), K, head, upb, cs);
                if (x == cudaSuccess) x = launch_dst_row_jobs<R>(A0.ra, (const DstRowArgs<R>*)arr(L.ra), K, head, upb, cs);
                if (x == cudaSuccess) x = launch_jobs_check(K, dchk, st, kmax_all, (unsigned long long)hin, cs);
                if (x == cudaSuccess) x = launch_col_jobs<R>(A0.cai, (const ColArgs<R>*)arr(L.cai), K, tail, upb, cs);
                if (x == cudaSuccess) x = launch_row_inverse_jobs<R>(A0.iai, (const InvArgs<R>*)arr(L.iai), K, tail, upb, cs);
                cudaGraph_t got = nullptr;
                const cudaError_t x2 = cudaStreamEndCapture(cs, &got);
                if (x != cudaSuccess) { e = x; where = "iteration launches"; goto graph_done; }
                if (x2 != cudaSuccess) { e = x2; where = "cudaStreamEndCapture(iteration)"; goto graph_done; }
            }
            // after the iterations: statistics and the next theta step
            PIDE_GTRY(cudaStreamBeginCaptureToGraph(cs, body_o, &inner, nullptr, 1, cudaStreamCaptureModeRelaxed));
            {
                const cudaError_t x = launch_step_tally(K, st, (const int*)arr(L.step_end), Tused,
                                                        (unsigned long long)hout, cs);
                cudaGraph_t got = nullptr;
                const cudaError_t x2 = cudaStreamEndCapture(cs, &got);
                if (x != cudaSuccess) { e = x; where = "launch_step_tally"; goto graph_done; }
                if (x2 != cudaSuccess) { e = x2; where = "cudaStreamEndCapture(tally)"; goto graph_done; }
            }
        }
        PIDE_GTRY(cudaGraphInstantiate(&ex, g, 0));
        PIDE_GTRY(cudaGraphLaunch(ex, s));
    }
graph_done:
#undef PIDE_GTRY
    if (e != cudaSuccess) {
        if (ex) cudaGraphExecDestroy(ex);
        cudaGraphDestroy(g);
        H->err = std::string("multi-job loop graph: ") + where + ": " + cudaGetErrorString(e);
        H->broken = true;
        return fail(H, PIDE2D_ERR_CUDA);
    }
    // 3. one synchronisation; the statistics back to the handles
    std::vector<int> tot(K), mx(K), nc(K);
    std::vector<double> lastv(K);
    {
        const cudaError_t es = cudaStreamSynchronize(s);
        cudaGraphExecDestroy(ex);
        cudaGraphDestroy(g);
        PIDE_CUDA(es);
        PIDE_CUDA(cudaMemcpyAsync(tot.data(), st.it_total, 4 * (size_t)K, cudaMemcpyDeviceToHost, s));
        PIDE_CUDA(cudaMemcpyAsync(mx.data(), st.it_max, 4 * (size_t)K, cudaMemcpyDeviceToHost, s));
        PIDE_CUDA(cudaMemcpyAsync(nc.data(), st.nonconv, 4 * (size_t)K, cudaMemcpyDeviceToHost, s));
        PIDE_CUDA(cudaMemcpyAsync(lastv.data(), st.last, 8 * (size_t)K, cudaMemcpyDeviceToHost, s));
        PIDE_CUDA(cudaStreamSynchronize(s));
    }
    for (int j = 0; j < K; ++j) {
        pide2d* Hj = hs[j];
        const int N = Hj->L.g.N;
        Hj->stats.fp_iters_total += tot[j];
        Hj->stats.fp_iters_max = std::max(Hj->stats.fp_iters_max, mx[j]);
        Hj->stats.cell_iters += (double)N * N * (double)(tot[j] + Tused);
        Hj->stats.last_resid = lastv[j];
        if (nc[j]) {
            Hj->err = "fixed-point iteration not converged in a theta step (multi-job loop)";
            Hj->group_nonconv = true;
        }
    }
    return PIDE2D_OK;
}

namespace pide {
void set_handle_stream(pide2d_t* h, void* stream) { h->stream = static_cast<cudaStream_t>(stream); }

pide2d_status solve_group(pide2d_t* const* hs, int K, void* scratch, int upb, std::string* err) {
    return hs[0]->grid.precision == PIDE2D_FP64 ? group_solve<double>(hs, K, (char*)scratch, upb, err)
                                                : group_solve<float>(hs, K, (char*)scratch, upb, err);
}

// Timed trial of the multi-job launch shape: the increment column pass
// (forward FFT, product with the weight spectrum, inverse FFT) of K fresh
// handles of one geometry, `reps` times with upb FFT units per block.  The
// pass works in place on each handle's spectrum buffer, which the time loop
// rewrites before reading, so the trial leaves the solution untouched.
template <typename R>
static pide2d_status time_col(pide2d* const* hs, int K, char* scratch, int upb, int reps, double* ms) {
    pide2d* H = hs[0];
    cudaStream_t s = H->stream;
    std::vector<ColArgs<R>> arr(K);
    for (int j = 0; j < K; ++j) {
        pide2d* Hj = hs[j];
        SolveSpec<R> sp{};
        sp.Y = (St<R>*)Hj->field(0);
        sp.BY = (St<R>*)Hj->field(Hj->by);
        sp.W = Hj->at<St<R>>(R_W);
        sp.far = 1;
        sp.Kd = Hj->contract.strike;
        sp.Wh = Hj->at<void>(R_WH);
        sp.Whi = Hj->at<void>(R_WHI);
        sp.theta = Hj->theta;
        sp.ht = Hj->dt;
        SolveArgs<R> A;
        build_solve_args<R>(Hj, sp, &A);
        arr[j] = A.cai;
    }
    PIDE_CUDA(cudaMemcpyAsync(scratch, arr.data(), sizeof(ColArgs<R>) * K, cudaMemcpyHostToDevice, s));
    const JobsCtl all{nullptr, nullptr, nullptr, 0};
    cudaEvent_t e0, e1;
    PIDE_CUDA(cudaEventCreate(&e0));
    PIDE_CUDA(cudaEventCreate(&e1));
    pide2d_status st = PIDE2D_OK;
    cudaError_t e = launch_col_jobs<R>(arr[0], (const ColArgs<R>*)scratch, K, all, upb, s);   // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_col_jobs<R>(arr[0], (const ColArgs<R>*)scratch, K, all, upb, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e != cudaSuccess) {
        H->err = std::string("launch-shape trial: ") + cudaGetErrorString(e);
        H->broken = true;
        st = PIDE2D_ERR_CUDA;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = (double)t / reps;
    return st;
}

pide2d_status time_col_jobs(pide2d_t* const* hs, int K, void* scratch, int upb, int reps, double* ms, std::string* err) {
    const pide2d_status st = hs[0]->grid.precision == PIDE2D_FP64 ? time_col<double>(hs, K, (char*)scratch, upb, reps, ms)
                                                                  : time_col<float>(hs, K, (char*)scratch, upb, reps, ms);
    if (st != PIDE2D_OK) *err = hs[0]->err;
    return st;
}
}  // namespace pide

// ---------------------------------------------------------------------------
// discrete adjoint of the time loop (see adjoint.cu for the recursion)
// ---------------------------------------------------------------------------
// B_w with the weight spectrum Wh applied to a full node field V (far field
// g(s, tau) with discounted strike Kd in the halo when far = 1, zero when
// far = 0), interior result written to the FP64 field `out` (pitch ldS)
template <typename R>
static pide2d_status jump_apply(pide2d* H, const St<R>* V, int far, double Kd, const void* Wh, double* out) {
    const Geometry g = H->L.g;
    const int N = g.N;
    FwdArgs<R> fa{};
    fa.g = g;
    fa.mode = far ? FWD_FULL : FWD_FULL0;
    fa.Y = V;
    fa.E1 = (const R*)(sizeof(R) == 4 ? (const void*)H->at<float>(R_E1F) : (const void*)H->at<double>(R_E1D));
    fa.E2 = (const R*)(sizeof(R) == 4 ? (const void*)H->at<float>(R_E2F) : (const void*)H->at<double>(R_E2D));
    fa.Kd = (R)Kd;
    fa.payoff = H->contract.payoff;
    fa.S = H->at<void>(R_S);
    fa.pair0 = 0;
    fa.npairs = N + 1;
    fa.tw = H->at<void>(R_TWR);
    PIDE_CUDA(launch_row_forward<R>(fa, H->stream));
    ColArgs<R> ca{};
    ca.g = g;
    ca.mode = COL_FULL;
    ca.S = H->at<void>(R_S);
    ca.Wh = Wh;
    ca.rlo = 0;
    ca.rhi = g.P + 2;
    ca.tw = H->at<void>(R_TWR);
    PIDE_CUDA(launch_col<R>(ca, H->stream));
    InvArgs<R> ia{};
    ia.g = g;
    ia.mode = INV_OUT;
    ia.do_resid = 0;
    ia.S = H->at<void>(R_S);
    ia.out = out;
    ia.tw = H->at<void>(R_TWR);
    PIDE_CUDA(launch_row_inverse<R>(ia, H->stream));
    return PIDE2D_OK;
}

namespace {
struct SavedState {
    std::vector<int> hist, freel;
    int bv, by, steps_done;
    pide2d_stats stats;
    bool last_step_device;
};
}  // namespace

// the contributions of one stored state V^j (far field at tau_j) with the
// coefficient field xi: <xi, V>, <xi, D-parts V>, and for the weights the
// spectral product conj(xi^) V~^ added to the FP64 accumulator: summed over
// the states and inverted once, it gives C(l) = sum_j sum_m xi_j(m) V~_j(m+l+1/2),
// and <xi_j, B_{dw} V_j> summed over j = sum_l dw(l) C(l) for every direction
template <typename R>
static pide2d_status state_dots(pide2d* H, const TapeLayout& t, const St<R>* V, double tau, int ndirs) {
    const Geometry g = H->L.g;
    const int N = g.N;
    char* scr = H->tape.base + t.scr;
    double* part = reinterpret_cast<double*>(scr + 3 * t.omega + t.part + kMomentBytes + 2 * 256 + t.rows);
    double* acc = reinterpret_cast<double*>(H->tape.base + t.acc);
    const double* xi = reinterpret_cast<const double*>(H->tape.base + t.adj + A_XI * t.field);
    PIDE_CUDA(launch_dots_state<R>(g, xi, V, part, acc, 1.0, H->stream));
    if (ndirs == 0) return PIDE2D_OK;
    const void* tw = H->at<void>(R_TWR);
    // V~ (midpoints, far field at tau) into the handle's spectrum buffer
    FwdArgs<R> fa{};
    fa.g = g;
    fa.mode = FWD_FULL;
    fa.Y = V;
    fa.E1 = (const R*)(sizeof(R) == 4 ? (const void*)H->at<float>(R_E1F) : (const void*)H->at<double>(R_E1D));
    fa.E2 = (const R*)(sizeof(R) == 4 ? (const void*)H->at<float>(R_E2F) : (const void*)H->at<double>(R_E2D));
    fa.Kd = (R)(H->contract.strike * std::exp(-H->model.r * tau));
    fa.payoff = H->contract.payoff;
    fa.S = H->at<void>(R_S);
    fa.pair0 = 0;
    fa.npairs = N + 1;
    fa.tw = tw;
    PIDE_LAUNCH(PIDE2D_KERNEL_ROW_FORWARD_FULL, launch_row_forward<R>(fa, H->stream));
    // xi (raw, at the increment positions) into the adjoint's spectrum rows
    R* xr = H->at<R>(R_DLT);
    PIDE_CUDA(launch_field_to_r<R>(g, xi, xr, H->stream));
    FwdArgs<R> fx{};
    fx.g = g;
    fx.mode = FWD_INCR;
    fx.D = xr;
    fx.S = H->tape.base + t.specx;
    fx.pair0 = N / 4 + 1;
    fx.npairs = N / 2;
    fx.tw = tw;
    PIDE_LAUNCH(PIDE2D_KERNEL_ROW_FORWARD_INCR, launch_row_forward<R>(fx, H->stream));
    PIDE_LAUNCH(PIDE2D_KERNEL_COL_FULL,
                launch_corr_col<R>(g, H->at<void>(R_S), H->tape.base + t.specx, N / 2 + 2, N / 2 + N + 2,
                                   reinterpret_cast<double*>(H->tape.base + t.cacc), tw, H->stream));
    return PIDE2D_OK;
}

template <typename R>
static pide2d_status do_adjoint(pide2d* H, const pide2d_model* dirs, int ndirs, double* grad) {
    const Geometry g = H->L.g;
    const int N = g.N;
    cudaStream_t s = H->stream;
    const TapeLayout t = tape_layout(H->L, H->n_steps, H->tape.interval, H->tape.ndirs);
    const size_t fb = H->L.size[R_V0];
    char* tb = H->tape.base;
    char* scr = tb + t.scr;
    double* om_p = reinterpret_cast<double*>(scr);
    double* om_m = reinterpret_cast<double*>(scr + t.omega);
    double* om_d = reinterpret_cast<double*>(scr + 2 * t.omega);
    double* part = reinterpret_cast<double*>(scr + 3 * t.omega);
    double* moment = reinterpret_cast<double*>(scr + 3 * t.omega + t.part);
    double* par_p = reinterpret_cast<double*>(scr + 3 * t.omega + t.part + kMomentBytes);
    double* par_m = reinterpret_cast<double*>(scr + 3 * t.omega + t.part + kMomentBytes + 256);
    void* rows = scr + 3 * t.omega + t.part + kMomentBytes + 512;
    double* dpart = reinterpret_cast<double*>(scr + 3 * t.omega + t.part + kMomentBytes + 512 + t.rows);
    double* acc = reinterpret_cast<double*>(tb + t.acc);
    auto afield = [&](int i) { return tb + t.adj + (size_t)i * t.field; };
    St<R>* lam = reinterpret_cast<St<R>*>(afield(A_LAM));
    St<R>* mu = reinterpret_cast<St<R>*>(afield(A_MU));
    St<R>* bmu = reinterpret_cast<St<R>*>(afield(A_BMU));
    St<R>* nu = reinterpret_cast<St<R>*>(afield(A_NU));
    double* xi = reinterpret_cast<double*>(afield(A_XI));
    double* pend = reinterpret_cast<double*>(afield(A_PEND));
    double* out = H->at<double>(R_OUT);
    void* whf = tb + t.spec;
    void* whif = tb + t.spec + t.spec1;

    // the final state is put back at the end
    PIDE_CUDA(cudaStreamSynchronize(s));
    SavedState sv{H->hist, H->freel, H->bv, H->by, H->steps_done, H->stats, H->last_step_device};
    for (size_t i = 0; i < H->hist.size(); ++i)
        PIDE_CUDA(cudaMemcpyAsync(tb + t.fin + i * t.field, H->field(H->hist[i]), fb, cudaMemcpyDeviceToDevice, s));
    PIDE_CUDA(cudaMemcpyAsync(tb + t.fin + 4 * t.field, H->field(H->bv), fb, cudaMemcpyDeviceToDevice, s));

    // derivatives of the weights and rates along each direction: central
    // differences of the FP64 precompute (eqs. 3.3, 3.5, 3.6)
    std::vector<double> dpar((size_t)ndirs * 9);
    for (int k = 0; k < ndirs; ++k) {
        const pide2d_model& d = dirs[k];
        const double fields[7] = {d.delta, d.lambda, d.eta[0], d.eta[1], d.rho[0], d.rho[1], d.rho[2]};
        const double base[7] = {H->model.delta, H->model.lambda, H->model.eta[0], H->model.eta[1],
                                H->model.rho[0], H->model.rho[1], H->model.rho[2]};
        double ratio = 0.0;
        for (int i = 0; i < 7; ++i) ratio = std::fmax(ratio, std::fabs(fields[i]) / std::fmax(std::fabs(base[i]), 1e-3));
        if (!(ratio > 0.0) || !std::isfinite(ratio)) {
            for (int i = 0; i < 9; ++i) dpar[(size_t)k * 9 + i] = 0.0;
            PIDE_CUDA(cudaMemsetAsync(tb + t.dw + (size_t)k * t.omega, 0, (size_t)N * N * 8, s));
            continue;
        }
        const double eps = 1e-5 / ratio;
        pide2d_model mp = H->model, mm = H->model;
        mp.delta += eps * d.delta;           mm.delta -= eps * d.delta;
        mp.lambda += eps * d.lambda;         mm.lambda -= eps * d.lambda;
        for (int i = 0; i < 2; ++i) { mp.eta[i] += eps * d.eta[i]; mm.eta[i] -= eps * d.eta[i]; }
        for (int i = 0; i < 3; ++i) { mp.rho[i] += eps * d.rho[i]; mm.rho[i] -= eps * d.rho[i]; }
        pide2d_status ps = run_precompute(H, mp, om_p, part, moment, par_p);
        if (ps != PIDE2D_OK) return ps;
        ps = run_precompute(H, mm, om_m, part, moment, par_m);
        if (ps != PIDE2D_OK) return ps;
        PIDE_CUDA(launch_central_difference(om_p, om_m, 0.5 / eps, reinterpret_cast<double*>(tb + t.dw + (size_t)k * t.omega),
                                            (size_t)N * N, s));
        double hp[9], hm[9];
        PIDE_CUDA(cudaMemcpyAsync(hp, par_p, 9 * 8, cudaMemcpyDeviceToHost, s));
        PIDE_CUDA(cudaMemcpyAsync(hm, par_m, 9 * 8, cudaMemcpyDeviceToHost, s));
        PIDE_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < 9; ++i) dpar[(size_t)k * 9 + i] = (hp[i] - hm[i]) * (0.5 / eps);
    }
    // the transposed jump operator: the same correlation with the weights
    // flipped in both axes (w'_l = w_{-l-1}, which also carries the midpoint
    // interpolation over to its transpose)
    PIDE_CUDA(launch_flip_weights(H->at<double>(R_OMEGA), om_d, N, s));
    {
        const pide2d_status ws = weight_spectrum<R>(H, om_d, whf, whif, rows);
        if (ws != PIDE2D_OK) return ws;
    }

    // lambda^{S} = e_{S0}; everything else zero
    for (int i = 0; i < A_COUNT; ++i) PIDE_CUDA(cudaMemsetAsync(afield(i), 0, t.field, s));
    PIDE_CUDA(cudaMemsetAsync(acc, 0, (size_t)(kAdjAcc + ndirs) * 8, s));
    PIDE_CUDA(cudaMemsetAsync(tb + t.cacc, 0, (size_t)(N + 1) * (2 * N) * 16, s));
    {
        const St<R> one = st_host_one<R>();
        PIDE_CUDA(cudaMemcpyAsync(lam + (size_t)(N / 2) * g.ldS + N / 2, &one, sizeof one, cudaMemcpyHostToDevice, s));
        PIDE_CUDA(cudaStreamSynchronize(s));
    }
    const double hg = H->h;
    const double rw = H->par[1], a11 = H->par[4], a12 = H->par[5], a22 = H->par[6];
    const double d11 = 0.5 * a11 / (hg * hg), d22 = 0.5 * a22 / (hg * hg), d12 = 0.25 * a12 / (hg * hg);
    pide2d_status worst = PIDE2D_OK;

    H->force_host_loop = true;
    for (int seg = t.nckpt - 1; seg >= 0; --seg) {
        // replay the segment forward, keeping every theta step
        pide2d_status rs = restore_checkpoint(H, seg);
        if (rs != PIDE2D_OK) { H->force_host_loop = false; return rs; }
        H->seg_record = true;
        H->seg_slot = 0;
        H->seg_meta.clear();
        const int n_end = std::min((seg + 1) * H->tape.interval, H->n_steps);
        while (H->steps_done < n_end) {
            int k = 0;
            double r = 0.0;
            rs = do_step<R>(H, &k, &r);
            if (rs == PIDE2D_ERR_CUDA || rs == PIDE2D_ERR_ARG || rs == PIDE2D_ERR_STATE) {
                H->seg_record = false;
                H->force_host_loop = false;
                return rs;
            }
        }
        H->seg_record = false;
        // backwards through the segment's theta steps
        for (int slot = H->seg_slot - 1; slot >= 0; --slot) {
            const pide2d::StepMeta m = H->seg_meta[slot];
            const double htt = m.ht * m.theta, htm = m.ht * (1.0 - m.theta);
            const St<R>* Vs = reinterpret_cast<const St<R>*>(tape_seg(H, t, slot, 0));
            const St<R>* Vp = reinterpret_cast<const St<R>*>(slot > 0 ? tape_seg(H, t, slot - 1, 0)
                                                                        : tape_ckpt(H, t, seg, 0));
            const St<R>* BVp = reinterpret_cast<const St<R>*>(slot > 0 ? tape_seg(H, t, slot - 1, 1)
                                                                         : tape_ckpt(H, t, seg, 4));
            // mu = A^{-T} lambda: the forward solver with the flipped weights and a zero far field
            SolveSpec<R> sp{};
            sp.Y = mu;
            sp.BY = bmu;
            sp.W = lam;
            sp.far = 0;
            sp.Kd = 0.0;
            sp.Wh = whf;
            sp.Whi = whif;
            sp.theta = m.theta;
            sp.ht = m.ht;
            sp.step_end = 1;
            sp.device_loop = false;
            int k = 0;
            double r = 0.0;
            bool conv = false;
            rs = fixed_point_solve<R>(H, sp, &k, &r, &conv);
            if (rs != PIDE2D_OK) { H->force_host_loop = false; return rs; }
            if (!conv) worst = PIDE2D_ERR_NOT_CONVERGED;
            // nu = T_SL^T mu
            const double q[2] = {H->par[7] * m.ht / hg, H->par[8] * m.ht / hg};
            SlWeights w{};
            int o1 = 0, o2 = 0;
            sl_stencil(H->sl_order, q[0], &o1, w.w1, w.dw1);
            sl_stencil(H->sl_order, q[1], &o2, w.w2, w.dw2);
            const int nt = H->sl_order == 1 ? 2 : 4;
            PIDE_CUDA(launch_sl_transpose<R>(g, mu, nu, o1, o2, nt, w, s));
            // <mu, dT_SL/dq_i Z>: the departure shift q = b h_t / h
            SlShiftArgs<R> sa{};
            sa.mu = mu;
            sa.V = Vp;
            sa.BV = BVp;
            sa.htm = htm;
            sa.rw = rw;
            sa.d11 = d11;
            sa.d22 = d22;
            sa.d12 = d12;
            sa.o1 = o1;
            sa.o2 = o2;
            sa.nt = nt;
            sa.w = w;
            sa.E1d = H->at<double>(R_E1D);
            sa.E2d = H->at<double>(R_E2D);
            sa.Kd_prev = H->contract.strike * std::exp(-H->model.r * m.tau_prev);
            sa.payoff = H->contract.payoff;
            PIDE_CUDA(launch_sl_shift_dots<R>(g, sa, dpart, acc + 4, m.ht / hg, s));
            // xi = h_t theta mu + (the h_t (1-theta) nu of the step after); the state V^s
            PIDE_CUDA(launch_adj_xi<R>(g, mu, nu, xi, pend, htt, htm, s));
            rs = state_dots<R>(H, t, Vs, m.tau, ndirs);
            if (rs != PIDE2D_OK) { H->force_host_loop = false; return rs; }
            // lambda^{s-1} = nu + htm ((D - r_w) nu + B^T nu)
            if (htm != 0.0) {
                rs = jump_apply<R>(H, nu, 0, 0.0, whf, out);
                if (rs != PIDE2D_OK) { H->force_host_loop = false; return rs; }
                PIDE_CUDA(launch_adj_combine<R>(g, nu, out, lam, htm, rw, d11, d22, d12, s));
            } else {
                PIDE_CUDA(cudaMemcpyAsync(lam, nu, fb, cudaMemcpyDeviceToDevice, s));
            }
        }
    }
    // V^0 (the payoff, far field at tau = 0) with the remaining h_t (1-theta) nu
    PIDE_CUDA(launch_adj_xi<R>(g, mu, nullptr, xi, pend, 0.0, 0.0, s));
    {
        const pide2d_status rs = state_dots<R>(H, t, reinterpret_cast<const St<R>*>(tape_ckpt(H, t, 0, 0)), 0.0, ndirs);
        if (rs != PIDE2D_OK) { H->force_host_loop = false; return rs; }
    }
    H->force_host_loop = false;
    // the correlation at the lags, and <dw_k, C> for every direction
    if (ndirs > 0) {
        double* C = reinterpret_cast<double*>(tb + t.cfield);
        double* dp = reinterpret_cast<double*>(scr + 3 * t.omega + t.part + kMomentBytes + 2 * 256 + t.rows);
        PIDE_CUDA(launch_corr_finish<double>(g, reinterpret_cast<double*>(tb + t.cacc), C, H->at<void>(R_TWD), s));
        for (int k = 0; k < ndirs; ++k)
            PIDE_CUDA(launch_dot_plain(g, reinterpret_cast<const double*>(tb + t.dw + (size_t)k * t.omega), C,
                                       (size_t)N * N, dp, acc + kAdjAcc + k, s));
    }

    // put the final state back
    for (size_t i = 0; i < sv.hist.size(); ++i)
        PIDE_CUDA(cudaMemcpyAsync(H->field(sv.hist[i]), tb + t.fin + i * t.field, fb, cudaMemcpyDeviceToDevice, s));
    PIDE_CUDA(cudaMemcpyAsync(H->field(sv.bv), tb + t.fin + 4 * t.field, fb, cudaMemcpyDeviceToDevice, s));
    H->hist = sv.hist;
    H->freel = sv.freel;
    H->bv = sv.bv;
    H->by = sv.by;
    H->steps_done = sv.steps_done;
    H->stats = sv.stats;
    H->last_step_device = sv.last_step_device;

    std::vector<double> a(kAdjAcc + ndirs);
    PIDE_CUDA(cudaMemcpyAsync(a.data(), acc, a.size() * 8, cudaMemcpyDeviceToHost, s));
    PIDE_CUDA(cudaStreamSynchronize(s));
    // dJ/dp = <G, dw> + sum_ij da_ij <xi, D_ij V> - dr_w <xi, V> + sum_i db_i <mu, dT/dq_i Z> h_t/h
    for (int k = 0; k < ndirs; ++k) {
        const double* dp = &dpar[(size_t)k * 9];   // sum_w, r_w, kappa1, kappa2, a11, a12, a22, b1, b2
        const double ih2 = 1.0 / (hg * hg);
        grad[k] = a[kAdjAcc + k] + ih2 * (0.5 * dp[4] * a[1] + 0.25 * dp[5] * a[2] + 0.5 * dp[6] * a[3]) -
                  dp[1] * a[0] + dp[7] * a[4] + dp[8] * a[5];
    }
    return worst;
}

// ---------------------------------------------------------------------------
// price-space jump operator on the paper's non-uniform price grid
// (B_w = T_out I~ C T_in, eqs. 3.12-3.17): tables, weights and spectrum at
// creation, five kernels per application
// ---------------------------------------------------------------------------
struct pide2d_price {
    pide2d_model model;
    int precision;
    int nx1, nz, nin, nout, P;
    double hz;
    int ny_minus, ny_plus;
    cudaStream_t stream;
    char* ws;
    size_t off_gl, off_omega, off_pad, off_part, off_moment, off_params, off_rows, off_wh, off_twr, off_twd,
        off_tin_s, off_tin_w, off_tout_t, off_tout_u, off_A, off_S, off_By, off_loop, total;
    std::vector<double> x;         // the price nodes
    double par[9];
    std::string err;
    bool broken = false;
    // instantiated BiCGSTAB graphs, one per system (c0, c1), and their capture stream
    struct BicgGraph {
        double c0, c1;
        cudaGraph_t g;
        cudaGraphExec_t ex;
    };
    std::vector<BicgGraph> bicg;
    cudaStream_t cap = nullptr;
    template <typename T> T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
    ~pide2d_price() {
        if (!bicg.empty()) cudaStreamSynchronize(stream);
        for (auto& b : bicg) {
            cudaGraphExecDestroy(b.ex);
            cudaGraphDestroy(b.g);
        }
        if (cap) cudaStreamDestroy(cap);
    }
};

namespace {

int pow2_at_least(int n) {
    int p = 16;
    while (p < n) p *= 2;
    return p;
}

// cubic Lagrange weights at t over the four nodes starting at s0
void lagrange4(const double* nodes, int s0, double t, double w[4]) {
    for (int q = 0; q < 4; ++q) {
        double v = 1.0;
        for (int r = 0; r < 4; ++r)
            if (r != q) v *= (t - nodes[s0 + r]) / (nodes[s0 + q] - nodes[s0 + r]);
        w[q] = v;
    }
}

// first index k with nodes[k] <= t < nodes[k+1] (clamped to [0, n-2])
int bracket(const std::vector<double>& nodes, double t) {
    int lo = 0, hi = (int)nodes.size() - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (nodes[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

std::string check_price_grid(const pide2d_price_grid* g) {
    if (!g || !g->x) return "price grid or its nodes are NULL";
    if (g->nx < 4 || g->nx > 8192) return "price grid: 4 <= nx <= 8192";
    if (g->x[0] != 0.0) return "price grid: x[0] must be 0";
    for (int i = 0; i < g->nx; ++i)
        if (!(g->x[i + 1] > g->x[i]) || !std::isfinite(g->x[i + 1])) return "price grid: nodes must increase";
    if (g->n_z < 2 || !(g->h_z > 0.0) || !std::isfinite(g->h_z)) return "price grid: n_z >= 2 and h_z > 0";
    if (g->ny_minus + g->ny_plus + 1 < 4) return "price grid: at least four y_out points";
    if (g->precision != PIDE2D_FP64 && g->precision != PIDE2D_FP32_BULK) return "price grid: precision invalid";
    return "";
}

struct PriceSizes {
    int nx1, nz, nin, nout, P;
};

PriceSizes price_sizes(const pide2d_price_grid* g) {
    PriceSizes z{};
    z.nx1 = g->nx + 1;
    z.nz = g->n_z;
    z.nin = g->ny_minus + g->ny_plus + 2 * g->n_z;
    z.nout = g->ny_minus + g->ny_plus + 1;
    z.P = pow2_at_least(std::max(z.nin, 4 * z.nz));   // Omega must fit the top-left quarter
    return z;
}

template <typename R>
void price_layout(pide2d_price* H) {
    const int P = H->P;
    const int ng = spectrum_groups<R>(P);
    const int nzz = 2 * H->nz;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align256(bytes);
        return at;
    };
    H->off_gl = take((size_t)(kGlTotal + kKtabMax) * 8);
    H->off_omega = take((size_t)nzz * nzz * 8);
    H->off_pad = take((size_t)(P / 2) * (P / 2) * 8);
    H->off_part = take((size_t)((nzz * nzz + 255) / 256) * 3 * 8);
    H->off_moment = take(moment_doubles() * 8);
    H->off_params = take(16 * 8);
    H->off_rows = take((size_t)spectrum_groups<double>(P) * P * cgroup_bytes<double>());
    H->off_wh = take((size_t)ng * P * cgroup_bytes<R>());
    H->off_twr = take((size_t)tw_entries(P) * 2 * sizeof(R));
    H->off_twd = take((size_t)tw_entries(P) * 16);
    H->off_tin_s = take((size_t)H->nin * 4);
    H->off_tin_w = take((size_t)H->nin * 4 * 8);
    H->off_tout_t = take((size_t)H->nx1 * 4);
    H->off_tout_u = take((size_t)H->nx1 * 4 * 8);
    H->off_A = take((size_t)P * P * sizeof(R));
    H->off_S = take((size_t)ng * P * cgroup_bytes<R>());
    H->off_By = take((size_t)H->nout * H->nout * 8);
    H->off_loop = o;                // the time-loop fields follow (ps_loop_bytes)
    H->total = o;
}

}  // namespace

#define PIDE_PCUDA(call)                                                                  \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            H->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
            H->broken = true;                                                             \
            return PIDE2D_ERR_CUDA;                                                       \
        }                                                                                 \
    } while (0)

template <typename R>
static pide2d_status price_create(pide2d_price* H, const pide2d_price_grid* g) {
    cudaStream_t s = H->stream;
    const int P = H->P, nin = H->nin, nout = H->nout, nx1 = H->nx1;
    std::vector<double> x(g->x, g->x + nx1);
    // T_in: x-grid -> y_in (v = 0 beyond x_max); T_out: y_out -> x-grid (linear below y_out)
    std::vector<int> ts(nin), tt(nx1);
    std::vector<double> tw(4 * (size_t)nin, 0.0), tu(4 * (size_t)nx1, 0.0);
    for (int j = 0; j < nin; ++j) {
        const double y = std::exp((j - H->nz - H->ny_minus + 0.5) * H->hz);
        if (y > x[nx1 - 1]) {
            ts[j] = -1;
            continue;
        }
        const int k = bracket(x, y);
        const int s0 = std::min(std::max(k - 1, 0), nx1 - 4);
        ts[j] = s0;
        lagrange4(x.data(), s0, y, &tw[4 * (size_t)j]);
    }
    std::vector<double> yo(nout);
    for (int i = 0; i < nout; ++i) yo[i] = std::exp((i - H->ny_minus) * H->hz);
    for (int m = 0; m < nx1; ++m) {
        const double t = x[m];
        double* u = &tu[4 * (size_t)m];
        if (t < yo[0] || t > yo[nout - 1]) {
            const int j = t < yo[0] ? 0 : nout - 2;
            tt[m] = j;
            u[0] = (yo[j + 1] - t) / (yo[j + 1] - yo[j]);
            u[1] = (t - yo[j]) / (yo[j + 1] - yo[j]);
            continue;
        }
        const int k = bracket(yo, t);
        const int s0 = std::min(std::max(k - 1, 0), nout - 4);
        tt[m] = s0;
        lagrange4(yo.data(), s0, t, u);
    }
    const std::vector<double> gl = quadrature_nodes();
    PIDE_PCUDA(cudaMemsetAsync(H->ws, 0, H->total, s));
    PIDE_PCUDA(cudaMemcpyAsync(H->at<double>(H->off_gl), gl.data(), gl.size() * 8, cudaMemcpyHostToDevice, s));
    PIDE_PCUDA(cudaMemcpyAsync(H->at<int>(H->off_tin_s), ts.data(), ts.size() * 4, cudaMemcpyHostToDevice, s));
    PIDE_PCUDA(cudaMemcpyAsync(H->at<double>(H->off_tin_w), tw.data(), tw.size() * 8, cudaMemcpyHostToDevice, s));
    PIDE_PCUDA(cudaMemcpyAsync(H->at<int>(H->off_tout_t), tt.data(), tt.size() * 4, cudaMemcpyHostToDevice, s));
    PIDE_PCUDA(cudaMemcpyAsync(H->at<double>(H->off_tout_u), tu.data(), tu.size() * 8, cudaMemcpyHostToDevice, s));
    PIDE_PCUDA(launch_twiddles<R>(P, H->at<void>(H->off_twr), s));
    PIDE_PCUDA(launch_twiddles<double>(P, H->at<void>(H->off_twd), s));
    // weights on the z-lattice (N_z = nz, width hz), then conj(fft2(Omega padded))/P^2
    const int nzz = 2 * H->nz;
    PIDE_PCUDA(precompute_core(nzz, H->hz, H->at<double>(H->off_gl), H->model, H->at<double>(H->off_omega),
                               H->at<double>(H->off_part), H->at<double>(H->off_moment),
                               H->at<double>(H->off_params), s));
    PIDE_PCUDA(cudaMemcpy2DAsync(H->at<double>(H->off_pad), (size_t)(P / 2) * 8, H->at<double>(H->off_omega),
                                 (size_t)nzz * 8, (size_t)nzz * 8, nzz, cudaMemcpyDeviceToDevice, s));
    Geometry gd{};
    gd.N = P / 2;
    gd.P = P;
    gd.rows = P;
    gd.ng = spectrum_groups<double>(P);
    FwdArgs<double> wa{};
    wa.g = gd;
    wa.mode = FWD_WEIGHTS;
    wa.omega = H->at<double>(H->off_pad);
    wa.S = H->at<void>(H->off_rows);
    wa.pair0 = 0;
    wa.npairs = P / 4;
    wa.tw = H->at<void>(H->off_twd);
    PIDE_PCUDA(launch_row_forward<double>(wa, s));
    PIDE_PCUDA(launch_weights_col<R>(gd, H->at<void>(H->off_rows), H->at<void>(H->off_wh), nullptr,
                                     H->at<void>(H->off_twd), s));
    PIDE_PCUDA(cudaMemcpyAsync(H->par, H->at<double>(H->off_params), 9 * 8, cudaMemcpyDeviceToHost, s));
    PIDE_PCUDA(cudaStreamSynchronize(s));
    for (double v : H->par)
        if (!std::isfinite(v)) {
            H->err = "price-space precompute: rates are not finite";
            return PIDE2D_ERR_ARG;
        }
    return PIDE2D_OK;
}

template <typename R>
static pide2d_status price_apply(pide2d_price* H, const double* V, double* out) {
    cudaStream_t s = H->stream;
    const int P = H->P;
    R* A = H->at<R>(H->off_A);
    void* S = H->at<void>(H->off_S);
    const void* tw = H->at<void>(H->off_twr);
    PIDE_PCUDA(launch_ps_tin<R>(P, H->nin, H->nx1, H->at<int>(H->off_tin_s), H->at<double>(H->off_tin_w), V, A, s));
    PIDE_PCUDA(launch_ps_rows_fwd<R>(P, A, H->nin, S, tw, s));
    PIDE_PCUDA(launch_ps_col<R>(P, S, H->at<void>(H->off_wh), H->nin, H->nout, tw, s));
    PIDE_PCUDA(launch_ps_rows_inv<R>(P, S, H->nout, H->at<double>(H->off_By), H->nout, tw, s));
    PIDE_PCUDA(launch_ps_tout(H->nx1, H->nout, H->at<int>(H->off_tout_t), H->at<double>(H->off_tout_u),
                              H->at<double>(H->off_By), H->nout, out, s));
    PIDE_PCUDA(cudaStreamSynchronize(s));
    return PIDE2D_OK;
}

// ---------------------------------------------------------------------------
// the price-space time loop (Sec. 3.3 on the paper's grid), FP64 fields:
// explicit part, T_SL, fixed-point iteration with the price-space jump
// operator, each implicit system solved by Jacobi-preconditioned BiCGSTAB
// ---------------------------------------------------------------------------
namespace {
enum PsField { F_V0, F_V1, F_V2, F_V3, F_V4, F_BV, F_W, F_Z, F_Y, F_YN, F_BY, F_B, F_R, F_RH, F_P, F_VV, F_YY,
               F_S, F_ZZ, F_T, F_DINV, F_COUNT };

double ps_H(double t) { return t > 0.0 ? t * t * t / 6.0 : 0.0; }

// int_{a1}^{b1} int_{a2}^{b2} max(K - (x1 + x2)/2, 0): the positive part of an affine function
// integrated twice in closed form
double ps_put_cell(double K, double a1, double b1, double a2, double b2) {
    return 4.0 * (ps_H(K - 0.5 * a1 - 0.5 * a2) - ps_H(K - 0.5 * a1 - 0.5 * b2) - ps_H(K - 0.5 * b1 - 0.5 * a2) +
                  ps_H(K - 0.5 * b1 - 0.5 * b2));
}

// departure-point tables of one axis: x e^{k ht}, cubic Lagrange, linear beyond x_max
void ps_sl_table(const std::vector<double>& x, double kappa, double ht, std::vector<int>& s, std::vector<double>& w) {
    const int n1 = (int)x.size();
    s.assign(n1, 0);
    w.assign(4 * (size_t)n1, 0.0);
    const double f = std::exp(kappa * ht);
    for (int m = 0; m < n1; ++m) {
        const double t = x[m] * f;
        double* u = &w[4 * (size_t)m];
        if (t > x[n1 - 1]) {
            s[m] = n1 - 4;
            u[2] = (x[n1 - 1] - t) / (x[n1 - 1] - x[n1 - 2]);
            u[3] = (t - x[n1 - 2]) / (x[n1 - 1] - x[n1 - 2]);
            continue;
        }
        const int k = bracket(x, t);
        const int s0 = std::min(std::max(k - 1, 0), n1 - 4);
        s[m] = s0;
        lagrange4(x.data(), s0, t, u);
    }
}
}  // namespace

static size_t ps_field_bytes(int nx1) { return align256((size_t)nx1 * nx1 * 8); }

static size_t ps_loop_bytes(int nx1) {
    return (size_t)F_COUNT * ps_field_bytes(nx1) + 3 * align256((size_t)nx1 * 3 * 8) + 2 * align256((size_t)nx1 * 4) +
           2 * align256((size_t)nx1 * 4 * 8) + align256((size_t)ps_reduction_blocks() * 3 * 8) + 256 + 256;
}

static pide2d_status price_solve(pide2d_price* H, const pide2d_contract* c, double theta, int n_steps, double tol,
                                 int damping, int kmax, double* values_out, pide2d_stats* stats) {
    cudaStream_t s = H->stream;
    const int n1 = H->nx1;
    const size_t n = (size_t)n1 * n1;
    char* base = H->ws + H->off_loop;
    auto fld = [&](int i) { return reinterpret_cast<double*>(base + (size_t)i * ps_field_bytes(n1)); };
    char* q = base + (size_t)F_COUNT * ps_field_bytes(n1);
    auto take = [&](size_t bytes) {
        char* at = q;
        q += align256(bytes);
        return at;
    };
    double* dx = reinterpret_cast<double*>(take((size_t)n1 * 3 * 8));
    double* da1 = reinterpret_cast<double*>(take((size_t)n1 * 3 * 8));
    double* db2 = reinterpret_cast<double*>(take((size_t)n1 * 3 * 8));
    int* ds1 = reinterpret_cast<int*>(take((size_t)n1 * 4));
    int* ds2 = reinterpret_cast<int*>(take((size_t)n1 * 4));
    double* dw1 = reinterpret_cast<double*>(take((size_t)n1 * 4 * 8));
    double* dw2 = reinterpret_cast<double*>(take((size_t)n1 * 4 * 8));
    double* part = reinterpret_cast<double*>(take((size_t)ps_reduction_blocks() * 3 * 8));
    double* res = reinterpret_cast<double*>(q);
    PsBicg* bst = reinterpret_cast<PsBicg*>(q + 256);
    const std::vector<double>& x = H->x;
    // central differences on the non-uniform grid (Sec. 3.2.1); row 0 zero, last row:
    // second difference zero, first difference backward
    std::vector<double> a1(3 * (size_t)n1, 0.0), b2(3 * (size_t)n1, 0.0);
    for (int m = 1; m < n1 - 1; ++m) {
        const double hm = x[m] - x[m - 1], hp = x[m + 1] - x[m];
        a1[3 * m + 0] = -hp / (hm * (hm + hp));
        a1[3 * m + 1] = (hp - hm) / (hm * hp);
        a1[3 * m + 2] = hm / (hp * (hm + hp));
        b2[3 * m + 0] = 2.0 / (hm * (hm + hp));
        b2[3 * m + 1] = -2.0 / (hm * hp);
        b2[3 * m + 2] = 2.0 / (hp * (hm + hp));
    }
    const double hN = x[n1 - 1] - x[n1 - 2];
    a1[3 * (n1 - 1) + 0] = -1.0 / hN;
    a1[3 * (n1 - 1) + 1] = 1.0 / hN;
    PIDE_PCUDA(cudaMemcpyAsync(dx, x.data(), n1 * 8, cudaMemcpyHostToDevice, s));
    PIDE_PCUDA(cudaMemcpyAsync(da1, a1.data(), a1.size() * 8, cudaMemcpyHostToDevice, s));
    PIDE_PCUDA(cudaMemcpyAsync(db2, b2.data(), b2.size() * 8, cudaMemcpyHostToDevice, s));
    PsDiff d{n1, dx, da1, db2, H->par[4], H->par[5], H->par[6]};
    const double rw = H->par[1], k1 = H->par[2], k2 = H->par[3];

    // V^0: the payoff, cell-averaged on cells that meet the kink (Sec. 3.2.3)
    {
        const double K = c->strike;
        std::vector<double> lo(n1), hi(n1), v0(n);
        for (int m = 0; m < n1; ++m) {
            lo[m] = m == 0 ? -0.5 * (x[0] + x[1]) : 0.5 * (x[m - 1] + x[m]);
            hi[m] = m == n1 - 1 ? 2.0 * x[n1 - 1] - 0.5 * (x[n1 - 2] + x[n1 - 1]) : 0.5 * (x[m] + x[m + 1]);
        }
        for (int m2 = 0; m2 < n1; ++m2)
            for (int m1 = 0; m1 < n1; ++m1) {
                const bool kink = lo[m1] + lo[m2] < 2 * K && hi[m1] + hi[m2] > 2 * K;
                double put = std::max(K - 0.5 * (x[m1] + x[m2]), 0.0);
                double lin = 0.5 * (x[m1] + x[m2]) - K;
                if (kink) {
                    const double area = (hi[m1] - lo[m1]) * (hi[m2] - lo[m2]);
                    put = ps_put_cell(K, lo[m1], hi[m1], lo[m2], hi[m2]) / area;
                    lin = 0.25 * (lo[m1] + hi[m1] + lo[m2] + hi[m2]) - K;
                }
                v0[(size_t)m2 * n1 + m1] = c->payoff == PIDE2D_CALL_AVG ? put + lin : put;
            }
        PIDE_PCUDA(cudaMemcpyAsync(fld(F_V0), v0.data(), n * 8, cudaMemcpyHostToDevice, s));
        PIDE_PCUDA(cudaStreamSynchronize(s));
    }
    auto apply_jump = [&](const double* V, double* out) -> pide2d_status {
        return H->precision == PIDE2D_FP64 ? price_apply<double>(H, V, out) : price_apply<float>(H, V, out);
    };
    // BiCGSTAB with Jacobi preconditioning for (c0 I - c1 D) X = B, X holding the
    // start: one graph launch (set-up and a while-node over the iterations, the
    // scalars on the device), then one read of the solver state
    constexpr int kBicgMaxIt = 20000;
    constexpr size_t kBicgGraphs = 8;
    auto bicgstab = [&](double c0, double c1, const double* Bv, double* X, int* its) -> pide2d_status {
        cudaGraphExec_t ex = nullptr;
        for (const auto& bg : H->bicg)
            if (bg.c0 == c0 && bg.c1 == c1) ex = bg.ex;
        if (!ex) {
            if (!H->cap) PIDE_PCUDA(cudaStreamCreateWithFlags(&H->cap, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            PIDE_PCUDA(cudaGraphCreate(&g, 0));
            const PsBicgArgs ba{d, n, c0, c1, Bv, X, fld(F_R), fld(F_RH), fld(F_P), fld(F_VV), fld(F_YY), fld(F_S),
                                fld(F_ZZ), fld(F_T), fld(F_DINV), part, res, bst, kBicgMaxIt};
            const char* where = "";
            cudaError_t e = record_ps_bicg(g, H->cap, ba, &where);
            if (e == cudaSuccess) {
                e = cudaGraphInstantiate(&ex, g, 0);
                where = "cudaGraphInstantiate";
            }
            if (e != cudaSuccess) {
                cudaGraphDestroy(g);
                H->err = std::string("price-space BiCGSTAB graph: ") + where + ": " + cudaGetErrorString(e);
                H->broken = true;
                return PIDE2D_ERR_CUDA;
            }
            if (H->bicg.size() >= kBicgGraphs) {
                PIDE_PCUDA(cudaStreamSynchronize(s));       // the oldest may still be queued
                cudaGraphExecDestroy(H->bicg.front().ex);
                cudaGraphDestroy(H->bicg.front().g);
                H->bicg.erase(H->bicg.begin());
            }
            H->bicg.push_back({c0, c1, g, ex});
        }
        PIDE_PCUDA(cudaGraphLaunch(ex, s));
        PsBicg hb{};
        PIDE_PCUDA(cudaMemcpyAsync(&hb, bst, sizeof hb, cudaMemcpyDeviceToHost, s));
        PIDE_PCUDA(cudaStreamSynchronize(s));
        *its = hb.it;
        if (!(hb.rn <= hb.lim)) {
            H->err = "price-space BiCGSTAB did not reach its tolerance";
            return PIDE2D_ERR_NOT_CONVERGED;
        }
        return PIDE2D_OK;
    };

    std::vector<int> hist{F_V0};
    std::vector<int> freel{F_V4, F_V3, F_V2, F_V1};
    int cur = F_V0;
    pide2d_status st = apply_jump(fld(F_V0), fld(F_BV));
    if (st != PIDE2D_OK) return st;
    pide2d_stats S{};
    const double T = c->maturity, ht_full = T / n_steps;
    std::vector<int> sl1, sl2;
    std::vector<double> wl1, wl2;
    // one theta step from V (field cur) with B_w V in F_BV; start in F_Y; result into `out_field`
    auto theta_step = [&](int out_field, double ht, double th) -> pide2d_status {
        const double htm = ht * (1.0 - th), htt = ht * th;
        double* V = fld(cur);
        PIDE_PCUDA(launch_ps_diff(d, V, 1.0 - htm * rw, htm, fld(F_BV), htm, fld(F_Z), s));
        ps_sl_table(x, k1, ht, sl1, wl1);
        ps_sl_table(x, k2, ht, sl2, wl2);
        PIDE_PCUDA(cudaMemcpyAsync(ds1, sl1.data(), n1 * 4, cudaMemcpyHostToDevice, s));
        PIDE_PCUDA(cudaMemcpyAsync(ds2, sl2.data(), n1 * 4, cudaMemcpyHostToDevice, s));
        PIDE_PCUDA(cudaMemcpyAsync(dw1, wl1.data(), wl1.size() * 8, cudaMemcpyHostToDevice, s));
        PIDE_PCUDA(cudaMemcpyAsync(dw2, wl2.data(), wl2.size() * 8, cudaMemcpyHostToDevice, s));
        PIDE_PCUDA(launch_ps_sl(n1, ds1, dw1, ds2, dw2, fld(F_Z), fld(F_W), s));
        const double c0 = 1.0 + htt * rw, c1 = htt;
        PIDE_PCUDA(launch_ps_diag_inv(d, c0, c1, fld(F_DINV), s));
        double err = 0.0;
        int k = 0;
        for (k = 1; k <= kmax; ++k) {
            // B_w Y^{k-1} = B_w Y^{k-2} + B_w (Y^{k-1} - Y^{k-2}) after the first iteration: in
            // FP32-bulk the rounding then shrinks with the increment and the test (3.25) can
            // reach tolerances far below FP32's unit roundoff; F_T holds the increment
            if (k == 1) {
                pide2d_status js = apply_jump(fld(F_Y), fld(F_BY));
                if (js != PIDE2D_OK) return js;
            } else {
                pide2d_status js = apply_jump(fld(F_T), fld(F_ZZ));
                if (js != PIDE2D_OK) return js;
                PIDE_PCUDA(launch_ps_axpy(n, 1.0, fld(F_BY), 1.0, fld(F_ZZ), 0.0, nullptr, nullptr, fld(F_BY), s));
            }
            PIDE_PCUDA(launch_ps_axpy(n, htt, fld(F_BY), 1.0, fld(F_W), 0.0, nullptr, nullptr, fld(F_B), s));
            PIDE_PCUDA(cudaMemcpyAsync(fld(F_YN), fld(F_Y), n * 8, cudaMemcpyDeviceToDevice, s));
            int its = 0;
            const pide2d_status js = bicgstab(c0, c1, fld(F_B), fld(F_YN), &its);
            if (js != PIDE2D_OK) return js;
            PIDE_PCUDA(launch_ps_maxrel(n, fld(F_YN), fld(F_Y), part, res, s));
            PIDE_PCUDA(cudaMemcpyAsync(&err, res, 8, cudaMemcpyDeviceToHost, s));
            PIDE_PCUDA(launch_ps_axpy(n, 1.0, fld(F_YN), -1.0, fld(F_Y), 0.0, nullptr, nullptr, fld(F_T), s));
            PIDE_PCUDA(cudaMemcpyAsync(fld(F_Y), fld(F_YN), n * 8, cudaMemcpyDeviceToDevice, s));
            PIDE_PCUDA(cudaStreamSynchronize(s));
            if (err < tol) break;
        }
        if (k > kmax) {
            H->err = "price-space fixed-point iteration not converged";
            return PIDE2D_ERR_NOT_CONVERGED;
        }
        PIDE_PCUDA(cudaMemcpyAsync(fld(out_field), fld(F_Y), n * 8, cudaMemcpyDeviceToDevice, s));
        pide2d_status js = apply_jump(fld(out_field), fld(F_BV));
        if (js != PIDE2D_OK) return js;
        S.fp_iters_total += k;
        S.cell_iters += (double)n * (k + 1);
        return PIDE2D_OK;
    };
    int first = 1;
    if (damping) {
        const int v0 = cur;
        for (int j = 0; j < 4; ++j) {
            const int res = freel.back();
            freel.pop_back();
            PIDE_PCUDA(cudaMemcpyAsync(fld(F_Y), fld(cur), n * 8, cudaMemcpyDeviceToDevice, s));
            st = theta_step(res, ht_full / 4.0, 1.0);
            if (st != PIDE2D_OK) return st;
            if (cur != v0) freel.push_back(cur);
            cur = res;
        }
        hist = {cur, v0};
        first = 2;
        S.steps_done = 1;
    }
    for (int step = first; step <= n_steps; ++step) {
        // Y^{n,0}: polynomial extrapolation of the history (eq. 3.26)
        const int cnt = (int)hist.size() < 4 ? (int)hist.size() : 4;
        static const double coef[4][4] = {{1, 0, 0, 0}, {2, -1, 0, 0}, {3, -3, 1, 0}, {4, -6, 4, -1}};
        const double* cf = coef[cnt - 1];
        PIDE_PCUDA(launch_ps_axpy(n, cf[0], fld(hist[0]), cf[1], cnt > 1 ? fld(hist[1]) : nullptr, cf[2],
                                  cnt > 2 ? fld(hist[2]) : nullptr, nullptr, fld(F_Y), s));
        if (cnt > 3) PIDE_PCUDA(launch_ps_axpy(n, 1.0, fld(F_Y), cf[3], fld(hist[3]), 0.0, nullptr, nullptr, fld(F_Y), s));
        const int res = freel.back();
        freel.pop_back();
        cur = hist[0];
        st = theta_step(res, ht_full, theta);
        if (st != PIDE2D_OK) return st;
        hist.insert(hist.begin(), res);
        if (hist.size() > 4) {
            freel.push_back(hist.back());
            hist.pop_back();
        }
        cur = res;
        S.steps_done = step;
    }
    if (values_out) PIDE_PCUDA(cudaMemcpyAsync(values_out, fld(hist[0]), n * 8, cudaMemcpyDefault, s));
    PIDE_PCUDA(cudaStreamSynchronize(s));
    if (stats) *stats = S;
    return PIDE2D_OK;
}

// ---------------------------------------------------------------------------
// public entry points
// ---------------------------------------------------------------------------
extern "C" {

pide2d_status pide2d_workspace_bytes(const pide2d_grid* grid, size_t* bytes) {
    const std::string e = check_grid(grid);
    if (!e.empty() || !bytes) {
        g_create_error = e.empty() ? "bytes is NULL" : e;
        return PIDE2D_ERR_ARG;
    }
    Layout L;
    layout_for(grid, L);
    *bytes = L.total;
    return PIDE2D_OK;
}

pide2d_status pide2d_create(const pide2d_grid* grid, const pide2d_model* model, const pide2d_contract* contract,
                            double theta, double dt, double fp_tol, const pide2d_options* opts, void* workspace,
                            size_t workspace_bytes, void* cuda_stream, pide2d_t** out) {
    if (out) *out = nullptr;
    if (!out) { g_create_error = "out is NULL"; return PIDE2D_ERR_ARG; }
    std::string e = check_grid(grid);
    if (e.empty() && !model) e = "model is NULL";
    if (e.empty() && !contract) e = "contract is NULL";
    if (e.empty()) {
        const pide2d_model& m = *model;
        const double det = m.rho[0] * m.rho[2] - m.rho[1] * m.rho[1];
        if (!(m.alpha >= 0.0 && m.alpha < 1.0)) e = "model.alpha must be in [0, 1)";
        else if (!(m.delta > 0.0) || !(m.lambda > 0.0)) e = "model.delta and model.lambda must be positive";
        else if (!(m.rho[0] > 0.0) || !(det > 0.0)) e = "model.rho must be positive definite";
        else if (!(m.lambda > m.eta[0] + 0.5 * m.rho[0]) || !(m.lambda > m.eta[1] + 0.5 * m.rho[2]))
            e = "E[exp L_i(1)] is infinite: need lambda > eta_i + rho_ii/2";
        else if (!std::isfinite(m.r)) e = "model.r must be finite";
        else {
            const double sd = m.sigma_cov[0] * m.sigma_cov[2] - m.sigma_cov[1] * m.sigma_cov[1];
            if (m.sigma_cov[0] < 0.0 || m.sigma_cov[2] < 0.0 || sd < 0.0) e = "model.sigma_cov must be PSD";
        }
    }
    if (e.empty()) {
        const pide2d_contract& c = *contract;
        if (c.payoff < 0 || c.payoff > 2) e = "contract.payoff invalid";
        else if (!(c.strike > 0.0) || !(c.maturity > 0.0)) e = "contract strike and maturity must be positive";
    }
    int n_steps = 0;
    if (e.empty()) {
        if (!(theta >= 0.5 && theta <= 1.0)) e = "theta must be in [0.5, 1]";
        else if (!(dt > 0.0) || !(fp_tol > 0.0)) e = "dt and fp_tol must be positive";
        else {
            const double ns = contract->maturity / dt;
            n_steps = (int)std::llround(ns);
            if (n_steps < 1 || std::fabs(ns - n_steps) > 1e-9 * ns) e = "maturity/dt must be an integer >= 1";
        }
    }
    if (e.empty() && opts && (opts->kmax < 0 || opts->kmax > 100000)) e = "opts.kmax out of range";
    if (e.empty() && opts && (opts->host_loop < 0 || opts->host_loop > 1)) e = "opts.host_loop must be 0 or 1";
    if (!e.empty()) { g_create_error = e; return PIDE2D_ERR_ARG; }

    Layout L;
    layout_for(grid, L);
    if (!workspace || ((uintptr_t)workspace & 255) != 0 || workspace_bytes < L.total) {
        char buf[200];
        std::snprintf(buf, sizeof buf, "workspace must be 256-byte aligned device memory of >= %zu bytes", L.total);
        g_create_error = buf;
        return PIDE2D_ERR_WORKSPACE;
    }
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, workspace) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        g_create_error = "workspace is not device memory";
        return PIDE2D_ERR_WORKSPACE;
    }

    pide2d* H = new (std::nothrow) pide2d();
    if (!H) { g_create_error = "out of host memory"; return PIDE2D_ERR_ARG; }
    H->grid = *grid;
    H->model = *model;
    H->contract = *contract;
    H->theta = theta;
    H->dt = dt;
    H->tol = fp_tol;
    H->kmax = (opts && opts->kmax > 0) ? opts->kmax : 100;
    H->damping = opts ? (opts->damping != 0) : 1;
    H->host_loop = opts ? (opts->host_loop != 0) : 0;
    H->n_steps = n_steps;
    H->sl_order = grid->sl_order == 0 ? 3 : grid->sl_order;
    H->L = L;
    H->stream = (cudaStream_t)cuda_stream;
    H->ws = (char*)workspace;
    H->h = 2.0 * grid->half_width / grid->n;
    H->s_lo1 = grid->s_center[0] - grid->half_width;
    H->s_lo2 = grid->s_center[1] - grid->half_width;
    H->steps_done = 0;
    std::memset(&H->stats, 0, sizeof H->stats);
    H->broken = false;
    const pide2d_status st = (grid->precision == PIDE2D_FP64) ? do_create<double>(H) : do_create<float>(H);
    if (st != PIDE2D_OK) {
        g_create_error = H->err;
        delete H;
        return st;
    }
    *out = H;
    return PIDE2D_OK;
}

static pide2d_status step_nosync(pide2d_t* H, int* fp_iters, double* fp_resid) {
    if (H->broken) { H->err = "handle unusable after a CUDA error"; return PIDE2D_ERR_STATE; }
    if (H->steps_done >= H->n_steps) { H->err = "all time steps done"; return PIDE2D_ERR_STATE; }
    return H->grid.precision == PIDE2D_FP64 ? do_step<double>(H, fp_iters, fp_resid)
                                            : do_step<float>(H, fp_iters, fp_resid);
}

pide2d_status pide2d_step(pide2d_t* H, int* fp_iters, double* fp_resid) {
    if (!H) return PIDE2D_ERR_ARG;
    pide2d_status s = step_nosync(H, fp_iters, fp_resid);
    if (s == PIDE2D_ERR_CUDA || s == PIDE2D_ERR_STATE || s == PIDE2D_ERR_ARG || !H->last_step_device) return s;
    const pide2d_status r = read_ctl(H);
    if (r != PIDE2D_OK) return r;
    if (fp_iters) *fp_iters = H->ctl.last_step_k;
    if (fp_resid) *fp_resid = H->ctl.step_resid;
    const pide2d_status c = check_device_convergence(H);
    return s != PIDE2D_OK ? s : c;
}

pide2d_status pide2d_solve(pide2d_t* H, double* price, double* values_out, pide2d_stats* stats) {
    if (!H) return PIDE2D_ERR_ARG;
    if (H->broken) { H->err = "handle unusable after a CUDA error"; return PIDE2D_ERR_STATE; }
    pide2d_status worst = PIDE2D_OK;
    while (H->steps_done < H->n_steps) {
        // device-loop steps are queued back to back; the host waits once, below
        const pide2d_status s = step_nosync(H, nullptr, nullptr);
        if (s == PIDE2D_ERR_CUDA || s == PIDE2D_ERR_STATE || s == PIDE2D_ERR_ARG) return s;
        if (s != PIDE2D_OK) worst = s;
    }
    {
        const pide2d_status r = read_ctl(H);
        if (r != PIDE2D_OK) return r;
        if (check_device_convergence(H) != PIDE2D_OK) worst = PIDE2D_ERR_NOT_CONVERGED;
        if (H->group_nonconv) worst = PIDE2D_ERR_NOT_CONVERGED;
    }
    if (price) {
        const pide2d_status s = H->grid.precision == PIDE2D_FP64 ? do_price<double>(H, price) : do_price<float>(H, price);
        if (s != PIDE2D_OK) return s;
    }
    if (values_out) {
        const pide2d_status s = pide2d_get_values(H, values_out);
        if (s != PIDE2D_OK) return s;
    }
    if (stats) *stats = combined_stats(H);
    return worst;
}

pide2d_status pide2d_get_values(pide2d_t* H, double* dst) {
    if (!H || !dst) return PIDE2D_ERR_ARG;
    if (H->broken) return PIDE2D_ERR_STATE;
    return H->grid.precision == PIDE2D_FP64 ? do_get_values<double>(H, dst) : do_get_values<float>(H, dst);
}

pide2d_status pide2d_get_weights(pide2d_t* H, double* omega_out, double* rates_out) {
    if (!H) return PIDE2D_ERR_ARG;
    if (H->broken) return PIDE2D_ERR_STATE;
    const int N = H->grid.n;
    if (omega_out) {
        PIDE_CUDA(cudaMemcpyAsync(omega_out, H->at<double>(R_OMEGA), (size_t)N * N * 8, cudaMemcpyDefault, H->stream));
        PIDE_CUDA(cudaStreamSynchronize(H->stream));
    }
    if (rates_out) {
        PIDE_CUDA(cudaMemcpy(rates_out, H->par, 9 * 8, cudaMemcpyDefault));
    }
    return PIDE2D_OK;
}

pide2d_status pide2d_greeks(pide2d_t* H, double* delta1, double* delta2, double* gamma11, double* gamma12,
                            double* gamma22) {
    if (!H) return PIDE2D_ERR_ARG;
    if (H->broken) return PIDE2D_ERR_STATE;
    double* const outs[5] = {delta1, delta2, gamma11, gamma12, gamma22};
    return H->grid.precision == PIDE2D_FP64 ? do_greeks<double>(H, outs) : do_greeks<float>(H, outs);
}

pide2d_status pide2d_apply_jump(pide2d_t* H, const double* U, double tau, int far_field, double* out) {
    if (!H || !U || !out) return PIDE2D_ERR_ARG;
    if (H->broken) return PIDE2D_ERR_STATE;
    return H->grid.precision == PIDE2D_FP64 ? do_apply_jump<double>(H, U, tau, far_field, out)
                                            : do_apply_jump<float>(H, U, tau, far_field, out);
}

pide2d_status pide2d_iteration_probe(pide2d_t* H, const double* r, double ht, double theta, double* delta_out,
                                     double* bdelta_out, double* stop_out) {
    if (!H || !r) return PIDE2D_ERR_ARG;
    if (H->broken) return PIDE2D_ERR_STATE;
    if (!(ht > 0.0) || !(theta > 0.0) || !(theta <= 1.0)) {
        H->err = "iteration probe: ht must be > 0 and theta in (0, 1]";
        return PIDE2D_ERR_ARG;
    }
    return H->grid.precision == PIDE2D_FP64
               ? do_iteration_probe<double>(H, r, ht, theta, delta_out, bdelta_out, stop_out)
               : do_iteration_probe<float>(H, r, ht, theta, delta_out, bdelta_out, stop_out);
}

pide2d_status pide2d_profile(pide2d_t* H, int enable) {
    if (!H) return PIDE2D_ERR_ARG;
    if (enable) {
        for (auto& r : H->recs) {
            H->pool.push_back(r.a);
            H->pool.push_back(r.b);
        }
        H->recs.clear();
    }
    H->prof = enable != 0;
    return PIDE2D_OK;
}

pide2d_status pide2d_profile_read(pide2d_t* H, pide2d_kernel_times* out) {
    if (!H || !out) return PIDE2D_ERR_ARG;
    std::memset(out, 0, sizeof *out);
    PIDE_CUDA(cudaStreamSynchronize(H->stream));
    for (const auto& r : H->recs) {
        float ms = 0.f;
        PIDE_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        out->launches[r.cls] += 1;
        out->ms[r.cls] += ms;
    }
    return PIDE2D_OK;
}

pide2d_status pide2d_tape_bytes(pide2d_t* H, int interval, int ndirs, size_t* bytes) {
    if (!H || !bytes || interval < 1 || ndirs < 0 || ndirs > 16) return PIDE2D_ERR_ARG;
    *bytes = tape_layout(H->L, H->n_steps, interval, ndirs).total;
    return PIDE2D_OK;
}

pide2d_status pide2d_record(pide2d_t* H, void* tape, size_t bytes, int interval, int ndirs) {
    if (!H) return PIDE2D_ERR_ARG;
    if (H->broken) return PIDE2D_ERR_STATE;
    if (H->steps_done != 0) { H->err = "pide2d_record must precede the first step"; return PIDE2D_ERR_STATE; }
    if (interval < 1 || ndirs < 0 || ndirs > 16) { H->err = "interval >= 1 and 0 <= ndirs <= 16"; return PIDE2D_ERR_ARG; }
    const TapeLayout t = tape_layout(H->L, H->n_steps, interval, ndirs);
    if (!tape || ((uintptr_t)tape & 255) != 0 || bytes < t.total) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "tape must be 256-byte aligned device memory of >= %zu bytes", t.total);
        H->err = buf;
        return PIDE2D_ERR_WORKSPACE;
    }
    H->tape.base = static_cast<char*>(tape);
    H->tape.bytes = bytes;
    H->tape.interval = interval;
    H->tape.ndirs = ndirs;
    H->tape.nckpt = t.nckpt;
    H->tape.seg_slots = t.seg_slots;
    H->tape.ckpt_cnt.assign(t.nckpt, 0);
    return PIDE2D_OK;
}

pide2d_status pide2d_adjoint(pide2d_t* H, const pide2d_model* dirs, int ndirs, double* grad) {
    if (!H || (ndirs > 0 && (!dirs || !grad)) || ndirs < 0) return PIDE2D_ERR_ARG;
    if (H->broken) { H->err = "handle unusable after a CUDA error"; return PIDE2D_ERR_STATE; }
    if (!H->tape.base) { H->err = "no tape: call pide2d_record before the first step"; return PIDE2D_ERR_STATE; }
    if (H->steps_done != H->n_steps) { H->err = "pide2d_adjoint needs the finished solve"; return PIDE2D_ERR_STATE; }
    if (ndirs > H->tape.ndirs) { H->err = "more directions than the tape was sized for"; return PIDE2D_ERR_ARG; }
    {
        const pide2d_status r = read_ctl(H);
        if (r != PIDE2D_OK) return r;
    }
    return H->grid.precision == PIDE2D_FP64 ? do_adjoint<double>(H, dirs, ndirs, grad)
                                            : do_adjoint<float>(H, dirs, ndirs, grad);
}

// ---------------------------------------------------------------------------
// workload parameterisation (Appendix A, Table A5): a unit-mean tempered-
// stable subordinator with variance kappa time-changes a Brownian motion with
// drift beta and covariance [[s1^2, c s1 s2], [c s1 s2, s2^2]]
// ---------------------------------------------------------------------------
static std::string check_workload(const pide2d_workload* w) {
    if (!w) return "workload is NULL";
    if (!(w->alpha >= 0.0 && w->alpha < 1.0)) return "workload.alpha must lie in [0, 1)";
    if (!(w->kappa > 0.0) || !std::isfinite(w->kappa)) return "workload.kappa must be positive";
    if (!(w->sigma[0] > 0.0) || !(w->sigma[1] > 0.0) || !std::isfinite(w->sigma[0]) || !std::isfinite(w->sigma[1]))
        return "workload.sigma must be positive";
    if (!(std::fabs(w->corr) < 1.0)) return "workload.corr must lie in (-1, 1)";
    if (!std::isfinite(w->beta[0]) || !std::isfinite(w->beta[1]) || !std::isfinite(w->r))
        return "workload.beta and r must be finite";
    return "";
}

pide2d_status pide2d_model_from_workload(const pide2d_workload* w, pide2d_model* out) {
    const std::string e = check_workload(w);
    if (!e.empty() || !out) {
        pide::set_global_error(e.empty() ? "model is NULL" : e);
        return PIDE2D_ERR_ARG;
    }
    // Table A5: E G(1) = delta Gamma(1 - alpha) / lambda^(1 - alpha) = 1 and
    // V G(1) / E G(1) = (1 - alpha) / lambda = kappa
    const double lam = (1.0 - w->alpha) / w->kappa;
    std::memset(out, 0, sizeof *out);
    out->alpha = w->alpha;
    out->lambda = lam;
    out->delta = std::pow(lam, 1.0 - w->alpha) / std::tgamma(1.0 - w->alpha);
    out->eta[0] = w->beta[0];
    out->eta[1] = w->beta[1];
    const double s1 = w->sigma[0], s2 = w->sigma[1];
    out->rho[0] = s1 * s1;
    out->rho[1] = w->corr * s1 * s2;
    out->rho[2] = s2 * s2;
    out->r = w->r;
    return PIDE2D_OK;
}

pide2d_status pide2d_workload_directions(const pide2d_workload* w, pide2d_model* dirs) {
    pide2d_model m;
    const pide2d_status st = pide2d_model_from_workload(w, &m);
    if (st != PIDE2D_OK) return st;
    if (!dirs) {
        pide::set_global_error("dirs is NULL");
        return PIDE2D_ERR_ARG;
    }
    std::memset(dirs, 0, 6 * sizeof *dirs);
    const double s1 = w->sigma[0], s2 = w->sigma[1], c = w->corr;
    dirs[0].rho[0] = 2.0 * s1;                   // sigma1
    dirs[0].rho[1] = c * s2;
    dirs[1].rho[1] = c * s1;                     // sigma2
    dirs[1].rho[2] = 2.0 * s2;
    dirs[2].rho[1] = s1 * s2;                    // corr
    // kappa: d lambda / d kappa = -lambda / kappa, d delta / d kappa = -(1 - alpha) delta / kappa
    dirs[3].lambda = -m.lambda / w->kappa;
    dirs[3].delta = -(1.0 - w->alpha) * m.delta / w->kappa;
    dirs[4].eta[0] = 1.0;                        // beta1
    dirs[5].eta[1] = 1.0;                        // beta2
    return PIDE2D_OK;
}

pide2d_status pide2d_adjoint_workload(pide2d_t* H, const pide2d_workload* w, double* grad) {
    if (!H || !grad) return PIDE2D_ERR_ARG;
    pide2d_model m, dirs[6];
    if (pide2d_workload_directions(w, dirs) != PIDE2D_OK || pide2d_model_from_workload(w, &m) != PIDE2D_OK) {
        H->err = g_create_error;
        return PIDE2D_ERR_ARG;
    }
    // the handle must price this workload's model
    auto close = [](double a, double b) { return std::fabs(a - b) <= 1e-12 * std::max(1.0, std::fabs(b)); };
    const pide2d_model& hm = H->model;
    const bool same = close(hm.alpha, m.alpha) && close(hm.delta, m.delta) && close(hm.lambda, m.lambda) &&
                      close(hm.eta[0], m.eta[0]) && close(hm.eta[1], m.eta[1]) && close(hm.rho[0], m.rho[0]) &&
                      close(hm.rho[1], m.rho[1]) && close(hm.rho[2], m.rho[2]) && close(hm.r, m.r);
    if (!same) {
        H->err = "pide2d_adjoint_workload: the handle was not created with this workload's model";
        return PIDE2D_ERR_ARG;
    }
    return pide2d_adjoint(H, dirs, 6, grad);
}

pide2d_status pide2d_price_sinh_grid(int nx, double strike, double x_max, double z_iii, double frac,
                                     double* x_out, pide2d_price_grid* grid) {
    if (nx < 4 || nx > 8192 || !(strike > 0.0) || !(x_max > 0.0) || !(z_iii > 0.0) || !(frac > 0.0 && frac < 1.0) ||
        !x_out || !grid) {
        pide::set_global_error("pide2d_price_sinh_grid: invalid arguments");
        return PIDE2D_ERR_ARG;
    }
    const double x_int = 2.5 * strike;
    const double F = std::max(frac, x_int / x_max);
    if (F < 1.0) {
        // c with xi_int / xi_max = F, xi_int = x_int / c, xi_max = xi_int + asinh((x_max - x_int) / c);
        // the ratio falls from 1 (c -> 0) to x_int / x_max (c -> infinity): bisection on log c
        auto ratio = [&](double c) { return 1.0 / (1.0 + c / x_int * std::asinh((x_max - x_int) / c)); };
        double lo = std::log(1e-6 * x_int), hi = std::log(1e6 * x_max);
        for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(hi)); ++it) {
            const double mid = 0.5 * (lo + hi);
            if (ratio(std::exp(mid)) > F) lo = mid;
            else hi = mid;
        }
        const double c = std::exp(0.5 * (lo + hi));
        const double xi_int = x_int / c, xi_max = xi_int + std::asinh((x_max - x_int) / c);
        for (int m = 0; m <= nx; ++m) {
            const double xi = m * (xi_max / nx);
            x_out[m] = xi <= xi_int ? c * xi : x_int + c * std::sinh(xi - xi_int);
        }
    } else {
        for (int m = 0; m <= nx; ++m) x_out[m] = m * (x_max / nx);
    }
    x_out[nx] = x_max;
    grid->nx = nx;
    grid->x = x_out;
    grid->n_z = 2 * nx;
    grid->h_z = z_iii / grid->n_z;
    grid->ny_minus = (int)std::ceil(-std::log(x_out[1]) / grid->h_z);
    grid->ny_plus = (int)std::ceil(std::log(x_max) / grid->h_z);
    return PIDE2D_OK;
}

pide2d_status pide2d_price_workspace_bytes(const pide2d_price_grid* g, size_t* bytes) {
    const std::string e = check_price_grid(g);
    if (!e.empty() || !bytes) {
        g_create_error = e.empty() ? "bytes is NULL" : e;
        return PIDE2D_ERR_ARG;
    }
    const PriceSizes z = price_sizes(g);
    if (z.P > (g->precision == PIDE2D_FP64 ? 4096 : 8192)) {
        g_create_error = "price grid: the transform length exceeds 8192 (4096 in FP64)";
        return PIDE2D_ERR_UNSUPPORTED;
    }
    pide2d_price tmp;
    tmp.nx1 = z.nx1;
    tmp.nz = z.nz;
    tmp.nin = z.nin;
    tmp.nout = z.nout;
    tmp.P = z.P;
    if (g->precision == PIDE2D_FP64) price_layout<double>(&tmp);
    else price_layout<float>(&tmp);
    *bytes = tmp.total + ps_loop_bytes(z.nx1);
    return PIDE2D_OK;
}

pide2d_status pide2d_price_create(const pide2d_price_grid* g, const pide2d_model* model, void* workspace,
                                  size_t workspace_bytes, void* cuda_stream, pide2d_price_t** out) {
    if (out) *out = nullptr;
    if (!out || !model) { g_create_error = "out or model is NULL"; return PIDE2D_ERR_ARG; }
    size_t need = 0;
    const pide2d_status st0 = pide2d_price_workspace_bytes(g, &need);
    if (st0 != PIDE2D_OK) return st0;
    const double det = model->rho[0] * model->rho[2] - model->rho[1] * model->rho[1];
    if (!(model->alpha >= 0.0 && model->alpha < 1.0) || !(model->delta > 0.0) || !(model->lambda > 0.0) ||
        !(model->rho[0] > 0.0) || !(det > 0.0)) {
        g_create_error = "model invalid (alpha in [0,1), delta, lambda > 0, rho positive definite)";
        return PIDE2D_ERR_ARG;
    }
    if (!workspace || ((uintptr_t)workspace & 255) != 0 || workspace_bytes < need) {
        g_create_error = "workspace must be 256-byte aligned device memory of >= pide2d_price_workspace_bytes";
        return PIDE2D_ERR_WORKSPACE;
    }
    pide2d_price* H = new (std::nothrow) pide2d_price();
    if (!H) { g_create_error = "out of host memory"; return PIDE2D_ERR_ARG; }
    const PriceSizes z = price_sizes(g);
    H->model = *model;
    H->precision = g->precision;
    H->nx1 = z.nx1;
    H->nz = z.nz;
    H->nin = z.nin;
    H->nout = z.nout;
    H->P = z.P;
    H->hz = g->h_z;
    H->ny_minus = g->ny_minus;
    H->ny_plus = g->ny_plus;
    H->stream = (cudaStream_t)cuda_stream;
    H->ws = (char*)workspace;
    if (g->precision == PIDE2D_FP64) price_layout<double>(H);
    else price_layout<float>(H);
    H->x.assign(g->x, g->x + z.nx1);
    const pide2d_status st = g->precision == PIDE2D_FP64 ? price_create<double>(H, g) : price_create<float>(H, g);
    if (st != PIDE2D_OK) {
        g_create_error = H->err;
        delete H;
        return st;
    }
    *out = H;
    return PIDE2D_OK;
}

pide2d_status pide2d_price_apply_jump(pide2d_price_t* H, const double* V, double* out) {
    if (!H || !V || !out) return PIDE2D_ERR_ARG;
    if (H->broken) return PIDE2D_ERR_STATE;
    return H->precision == PIDE2D_FP64 ? price_apply<double>(H, V, out) : price_apply<float>(H, V, out);
}

pide2d_status pide2d_price_solve(pide2d_price_t* H, const pide2d_contract* c, double theta, int n_steps,
                                 double fp_tol, const pide2d_options* opts, double* values_out, pide2d_stats* stats) {
    if (!H || !c) return PIDE2D_ERR_ARG;
    if (H->broken) return PIDE2D_ERR_STATE;
    if (c->payoff != PIDE2D_PUT_AVG && c->payoff != PIDE2D_CALL_AVG) {
        H->err = "price-space solve: put or call on the average";
        return PIDE2D_ERR_ARG;
    }
    if (!(c->strike > 0.0) || !(c->maturity > 0.0) || n_steps < 1 || !(theta >= 0.5 && theta <= 1.0) ||
        !(fp_tol > 0.0)) {
        H->err = "price-space solve: strike, maturity, fp_tol > 0, n_steps >= 1, theta in [0.5, 1]";
        return PIDE2D_ERR_ARG;
    }
    const int kmax = (opts && opts->kmax > 0) ? opts->kmax : 100;
    const int damping = opts ? (opts->damping != 0) : 1;
    return price_solve(H, c, theta, n_steps, fp_tol, damping, kmax, values_out, stats);
}

pide2d_status pide2d_price_get_weights(pide2d_price_t* H, double* omega_out, double* rates_out) {
    if (!H) return PIDE2D_ERR_ARG;
    if (H->broken) return PIDE2D_ERR_STATE;
    if (omega_out) {
        const size_t n = (size_t)(2 * H->nz) * (2 * H->nz);
        PIDE_PCUDA(cudaMemcpyAsync(omega_out, H->at<double>(H->off_omega), n * 8, cudaMemcpyDefault, H->stream));
        PIDE_PCUDA(cudaStreamSynchronize(H->stream));
    }
    if (rates_out) std::memcpy(rates_out, H->par, 9 * 8);
    return PIDE2D_OK;
}

const char* pide2d_price_last_error(const pide2d_price_t* H) { return H ? H->err.c_str() : g_create_error.c_str(); }

void pide2d_price_destroy(pide2d_price_t* H) { delete H; }

const char* pide2d_last_error(const pide2d_t* H) {
    if (!H) return g_create_error.c_str();
    return H->err.c_str();
}

void pide2d_destroy(pide2d_t* H) {
    if (!H) return;
    for (auto& r : H->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : H->pool) cudaEventDestroy(e);
    if (!H->graphs.empty()) cudaStreamSynchronize(H->stream);
    for (auto& g : H->graphs) {
        cudaGraphExecDestroy(g.exec);
        cudaGraphDestroy(g.graph);
    }
    if (H->cap) cudaStreamDestroy(H->cap);
    delete H;
}

}  // extern "C"
