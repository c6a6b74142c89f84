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
    R_E1D, R_E2D, R_E1F, R_E2F, R_SIN2D, R_SIN2R,
    R_OMEGA, R_PART, R_PARAMS, R_MOMENT, R_GL, R_RESID,
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
    g.ng = (g.P / 2 + 1 + cgroup<R>() - 1) / cgroup<R>();
    g.nge = N / rgroup<R>();
    g.ldS = round_up(N + 1, 32);
    g.ldR = round_up(N + 1, 32);
    g.eoff = N / 2 + 3;
    const size_t fieldS = (size_t)(N + 1) * g.ldS * 8;
    const size_t fieldR = (size_t)(N + 1) * g.ldR * sizeof(R);
    for (int i = R_V0; i <= R_OUT; ++i) L.size[i] = fieldS;
    L.size[R_RES] = L.size[R_DLT] = fieldR;
    L.size[R_S] = (size_t)g.ng * g.rows * 16;
    L.size[R_WH] = L.size[R_WHI] = (size_t)g.ng * g.P * 16;
    L.size[R_E] = (size_t)g.nge * N * 16;
    L.size[R_TWR] = (size_t)g.P * 2 * sizeof(R);
    L.size[R_TWD] = (size_t)g.P * 16;
    const size_t tl = (size_t)(2 * N + 7);
    L.size[R_E1D] = L.size[R_E2D] = tl * 8;
    L.size[R_E1F] = L.size[R_E2F] = tl * 4;
    L.size[R_SIN2D] = (size_t)(N + 1) * 8;
    L.size[R_SIN2R] = (size_t)(N + 1) * sizeof(R);
    L.size[R_OMEGA] = (size_t)N * N * 8;
    L.size[R_PART] = (size_t)((N * N + 255) / 256) * 3 * 8;
    L.size[R_PARAMS] = 16 * 8;
    L.size[R_MOMENT] = 4 * 8;
    L.size[R_GL] = (size_t)kGlTotal * 8;
    L.size[R_RESID] = 16;
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
    if (g->precision == PIDE2D_FP64 && g->n > 2048) return "FP64 mode supports n <= 2048";
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
    int kmax, damping, n_steps, sl_order;
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
// one theta step (eq. 3.23) by the fixed-point iteration (3.24)-(3.26)
// ---------------------------------------------------------------------------
template <typename R>
static pide2d_status theta_step(pide2d* H, const int* list, int cnt, double theta, double ht, double tau_prev,
                                double tau, int res, int* iters_out, double* resid_out) {
    const Geometry g = H->L.g;
    const int N = g.N;
    const double hg = H->h;
    const double htt = ht * theta, htm = ht * (1.0 - theta);
    const double rw = H->par[1], a11 = H->par[4], a12 = H->par[5], a22 = H->par[6];
    const R d11 = (R)(0.5 * a11 / (hg * hg)), d22 = (R)(0.5 * a22 / (hg * hg)), d12 = (R)(0.25 * a12 / (hg * hg));
    const double Kd_prev = H->contract.strike * std::exp(-H->model.r * tau_prev);
    const double Kd_now = H->contract.strike * std::exp(-H->model.r * tau);
    St<R>* Y = (St<R>*)H->field(res);
    St<R>* W = H->at<St<R>>(R_W);
    St<R>* BV = (St<R>*)H->field(H->bv);
    St<R>* BY = (St<R>*)H->field(H->by);
    R* rres = H->at<R>(R_RES);
    R* dlt = H->at<R>(R_DLT);
    R* E = H->at<R>(R_E);
    const void* tw = H->at<void>(R_TWR);

    // Algorithm 1 steps 2-3: W and Y^{n,0}
    PrepArgs<R> pa{};
    pa.g = g;
    for (int i = 0; i < 4; ++i) pa.V[i] = (const St<R>*)H->field(list[i < cnt ? i : 0]);
    pa.hcount = cnt;
    pa.BV = BV;
    pa.W = W;
    pa.Y = Y;
    pa.cz = rres;            // the residual field is free until the first sweep of the step
    pa.htm = (R)htm;
    pa.rw = (R)rw;
    pa.d11 = d11;
    pa.d22 = d22;
    pa.d12 = d12;
    const double q[2] = {H->par[7] * ht / hg, H->par[8] * ht / hg};
    // the departure stencil and the far-field tables reach N/4 cells at most
    if (!(std::fabs(q[0]) <= N / 4) || !(std::fabs(q[1]) <= N / 4)) {
        H->err = "semi-Lagrangian shift exceeds N/4 cells: time step too large";
        return PIDE2D_ERR_ARG;
    }
    int o[2];
    double w[2][4];
    for (int ax = 0; ax < 2; ++ax) {
        const int fl = (int)std::floor(q[ax]);
        const double f = q[ax] - fl;
        if (H->sl_order == 1) {
            o[ax] = fl;
            w[ax][0] = 1.0 - f;
            w[ax][1] = f;
            w[ax][2] = w[ax][3] = 0.0;
        } else {
            o[ax] = fl - 1;
            w[ax][0] = -f * (f - 1.0) * (f - 2.0) / 6.0;
            w[ax][1] = (f + 1.0) * (f - 1.0) * (f - 2.0) / 2.0;
            w[ax][2] = -(f + 1.0) * f * (f - 2.0) / 2.0;
            w[ax][3] = (f + 1.0) * f * (f - 1.0) / 6.0;
        }
    }
    pa.o1 = o[0];
    pa.o2 = o[1];
    pa.nt = H->sl_order == 1 ? 2 : 4;
    for (int i = 0; i < 4; ++i) {
        pa.w1[i] = (R)w[0][i];
        pa.w2[i] = (R)w[1][i];
    }
    pa.E1d = H->at<double>(R_E1D);
    pa.E2d = H->at<double>(R_E2D);
    pa.Kd_prev = Kd_prev;
    pa.Kd_now = Kd_now;
    pa.payoff = H->contract.payoff;
    PIDE_LAUNCH(PIDE2D_KERNEL_PREP, launch_prep<R>(pa, H->stream));

    // B_w Y^{n,0} by a full sweep (with far field) and the first residual
    FwdArgs<R> fa{};
    fa.g = g;
    fa.mode = FWD_FULL;
    fa.Y = Y;
    fa.D = dlt;
    fa.E1 = (const R*)(sizeof(R) == 4 ? (const void*)H->at<float>(R_E1F) : (const void*)H->at<double>(R_E1D));
    fa.E2 = (const R*)(sizeof(R) == 4 ? (const void*)H->at<float>(R_E2F) : (const void*)H->at<double>(R_E2D));
    fa.Kd = (R)Kd_now;
    fa.payoff = H->contract.payoff;
    fa.S = H->at<void>(R_S);
    fa.pair0 = 0;
    fa.npairs = N + 1;
    fa.tw = tw;
    PIDE_LAUNCH(PIDE2D_KERNEL_ROW_FORWARD_FULL, launch_row_forward<R>(fa, H->stream));
    ColArgs<R> ca{};
    ca.g = g;
    ca.mode = COL_FULL;
    ca.S = H->at<void>(R_S);
    ca.Wh = H->at<void>(R_WH);
    ca.rlo = 0;
    ca.rhi = g.P + 2;
    ca.tw = tw;
    PIDE_LAUNCH(PIDE2D_KERNEL_COL_FULL, launch_col<R>(ca, H->stream));
    InvArgs<R> ia{};
    ia.g = g;
    ia.mode = INV_FULL;
    ia.do_resid = 1;
    ia.S = H->at<void>(R_S);
    ia.BY = BY;
    ia.Y = Y;
    ia.W = W;
    ia.r = rres;
    ia.D = dlt;
    ia.htt = (R)htt;
    ia.cid = (R)(1.0 + htt * rw);
    ia.d11 = d11;
    ia.d22 = d22;
    ia.d12 = d12;
    ia.rw = (R)rw;
    ia.E = E;
    ia.tw = tw;
    PIDE_LAUNCH(PIDE2D_KERNEL_ROW_INVERSE_FULL, launch_row_inverse<R>(ia, H->stream));

    DstColArgs<R> da{};
    da.g = g;
    da.E = E;
    da.sin2 = H->at<R>(R_SIN2R);
    da.c0 = 1.0 + htt * rw;
    da.c1 = 2.0 * htt * a11 / (hg * hg);
    da.c2 = 2.0 * htt * a22 / (hg * hg);
    da.scale = (2.0 / N) * (2.0 / N);
    da.tw = tw;
    DstRowArgs<R> ra{};
    ra.g = g;
    ra.E = E;
    ra.Y = Y;
    ra.D = dlt;
    ra.resid = H->at<void>(R_RESID);
    ra.S = H->at<void>(R_S);
    ra.tw = tw;

    fa.mode = FWD_INCR;
    fa.pair0 = (N / 2 + 2) / 2;
    fa.npairs = N / 2;
    ca.mode = COL_INCR;
    ca.Wh = H->at<void>(R_WHI);
    ca.rlo = N / 2 + 2;
    ca.rhi = N / 2 + N + 2;
    ia.mode = INV_INCR;

    int k = 0;
    double resid = 0.0;
    bool conv = false;
    for (k = 1; k <= H->kmax; ++k) {
        PIDE_LAUNCH(PIDE2D_KERNEL_DST_COL, launch_dst_col<R>(da, H->stream));
        PIDE_CUDA(cudaMemsetAsync(H->at<void>(R_RESID), 0, 16, H->stream));
        PIDE_LAUNCH(PIDE2D_KERNEL_DST_ROW, launch_dst_row<R>(ra, H->stream));
        R rhost = 0;
        PIDE_CUDA(cudaMemcpyAsync(&rhost, H->at<void>(R_RESID), sizeof(R), cudaMemcpyDeviceToHost, H->stream));
        PIDE_CUDA(cudaStreamSynchronize(H->stream));
        resid = (double)rhost;
        conv = resid < H->tol;
        // B_w of the increment keeps B_w Y^{n,k} current (needed for the next W);
        // its row pass ran inside k_dst_row
        PIDE_LAUNCH(PIDE2D_KERNEL_COL_INCR, launch_col<R>(ca, H->stream));
        ia.do_resid = conv ? 0 : 1;
        PIDE_LAUNCH(PIDE2D_KERNEL_ROW_INVERSE_INCR, launch_row_inverse<R>(ia, H->stream));
        if (conv) break;
    }
    if (!conv) k = H->kmax;
    std::swap(H->bv, H->by);
    *iters_out = k;
    *resid_out = resid;
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
                                                  res, &k, &r);
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
        const pide2d_status s = theta_step<R>(H, H->hist.data(), cnt, H->theta, dt, (n - 1) * dt, n * dt, res, &k, &r);
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
    H->stats.fp_iters_total += ktot;
    if (ktot > H->stats.fp_iters_max) H->stats.fp_iters_max = ktot;
    H->stats.last_resid = r;
    if (iters) *iters = ktot;
    if (resid) *resid = r;
    return st;
}

template <typename R>
static pide2d_status do_create(pide2d* H) {
    const Geometry g = H->L.g;
    const int N = g.N;
    cudaStream_t s = H->stream;
    // quadrature nodes
    std::vector<double> gl(kGlTotal);
    double* p = gl.data();
    gauss_legendre(kGlNear, p, p + kGlNear);
    gauss_legendre(kGlFar, p + 2 * kGlNear, p + 2 * kGlNear + kGlFar);
    gauss_legendre(kGlEdge, p + 2 * (kGlNear + kGlFar), p + 2 * (kGlNear + kGlFar) + kGlEdge);
    gauss_legendre(kGlPay, p + 2 * (kGlNear + kGlFar + kGlEdge), p + 2 * (kGlNear + kGlFar + kGlEdge) + kGlPay);
    double* pv = p + 2 * (kGlNear + kGlFar + kGlEdge + kGlPay);
    gauss_legendre(kGlVfar, pv, pv + kGlVfar);
    double* dgl = H->at<double>(R_GL);
    PIDE_CUDA(cudaMemsetAsync(H->ws, 0, H->L.total, s));
    PIDE_CUDA(cudaMemcpyAsync(dgl, gl.data(), gl.size() * 8, cudaMemcpyHostToDevice, s));

    // tables
    PIDE_CUDA(launch_tables(N, H->s_lo1, H->s_lo2, H->h, H->at<double>(R_E1D), H->at<double>(R_E2D),
                            H->at<float>(R_E1F), H->at<float>(R_E2F), H->at<double>(R_SIN2D), s));
    PIDE_CUDA(launch_twiddles<R>(g.P, H->at<void>(R_TWR), s));
    PIDE_CUDA(launch_twiddles<double>(g.P, H->at<void>(R_TWD), s));

    // Levy density constants (Sec. 4)
    const pide2d_model& m = H->model;
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

    WeightJob j{};
    j.N = N;
    j.h = H->h;
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
    PIDE_CUDA(launch_weights(L, j, H->at<double>(R_OMEGA), H->at<double>(R_PART), &nblocks, s));
    const double* edge = dgl + 2 * (kGlNear + kGlFar);
    PIDE_CUDA(launch_moment(L, 2.0 * H->h, edge, edge + kGlEdge, kGlEdge, kTanhSinhStep, H->at<double>(R_MOMENT), s));
    PIDE_CUDA(launch_finalize(H->at<double>(R_PART), nblocks, H->at<double>(R_MOMENT), m.r, m.sigma_cov,
                              H->at<double>(R_PARAMS), s));

    // omega-hat = conj(fft2(Omega padded))/P^2 (eq. 3.13): FP64 row spectra in
    // the (not yet used) state-field region, then FP64 column FFTs
    Geometry gd = g;
    gd.rows = g.P;
    gd.ng = g.P / 2 + 1;
    FwdArgs<double> wa{};
    wa.g = gd;
    wa.mode = FWD_WEIGHTS;
    wa.omega = H->at<double>(R_OMEGA);
    wa.S = H->field(0);
    wa.pair0 = 0;
    wa.npairs = N / 2;
    wa.tw = H->at<void>(R_TWD);
    PIDE_CUDA(launch_row_forward<double>(wa, s));
    PIDE_CUDA(launch_weights_col<R>(gd, H->field(0), H->at<void>(R_WH), H->at<void>(R_WHI), H->at<void>(R_TWD), s));
    PIDE_CUDA(cudaMemsetAsync(H->field(0), 0, H->L.off[R_RES] - H->L.off[R_V0], s));

    PIDE_CUDA(cudaMemcpyAsync(H->par, H->at<double>(R_PARAMS), 9 * 8, cudaMemcpyDeviceToHost, s));
    // sin^2 table in the transform precision
    PIDE_CUDA(cudaStreamSynchronize(s));
    {
        std::vector<R> s2(N + 1);
        std::vector<double> s2d(N + 1);
        PIDE_CUDA(cudaMemcpy(s2d.data(), H->at<double>(R_SIN2D), (N + 1) * 8, cudaMemcpyDeviceToHost));
        for (int i = 0; i <= N; ++i) s2[i] = (R)s2d[i];
        PIDE_CUDA(cudaMemcpy(H->at<R>(R_SIN2R), s2.data(), (N + 1) * sizeof(R), cudaMemcpyHostToDevice));
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

pide2d_status pide2d_step(pide2d_t* H, int* fp_iters, double* fp_resid) {
    if (!H) return PIDE2D_ERR_ARG;
    if (H->broken) { H->err = "handle unusable after a CUDA error"; return PIDE2D_ERR_STATE; }
    if (H->steps_done >= H->n_steps) { H->err = "all time steps done"; return PIDE2D_ERR_STATE; }
    return H->grid.precision == PIDE2D_FP64 ? do_step<double>(H, fp_iters, fp_resid)
                                            : do_step<float>(H, fp_iters, fp_resid);
}

pide2d_status pide2d_solve(pide2d_t* H, double* price, double* values_out, pide2d_stats* stats) {
    if (!H) return PIDE2D_ERR_ARG;
    if (H->broken) { H->err = "handle unusable after a CUDA error"; return PIDE2D_ERR_STATE; }
    pide2d_status worst = PIDE2D_OK;
    while (H->steps_done < H->n_steps) {
        const pide2d_status s = pide2d_step(H, nullptr, nullptr);
        if (s == PIDE2D_ERR_CUDA || s == PIDE2D_ERR_STATE) return s;
        if (s != PIDE2D_OK) worst = s;
    }
    if (price) {
        const pide2d_status s = H->grid.precision == PIDE2D_FP64 ? do_price<double>(H, price) : do_price<float>(H, price);
        if (s != PIDE2D_OK) return s;
    }
    if (values_out) {
        const pide2d_status s = pide2d_get_values(H, values_out);
        if (s != PIDE2D_OK) return s;
    }
    if (stats) *stats = H->stats;
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
    delete H;
}

}  // extern "C"
