// T_out of the price-space jump operator (eq. 3.15): from the y_out lattice
// back to the non-uniform price grid, cubic Lagrange per axis (linear
// extrapolation below y_out is encoded in the tables as two taps).
#include <cuda_runtime.h>

#include <vector>

#include "internal.h"

namespace pide {

__global__ void k_ps_tout(int nx1, int nout, const int* __restrict__ t, const double* __restrict__ u,
                          const double* __restrict__ By, int ldB, double* __restrict__ out) {
    const int m1 = blockIdx.x * blockDim.x + threadIdx.x;
    const int m2 = blockIdx.y * blockDim.y + threadIdx.y;
    if (m1 >= nx1 || m2 >= nx1) return;
    const int a1 = t[m1], a2 = t[m2];
    double acc = 0.0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const double wb = u[m2 * 4 + b];
        if (wb == 0.0) continue;
        const double* row = By + (size_t)(a2 + b) * ldB + a1;
        double r = 0.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const double wc = u[m1 * 4 + c];
            if (wc != 0.0) r += wc * row[c];
        }
        acc += wb * r;
    }
    out[(size_t)m2 * nx1 + m1] = acc;
}

cudaError_t launch_ps_tout(int nx1, int nout, const int* t, const double* u, const double* By, int ldB, double* out,
                           cudaStream_t st) {
    (void)nout;
    const dim3 blk(32, 8), grd((nx1 + 31) / 32, (nx1 + 7) / 8);
    k_ps_tout<<<grd, blk, 0, st>>>(nx1, nout, t, u, By, ldB, out);
    return cudaGetLastError();
}

}  // namespace pide

// ---------------------------------------------------------------------------
// the price-space time loop (Sec. 3.3 on the paper's grid), FP64
// ---------------------------------------------------------------------------
namespace pide {

namespace {
constexpr int kBX = 32, kBY = 8;
__device__ __forceinline__ int clampi(int v, int hi) { return v < 0 ? 0 : (v > hi ? hi : v); }
}  // namespace

// D v (Sec. 3.2.1) at node (m1, m2): per-axis three-point coefficients a1 (first
// difference) and b2 (second difference), boundary rows encoded in the tables
__device__ __forceinline__ double ps_dv(const PsDiff& d, const double* v, int m1, int m2) {
    const int n = d.n1, N = n - 1;
    double d2x = 0.0, d2y = 0.0, mix = 0.0;
#pragma unroll
    for (int i = -1; i <= 1; ++i) {
        const int q1 = clampi(m1 + i, N), q2 = clampi(m2 + i, N);
        d2x += d.b2[m1 * 3 + i + 1] * v[(size_t)m2 * n + q1];
        d2y += d.b2[m2 * 3 + i + 1] * v[(size_t)q2 * n + m1];
        const double a2 = d.a1[m2 * 3 + i + 1];
        if (a2 != 0.0) {
#pragma unroll
            for (int j = -1; j <= 1; ++j) mix += a2 * d.a1[m1 * 3 + j + 1] * v[(size_t)q2 * n + clampi(m1 + j, N)];
        }
    }
    const double x1 = d.x[m1], x2 = d.x[m2];
    return 0.5 * d.A11 * x1 * x1 * d2x + d.A12 * x1 * x2 * mix + 0.5 * d.A22 * x2 * x2 * d2y;
}

// out = alpha v + beta D v + gamma w (w may be NULL)
__global__ void k_ps_diff(PsDiff d, const double* __restrict__ v, double alpha, double beta,
                          const double* __restrict__ w, double gamma, double* __restrict__ out) {
    const int m1 = blockIdx.x * blockDim.x + threadIdx.x, m2 = blockIdx.y * blockDim.y + threadIdx.y;
    if (m1 >= d.n1 || m2 >= d.n1) return;
    const size_t i = (size_t)m2 * d.n1 + m1;
    double r = alpha * v[i] + beta * ps_dv(d, v, m1, m2);
    if (w) r += gamma * w[i];
    out[i] = r;
}

// inverse of the diagonal of c0 I - c1 D (Jacobi preconditioner)
__global__ void k_ps_diag_inv(PsDiff d, double c0, double c1, double* __restrict__ dinv) {
    const int m1 = blockIdx.x * blockDim.x + threadIdx.x, m2 = blockIdx.y * blockDim.y + threadIdx.y;
    if (m1 >= d.n1 || m2 >= d.n1) return;
    const double x1 = d.x[m1], x2 = d.x[m2];
    const double dd = 0.5 * d.A11 * x1 * x1 * d.b2[m1 * 3 + 1] + d.A12 * x1 * x2 * d.a1[m2 * 3 + 1] * d.a1[m1 * 3 + 1] +
                      0.5 * d.A22 * x2 * x2 * d.b2[m2 * 3 + 1];
    dinv[(size_t)m2 * d.n1 + m1] = 1.0 / (c0 - c1 * dd);
}

// elementwise: out = a x + b y + c z (y, z may be NULL), or with dinv: out = dinv * (a x + b y)
// out may be one of x, y, z (each element is read before it is written): no __restrict__
__global__ void k_ps_axpy(size_t n, double a, const double* x, double b, const double* y, double c,
                          const double* z, const double* dinv, double* out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double r = a * x[i];
    if (y) r += b * y[i];
    if (z) r += c * z[i];
    if (dinv) r *= dinv[i];
    out[i] = r;
}

// up to three dot products <x_k, y_k> as per-block partials
__global__ void k_ps_dots(size_t n, int nd, PsDots dp, double* __restrict__ part) {
    __shared__ double red[3][256];
    double acc[3] = {0.0, 0.0, 0.0};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        for (int k = 0; k < nd; ++k) acc[k] += dp.x[k][i] * dp.y[k][i];
    for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) part[(size_t)blockIdx.x * 3 + k] = red[k][0];
}

__global__ void k_ps_maxrel(size_t n, const double* __restrict__ a, const double* __restrict__ b,
                            double* __restrict__ part) {
    __shared__ double red[256];
    double m = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(a[i] - b[i]) / fmax(1.0, fabs(a[i])));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// fixed-order sums (kind 0) or maxima (kind 1) of per-block partials into res[0..nd)
__global__ void k_ps_finish(const double* __restrict__ part, int nblocks, int nd, int kind, double* __restrict__ res) {
    __shared__ double red[256];
    for (int k = 0; k < nd; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
            const double v = part[(size_t)b * (kind ? 1 : 3) + k];
            s = kind ? fmax(s, v) : s + v;
        }
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] = kind ? fmax(red[threadIdx.x], red[threadIdx.x + o])
                                                              : red[threadIdx.x] + red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) res[k] = red[0];
        __syncthreads();
    }
}

constexpr int kPsRedBlocks = 304;      // 2 x 152 SMs

cudaError_t launch_ps_diff(const PsDiff& d, const double* v, double alpha, double beta, const double* w, double gamma,
                           double* out, cudaStream_t s) {
    const dim3 blk(kBX, kBY), grd((d.n1 + kBX - 1) / kBX, (d.n1 + kBY - 1) / kBY);
    k_ps_diff<<<grd, blk, 0, s>>>(d, v, alpha, beta, w, gamma, out);
    return cudaGetLastError();
}
cudaError_t launch_ps_diag_inv(const PsDiff& d, double c0, double c1, double* dinv, cudaStream_t s) {
    const dim3 blk(kBX, kBY), grd((d.n1 + kBX - 1) / kBX, (d.n1 + kBY - 1) / kBY);
    k_ps_diag_inv<<<grd, blk, 0, s>>>(d, c0, c1, dinv);
    return cudaGetLastError();
}
cudaError_t launch_ps_axpy(size_t n, double a, const double* x, double b, const double* y, double c, const double* z,
                           const double* dinv, double* out, cudaStream_t s) {
    k_ps_axpy<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, x, b, y, c, z, dinv, out);
    return cudaGetLastError();
}
int ps_reduction_blocks() { return kPsRedBlocks; }
cudaError_t launch_ps_dots(size_t n, int nd, const PsDots& dp, double* part, double* res, cudaStream_t s) {
    k_ps_dots<<<kPsRedBlocks, 256, 0, s>>>(n, nd, dp, part);
    k_ps_finish<<<1, 256, 0, s>>>(part, kPsRedBlocks, nd, 0, res);
    return cudaGetLastError();
}
// ---------------------------------------------------------------------------
// BiCGSTAB with the scalars on the device.  The vector updates read alpha,
// beta and omega from PsBicg; each scalar step is one thread; the loop is a
// CUDA-graph while-node whose condition the scalar steps set (no host round
// trip per iteration).  Same recurrences and reductions as a host-driven loop.
// ---------------------------------------------------------------------------
__global__ void k_bicg_init(const double* __restrict__ res, PsBicg* __restrict__ st, int maxit,
                            unsigned long long hnd) {
    PsBicg q{};
    const double bn = sqrt(res[0]);                   // res: <B, B>, <r, r>
    q.lim = 1e-13 * (bn > 0.0 ? bn : 1.0);
    q.rn = sqrt(res[1]);
    q.rho = 1.0;
    q.alpha = 1.0;
    q.omega = 1.0;
    q.rho_new = res[1];
    *st = q;
    cudaGraphSetConditional((cudaGraphConditionalHandle)hnd, (q.rn > q.lim && maxit > 0) ? 1u : 0u);
}
// p = r (first iteration) or r + beta p - beta omega v, beta = (rho_new / rho)(alpha / omega)
__global__ void k_bicg_p(size_t n, const PsBicg* __restrict__ st, const double* __restrict__ r, double* p,
                         const double* __restrict__ v) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const PsBicg q = *st;
    if (q.it == 0) {
        p[i] = r[i];
    } else {
        const double beta = (q.rho_new / q.rho) * (q.alpha / q.omega);
        p[i] = 1.0 * r[i] + beta * p[i] + (-beta * q.omega) * v[i];
    }
}
__global__ void k_bicg_alpha(const double* __restrict__ res, PsBicg* __restrict__ st) {
    st->alpha = st->rho_new / res[0];                 // res: <rh, v>
}
// s = r - alpha v
__global__ void k_bicg_s(size_t n, const PsBicg* __restrict__ st, const double* __restrict__ r,
                         const double* __restrict__ v, double* __restrict__ s) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    s[i] = 1.0 * r[i] + (-st->alpha) * v[i];
}
// res: <t, s>, <t, t>, <s, s>: converged on s (the loop ends), else omega
__global__ void k_bicg_omega(const double* __restrict__ res, PsBicg* __restrict__ st, unsigned long long hnd) {
    PsBicg q = *st;
    q.it += 1;
    const double sn = sqrt(res[2]);
    if (sn <= q.lim) {
        q.done = 1;
        q.rn = sn;
        cudaGraphSetConditional((cudaGraphConditionalHandle)hnd, 0u);
    } else {
        q.omega = res[0] / res[1];
    }
    *st = q;
}
// X += alpha y (+ omega z), r = s - omega t (unless converged on s)
__global__ void k_bicg_xr(size_t n, const PsBicg* __restrict__ st, double* X, const double* __restrict__ y,
                          const double* __restrict__ z, const double* __restrict__ s, const double* __restrict__ t,
                          double* __restrict__ r) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const PsBicg q = *st;
    if (q.done) {
        X[i] = 1.0 * X[i] + q.alpha * y[i];
    } else {
        X[i] = 1.0 * X[i] + q.alpha * y[i] + q.omega * z[i];
        r[i] = 1.0 * s[i] + (-q.omega) * t[i];
    }
}
// res: <r, r>, <rh, r>: the residual norm, the next rho and the loop condition
__global__ void k_bicg_rho(const double* __restrict__ res, PsBicg* __restrict__ st, int maxit,
                           unsigned long long hnd) {
    PsBicg q = *st;
    if (q.done) return;                               // the condition was cleared at convergence on s
    q.rho = q.rho_new;
    q.rn = sqrt(res[0]);
    q.rho_new = res[1];
    *st = q;
    cudaGraphSetConditional((cudaGraphConditionalHandle)hnd, (q.rn > q.lim && q.it < maxit) ? 1u : 0u);
}

cudaError_t record_ps_bicg(cudaGraph_t g, cudaStream_t cs, const PsBicgArgs& a, const char** where) {
    cudaError_t e = cudaSuccess;
#define PS_GTRY(call)                \
    do {                             \
        e = (call);                  \
        if (e != cudaSuccess) {      \
            *where = #call;          \
            return e;                \
        }                            \
    } while (0)
    const size_t n = a.n;
    const unsigned nb = (unsigned)((n + 255) / 256);
    cudaGraphConditionalHandle hnd;
    PS_GTRY(cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault));
    // set-up: r = B - (c0 X - c1 D X), rh = r, <B, B>, <r, r>, the stopping level
    PS_GTRY(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    {
        cudaError_t x = launch_ps_diff(a.d, a.X, a.c0, -a.c1, nullptr, 0.0, a.r, cs);
        if (x == cudaSuccess) x = launch_ps_axpy(n, 1.0, a.B, -1.0, a.r, 0.0, nullptr, nullptr, a.r, cs);
        if (x == cudaSuccess) x = cudaMemcpyAsync(a.rh, a.r, n * 8, cudaMemcpyDeviceToDevice, cs);
        if (x == cudaSuccess) x = launch_ps_dots(n, 2, PsDots{{a.B, a.r, nullptr}, {a.B, a.r, nullptr}}, a.part, a.res, cs);
        if (x == cudaSuccess) {
            k_bicg_init<<<1, 1, 0, cs>>>(a.res, a.st, a.maxit, (unsigned long long)hnd);
            x = cudaGetLastError();
        }
        cudaGraph_t got = nullptr;
        const cudaError_t x2 = cudaStreamEndCapture(cs, &got);
        if (x != cudaSuccess) { *where = "BiCGSTAB set-up launches"; return x; }
        if (x2 != cudaSuccess) { *where = "cudaStreamEndCapture(set-up)"; return x2; }
    }
    // the set-up is a chain: its last node has no dependents
    size_t nn = 0;
    PS_GTRY(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    PS_GTRY(cudaGraphGetNodes(g, nodes.data(), &nn));
    std::vector<cudaGraphNode_t> leaves;
    for (auto nd : nodes) {
        size_t nd_out = 0;
        PS_GTRY(cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &nd_out));
        if (nd_out == 0) leaves.push_back(nd);
    }
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hnd;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop = nullptr;
    PS_GTRY(cudaGraphAddNode(&loop, g, leaves.data(), nullptr, leaves.size(), &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    // one BiCGSTAB iteration
    PS_GTRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    {
        cudaError_t x = cudaSuccess;
        k_bicg_p<<<nb, 256, 0, cs>>>(n, a.st, a.r, a.p, a.v);
        x = cudaGetLastError();
        if (x == cudaSuccess) x = launch_ps_axpy(n, 1.0, a.p, 0.0, nullptr, 0.0, nullptr, a.dinv, a.y, cs);
        if (x == cudaSuccess) x = launch_ps_diff(a.d, a.y, a.c0, -a.c1, nullptr, 0.0, a.v, cs);
        if (x == cudaSuccess) x = launch_ps_dots(n, 1, PsDots{{a.rh, nullptr, nullptr}, {a.v, nullptr, nullptr}}, a.part, a.res, cs);
        if (x == cudaSuccess) {
            k_bicg_alpha<<<1, 1, 0, cs>>>(a.res, a.st);
            x = cudaGetLastError();
        }
        if (x == cudaSuccess) {
            k_bicg_s<<<nb, 256, 0, cs>>>(n, a.st, a.r, a.v, a.s);
            x = cudaGetLastError();
        }
        if (x == cudaSuccess) x = launch_ps_axpy(n, 1.0, a.s, 0.0, nullptr, 0.0, nullptr, a.dinv, a.z, cs);
        if (x == cudaSuccess) x = launch_ps_diff(a.d, a.z, a.c0, -a.c1, nullptr, 0.0, a.t, cs);
        if (x == cudaSuccess) x = launch_ps_dots(n, 3, PsDots{{a.t, a.t, a.s}, {a.s, a.t, a.s}}, a.part, a.res, cs);
        if (x == cudaSuccess) {
            k_bicg_omega<<<1, 1, 0, cs>>>(a.res, a.st, (unsigned long long)hnd);
            x = cudaGetLastError();
        }
        if (x == cudaSuccess) {
            k_bicg_xr<<<nb, 256, 0, cs>>>(n, a.st, a.X, a.y, a.z, a.s, a.t, a.r);
            x = cudaGetLastError();
        }
        if (x == cudaSuccess) x = launch_ps_dots(n, 2, PsDots{{a.r, a.rh, nullptr}, {a.r, a.r, nullptr}}, a.part, a.res, cs);
        if (x == cudaSuccess) {
            k_bicg_rho<<<1, 1, 0, cs>>>(a.res, a.st, a.maxit, (unsigned long long)hnd);
            x = cudaGetLastError();
        }
        cudaGraph_t got = nullptr;
        const cudaError_t x2 = cudaStreamEndCapture(cs, &got);
        if (x != cudaSuccess) { *where = "BiCGSTAB iteration launches"; return x; }
        if (x2 != cudaSuccess) { *where = "cudaStreamEndCapture(iteration)"; return x2; }
    }
#undef PS_GTRY
    return cudaSuccess;
}

cudaError_t launch_ps_maxrel(size_t n, const double* a, const double* b, double* part, double* res, cudaStream_t s) {
    k_ps_maxrel<<<kPsRedBlocks, 256, 0, s>>>(n, a, b, part);
    k_ps_finish<<<1, 256, 0, s>>>(part, kPsRedBlocks, 1, 1, res);
    return cudaGetLastError();
}

}  // namespace pide

namespace pide {

// W[m2][m1] = sum_{b,c} w2[m2][b] w1[m1][c] Z[s2[m2]+b][s1[m1]+c]: the departure interpolation T_SL
__global__ void k_ps_sl(int n1, const int* __restrict__ s1, const double* __restrict__ w1, const int* __restrict__ s2,
                        const double* __restrict__ w2, const double* __restrict__ Z, double* __restrict__ W) {
    const int m1 = blockIdx.x * blockDim.x + threadIdx.x, m2 = blockIdx.y * blockDim.y + threadIdx.y;
    if (m1 >= n1 || m2 >= n1) return;
    const int a1 = s1[m1], a2 = s2[m2];
    double acc = 0.0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const double* row = Z + (size_t)(a2 + b) * n1 + a1;
        double r = 0.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) r += w1[m1 * 4 + c] * row[c];
        acc += w2[m2 * 4 + b] * r;
    }
    W[(size_t)m2 * n1 + m1] = acc;
}

cudaError_t launch_ps_sl(int n1, const int* s1, const double* w1, const int* s2, const double* w2, const double* Z,
                         double* W, cudaStream_t s) {
    const dim3 blk(kBX, kBY), grd((n1 + kBX - 1) / kBX, (n1 + kBY - 1) / kBY);
    k_ps_sl<<<grd, blk, 0, s>>>(n1, s1, w1, s2, w2, Z, W);
    return cudaGetLastError();
}

}  // namespace pide
