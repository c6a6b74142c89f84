// Kernels of the discrete adjoint of the time loop (Sec. 3 scheme, Algorithm 1).
//
// One theta step maps V^{s-1} to V^s by
//   W   = T_SL[Z],  Z = V^{s-1} + h_t (1-theta) ((D - r_w) V^{s-1} + B V^{s-1})   (eqs. 3.19-3.22)
//   (1 + h_t theta r_w) V^s - h_t theta D V^s - h_t theta B V^s = W                (eq. 3.23)
// with the far field g on the ring and the halo.  Going backwards, the
// adjoint variable lambda_s of V^s gives mu_s = A_s^{-T} lambda_s (solved by
// the forward machinery with the flipped weights, see pide2d_adjoint) and
//   nu_s = T_SL^T mu_s,   lambda_{s-1} = nu_s + h_t (1-theta) ((D - r_w) nu_s + B^T nu_s).
// The kernels here are the pieces that the forward path has no use for: the
// transposed departure interpolation, the combination above, and the FP64
// dot products that contract the adjoint fields with the derivatives of the
// operators (weights, diffusion coefficients, r_w and the departure shift).
// Dot products are written as per-block partial sums and added up by one
// block in a fixed order, so the gradient is reproducible bit for bit.
#include <cuda_runtime.h>

#include "internal.h"
#include "state.cuh"

namespace pide {

namespace {

constexpr int kBX = 32, kBY = 8;

__device__ __forceinline__ double dget(const float2* p, size_t i) { return st_dbl(p[i]); }
__device__ __forceinline__ double dget(const double* p, size_t i) { return p[i]; }

// D applied at interior index idx of a full node field (ring included), FP64
template <typename T>
__device__ __forceinline__ void stencil_parts(const T* V, size_t idx, int ld, double* dxx, double* dyy, double* dxy) {
    const double c = dget(V, idx);
    *dxx = dget(V, idx + 1) + dget(V, idx - 1) - 2.0 * c;
    *dyy = dget(V, idx + ld) + dget(V, idx - ld) - 2.0 * c;
    *dxy = (dget(V, idx + ld + 1) - dget(V, idx - ld + 1)) - (dget(V, idx + ld - 1) - dget(V, idx - ld - 1));
}

template <int ND>
__device__ __forceinline__ void block_partials(double (&v)[ND], double* part) {
    __shared__ double red[ND][kBX * kBY / 32];
    const int lane = (threadIdx.y * kBX + threadIdx.x) & 31;
    const int warp = (threadIdx.y * kBX + threadIdx.x) >> 5;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        double x = v[d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[d][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const int b = blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            double s = 0.0;
            for (int w = 0; w < kBX * kBY / 32; ++w) s += red[d][w];
            part[(size_t)b * ND + d] = s;
        }
    }
}

}  // namespace

__global__ void k_flip_weights(const double* om, double* out, int N) {
    const int i1 = blockIdx.x * blockDim.x + threadIdx.x;
    const int i2 = blockIdx.y * blockDim.y + threadIdx.y;
    if (i1 >= N || i2 >= N) return;
    out[(size_t)i2 * N + i1] = om[(size_t)(N - 1 - i2) * N + (N - 1 - i1)];
}

__global__ void k_central_difference(const double* a, const double* b, double s, double* out, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (a[i] - b[i]) * s;
}

// nu_j = sum_{b,c} w2_b w1_c mu[j2 - o2 - b][j1 - o1 - c] over interior mu; ring of nu = 0
template <typename R>
__global__ void k_sl_transpose(Geometry g, const St<R>* mu, St<R>* nu, int o1, int o2, int nt, SlWeights w) {
    const int N = g.N;
    const int j1 = blockIdx.x * blockDim.x + threadIdx.x;
    const int j2 = blockIdx.y * blockDim.y + threadIdx.y;
    if (j1 > N || j2 > N) return;
    const size_t idx = (size_t)j2 * g.ldS + j1;
    if (j1 == 0 || j2 == 0 || j1 == N || j2 == N) {
        nu[idx] = st_make<St<R>>(0.0);
        return;
    }
    double acc = 0.0;
    for (int b = 0; b < nt; ++b) {
        const int m2 = j2 - o2 - b;
        if (m2 < 1 || m2 > N - 1) continue;
        double row = 0.0;
        for (int c = 0; c < nt; ++c) {
            const int m1 = j1 - o1 - c;
            if (m1 < 1 || m1 > N - 1) continue;
            row += w.w1[c] * dget(mu, (size_t)m2 * g.ldS + m1);
        }
        acc += w.w2[b] * row;
    }
    nu[idx] = st_make<St<R>>(acc);
}

// lambda = nu + htm ((D - r_w) nu + B^T nu) at interior nodes (nu is zero on the ring)
template <typename R>
__global__ void k_adj_combine(Geometry g, const St<R>* nu, const double* bnu, St<R>* lam, double htm, double rw,
                              double d11, double d22, double d12) {
    const int N = g.N;
    const int m1 = blockIdx.x * blockDim.x + threadIdx.x;
    const int m2 = blockIdx.y * blockDim.y + threadIdx.y;
    if (m1 > N || m2 > N) return;
    const size_t idx = (size_t)m2 * g.ldS + m1;
    if (m1 == 0 || m2 == 0 || m1 == N || m2 == N) {
        lam[idx] = st_make<St<R>>(0.0);
        return;
    }
    double dxx, dyy, dxy;
    stencil_parts(nu, idx, g.ldS, &dxx, &dyy, &dxy);
    const double v = dget(nu, idx);
    lam[idx] = st_make<St<R>>(v + htm * (d11 * dxx + d22 * dyy + d12 * dxy - rw * v + bnu[idx]));
}

// xi = htt mu + pend;  pend = htm_s nu  (interior; FP64 fields of pitch ldS)
template <typename R>
__global__ void k_adj_xi(Geometry g, const St<R>* mu, const St<R>* nu, double* xi, double* pend, double htt,
                         double htm_s) {
    const int N = g.N;
    const int m1 = blockIdx.x * blockDim.x + threadIdx.x;
    const int m2 = blockIdx.y * blockDim.y + threadIdx.y;
    if (m1 > N || m2 > N) return;
    const size_t idx = (size_t)m2 * g.ldS + m1;
    if (m1 == 0 || m2 == 0 || m1 == N || m2 == N) {
        xi[idx] = 0.0;
        pend[idx] = 0.0;
        return;
    }
    xi[idx] = htt * dget(mu, idx) + pend[idx];
    pend[idx] = nu ? htm_s * dget(nu, idx) : 0.0;
}

// partial sums of <xi, V>, <xi, dxx V>, <xi, dxy V>, <xi, dyy V> over the interior
template <typename R>
__global__ void __launch_bounds__(kBX* kBY) k_dots_state(Geometry g, const double* xi, const St<R>* V, double* part) {
    const int N = g.N;
    const int m1 = blockIdx.x * blockDim.x + threadIdx.x;
    const int m2 = blockIdx.y * blockDim.y + threadIdx.y;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (m1 >= 1 && m2 >= 1 && m1 <= N - 1 && m2 <= N - 1) {
        const size_t idx = (size_t)m2 * g.ldS + m1;
        const double x = xi[idx];
        double dxx, dyy, dxy;
        stencil_parts(V, idx, g.ldS, &dxx, &dyy, &dxy);
        v[0] = x * dget(V, idx);
        v[1] = x * dxx;
        v[2] = x * dxy;
        v[3] = x * dyy;
    }
    block_partials<4>(v, part);
}

// partial sums of <xi, out> over the interior (out: FP64 field of pitch ldS)
__global__ void __launch_bounds__(kBX* kBY) k_dot_field(Geometry g, const double* xi, const double* out, double* part) {
    const int N = g.N;
    const int m1 = blockIdx.x * blockDim.x + threadIdx.x;
    const int m2 = blockIdx.y * blockDim.y + threadIdx.y;
    double v[1] = {0.0};
    if (m1 >= 1 && m2 >= 1 && m1 <= N - 1 && m2 <= N - 1) {
        const size_t idx = (size_t)m2 * g.ldS + m1;
        v[0] = xi[idx] * out[idx];
    }
    block_partials<1>(v, part);
}

// partial sums of <mu, dT_SL/dq_1 Zx> and <mu, dT_SL/dq_2 Zx>, with Zx = V + htm ((D - r_w) V + BV)
// at interior nodes and the far field g(s, tau_{s-1}) elsewhere (as in the forward W)
template <typename R>
__global__ void __launch_bounds__(kBX* kBY) k_sl_shift_dots(Geometry g, SlShiftArgs<R> a, double* part) {
    const int N = g.N;
    const int m1 = blockIdx.x * blockDim.x + threadIdx.x;
    const int m2 = blockIdx.y * blockDim.y + threadIdx.y;
    double v[2] = {0.0, 0.0};
    if (m1 >= 1 && m2 >= 1 && m1 <= N - 1 && m2 <= N - 1) {
        const int ld = g.ldS;
        double s1 = 0.0, s2 = 0.0;
        for (int b = 0; b < a.nt; ++b) {
            const int q2 = m2 + a.o2 + b;
            double r1 = 0.0, r2 = 0.0;
            for (int c = 0; c < a.nt; ++c) {
                const int q1 = m1 + a.o1 + c;
                double z;
                if (q1 >= 1 && q1 <= N - 1 && q2 >= 1 && q2 <= N - 1) {
                    const size_t qi = (size_t)q2 * ld + q1;
                    const double vq = dget(a.V, qi);
                    z = vq;
                    if (a.htm != 0.0) {
                        double dxx, dyy, dxy;
                        stencil_parts(a.V, qi, ld, &dxx, &dyy, &dxy);
                        z += a.htm * (a.d11 * dxx + a.d22 * dyy + a.d12 * dxy - a.rw * vq + dget(a.BV, qi));
                    }
                } else {
                    z = far_value<double>(a.payoff, a.Kd_prev, a.E1d[q1 + g.eoff], a.E2d[q2 + g.eoff]);
                }
                r1 += a.w.dw1[c] * z;
                r2 += a.w.w1[c] * z;
            }
            s1 += a.w.w2[b] * r1;
            s2 += a.w.dw2[b] * r2;
        }
        const double mu = dget(a.mu, (size_t)m2 * ld + m1);
        v[0] = mu * s1;
        v[1] = mu * s2;
    }
    block_partials<2>(v, part);
}

// dst (R field, pitch ldR) = src (FP64 field, pitch ldS) at the interior nodes
template <typename R>
__global__ void k_field_to_r(Geometry g, const double* src, R* dst) {
    const int m1 = blockIdx.x * blockDim.x + threadIdx.x;
    const int m2 = blockIdx.y * blockDim.y + threadIdx.y;
    if (m1 < 1 || m2 < 1 || m1 > g.N - 1 || m2 > g.N - 1) return;
    dst[(size_t)m2 * g.ldR + m1] = (R)src[(size_t)m2 * g.ldS + m1];
}

// per-block partial sums of a[i] b[i], i < n (grid-stride, a fixed number of blocks)
__global__ void k_dot_plain(const double* a, const double* b, size_t n, double* part) {
    __shared__ double red[256];
    double x = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x += a[i] * b[i];
    red[threadIdx.x] = x;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// acc[d] += scale * sum_b part[b][d], one block, fixed order
__global__ void k_reduce_add(const double* part, int nblocks, int nd, double* acc, double scale) {
    __shared__ double red[256];
    for (int d = 0; d < nd; ++d) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += part[(size_t)b * nd + d];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) acc[d] += scale * red[0];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
namespace {
dim3 node_grid(int N) { return dim3((N + 1 + kBX - 1) / kBX, (N + 1 + kBY - 1) / kBY); }
}  // namespace

int adjoint_dot_blocks(int N) {
    const dim3 gr = node_grid(N);
    return (int)(gr.x * gr.y);
}

cudaError_t launch_flip_weights(const double* om, double* out, int N, cudaStream_t s) {
    k_flip_weights<<<dim3((N + 31) / 32, (N + 7) / 8), dim3(32, 8), 0, s>>>(om, out, N);
    return cudaGetLastError();
}

cudaError_t launch_central_difference(const double* a, const double* b, double scale, double* out, size_t n,
                                      cudaStream_t s) {
    k_central_difference<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, b, scale, out, n);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_sl_transpose(const Geometry& g, const St<R>* mu, St<R>* nu, int o1, int o2, int nt,
                                const SlWeights& w, cudaStream_t s) {
    k_sl_transpose<R><<<node_grid(g.N), dim3(kBX, kBY), 0, s>>>(g, mu, nu, o1, o2, nt, w);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_adj_combine(const Geometry& g, const St<R>* nu, const double* bnu, St<R>* lam, double htm,
                               double rw, double d11, double d22, double d12, cudaStream_t s) {
    k_adj_combine<R><<<node_grid(g.N), dim3(kBX, kBY), 0, s>>>(g, nu, bnu, lam, htm, rw, d11, d22, d12);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_adj_xi(const Geometry& g, const St<R>* mu, const St<R>* nu, double* xi, double* pend, double htt,
                          double htm_s, cudaStream_t s) {
    k_adj_xi<R><<<node_grid(g.N), dim3(kBX, kBY), 0, s>>>(g, mu, nu, xi, pend, htt, htm_s);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_dots_state(const Geometry& g, const double* xi, const St<R>* V, double* part, double* acc,
                              double scale, cudaStream_t s) {
    const int nb = adjoint_dot_blocks(g.N);
    k_dots_state<R><<<node_grid(g.N), dim3(kBX, kBY), 0, s>>>(g, xi, V, part);
    k_reduce_add<<<1, 256, 0, s>>>(part, nb, 4, acc, scale);
    return cudaGetLastError();
}

cudaError_t launch_dot_field(const Geometry& g, const double* xi, const double* out, double* part, double* acc,
                             cudaStream_t s) {
    const int nb = adjoint_dot_blocks(g.N);
    k_dot_field<<<node_grid(g.N), dim3(kBX, kBY), 0, s>>>(g, xi, out, part);
    k_reduce_add<<<1, 256, 0, s>>>(part, nb, 1, acc, 1.0);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_field_to_r(const Geometry& g, const double* src, R* dst, cudaStream_t s) {
    k_field_to_r<R><<<node_grid(g.N), dim3(kBX, kBY), 0, s>>>(g, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_dot_plain(const Geometry& g, const double* a, const double* b, size_t n, double* part, double* acc,
                             cudaStream_t s) {
    const int nb = adjoint_dot_blocks(g.N);
    k_dot_plain<<<nb, 256, 0, s>>>(a, b, n, part);
    k_reduce_add<<<1, 256, 0, s>>>(part, nb, 1, acc, 1.0);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_sl_shift_dots(const Geometry& g, const SlShiftArgs<R>& a, double* part, double* acc, double scale,
                                 cudaStream_t s) {
    const int nb = adjoint_dot_blocks(g.N);
    k_sl_shift_dots<R><<<node_grid(g.N), dim3(kBX, kBY), 0, s>>>(g, a, part);
    k_reduce_add<<<1, 256, 0, s>>>(part, nb, 2, acc, scale);
    return cudaGetLastError();
}

#define PIDE_ADJ_INSTANTIATE(R)                                                                                   \
    template cudaError_t launch_sl_transpose<R>(const Geometry&, const St<R>*, St<R>*, int, int, int,             \
                                                const SlWeights&, cudaStream_t);                                   \
    template cudaError_t launch_adj_combine<R>(const Geometry&, const St<R>*, const double*, St<R>*, double,      \
                                               double, double, double, double, cudaStream_t);                      \
    template cudaError_t launch_adj_xi<R>(const Geometry&, const St<R>*, const St<R>*, double*, double*, double,  \
                                          double, cudaStream_t);                                                   \
    template cudaError_t launch_dots_state<R>(const Geometry&, const double*, const St<R>*, double*, double*,     \
                                              double, cudaStream_t);                                               \
    template cudaError_t launch_sl_shift_dots<R>(const Geometry&, const SlShiftArgs<R>&, double*, double*, double, \
                                                 cudaStream_t);                                                    \
    template cudaError_t launch_field_to_r<R>(const Geometry&, const double*, R*, cudaStream_t);
PIDE_ADJ_INSTANTIATE(float)
PIDE_ADJ_INSTANTIATE(double)
#undef PIDE_ADJ_INSTANTIATE

}  // namespace pide
