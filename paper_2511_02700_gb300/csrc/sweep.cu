// Time-stepping kernels of pide2d: the jump sum B_w by zero-padded 2D FFT
// cross-correlation (eqs. 3.10-3.17), the diffusion solve by DST-I, and the
// semi-Lagrangian explicit part (Algorithm 1, steps 1-4).
//
// Data flow of one fixed-point iteration (all transforms length P = 2N):
//   k_row_forward  rows of T_in U (midpoints along s1), packed two real rows
//                  per complex FFT, R2C spectra -> S[group][row][c]
//   k_col          per spectrum column: midpoints along s2, forward FFT,
//                  product with conj(w^)/P^2, inverse FFT, keep rows 1..N
//   k_row_inverse  per row pair: C2R, B_w at the interior nodes, state and
//                  residual update, then the row DST-I of the residual -> E
//   k_dst_col      per column pair: DST-I, divide by the eigenvalues of the
//                  diffusion operator, DST-I back
//   k_dst_row      per row pair: DST-I back to nodes = increment, state
//                  update and the eq. 3.25 maximum
// DST-I of length N-1 is the imaginary part of the length-2N DFT of the
// odd extension, so every pass uses the same block FFT.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "state.cuh"

namespace pide {

namespace {

constexpr int kMaxThreads = 512;

inline int units_per_cta(int P) {
    const int nt = P / 16;
    const int u = 128 / nt;
    return u < 1 ? 1 : u;
}
__host__ __device__ inline int unit_len(int P) { return padded_len(P) + 4; }

template <typename R>
__device__ __forceinline__ R midpoint(const R* u, int i) {
    // cubic Lagrange at the midpoint of nodes i+1, i+2 from nodes i..i+3
    return R(-0.0625) * (u[i] + u[i + 3]) + R(0.5625) * (u[i + 1] + u[i + 2]);
}

template <typename R>
__device__ __forceinline__ R node_value(const FwdArgs<R>& a, int m1, int m2) {
    const int N = a.g.N;
    const bool in = (m1 >= 1 && m1 <= N - 1 && m2 >= 1 && m2 <= N - 1);
    if (a.mode == FWD_INCR) return in ? a.D[(size_t)m2 * a.g.ldR + m1] : R(0);
    if (in) return st_r(a.Y[(size_t)m2 * a.g.ldS + m1]);
    if (a.mode == FWD_FULL0) return R(0);
    return far_value<R>(a.payoff, a.Kd, a.E1[m1 + a.g.eoff], a.E2[m2 + a.g.eoff]);
}

// D applied to a state field at interior index idx (pitch ld)
template <typename S, typename R>
__device__ __forceinline__ R diff_state(const S* Y, size_t idx, int ld, R d11, R d22, R d12) {
    const S c = Y[idx];
    const R dxx = st_diff(Y[idx + 1], c) + st_diff(Y[idx - 1], c);
    const R dyy = st_diff(Y[idx + ld], c) + st_diff(Y[idx - ld], c);
    const R dxy = st_diff(Y[idx + ld + 1], Y[idx - ld + 1]) - st_diff(Y[idx + ld - 1], Y[idx - ld - 1]);
    return d11 * dxx + d22 * dyy + d12 * dxy;
}
template <typename R>
__device__ __forceinline__ R diff_plain(const R* D, size_t idx, int ld, R d11, R d22, R d12) {
    const R c = D[idx];
    const R dxx = D[idx + 1] + D[idx - 1] - R(2) * c;
    const R dyy = D[idx + ld] + D[idx - ld] - R(2) * c;
    const R dxy = (D[idx + ld + 1] - D[idx - ld + 1]) - (D[idx + ld - 1] - D[idx - ld - 1]);
    return d11 * dxx + d22 * dyy + d12 * dxy;
}

template <typename R> struct ResidAtomic;
template <> struct ResidAtomic<float> {
    static __device__ void max(void* p, float v) { atomicMax((unsigned int*)p, __float_as_uint(v)); }
};
template <> struct ResidAtomic<double> {
    static __device__ void max(void* p, double v) {
        atomicMax((unsigned long long*)p, (unsigned long long)__double_as_longlong(v));
    }
};

template <typename K>
void set_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// ---------------------------------------------------------------------------
// forward row pass
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kMaxThreads) k_row_forward(FwdArgs<R> a) {
    using C = cpx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = a.g.P, N = a.g.N, nt = P >> 4;
    const int unit = threadIdx.x / nt, t = threadIdx.x - unit * nt;
    C* buf = reinterpret_cast<C*>(smem_raw) + (size_t)unit * unit_len(P);
    R* nodes = reinterpret_cast<R*>(buf);
    const int p = blockIdx.x * (blockDim.x / nt) + unit;
    const bool valid = p < a.npairs;
    const int rho = 2 * (a.pair0 + p);
    C z[16];
    if (a.mode == FWD_WEIGHTS) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int i = t + q * nt;
            R wa = 0, wb = 0;
            if (valid && i < N) {
                if (rho < N) wa = (R)a.omega[(size_t)rho * N + i];
                if (rho + 1 < N) wb = (R)a.omega[(size_t)(rho + 1) * N + i];
            }
            z[q] = mk<R>(wa, wb);
        }
    } else {
        const int m2a = rho - N / 2 - 1;
        for (int idx = t; idx < P + 2; idx += nt) {
            const int m1 = idx - N / 2 - 1;
            nodes[idx] = valid ? node_value(a, m1, m2a) : R(0);
            nodes[P + 2 + idx] = valid ? node_value(a, m1, m2a + 1) : R(0);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int i = t + q * nt;
            R ua = 0, ub = 0;
            if (i <= P - 2) {
                ua = midpoint(nodes, i);
                ub = midpoint(nodes + P + 2, i);
            }
            z[q] = mk<R>(ua, ub);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) buf[padi(t + q * nt)] = z[q];
    __syncthreads();
    block_fft<R, -1>(buf, P, t, (const C*)a.tw);

    constexpr int Gc = cgroup<R>();
    C* S = (C*)a.S;
    const int rows = a.g.rows;
    for (int g = t; g < a.g.ng; g += nt) {
#pragma unroll
        for (int c = 0; c < Gc; ++c) {
            const int k = g * Gc + c;
            C xa = mk<R>(0, 0), xb = mk<R>(0, 0);
            if (k <= P / 2) {
                const C zk = buf[padi(k)];
                const C zm = buf[padi((P - k) & (P - 1))];
                xa = mk<R>(R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y - zm.y));
                xb = mk<R>(R(0.5) * (zk.y + zm.y), R(-0.5) * (zk.x - zm.x));
            }
            if (valid) {
                S[((size_t)g * rows + rho) * Gc + c] = xa;
                S[((size_t)g * rows + rho + 1) * Gc + c] = xb;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// column pass: midpoints along s2, FFT, spectral product, inverse FFT
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kMaxThreads) k_col(ColArgs<R> a) {
    using C = cpx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = a.g.P, N = a.g.N, nt = P >> 4;
    const int unit = threadIdx.x / nt, t = threadIdx.x - unit * nt;
    C* buf = reinterpret_cast<C*>(smem_raw) + (size_t)unit * unit_len(P);
    const int k1 = blockIdx.x * (blockDim.x / nt) + unit;
    const bool valid = k1 <= P / 2;
    constexpr int Gc = cgroup<R>();
    const int g = k1 / Gc, c = k1 - g * Gc;
    C* col = (C*)a.S + (size_t)g * a.g.rows * Gc + c;
    C z[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int i = t + q * nt;
        C v = mk<R>(0, 0);
        if (valid && i <= P - 2) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int rho = i + e;
                if (rho >= a.rlo && rho < a.rhi) {
                    const C x = col[(size_t)rho * Gc];
                    const R w = (e == 0 || e == 3) ? R(-0.0625) : R(0.5625);
                    v.x += w * x.x;
                    v.y += w * x.y;
                }
            }
        }
        z[q] = v;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) buf[padi(t + q * nt)] = z[q];
    __syncthreads();
    block_fft<R, -1>(buf, P, t, (const C*)a.tw);
    const C* wh = (const C*)a.Wh + (size_t)g * P * Gc + c;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int k2 = t + q * nt;
        const C w = valid ? wh[(size_t)k2 * Gc] : mk<R>(0, 0);
        buf[padi(k2)] = cmul(buf[padi(k2)], w);
    }
    __syncthreads();
    block_fft<R, +1>(buf, P, t, (const C*)a.tw);
    if (valid) {
        for (int m = 1 + t; m <= N; m += nt) col[(size_t)(m - 1) * Gc] = buf[padi(m)];
    }
}

// ---------------------------------------------------------------------------
// inverse row pass + state/residual update + row DST of the residual
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kMaxThreads) k_row_inverse(InvArgs<R> a) {
    using C = cpx<R>;
    using S_ = St<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = a.g.P, N = a.g.N, nt = P >> 4;
    const int unit = threadIdx.x / nt, t = threadIdx.x - unit * nt;
    C* buf = reinterpret_cast<C*>(smem_raw) + (size_t)unit * unit_len(P);
    const int p = blockIdx.x * (blockDim.x / nt) + unit;
    const int m2 = 2 * p + 1;
    const bool valid = m2 <= N - 1;
    const bool hasb = valid && (m2 + 1 <= N - 1);
    constexpr int Gc = cgroup<R>();
    const C* S = (const C*)a.S;
    const int rows = a.g.rows;
    for (int g = t; g < a.g.ng; g += nt) {
#pragma unroll
        for (int c = 0; c < Gc; ++c) {
            const int k = g * Gc + c;
            if (k > P / 2) continue;
            C xa = mk<R>(0, 0), xb = mk<R>(0, 0);
            if (valid) {
                xa = S[((size_t)g * rows + (m2 - 1)) * Gc + c];
                xb = S[((size_t)g * rows + m2) * Gc + c];
            }
            if (k == 0 || k == P / 2) { xa.y = 0; xb.y = 0; }
            buf[padi(k)] = mk<R>(xa.x - xb.y, xa.y + xb.x);
            if (k > 0 && k < P / 2) buf[padi(P - k)] = mk<R>(xa.x + xb.y, xb.x - xa.y);
        }
    }
    __syncthreads();
    block_fft<R, +1>(buf, P, t, (const C*)a.tw);

    const int ld = a.g.ldS, ldR = a.g.ldR;
    R ra[8], rb[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int m1 = t + q * nt;
        ra[q] = 0;
        rb[q] = 0;
        if (!valid || m1 < 1 || m1 > N - 1) continue;
        const C zz = buf[padi(m1)];
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            if (half == 1 && !hasb) break;
            const int row = m2 + half;
            const R zv = half == 0 ? zz.x : zz.y;
            const size_t idx = (size_t)row * ld + m1;
            const size_t idr = (size_t)row * ldR + m1;
            R rr = 0;
            if (a.mode == INV_OUT) {
                a.out[idx] = (double)zv;
            } else if (a.mode == INV_FULL) {
                a.BY[idx] = st_from_r<S_, R>(zv);
                if (a.do_resid) {
                    const S_ y = a.Y[idx];
                    rr = st_diff(a.W[idx], y) + a.htt * zv - a.htt * a.rw * st_r(y)
                         + a.htt * diff_state(a.Y, idx, ld, a.d11, a.d22, a.d12);
                }
            } else {  // INV_INCR
                a.BY[idx] = st_add(a.BY[idx], zv);
                if (a.do_resid) {
                    const R d = a.D[idr];
                    rr = a.r[idr] + a.htt * zv - (a.cid * d - a.htt * diff_plain(a.D, idr, ldR, a.d11, a.d22, a.d12));
                }
            }
            if (a.do_resid) a.r[idr] = rr;
            if (half == 0) ra[q] = rr; else rb[q] = rr;
        }
    }
    if (!a.do_resid) return;   // uniform across the block
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int m1 = t + q * nt;
        if (m1 == 0) {
            buf[padi(0)] = mk<R>(0, 0);
            buf[padi(N)] = mk<R>(0, 0);
        } else {
            buf[padi(m1)] = mk<R>(ra[q], rb[q]);
            buf[padi(P - m1)] = mk<R>(-ra[q], -rb[q]);
        }
    }
    __syncthreads();
    block_fft<R, -1>(buf, P, t, (const C*)a.tw);
    constexpr int GE = rgroup<R>();
    for (int gE = t; gE < a.g.nge; gE += nt) {
#pragma unroll
        for (int c = 0; c < GE; ++c) {
            const int k = gE * GE + c;
            const C zz = buf[padi(k)];
            const R va = k >= 1 ? R(-0.5) * zz.y : R(0);
            const R vb = k >= 1 ? R(0.5) * zz.x : R(0);
            if (valid) a.E[((size_t)gE * N + m2) * GE + c] = va;
            if (hasb) a.E[((size_t)gE * N + m2 + 1) * GE + c] = vb;
        }
    }
}

// ---------------------------------------------------------------------------
// column DST pass with the eigenvalue division
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kMaxThreads) k_dst_col(DstColArgs<R> a) {
    using C = cpx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = a.g.P, N = a.g.N, nt = P >> 4;
    const int unit = threadIdx.x / nt, t = threadIdx.x - unit * nt;
    C* buf = reinterpret_cast<C*>(smem_raw) + (size_t)unit * unit_len(P);
    const int u = blockIdx.x * (blockDim.x / nt) + unit;
    const int ka = 2 * u, kb = ka + 1;
    const bool valid = ka < N;
    constexpr int GE = rgroup<R>();
    const int gE = ka / GE, ca = ka - gE * GE, cb = ca + 1;
    R* col = a.E + (size_t)gE * N * GE;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int i = t + q * nt;
        const int j = i <= N ? i : P - i;
        const R sg = i <= N ? R(1) : R(-1);
        R xa = 0, xb = 0;
        if (valid && j >= 1 && j <= N - 1) {
            xa = sg * col[(size_t)j * GE + ca];
            xb = sg * col[(size_t)j * GE + cb];
        }
        buf[padi(i)] = mk<R>(xa, xb);
    }
    __syncthreads();
    block_fft<R, -1>(buf, P, t, (const C*)a.tw);
    R ta[8], tb[8];
    const R c0 = (R)a.c0, c1 = (R)a.c1, c2 = (R)a.c2, sc = (R)a.scale;
    const R sa = valid ? (R)a.sin2[ka] : R(0);
    const R sb = valid ? (R)a.sin2[kb] : R(0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int k2 = t + q * nt;
        const C zz = buf[padi(k2)];
        const R s2 = (R)a.sin2[k2];
        ta[q] = k2 >= 1 ? R(-0.5) * zz.y * sc / (c0 + c1 * sa + c2 * s2) : R(0);
        tb[q] = k2 >= 1 ? R(0.5) * zz.x * sc / (c0 + c1 * sb + c2 * s2) : R(0);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int k2 = t + q * nt;
        if (k2 == 0) {
            buf[padi(0)] = mk<R>(0, 0);
            buf[padi(N)] = mk<R>(0, 0);
        } else {
            buf[padi(k2)] = mk<R>(ta[q], tb[q]);
            buf[padi(P - k2)] = mk<R>(-ta[q], -tb[q]);
        }
    }
    __syncthreads();
    block_fft<R, -1>(buf, P, t, (const C*)a.tw);
    if (valid) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int m2 = t + q * nt;
            if (m2 < 1) continue;
            const C zz = buf[padi(m2)];
            col[(size_t)m2 * GE + ca] = R(-0.5) * zz.y;
            col[(size_t)m2 * GE + cb] = R(0.5) * zz.x;
        }
    }
}

// ---------------------------------------------------------------------------
// row DST back to nodes: increment, state update, eq. 3.25 maximum
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kMaxThreads) k_dst_row(DstRowArgs<R> a) {
    using C = cpx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = a.g.P, N = a.g.N, nt = P >> 4;
    const int units = blockDim.x / nt;
    const int unit = threadIdx.x / nt, t = threadIdx.x - unit * nt;
    C* buf = reinterpret_cast<C*>(smem_raw) + (size_t)unit * unit_len(P);
    R* red = reinterpret_cast<R*>(reinterpret_cast<C*>(smem_raw) + (size_t)units * unit_len(P));
    const int p = blockIdx.x * units + unit;
    const int m2 = 2 * p + 1;
    const bool valid = m2 <= N - 1;
    const bool hasb = valid && (m2 + 1 <= N - 1);
    constexpr int GE = rgroup<R>();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int i = t + q * nt;
        const int j = i <= N ? i : P - i;
        const R sg = i <= N ? R(1) : R(-1);
        R ea = 0, eb = 0;
        if (valid && j >= 1 && j <= N - 1) {
            const int gE = j / GE, c = j - gE * GE;
            ea = sg * a.E[((size_t)gE * N + m2) * GE + c];
            if (hasb) eb = sg * a.E[((size_t)gE * N + m2 + 1) * GE + c];
        }
        buf[padi(i)] = mk<R>(ea, eb);
    }
    __syncthreads();
    block_fft<R, -1>(buf, P, t, (const C*)a.tw);
    R rmax = 0;
    const int ld = a.g.ldS, ldR = a.g.ldR;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int m1 = t + q * nt;
        if (!valid || m1 < 1) continue;
        const C zz = buf[padi(m1)];
        const R da = R(-0.5) * zz.y, db = R(0.5) * zz.x;
        {
            const size_t idx = (size_t)m2 * ld + m1;
            const St<R> y = st_add(a.Y[idx], da);
            a.Y[idx] = y;
            a.D[(size_t)m2 * ldR + m1] = da;
            rmax = fmax(rmax, fabs(da) / fmax(R(1), fabs(st_r(y))));
        }
        if (hasb) {
            const size_t idx = (size_t)(m2 + 1) * ld + m1;
            const St<R> y = st_add(a.Y[idx], db);
            a.Y[idx] = y;
            a.D[(size_t)(m2 + 1) * ldR + m1] = db;
            rmax = fmax(rmax, fabs(db) / fmax(R(1), fabs(st_r(y))));
        }
    }
    // block maximum, one atomic per block
    for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
    if (lane == 0) red[warp] = rmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        R m = 0;
        for (int w = 0; w < nwarp; ++w) m = fmax(m, red[w]);
        ResidAtomic<R>::max(a.resid, m);
    }
}

// ---------------------------------------------------------------------------
// per-step preparation: W = T_SL[Z] (Algorithm 1 step 2), Y^{n,0} (eq. 3.26),
// far field on the boundary ring of Y
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ double far_dbl(const PrepArgs<R>& a, int q1, int q2, double Kd) {
    return (double)far_value<double>(a.payoff, Kd, a.E1d[q1 + a.g.eoff], a.E2d[q2 + a.g.eoff]);
}

template <typename R>
__device__ __forceinline__ R explicit_inc(const PrepArgs<R>& a, int q1, int q2) {
    // Z - V at an interior node: h_t (1-theta) (D V - r_w V + B V)
    if (a.htm == R(0)) return R(0);
    const int ld = a.g.ldS;
    const size_t idx = (size_t)q2 * ld + q1;
    const St<R>* V = a.V[0];
    return a.htm * (diff_state(V, idx, ld, a.d11, a.d22, a.d12) - a.rw * st_r(V[idx]) + st_r(a.BV[idx]));
}

template <typename R>
__global__ void k_prep(PrepArgs<R> a) {
    const int N = a.g.N;
    const int m1 = blockIdx.x * blockDim.x + threadIdx.x;
    const int m2 = blockIdx.y * blockDim.y + threadIdx.y;
    if (m1 > N || m2 > N) return;
    const int ld = a.g.ldS;
    const size_t idx = (size_t)m2 * ld + m1;
    using S_ = St<R>;
    if (m1 == 0 || m2 == 0 || m1 == N || m2 == N) {
        a.Y[idx] = st_make<S_>(far_dbl(a, m1, m2, a.Kd_now));
        return;
    }
    const S_* V = a.V[0];
    const S_ v = V[idx];
    const R czm = explicit_inc(a, m1, m2);
    R corr = czm;
    for (int b = 0; b < a.nt; ++b) {
        const int q2 = m2 + a.o2 + b;
        for (int c = 0; c < a.nt; ++c) {
            const int q1 = m1 + a.o1 + c;
            R dz;
            if (q1 >= 1 && q1 <= N - 1 && q2 >= 1 && q2 <= N - 1) {
                dz = st_diff(V[(size_t)q2 * ld + q1], v) + explicit_inc(a, q1, q2) - czm;
            } else {
                dz = (R)(far_dbl(a, q1, q2, a.Kd_prev) - st_dbl(v)) - czm;
            }
            corr += a.w1[c] * a.w2[b] * dz;
        }
    }
    a.W[idx] = st_add(v, corr);
    R e = 0;
    if (a.hcount == 2) {
        e = -st_diff(a.V[1][idx], v);
    } else if (a.hcount == 3) {
        e = R(-3) * st_diff(a.V[1][idx], v) + st_diff(a.V[2][idx], v);
    } else if (a.hcount >= 4) {
        e = R(-6) * st_diff(a.V[1][idx], v) + R(4) * st_diff(a.V[2][idx], v) - st_diff(a.V[3][idx], v);
    }
    a.Y[idx] = st_add(v, e);
}

// ---------------------------------------------------------------------------
// omega-hat: FP64 forward column FFT of the FP64 row spectra of Omega
// ---------------------------------------------------------------------------
template <typename RO>
__global__ void __launch_bounds__(kMaxThreads) k_weights_col(Geometry g, const double2* Sd, cpx<RO>* Wh,
                                                             const double2* twd) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = g.P, N = g.N, nt = P >> 4;
    const int unit = threadIdx.x / nt, t = threadIdx.x - unit * nt;
    double2* buf = reinterpret_cast<double2*>(smem_raw) + (size_t)unit * unit_len(P);
    const int k1 = blockIdx.x * (blockDim.x / nt) + unit;
    const bool valid = k1 <= P / 2;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int i = t + q * nt;
        double2 v = mk<double>(0, 0);
        if (valid && i < N) v = Sd[(size_t)k1 * P + i];   // rows >= N of the padded Omega are zero
        buf[padi(i)] = v;
    }
    __syncthreads();
    block_fft<double, -1>(buf, P, t, twd);
    if (!valid) return;
    constexpr int Go = cgroup<RO>();
    const int go = k1 / Go, co = k1 - go * Go;
    const double inv = 1.0 / ((double)P * (double)P);
    for (int k2 = t; k2 < P; k2 += nt) {
        const double2 w = buf[padi(k2)];
        Wh[((size_t)go * P + k2) * Go + co] = mk<RO>((RO)(w.x * inv), (RO)(-w.y * inv));
    }
}

template <typename R>
__global__ void k_state_from_double(Geometry g, const double* src, int lds, St<R>* dst) {
    const int m1 = blockIdx.x * blockDim.x + threadIdx.x, m2 = blockIdx.y * blockDim.y + threadIdx.y;
    if (m1 > g.N || m2 > g.N) return;
    dst[(size_t)m2 * g.ldS + m1] = st_make<St<R>>(src[(size_t)m2 * lds + m1]);
}
template <typename R>
__global__ void k_state_to_double(Geometry g, const St<R>* src, double* dst, int ldd) {
    const int m1 = blockIdx.x * blockDim.x + threadIdx.x, m2 = blockIdx.y * blockDim.y + threadIdx.y;
    if (m1 > g.N || m2 > g.N) return;
    dst[(size_t)m2 * ldd + m1] = st_dbl(src[(size_t)m2 * g.ldS + m1]);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename R>
cudaError_t launch_row_forward(const FwdArgs<R>& a, cudaStream_t s) {
    const int P = a.g.P, nt = P / 16, u = units_per_cta(P);
    const size_t smem = (size_t)u * unit_len(P) * sizeof(cpx<R>);
    set_smem(k_row_forward<R>, smem);
    const int blocks = (a.npairs + u - 1) / u;
    k_row_forward<R><<<blocks, u * nt, smem, s>>>(a);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_col(const ColArgs<R>& a, cudaStream_t s) {
    const int P = a.g.P, nt = P / 16, u = units_per_cta(P);
    const size_t smem = (size_t)u * unit_len(P) * sizeof(cpx<R>);
    set_smem(k_col<R>, smem);
    const int blocks = (P / 2 + 1 + u - 1) / u;
    k_col<R><<<blocks, u * nt, smem, s>>>(a);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_row_inverse(const InvArgs<R>& a, cudaStream_t s) {
    const int P = a.g.P, nt = P / 16, u = units_per_cta(P);
    const size_t smem = (size_t)u * unit_len(P) * sizeof(cpx<R>);
    set_smem(k_row_inverse<R>, smem);
    const int pairs = a.g.N / 2;
    k_row_inverse<R><<<(pairs + u - 1) / u, u * nt, smem, s>>>(a);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_dst_col(const DstColArgs<R>& a, cudaStream_t s) {
    const int P = a.g.P, nt = P / 16, u = units_per_cta(P);
    const size_t smem = (size_t)u * unit_len(P) * sizeof(cpx<R>);
    set_smem(k_dst_col<R>, smem);
    const int pairs = a.g.N / 2;
    k_dst_col<R><<<(pairs + u - 1) / u, u * nt, smem, s>>>(a);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_dst_row(const DstRowArgs<R>& a, cudaStream_t s) {
    const int P = a.g.P, nt = P / 16, u = units_per_cta(P);
    const size_t smem = (size_t)u * unit_len(P) * sizeof(cpx<R>) + 32 * sizeof(R);
    set_smem(k_dst_row<R>, smem);
    const int pairs = a.g.N / 2;
    k_dst_row<R><<<(pairs + u - 1) / u, u * nt, smem, s>>>(a);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_prep(const PrepArgs<R>& a, cudaStream_t s) {
    const dim3 blk(32, 8);
    const dim3 grd((a.g.N + 1 + 31) / 32, (a.g.N + 1 + 7) / 8);
    k_prep<R><<<grd, blk, 0, s>>>(a);
    return cudaGetLastError();
}
template <typename RO>
cudaError_t launch_weights_col(const Geometry& g, const void* Sd, void* Wh, const void* twd, cudaStream_t s) {
    const int P = g.P, nt = P / 16, u = units_per_cta(P);
    const size_t smem = (size_t)u * unit_len(P) * sizeof(double2);
    set_smem(k_weights_col<RO>, smem);
    const int blocks = (P / 2 + 1 + u - 1) / u;
    k_weights_col<RO><<<blocks, u * nt, smem, s>>>(g, (const double2*)Sd, (cpx<RO>*)Wh, (const double2*)twd);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_state_from_double(const Geometry& g, const double* src, int lds, St<R>* dst, cudaStream_t s) {
    const dim3 blk(32, 8), grd((g.N + 1 + 31) / 32, (g.N + 1 + 7) / 8);
    k_state_from_double<R><<<grd, blk, 0, s>>>(g, src, lds, dst);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_state_to_double(const Geometry& g, const St<R>* src, double* dst, int ldd, cudaStream_t s) {
    const dim3 blk(32, 8), grd((g.N + 1 + 31) / 32, (g.N + 1 + 7) / 8);
    k_state_to_double<R><<<grd, blk, 0, s>>>(g, src, dst, ldd);
    return cudaGetLastError();
}

#define PIDE_INSTANTIATE(R)                                                                         \
    template cudaError_t launch_row_forward<R>(const FwdArgs<R>&, cudaStream_t);                    \
    template cudaError_t launch_col<R>(const ColArgs<R>&, cudaStream_t);                            \
    template cudaError_t launch_row_inverse<R>(const InvArgs<R>&, cudaStream_t);                    \
    template cudaError_t launch_dst_col<R>(const DstColArgs<R>&, cudaStream_t);                     \
    template cudaError_t launch_dst_row<R>(const DstRowArgs<R>&, cudaStream_t);                     \
    template cudaError_t launch_prep<R>(const PrepArgs<R>&, cudaStream_t);                          \
    template cudaError_t launch_weights_col<R>(const Geometry&, const void*, void*, const void*,    \
                                               cudaStream_t);                                       \
    template cudaError_t launch_state_from_double<R>(const Geometry&, const double*, int, St<R>*,  \
                                                     cudaStream_t);                                 \
    template cudaError_t launch_state_to_double<R>(const Geometry&, const St<R>*, double*, int,    \
                                                   cudaStream_t);
PIDE_INSTANTIATE(float)
PIDE_INSTANTIATE(double)
#undef PIDE_INSTANTIATE

}  // namespace pide
