// Time-stepping kernels of pide2d (templates; instantiated per precision in
// sweep_f32.cu and sweep_f64.cu): the jump sum B_w by zero-padded 2D FFT
// cross-correlation (eqs. 3.10-3.17), the diffusion solve (row DST-I and
// tridiagonal column solves), and the
// semi-Lagrangian explicit part (Algorithm 1, steps 1-4).
//
// Data flow of one fixed-point iteration (all transforms length P = 2N):
//   k_row_forward  rows of T_in U (midpoints along s1), packed two real rows
//                  per complex FFT, R2C spectra -> S[group][row][c]
//   k_col          per spectrum column: midpoints along s2, forward FFT,
//                  product with conj(w^)/P^2, inverse FFT, keep rows 1..N
//   k_row_inverse  per row pair: C2R, B_w at the interior nodes, state and
//                  residual update, then the row DST-I of the residual -> E
//   k_col_solve    per column pair of row-DST modes: the tridiagonal solve of
//                  the diffusion operator along s2 (two block scans)
//   k_dst_row      per row pair: DST-I back to nodes = increment, state
//                  update and the eq. 3.25 maximum
// DST-I of length N-1 is the imaginary part of the length-2N DFT of the
// odd extension, so every transform uses the same block FFT.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "state.cuh"

namespace pide {

namespace {

// Launch shape of the FFT kernels for transform length P: FFT units of P/16
// threads, at least 128 threads per block; the register target (64 in FP32,
// 128 in FP64) fixes the minimum number of resident blocks per SM.
template <typename R, int P> struct Cfg {
    static constexpr int NT = P / 16;
    static constexpr int UNITS = NT >= 128 ? 1 : 128 / NT;
    static constexpr int THREADS = UNITS * NT;
    static constexpr int ULEN = padded_len(P) + 4;
    static constexpr int MINB = (sizeof(R) == 4 ? 1024 : 512) / THREADS;
    static constexpr size_t SMEM = (size_t)UNITS * ULEN * sizeof(cpx<R>);
    // multi-job kernels: launched with any number of units per block up to
    // MAXT threads (the batch picks it by timed trials), same register target
    static constexpr int MAXT = THREADS > 512 ? THREADS : 512;
    static constexpr int JMINB = (sizeof(R) == 4 ? 1024 : 512) / MAXT > 0 ? (sizeof(R) == 4 ? 1024 : 512) / MAXT : 1;
};

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
    if (a.mode == FWD_DIFF) {
        if (in) {
            const size_t idx = (size_t)m2 * a.g.ldS + m1;
            return st_diff(a.Y[idx], a.Yref[idx]);
        }
        return far_diff<R>(a.payoff, a.Kd, a.Kd_prev, a.dKd, a.E1[m1 + a.g.eoff], a.E2[m2 + a.g.eoff]);
    }
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
// The increment D of a fixed-point iteration solves M D = r(Y) exactly, M being
// (1 + h_t theta r_w) I minus h_t theta times the non-mixed part of D, which the
// DST-I inverts (eq. 3.24 with the mixed term lagged).  The residual of Y + D is
// then r(Y) + h_t theta B D - (M D - h_t theta a12 delta_12 D)
//     = h_t theta (B D + a12 delta_12 D):
// the B D of this sweep and the mixed difference of D, with no cancellation
// between r(Y) and M D.  (The residual is formed from the full operator at the
// start of every step, so rounding in the DST does not accumulate across steps.)
// The mixed difference of D at (row, x) is f(x + 1) - f(x - 1) with
// f(x) = D[row + 1][x] - D[row - 1][x] (dcol below).

// |d| / max(1, |y|) to select the node of a block's eq. 3.25 maximum: in FP32
// the fast division (2 ulp; max(1, |y|) stays far below 2^126), since the
// selected node is evaluated again in FP64; in FP64 the exact quotient
__device__ __forceinline__ float stop_ratio(float d, float y) { return __fdividef(fabsf(d), fmaxf(1.f, fabsf(y))); }
__device__ __forceinline__ double stop_ratio(double d, double y) { return fabs(d) / fmax(1.0, fabs(y)); }

// a warp's candidate for the eq. 3.25 maximum (shared-memory reduction slot)
struct StopCand {
    double q;      // its ratio in the transform precision (-1: no node)
    double d;      // its increment
    double y;      // its state value (FP64 of the stored state)
    int bad;       // a non-finite ratio or state was seen
    int pad;
};
__device__ __forceinline__ float2 shfl_xor_state(float2 y, int o) {
    return make_float2(__shfl_xor_sync(0xffffffffu, y.x, o), __shfl_xor_sync(0xffffffffu, y.y, o));
}
__device__ __forceinline__ double shfl_xor_state(double y, int o) { return __shfl_xor_sync(0xffffffffu, y, o); }
__device__ __forceinline__ float2 shfl_up_state(float2 y, int o) {
    return make_float2(__shfl_up_sync(0xffffffffu, y.x, o), __shfl_up_sync(0xffffffffu, y.y, o));
}
__device__ __forceinline__ double shfl_up_state(double y, int o) { return __shfl_up_sync(0xffffffffu, y, o); }
__device__ __forceinline__ float2 shfl_down_state(float2 y, int o) {
    return make_float2(__shfl_down_sync(0xffffffffu, y.x, o), __shfl_down_sync(0xffffffffu, y.y, o));
}
__device__ __forceinline__ double shfl_down_state(double y, int o) { return __shfl_down_sync(0xffffffffu, y, o); }

template <typename K>
void set_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

#define PIDE_FFT_KERNEL(R, P) __global__ void __launch_bounds__(Cfg<R, P>::THREADS, Cfg<R, P>::MINB)
#define PIDE_FFT_JOBS_KERNEL(R, P) __global__ void __launch_bounds__(Cfg<R, P>::MAXT, Cfg<R, P>::JMINB)

// Split the packed transform of two real rows in buf (natural order) into the
// two rows' spectra (Hermitian symmetry) and write them as spectrum rows rho and
// rho + 1 of S [group][row][c].  In FP32 a group's two columns of one row are 16
// contiguous bytes, written with one store.
template <typename R, int P>
__device__ __forceinline__ void store_spectrum_rows(const cpx<R>* buf, cpx<R>* S, int rows, int ng, int rho, int t,
                                                    bool valid) {
    using C = cpx<R>;
    constexpr int NT = P / 16;
    constexpr int Gc = cgroup<R>();
    auto split = [&](int k, C& xa, C& xb) {
        xa = mk<R>(0, 0);
        xb = mk<R>(0, 0);
        if (k <= P / 2) {
            const C zk = buf[padi(k)];
            const C zm = buf[padi((P - k) & (P - 1))];
            xa = mk<R>(R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y - zm.y));
            xb = mk<R>(R(0.5) * (zk.y + zm.y), R(-0.5) * (zk.x - zm.x));
        }
    };
    for (int g = t; g < ng; g += NT) {
        if constexpr (sizeof(R) == 4 && Gc == 2) {
            C a0, b0, a1, b1;
            split(2 * g, a0, b0);
            split(2 * g + 1, a1, b1);
            if (valid) {
                float4* row = reinterpret_cast<float4*>(S + ((size_t)g * rows + rho) * Gc);
                row[0] = make_float4(a0.x, a0.y, a1.x, a1.y);
                row[1] = make_float4(b0.x, b0.y, b1.x, b1.y);
            }
        } else {
#pragma unroll
            for (int c = 0; c < Gc; ++c) {
                C xa, xb;
                split(g * Gc + c, xa, xb);
                if (valid) {
                    S[((size_t)g * rows + rho) * Gc + c] = xa;
                    S[((size_t)g * rows + rho + 1) * Gc + c] = xb;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// forward row pass: T_in along s1 (from staged nodes) + packed R2C
// ---------------------------------------------------------------------------
template <typename R, int P>
__device__ __forceinline__ void row_forward_body(const FwdArgs<R>& a, int upb) {
    using C = cpx<R>;
    using CF = Cfg<R, P>;
    constexpr int NT = CF::NT, N = P / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int unit = threadIdx.x / NT, t = threadIdx.x - unit * NT;
    C* buf = reinterpret_cast<C*>(smem_raw) + (size_t)unit * CF::ULEN;
    R* nodes = reinterpret_cast<R*>(buf);
    const int p = blockIdx.x * upb + unit;
    const bool valid = p < a.npairs;
    const int rho = 2 * (a.pair0 + p);
    const C* tw = (const C*)a.tw;
    if (a.mode == FWD_WEIGHTS) {
        auto load = [&](int i) -> C {
            R wa = 0, wb = 0;
            if (valid && i < N) {
                if (rho < N) wa = (R)a.omega[(size_t)rho * N + i];
                if (rho + 1 < N) wb = (R)a.omega[(size_t)(rho + 1) * N + i];
            }
            return mk<R>(wa, wb);
        };
        block_fft<R, -1, P>(buf, t, tw, load, SmemStore<R>{buf});
    } else if (a.mode == FWD_INCR) {
        // raw increment rows at positions p = m1 + N/2 + 1; the cubic midpoint
        // interpolation along s1 is a factor of the increment weight spectrum
        const int m2a = rho - N / 2 - 1;
        const R* ra = a.D + (size_t)m2a * a.g.ldR;
        const bool va = valid && m2a >= 1 && m2a <= N - 1;
        const bool vb = valid && m2a + 1 >= 1 && m2a + 1 <= N - 1;
        auto load = [&](int i) -> C {
            const int m1 = i - N / 2 - 1;
            if (m1 < 1 || m1 > N - 1) return mk<R>(0, 0);
            return mk<R>(va ? ra[m1] : R(0), vb ? ra[a.g.ldR + m1] : R(0));
        };
        block_fft<R, -1, P>(buf, t, tw, load, SmemStore<R>{buf});
    } else {
        const int m2a = rho - N / 2 - 1;
        const bool ina = valid && m2a >= 1 && m2a <= N - 1;          // row m2a has interior nodes
        const bool inb = valid && m2a + 1 >= 1 && m2a + 1 <= N - 1;
        // far-field (halo) positions first: no state loads; a compile-time trip
        // count lets the loop unroll
#pragma unroll
        for (int q = 0; q < (P + 2 + NT - 1) / NT; ++q) {
            const int idx = t + q * NT;
            if (idx < P + 2) {
                const int m1 = idx - N / 2 - 1;
                const bool colin = m1 >= 1 && m1 <= N - 1;
                if (!(ina && colin)) nodes[idx] = valid ? node_value(a, m1, m2a) : R(0);
                if (!(inb && colin)) nodes[P + 2 + idx] = valid ? node_value(a, m1, m2a + 1) : R(0);
            }
        }
        // interior positions m1 = 1 + t + NT b: the state loads of four columns of
        // both rows go out together
        const St<R>* Ya = a.Y + (size_t)m2a * a.g.ldS;
        const St<R>* Ra = a.mode == FWD_DIFF ? a.Yref + (size_t)m2a * a.g.ldS : nullptr;
        const int ldS = a.g.ldS;
#pragma unroll
        for (int b0 = 0; b0 < N / NT; b0 += 4) {
            St<R> ya[4], yb[4], za[4], zb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int m1 = 1 + t + NT * (b0 + i);
                const bool ok = m1 <= N - 1;
                const St<R> zero = st_from_r<St<R>, R>(R(0));
                ya[i] = (ina && ok) ? Ya[m1] : zero;
                yb[i] = (inb && ok) ? Ya[ldS + m1] : zero;
                za[i] = (Ra && ina && ok) ? Ra[m1] : zero;
                zb[i] = (Ra && inb && ok) ? Ra[ldS + m1] : zero;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int m1 = 1 + t + NT * (b0 + i);
                if (m1 > N - 1) continue;
                const int idx = m1 + N / 2 + 1;
                if (ina) nodes[idx] = Ra ? st_diff(ya[i], za[i]) : st_r(ya[i]);
                if (inb) nodes[P + 2 + idx] = Ra ? st_diff(yb[i], zb[i]) : st_r(yb[i]);
            }
        }
        __syncthreads();
        auto load = [&](int i) -> C {
            if (i > P - 2) return mk<R>(0, 0);
            return mk<R>(midpoint(nodes, i), midpoint(nodes + P + 2, i));
        };
        block_fft<R, -1, P>(buf, t, tw, load, SmemStore<R>{buf});
    }
    store_spectrum_rows<R, P>(buf, (C*)a.S, a.g.rows, a.g.ng, rho, t, valid);
}
template <typename R, int P>
PIDE_FFT_KERNEL(R, P) k_row_forward(const __grid_constant__ FwdArgs<R> a) { row_forward_body<R, P>(a, Cfg<R, P>::UNITS); }
template <typename R, int P>
PIDE_FFT_JOBS_KERNEL(R, P) k_row_forward_jobs(const FwdArgs<R>* __restrict__ arr, JobsCtl jc) {
    if (jc.skip(blockIdx.y)) return;
    row_forward_body<R, P>(arr[blockIdx.y], blockDim.x / Cfg<R, P>::NT);
}

// ---------------------------------------------------------------------------
// column pass: staged column, T_in along s2 in the first stage, product with
// conj(w^)/P^2 in the last forward stage, inverse FFT writing rows 1..N
// ---------------------------------------------------------------------------
// loader of an increment column: rows rlo..rhi-1 of the column group (zero elsewhere)
template <typename R, int P>
struct IncrColLoad {
    static constexpr unsigned zero_mask = P >= 32 ? 0xE00Fu : 0u;   // r in {0..3, 13..15}
    const cpx<R>* col;
    int rlo, rhi;
    bool valid;
    __device__ __forceinline__ cpx<R> operator()(int rho) const {
        return (valid && rho >= rlo && rho < rhi) ? col[(size_t)rho * cgroup<R>()] : mk<R>(0, 0);
    }
};

// INCR: compiled for COL_INCR only, else for COL_FULL (each with its own register allocation)
template <typename R, int P, bool INCR>
__device__ __forceinline__ void col_body(const ColArgs<R>& a, int upb) {
    using C = cpx<R>;
    using CF = Cfg<R, P>;
    constexpr int NT = CF::NT, N = P / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int unit = threadIdx.x / NT, t = threadIdx.x - unit * NT;
    C* buf = reinterpret_cast<C*>(smem_raw) + (size_t)unit * CF::ULEN;
    const int k1 = blockIdx.x * upb + unit;
    const bool valid = k1 <= P / 2;
    constexpr int Gc = cgroup<R>();
    const int g = k1 / Gc, c = k1 - g * Gc;
    C* col = (C*)a.S + (size_t)g * a.g.rows * Gc + c;
    const C* tw = (const C*)a.tw;
    // the weight spectrum is column-major (column k1 at Wh + k1 P): the block's
    // column is contiguous, and comes into L2 while the forward transform runs
    const C* wh = (const C*)a.Wh + (size_t)k1 * P;
    if (t == 0 && valid) l2_prefetch(wh, (size_t)P * sizeof(C));
    // look ahead: the column a block resident one wave later (MINB blocks on each
    // of 152 SMs) will transform; its group's input rows come into L2 now, a
    // quarter from each of the group's blocks
    if (t == 0) {
        const int kn = k1 + CF::MINB * 152;
        if (kn <= P / 2 && a.rhi > a.rlo) {
            const int gn = kn / Gc, cn = kn - gn * Gc, len = a.rhi - a.rlo;
            const int r0 = a.rlo + (cn * len) / Gc, r1 = a.rlo + ((cn + 1) * len) / Gc;
            l2_prefetch((const C*)a.S + ((size_t)gn * a.g.rows + r0) * Gc, (size_t)(r1 - r0) * Gc * sizeof(C));
        }
    }
    auto store_mul = [&](int k2, C v) {
        const C w = valid ? __ldg(&wh[k2]) : mk<R>(0, 0);
        buf[padi(k2)] = cmul(v, w);
    };
    if constexpr (INCR) {
        // raw rows; the midpoint interpolation along s2 is in the weight spectrum.
        // Rows outside [N/2 + 2, 3N/2 + 2) are zero, so first-stage inputs
        // j + r P/16 with r in {0..3, 13..15} always are (P >= 32)
        block_fft<R, -1, P>(buf, t, tw, IncrColLoad<R, P>{col, a.rlo, a.rhi, valid}, store_mul);
    } else {
        // (constant trip count with a guard: the loop unrolls and its loads go out together)
#pragma unroll
        for (int q = 0; q < (P + 2 + NT - 1) / NT; ++q) {
            const int rho = t + q * NT;
            if (rho < P + 2)
                buf[padi(rho)] = (valid && rho >= a.rlo && rho < a.rhi) ? col[(size_t)rho * Gc] : mk<R>(0, 0);
        }
        __syncthreads();
        auto load = [&](int i) -> C {
            if (i > P - 2) return mk<R>(0, 0);
            const C x0 = buf[padi(i)], x1 = buf[padi(i + 1)], x2 = buf[padi(i + 2)], x3 = buf[padi(i + 3)];
            return mk<R>(R(-0.0625) * (x0.x + x3.x) + R(0.5625) * (x1.x + x2.x),
                         R(-0.0625) * (x0.y + x3.y) + R(0.5625) * (x1.y + x2.y));
        };
        block_fft<R, -1, P>(buf, t, tw, load, store_mul);
    }
    auto store_out = [&](int m, C v) {
        if (valid && m >= 1 && m <= N) col[(size_t)(m - 1) * Gc] = v;
    };
    block_fft<R, +1, P>(buf, t, tw, SmemLoad<R>{buf}, store_out);
}
template <typename R, int P, bool INCR>
PIDE_FFT_KERNEL(R, P) k_col(const __grid_constant__ ColArgs<R> a) { col_body<R, P, INCR>(a, Cfg<R, P>::UNITS); }
template <typename R, int P, bool INCR>
PIDE_FFT_JOBS_KERNEL(R, P) k_col_jobs(const ColArgs<R>* __restrict__ arr, JobsCtl jc) {
    if (jc.skip(blockIdx.y)) return;
    col_body<R, P, INCR>(arr[blockIdx.y], blockDim.x / Cfg<R, P>::NT);
}

// ---------------------------------------------------------------------------
// inverse row pass: Hermitian-extended packed spectrum in the first stage,
// B_w at the interior nodes + state/residual update in the last stage, which
// also lays out the odd extension of the residual for the row DST
// ---------------------------------------------------------------------------
// L2 prefetch of the field rows the inverse row pass's epilogue reads for
// rows m2 (and m2 + 1): they arrive while the transform runs
template <typename R>
__device__ __forceinline__ void prefetch_inverse_rows(const InvArgs<R>& a, const St<R>* BYv, int m2, bool hasb,
                                                      bool do_resid) {
    using S_ = St<R>;
    const int N = a.g.N, ld = a.g.ldS, ldR = a.g.ldR;
    const int nr = hasb ? 2 : 1;
    const int lo = m2 - 1, hi = m2 + 2 < N ? m2 + 2 : N;     // stencil rows, inside the N + 1 rows
    if (a.mode == INV_INCR) {
        l2_prefetch(BYv + (size_t)m2 * ld, (size_t)nr * ld * sizeof(S_));
        if (do_resid) l2_prefetch(a.D + (size_t)lo * ldR, (size_t)(hi - lo + 1) * ldR * sizeof(R));
    } else if (a.mode == INV_FULL && do_resid) {
        l2_prefetch(a.W + (size_t)m2 * ld, (size_t)nr * ld * sizeof(S_));
        l2_prefetch(a.Y + (size_t)lo * ld, (size_t)(hi - lo + 1) * ld * sizeof(S_));
        if (a.BV) l2_prefetch(a.BV + (size_t)m2 * ld, (size_t)nr * ld * sizeof(S_));
    }
}

// f(x) = D[row + 1][x] - D[row - 1][x] at column x (the mixed difference of an
// increment at (row, x +- 1) is f(x + 1) - f(x - 1))
template <typename R>
__device__ __forceinline__ R dcol(const R* D, int ldR, int row, int x) {
    const R* c = D + (size_t)row * ldR + x;
    return c[ldR] - c[-ldR];
}

// Epilogue of the increment inverse row pass in coalesced order: outputs
// m1 = t + NT b (b = 0..7) of rows m2 and m2 + 1, their C2R values in buf.
// B_w Y += zz; the residual h_t theta (zz + a12 d12 D) of the increment
// identity goes to buf as the odd extension for the row DST.  The loads of
// four outputs are issued together, and the neighbours x -+ 1 of the mixed
// difference come from the adjacent lanes (direct loads at warp edges).
template <typename R, int P>
__device__ __forceinline__ void incr_epilogue(const InvArgs<R>& a, St<R>* BYv, cpx<R>* buf, int t, int m2, bool valid,
                                              bool hasb, bool do_resid) {
    using C = cpx<R>;
    using S_ = St<R>;
    constexpr int NT = P / 16, N = P / 2, NB = N / NT;
    constexpr bool SHFL = NT >= 32;
    constexpr int EB = 4;             // outputs whose loads go out together
    const int ld = a.g.ldS, ldR = a.g.ldR;
    const int lane = threadIdx.x & 31;
    const S_ zero = st_from_r<S_, R>(R(0));
#pragma unroll
    for (int b0 = 0; b0 < NB; b0 += EB) {
        S_ ya[EB], yb[EB];
        R fa[EB], fb[EB];
#pragma unroll
        for (int i = 0; i < EB; ++i) {
            const int m1 = t + NT * (b0 + i);
            const size_t idx = (size_t)m2 * ld + m1;
            ya[i] = valid ? BYv[idx] : zero;
            yb[i] = hasb ? BYv[idx + ld] : zero;
            fa[i] = (do_resid && valid) ? dcol(a.D, ldR, m2, m1) : R(0);
            fb[i] = (do_resid && hasb) ? dcol(a.D, ldR, m2 + 1, m1) : R(0);
        }
#pragma unroll
        for (int i = 0; i < EB; ++i) {
            const int m1 = t + NT * (b0 + i);
            R fal, far_, fbl, fbr;
            if constexpr (SHFL) {
                fal = __shfl_up_sync(0xffffffffu, fa[i], 1);
                far_ = __shfl_down_sync(0xffffffffu, fa[i], 1);
                fbl = __shfl_up_sync(0xffffffffu, fb[i], 1);
                fbr = __shfl_down_sync(0xffffffffu, fb[i], 1);
                if (lane == 0 && m1 >= 1 && do_resid) {
                    fal = valid ? dcol(a.D, ldR, m2, m1 - 1) : R(0);
                    fbl = hasb ? dcol(a.D, ldR, m2 + 1, m1 - 1) : R(0);
                }
                if (lane == 31 && do_resid) {
                    far_ = valid ? dcol(a.D, ldR, m2, m1 + 1) : R(0);
                    fbr = hasb ? dcol(a.D, ldR, m2 + 1, m1 + 1) : R(0);
                }
            } else {
                const bool in = do_resid && m1 >= 1;
                fal = (in && valid) ? dcol(a.D, ldR, m2, m1 - 1) : R(0);
                far_ = (in && valid) ? dcol(a.D, ldR, m2, m1 + 1) : R(0);
                fbl = (in && hasb) ? dcol(a.D, ldR, m2 + 1, m1 - 1) : R(0);
                fbr = (in && hasb) ? dcol(a.D, ldR, m2 + 1, m1 + 1) : R(0);
            }
            if (m1 < 1) continue;
            R rra = R(0), rrb = R(0);
            if (valid) {
                const size_t idx = (size_t)m2 * ld + m1;
                const C zz = buf[padi(m1)];
                const R zva = zz.x, zvb = zz.y;
                BYv[idx] = st_add(ya[i], zva);
                if (do_resid) rra = a.htt * (zva + a.d12 * (far_ - fal));
                if (hasb) {
                    BYv[idx + ld] = st_add(yb[i], zvb);
                    if (do_resid) rrb = a.htt * (zvb + a.d12 * (fbr - fbl));
                }
            }
            if (do_resid) {
                buf[padi(m1)] = mk<R>(rra, rrb);
                buf[padi(P - m1)] = mk<R>(-rra, -rrb);
            }
        }
    }
}

// Epilogue of the full inverse row pass (INV_FULL, INV_OUT) in coalesced order:
// outputs m1 = t + NT b of rows m2 and m2 + 1, their C2R values zz in buf.
// INV_OUT writes zz.  INV_FULL sets B_w Y (= B_w V^{n-1} + zz after a difference
// sweep, else zz) and forms the step's first residual with the full operator,
//     W - Y + h_t theta (B_w Y - r_w Y) + h_t theta D Y,
// as the odd extension for the row DST.  Each column's four state rows
// m2 - 1 .. m2 + 2 are loaded once; the stencil's neighbours m1 -+ 1 (the
// states of rows m2, m2 + 1 and the vertical differences of the mixed term)
// come from the adjacent lanes, with direct loads at the warp edges.
template <typename R, int P>
__device__ __forceinline__ void full_epilogue(const InvArgs<R>& a, St<R>* BYv, cpx<R>* buf, int t, int m2,
                                              bool valid, bool hasb, bool do_resid) {
    using C = cpx<R>;
    using S_ = St<R>;
    constexpr int NT = P / 16, N = P / 2, NB = N / NT;
    constexpr bool SHFL = NT >= 32;
    constexpr int EB = 1;             // outputs whose loads go out together
    const int ld = a.g.ldS;
    const int lane = threadIdx.x & 31;
    const S_ zero = st_from_r<S_, R>(R(0));
    const bool full = a.mode == INV_FULL;
    const bool stencil = full && do_resid;
    const S_* Y = a.Y;
    // the column at m1 of rows m2 - 1 .. m2 + 2 (rows beyond the grid read as zero)
    auto column = [&](int m1, S_& ym, S_& y0, S_& y1, S_& y2) {
        const size_t idx = (size_t)m2 * ld + m1;
        ym = valid ? Y[idx - ld] : zero;
        y0 = valid ? Y[idx] : zero;
        y1 = valid ? Y[idx + ld] : zero;
        y2 = hasb ? Y[idx + 2 * ld] : zero;
    };
#pragma unroll
    for (int b0 = 0; b0 < NB; b0 += EB) {
        S_ ym[EB], y0[EB], y1[EB], y2[EB], w0[EB], w1[EB], v0[EB], v1[EB];
#pragma unroll
        for (int i = 0; i < EB; ++i) {
            const int m1 = t + NT * (b0 + i);
            const size_t idx = (size_t)m2 * ld + m1;
            ym[i] = y0[i] = y1[i] = y2[i] = w0[i] = w1[i] = v0[i] = v1[i] = zero;
            if (stencil) {
                column(m1, ym[i], y0[i], y1[i], y2[i]);
                w0[i] = valid ? a.W[idx] : zero;
                w1[i] = hasb ? a.W[idx + ld] : zero;
            }
            if (full && a.BV) {
                v0[i] = valid ? a.BV[idx] : zero;
                v1[i] = hasb ? a.BV[idx + ld] : zero;
            }
        }
#pragma unroll
        for (int i = 0; i < EB; ++i) {
            const int m1 = t + NT * (b0 + i);
            // the neighbours' states of rows m2, m2 + 1 and vertical differences
            // f0 = Y[m2 + 1] - Y[m2 - 1], f1 = Y[m2 + 2] - Y[m2]
            S_ aL = zero, aR = zero, bL = zero, bR = zero;
            R f0L = 0, f0R = 0, f1L = 0, f1R = 0;
            if (stencil) {
                const R f0 = st_diff(y1[i], ym[i]), f1 = st_diff(y2[i], y0[i]);
                if constexpr (SHFL) {
                    f0L = __shfl_up_sync(0xffffffffu, f0, 1);
                    f0R = __shfl_down_sync(0xffffffffu, f0, 1);
                    f1L = __shfl_up_sync(0xffffffffu, f1, 1);
                    f1R = __shfl_down_sync(0xffffffffu, f1, 1);
                    aL = shfl_up_state(y0[i], 1);
                    aR = shfl_down_state(y0[i], 1);
                    bL = shfl_up_state(y1[i], 1);
                    bR = shfl_down_state(y1[i], 1);
                    if (lane == 0 && m1 >= 1) {
                        S_ q0, q1, q2, q3;
                        column(m1 - 1, q0, q1, q2, q3);
                        f0L = st_diff(q2, q0);
                        f1L = st_diff(q3, q1);
                        aL = q1;
                        bL = q2;
                    }
                    if (lane == 31) {
                        S_ q0, q1, q2, q3;
                        column(m1 + 1, q0, q1, q2, q3);
                        f0R = st_diff(q2, q0);
                        f1R = st_diff(q3, q1);
                        aR = q1;
                        bR = q2;
                    }
                } else if (m1 >= 1) {
                    S_ q0, q1, q2, q3;
                    column(m1 - 1, q0, q1, q2, q3);
                    f0L = st_diff(q2, q0);
                    f1L = st_diff(q3, q1);
                    aL = q1;
                    bL = q2;
                    column(m1 + 1, q0, q1, q2, q3);
                    f0R = st_diff(q2, q0);
                    f1R = st_diff(q3, q1);
                    aR = q1;
                    bR = q2;
                }
            }
            if (m1 < 1) continue;
            const C zz = buf[padi(m1)];
            R rr0 = R(0), rr1 = R(0);
            if (valid) {
                const size_t idx = (size_t)m2 * ld + m1;
                if (!full) {
                    a.out[idx] = (double)zz.x;
                    if (hasb) a.out[idx + ld] = (double)zz.y;
                } else {
                    BYv[idx] = a.BV ? st_add(v0[i], zz.x) : st_from_r<S_, R>(zz.x);
                    if (hasb) BYv[idx + ld] = a.BV ? st_add(v1[i], zz.y) : st_from_r<S_, R>(zz.y);
                    if (do_resid) {
                        // D Y as in diff_state: d11 dxx + d22 dyy + d12 dxy
                        const R dy0 = a.d11 * (st_diff(aR, y0[i]) + st_diff(aL, y0[i])) +
                                      a.d22 * (st_diff(y1[i], y0[i]) + st_diff(ym[i], y0[i])) + a.d12 * (f0R - f0L);
                        const R jb0 = a.BV ? jump_gen(v0[i], y0[i], a.rw, a.rw_lo) + zz.x
                                           : zz.x - a.rw * st_r(y0[i]);
                        rr0 = st_diff(w0[i], y0[i]) + a.htt * jb0 + a.htt * dy0;
                        if (hasb) {
                            const R dy1 = a.d11 * (st_diff(bR, y1[i]) + st_diff(bL, y1[i])) +
                                          a.d22 * (st_diff(y2[i], y1[i]) + st_diff(y0[i], y1[i])) + a.d12 * (f1R - f1L);
                            const R jb1 = a.BV ? jump_gen(v1[i], y1[i], a.rw, a.rw_lo) + zz.y
                                               : zz.y - a.rw * st_r(y1[i]);
                            rr1 = st_diff(w1[i], y1[i]) + a.htt * jb1 + a.htt * dy1;
                        }
                    }
                }
            }
            if (do_resid) {
                buf[padi(m1)] = mk<R>(rr0, rr1);
                buf[padi(P - m1)] = mk<R>(-rr0, -rr1);
            }
        }
    }
}

// INCR: compiled for the increment mode only (INV_INCR), else for INV_FULL / INV_OUT,
// so the two epilogues do not share one register allocation
template <typename R, int P, bool INCR>
__device__ __forceinline__ void row_inverse_body(const InvArgs<R>& a, int upb) {
    using C = cpx<R>;
    using S_ = St<R>;
    using CF = Cfg<R, P>;
    constexpr int NT = CF::NT, N = P / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int unit = threadIdx.x / NT, t = threadIdx.x - unit * NT;
    C* buf = reinterpret_cast<C*>(smem_raw) + (size_t)unit * CF::ULEN;
    const int p = blockIdx.x * upb + unit;
    const int m2 = 2 * p + 1;
    const bool valid = m2 <= N - 1;
    const bool hasb = valid && (m2 + 1 <= N - 1);
    constexpr int Gc = cgroup<R>();
    const C* S = (const C*)a.S;
    const int rows = a.g.rows;
    const C* tw = (const C*)a.tw;
    // the device-side fixed-point loop decides on the device whether a residual is needed
    const bool do_resid = a.conv_flag ? (*a.conv_flag == 0) : (a.do_resid != 0);
    const int ld = a.g.ldS, ldR = a.g.ldR;
    S_* const BYv = a.BYind ? *a.BYind : a.BY;
    if (t == 0 && valid) prefetch_inverse_rows(a, BYv, m2, hasb, do_resid);
    // the two spectrum rows, each value read once (the Hermitian extension uses
    // every k twice): k at plain indices 2k, 2k + 1 of buf, which the first stage
    // reads completely before it writes
    // (a constant trip count with a guard, so the loop unrolls and its loads go out together)
#pragma unroll
    for (int q = 0; q < (P / 2 + NT) / NT; ++q) {
        const int k = t + q * NT;
        if (k <= P / 2) {
            C xa = mk<R>(0, 0), xb = mk<R>(0, 0);
            if (valid) {
                const int g = k / Gc, c = k - g * Gc;
                xa = S[((size_t)g * rows + (m2 - 1)) * Gc + c];
                xb = S[((size_t)g * rows + m2) * Gc + c];
            }
            buf[2 * k] = xa;
            buf[2 * k + 1] = xb;
        }
    }
    __syncthreads();
    auto load = [&](int pos) -> C {
        const bool hi = pos > P / 2;
        const int k = hi ? P - pos : pos;
        C xa = buf[2 * k], xb = buf[2 * k + 1];
        if (k == 0 || k == P / 2) { xa.y = 0; xb.y = 0; }
        if (hi) { xa.y = -xa.y; xb.y = -xb.y; }
        return mk<R>(xa.x - xb.y, xa.y + xb.x);
    };
    if constexpr (INCR) {
        // the C2R into buf in natural order, then the epilogue in coalesced order
        // (each thread reads the C2R values at its own m1 < N and writes the
        // residual at m1 and P - m1 > N, whose C2R values nobody reads, and
        // at 0 and N: no thread reads another thread's overwritten value)
        block_fft<R, +1, P, false>(buf, t, tw, load, SmemStore<R>{buf});
        incr_epilogue<R, P>(a, BYv, buf, t, m2, valid, hasb, do_resid);
        if (do_resid && t == 0) {
            buf[padi(0)] = mk<R>(0, 0);
            buf[padi(N)] = mk<R>(0, 0);
        }
        __syncthreads();
    } else {
        block_fft<R, +1, P, false>(buf, t, tw, load, SmemStore<R>{buf});
        full_epilogue<R, P>(a, BYv, buf, t, m2, valid, hasb, do_resid);
        if (do_resid && t == 0) {
            buf[padi(0)] = mk<R>(0, 0);
            buf[padi(N)] = mk<R>(0, 0);
        }
        __syncthreads();
    }
    if (!do_resid) return;   // uniform across the block
    constexpr int GE = rgroup<R>();
    auto store_e = [&](int k, C zz) {
        if (k >= N) return;
        const int gE = k / GE, c = k - gE * GE;
        const R va = k >= 1 ? R(-0.5) * zz.y : R(0);
        const R vb = k >= 1 ? R(0.5) * zz.x : R(0);
        if (valid) a.E[((size_t)gE * N + m2) * GE + c] = va;
        if (hasb) a.E[((size_t)gE * N + m2 + 1) * GE + c] = vb;
    };
    block_fft<R, -1, P>(buf, t, tw, SmemLoad<R>{buf}, store_e);
}
// The single-job kernel reads its arguments from a shared-memory copy: inlined
// from the parameter block itself, this FFT kernel needed several times the
// spill traffic (register allocation differs with the arguments' address space).
template <typename R, int P, bool INCR>
PIDE_FFT_KERNEL(R, P) k_row_inverse(const __grid_constant__ InvArgs<R> a0) {
    __shared__ InvArgs<R> sa;
    if (threadIdx.x == 0) sa = a0;
    __syncthreads();
    row_inverse_body<R, P, INCR>(sa, Cfg<R, P>::UNITS);
}
template <typename R, int P, bool INCR>
PIDE_FFT_JOBS_KERNEL(R, P) k_row_inverse_jobs(const InvArgs<R>* __restrict__ arr, JobsCtl jc) {
    if (jc.skip(blockIdx.y)) return;
    row_inverse_body<R, P, INCR>(arr[blockIdx.y], blockDim.x / Cfg<R, P>::NT);
}

// ---------------------------------------------------------------------------
// column solve of the non-mixed diffusion operator in the row-DST basis.
// After the row DST, mode k1 of A_0 acts along s2 as the constant-coefficient
// tridiagonal matrix T = c tridiag(-1, 2 + s, -1) on rows 1..N-1 (Dirichlet
// rows 0 and N), c = c2/4, s = (c0 + c1 sin^2(pi k1/2N))/c: its eigenvalues in
// the column DST basis are c0 + c1 sin^2(pi k1/2N) + c2 sin^2(pi k2/2N).  Its LU
// factors have a closed form: with q = e^{-th}, th = 2 asinh(sqrt(s)/2) (so
// q + 1/q = 2 + s) and psi_m = 1 - q^{2m}, the pivots are u_i = (c/q)
// psi_{i+1}/psi_i.  Scaled by psi, both substitutions become recursions with
// the constant multiplier q,
//     z_i = psi_i b_i + q z_{i-1}                       (z_0 = 0, rows upward)
//     t_i = (q/c) z_i / (psi_i psi_{i+1}) + q t_{i+1}   (t_N = 0, rows downward)
//     x_i = psi_i t_i,
// which a block evaluates as two scans over its threads' row chunks.  It is the
// Thomas algorithm with exact pivots (backward stable for the diagonally
// dominant T), equal to the column DST-I eigen-solve of the same matrix.
// ---------------------------------------------------------------------------
template <typename R, int P> struct ColSolveCfg {
    static constexpr int N = P / 2;
    static constexpr int RPT = N >= 512 ? 16 : (N >= 64 ? N / 32 : 1);  // rows per thread
    static constexpr int NTH = N / RPT >= 32 ? N / RPT : 32;             // threads (rows >= N are zero)
    static constexpr int NW = NTH / 32;
    // FP32: 64 registers (four 256-thread blocks per SM at N = 4096)
    static constexpr int MINB = sizeof(R) == 4 ? 1024 / NTH : 1;
    // the column pair staged in shared memory, one pad pair per 16 rows
    static constexpr int ROWS = NTH * RPT;
    static constexpr size_t SMEM = (size_t)(ROWS + ROWS / 16) * sizeof(cpx<R>);
};
__device__ __forceinline__ int col_pad(int row) { return row + (row >> 4); }

// The recursion y_t = v_t + Q y_{t-1} over the block's threads, in increasing
// thread order (REV = false) or decreasing (REV = true), for two columns at once
// (x and y of the pair): returns y at the previous thread's chunk end (0 for the
// first thread).  wsum: NW pairs of shared memory; one block barrier.
template <typename R, int NW, bool REV>
__device__ __forceinline__ cpx<R> chunk_carry(cpx<R> v, R Qa, R Qb, cpx<R>* wsum) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int l = REV ? 31 - lane : lane;
    const int wp = REV ? NW - 1 - w : w;
    R pa = Qa, pb = Qb, la = R(1), lb = R(1);   // Q^off, and Q^l accumulated bit by bit
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const R ua = REV ? __shfl_down_sync(0xffffffffu, v.x, off) : __shfl_up_sync(0xffffffffu, v.x, off);
        const R ub = REV ? __shfl_down_sync(0xffffffffu, v.y, off) : __shfl_up_sync(0xffffffffu, v.y, off);
        if (l >= off) {
            v.x += pa * ua;
            v.y += pb * ub;
        }
        if (l & off) {
            la *= pa;
            lb *= pb;
        }
        pa *= pa;
        pb *= pb;
    }
    // v: inclusive value at position l; pa, pb: Q^32
    R ea = REV ? __shfl_down_sync(0xffffffffu, v.x, 1) : __shfl_up_sync(0xffffffffu, v.x, 1);
    R eb = REV ? __shfl_down_sync(0xffffffffu, v.y, 1) : __shfl_up_sync(0xffffffffu, v.y, 1);
    if (l == 0) ea = eb = R(0);
    if constexpr (NW > 1) {
        if (l == 31) wsum[wp] = v;
        __syncthreads();
        R sa = R(0), sb = R(0);                 // the value at the end of warp position wp - 1
        for (int u = 0; u < wp; ++u) {
            const cpx<R> W = wsum[u];
            sa = sa * pa + W.x;
            sb = sb * pb + W.y;
        }
        ea += la * sa;
        eb += lb * sb;
    }
    return mk<R>(ea, eb);
}

// a / b: the fast FP32 quotient (2 ulp; the solve is the fixed point's
// preconditioner, so it sets only the contraction), exact in FP64
template <typename R> __device__ __forceinline__ R pc_div(R a, R b) {
    if constexpr (sizeof(R) == 4) return __fdividef(a, b);
    else return a / b;
}

// per column of the pair: th, q = e^{-th}, q^2, psi_1, q^RPT and q/c
template <typename R> struct ColConst {
    R th, q, qq, p1, Q, g;
};

template <typename R, int P>
__device__ __forceinline__ void col_solve_body(const ColSolveArgs<R>& a, int pair) {
    using C = cpx<R>;
    using SC = ColSolveCfg<R, P>;
    constexpr int N = SC::N, RPT = SC::RPT, NW = SC::NW;
    __shared__ C wsum[2][NW];
    __shared__ ColConst<R> kc[2];
    const int ka = 2 * pair;                    // columns ka, ka + 1 (mode k1 = column index)
    if (ka >= N) return;                        // uniform across the block
    constexpr int GE = rgroup<R>();
    const int gE = ka / GE, ce = ka - gE * GE;
    C* col = reinterpret_cast<C*>(a.E + (size_t)gE * N * GE + ce);   // row i at col[i * GE / 2]
    constexpr int RS = GE / 2;
    const int i0 = threadIdx.x * RPT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* stage = reinterpret_cast<C*>(smem_raw);
    // per column: q = e^{-th} and psi_1 once per block; psi_{m+1} = psi_m +
    // q^{2m} psi_1 (a sum of positive terms) regenerates a chunk's psi from
    // psi_{i0} and q^{2 i0} in each pass
    if (threadIdx.x < 2) {
        const R cc = R(0.25) * a.rc2;
        const R sv = (a.rc0 + a.rc1 * a.sin2[ka + threadIdx.x]) / cc;
        ColConst<R> k;
        k.th = R(2) * asinh(sqrt(sv) * R(0.5));
        k.q = exp(-k.th);
        k.qq = k.q * k.q;
        k.p1 = -expm1(R(-2) * k.th);
        k.Q = exp(-(R)RPT * k.th);
        k.g = k.q / cc;
        kc[threadIdx.x] = k;
    }
    // coalesced load of the pair (rows outside 1..N-1 are zero), then each
    // thread takes its chunk of RPT consecutive rows
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int i = (int)threadIdx.x + r * SC::NTH;
        stage[col_pad(i)] = (i >= 1 && i <= N - 1) ? col[(size_t)i * RS] : mk<R>(R(0), R(0));
    }
    __syncthreads();
    C v[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) v[r] = stage[col_pad(i0 + r)];
    const ColConst<R> ka_ = kc[0], kb_ = kc[1];
    const R q_a = ka_.q, q_b = kb_.q;
    const R Qa = ka_.Q, Qb = kb_.Q;             // q^RPT
    // psi_i = 1 to working precision once q^{2i} < 2^-25 (FP32; 2^-54 in FP64):
    // then the chunk's recursions need neither psi nor the quotient
    const R thmin = ka_.th < kb_.th ? ka_.th : kb_.th;
    const bool plain = R(2) * (R)i0 * thmin > (sizeof(R) == 4 ? R(18) : R(38));
    // forward: z_i = psi_i b_i + q z_{i-1}
    C acc = mk<R>(R(0), R(0));
    if (plain) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            acc.x = v[r].x + q_a * acc.x;
            acc.y = v[r].y + q_b * acc.y;
            v[r] = acc;
        }
    } else {
        R pa = -expm1(R(-2) * (R)i0 * ka_.th), pb = -expm1(R(-2) * (R)i0 * kb_.th);
        R ea = exp(R(-2) * (R)i0 * ka_.th), eb = exp(R(-2) * (R)i0 * kb_.th);
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            acc.x = pa * v[r].x + q_a * acc.x;
            acc.y = pb * v[r].y + q_b * acc.y;
            v[r] = acc;
            pa += ea * ka_.p1;
            pb += eb * kb_.p1;
            ea *= ka_.qq;
            eb *= kb_.qq;
        }
    }
    {
        const C cin = chunk_carry<R, NW, false>(acc, Qa, Qb, wsum[0]);
        R fa = q_a, fb = q_b;
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            v[r].x += fa * cin.x;
            v[r].y += fb * cin.y;
            fa *= q_a;
            fb *= q_b;
        }
    }
    // backward: t_i = (q/c) z_i / (psi_i psi_{i+1}) + q t_{i+1}
    if (plain) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const bool in = i0 + r <= N - 1;
            v[r].x = in ? ka_.g * v[r].x : R(0);
            v[r].y = in ? kb_.g * v[r].y : R(0);
        }
    } else {
        R pa = -expm1(R(-2) * (R)i0 * ka_.th), pb = -expm1(R(-2) * (R)i0 * kb_.th);
        R ea = exp(R(-2) * (R)i0 * ka_.th), eb = exp(R(-2) * (R)i0 * kb_.th);
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int i = i0 + r;
            const R na = pa + ea * ka_.p1, nb = pb + eb * kb_.p1;
            const bool in = i >= 1 && i <= N - 1;
            v[r].x = in ? pc_div(ka_.g * v[r].x, pa * na) : R(0);
            v[r].y = in ? pc_div(kb_.g * v[r].y, pb * nb) : R(0);
            pa = na;
            pb = nb;
            ea *= ka_.qq;
            eb *= kb_.qq;
        }
    }
    acc = mk<R>(R(0), R(0));
#pragma unroll
    for (int r = RPT - 1; r >= 0; --r) {
        acc.x = v[r].x + q_a * acc.x;
        acc.y = v[r].y + q_b * acc.y;
        v[r] = acc;
    }
    {
        const C cin = chunk_carry<R, NW, true>(acc, Qa, Qb, wsum[1]);
        R fa = q_a, fb = q_b;
#pragma unroll
        for (int r = RPT - 1; r >= 0; --r) {
            v[r].x += fa * cin.x;
            v[r].y += fb * cin.y;
            fa *= q_a;
            fb *= q_b;
        }
    }
    // x_i = psi_i t_i, with the row DST pair's normalisation, staged for a
    // coalesced store of rows 1..N-1 (the chunk reads of every thread ended
    // before the first scan's barrier)
    const R sc = a.rscale;
    if (plain) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) stage[col_pad(i0 + r)] = mk<R>(sc * v[r].x, sc * v[r].y);
    } else {
        R pa = -expm1(R(-2) * (R)i0 * ka_.th), pb = -expm1(R(-2) * (R)i0 * kb_.th);
        R ea = exp(R(-2) * (R)i0 * ka_.th), eb = exp(R(-2) * (R)i0 * kb_.th);
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            stage[col_pad(i0 + r)] = mk<R>(sc * pa * v[r].x, sc * pb * v[r].y);
            pa += ea * ka_.p1;
            pb += eb * kb_.p1;
            ea *= ka_.qq;
            eb *= kb_.qq;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int i = (int)threadIdx.x + r * SC::NTH;
        if (i >= 1 && i <= N - 1) col[(size_t)i * RS] = stage[col_pad(i)];
    }
}
template <typename R, int P>
__global__ void __launch_bounds__(ColSolveCfg<R, P>::NTH, ColSolveCfg<R, P>::MINB) k_col_solve(const __grid_constant__ ColSolveArgs<R> a) {
    col_solve_body<R, P>(a, blockIdx.x);
}
template <typename R, int P>
__global__ void __launch_bounds__(ColSolveCfg<R, P>::NTH, ColSolveCfg<R, P>::MINB) k_col_solve_jobs(const ColSolveArgs<R>* __restrict__ arr,
                                                                           JobsCtl jc) {
    if (jc.skip(blockIdx.y)) return;
    col_solve_body<R, P>(arr[blockIdx.y], blockIdx.x);
}

// ---------------------------------------------------------------------------
// row DST back to nodes: increment, state update, eq. 3.25 maximum, and the
// row pass of the increment's B_w sweep (packed R2C) in the same block
// ---------------------------------------------------------------------------
template <typename R, int P>
__device__ __forceinline__ void dst_row_body(const DstRowArgs<R>& a, int upb) {
    using C = cpx<R>;
    using CF = Cfg<R, P>;
    constexpr int NT = CF::NT, N = P / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int unit = threadIdx.x / NT, t = threadIdx.x - unit * NT;
    C* buf = reinterpret_cast<C*>(smem_raw) + (size_t)unit * CF::ULEN;
    StopCand* red = reinterpret_cast<StopCand*>(reinterpret_cast<C*>(smem_raw) + (size_t)upb * CF::ULEN);
    const int p = blockIdx.x * upb + unit;
    const int m2 = 2 * p + 1;
    const bool valid = m2 <= N - 1;
    const bool hasb = valid && (m2 + 1 <= N - 1);
    constexpr int GE = rgroup<R>();
    const C* tw = (const C*)a.tw;
    // the two DST rows, each value read once (the odd extension uses every j
    // twice), at plain indices of buf, which the first stage reads before it writes
    // (constant trip count with a guard: the loop unrolls and its loads go out together)
#pragma unroll
    for (int q = 0; q < (N + NT) / NT; ++q) {
        const int j = t + q * NT;
        if (j <= N) {
            R ea = 0, eb = 0;
            if (valid && j >= 1 && j <= N - 1) {
                const int gE = j / GE, c = j - gE * GE;
                ea = a.E[((size_t)gE * N + m2) * GE + c];
                if (hasb) eb = a.E[((size_t)gE * N + m2 + 1) * GE + c];
            }
            buf[j] = mk<R>(ea, eb);
        }
    }
    __syncthreads();
    auto load = [&](int i) -> C {
        const int j = i <= N ? i : P - i;
        const C e = buf[j];
        return i <= N ? e : mk<R>(-e.x, -e.y);
    };
    St<R>* const Yv = a.Yind ? *a.Yind : a.Y;
    // eq. 3.25: the thread's largest ratio |D| / max(1, |Y|) in the transform
    // precision selects a node, whose D and Y are kept; the block's selected
    // node is evaluated again in FP64 below, and that FP64 value is what the
    // stopping rule compares with tol.  A NaN ratio or Y marks the block
    // non-finite.
    R qmax = R(-1), dsel = R(0);
    St<R> ysel = st_from_r<St<R>, R>(R(0));
    bool bad = false;
    const int ld = a.g.ldS, ldR = a.g.ldR;
    // the state rows updated after the DST arrive in L2 while it runs
    if (t == 0 && valid) l2_prefetch(Yv + (size_t)m2 * ld, (size_t)(hasb ? 2 : 1) * ld * sizeof(St<R>));
    // the increment also enters the next B_w sweep: it is laid out at its
    // R2C position p = m1 + N/2 + 1 (zero elsewhere) for the second transform.
    // y0, y1: the states at (m2, m1) and (m2 + 1, m1), loaded beforehand
    auto update = [&](int m1, C zz, St<R> y0, St<R> y1) {
        R da = 0, db = 0;
        if (valid && m1 >= 1 && m1 < N) {
            da = R(-0.5) * zz.y;
            {
                const size_t idx = (size_t)m2 * ld + m1;
                const St<R> y = st_add(y0, da);
                Yv[idx] = y;
                a.D[(size_t)m2 * ldR + m1] = da;
                const R yr = st_r(y);
                const R q = stop_ratio(da, yr);
                bad |= !(q == q) || !(yr == yr);
                if (q > qmax) { qmax = q; dsel = da; ysel = y; }
            }
            if (hasb) {
                db = R(0.5) * zz.x;
                const size_t idx = (size_t)(m2 + 1) * ld + m1;
                const St<R> y = st_add(y1, db);
                Yv[idx] = y;
                a.D[(size_t)(m2 + 1) * ldR + m1] = db;
                const R yr = st_r(y);
                const R q = stop_ratio(db, yr);
                bad |= !(q == q) || !(yr == yr);
                if (q > qmax) { qmax = q; dsel = db; ysel = y; }
            }
        }
        buf[padi((m1 + N / 2 + 1) & (P - 1))] = mk<R>(da, db);
    };
    // the DST back into buf in natural order; then the update in coalesced
    // order (m1 = t + NT b), the state loads of four outputs issued together
    block_fft<R, -1, P>(buf, t, tw, load, SmemStore<R>{buf});
    {
        constexpr int NB = N / NT;
        C zz[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) zz[b] = buf[padi(t + NT * b)];
        __syncthreads();                    // every DST value is read before buf takes the R2C input
#pragma unroll
        for (int b = 0; b < NB; ++b) buf[padi((N + t + NT * b + N / 2 + 1) & (P - 1))] = mk<R>(0, 0);
        const St<R> zero = st_from_r<St<R>, R>(R(0));
#pragma unroll
        for (int b0 = 0; b0 < NB; b0 += 4) {
            St<R> y0[4], y1[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int m1 = t + NT * (b0 + i);
                const size_t idx = (size_t)m2 * ld + m1;
                y0[i] = (valid && m1 >= 1) ? Yv[idx] : zero;
                y1[i] = (hasb && m1 >= 1) ? Yv[idx + ld] : zero;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) update(t + NT * (b0 + i), zz[b0 + i], y0[i], y1[i]);
        }
        __syncthreads();
    }
    // (reduced here, before the second transform, so the candidate's registers
    // are free during it)
    // block maximum of eq. 3.25 in FP64, one atomic per block: the block's
    // node with the largest ratio in the transform precision is re-evaluated
    // in FP64 from its D and Y (as stored).  With FP32
    // ratios (two roundings of Y, 2 ulp of the quotient) the FP64 value found
    // is within 2^-20 relative of the exact FP64 maximum.
    for (int o = 16; o > 0; o >>= 1) {
        const R oq = __shfl_xor_sync(0xffffffffu, qmax, o);
        const R od = __shfl_xor_sync(0xffffffffu, dsel, o);
        const St<R> oy = shfl_xor_state(ysel, o);
        if (oq > qmax) { qmax = oq; dsel = od; ysel = oy; }
    }
    bad = __any_sync(0xffffffffu, bad);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
    if (lane == 0) red[warp] = StopCand{(double)qmax, (double)dsel, st_dbl(ysel), bad ? 1 : 0, 0};
    __syncthreads();
    if (threadIdx.x == 0) {
        StopCand c = red[0];
        for (int w = 1; w < nwarp; ++w) {
            const StopCand o = red[w];
            if (o.q > c.q) { c.q = o.q; c.d = o.d; c.y = o.y; }
            c.bad |= o.bad;
        }
        // +inf for a non-finite block: the loop stops, not converged
        const double v = c.bad ? __longlong_as_double(0x7ff0000000000000LL)
                               : (c.q >= 0.0 ? fabs(c.d) / fmax(1.0, fabs(c.y)) : 0.0);
        atomicMax((unsigned long long*)a.resid, (unsigned long long)__double_as_longlong(v));
    }
    // packed R2C of the two increment rows -> spectrum rows rho = m2 + N/2 + 1, +1
    // (the midpoint interpolation is a factor of the increment weight spectrum);
    // positions outside [N/2 + 2, 3N/2] are zero, so first-stage inputs
    // j + r P/16 with r in {0..3, 13..15} always are (P >= 32)
    block_fft<R, -1, P>(buf, t, tw, SmemLoad<R, (P >= 32 ? 0xE00Fu : 0u)>{buf}, SmemStore<R>{buf});
    store_spectrum_rows<R, P>(buf, (C*)a.S, a.g.rows, a.g.ng, m2 + N / 2 + 1, t, valid);
}
template <typename R, int P>
PIDE_FFT_KERNEL(R, P) k_dst_row(const __grid_constant__ DstRowArgs<R> a) { dst_row_body<R, P>(a, Cfg<R, P>::UNITS); }
template <typename R, int P>
PIDE_FFT_JOBS_KERNEL(R, P) k_dst_row_jobs(const DstRowArgs<R>* __restrict__ arr, JobsCtl jc) {
    if (jc.skip(blockIdx.y)) return;
    dst_row_body<R, P>(arr[blockIdx.y], blockDim.x / Cfg<R, P>::NT);
}

// ---------------------------------------------------------------------------
// row DST-I of an FP64 interior field into the DST buffer E: the same
// transform k_row_inverse applies to the residual before the column solve, here
// for a residual handed in by the caller (pide2d_iteration_probe)
// ---------------------------------------------------------------------------
template <typename R, int P>
PIDE_FFT_KERNEL(R, P) k_row_dst(Geometry g, const double* __restrict__ src, R* __restrict__ E, const void* twv) {
    using C = cpx<R>;
    using CF = Cfg<R, P>;
    constexpr int NT = CF::NT, N = P / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int unit = threadIdx.x / NT, t = threadIdx.x - unit * NT;
    C* buf = reinterpret_cast<C*>(smem_raw) + (size_t)unit * CF::ULEN;
    const int p = blockIdx.x * CF::UNITS + unit;
    const int m2 = 2 * p + 1;
    const bool valid = m2 <= N - 1;
    const bool hasb = valid && (m2 + 1 <= N - 1);
    const C* tw = (const C*)twv;
    // odd extension of rows m2, m2 + 1 packed into one complex sequence
    auto load = [&](int i) -> C {
        const int j = i <= N ? i : P - i;
        const R sg = i <= N ? R(1) : R(-1);
        R xa = 0, xb = 0;
        if (j >= 1 && j <= N - 1) {
            if (valid) xa = sg * (R)src[(size_t)m2 * g.ldS + j];
            if (hasb) xb = sg * (R)src[(size_t)(m2 + 1) * g.ldS + j];
        }
        return mk<R>(xa, xb);
    };
    constexpr int GE = rgroup<R>();
    auto store_e = [&](int k, C zz) {
        if (k >= N) return;
        const int gE = k / GE, c = k - gE * GE;
        const R va = k >= 1 ? R(-0.5) * zz.y : R(0);
        const R vb = k >= 1 ? R(0.5) * zz.x : R(0);
        if (valid) E[((size_t)gE * N + m2) * GE + c] = va;
        if (hasb) E[((size_t)gE * N + m2 + 1) * GE + c] = vb;
    };
    block_fft<R, -1, P>(buf, t, tw, load, store_e);
}

// ---------------------------------------------------------------------------
// per-step preparation: W = T_SL[Z] (Algorithm 1 step 2), Y^{n,0} (eq. 3.26),
// far field on the boundary ring of Y.  Z - V at interior nodes comes from
// k_explicit (one pass), so the SL taps read it instead of recomputing the
// stencil per tap.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ double far_dbl(const PrepArgs<R>& a, int q1, int q2, double Kd) {
    return (double)far_value<double>(a.payoff, Kd, a.E1d[q1 + a.g.eoff], a.E2d[q2 + a.g.eoff]);
}
// the far field at node (q1, q2) as a state value: FP64 in FP64 mode, a
// double-float pair from the split e^{s} tables in FP32-bulk mode (no FP64
// instruction in the step's preparation); prev selects tau_{n-1}, else tau_n
template <typename R>
__device__ __forceinline__ St<R> far_state(const PrepArgs<R>& a, int q1, int q2, bool prev) {
    if constexpr (sizeof(R) == 4) {
        const int i1 = q1 + a.g.eoff, i2 = q2 + a.g.eoff;
        return far_value_df(a.payoff, prev ? a.Kdp_h : a.Kdn_h, prev ? a.Kdp_l : a.Kdn_l, a.E1h[i1], a.E1l[i1],
                            a.E2h[i2], a.E2l[i2]);
    } else {
        return far_dbl(a, q1, q2, prev ? a.Kd_prev : a.Kd_now);
    }
}

// cz = h_t (1-theta) (D V - r_w V + B V) at interior nodes (Z - V of Algorithm 1 step 2)
template <typename R>
__device__ __forceinline__ void explicit_body(const PrepArgs<R>& a) {
    const int N = a.g.N;
    const int m1 = blockIdx.x * blockDim.x + threadIdx.x;
    const int m2 = blockIdx.y * blockDim.y + threadIdx.y;
    if (m1 < 1 || m2 < 1 || m1 > N - 1 || m2 > N - 1) return;
    const int ld = a.g.ldS;
    const size_t idx = (size_t)m2 * ld + m1;
    const St<R>* V = a.V[0];
    a.cz[(size_t)m2 * a.g.ldR + m1] =
        a.htm * (diff_state(V, idx, ld, a.d11, a.d22, a.d12) + jump_gen(a.BV[idx], V[idx], a.rw, a.rw_lo));
}

template <typename R>
__global__ void k_explicit(const __grid_constant__ PrepArgs<R> a) { explicit_body<R>(a); }
template <typename R>
__global__ void k_explicit_jobs(const PrepArgs<R>* __restrict__ arr) {
    explicit_body<R>(arr[blockIdx.z]);
}

template <typename R, int NTAP>
__device__ __forceinline__ void prep_node(const PrepArgs<R>& a, int m1, int m2) {
    const int N = a.g.N;
    if (m1 > N || m2 > N) return;
    const int ld = a.g.ldS, ldR = a.g.ldR;
    const size_t idx = (size_t)m2 * ld + m1;
    using S_ = St<R>;
    if (m1 == 0 || m2 == 0 || m1 == N || m2 == N) {
        a.Y[idx] = far_state(a, m1, m2, false);
        return;
    }
    const S_* V = a.V[0];
    const S_ v = V[idx];
    const bool expl = a.htm != R(0);
    const R czm = expl ? a.cz[(size_t)m2 * ldR + m1] : R(0);
    // all taps inside the interior: the common case, branch-free and unrolled
    const bool inner = m1 + a.o1 >= 1 && m1 + a.o1 + NTAP - 1 <= N - 1 && m2 + a.o2 >= 1 &&
                       m2 + a.o2 + NTAP - 1 <= N - 1;
    R w1[NTAP], w2[NTAP];
#pragma unroll
    for (int c = 0; c < NTAP; ++c) {
        w1[c] = a.w1[c];
        w2[c] = a.w2[c];
    }
    R corr = czm;
    if (inner) {
        const S_* Vb = V + (size_t)(m2 + a.o2) * ld + (m1 + a.o1);
        const R* Cb = a.cz + (size_t)(m2 + a.o2) * ldR + (m1 + a.o1);
        S_ vv[NTAP][NTAP];
        R cc[NTAP][NTAP];
#pragma unroll
        for (int b = 0; b < NTAP; ++b)
#pragma unroll
            for (int c = 0; c < NTAP; ++c) {
                vv[b][c] = Vb[(size_t)b * ld + c];
                cc[b][c] = expl ? Cb[(size_t)b * ldR + c] : R(0);
            }
#pragma unroll
        for (int b = 0; b < NTAP; ++b) {
            R row = 0;
#pragma unroll
            for (int c = 0; c < NTAP; ++c) row += w1[c] * (st_diff(vv[b][c], v) + cc[b][c] - czm);
            corr += w2[b] * row;
        }
    } else {
#pragma unroll
        for (int b = 0; b < NTAP; ++b) {
            const int q2 = m2 + a.o2 + b;
            R row = 0;
#pragma unroll
            for (int c = 0; c < NTAP; ++c) {
                const int q1 = m1 + a.o1 + c;
                R dz;
                if (q1 >= 1 && q1 <= N - 1 && q2 >= 1 && q2 <= N - 1) {
                    dz = st_diff(V[(size_t)q2 * ld + q1], v) - czm;
                    if (expl) dz += a.cz[(size_t)q2 * ldR + q1];
                } else {
                    dz = st_diff(far_state(a, q1, q2, true), v) - czm;
                }
                row += w1[c] * dz;
            }
            corr += w2[b] * row;
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

// NC consecutive values of a row from position q (q's parity fixed per launch):
// 16-byte loads of state pairs (8-byte loads of R pairs) where aligned
template <int NC, int C>
__device__ __forceinline__ void load_pairs(const float2* row, int q, float2* v) {
    if constexpr (C + 1 < NC) {
        const float4 t = *reinterpret_cast<const float4*>(row + q + C);
        v[C] = make_float2(t.x, t.y);
        v[C + 1] = make_float2(t.z, t.w);
        load_pairs<NC, C + 2>(row, q, v);
    } else if constexpr (C < NC) {
        v[C] = row[q + C];
    }
}
template <int NC, int C>
__device__ __forceinline__ void load_pairs(const float* row, int q, float* v) {
    if constexpr (C + 1 < NC) {
        const float2 t = *reinterpret_cast<const float2*>(row + q + C);
        v[C] = t.x;
        v[C + 1] = t.y;
        load_pairs<NC, C + 2>(row, q, v);
    } else if constexpr (C < NC) {
        v[C] = row[q + C];
    }
}
template <int NC, typename T>
__device__ __forceinline__ void load_run(const T* row, int q, T* v) {
    if (q & 1) {
        v[0] = row[q];
        load_pairs<NC, 1>(row, q, v);
    } else {
        load_pairs<NC, 0>(row, q, v);
    }
}

// FP32-bulk: the interior nodes (m1, m2) and (m1 + 1, m2), m1 even, from one
// window of NTAP rows by NTAP + 1 columns (the same arithmetic per node as
// prep_node's interior path).  False, with nothing written, when a node is not
// interior or a tap leaves the interior.
template <int NTAP>
__device__ __forceinline__ bool prep_pair_f32(const PrepArgs<float>& a, int m1, int m2) {
    const int N = a.g.N;
    const int q0 = m1 + a.o1, r0 = m2 + a.o2;
    if (!(m1 >= 2 && m1 + 1 <= N - 1 && m2 >= 1 && m2 <= N - 1 && q0 >= 1 && q0 + NTAP <= N - 1 && r0 >= 1 &&
          r0 + NTAP - 1 <= N - 1))
        return false;
    constexpr int NC = NTAP + 1;
    const int ld = a.g.ldS, ldR = a.g.ldR;
    const size_t idx = (size_t)m2 * ld + m1;
    const float2* V = a.V[0];
    const float4 vp = *reinterpret_cast<const float4*>(V + idx);
    const float2 v0 = make_float2(vp.x, vp.y), v1 = make_float2(vp.z, vp.w);
    const bool expl = a.htm != 0.f;
    float czm0 = 0.f, czm1 = 0.f;
    if (expl) {
        const float2 c = *reinterpret_cast<const float2*>(a.cz + (size_t)m2 * ldR + m1);
        czm0 = c.x;
        czm1 = c.y;
    }
    float w1[NTAP], w2[NTAP];
#pragma unroll
    for (int c = 0; c < NTAP; ++c) {
        w1[c] = a.w1[c];
        w2[c] = a.w2[c];
    }
    float corr0 = czm0, corr1 = czm1;
#pragma unroll
    for (int b = 0; b < NTAP; ++b) {
        float2 vv[NC];
        float cc[NC];
        load_run<NC>(V + (size_t)(r0 + b) * ld, q0, vv);
        if (expl) {
            load_run<NC>(a.cz + (size_t)(r0 + b) * ldR, q0, cc);
        } else {
#pragma unroll
            for (int c = 0; c < NC; ++c) cc[c] = 0.f;
        }
        float row0 = 0.f, row1 = 0.f;
#pragma unroll
        for (int c = 0; c < NTAP; ++c) {
            row0 += w1[c] * (st_diff(vv[c], v0) + cc[c] - czm0);
            row1 += w1[c] * (st_diff(vv[c + 1], v1) + cc[c + 1] - czm1);
        }
        corr0 += w2[b] * row0;
        corr1 += w2[b] * row1;
    }
    const float2 W0 = st_add(v0, corr0), W1 = st_add(v1, corr1);
    *reinterpret_cast<float4*>(a.W + idx) = make_float4(W0.x, W0.y, W1.x, W1.y);
    float e0 = 0.f, e1 = 0.f;
    auto hist = [&](int k, float2& h0, float2& h1) {
        const float4 t = *reinterpret_cast<const float4*>(a.V[k] + idx);
        h0 = make_float2(t.x, t.y);
        h1 = make_float2(t.z, t.w);
    };
    if (a.hcount == 2) {
        float2 p0, p1;
        hist(1, p0, p1);
        e0 = -st_diff(p0, v0);
        e1 = -st_diff(p1, v1);
    } else if (a.hcount == 3) {
        float2 p0, p1, q0v, q1v;
        hist(1, p0, p1);
        hist(2, q0v, q1v);
        e0 = -3.f * st_diff(p0, v0) + st_diff(q0v, v0);
        e1 = -3.f * st_diff(p1, v1) + st_diff(q1v, v1);
    } else if (a.hcount >= 4) {
        float2 p0, p1, q0v, q1v, u0, u1;
        hist(1, p0, p1);
        hist(2, q0v, q1v);
        hist(3, u0, u1);
        e0 = -6.f * st_diff(p0, v0) + 4.f * st_diff(q0v, v0) - st_diff(u0, v0);
        e1 = -6.f * st_diff(p1, v1) + 4.f * st_diff(q1v, v1) - st_diff(u1, v1);
    }
    const float2 Y0 = st_add(v0, e0), Y1 = st_add(v1, e1);
    *reinterpret_cast<float4*>(a.Y + idx) = make_float4(Y0.x, Y0.y, Y1.x, Y1.y);
    return true;
}

// each thread prepares the nodes (2 tx, m2) and (2 tx + 1, m2)
template <typename R, int NTAP>
__device__ __forceinline__ void prep_body(const PrepArgs<R>& a) {
    const int m1 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int m2 = blockIdx.y * blockDim.y + threadIdx.y;
    if constexpr (sizeof(R) == 4) {
        if (prep_pair_f32<NTAP>(a, m1, m2)) return;
    }
    prep_node<R, NTAP>(a, m1, m2);
    prep_node<R, NTAP>(a, m1 + 1, m2);
}

template <typename R, int NTAP>
__global__ void __launch_bounds__(256) k_prep(const __grid_constant__ PrepArgs<R> a) { prep_body<R, NTAP>(a); }
template <typename R, int NTAP>
__global__ void __launch_bounds__(256) k_prep_jobs(const PrepArgs<R>* __restrict__ arr) {
    prep_body<R, NTAP>(arr[blockIdx.z]);
}

// ---------------------------------------------------------------------------
// price-space jump operator B_w = T_out I~ C T_in (eqs. 3.12-3.17 on the
// paper's non-uniform price grid): T_in into a P x P real array on the
// y_in lattice, the zero-padded correlation with Omega by row R2C, column
// (forward, * conj(w^)/P^2, inverse) and row C2R passes, T_out back
// ---------------------------------------------------------------------------
// A[j2][j1] = sum_{b,c} w[j2][b] w[j1][c] V[s[j2]+b][s[j1]+c] on j < nin (s = -1: beyond x_max, 0)
template <typename R>
__global__ void k_ps_tin(int P, int nin, int nx1, const int* __restrict__ s, const double* __restrict__ w,
                         const double* __restrict__ V, R* __restrict__ A) {
    const int j1 = blockIdx.x * blockDim.x + threadIdx.x;
    const int j2 = blockIdx.y * blockDim.y + threadIdx.y;
    if (j1 >= P || j2 >= P) return;
    double acc = 0.0;
    if (j1 < nin && j2 < nin) {
        const int a1 = s[j1], a2 = s[j2];
        if (a1 >= 0 && a2 >= 0) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const double* row = V + (size_t)(a2 + b) * nx1 + a1;
                double r = 0.0;
#pragma unroll
                for (int c = 0; c < 4; ++c) r += w[j1 * 4 + c] * row[c];
                acc += w[j2 * 4 + b] * r;
            }
        }
    }
    A[(size_t)j2 * P + j1] = (R)acc;
}

// rows 2p, 2p+1 of A (rows and columns >= nin are zero): packed R2C into S [group][row][c]
template <typename R, int P>
PIDE_FFT_KERNEL(R, P) k_ps_rows_fwd(const R* __restrict__ A, int nin, void* Sv, int rows, int ng, const void* twv) {
    using C = cpx<R>;
    using CF = Cfg<R, P>;
    constexpr int NT = CF::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int unit = threadIdx.x / NT, t = threadIdx.x - unit * NT;
    C* buf = reinterpret_cast<C*>(smem_raw) + (size_t)unit * CF::ULEN;
    const int p = blockIdx.x * CF::UNITS + unit;
    const int rho = 2 * p;
    const bool valid = rho < nin;
    const C* tw = (const C*)twv;
    auto load = [&](int i) -> C {
        R xa = 0, xb = 0;
        if (valid && i < nin) {
            xa = A[(size_t)rho * P + i];
            if (rho + 1 < nin) xb = A[(size_t)(rho + 1) * P + i];
        }
        return mk<R>(xa, xb);
    };
    block_fft<R, -1, P>(buf, t, tw, load, SmemStore<R>{buf});
    constexpr int Gc = cgroup<R>();
    C* S = (C*)Sv;
    for (int g = t; g < ng; g += NT) {
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

// column k1: rows < nin in, forward FFT, * Wh, inverse FFT, rows < nout out (in place)
template <typename R, int P>
PIDE_FFT_KERNEL(R, P) k_ps_col(void* Sv, const void* Whv, int rows, int nin, int nout, const void* twv) {
    using C = cpx<R>;
    using CF = Cfg<R, P>;
    constexpr int NT = CF::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int unit = threadIdx.x / NT, t = threadIdx.x - unit * NT;
    C* buf = reinterpret_cast<C*>(smem_raw) + (size_t)unit * CF::ULEN;
    const int k1 = blockIdx.x * CF::UNITS + unit;
    const bool valid = k1 <= P / 2;
    constexpr int Gc = cgroup<R>();
    const int g = k1 / Gc, c = k1 - g * Gc;
    C* col = (C*)Sv + (size_t)g * rows * Gc + c;
    const C* wh = (const C*)Whv + (size_t)k1 * P;      // column-major weight spectrum
    const C* tw = (const C*)twv;
    auto load = [&](int rho) -> C { return (valid && rho < nin) ? col[(size_t)rho * Gc] : mk<R>(0, 0); };
    auto store_mul = [&](int k2, C v) {
        const C w = valid ? __ldg(&wh[k2]) : mk<R>(0, 0);
        buf[padi(k2)] = cmul(v, w);
    };
    block_fft<R, -1, P>(buf, t, tw, load, store_mul);
    auto store_out = [&](int m, C v) {
        if (valid && m < nout) col[(size_t)m * Gc] = v;
    };
    block_fft<R, +1, P>(buf, t, tw, SmemLoad<R>{buf}, store_out);
}

// output rows 2p, 2p+1 (< nout): packed C2R of the Hermitian spectrum, By[row][m1] for m1 < nout
template <typename R, int P>
PIDE_FFT_KERNEL(R, P) k_ps_rows_inv(const void* Sv, int rows, int nout, double* __restrict__ By, int ldB,
                                    const void* twv) {
    using C = cpx<R>;
    using CF = Cfg<R, P>;
    constexpr int NT = CF::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int unit = threadIdx.x / NT, t = threadIdx.x - unit * NT;
    C* buf = reinterpret_cast<C*>(smem_raw) + (size_t)unit * CF::ULEN;
    const int p = blockIdx.x * CF::UNITS + unit;
    const int r = 2 * p;
    const bool valid = r < nout;
    constexpr int Gc = cgroup<R>();
    const C* S = (const C*)Sv;
    const C* tw = (const C*)twv;
    auto load = [&](int pos) -> C {
        const bool hi = pos > P / 2;
        const int k = hi ? P - pos : pos;
        C xa = mk<R>(0, 0), xb = mk<R>(0, 0);
        if (valid) {
            const int g = k / Gc, c = k - g * Gc;
            xa = S[((size_t)g * rows + r) * Gc + c];
            xb = S[((size_t)g * rows + r + 1) * Gc + c];
        }
        if (k == 0 || k == P / 2) { xa.y = 0; xb.y = 0; }
        if (hi) { xa.y = -xa.y; xb.y = -xb.y; }
        return mk<R>(xa.x - xb.y, xa.y + xb.x);
    };
    auto store = [&](int m1, C z) {
        if (!valid || m1 >= nout) return;
        By[(size_t)r * ldB + m1] = (double)z.x;
        if (r + 1 < nout) By[(size_t)(r + 1) * ldB + m1] = (double)z.y;
    };
    block_fft<R, +1, P>(buf, t, tw, load, store);
}

// ---------------------------------------------------------------------------
// omega-hat: FP64 forward column FFT of the FP64 row spectra of Omega
// ---------------------------------------------------------------------------
// Wh  = conj(w^)/P^2                      (full sweeps: midpoints taken in space)
// Whi = conj(w^ c^[k1] c^[k2])/P^2         (increment sweeps; skipped if NULL): c^[k] = sum_e c_e
// e^{-2 pi i e k/P} with the cubic midpoint weights c = (-1, 9, 9, -1)/16, so the
// midpoint interpolation of a field that vanishes outside the interior is a
// spectral factor (its support never wraps around at P = 2N).
template <typename RO, int P>
PIDE_FFT_KERNEL(double, P) k_weights_col(Geometry g, const double2* Sd, cpx<RO>* Wh, cpx<RO>* Whi,
                                         const double2* twd) {
    using CF = Cfg<double, P>;
    constexpr int NT = CF::NT, N = P / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int unit = threadIdx.x / NT, t = threadIdx.x - unit * NT;
    double2* buf = reinterpret_cast<double2*>(smem_raw) + (size_t)unit * CF::ULEN;
    const int k1 = blockIdx.x * CF::UNITS + unit;
    const bool valid = k1 <= P / 2;
    constexpr int Gd = cgroup<double>();
    const int gd = k1 / Gd, cd = k1 - gd * Gd;
    auto load = [&](int i) -> double2 {
        // rows >= N of the zero-padded Omega are zero
        return (valid && i < N) ? Sd[((size_t)gd * P + i) * Gd + cd] : mk<double>(0, 0);
    };
    const double inv = 1.0 / ((double)P * (double)P);
    auto chat = [&](int k) -> double2 {
        const double2 a1 = twd[k], a2 = twd[(2 * k) & (P - 1)], a3 = twd[(3 * k) & (P - 1)];
        return mk<double>(-0.0625 + 0.5625 * a1.x + 0.5625 * a2.x - 0.0625 * a3.x,
                          0.5625 * a1.y + 0.5625 * a2.y - 0.0625 * a3.y);
    };
    const double2 c1 = valid ? chat(k1) : mk<double>(0, 0);
    // column-major: column k1 at k1 P, contiguous for the column pass that reads it
    auto store = [&](int k2, double2 w) {
        if (!valid) return;
        const size_t o = (size_t)k1 * P + k2;
        Wh[o] = mk<RO>((RO)(w.x * inv), (RO)(-w.y * inv));
        if (Whi) {
            const double2 wc = cmul(cmul(w, c1), chat(k2));
            Whi[o] = mk<RO>((RO)(wc.x * inv), (RO)(-wc.y * inv));
        }
    };
    block_fft<double, -1, P>(buf, t, twd, load, store);
}

// ---------------------------------------------------------------------------
// the adjoint's weight contraction: C(l) = sum_j sum_m xi_j(m) V~_j(m + l + 1/2)
// (V~ the midpoints of T_in with the far field), so that for every direction
// <xi_j, B_{dw} V_j> summed over j equals sum_l dw(l) C(l).  The spectra of
// xi_j (raw rows at the increment positions) and of V~_j (midpoint rows)
// meet column by column; conj(xi^) V^ is accumulated in FP64 over all
// states, and one inverse transform at the end gives C.
// ---------------------------------------------------------------------------
// column k1: forward FFT of the V~ column (midpoints along s2, rows 0..P+1)
// and of the xi column (raw rows rlo..rhi-1); acc[k1][k2] += conj(X) A
template <typename R, int P>
PIDE_FFT_KERNEL(R, P) k_corr_col(Geometry g, const void* SV, const void* SX, int rlo, int rhi, double2* acc,
                                 const void* twv) {
    using C = cpx<R>;
    using CF = Cfg<R, P>;
    constexpr int NT = CF::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int unit = threadIdx.x / NT, t = threadIdx.x - unit * NT;
    C* bufA = reinterpret_cast<C*>(smem_raw) + (size_t)unit * 2 * CF::ULEN;
    C* bufX = bufA + CF::ULEN;
    const int k1 = blockIdx.x * CF::UNITS + unit;
    const bool valid = k1 <= P / 2;
    constexpr int Gc = cgroup<R>();
    const int gq = k1 / Gc, c = k1 - gq * Gc;
    const C* colA = (const C*)SV + (size_t)gq * g.rows * Gc + c;
    const C* colX = (const C*)SX + (size_t)gq * g.rows * Gc + c;
    const C* tw = (const C*)twv;
    for (int rho = t; rho < P + 2; rho += NT) bufA[padi(rho)] = valid ? colA[(size_t)rho * Gc] : mk<R>(0, 0);
    __syncthreads();
    auto loadA = [&](int i) -> C {
        if (i > P - 2) return mk<R>(0, 0);
        const C x0 = bufA[padi(i)], x1 = bufA[padi(i + 1)], x2 = bufA[padi(i + 2)], x3 = bufA[padi(i + 3)];
        return mk<R>(R(-0.0625) * (x0.x + x3.x) + R(0.5625) * (x1.x + x2.x),
                     R(-0.0625) * (x0.y + x3.y) + R(0.5625) * (x1.y + x2.y));
    };
    block_fft<R, -1, P>(bufA, t, tw, loadA, SmemStore<R>{bufA});
    auto loadX = [&](int rho) -> C {
        return (valid && rho >= rlo && rho < rhi) ? colX[(size_t)rho * Gc] : mk<R>(0, 0);
    };
    auto accum = [&](int k2, C x) {
        if (!valid) return;
        const C a = bufA[padi(k2)];
        double2* d = acc + (size_t)k1 * P + k2;
        const double xr = (double)x.x, xi = (double)x.y, ar = (double)a.x, ai = (double)a.y;
        double2 v = *d;
        v.x += xr * ar + xi * ai;           // conj(x) a
        v.y += xr * ai - xi * ar;
        *d = v;
    };
    block_fft<R, -1, P>(bufX, t, tw, loadX, accum);
}

// in place, column k1 of the FP64 accumulator: inverse FFT over k2
template <int P>
PIDE_FFT_KERNEL(double, P) k_corr_icol(double2* acc, const double2* twd) {
    using CF = Cfg<double, P>;
    constexpr int NT = CF::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int unit = threadIdx.x / NT, t = threadIdx.x - unit * NT;
    double2* buf = reinterpret_cast<double2*>(smem_raw) + (size_t)unit * CF::ULEN;
    const int k1 = blockIdx.x * CF::UNITS + unit;
    const bool valid = k1 <= P / 2;
    double2* col = acc + (size_t)k1 * P;
    auto load = [&](int k2) -> double2 { return valid ? col[k2] : mk<double>(0, 0); };
    auto store = [&](int q2, double2 v) {
        if (valid) col[q2] = v;
    };
    block_fft<double, +1, P>(buf, t, twd, load, store);
}

// lag row l2 (q2 = l2 - 1 mod P): Hermitian C2R over k1, C[l2 + N/2][l1 + N/2] = out(q1 = l1 - 1) / P^2
template <int P>
PIDE_FFT_KERNEL(double, P) k_corr_rows(const double2* acc, double* Cout, const double2* twd) {
    using CF = Cfg<double, P>;
    constexpr int NT = CF::NT, N = P / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int unit = threadIdx.x / NT, t = threadIdx.x - unit * NT;
    double2* buf = reinterpret_cast<double2*>(smem_raw) + (size_t)unit * CF::ULEN;
    const int r = blockIdx.x * CF::UNITS + unit;        // 0..N-1: l2 = r - N/2
    const bool valid = r < N;
    const int q2 = (r - N / 2 - 1 + P) & (P - 1);
    auto load = [&](int k) -> double2 {
        if (!valid) return mk<double>(0, 0);
        const bool hi = k > P / 2;
        const int kk = hi ? P - k : k;
        double2 v = acc[(size_t)kk * P + q2];
        if (kk == 0 || kk == P / 2) v.y = 0.0;
        if (hi) v.y = -v.y;
        return v;
    };
    const double inv = 1.0 / ((double)P * (double)P);
    auto store = [&](int q1, double2 v) {
        const int l1 = ((q1 + 1) & (P - 1));                 // l1 = q1 + 1 (mod P), wanted in [-N/2, N/2)
        const int i1 = l1 < N / 2 ? l1 + N / 2 : (l1 >= P - N / 2 ? l1 - (P - N / 2) : -1);
        if (valid && i1 >= 0) Cout[(size_t)r * N + i1] = v.x * inv;
    };
    block_fft<double, +1, P>(buf, t, twd, load, store);
}

// Greeks (Sec. 4, central differences) at interior nodes, in price space:
// which = 0: dV/dS1, 1: dV/dS2, 2: d2V/dS1^2, 3: d2V/dS1dS2, 4: d2V/dS2^2
template <typename R>
__global__ void k_greeks(Geometry g, const St<R>* V, const double* E1d, const double* E2d, double h, int which,
                         double* out, int ldo) {
    const int m1 = blockIdx.x * blockDim.x + threadIdx.x, m2 = blockIdx.y * blockDim.y + threadIdx.y;
    if (m1 < 1 || m2 < 1 || m1 > g.N - 1 || m2 > g.N - 1) return;
    const int ld = g.ldS;
    const size_t i = (size_t)m2 * ld + m1;
    const double S1 = E1d[m1 + g.eoff], S2 = E2d[m2 + g.eoff];
    const double c = st_dbl(V[i]);
    double r;
    if (which == 0) {
        r = (st_dbl(V[i + 1]) - st_dbl(V[i - 1])) / (2.0 * h) / S1;
    } else if (which == 1) {
        r = (st_dbl(V[i + ld]) - st_dbl(V[i - ld])) / (2.0 * h) / S2;
    } else if (which == 2) {
        const double v1 = (st_dbl(V[i + 1]) - st_dbl(V[i - 1])) / (2.0 * h);
        const double v11 = (st_dbl(V[i + 1]) - 2.0 * c + st_dbl(V[i - 1])) / (h * h);
        r = (v11 - v1) / (S1 * S1);
    } else if (which == 3) {
        r = (st_dbl(V[i + ld + 1]) - st_dbl(V[i - ld + 1]) - st_dbl(V[i + ld - 1]) + st_dbl(V[i - ld - 1])) /
            (4.0 * h * h) / (S1 * S2);
    } else {
        const double v2 = (st_dbl(V[i + ld]) - st_dbl(V[i - ld])) / (2.0 * h);
        const double v22 = (st_dbl(V[i + ld]) - 2.0 * c + st_dbl(V[i - ld])) / (h * h);
        r = (v22 - v2) / (S2 * S2);
    }
    out[(size_t)m2 * ldo + m1] = r;
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
// launchers: dispatch the compile-time transform length
// ---------------------------------------------------------------------------
#define PIDE_SWITCH_P(P, CASE)                                                              \
    switch (P) {                                                                            \
        case 16: CASE(16); case 32: CASE(32); case 64: CASE(64); case 128: CASE(128);       \
        case 256: CASE(256); case 512: CASE(512); case 1024: CASE(1024);                    \
        case 2048: CASE(2048); case 4096: CASE(4096); case 8192: CASE(8192);                \
        default: return cudaErrorInvalidValue;                                              \
    }

// time-loop kernels exist for every transform length in both precisions (an
// 8192-point FP64 unit takes 139 KB of dynamic shared memory, one block per SM)
template <typename R, int P> struct LoopSize { static constexpr bool ok = true; };

template <typename R, int P, class K, class A>
cudaError_t launch_fft_kernel(K kernel, const A& a, int work_units, size_t extra_smem, cudaStream_t s) {
    using CF = Cfg<R, P>;
    const size_t smem = CF::SMEM + extra_smem;
    set_smem(kernel, smem);
    const int blocks = (work_units + CF::UNITS - 1) / CF::UNITS;
    kernel<<<blocks, CF::THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

// units per block of a multi-job launch: upb <= 0 selects the single-job shape
template <typename R, int P>
int jobs_units(int upb) {
    using CF = Cfg<R, P>;
    if (upb <= 0) return CF::UNITS;
    const int mx = CF::MAXT / CF::NT;
    return upb < mx ? upb : mx;
}

template <typename R, int P, class K, class A>
cudaError_t launch_fft_kernel_jobs(K kernel, const A* arr, int njobs, JobsCtl jc, int work_units, size_t extra_smem,
                                   int upb, cudaStream_t s) {
    using CF = Cfg<R, P>;
    const int u = jobs_units<R, P>(upb);
    const size_t smem = (size_t)u * CF::ULEN * sizeof(cpx<R>) + extra_smem;
    set_smem(kernel, smem);
    const dim3 grid((work_units + u - 1) / u, njobs);
    kernel<<<grid, u * CF::NT, smem, s>>>(arr, jc);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_row_forward_jobs(const FwdArgs<R>& a0, const FwdArgs<R>* arr, int K, JobsCtl jc, int upb,
                              cudaStream_t s) {
#define CASE(PP) return launch_fft_kernel_jobs<R, PP>(k_row_forward_jobs<R, PP>, arr, K, jc, a0.npairs, 0, upb, s);
    PIDE_SWITCH_P(a0.g.P, CASE)
#undef CASE
}
template <typename R>
cudaError_t launch_col_jobs(const ColArgs<R>& a0, const ColArgs<R>* arr, int K, JobsCtl jc, int upb,
                              cudaStream_t s) {
#define CASE(PP)                                                                                             \
    if constexpr (LoopSize<R, PP>::ok) {                                                                     \
        if (a0.mode == COL_INCR)                                                                             \
            return launch_fft_kernel_jobs<R, PP>(k_col_jobs<R, PP, true>, arr, K, jc, PP / 2 + 1, 0, upb, s); \
        return launch_fft_kernel_jobs<R, PP>(k_col_jobs<R, PP, false>, arr, K, jc, PP / 2 + 1, 0, upb, s); \
    } else return cudaErrorInvalidValue;
    PIDE_SWITCH_P(a0.g.P, CASE)
#undef CASE
}
template <typename R>
cudaError_t launch_row_inverse_jobs(const InvArgs<R>& a0, const InvArgs<R>* arr, int K, JobsCtl jc, int upb,
                              cudaStream_t s) {
#define CASE(PP)                                                                                             \
    if constexpr (LoopSize<R, PP>::ok) {                                                                     \
        if (a0.mode == INV_INCR)                                                                             \
            return launch_fft_kernel_jobs<R, PP>(k_row_inverse_jobs<R, PP, true>, arr, K, jc, PP / 4, 0, upb, s); \
        return launch_fft_kernel_jobs<R, PP>(k_row_inverse_jobs<R, PP, false>, arr, K, jc, PP / 4, 0, upb, s); \
    } else return cudaErrorInvalidValue;
    PIDE_SWITCH_P(a0.g.P, CASE)
#undef CASE
}
template <typename R>
cudaError_t launch_col_solve_jobs(const ColSolveArgs<R>& a0, const ColSolveArgs<R>* arr, int K, JobsCtl jc, int upb,
                                  cudaStream_t s) {
    (void)upb;                               // one block per column pair
#define CASE(PP)                                                                                      \
    {                                                                                                 \
        using SC = ColSolveCfg<R, PP>;                                                                \
        set_smem(k_col_solve_jobs<R, PP>, SC::SMEM);                                                  \
        const dim3 grid(PP / 4, K);                                                                   \
        k_col_solve_jobs<R, PP><<<grid, SC::NTH, SC::SMEM, s>>>(arr, jc);                             \
        return cudaGetLastError();                                                                    \
    }
    PIDE_SWITCH_P(a0.g.P, CASE)
#undef CASE
}
template <typename R>
cudaError_t launch_dst_row_jobs(const DstRowArgs<R>& a0, const DstRowArgs<R>* arr, int K, JobsCtl jc, int upb,
                              cudaStream_t s) {
#define CASE(PP)                                                                                             \
    if constexpr (LoopSize<R, PP>::ok) return launch_fft_kernel_jobs<R, PP>(k_dst_row_jobs<R, PP>, arr, K, jc, PP / 4, 32 * sizeof(StopCand), upb, s); \
    else return cudaErrorInvalidValue;
    PIDE_SWITCH_P(a0.g.P, CASE)
#undef CASE
}
template <typename R>
cudaError_t launch_prep_jobs(const PrepArgs<R>& a0, const PrepArgs<R>* arr, int K, bool explicit_part, cudaStream_t s) {
    const dim3 blk(32, 8);
    const dim3 grd((a0.g.N + 1 + 31) / 32, (a0.g.N + 1 + 7) / 8, K);
    if (explicit_part) {
        k_explicit_jobs<R><<<grd, blk, 0, s>>>(arr);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const dim3 grp((a0.g.N + 1 + 63) / 64, (a0.g.N + 1 + 7) / 8, K);      // two nodes per thread
    if (a0.nt == 2) k_prep_jobs<R, 2><<<grp, blk, 0, s>>>(arr);
    else k_prep_jobs<R, 4><<<grp, blk, 0, s>>>(arr);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_row_forward(const FwdArgs<R>& a, cudaStream_t s) {
#define CASE(PP) return launch_fft_kernel<R, PP>(k_row_forward<R, PP>, a, a.npairs, 0, s);
    PIDE_SWITCH_P(a.g.P, CASE)
#undef CASE
}
template <typename R>
cudaError_t launch_col(const ColArgs<R>& a, cudaStream_t s) {
#define CASE(PP)                                                                       \
    if constexpr (LoopSize<R, PP>::ok) {                                               \
        if (a.mode == COL_INCR) return launch_fft_kernel<R, PP>(k_col<R, PP, true>, a, PP / 2 + 1, 0, s); \
        return launch_fft_kernel<R, PP>(k_col<R, PP, false>, a, PP / 2 + 1, 0, s); \
    } else return cudaErrorInvalidValue;
    PIDE_SWITCH_P(a.g.P, CASE)
#undef CASE
}
template <typename R>
cudaError_t launch_row_inverse(const InvArgs<R>& a, cudaStream_t s) {
#define CASE(PP)                                                                       \
    if constexpr (LoopSize<R, PP>::ok) {                                               \
        if (a.mode == INV_INCR) return launch_fft_kernel<R, PP>(k_row_inverse<R, PP, true>, a, PP / 4, 0, s); \
        return launch_fft_kernel<R, PP>(k_row_inverse<R, PP, false>, a, PP / 4, 0, s); \
    } else return cudaErrorInvalidValue;
    PIDE_SWITCH_P(a.g.P, CASE)
#undef CASE
}
template <typename R>
cudaError_t launch_col_solve(const ColSolveArgs<R>& a, cudaStream_t s) {
#define CASE(PP)                                                                                      \
    {                                                                                                 \
        using SC = ColSolveCfg<R, PP>;                                                                \
        set_smem(k_col_solve<R, PP>, SC::SMEM);                                                       \
        k_col_solve<R, PP><<<PP / 4, SC::NTH, SC::SMEM, s>>>(a);                                      \
        return cudaGetLastError();                                                                    \
    }
    PIDE_SWITCH_P(a.g.P, CASE)
#undef CASE
}
template <typename R>
cudaError_t launch_dst_row(const DstRowArgs<R>& a, cudaStream_t s) {
#define CASE(PP)                                                                       \
    if constexpr (LoopSize<R, PP>::ok) return launch_fft_kernel<R, PP>(k_dst_row<R, PP>, a, PP / 4, 32 * sizeof(StopCand), s); \
    else return cudaErrorInvalidValue;
    PIDE_SWITCH_P(a.g.P, CASE)
#undef CASE
}
template <typename R>
cudaError_t launch_row_dst(const Geometry& g, const double* src, R* E, const void* tw, cudaStream_t s) {
#define CASE(PP)                                                                                      \
    {                                                                                                 \
        using CF = Cfg<R, PP>;                                                                        \
        set_smem(k_row_dst<R, PP>, CF::SMEM);                                                         \
        k_row_dst<R, PP><<<(PP / 4 + CF::UNITS - 1) / CF::UNITS, CF::THREADS, CF::SMEM, s>>>(g, src, E, tw); \
        return cudaGetLastError();                                                                    \
    }
    PIDE_SWITCH_P(g.P, CASE)
#undef CASE
}
template <typename R>
cudaError_t launch_prep(const PrepArgs<R>& a, cudaStream_t s) {
    const dim3 blk(32, 8);
    const dim3 grd((a.g.N + 1 + 31) / 32, (a.g.N + 1 + 7) / 8);
    const dim3 grp((a.g.N + 1 + 63) / 64, (a.g.N + 1 + 7) / 8);     // two nodes per thread
    if (a.htm != R(0)) {
        k_explicit<R><<<grd, blk, 0, s>>>(a);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (a.nt == 2) k_prep<R, 2><<<grp, blk, 0, s>>>(a);
    else k_prep<R, 4><<<grp, blk, 0, s>>>(a);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_ps_tin(int P, int nin, int nx1, const int* s, const double* w, const double* V, R* A,
                          cudaStream_t st) {
    const dim3 blk(32, 8), grd((P + 31) / 32, (P + 7) / 8);
    k_ps_tin<R><<<grd, blk, 0, st>>>(P, nin, nx1, s, w, V, A);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_ps_rows_fwd(int P, const R* A, int nin, void* S, const void* tw, cudaStream_t st) {
    const int rows = P, ng = spectrum_groups<R>(P);
#define CASE(PP)                                                                                     \
    if constexpr (LoopSize<R, PP>::ok) {                                                             \
        using CF = Cfg<R, PP>;                                                                       \
        set_smem(k_ps_rows_fwd<R, PP>, CF::SMEM);                                                    \
        const int units = (nin + 1) / 2;                                                             \
        k_ps_rows_fwd<R, PP><<<(units + CF::UNITS - 1) / CF::UNITS, CF::THREADS, CF::SMEM, st>>>(A, nin, S, rows, ng, tw); \
        return cudaGetLastError();                                                                   \
    } else return cudaErrorInvalidValue;
    PIDE_SWITCH_P(P, CASE)
#undef CASE
}
template <typename R>
cudaError_t launch_ps_col(int P, void* S, const void* Wh, int nin, int nout, const void* tw, cudaStream_t st) {
#define CASE(PP)                                                                                     \
    if constexpr (LoopSize<R, PP>::ok) {                                                             \
        using CF = Cfg<R, PP>;                                                                       \
        set_smem(k_ps_col<R, PP>, CF::SMEM);                                                         \
        k_ps_col<R, PP><<<(PP / 2 + 1 + CF::UNITS - 1) / CF::UNITS, CF::THREADS, CF::SMEM, st>>>(S, Wh, PP, nin, nout, tw); \
        return cudaGetLastError();                                                                   \
    } else return cudaErrorInvalidValue;
    PIDE_SWITCH_P(P, CASE)
#undef CASE
}
template <typename R>
cudaError_t launch_ps_rows_inv(int P, const void* S, int nout, double* By, int ldB, const void* tw, cudaStream_t st) {
#define CASE(PP)                                                                                     \
    if constexpr (LoopSize<R, PP>::ok) {                                                             \
        using CF = Cfg<R, PP>;                                                                       \
        set_smem(k_ps_rows_inv<R, PP>, CF::SMEM);                                                    \
        const int units = (nout + 1) / 2;                                                            \
        k_ps_rows_inv<R, PP><<<(units + CF::UNITS - 1) / CF::UNITS, CF::THREADS, CF::SMEM, st>>>(S, PP, nout, By, ldB, tw); \
        return cudaGetLastError();                                                                   \
    } else return cudaErrorInvalidValue;
    PIDE_SWITCH_P(P, CASE)
#undef CASE
}
template <typename RO>
cudaError_t launch_weights_col(const Geometry& g, const void* Sd, void* Wh, void* Whi, const void* twd,
                               cudaStream_t s) {
#define CASE(PP)                                                                                   \
    {                                                                                              \
        using CF = Cfg<double, PP>;                                                                \
        set_smem(k_weights_col<RO, PP>, CF::SMEM);                                                 \
        k_weights_col<RO, PP><<<(PP / 2 + 1 + CF::UNITS - 1) / CF::UNITS, CF::THREADS, CF::SMEM, s>>>( \
            g, (const double2*)Sd, (cpx<RO>*)Wh, (cpx<RO>*)Whi, (const double2*)twd);               \
        return cudaGetLastError();                                                                 \
    }
    PIDE_SWITCH_P(g.P, CASE)
#undef CASE
}
template <typename R>
cudaError_t launch_corr_col(const Geometry& g, const void* SV, const void* SX, int rlo, int rhi, double* acc,
                            const void* tw, cudaStream_t s) {
#define CASE(PP)                                                                                      \
    {                                                                                                 \
        using CF = Cfg<R, PP>;                                                                        \
        const size_t sm = 2 * CF::SMEM;                                                               \
        if (sm > 227 * 1024) return cudaErrorInvalidValue;      /* two FP64 8192-point units */      \
        set_smem(k_corr_col<R, PP>, sm);                                                              \
        k_corr_col<R, PP><<<(PP / 2 + 1 + CF::UNITS - 1) / CF::UNITS, CF::THREADS, sm, s>>>(          \
            g, SV, SX, rlo, rhi, (double2*)acc, tw);                                                  \
        return cudaGetLastError();                                                                    \
    }
    PIDE_SWITCH_P(g.P, CASE)
#undef CASE
}
template <typename R>
cudaError_t launch_corr_finish(const Geometry& g, double* acc, double* Cout, const void* twd, cudaStream_t s) {
    if constexpr (sizeof(R) == 8) {
#define CASE(PP)                                                                                      \
        {                                                                                             \
            using CF = Cfg<double, PP>;                                                               \
            set_smem(k_corr_icol<PP>, CF::SMEM);                                                      \
            k_corr_icol<PP><<<(PP / 2 + 1 + CF::UNITS - 1) / CF::UNITS, CF::THREADS, CF::SMEM, s>>>(  \
                (double2*)acc, (const double2*)twd);                                                  \
            cudaError_t e = cudaGetLastError();                                                       \
            if (e != cudaSuccess) return e;                                                           \
            set_smem(k_corr_rows<PP>, CF::SMEM);                                                      \
            k_corr_rows<PP><<<(PP / 2 + CF::UNITS - 1) / CF::UNITS, CF::THREADS, CF::SMEM, s>>>(      \
                (const double2*)acc, Cout, (const double2*)twd);                                      \
            return cudaGetLastError();                                                                \
        }
        PIDE_SWITCH_P(g.P, CASE)
#undef CASE
    } else {
        return cudaErrorInvalidValue;       // the FP64 transforms are instantiated with the FP64 kernels
    }
}
template <typename R>
cudaError_t launch_greeks(const Geometry& g, const St<R>* V, const double* E1d, const double* E2d, double h,
                         int which, double* out, int ldo, cudaStream_t s) {
    const dim3 blk(32, 8), grd((g.N + 1 + 31) / 32, (g.N + 1 + 7) / 8);
    k_greeks<R><<<grd, blk, 0, s>>>(g, V, E1d, E2d, h, which, out, ldo);
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

}  // namespace pide
