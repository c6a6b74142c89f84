// Device building blocks shared by the pide2d kernels: complex arithmetic,
// the in-register small DFTs and the shared-memory block FFT.
//
// Block FFT.  One "FFT unit" is P/16 threads that each hold 16 complex
// values in registers; a length-P transform (P = 2^p, 16 <= P <= 8192) is a
// Stockham autosort sequence of radix-16 stages and at most one radix-2/4/8
// stage, exchanging through shared memory between stages.  Stage with
// radix R and span Ns: butterfly j reads buf[j + r P/R], multiplies by
// w_P^{(j mod Ns) r P/(Ns R)}, applies an R-point DFT and writes
// buf[(j - j mod Ns) R + j mod Ns + r Ns] (the autosort Stockham formulation
// of Govindaraju et al., SC'08).  Shared-memory addresses are padded with
// one element per 16 to break the bank conflicts of the first stage.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pide {

template <typename R> struct cpx_t;
template <> struct cpx_t<float> { using type = float2; };
template <> struct cpx_t<double> { using type = double2; };
template <typename R> using cpx = typename cpx_t<R>::type;

template <typename R> __device__ __forceinline__ cpx<R> mk(R x, R y) { cpx<R> c; c.x = x; c.y = y; return c; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { a.x *= s; a.y *= s; return a; }

// padded shared-memory index: one pad element per 16
__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int P) { return P + (P >> 4); }

// v * e^{DIR 2 pi i m / 16} for a compile-time m in [0, 16)
template <int DIR, int M, typename C>
__device__ __forceinline__ C mul_w16(C v) {
    using R = decltype(v.x);
    constexpr int m = M & 15;
    // cos(2 pi m/16), sin(2 pi m/16) for m = 0..15
    constexpr double c16[16] = {1.0, 0.92387953251128674, 0.70710678118654752, 0.38268343236508977,
                                0.0, -0.38268343236508977, -0.70710678118654752, -0.92387953251128674,
                                -1.0, -0.92387953251128674, -0.70710678118654752, -0.38268343236508977,
                                0.0, 0.38268343236508977, 0.70710678118654752, 0.92387953251128674};
    constexpr double s16[16] = {0.0, 0.38268343236508977, 0.70710678118654752, 0.92387953251128674,
                                1.0, 0.92387953251128674, 0.70710678118654752, 0.38268343236508977,
                                0.0, -0.38268343236508977, -0.70710678118654752, -0.92387953251128674,
                                -1.0, -0.92387953251128674, -0.70710678118654752, -0.38268343236508977};
    if constexpr (m == 0) {
        return v;
    } else if constexpr (m == 8) {
        C r; r.x = -v.x; r.y = -v.y; return r;
    } else if constexpr (m == 4) {          // multiply by DIR*i
        C r;
        if constexpr (DIR > 0) { r.x = -v.y; r.y = v.x; } else { r.x = v.y; r.y = -v.x; }
        return r;
    } else if constexpr (m == 12) {         // multiply by -DIR*i
        C r;
        if constexpr (DIR > 0) { r.x = v.y; r.y = -v.x; } else { r.x = -v.y; r.y = v.x; }
        return r;
    } else {
        const R c = (R)c16[m];
        const R s = (R)(DIR > 0 ? s16[m] : -s16[m]);
        C r; r.x = v.x * c - v.y * s; r.y = v.x * s + v.y * c; return r;
    }
}

template <int K, int L> struct brev_t {
    static constexpr int value = ((K & 1) << (L - 1)) | brev_t<(K >> 1), L - 1>::value;
};
template <int K> struct brev_t<K, 0> { static constexpr int value = 0; };

template <int N> struct log2_t { static constexpr int value = 1 + log2_t<N / 2>::value; };
template <> struct log2_t<1> { static constexpr int value = 0; };

// in-register radix-2 butterfly layer for the R-point DFT (iterative DIT)
template <int DIR, int RAD, int LEN, int I, int K, typename C>
__device__ __forceinline__ void dit_bfly(C* v) {
    if constexpr (I < RAD) {
        if constexpr (K < LEN / 2) {
            C a = v[I + K];
            C b = mul_w16<DIR, K*(16 / LEN)>(v[I + K + LEN / 2]);
            v[I + K] = cadd(a, b);
            v[I + K + LEN / 2] = csub(a, b);
            dit_bfly<DIR, RAD, LEN, I, K + 1>(v);
        } else {
            dit_bfly<DIR, RAD, LEN, I + LEN, 0>(v);
        }
    }
}
template <int DIR, int RAD, int LEN, typename C>
__device__ __forceinline__ void dit_layers(C* v) {
    if constexpr (LEN <= RAD) {
        dit_bfly<DIR, RAD, LEN, 0, 0>(v);
        dit_layers<DIR, RAD, LEN * 2>(v);
    }
}
template <int RAD, int I, typename C>
__device__ __forceinline__ void bitrev_perm(C* v) {
    if constexpr (I < RAD) {
        constexpr int J = brev_t<I, log2_t<RAD>::value>::value;
        if constexpr (J > I) { C t = v[I]; v[I] = v[J]; v[J] = t; }
        bitrev_perm<RAD, I + 1>(v);
    }
}
// X[k] = sum_n v[n] e^{DIR 2 pi i n k / RAD}, natural order in and out (RAD <= 16)
template <int DIR, int RAD, typename C>
__device__ __forceinline__ void dft_small(C* v) {
    bitrev_perm<RAD, 0>(v);
    dit_layers<DIR, RAD, 2>(v);
}

// One Stockham stage of radix RAD over the whole P-point sequence (see top).
// t in [0, P/16): this thread's index within its FFT unit.
template <typename R, int DIR, int RAD>
__device__ __forceinline__ void fft_stage(cpx<R>* buf, int P, int Ns, int t, const cpx<R>* __restrict__ tw) {
    constexpr int NB = 16 / RAD;            // butterflies per thread
    const int nt = P >> 4;
    const int stride = P / RAD;
    const int twstep = P / (Ns * RAD);
    cpx<R> v[16];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * nt;
#pragma unroll
        for (int r = 0; r < RAD; ++r) v[b * RAD + r] = buf[padi(j + r * stride)];
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * nt;
        const int k = j & (Ns - 1);
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                cpx<R> w = __ldg(&tw[k * r * twstep]);
                if (DIR > 0) w.y = -w.y;
                v[b * RAD + r] = cmul(v[b * RAD + r], w);
            }
        }
        dft_small<DIR, RAD>(&v[b * RAD]);
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * nt;
        const int k = j & (Ns - 1);
        const int base = (j - k) * RAD + k;
#pragma unroll
        for (int r = 0; r < RAD; ++r) buf[padi(base + r * Ns)] = v[b * RAD + r];
    }
    __syncthreads();
}

// Unscaled length-P complex DFT of buf (padded layout) in place:
// DIR = -1: X[k] = sum_j x[j] e^{-2 pi i jk/P}; DIR = +1: e^{+2 pi i jk/P}.
// tw[k] = e^{-2 pi i k/P}.  Every thread of the block must call it (it
// synchronises the block); buf must have been written and synchronised.
template <typename R, int DIR>
__device__ void block_fft(cpx<R>* buf, int P, int t, const cpx<R>* __restrict__ tw) {
    int Ns = 1;
    while (Ns * 16 <= P) {
        fft_stage<R, DIR, 16>(buf, P, Ns, t, tw);
        Ns *= 16;
    }
    const int rem = P / Ns;
    if (rem == 2) fft_stage<R, DIR, 2>(buf, P, Ns, t, tw);
    else if (rem == 4) fft_stage<R, DIR, 4>(buf, P, Ns, t, tw);
    else if (rem == 8) fft_stage<R, DIR, 8>(buf, P, Ns, t, tw);
}

// order-preserving bit pattern of a non-negative double (for atomicMax)
__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

}  // namespace pide
