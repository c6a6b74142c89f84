// Device building blocks shared by the pide2d kernels: complex arithmetic,
// the in-register small DFTs and the shared-memory block FFT.
//
// Block FFT.  One "FFT unit" is P/16 threads that each hold 16 complex
// values in registers; a length-P transform (P = 2^p, 16 <= P <= 8192, a
// compile-time constant) is a Stockham autosort sequence of radix-16 stages
// and at most one radix-2/4/8 stage, exchanging through shared memory
// between stages.  Stage with radix R and span Ns: butterfly j reads
// x[j + r P/R], multiplies by w_P^{(j mod Ns) r P/(Ns R)}, applies an R-point
// DFT and writes x[(j - j mod Ns) R + j mod Ns + r Ns] (the autosort
// Stockham formulation of Govindaraju et al., SC'08).  The first stage reads
// through a caller functor and the last stage writes through one, so input
// staging (midpoints, Hermitian or odd extensions) and output epilogues fuse
// into the transform.  Shared-memory addresses are padded with one element
// per 16 to break the bank conflicts of the first stage.
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

// Twiddle tables (complex, transform precision; w = e^{-2 pi i / P}):
//   [0, P)  w^k;
//   then per radix-16 stage with span NS = 16, 256, ... (16 NS <= P): NS rows of 8
//     entries, row k = w^{k TWS m} for m = 1, 2, 3, 4, 8, 12 (TWS = P / (16 NS)), 2 unused;
//   then, when P = 32 NS for a span NS = 16^j, the radix-32 stage: NS rows,
//     row k = w^{2 k m} for m = 1, 2, 3, 4, 8, 12, then w^k, 1 unused.
// Every entry is an FP64 value rounded once, so the fifteen twiddles w^{4a} w^b of a
// butterfly are at most two roundings from exact, and a row is three or four 16-byte loads.
__host__ __device__ constexpr int tw16_offset(int P, int NS) {
    int off = P;
    for (int s = 16; s < NS; s *= 16) off += 8 * s;
    return off;
}
__host__ __device__ constexpr int tw32_offset(int P) {
    int off = P;
    for (int s = 16; 16 * s <= P; s *= 16) off += 8 * s;
    return off;
}
__host__ __device__ constexpr bool tw_has_r32(int P) {
    int s = 1;
    while (32 * s < P) s *= 16;
    return 32 * s == P;
}
__host__ __device__ constexpr int tw_entries(int P) { return tw32_offset(P) + (tw_has_r32(P) ? 8 * (P / 32) : 0); }

// two adjacent table entries with one 16-byte load (two 16-byte loads in FP64)
template <typename R>
__device__ __forceinline__ void tw_pair(const cpx<R>* p, cpx<R>& a, cpx<R>& b) {
    if constexpr (sizeof(R) == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p));
        a = mk<R>(q.x, q.y);
        b = mk<R>(q.z, q.w);
    } else {
        a = __ldg(p);
        b = __ldg(p + 1);
    }
}

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

// v * e^{DIR 2 pi i m / 32} for a compile-time m in [0, 16)
template <int DIR, int M, typename C>
__device__ __forceinline__ C mul_w32(C v) {
    using R = decltype(v.x);
    static_assert(M >= 0 && M < 16, "m in [0, 16)");
    // cos(2 pi m/32), sin(2 pi m/32) for m = 0..15
    constexpr double c32[16] = {1.0, 0.98078528040323044, 0.92387953251128674, 0.83146961230254524,
                                0.70710678118654752, 0.55557023301960218, 0.38268343236508977, 0.19509032201612826,
                                0.0, -0.19509032201612826, -0.38268343236508977, -0.55557023301960218,
                                -0.70710678118654752, -0.83146961230254524, -0.92387953251128674, -0.98078528040323044};
    constexpr double s32[16] = {0.0, 0.19509032201612826, 0.38268343236508977, 0.55557023301960218,
                                0.70710678118654752, 0.83146961230254524, 0.92387953251128674, 0.98078528040323044,
                                1.0, 0.98078528040323044, 0.92387953251128674, 0.83146961230254524,
                                0.70710678118654752, 0.55557023301960218, 0.38268343236508977, 0.19509032201612826};
    if constexpr (M == 0) {
        return v;
    } else if constexpr (M == 8) {          // multiply by DIR*i
        C r;
        if constexpr (DIR > 0) { r.x = -v.y; r.y = v.x; } else { r.x = v.y; r.y = -v.x; }
        return r;
    } else {
        const R c = (R)c32[M];
        const R s = (R)(DIR > 0 ? s32[M] : -s32[M]);
        C r; r.x = v.x * c - v.y * s; r.y = v.x * s + v.y * c; return r;
    }
}
// v[q] *= e^{DIR 2 pi i q / 32} for q = Q..15 where `on`, unchanged elsewhere
template <int DIR, int Q, typename C>
__device__ __forceinline__ void mul_w32_sel(C* v, bool on) {
    if constexpr (Q < 16) {
        const C m = mul_w32<DIR, Q>(v[Q]);
        if (on) v[Q] = m;
        mul_w32_sel<DIR, Q + 1>(v, on);
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

// Loader/storer of the shared-memory buffer (padded layout).  The stage
// calls them with positions base + r * step; when both base and step are
// multiples of 16 (or step < 16 with base a multiple of 16 and r*step < 16)
// the padding distributes, padi(base + r*step) = padi(base) + r*padi(step),
// and the stage uses the *_at forms with one padded base per thread.
template <typename R, unsigned ZM = 0u> struct SmemLoad {
    cpx<R>* buf;
    __device__ __forceinline__ cpx<R> operator()(int i) const { return buf[padi(i)]; }
    __device__ __forceinline__ cpx<R> at(int pbase, int poff) const { return buf[pbase + poff]; }
    static constexpr bool smem = true;
    static constexpr unsigned zero_mask = ZM;     // see zero_mask_of below
};
template <typename R> struct SmemStore {
    cpx<R>* buf;
    __device__ __forceinline__ void operator()(int i, cpx<R> v) const { buf[padi(i)] = v; }
    __device__ __forceinline__ void at(int pbase, int poff, cpx<R> v) const { buf[pbase + poff] = v; }
    static constexpr bool smem = true;
};
template <class T, class = void> struct is_smem_io { static constexpr bool value = false; };
template <class T> struct is_smem_io<T, decltype((void)T::smem, void())> { static constexpr bool value = T::smem; };
// A first-stage loader may declare `zero_mask`: bit r set means that input
// j + r P/16 of every radix-16 butterfly is zero, so the stage skips the load
// and the transform folds the zero at compile time.
template <class T, class = void> struct zero_mask_of { static constexpr unsigned value = 0u; };
template <class T> struct zero_mask_of<T, decltype((void)T::zero_mask, void())> {
    static constexpr unsigned value = T::zero_mask;
};

// One Stockham stage of radix RAD (compile-time P and span NS); t in [0, P/16)
// is the thread's index in its FFT unit.  The stage reads its inputs through
// `load` (position -> value), synchronises the block, and writes its outputs
// through `store` (position, value), then synchronises again.  Intermediate
// stages use the shared buffer; the first stage may read from anywhere (global
// memory, a staged raw array) and the last stage may write anywhere.
template <typename R, int DIR, int RAD, int P, int NS, class L, class S>
__device__ __forceinline__ void fft_stage(int t, const cpx<R>* __restrict__ tw, const L& load, const S& store) {
    constexpr int NB = 16 / RAD;            // butterflies per thread
    constexpr int NT = P / 16;
    constexpr int STRIDE = P / RAD;
    constexpr int TWS = P / (NS * RAD);
    cpx<R> v[16];
    constexpr unsigned ZM = (RAD == 16 && NS == 1) ? zero_mask_of<L>::value : 0u;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * NT;
        if constexpr (is_smem_io<L>::value && STRIDE % 16 == 0) {
            const int pj = padi(j);
#pragma unroll
            for (int r = 0; r < RAD; ++r) {
                if ((ZM >> r) & 1u) v[b * RAD + r] = mk<R>(R(0), R(0));
                else v[b * RAD + r] = load.at(pj, r * (STRIDE + STRIDE / 16));
            }
        } else {
#pragma unroll
            for (int r = 0; r < RAD; ++r) {
                if ((ZM >> r) & 1u) v[b * RAD + r] = mk<R>(R(0), R(0));
                else v[b * RAD + r] = load(j + r * STRIDE);
            }
        }
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * NT;
        if constexpr (NS > 1) {
            const int k = j & (NS - 1);
            if constexpr (RAD == 16) {
                // w^r = w^{4a} w^b (r = 4a + b): the row of the stage's table holds
                // w^b and w^{4a}; nine products form the rest
                static_assert(TWS * NS * 16 == P, "radix-16 table row");
                const cpx<R>* T = tw + tw16_offset(P, NS) + 8 * k;
                cpx<R> wb[4], wa[4];
                tw_pair<R>(T, wb[1], wb[2]);
                tw_pair<R>(T + 2, wb[3], wa[1]);
                tw_pair<R>(T + 4, wa[2], wa[3]);
                if (DIR > 0) {
#pragma unroll
                    for (int q = 1; q < 4; ++q) { wb[q].y = -wb[q].y; wa[q].y = -wa[q].y; }
                }
#pragma unroll
                for (int r = 1; r < 16; ++r) {
                    const int qa = r >> 2, qb = r & 3;
                    cpx<R> w;
                    if (qa == 0) w = wb[qb];
                    else if (qb == 0) w = wa[qa];
                    else w = cmul(wa[qa], wb[qb]);
                    v[b * RAD + r] = cmul(v[b * RAD + r], w);
                }
            } else {
#pragma unroll
                for (int r = 1; r < RAD; ++r) {
                    cpx<R> w = __ldg(&tw[k * (r * TWS)]);
                    if (DIR > 0) w.y = -w.y;
                    v[b * RAD + r] = cmul(v[b * RAD + r], w);
                }
            }
        }
        dft_small<DIR, RAD>(&v[b * RAD]);
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * NT;
        const int k = j & (NS - 1);
        const int base = (j - k) * RAD + k;
        if constexpr (is_smem_io<S>::value && (NS % 16 == 0 || (NS == 1 && RAD == 16))) {
            // NS = 1: base is a multiple of 16 and r < 16; NS % 16 == 0: r*NS is
            const int pb = padi(base);
#pragma unroll
            for (int r = 0; r < RAD; ++r) store.at(pb, r * (NS + NS / 16), v[b * RAD + r]);
        } else {
#pragma unroll
            for (int r = 0; r < RAD; ++r) store(base + r * NS, v[b * RAD + r]);
        }
    }
    __syncthreads();
}

// The last Stockham stage when P = 32 NS: a radix-32 butterfly per pair of
// lanes, so a length 16^k * 2 transform needs no separate radix-2 pass
// through shared memory.  With r = 2m + h, lane h of the pair (h = t & 1)
// takes the inputs r = 2m + h, twiddles them by w^{k r} = w^{2km} w^{kh}, and
// forms Y_h[q] = sum_m v_m e^{DIR 2 pi i m q / 16}; the outputs are
//   X[q + 16 p] = sum_h e^{DIR 2 pi i h (q + 16 p) / 32} w^{kh} Y_h[q],
// a radix-2 butterfly across the pair (one shuffle per value): lane h
// finishes q in [8h, 8h + 8) for p = 0, 1.
template <typename R, int DIR, int P, int NS, class L, class S>
__device__ __forceinline__ void fft_stage_r32(int t, const cpx<R>* __restrict__ tw, const L& load, const S& store) {
    static_assert(NS * 32 == P, "radix-32 stage must be the last one");
    const int j = t >> 1, h = t & 1;        // butterfly j = k < NS
    const int k = j;
    cpx<R> v[16];
    if constexpr (is_smem_io<L>::value && (2 * NS) % 16 == 0) {
        const int pb = padi(j + h * NS);
        constexpr int ST = 2 * NS + (2 * NS) / 16;
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = load.at(pb, m * ST);
    } else {
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = load(j + (2 * m + h) * NS);
    }
    // the stage's table row k: w^{2km} for m = 1, 2, 3, 4, 8, 12, then w^k
    const cpx<R>* T = tw + tw32_offset(P) + 8 * k;
    cpx<R> wk, unused;
    tw_pair<R>(T + 6, wk, unused);
    if (DIR > 0) wk.y = -wk.y;
    if constexpr (NS > 1) {
        // w^{2km} = w^{2k(4a+b)} as in fft_stage
        cpx<R> wb[4], wa[4];
        tw_pair<R>(T, wb[1], wb[2]);
        tw_pair<R>(T + 2, wb[3], wa[1]);
        tw_pair<R>(T + 4, wa[2], wa[3]);
        if (DIR > 0) {
#pragma unroll
            for (int q = 1; q < 4; ++q) { wb[q].y = -wb[q].y; wa[q].y = -wa[q].y; }
        }
#pragma unroll
        for (int m = 1; m < 16; ++m) {
            const int qa = m >> 2, qb = m & 3;
            cpx<R> w;
            if (qa == 0) w = wb[qb];
            else if (qb == 0) w = wa[qa];
            else w = cmul(wa[qa], wb[qb]);
            v[m] = cmul(v[m], w);
        }
    }
    dft_small<DIR, 16>(v);
    // Z_h[q] = w^{h (k + q NS)} Y_h[q] = w^{hk} e^{DIR 2 pi i h q / 32} Y_h[q] (NS = P/32;
    // the identity for h = 0): one table load and compile-time constants
    if (h) {
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = cmul(v[q], wk);
    }
    mul_w32_sel<DIR, 0>(v, h != 0);
    __syncthreads();                        // every input of the stage is read before any store
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const cpx<R> send = h ? v[i] : v[8 + i];
        const cpx<R> own = h ? v[8 + i] : v[i];
        cpx<R> recv;
        recv.x = __shfl_xor_sync(0xffffffffu, send.x, 1);
        recv.y = __shfl_xor_sync(0xffffffffu, send.y, 1);
        const cpx<R> z0 = h ? recv : own;   // Z_0[8h + i]
        const cpx<R> z1 = h ? own : recv;   // Z_1[8h + i]
        const int q = 8 * h + i;
        store(k + q * NS, mk<R>(z0.x + z1.x, z0.y + z1.y));
        store(k + (q + 16) * NS, mk<R>(z0.x - z1.x, z0.y - z1.y));
    }
    __syncthreads();
}

// Stages NS, 16 NS, ... of a length-P transform: radix 16 while it fits; a
// remainder of 2 is merged into the last radix-16 stage (radix 32 across lane
// pairs), a remainder of 4 or 8 is one more stage.  `load` feeds the first of
// them, `store` takes the last one's outputs (natural order); the others go
// through `buf`.
template <typename R, int DIR, int P, int NS, bool FUSE2, class L, class S>
__device__ __forceinline__ void fft_from(cpx<R>* buf, int t, const cpx<R>* __restrict__ tw, const L& load,
                                         const S& store) {
    constexpr int RAD = (NS * 16 <= P) ? 16 : P / NS;
    if constexpr (NS * RAD == P) {
        fft_stage<R, DIR, RAD, P, NS>(t, tw, load, store);
    } else if constexpr (FUSE2 && NS * 32 == P) {
        fft_stage_r32<R, DIR, P, NS>(t, tw, load, store);
    } else {
        fft_stage<R, DIR, RAD, P, NS>(t, tw, load, SmemStore<R>{buf});
        fft_from<R, DIR, P, NS * RAD, FUSE2>(buf, t, tw, SmemLoad<R>{buf}, store);
    }
}

// Unscaled length-P complex DFT (DIR = -1: e^{-2 pi i jk/P}, DIR = +1: e^{+...})
// with input x[j] = load(j) and output X[k] handed to store(k, X[k]);
// tw is the twiddle table laid out as tw_entries(P) above.  FUSE2 = false keeps a remainder of 2 as its own
// stage (for store functors heavy enough that the radix-32 stage spills).  Every thread of the block must call it (it
// synchronises the block); inputs read from `buf` must have been written and
// synchronised before the call.
template <typename R, int DIR, int P, bool FUSE2 = true, class L, class S>
__device__ __forceinline__ void block_fft(cpx<R>* buf, int t, const cpx<R>* __restrict__ tw, const L& load,
                                          const S& store) {
    fft_from<R, DIR, P, 1, FUSE2>(buf, t, tw, load, store);
}

// Hint to the bulk-copy engine to bring [p, p + bytes) into L2 (no wait, no
// completion event).  The range is narrowed to 16-byte boundaries inside it,
// as the instruction requires, so it never reaches past the caller's range.
__device__ __forceinline__ void l2_prefetch(const void* p, size_t bytes) {
    const uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15;
    const uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
    if (e > a) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)(e - a)) : "memory");
}

// order-preserving bit pattern of a non-negative double (for atomicMax)
__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

}  // namespace pide
