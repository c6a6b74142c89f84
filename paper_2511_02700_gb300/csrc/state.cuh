// State arithmetic.  FP64 mode: plain double.  FP32-bulk mode: a
// double-float pair (hi, lo) with value hi + lo, updated only by adding an
// FP32 increment (Knuth's error-free two-sum followed by a renormalising
// fast two-sum), and read back either as an FP32 value or as an FP32
// difference of two nearby states.  This keeps ~48 significant bits in
// the stored solution while all arithmetic runs on the FP32 pipes.
#pragma once

#include <cuda_runtime.h>

namespace pide {

__device__ __forceinline__ float2 st_add(float2 a, float b) {
    const float s = a.x + b;
    const float bb = s - a.x;
    float e = (a.x - (s - bb)) + (b - bb);
    e += a.y;
    const float hi = s + e;
    const float lo = e - (hi - s);
    return make_float2(hi, lo);
}
__device__ __forceinline__ double st_add(double a, double b) { return a + b; }

__device__ __forceinline__ float st_diff(float2 a, float2 b) { return (a.x - b.x) + (a.y - b.y); }
__device__ __forceinline__ double st_diff(double a, double b) { return a - b; }

__device__ __forceinline__ float st_r(float2 a) { return a.x + a.y; }
__device__ __forceinline__ double st_r(double a) { return a; }

__device__ __forceinline__ double st_dbl(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ double st_dbl(double a) { return a; }

template <typename S> __device__ __forceinline__ S st_make(double v);
template <> __device__ __forceinline__ float2 st_make<float2>(double v) {
    const float hi = __double2float_rn(v);
    return make_float2(hi, __double2float_rn(v - (double)hi));
}
template <> __device__ __forceinline__ double st_make<double>(double v) { return v; }

template <typename S, typename R> __device__ __forceinline__ S st_from_r(R v);
template <> __device__ __forceinline__ float2 st_from_r<float2, float>(float v) { return make_float2(v, 0.f); }
template <> __device__ __forceinline__ double st_from_r<double, double>(double v) { return v; }

// B_w V - r_w V at a node, from the state values bv = (B_w V)(s) and v = V(s)
// and r_w = rh + rl.  Both products are ~sum(w) |V|, so in FP32-bulk mode the
// difference is formed in double-float arithmetic: rh * v.x = p + pe exactly
// (FMA), and bv.x - p is exact when the two are within a factor of two
// (Sterbenz), which is the cancelling case.
__device__ __forceinline__ float jump_gen(float2 bv, float2 v, float rh, float rl) {
    const float p = rh * v.x;
    const float pe = fmaf(rh, v.x, -p);
    const float t = bv.x - p;
    return t + ((bv.y - pe) - (rh * v.y + rl * v.x));
}
__device__ __forceinline__ double jump_gen(double bv, double v, double rh, double rl) { return bv - (rh + rl) * v; }

// far field g(s, tau): the payoff with the strike discounted, Kd = K e^{-r tau}
template <typename R>
__device__ __forceinline__ R far_value(int payoff, R Kd, R e1, R e2) {
    if (payoff == 0) return fmax(Kd - R(0.5) * (e1 + e2), R(0));
    if (payoff == 1) return fmax(R(0.5) * (e1 + e2) - Kd, R(0));
    return fmax(Kd - e1, R(0));
}

// The far field g(s, tau) as a double-float pair from double-float inputs: e^{s1}
// = e1h + e1l, e^{s2} = e2h + e2l, K e^{-r tau} = kh + kl.  Knuth's two-sum keeps
// every sum exact to about 48 bits, so the value matches the FP64 evaluation to
// the pair's precision without an FP64 instruction.
__device__ __forceinline__ float2 df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return make_float2(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ float2 df_norm(float hi, float lo) {
    const float s = hi + lo;
    return make_float2(s, lo - (s - hi));
}
__device__ __forceinline__ float2 far_value_df(int payoff, float kh, float kl, float e1h, float e1l, float e2h,
                                               float e2l) {
    float ah, al;                            // the payoff's argument a: (e1 + e2)/2, or e1
    if (payoff == 2) {
        ah = e1h;
        al = e1l;
    } else {
        const float2 t = df_two_sum(e1h, e2h);
        const float2 u = df_norm(t.x, t.y + (e1l + e2l));
        ah = 0.5f * u.x;
        al = 0.5f * u.y;
    }
    // g = k - a (puts) or a - k (call), then max(g, 0)
    const float sgn = payoff == 1 ? -1.0f : 1.0f;
    const float2 d = df_two_sum(sgn * kh, -sgn * ah);
    const float2 g = df_norm(d.x, d.y + sgn * (kl - al));
    if (g.x < 0.0f || (g.x == 0.0f && g.y <= 0.0f)) return make_float2(0.0f, 0.0f);
    return g;
}

// g(s, tau) - g(s, tau_prev) with k0 = K e^{-r tau}, k1 = K e^{-r tau_prev} and
// dk = k0 - k1 rounded once from FP64: piecewise in the payoff's argument a,
// so no difference of two nearby far-field values is rounded
template <typename R>
__device__ __forceinline__ R far_diff(int payoff, R k0, R k1, R dk, R e1, R e2) {
    const R a = payoff == 2 ? e1 : R(0.5) * (e1 + e2);
    const R lo = fmin(k0, k1), hi = fmax(k0, k1);
    if (payoff == 1) {                      // call: max(a - k, 0)
        if (a <= lo) return R(0);
        if (a >= hi) return -dk;
        return k0 < k1 ? a - k0 : k1 - a;
    }
    if (a >= hi) return R(0);               // puts: max(k - a, 0)
    if (a <= lo) return dk;
    return k0 > k1 ? k0 - a : a - k1;
}

}  // namespace pide
