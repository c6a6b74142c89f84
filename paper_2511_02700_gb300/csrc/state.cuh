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

// far field g(s, tau): the payoff with the strike discounted, Kd = K e^{-r tau}
template <typename R>
__device__ __forceinline__ R far_value(int payoff, R Kd, R e1, R e2) {
    if (payoff == 0) return fmax(Kd - R(0.5) * (e1 + e2), R(0));
    if (payoff == 1) return fmax(R(0.5) * (e1 + e2) - Kd, R(0));
    return fmax(Kd - e1, R(0));
}

}  // namespace pide
