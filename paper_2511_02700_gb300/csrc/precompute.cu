// Precomputation of Algorithm 1 on the device, in FP64: the NTS Levy
// density (Sec. 4), the modified-midpoint weights (eq. 3.5), the
// artificial-diffusion moment over R_I (eq. 3.3), the rates of eq. 3.6,
// the payoff with cell averaging (eq. 3.18) and small lookup tables.
//
// Bessel K_nu.  K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt, evaluated
// with the trapezoidal rule, which converges geometrically for this
// analytic integrand (Gil, Segura, Temme, "Numerical Methods for Special
// Functions", SIAM 2007, Sec. 5.4).  The step h = min(1/6, 0.6/sqrt(x))
// keeps the strip-of-analyticity error below 1e-16 relative for x up to
// several hundred (the integrand narrows like 1/sqrt(x)); the exponentially
// scaled form e^x K_nu(x) is summed so nothing underflows.
//
// R_I moment.  int_{[-H,H]^2} z z^T l(z) dz: four triangles with apex at
// the origin, z = rho (e + t f), dz = rho drho dt; the rho integral (with
// its rho^(1-2 alpha) apex behaviour) uses the tanh-sinh rule of Takahasi
// and Mori (1974), the edge integral Gauss-Legendre.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "internal.h"
#include "state.cuh"

namespace pide {

// e^x K_nu(x), x > 0
__device__ double bessel_k_scaled(double nu, double x) {
    const double h = fmin(1.0 / 6.0, 0.6 / sqrt(x));
    double s = 0.5;
    for (int k = 1; k < 4000; ++k) {
        const double t = k * h;
        const double sh = sinh(0.5 * t);
        const double term = exp(-2.0 * x * sh * sh) * cosh(nu * t);
        s += term;
        if (term < 1e-18 * s) break;
    }
    return s * h;
}


// ln(e^x K_nu(x)): 8-point Lagrange interpolation in u = ln x on the
// model's table (nodes base..base+7 around u), else the trapezoidal sum.  In u
// the function is smooth (slope -nu for small x, -1/2 for large x); at a node
// spacing of 0.01 the interpolation error is below 1e-14 absolute, the
// rounding level of the sum it replaces.
__device__ double log_ek(const LevyParams& L, double x) {
    if (L.ktab) {
        const double f = (log(x) - L.ku0) * L.kidu;
        const int base = (int)floor(f) - 3;
        if (base >= 0 && base + 7 < L.kn) {
            const double t = f - (double)base;             // in [3, 4)
            // l_a(t) = prod_{b != a} (t - b) / (a - b) = pre_a suf_a c_a
            constexpr double c[8] = {-1.0 / 5040.0, 1.0 / 720.0, -1.0 / 240.0, 1.0 / 144.0,
                                     -1.0 / 144.0,  1.0 / 240.0, -1.0 / 720.0, 1.0 / 5040.0};
            double pre[8], suf[8];
            pre[0] = 1.0;
#pragma unroll
            for (int a = 1; a < 8; ++a) pre[a] = pre[a - 1] * (t - (double)(a - 1));
            suf[7] = 1.0;
#pragma unroll
            for (int a = 6; a >= 0; --a) suf[a] = suf[a + 1] * (t - (double)(a + 1));
            const double* T = L.ktab + base;
            double v = 0.0;
#pragma unroll
            for (int a = 0; a < 8; ++a) v += (pre[a] * suf[a] * c[a]) * T[a];
            return v;
        }
    }
    return log(bessel_k_scaled(L.nu, x));
}

// x^nu K_nu(x), bounded as x -> 0 (limit 2^(nu-1) Gamma(nu))
__device__ double xnu_knu(const LevyParams& L, double x) {
    if (x < 1e-8) return exp2(L.nu - 1.0) * L.gamma_nu;
    return exp(L.nu * log(x) - x + log_ek(L, x));
}

// l(z), Sec. 4
__device__ double levy_density(const LevyParams& L, double z1, double z2) {
    const double zn = sqrt(L.Ri11 * z1 * z1 + 2.0 * L.Ri12 * z1 * z2 + L.Ri22 * z2 * z2);
    const double x = L.c1 * zn;
    return exp(L.logpref + log_ek(L, x) - x - L.nu * log(zn) + L.b1 * z1 + L.b2 * z2);
}

// the table of log_ek: ln(e^x K_nu(x)) at x = e^{u0 + i du}, i < n.  One warp per
// entry: lane l sums the trapezoidal terms k = l + 1 + 32 j of bessel_k_scaled
// until they fall below 1e-18 of its partial sum (past the integrand's peak they
// only decrease), then the warp adds the lane sums
__global__ void k_ktab(double nu, double u0, double du, int n, double* tab) {
    const int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;                               // uniform across the warp
    const double x = exp(u0 + (double)i * du);
    const double h = fmin(1.0 / 6.0, 0.6 / sqrt(x));
    double s = 0.0;
    for (int k = lane + 1; k < 4000; k += 32) {
        const double t = k * h;
        const double sh = sinh(0.5 * t);
        const double term = exp(-2.0 * x * sh * sh) * cosh(nu * t);
        s += term;
        if (term < 1e-18 * s || term == 0.0) break;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) tab[i] = log((0.5 + s) * h);
}

// R_II cells up to this ||z_l||_inf / h (the 10-point rule, 100 nodes) take a
// warp each (k_weights_near); the cells beyond, with 36 or 16 nodes, are
// numerous enough to fill the GPU one thread per cell, at full lane use
__host__ __device__ __forceinline__ int weights_warp_zone(const WeightJob& j) { return j.M2 < 8 ? j.M2 : 8; }

// the R_II cell integral at node (a, b) of its product rule (eq. 3.5 with the
// |z|^2 factor of the modified midpoint rule)
__device__ __forceinline__ double rii_node(const LevyParams& L, double c1, double c2, double h, const double* gx,
                                           const double* gw, int a, int b) {
    const double za = c1 + 0.5 * h * gx[a], zb = c2 + 0.5 * h * gx[b];
    return gw[a] * gw[b] * (za * za + zb * zb) * levy_density(L, za, zb);
}

// R_II cells with ||z_l||_inf / h in (2, weights_warp_zone]: one warp per cell of
// the square around the origin, the rule's 100 nodes strided over the lanes
// (at GB300's FP64 rate a cell's 100 density evaluations on one thread are the
// tail of k_weights otherwise); the lane sums are added in a fixed order
__global__ void k_weights_near(LevyParams L, WeightJob j, double* omega) {
    const int Z = weights_warp_zone(j);
    const int side = 2 * Z;
    const int wcell = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (wcell >= side * side) return;                 // uniform across the warp
    const int q2 = wcell / side, q1 = wcell - q2 * side;
    const int l1 = q1 - Z, l2 = q2 - Z;               // cells l = -Z .. Z - 1 around the origin
    const double inf = fmax(fabs(l1 + 0.5), fabs(l2 + 0.5));
    if (inf <= 2.0 || inf > (double)Z) return;
    const int n = j.n_near;                           // inf <= 8: the 10-point rule
    const double* gx = j.gl_near_x;
    const double* gw = j.gl_near_w;
    const double c1 = (l1 + 0.5) * j.h, c2 = (l2 + 0.5) * j.h;
    double acc = 0.0;
    for (int k = lane; k < n * n; k += 32) acc += rii_node(L, c1, c2, j.h, gx, gw, k / n, k - (k / n) * n);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        const int N = j.N;
        omega[(size_t)(l2 + N / 2) * N + (l1 + N / 2)] = acc * 0.25 * j.h * j.h / (c1 * c1 + c2 * c2);
    }
}

// ---------------------------------------------------------------------------
// weights, eq. 3.5; one thread per cell, per-block partial sums of
// (w, w (e^{z1} - 1), w (e^{z2} - 1)) for the deterministic final reduction
// ---------------------------------------------------------------------------
__global__ void k_weights(LevyParams L, WeightJob j, double* omega, double* partials) {
    const int N = j.N;
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    double w = 0.0, e1 = 0.0, e2 = 0.0;
    if (cell < N * N) {
        const int i2 = cell / N, i1 = cell - i2 * N;
        const int l1 = i1 - N / 2, l2 = i2 - N / 2;
        const double c1 = (l1 + 0.5) * j.h, c2 = (l2 + 0.5) * j.h;
        const double inf = fmax(fabs(l1 + 0.5), fabs(l2 + 0.5));   // ||z_l||_inf / h
        if (inf <= 2.0) {
            w = 0.0;                                               // R_I
        } else if (inf <= (double)weights_warp_zone(j)) {
            w = omega[cell];                                       // R_II near the origin: k_weights_near
        } else if (inf <= (double)j.M2) {                          // R_II
            // Gauss-Legendre order by distance from the singular origin (in
            // cells): 10 up to 8 cells, 6 up to 24 cells (or on coarse grids),
            // 4 beyond -- each within ~1e-14 relative of a 24-point rule
            const bool near = inf <= 8.0;
            const bool far = inf > 24.0 && N >= 1024;
            const int n = near ? j.n_near : (far ? j.n_vfar : j.n_far);
            const double* gx = near ? j.gl_near_x : (far ? j.gl_vfar_x : j.gl_far_x);
            const double* gw = near ? j.gl_near_w : (far ? j.gl_vfar_w : j.gl_far_w);
            double acc = 0.0;
            for (int a = 0; a < n; ++a) {
                const double za = c1 + 0.5 * j.h * gx[a];
                double inner = 0.0;
                for (int b = 0; b < n; ++b) {
                    const double zb = c2 + 0.5 * j.h * gx[b];
                    inner += gw[b] * (za * za + zb * zb) * levy_density(L, za, zb);
                }
                acc += gw[a] * inner;
            }
            w = acc * 0.25 * j.h * j.h / (c1 * c1 + c2 * c2);
        } else {                                                   // R_III
            w = levy_density(L, c1, c2) * j.h * j.h;
        }
        omega[cell] = w;
        e1 = w * expm1(c1);
        e2 = w * expm1(c2);
    }
    __shared__ double sw[256], s1[256], s2[256];
    sw[threadIdx.x] = w;
    s1[threadIdx.x] = e1;
    s2[threadIdx.x] = e2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sw[threadIdx.x] += sw[threadIdx.x + o];
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = sw[0];
        partials[3 * blockIdx.x + 1] = s1[0];
        partials[3 * blockIdx.x + 2] = s2[0];
    }
}

// ---------------------------------------------------------------------------
// eq. 3.3 moment over R_I = [-H, H]^2 (one block)
// ---------------------------------------------------------------------------
// kMomentBlocks blocks each sum a strided share of the nodes into part[3 b ..];
// k_moment_sum adds the partial sums in block order (deterministic)
__global__ void k_moment(LevyParams L, double H, const double* glx, const double* glw, int ngl, double tsh,
                         double* part) {
    const double pi = 3.141592653589793;
    const int kmax = (int)(6.5 / tsh);
    const int nts = 2 * kmax + 1;
    const int total = 4 * ngl * nts;
    double m11 = 0.0, m12 = 0.0, m22 = 0.0;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
        const int e = it / (ngl * nts);
        const int rem = it - e * ngl * nts;
        const int ti = rem / nts;
        const int k = rem - ti * nts - kmax;
        // tanh-sinh node on [0, H]: rho = H / (1 + e^{-u}), u = pi sinh(k tsh)
        const double tt = k * tsh;
        const double u = pi * sinh(tt);
        if (u < -740.0) continue;
        const double eu = exp(-fabs(u));
        const double rho = u < 0.0 ? H * eu / (1.0 + eu) : H / (1.0 + eu);
        const double wr = H * tsh * pi * cosh(tt) * eu / ((1.0 + eu) * (1.0 + eu));
        if (!(rho > 0.0) || !(wr > 0.0)) continue;
        const double t = glx[ti];
        double d1, d2;
        if (e == 0) { d1 = 1.0; d2 = t; }
        else if (e == 1) { d1 = -1.0; d2 = t; }
        else if (e == 2) { d1 = t; d2 = 1.0; }
        else { d1 = t; d2 = -1.0; }
        const double dn = sqrt(L.Ri11 * d1 * d1 + 2.0 * L.Ri12 * d1 * d2 + L.Ri22 * d2 * d2);
        const double ed = L.b1 * d1 + L.b2 * d2;
        // rho^3 d d^T l(rho d) = rho^(1-2 alpha) d d^T F, F = rho^(2 nu) l(rho d)
        const double F = L.pref0 * xnu_knu(L, L.c1 * dn * rho) * pow(dn, -2.0 * L.nu) * exp(rho * ed);
        const double g = wr * glw[ti] * pow(rho, 1.0 - 2.0 * L.alpha) * F;
        m11 += g * d1 * d1;
        m12 += g * d1 * d2;
        m22 += g * d2 * d2;
    }
    __shared__ double a[256], b[256], c[256];
    a[threadIdx.x] = m11;
    b[threadIdx.x] = m12;
    c[threadIdx.x] = m22;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            a[threadIdx.x] += a[threadIdx.x + o];
            b[threadIdx.x] += b[threadIdx.x + o];
            c[threadIdx.x] += c[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = a[0];
        part[3 * blockIdx.x + 1] = b[0];
        part[3 * blockIdx.x + 2] = c[0];
    }
}
__global__ void k_moment_sum(const double* part, int nb, double* out3) {
    if (threadIdx.x < 3) {
        double acc = 0.0;
        for (int b = 0; b < nb; ++b) acc += part[3 * b + threadIdx.x];
        out3[threadIdx.x] = acc;
    }
}

// params: [0] sum w, [1] r_w, [2] kappa1, [3] kappa2, [4] a11, [5] a12, [6] a22, [7] b1, [8] b2.
// One block; each thread sums a fixed strided subset of the block partials,
// then a fixed-order tree: the result does not depend on scheduling.
__global__ void k_finalize(const double* partials, int nblocks, const double* moment, double r, double s11,
                           double s12, double s22, double* params) {
    __shared__ double a[1024], b[1024], c[1024];
    double sw = 0.0, e1 = 0.0, e2 = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
        sw += partials[3 * i];
        e1 += partials[3 * i + 1];
        e2 += partials[3 * i + 2];
    }
    a[threadIdx.x] = sw;
    b[threadIdx.x] = e1;
    c[threadIdx.x] = e2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            a[threadIdx.x] += a[threadIdx.x + o];
            b[threadIdx.x] += b[threadIdx.x + o];
            c[threadIdx.x] += c[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double a11 = s11 + moment[0], a12 = s12 + moment[1], a22 = s22 + moment[2];
    params[0] = a[0];
    params[1] = r + a[0];
    params[2] = r - b[0];
    params[3] = r - c[0];
    params[4] = a11;
    params[5] = a12;
    params[6] = a22;
    params[7] = params[2] - 0.5 * a11;
    params[8] = params[3] - 0.5 * a22;
}

// e^{s_m} tables for m in [-N/2-3, N+N/2+3] and sin^2(pi k/(2N)), k = 0..N
__global__ void k_tables(int N, double s1, double s2, double h, double* E1d, double* E2d, float* E1f, float* E2f,
                         float* E1l, float* E2l, double* sin2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int len = 2 * N + 7;
    if (i < len) {
        const int m = i - (N / 2 + 3);
        const double a = exp(s1 + m * h), b = exp(s2 + m * h);
        E1d[i] = a;
        E2d[i] = b;
        E1f[i] = (float)a;
        E2f[i] = (float)b;
        // the FP32 rounding errors: (E1f, E1l) is e^{s} to about 48 bits
        E1l[i] = (float)(a - (double)E1f[i]);
        E2l[i] = (float)(b - (double)E2f[i]);
    }
    if (i <= N) {
        const double s = sinpi(0.5 * i / N);
        sin2[i] = s * s;
    }
}

template <typename R>
__global__ void k_twiddles(int P, cpx<R>* tw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tw_entries(P)) return;
    // exponent of w = e^{-2 pi i / P} held by entry i (layout in common.cuh)
    long long e = i;
    if (i >= P) {
        const int m16[8] = {1, 2, 3, 4, 8, 12, 0, 0};
        const int m32[8] = {2, 4, 6, 8, 16, 24, 1, 0};
        int off = P;
        bool r16 = false;
        for (int sp = 16; 16 * sp <= P; sp *= 16) {
            if (i < off + 8 * sp) {
                const int k = (i - off) / 8, slot = (i - off) % 8;
                e = (long long)k * (P / (16 * sp)) * m16[slot];
                r16 = true;
                break;
            }
            off += 8 * sp;
        }
        if (!r16) {
            const int k = (i - off) / 8, slot = (i - off) % 8;
            e = (long long)k * m32[slot];
        }
        e %= P;
    }
    double s, c;
    sincospi(2.0 * (double)e / P, &s, &c);
    tw[i] = mk<R>((R)c, (R)(-s));
}

// ---------------------------------------------------------------------------
// payoff with cell averaging (eq. 3.18) in log coordinates; ring = g(s, 0)
// ---------------------------------------------------------------------------
__device__ double inner_put_avg(double c, double a, double b) {
    if (c <= 0.0) return 0.0;
    const double up = fmin(b, log(2.0 * c));
    if (up <= a) return 0.0;
    return c * (up - a) - 0.5 * (exp(up) - exp(a));
}
__device__ double inner_call_avg(double c, double a, double b) {
    if (c <= 0.0) return 0.5 * (exp(b) - exp(a)) - c * (b - a);
    const double lo = fmax(a, log(2.0 * c));
    if (lo >= b) return 0.0;
    return 0.5 * (exp(b) - exp(lo)) - c * (b - lo);
}

__device__ double cell_avg(int payoff, double K, double a1, double b1, double a2, double b2, const double* gx,
                           const double* gw, int n) {
    const double area = (b1 - a1) * (b2 - a2);
    if (payoff == 2) {
        const double up = fmin(b1, log(K));
        const double v = up <= a1 ? 0.0 : K * (up - a1) - (exp(up) - exp(a1));
        return v * (b2 - a2) / area;
    }
    // break points of the s2 integrand where the kink leaves the cell through s1 = b1 or s1 = a1
    double pts[4];
    int np = 0;
    pts[np++] = a2;
    const double qb = 2.0 * K - exp(b1), qa = 2.0 * K - exp(a1);
    if (qb > 0.0) { const double tb = log(qb); if (tb > a2 && tb < b2) pts[np++] = tb; }
    if (qa > 0.0) { const double ta = log(qa); if (ta > a2 && ta < b2) pts[np++] = ta; }
    pts[np++] = b2;
    double v = 0.0;
    for (int s = 0; s + 1 < np; ++s) {
        const double lo = pts[s], hi = pts[s + 1];
        const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
        double acc = 0.0;
        for (int i = 0; i < n; ++i) {
            const double s2 = mid + half * gx[i];
            const double c = K - 0.5 * exp(s2);
            acc += gw[i] * (payoff == 0 ? inner_put_avg(c, a1, b1) : inner_call_avg(c, a1, b1));
        }
        v += acc * half;
    }
    return v / area;
}

template <typename R>
__global__ void k_payoff(Geometry g, const double* E1d, const double* E2d, double s1lo, double s2lo, double h,
                         double K, int payoff, const double* gx, const double* gw, int n, St<R>* V) {
    const int m1 = blockIdx.x * blockDim.x + threadIdx.x, m2 = blockIdx.y * blockDim.y + threadIdx.y;
    const int N = g.N;
    if (m1 > N || m2 > N) return;
    const double e1 = E1d[m1 + g.eoff], e2 = E2d[m2 + g.eoff];
    double v = far_value<double>(payoff, K, e1, e2);
    const bool interior = m1 >= 1 && m1 <= N - 1 && m2 >= 1 && m2 <= N - 1;
    if (interior) {
        const double a1 = s1lo + (m1 - 0.5) * h, b1 = a1 + h;
        const double a2 = s2lo + (m2 - 0.5) * h, b2 = a2 + h;
        bool crosses;
        if (payoff == 2) crosses = exp(a1) < K && K < exp(b1);
        else crosses = exp(a1) + exp(a2) < 2.0 * K && 2.0 * K < exp(b1) + exp(b2);
        if (crosses) v = cell_avg(payoff, K, a1, b1, a2, b2, gx, gw, n);
    }
    V[(size_t)m2 * g.ldS + m1] = st_make<St<R>>(v);
}

template <typename R>
__global__ void k_ring(Geometry g, const double* E1d, const double* E2d, double Kd, int payoff, St<R>* Y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = g.N;
    if (i > N) return;
    const int ms[4][2] = {{i, 0}, {i, N}, {0, i}, {N, i}};
    for (int s = 0; s < 4; ++s) {
        const int m1 = ms[s][0], m2 = ms[s][1];
        Y[(size_t)m2 * g.ldS + m1] = st_make<St<R>>(far_value<double>(payoff, Kd, E1d[m1 + g.eoff], E2d[m2 + g.eoff]));
    }
}

// ---------------------------------------------------------------------------
cudaError_t launch_weights(const LevyParams& L, const WeightJob& j, double* omega, double* partials, int* nblocks,
                           cudaStream_t s) {
    const int cells = j.N * j.N;
    const int nb = (cells + 255) / 256;
    *nblocks = nb;
    const int side = 2 * weights_warp_zone(j);
    k_weights_near<<<(side * side + 7) / 8, 256, 0, s>>>(L, j, omega);       // eight cells per block
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_weights<<<nb, 256, 0, s>>>(L, j, omega, partials);
    return cudaGetLastError();
}
cudaError_t launch_moment(const LevyParams& L, double H, const double* glx, const double* glw, int ngl, double tsh,
                          double* out3, cudaStream_t s) {
    // out3 holds the three moments, then kMomentBlocks x 3 partial sums (moment_doubles())
    double* part = out3 + 4;
    k_moment<<<kMomentBlocks, 256, 0, s>>>(L, H, glx, glw, ngl, tsh, part);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_moment_sum<<<1, 32, 0, s>>>(part, kMomentBlocks, out3);
    return cudaGetLastError();
}
cudaError_t launch_finalize(const double* partials, int nblocks, const double* moment, double r,
                            const double* sigma_cov, double* params, cudaStream_t s) {
    k_finalize<<<1, 1024, 0, s>>>(partials, nblocks, moment, r, sigma_cov[0], sigma_cov[1], sigma_cov[2], params);
    return cudaGetLastError();
}
cudaError_t launch_ktab(double nu, double u0, double du, int n, double* tab, cudaStream_t s) {
    k_ktab<<<(n + 3) / 4, 128, 0, s>>>(nu, u0, du, n, tab);      // four entries per block
    return cudaGetLastError();
}
cudaError_t launch_tables(int N, double s_lo1, double s_lo2, double h, double* E1d, double* E2d, float* E1f,
                          float* E2f, float* E1l, float* E2l, double* sin2, cudaStream_t s) {
    const int len = 2 * N + 7;   // nodes m = -N/2-3 .. N+N/2+3
    k_tables<<<(len + 255) / 256, 256, 0, s>>>(N, s_lo1, s_lo2, h, E1d, E2d, E1f, E2f, E1l, E2l, sin2);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_twiddles(int P, void* tw, cudaStream_t s) {
    k_twiddles<R><<<(tw_entries(P) + 255) / 256, 256, 0, s>>>(P, (cpx<R>*)tw);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_payoff(const Geometry& g, const double* E1d, const double* E2d, double s_lo1, double s_lo2,
                          double h, double K, int payoff, const double* glx, const double* glw, int ngl, St<R>* V,
                          cudaStream_t s) {
    const dim3 blk(32, 8), grd((g.N + 1 + 31) / 32, (g.N + 1 + 7) / 8);
    k_payoff<R><<<grd, blk, 0, s>>>(g, E1d, E2d, s_lo1, s_lo2, h, K, payoff, glx, glw, ngl, V);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_ring(const Geometry& g, const double* E1d, const double* E2d, double Kd, int payoff, St<R>* Y,
                        cudaStream_t s) {
    k_ring<R><<<(g.N + 1 + 127) / 128, 128, 0, s>>>(g, E1d, E2d, Kd, payoff, Y);
    return cudaGetLastError();
}

template cudaError_t launch_twiddles<float>(int, void*, cudaStream_t);
template cudaError_t launch_twiddles<double>(int, void*, cudaStream_t);
template cudaError_t launch_payoff<float>(const Geometry&, const double*, const double*, double, double, double,
                                          double, int, const double*, const double*, int, St<float>*, cudaStream_t);
template cudaError_t launch_payoff<double>(const Geometry&, const double*, const double*, double, double, double,
                                           double, int, const double*, const double*, int, St<double>*,
                                           cudaStream_t);
template cudaError_t launch_ring<float>(const Geometry&, const double*, const double*, double, int, St<float>*,
                                        cudaStream_t);
template cudaError_t launch_ring<double>(const Geometry&, const double*, const double*, double, int, St<double>*,
                                         cudaStream_t);

}  // namespace pide
