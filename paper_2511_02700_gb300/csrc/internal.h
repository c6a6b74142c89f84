// Host-side interface between the pide2d translation units: argument blocks
// of the kernels and their launchers.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace pide {

// State element: FP64 mode keeps double; FP32-bulk mode keeps a double-float
// pair (hi, lo) in a float2 so every state update runs on FP32 units.
template <typename R> struct state_t;
template <> struct state_t<float> { using type = float2; };
template <> struct state_t<double> { using type = double; };
template <typename R> using St = typename state_t<R>::type;

// spectrum column groups: 16 bytes of complex values per (group, row)
template <typename R> __host__ __device__ constexpr int cgroup() { return 16 / (2 * (int)sizeof(R)); }
// DST column groups: 16 bytes of real values per (group, row)
template <typename R> __host__ __device__ constexpr int rgroup() { return 16 / (int)sizeof(R); }
// bytes of one (group, row) entry of the spectrum and of the DST buffer
template <typename R> constexpr size_t cgroup_bytes() { return (size_t)cgroup<R>() * 2 * sizeof(R); }
template <typename R> constexpr size_t rgroup_bytes() { return (size_t)rgroup<R>() * sizeof(R); }
// spectrum column groups of a length-P transform (P/2 + 1 columns)
template <typename R> constexpr int spectrum_groups(int P) { return (P / 2 + 1 + cgroup<R>() - 1) / cgroup<R>(); }

enum FwdMode { FWD_FULL = 0, FWD_FULL0 = 1, FWD_INCR = 2, FWD_WEIGHTS = 3, FWD_DIFF = 4 };
enum ColMode { COL_FULL = 0, COL_INCR = 1 };
enum InvMode { INV_FULL = 0, INV_INCR = 1, INV_OUT = 2 };

struct Geometry {
    int N, P;          // grid and padded transform length (P = 2N)
    int rows;          // rows of the spectrum buffer (P + 2)
    int ng;            // spectrum column groups
    int nge;           // DST column groups (N / rgroup)
    int ldS;           // pitch (elements) of state fields, (N+1) rows
    int ldR;           // pitch (elements) of R fields, (N+1) rows
    int eoff;          // index offset of node m in the exp tables (N/2 + 3)
};

template <typename R> struct FwdArgs {
    Geometry g;
    int mode;
    const St<R>* Y;          // FULL/FULL0/DIFF: field whose interior is transformed
    const St<R>* Yref;       // DIFF: the interior transformed is Y - Yref
    const R* D;              // INCR: increment field (ring zero)
    const double* omega;     // WEIGHTS: N x N weights [l2][l1]
    const R* E1; const R* E2;// e^{s_m} tables (transform precision)
    R Kd;                    // K e^{-r tau} for the far field
    R Kd_prev, dKd;          // DIFF: the halo is g(tau) - g(tau_prev); dKd = Kd - Kd_prev (rounded from FP64)
    int payoff;
    void* S;                 // spectrum out (cpx<R>, or cpx<double> for WEIGHTS)
    int pair0, npairs;       // row pairs (rho = 2 (pair0 + p), +1)
    const void* tw;          // twiddles of the transform precision
};

template <typename R> struct ColArgs {
    Geometry g;
    int mode;
    void* S;                 // cpx<R> spectrum, in place
    const void* Wh;          // cpx<R> conj(w^)/P^2 (FULL) or with the midpoint factors (INCR), [group][k2][c]
    int rlo, rhi;            // spectrum rows holding data
    const void* tw;
};

template <typename R> struct InvArgs {
    Geometry g;
    int mode;
    int do_resid;
    const int* conv_flag;    // device flag; when set, do_resid = !*conv_flag (device-side loop)
    const void* S;
    St<R>* BY;               // FULL: set (BV + the sweep when BV is given), INCR: accumulate
    const St<R>* BV;         // FULL: B_w V^{n-1} when the sweep transformed Y - V^{n-1} (else NULL)
    St<R>* const* BYind;     // device-side loop: BY is read from *BYind
    double* out;             // OUT: plain FP64 result field (pitch ldS)
    const St<R>* Y;          // FULL: Y^0 (with ring)
    const St<R>* W;          // FULL: W
    R* r;                    // (unused) residual field
    const R* D;              // INCR: increment field
    R htt, cid, d11, d22, d12, rw;   // h_t theta, 1 + h_t theta r_w, a11/(2h^2), a22/(2h^2), a12/(4h^2), r_w
    R rw_lo;                 // r_w - rw (the low part of r_w in the transform precision)
    R* E;                    // DST rows output
    const void* tw;
};

template <typename R> struct ColSolveArgs {
    Geometry g;
    R* E;                    // row-DST modes, solved in place
    const R* sin2;           // sin^2(pi k / (2N)), k = 0..N
    R rc0, rc1, rc2;         // A_0's eigenvalues c0 + c1 sin2[k1] + c2 sin2[k2], rounded once on the host
    R rscale;                // 2/N, the row DST pair's normalisation
};

template <typename R> struct DstRowArgs {
    Geometry g;
    const R* E;
    St<R>* Y;
    St<R>* const* Yind;      // device-side loop: Y is read from *Yind (set per step on the device)
    R* D;                    // increment out (interior)
    void* resid;             // FP64 max of |D| / max(1, |Y|) (eq. 3.25), as unsigned 64-bit bits
    void* S;                 // spectrum rows of the increment (R2C), cpx<R>
    const void* tw;
};

template <typename R> struct PrepArgs {
    Geometry g;
    const St<R>* V[4];       // history, latest first
    int hcount;
    const St<R>* BV;
    St<R>* W;
    St<R>* Y;
    R* cz;                   // Z - V at interior nodes (R field, pitch ldR)
    R htm;                   // h_t (1 - theta)
    R rw, d11, d22, d12;     // r_w and D coefficients
    R rw_lo;                 // r_w - rw
    int o1, o2, nt;          // SL: first tap offsets, taps per axis (2 or 4)
    R w1[4], w2[4];          // SL weights per axis
    const double* E1d; const double* E2d;   // e^{s} in FP64
    const float* E1h; const float* E1l;     // e^{s} as double-float pairs (FP32-bulk far field)
    const float* E2h; const float* E2l;
    double Kd_prev, Kd_now;  // K e^{-r tau_{n-1}}, K e^{-r tau_n}
    float Kdp_h, Kdp_l, Kdn_h, Kdn_l;        // the same as double-float pairs
    int payoff;
};

// Multi-job launches: grid dimension y (z for the 2D node kernels) indexes
// the job, whose arguments are read from a device array.  Inside the
// fixed-point loop a job that has stopped skips its blocks.
struct JobsCtl {
    const int* conv;         // per job: 1 once its loop stopped (converged, kmax or non-finite)
    const int* kconv;        // per job: the iteration at which it stopped
    const int* iter;         // the current iteration, 1-based, on the device (written by the check kernel)
    int mode;                // 0: every job; 1: jobs still iterating; 2: those and the ones stopped at *iter
#ifdef __CUDACC__
    __device__ __forceinline__ bool skip(int j) const {
        if (mode == 0) return false;
        const int c = conv[j];
        if (mode == 1) return c != 0;
        return c != 0 && kconv[j] < *iter;
    }
#endif
};

// launchers (sweep.cu), explicitly instantiated for float and double
template <typename R> cudaError_t launch_row_forward(const FwdArgs<R>& a, cudaStream_t s);
template <typename R> cudaError_t launch_col(const ColArgs<R>& a, cudaStream_t s);
template <typename R> cudaError_t launch_row_inverse(const InvArgs<R>& a, cudaStream_t s);
template <typename R> cudaError_t launch_col_solve(const ColSolveArgs<R>& a, cudaStream_t s);
template <typename R> cudaError_t launch_dst_row(const DstRowArgs<R>& a, cudaStream_t s);
template <typename R> cudaError_t launch_prep(const PrepArgs<R>& a, cudaStream_t s);
// the adjoint's weight contraction: acc[k1][k2] += conj(X) A for the spectra of the
// midpoint field (SV, full rows) and of xi (SX, raw rows rlo..rhi-1), FP64 accumulator
// (P/2 + 1) x P; corr_finish (FP64 handles' instantiation) inverts it into the N x N lag
// array Cout [l2 + N/2][l1 + N/2]
template <typename R> cudaError_t launch_corr_col(const Geometry& g, const void* SV, const void* SX, int rlo, int rhi,
                                                 double* acc, const void* tw, cudaStream_t s);
template <typename R> cudaError_t launch_corr_finish(const Geometry& g, double* acc, double* Cout, const void* twd,
                                                    cudaStream_t s);
// row DST-I of an FP64 interior field (pitch g.ldS) into the DST buffer E
template <typename R> cudaError_t launch_row_dst(const Geometry& g, const double* src, R* E, const void* tw,
                                                cudaStream_t s);
// the same kernels over K jobs of one geometry (a0: any job's arguments, for the launch shape)
// (upb: FFT units per block, <= 0 for the single-job shape; capped at 512 threads)
template <typename R> cudaError_t launch_row_forward_jobs(const FwdArgs<R>& a0, const FwdArgs<R>* arr, int K,
                                                         JobsCtl jc, int upb, cudaStream_t s);
template <typename R> cudaError_t launch_col_jobs(const ColArgs<R>& a0, const ColArgs<R>* arr, int K, JobsCtl jc,
                                                 int upb, cudaStream_t s);
template <typename R> cudaError_t launch_row_inverse_jobs(const InvArgs<R>& a0, const InvArgs<R>* arr, int K,
                                                         JobsCtl jc, int upb, cudaStream_t s);
template <typename R> cudaError_t launch_col_solve_jobs(const ColSolveArgs<R>& a0, const ColSolveArgs<R>* arr, int K,
                                                     JobsCtl jc, int upb, cudaStream_t s);
template <typename R> cudaError_t launch_dst_row_jobs(const DstRowArgs<R>& a0, const DstRowArgs<R>* arr, int K,
                                                     JobsCtl jc, int upb, cudaStream_t s);
// the single-job units per block of the FFT kernels at transform length P (0 if P is unsupported)
int fft_units_per_block(int P, int prec_bytes);
template <typename R> cudaError_t launch_prep_jobs(const PrepArgs<R>& a0, const PrepArgs<R>* arr, int K,
                                                  bool explicit_part, cudaStream_t s);
// price-space jump operator (eqs. 3.12-3.17 on the paper's price grid); P x P transforms
template <typename R> cudaError_t launch_ps_tin(int P, int nin, int nx1, const int* s, const double* w,
                                               const double* V, R* A, cudaStream_t st);
template <typename R> cudaError_t launch_ps_rows_fwd(int P, const R* A, int nin, void* S, const void* tw,
                                                    cudaStream_t st);
template <typename R> cudaError_t launch_ps_col(int P, void* S, const void* Wh, int nin, int nout, const void* tw,
                                               cudaStream_t st);
template <typename R> cudaError_t launch_ps_rows_inv(int P, const void* S, int nout, double* By, int ldB,
                                                    const void* tw, cudaStream_t st);
cudaError_t launch_ps_tout(int nx1, int nout, const int* t, const double* u, const double* By, int ldB, double* out,
                           cudaStream_t st);
// price-space diffusion and the Krylov solve around it (price_space.cu), FP64
struct PsDiff {
    int n1;                  // nodes per axis
    const double* x;         // [n1] price nodes
    const double* a1;        // [n1][3] first-difference coefficients (row 0 zero, last row backward)
    const double* b2;        // [n1][3] second-difference coefficients (first and last rows zero)
    double A11, A12, A22;    // sigma_w sigma_w^T
};
cudaError_t launch_ps_diff(const PsDiff& d, const double* v, double alpha, double beta, const double* w, double gamma,
                           double* out, cudaStream_t s);
cudaError_t launch_ps_diag_inv(const PsDiff& d, double c0, double c1, double* dinv, cudaStream_t s);
cudaError_t launch_ps_axpy(size_t n, double a, const double* x, double b, const double* y, double c, const double* z,
                           const double* dinv, double* out, cudaStream_t s);
int ps_reduction_blocks();
struct PsDots {
    const double* x[3];
    const double* y[3];
};
cudaError_t launch_ps_dots(size_t n, int nd, const PsDots& dp, double* part, double* res, cudaStream_t s);
// one Jacobi-preconditioned BiCGSTAB solve of (c0 I - c1 D) X = B with its
// scalars in device memory: record_ps_bicg builds it as a CUDA graph (set-up,
// then a while-node over the iterations), so a solve is one graph launch
struct PsBicg {
    double rho, rho_new, alpha, omega;
    double rn, lim;          // the residual norm and the stopping level 1e-13 |B|
    int it, done;            // iterations done; 1 once the half-step residual met lim
};
struct PsBicgArgs {
    PsDiff d;
    size_t n;
    double c0, c1;
    const double* B;
    double* X;               // the start in, the solution out
    double *r, *rh, *p, *v, *y, *s, *z, *t;
    const double* dinv;      // the Jacobi preconditioner
    double* part;            // ps_reduction_blocks() x 3 partial sums
    double* res;             // 3 doubles
    PsBicg* st;
    int maxit;
};
cudaError_t record_ps_bicg(cudaGraph_t g, cudaStream_t cap, const PsBicgArgs& a, const char** where);
cudaError_t launch_ps_maxrel(size_t n, const double* a, const double* b, double* part, double* res, cudaStream_t s);
cudaError_t launch_ps_sl(int n1, const int* s1, const double* w1, const int* s2, const double* w2, const double* Z,
                         double* W, cudaStream_t s);
// omega-hat: forward column FFT of the FP64 row spectra, written as cpx<RO>
template <typename RO> cudaError_t launch_weights_col(const Geometry& g, const void* Sd, void* Wh, void* Whi,
                                                       const void* twd, cudaStream_t s);
template <typename R> cudaError_t launch_state_from_double(const Geometry& g, const double* src, int ld_src,
                                                          St<R>* dst, cudaStream_t s);
template <typename R> cudaError_t launch_greeks(const Geometry& g, const St<R>* V, const double* E1d,
                                                const double* E2d, double h, int which, double* out, int ldo,
                                                cudaStream_t s);
template <typename R> cudaError_t launch_state_to_double(const Geometry& g, const St<R>* src, double* dst,
                                                        int ld_dst, cudaStream_t s);

// device-side fixed-point loop control (loop_ctl.cu)
struct FpCtl {
    int k;                   // iterations of the current theta step (reset per step)
    int conv;                // 1 once the eq. 3.25 test passed in the current step
    int total;               // iterations over all steps run by the device loop
    int step_k;              // iterations of the current time step (the damped step has four theta steps)
    int max_step;            // largest per-time-step count
    int last_step_k;         // count of the last completed time step
    int nonconv;             // theta steps that stopped at kmax or on a non-finite residual
    int substeps;            // theta steps run by the device loop
    double last_resid;       // last eq. 3.25 quantity
    double step_resid;       // its value at the end of the last completed time step
    void* Y;                 // fields of the current theta step (the loop graph reads them here)
    void* BY;
    int step_end;            // 1 if the current theta step ends a time step
};
// discrete adjoint (adjoint.cu)
struct SlWeights {
    double w1[4], w2[4];     // departure weights per axis (eq. 3.22)
    double dw1[4], dw2[4];   // their derivatives with respect to the shift in cells
};
template <typename R> struct SlShiftArgs {
    const St<R>* mu;         // adjoint of V^s
    const St<R>* V;          // V^{s-1} (ring included)
    const St<R>* BV;         // B_w V^{s-1}
    double htm, rw, d11, d22, d12;
    int o1, o2, nt;
    SlWeights w;
    const double* E1d; const double* E2d;
    double Kd_prev;          // K e^{-r tau_{s-1}}
    int payoff;
};
int adjoint_dot_blocks(int N);
cudaError_t launch_flip_weights(const double* om, double* out, int N, cudaStream_t s);
cudaError_t launch_central_difference(const double* a, const double* b, double scale, double* out, size_t n,
                                      cudaStream_t s);
template <typename R> cudaError_t launch_sl_transpose(const Geometry& g, const St<R>* mu, St<R>* nu, int o1, int o2,
                                                     int nt, const SlWeights& w, cudaStream_t s);
template <typename R> cudaError_t launch_adj_combine(const Geometry& g, const St<R>* nu, const double* bnu,
                                                    St<R>* lam, double htm, double rw, double d11, double d22,
                                                    double d12, cudaStream_t s);
template <typename R> cudaError_t launch_adj_xi(const Geometry& g, const St<R>* mu, const St<R>* nu, double* xi,
                                               double* pend, double htt, double htm_s, cudaStream_t s);
template <typename R> cudaError_t launch_dots_state(const Geometry& g, const double* xi, const St<R>* V, double* part,
                                                   double* acc, double scale, cudaStream_t s);
cudaError_t launch_dot_field(const Geometry& g, const double* xi, const double* out, double* part, double* acc,
                             cudaStream_t s);
// *acc += sum_i a[i] b[i], i < n (adjoint_dot_blocks(g.N) partials in part)
cudaError_t launch_dot_plain(const Geometry& g, const double* a, const double* b, size_t n, double* part, double* acc,
                             cudaStream_t s);
template <typename R> cudaError_t launch_field_to_r(const Geometry& g, const double* src, R* dst, cudaStream_t s);
template <typename R> cudaError_t launch_sl_shift_dots(const Geometry& g, const SlShiftArgs<R>& a, double* part,
                                                      double* acc, double scale, cudaStream_t s);

template <typename R> cudaError_t launch_fp_check(const void* resid, FpCtl* ctl, double tol, int kmax,
                                                 unsigned long long cond_handle, cudaStream_t s);
cudaError_t launch_fp_tally(FpCtl* ctl, cudaStream_t s);

// multi-job loop control (loop_ctl.cu)
struct JobCheck {
    const void* resid;       // the job's FP64 eq. 3.25 maximum (reset to 0 after each read)
    double tol;
    int kmax;
    int pad;
};
struct JobsState {
    int* conv;               // [K] 1 once the job's loop stopped
    int* kconv;              // [K] iteration at which it stopped
    int* kcount;             // [K] iterations of the current theta step
    int* nonconv;            // [K] 1 if a theta step stopped without meeting the tolerance
    double* last;            // [K] last eq. 3.25 quantity
    int* active;             // jobs still iterating after the last check
    int* iter;               // the current iteration of the theta step (1-based after the first check)
    // statistics over the whole time loop, per job
    int* it_total;           // [K] fixed-point iterations
    int* it_step;            // [K] iterations of the current time step (the damped step has four theta steps)
    int* it_max;             // [K] largest per-time-step count
    int* step;               // theta steps done (one counter for the chunk)
};
// resets the per-job stopping state and arms the graph condition `inner` of the iteration loop
template <typename R> cudaError_t launch_jobs_reset(int K, const JobCheck* jc, JobsState st, unsigned long long inner,
                                                  cudaStream_t s);
// the stopping rule of every job after iteration *st.iter + 1 (incremented here); clears the
// graph condition `cond` when no job iterates any more or kmax_all iterations were run
cudaError_t launch_jobs_check(int K, const JobCheck* jc, JobsState st, int kmax_all, unsigned long long cond,
                              cudaStream_t s);
// dst (bytes) = blobs + (*st.step) * bytes: the argument arrays of the chunk's current theta step
cudaError_t launch_step_select(const void* blobs, size_t bytes, JobsState st, void* dst, cudaStream_t s);
// end of a theta step: fold each job's count into the statistics, advance *st.step, clear the
// graph condition `cond` after `steps` theta steps; step_end[t] = 1 if theta step t ends a time step
cudaError_t launch_step_tally(int K, JobsState st, const int* step_end, int steps, unsigned long long cond,
                              cudaStream_t s);
cudaError_t launch_fp_setup(FpCtl* ctl, void* Y, void* BY, int step_end, cudaStream_t s);

// precompute (precompute.cu)
struct LevyParams {
    double alpha, nu, c1, logpref, Ri11, Ri12, Ri22, b1, b2;  // l(z) pieces
    double pref0;            // delta / (pi sqrt(det rho))
    double gamma_nu;         // Gamma(nu)
    // ln(e^x K_nu(x)) at u = ku0 + i / kidu, i < kn (NULL: no table)
    const double* ktab;
    double ku0, kidu;
    int kn;
};
constexpr int kKtabMax = 4096;          // entries of the K_nu table (after the quadrature nodes)
cudaError_t launch_ktab(double nu, double u0, double du, int n, double* tab, cudaStream_t s);
struct WeightJob {
    int N;
    double h;
    int M2;                  // z_II / h
    const double* gl_near_x; const double* gl_near_w; int n_near;
    const double* gl_far_x; const double* gl_far_w; int n_far;
    const double* gl_vfar_x; const double* gl_vfar_w; int n_vfar;
};
cudaError_t launch_weights(const LevyParams& L, const WeightJob& j, double* omega, double* partials,
                           int* nblocks, cudaStream_t s);
// the R_I moment (eq. 3.3): blocks of the quadrature and the doubles of its buffer
// (three moments, one spare, then the blocks' partial sums)
constexpr int kMomentBlocks = 64;
constexpr size_t moment_doubles() { return 4 + 3 * (size_t)kMomentBlocks; }
cudaError_t launch_moment(const LevyParams& L, double H, const double* glx, const double* glw, int ngl,
                          double tsh, double* out3, cudaStream_t s);
cudaError_t launch_finalize(const double* partials, int nblocks, const double* moment, double r,
                            const double* sigma_cov, double* params, cudaStream_t s);
cudaError_t launch_tables(int N, double s_lo1, double s_lo2, double h, double* E1d, double* E2d,
                          float* E1f, float* E2f, float* E1l, float* E2l, double* sin2, cudaStream_t s);
template <typename R> cudaError_t launch_twiddles(int P, void* tw, cudaStream_t s);
template <typename R> cudaError_t launch_payoff(const Geometry& g, const double* E1d, const double* E2d,
                                               double s_lo1, double s_lo2, double h, double K, int payoff,
                                               const double* glx, const double* glw, int ngl,
                                               St<R>* V, cudaStream_t s);
template <typename R> cudaError_t launch_ring(const Geometry& g, const double* E1d, const double* E2d,
                                             double Kd, int payoff, St<R>* Y, cudaStream_t s);

}  // namespace pide
