/*
 * pide2d -- C ABI of a GB300 (sm_103a) solver for two-asset European options
 * under an exponential Levy model with a bivariate Normal Tempered Stable
 * (NTS) jump measure, following Moda, in 't Hout, Vanmaele and Benth,
 * "Numerical valuation of European options under two-asset
 * infinite-activity exponential Levy models" (arXiv 2511.02700).
 *
 * What is computed (paper references in brackets):
 *   u_t = A_w u - r_w u on a uniform log-price grid   [Sec. 3.1, eq. 3.7]
 *   weights w_l of the modified midpoint rule          [eq. 3.5]
 *   artificial diffusion sigma_w sigma_w^T            [eq. 3.3, eq. 3.6]
 *   jump sum B_w V by zero-padded 2D FFT correlation  [eqs. 3.10-3.17]
 *   semi-Lagrangian theta-scheme with damping          [eqs. 3.19-3.23]
 *   fixed-point iteration, stop rule, extrapolation    [eqs. 3.24-3.26]
 *   in the order of Algorithm 1.
 *
 * Grid.  h = 2L/N, s_m = s_center - L + m h, m = 0..N per axis; the nodes
 * 0 and N carry the far-field value g(s, tau) (Dirichlet); the interior
 * nodes 1..N-1 are unknowns; ln S0 = s_center is node N/2.  The jump grid
 * is z_l = (l + 1/2) h, l = -N/2..N/2-1 (z_max^III = L).  Value arrays
 * exchanged through this ABI are (N+1) x (N+1) doubles, row-major
 * [m2][m1] (m1 fastest, the vector ordering of eq. 3.7).
 *
 * Memory and streams.  The caller owns every byte of device memory: it
 * passes one workspace of pide2d_workspace_bytes() bytes (device memory,
 * 256-byte aligned) to pide2d_create(), and the library never allocates
 * device memory.  All kernels run on the CUDA stream given at creation;
 * a call returns after the work it queued has finished only where stated.
 * The handle itself (a small host struct) is allocated by pide2d_create()
 * and freed by pide2d_destroy().
 *
 * Errors.  Every entry point returns a pide2d_status; nothing throws across
 * the ABI.  A non-OK status leaves a message readable by
 * pide2d_last_error().  After PIDE2D_ERR_CUDA the handle must only be
 * destroyed.
 */
#ifndef PIDE2D_H
#define PIDE2D_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PIDE2D_OK = 0,
    PIDE2D_ERR_ARG = 1,            /* invalid argument or model parameter      */
    PIDE2D_ERR_CUDA = 2,           /* a CUDA runtime call or launch failed     */
    PIDE2D_ERR_WORKSPACE = 3,      /* workspace NULL, too small or misaligned  */
    PIDE2D_ERR_NOT_CONVERGED = 4,  /* fixed-point cap reached (eq. 3.25 unmet) */
    PIDE2D_ERR_STATE = 5,          /* call not valid in the handle's state     */
    PIDE2D_ERR_UNSUPPORTED = 6     /* valid but not provided by this build     */
} pide2d_status;

/* payoff phi of the contract; g(s, tau) is phi with K replaced by K e^{-r tau} */
enum {
    PIDE2D_PUT_AVG = 0,     /* max(K - (S1 + S2)/2, 0): the paper's Sec. 4 option  */
    PIDE2D_CALL_AVG = 1,    /* max((S1 + S2)/2 - K, 0)                            */
    PIDE2D_PUT_ASSET1 = 2   /* max(K - S1, 0): single-asset reduction (tests)     */
};

/* Arithmetic of the transforms (FFT, DST, interpolation, stencils).  In both
 * modes the weights, sigma_w sigma_w^T and the rates are computed in FP64, the
 * eq. 3.25 stopping quantity that is compared with fp_tol is an FP64 value,
 * and the price is read out in FP64.  The state fields (V history, Y, W,
 * B_w Y) are FP64 in PIDE2D_FP64 mode and double-float pairs of FP32 values
 * (hi + lo, about 48 significant bits) in PIDE2D_FP32_BULK mode.  In
 * FP32-bulk mode the node that attains the eq. 3.25 maximum of a block is
 * chosen by FP32 ratios and its ratio is then evaluated in FP64, so the value
 * compared with fp_tol is within 2^-20 relative of the exact FP64 maximum. */
enum { PIDE2D_FP64 = 0, PIDE2D_FP32_BULK = 1 };

/* Spatial grid [Sec. 3.2, uniform in log price]. */
typedef struct {
    int n;                /* N: power of two, 8 <= N <= 4096 (both precisions)  */
    int n_z;              /* N_z: 0 or N/2 (z_max^III = L); other values ERR_ARG */
    double s_center[2];   /* ln S0 per axis (node N/2)                            */
    double half_width;    /* L > 0                                                */
    int sl_order;         /* semi-Lagrangian interpolation: 1 linear, 3 cubic     */
                          /* (0 selects 3, the paper's choice, Sec. 4)            */
    int precision;        /* PIDE2D_FP64 or PIDE2D_FP32_BULK                      */
} pide2d_grid;

/* NTS model in the paper's notation [Sec. 4, Table 2, Appendix A]. */
typedef struct {
    double alpha;         /* 0 <= alpha < 1 (tempered-stable index)               */
    double delta;         /* > 0                                                  */
    double lambda;        /* > 0                                                  */
    double eta[2];        /* Brownian drift of the subordinated BM                */
    double rho[3];        /* rho11, rho12, rho22: positive definite               */
    double r;             /* riskless rate                                        */
    double sigma_cov[3];  /* sigma sigma^T of eq. 2.3 (0 in all the paper's runs) */
} pide2d_model;

typedef struct {
    int payoff;           /* PIDE2D_PUT_AVG, PIDE2D_CALL_AVG, PIDE2D_PUT_ASSET1   */
    double strike;        /* K > 0                                                */
    double maturity;      /* T > 0                                                */
} pide2d_contract;

/* Optional settings; pass NULL for the defaults in brackets. */
typedef struct {
    int kmax;             /* fixed-point iteration cap per time step [100]        */
    int damping;          /* 1: first step = four theta = 1 steps of dt/4 [1]     */
    int host_loop;        /* 0: the fixed-point loop of each theta step runs on   */
                          /*    the device, as a CUDA graph whose while-node     */
                          /*    evaluates eq. 3.25 itself -- no host round trip  */
                          /*    per iteration [0];                               */
                          /* 1: the host reads the eq. 3.25 quantity after each  */
                          /*    iteration and launches the next one.  Tracing    */
                          /*    (pide2d_profile) always uses the host loop.      */
    int fixed_shapes;     /* batches only: 1 keeps `lanes` and the single-job   */
                          /*    launch shapes; 0 picks both per geometry group   */
                          /*    by timed trials on its first chunk [0]           */
} pide2d_options;

typedef struct {
    int steps_done;       /* time steps completed (damped first step counts 1)    */
    int fp_iters_total;   /* fixed-point iterations summed over all steps         */
    int fp_iters_max;     /* largest per-step count                               */
    double last_resid;    /* last eq. 3.25 quantity of the last step              */
    double cell_iters;    /* N^2 * (fixed-point iterations + 1) summed: the number */
                          /* of grid-cell applications of B_w                     */
} pide2d_stats;

typedef struct pide2d pide2d_t;

/* Bytes of device workspace pide2d_create() needs for this grid.
 * Errors: ERR_ARG for an invalid grid. */
pide2d_status pide2d_workspace_bytes(const pide2d_grid* grid, size_t* bytes);

/* Precomputes everything Algorithm 1 lists before time stepping, on the
 * device: the weights w (eq. 3.5; FP64), sigma_w sigma_w^T, kappa_w, r_w
 * (eqs. 3.3, 3.6; FP64), the weight spectrum conj(fft(C_1)) (eq. 3.13),
 * the payoff with cell averaging (eq. 3.18) and B_w V^0.
 * theta in [0.5, 1], dt > 0 with T/dt an integer (N_t), fp_tol > 0 (eq. 3.25).
 * workspace: device pointer, >= pide2d_workspace_bytes(), 256-byte aligned,
 * owned by the caller and used exclusively by this handle until destroy.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Blocks until the precomputation has finished.  On error *out is NULL.
 * Errors: ERR_ARG (grid, model -- rho not PD, alpha outside [0,1), delta or
 * lambda not positive, E[exp L_i(1)] infinite, i.e. lambda <= eta_i + rho_ii/2
 * by the Table A6 exponent --, contract, theta, dt, tol), ERR_WORKSPACE,
 * ERR_CUDA. */
pide2d_status pide2d_create(const pide2d_grid* grid, const pide2d_model* model,
                            const pide2d_contract* contract, double theta, double dt,
                            double fp_tol, const pide2d_options* opts,
                            void* workspace, size_t workspace_bytes, void* cuda_stream,
                            pide2d_t** out);

/* One time step of Algorithm 1 (the first call performs the four damped
 * steps when damping is on).  With the device loop it synchronises with the
 * stream once, at the end of the step, to read the iteration count; with
 * host_loop = 1 once per fixed-point iteration.
 * fp_iters / fp_resid: optional outputs (NULL allowed).
 * Errors: ERR_STATE after the last step, ERR_NOT_CONVERGED (state advanced
 * with the last iterate), ERR_CUDA. */
pide2d_status pide2d_step(pide2d_t* h, int* fp_iters, double* fp_resid);

/* Runs the remaining time steps, then writes the value at the valuation
 * node (N/2, N/2) = S0 to *price (FP64).  With the device loop the steps are
 * queued without any host synchronisation in between.  values_out: NULL or a pointer
 * (device or host) to (N+1)^2 doubles receiving V^{N_t} [m2][m1].
 * stats: optional.  Blocks until done. */
pide2d_status pide2d_solve(pide2d_t* h, double* price, double* values_out, pide2d_stats* stats);

/* Copies the current value array V^n, (N+1)^2 doubles [m2][m1], to dst
 * (device or host pointer).  Blocks until the copy has finished. */
pide2d_status pide2d_get_values(pide2d_t* h, double* dst);

/* Copies the device-computed quadrature data: omega_out (optional) receives
 * the (N)^2 weights w_{l1 l2} as [l2 + N/2][l1 + N/2] (eq. 3.5); rates_out
 * (optional, 9 doubles) receives sum w, r_w, kappa_w^1, kappa_w^2,
 * a11, a12, a22 (sigma_w sigma_w^T), b1, b2 (b = kappa_w - diag(a)/2, the
 * log-space departure drift).  Pointers may be device or host. */
pide2d_status pide2d_get_weights(pide2d_t* h, double* omega_out, double* rates_out);

/* Greeks of the current value array V^n at the interior nodes, by the
 * second-order central differences of Sec. 4 taken in log price and mapped
 * to price space: Delta_i = V_{s_i}/S_i, Gamma_ii = (V_{s_i s_i} - V_{s_i})/S_i^2,
 * Gamma_12 = V_{s_1 s_2}/(S_1 S_2) (FP64).  Each output is NULL (skipped) or
 * (N+1)^2 doubles [m2][m1] (device or host); only interior entries are
 * written.  Blocks until done. */
pide2d_status pide2d_greeks(pide2d_t* h, double* delta1, double* delta2, double* gamma11,
                            double* gamma12, double* gamma22);

/* The jump sum (B_w U)(s_m) at the interior nodes for a caller field:
 * U is (N+1)^2 doubles [m2][m1] (device or host) whose interior nodes are
 * used; every node outside the interior takes g(s, tau) when far_field is
 * 1, or 0 when it is 0.  out (device or host, (N+1)^2 doubles) receives B_w U
 * at the interior nodes; its other entries are left unchanged.  Runs the
 * same FFT kernels as the time stepping (eq. 3.17).  Blocks. */
pide2d_status pide2d_apply_jump(pide2d_t* h, const double* U, double tau, int far_field,
                                double* out);

/* Diagnostic: one iteration of the fixed-point loop (eqs. 3.24-3.25) as the
 * time loop runs it, applied to a caller residual r.  With
 *   M = (1 + ht theta r_w) I - ht theta (a11/2 d11 + a22/2 d22)
 * on the interior nodes (zero Dirichlet ring; the eq. 3.24 operator without
 * its mixed term, which the loop carries in the fixed point), it computes
 *   delta  = M^{-1} r         (DST-I along rows, tridiagonal solves along
 *                              columns for each row mode, DST-I back),
 *   bdelta = B_w delta        (the increment sweep of eq. 3.17: zero far field,
 *                              the midpoint interpolation of T_in folded into
 *                              the weight spectrum),
 *   *stop  = max |delta| / max(1, |delta|)  (eq. 3.25 for an iterate from 0),
 * through the same kernels and launch shapes as the time loop (row DST of r,
 * column solve pass, row DST pass with the R2C rows of delta, column pass,
 * inverse row pass).
 *   r           (N+1)^2 doubles [m2][m1], device or host; interior nodes used
 *   ht, theta   ht > 0, 0 < theta <= 1
 *   delta_out, bdelta_out  NULL or (N+1)^2 doubles (device or host); only the
 *               interior entries are written
 *   stop_out    NULL or one host double
 * Uses the handle's scratch fields only (callable between time steps without
 * changing the solution).  Blocks until done.  Errors: ERR_ARG, ERR_STATE,
 * ERR_CUDA. */
pide2d_status pide2d_iteration_probe(pide2d_t* h, const double* r, double ht, double theta,
                                     double* delta_out, double* bdelta_out, double* stop_out);

/* Kernel classes of the time loop, for pide2d_profile_read(). */
enum {
    PIDE2D_KERNEL_PREP = 0,            /* W = T_SL[...] and Y^{n,0} (Algorithm 1 steps 2-3)   */
    PIDE2D_KERNEL_ROW_FORWARD_FULL,    /* row pass of B_w Y^{n,0} (with far field)            */
    PIDE2D_KERNEL_ROW_FORWARD_INCR,    /* (unused: the increment row pass runs in DST_ROW)     */
    PIDE2D_KERNEL_COL_FULL,            /* column pass (FFT, product, inverse FFT), full rows   */
    PIDE2D_KERNEL_COL_INCR,            /* column pass of an increment                          */
    PIDE2D_KERNEL_ROW_INVERSE_FULL,    /* inverse row pass + first residual + row DST          */
    PIDE2D_KERNEL_ROW_INVERSE_INCR,    /* inverse row pass + residual update + row DST         */
    PIDE2D_KERNEL_COL_SOLVE,           /* tridiagonal solves along s2 of the row-DST modes    */
    PIDE2D_KERNEL_DST_ROW,             /* row DST back, state update, eq. 3.25 maximum, and   */
                                       /* the row pass of the increment's B_w sweep         */
    PIDE2D_KERNEL_CLASSES = 9
};

typedef struct {
    int launches[16];                  /* per class, since profiling was enabled               */
    double ms[16];                     /* summed CUDA-event durations per class                */
} pide2d_kernel_times;

/* Tracing: enable != 0 brackets every later time-loop kernel launch with a
 * pair of CUDA events on the handle's stream and clears earlier records;
 * enable == 0 stops recording.  The events are host-side resources created
 * on demand and kept until destroy (no device memory).  Errors: ERR_CUDA. */
pide2d_status pide2d_profile(pide2d_t* h, int enable);

/* Waits for the stream, then sums the recorded event pairs per kernel class
 * into *out.  Errors: ERR_ARG (out NULL), ERR_CUDA. */
pide2d_status pide2d_profile_read(pide2d_t* h, pide2d_kernel_times* out);

/* ------------------------------------------------------------------------
 * Discrete adjoint: the gradient of the price V^{N_t}(S0) with respect to
 * model parameters, exact for the discrete scheme of Algorithm 1 (up to
 * the fixed-point tolerance).  Going backwards through the theta steps, each
 * step solves the transposed system of eq. 3.23 with the same fixed-point
 * machinery (the transposed jump sum is the correlation with the weights
 * flipped in both axes; the diffusion solve is symmetric), applies the
 * transposed departure interpolation (the mirrored stencil of eq. 3.22) and
 * contracts the adjoint fields with the derivatives of the weights (eq. 3.5),
 * of sigma_w sigma_w^T, r_w and kappa_w (eqs. 3.3, 3.6) and of the departure
 * shift.  The derivatives of the precomputed quantities along each
 * direction are central differences of the FP64 precompute (relative step
 * 1e-5).  The time loop is replayed from checkpoints taken every
 * `interval` time steps.
 * ------------------------------------------------------------------------ */

/* Bytes of device tape for pide2d_record with this interval (>= 1) and up to
 * ndirs (<= 16) directions. */
pide2d_status pide2d_tape_bytes(pide2d_t* h, int interval, int ndirs, size_t* bytes);

/* Records checkpoints of the time loop into `tape` (device memory, 256-byte
 * aligned, >= pide2d_tape_bytes, caller-owned, untouched by anything else
 * until destroy).  Must be called before the first step.
 * Errors: ERR_STATE (steps already taken), ERR_ARG, ERR_WORKSPACE. */
pide2d_status pide2d_record(pide2d_t* h, void* tape, size_t bytes, int interval, int ndirs);

/* After pide2d_solve: grad[k] = d V^{N_t}(S0) / d eps of the model
 * model + eps * dirs[k] (only delta, lambda, eta and rho of dirs[k] are
 * used; alpha, r and sigma_cov are held fixed), k < ndirs (host arrays).
 * Replays the time loop segment by segment (one more forward solve) and
 * leaves the final values V^{N_t} in place.  Blocks until done.
 * Errors: ERR_STATE (no tape or the solve is not finished), ERR_ARG,
 * ERR_NOT_CONVERGED (an adjoint solve hit kmax; grad still written), ERR_CUDA. */
pide2d_status pide2d_adjoint(pide2d_t* h, const pide2d_model* dirs, int ndirs, double* grad);

/* ------------------------------------------------------------------------
 * Workload parameterisation [Appendix A, Table A5]: the NTS process as a
 * Brownian motion with drift beta and volatilities sigma, correlation corr,
 * time-changed by a unit-mean tempered-stable subordinator G with index
 * alpha and variance V[G(1)] = kappa.  Table A5 gives E[G(1)] =
 * delta Gamma(1-alpha) / lambda^(1-alpha) and V[G(1)] / E[G(1)] =
 * (1-alpha) / lambda, so
 *   lambda = (1 - alpha) / kappa,  delta = lambda^(1-alpha) / Gamma(1-alpha),
 *   eta = beta,  rho = [[s1^2, corr s1 s2], [corr s1 s2, s2^2]],
 * and the paper's extra Gaussian part sigma sigma^T is 0 (as in its Sec. 4).
 * ------------------------------------------------------------------------ */
typedef struct {
    double alpha;         /* 0 <= alpha < 1                                        */
    double kappa;         /* variance of G(1), > 0                                 */
    double beta[2];       /* Brownian drift                                        */
    double sigma[2];      /* Brownian volatilities, > 0                            */
    double corr;          /* Brownian correlation, |corr| < 1                      */
    double r;             /* riskless rate                                         */
} pide2d_workload;

/* The pide2d_model of a workload (the mapping above; host only).
 * Errors: ERR_ARG (invalid workload or NULL out; message via
 * pide2d_last_error(NULL)). */
pide2d_status pide2d_model_from_workload(const pide2d_workload* w, pide2d_model* out);

/* dirs[0..5] (host, 6 structs) receive the derivatives of that model with
 * respect to sigma1, sigma2, corr, kappa, beta1, beta2: the directions
 * pide2d_adjoint takes for the workload's gradient.  Errors: ERR_ARG. */
pide2d_status pide2d_workload_directions(const pide2d_workload* w, pide2d_model* dirs);

/* pide2d_adjoint along the six workload directions: grad[0..5] (host) =
 * d V^{N_t}(S0) / d (sigma1, sigma2, corr, kappa, beta1, beta2).  The handle
 * must have been created with pide2d_model_from_workload(w) and recorded with
 * ndirs >= 6.  Errors: ERR_ARG (NULL, invalid workload, or a handle whose
 * model is not w's), and those of pide2d_adjoint. */
pide2d_status pide2d_adjoint_workload(pide2d_t* h, const pide2d_workload* w, double* grad);

/* ------------------------------------------------------------------------
 * Batches: many independent pricings on one GPU (one time loop each, as in
 * Algorithm 1).  Jobs of one geometry (n, precision, sl_order, number of
 * steps) are advanced in lockstep, up to `lanes` at a time: every kernel of
 * a theta step and of each fixed-point iteration is launched once for all
 * of them, and a job whose iteration has converged skips its share.  The
 * whole time loop of such a chunk is one CUDA graph (a while-node over the
 * theta steps around a while-node over the fixed-point iterations, both
 * ended on the device), launched once; the host waits once per chunk.
 * ------------------------------------------------------------------------ */
typedef struct {
    pide2d_grid grid;
    pide2d_model model;
    pide2d_contract contract;
    double theta;         /* as for pide2d_create                                  */
    double dt;
    double fp_tol;
} pide2d_job;

typedef struct {
    int jobs_done;        /* jobs that produced a price (including NOT_CONVERGED)  */
    int failures;         /* jobs whose status was not OK                          */
    int fp_iters_total;   /* fixed-point iterations over all jobs                  */
    double cell_iters;    /* cell-applications of B_w over all jobs                */
    int tuned;            /* geometry groups whose launch shape was picked by     */
                          /* timed trials (the first 8 are listed below)          */
    int tune_n[8];        /* the group's grid size N                              */
    int tune_units[8];    /* FFT units per block of its multi-job kernels         */
    int tune_lanes[8];    /* jobs per chunk                                       */
    double tune_us_per_job[8];  /* the winning trial: microseconds per job of one */
                                /* column pass of the fixed-point iteration       */
    double create_s;      /* host wall time in the per-job precomputes             */
    double tune_s;        /* host wall time in the launch-shape trials             */
    double loop_s;        /* host wall time in the chunks' time loops              */
} pide2d_batch_stats;

/* Workspace for pide2d_batch_solve: min(lanes, count) lanes of the largest
 * job's pide2d_workspace_bytes (256-byte rounded), plus the argument arrays
 * of the multi-job launches for every theta step of the longest job.
 * 1 <= lanes <= 1024.  Errors: ERR_ARG. */
pide2d_status pide2d_batch_workspace_bytes(const pide2d_job* jobs, int count, int lanes, size_t* bytes);

/* Prices `count` jobs: prices[j] (host, count doubles) receives job j's value
 * at S0; statuses (host, count ints, optional) each job's status; stats
 * optional.  opts->host_loop is ignored (the multi-job loop runs on the
 * device).  All jobs of a chunk share damping.  workspace: device,
 * >= pide2d_batch_workspace_bytes(), 256-byte aligned, caller-owned.  Uses
 * the calling thread's current device; creates and destroys a few
 * non-blocking streams and host threads (no device allocation).  Blocks
 * until every job is done.  Returns OK if every job succeeded, else the
 * status of a failed job (ERR_CUDA first); message via pide2d_last_error(NULL). */
pide2d_status pide2d_batch_solve(const pide2d_job* jobs, int count, const pide2d_options* opts, int lanes,
                                 void* workspace, size_t workspace_bytes, double* prices, int* statuses,
                                 pide2d_batch_stats* stats);

/* ------------------------------------------------------------------------
 * The paper's price-space jump operator (Secs. 3.2.2, 4): on a non-uniform
 * price grid x_0 = 0 < x_1 < ... < x_nx (for example the paper's sinh grid),
 *   B_w V = T_out I~ C T_in V       (eqs. 3.12-3.17),
 * with T_in cubic Lagrange in price from the x-grid to the log lattice
 * y_in_m = e^{(m + 1/2) h_z}, m = -n_z - ny_minus .. n_z + ny_plus - 1 (v = 0
 * beyond x_nx), C the cross-correlation with the weights w on the z-lattice
 * of N_z = n_z cells of width h_z (eq. 3.5), I~ keeping
 * y_out_m = e^{m h_z}, m = -ny_minus .. ny_plus, and T_out cubic Lagrange in
 * price from y_out back to the x-grid (linear extrapolation for nodes below
 * y_out_{-ny_minus}).  The correlation is a zero-padded FFT of length
 * P = the least power of two >= max(#in, 4 n_z); the kept outputs equal
 * the paper's circulant of size #in (no wrap-around reaches them).
 * ------------------------------------------------------------------------ */
typedef struct {
    int nx;               /* the grid has nx + 1 nodes per axis, 4 <= nx <= 8192 */
    const double* x;      /* host: nx + 1 increasing nodes, x[0] = 0            */
    int n_z;              /* N_z >= 2                                           */
    double h_z;           /* z- and y-lattice spacing > 0                       */
    int ny_minus, ny_plus;/* y_out index range (either may be negative)         */
    int precision;        /* PIDE2D_FP64 (P <= 4096) or PIDE2D_FP32_BULK (FP32  */
                          /* transforms, P <= 8192); the tables are FP64        */
} pide2d_price_grid;

typedef struct pide2d_price pide2d_price_t;

/* Workspace bytes for this grid.  Errors: ERR_ARG, ERR_UNSUPPORTED (P too large). */
/* The paper's non-uniform price grid (Sec. 4), host-side, no GPU work:
 * uniform x = c xi on [0, x_int = 2.5 K], then x_int + c sinh(xi - xi_int) up
 * to x_max, on nx + 1 equidistant xi nodes, with c chosen so that
 * xi_int / xi_max = max(frac, x_int / x_max) (c = infinity, i.e. a uniform grid,
 * when x_int >= x_max); the z-lattice N_z = 2 nx cells of h_z = z_iii / N_z
 * (z_iii = z_max^III); the y_out range from the first positive node to
 * x_max: ny_minus = ceil(-ln x_1 / h_z), ny_plus = ceil(ln x_max / h_z).
 *   x_out  host, nx + 1 doubles (written); grid->x is set to x_out.
 * Errors: ERR_ARG (nx < 4 or > 8192, K, x_max, z_iii <= 0, frac outside
 * (0, 1), NULL pointers); message via pide2d_last_error(NULL). */
pide2d_status pide2d_price_sinh_grid(int nx, double strike, double x_max, double z_iii, double frac,
                                     double* x_out, pide2d_price_grid* grid);

pide2d_status pide2d_price_workspace_bytes(const pide2d_price_grid* grid, size_t* bytes);

/* Builds the interpolation tables (host, FP64), the weights w, sigma_w sigma_w^T
 * and the rates of `model` on the z-lattice (device, FP64) and the weight
 * spectrum.  workspace: device, 256-byte aligned, >= the bytes above,
 * caller-owned.  Blocks until done.  Errors: ERR_ARG, ERR_WORKSPACE, ERR_CUDA,
 * ERR_UNSUPPORTED. */
pide2d_status pide2d_price_create(const pide2d_price_grid* grid, const pide2d_model* model, void* workspace,
                                  size_t workspace_bytes, void* cuda_stream, pide2d_price_t** out);

/* out = B_w V on the (nx+1)^2 price grid; V and out: device, (nx+1)^2 doubles,
 * [m2][m1].  Blocks until done.  Errors: ERR_ARG, ERR_STATE, ERR_CUDA. */
pide2d_status pide2d_price_apply_jump(pide2d_price_t* h, const double* V, double* out);

/* Algorithm 1 in price space on this grid (Sec. 3.3): V^0 the payoff of
 * `contract` (put or call on the average) cell-averaged near the kink, then
 * n_steps theta steps (the first damped unless opts->damping = 0), each
 *   (I - h_t theta (D + B_w - r_w I)) V^n = T_SL (I + h_t (1-theta)(D + B_w - r_w I)) V^{n-1}
 * with D the central differences on the non-uniform grid (rows at x = 0
 * zero, second difference zero and first difference backward at x_max),
 * T_SL cubic Lagrange at x e^{kappa_w h_t} (linear beyond x_max), and the
 * fixed-point iteration (3.24)-(3.25) to fp_tol, each implicit system
 * solved by Jacobi-preconditioned BiCGSTAB to a relative residual of 1e-13.
 * FP64 fields; the jump operator in the handle's precision.
 * values_out: device or host, (nx+1)^2 doubles [m2][m1].  Blocks.
 * Errors: ERR_ARG, ERR_NOT_CONVERGED, ERR_CUDA. */
pide2d_status pide2d_price_solve(pide2d_price_t* h, const pide2d_contract* contract, double theta, int n_steps,
                                 double fp_tol, const pide2d_options* opts, double* values_out, pide2d_stats* stats);

/* The weights (2 n_z)^2 as [l2 + n_z][l1 + n_z] (omega_out, device or host) and
 * the 9 rates of pide2d_get_weights (rates_out, host).  Either may be NULL. */
pide2d_status pide2d_price_get_weights(pide2d_price_t* h, double* omega_out, double* rates_out);

const char* pide2d_price_last_error(const pide2d_price_t* h);
void pide2d_price_destroy(pide2d_price_t* h);

/* The jump sum of a field U with given weights and a zero far field -- the
 * same sum pide2d_apply_jump computes with far_field = 0 -- without any
 * device allocation.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory -- e.g. a plugin in a host
 * process whose memory manager owns the whole device, or a service that must
 * not call cudaMalloc (it can synchronise the device) after start-up.  Its
 * scratch is a fixed 7.2 MB device array inside the library, present on
 * every GPU where the library is loaded until the process exits; hence
 * n <= 256.
 *   n      power of two in [8, 256] (FP64 arithmetic, N_z = n/2)
 *   omega  device, n x n doubles, the weights [l2 + n/2][l1 + n/2] in the
 *          layout pide2d_get_weights returns them
 *   U      device, (n+1)^2 doubles [m2][m1]; its interior nodes are used and
 *          every other node counts as 0
 *   out    device, (n+1)^2 doubles; receives B_w U at the interior nodes, the
 *          other entries are left unchanged
 *   cuda_stream  the stream the work is queued on (NULL = legacy default)
 * Returns after queuing; the result is ready when the stream gets there.
 * The first call on a device looks up the scratch's device address
 * (cudaGetSymbolAddress) and caches it: make that first call before any
 * stream capture.  All calls share the one scratch array and nothing is
 * cleared between calls (each call writes every scratch entry it reads), so
 * calls whose GPU work overlaps -- on different streams or host threads --
 * race and must be serialised by the caller.
 * Errors: ERR_ARG (n out of range or not a power of two, NULL pointer),
 * ERR_CUDA; message via pide2d_last_error(NULL). */
pide2d_status pide2d_jump_static(int n, const double* omega, const double* U, double* out,
                                 void* cuda_stream);

/* Human-readable message for the last non-OK status on this handle (or of
 * the last failed pide2d_create when h is NULL).  Never NULL. */
const char* pide2d_last_error(const pide2d_t* h);

/* Frees the handle (not the workspace).  NULL is ignored. */
void pide2d_destroy(pide2d_t* h);

#ifdef __cplusplus
}
#endif

#endif /* PIDE2D_H */
