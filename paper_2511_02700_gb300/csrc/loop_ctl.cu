// Device-side control of the fixed-point iteration (eqs. 3.24-3.25).
//
// The iteration body of one theta step runs as the body of a CUDA-graph
// while-node; k_fp_check evaluates the stopping rule on the device and ends
// the loop, so a step needs no host round trip per iteration.  The loop
// always ends: at convergence, at kmax iterations, or on a non-finite
// residual.  k_fp_tally folds the step's count into running statistics that
// the host reads when it synchronises.  The fields a step iterates on are
// read by the loop kernels from FpCtl (written by k_fp_setup before each
// launch), so one instantiated graph serves every step with the same h_t
// and theta.
#include <cuda_runtime.h>

#include "internal.h"

namespace pide {

// resid: the FP64 eq. 3.25 quantity of the iteration (written by k_dst_row in
// both precisions)
template <typename R>
__global__ void k_fp_check(const double* resid, FpCtl* c, double tol, int kmax, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double r = *resid;
    const int k = c->k + 1;
    c->k = k;
    const bool conv = r < tol;
    c->conv = conv ? 1 : 0;
    c->last_resid = r;
    if (conv || k >= kmax || !isfinite(r)) cudaGraphSetConditional(h, 0);
}

__global__ void k_fp_setup(FpCtl* c, void* Y, void* BY, int step_end) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    c->Y = Y;
    c->BY = BY;
    c->step_end = step_end;
}

__global__ void k_fp_tally(FpCtl* c) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int k = c->k;
    const int step_end = c->step_end;
    c->total += k;
    c->substeps += 1;
    c->step_k += k;
    if (!c->conv) c->nonconv += 1;
    if (step_end) {
        c->last_step_k = c->step_k;
        if (c->step_k > c->max_step) c->max_step = c->step_k;
        c->step_k = 0;
        c->step_resid = c->last_resid;
    }
}

template <typename R>
cudaError_t launch_fp_check(const void* resid, FpCtl* ctl, double tol, int kmax, unsigned long long cond_handle,
                            cudaStream_t s) {
    k_fp_check<R><<<1, 32, 0, s>>>((const double*)resid, ctl, tol, kmax, (cudaGraphConditionalHandle)cond_handle);
    return cudaGetLastError();
}

cudaError_t launch_fp_tally(FpCtl* ctl, cudaStream_t s) {
    k_fp_tally<<<1, 32, 0, s>>>(ctl);
    return cudaGetLastError();
}

cudaError_t launch_fp_setup(FpCtl* ctl, void* Y, void* BY, int step_end, cudaStream_t s) {
    k_fp_setup<<<1, 32, 0, s>>>(ctl, Y, BY, step_end);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// multi-job fixed-point loop (one launch per kernel over all jobs of a group):
// the stopping rule of each job, and the count of jobs still iterating
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_jobs_reset(int K, const JobCheck* jc, JobsState st) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < K; j += gridDim.x * blockDim.x) {
        st.conv[j] = 0;
        st.kconv[j] = 0;
        st.kcount[j] = 0;
        *(double*)jc[j].resid = 0.0;
    }
}

template <typename R>
__global__ void k_jobs_check(int K, const JobCheck* jc, JobsState st, int iter) {
    __shared__ int act;
    if (threadIdx.x == 0) act = 0;
    __syncthreads();
    int mine = 0;
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        if (st.conv[j]) continue;
        double* rp = (double*)jc[j].resid;
        const double r = *rp;
        *rp = 0.0;                          // the next iteration's maximum starts from zero
        st.kcount[j] = iter;
        st.last[j] = r;
        const bool ok = r < jc[j].tol;
        if (ok || iter >= jc[j].kmax || !isfinite(r)) {
            st.conv[j] = 1;
            st.kconv[j] = iter;
            if (!ok) st.nonconv[j] = 1;
        } else {
            ++mine;
        }
    }
    if (mine) atomicAdd(&act, mine);
    __syncthreads();
    if (threadIdx.x == 0) *st.active = act;
}

template <typename R>
cudaError_t launch_jobs_reset(int K, const JobCheck* jc, JobsState st, cudaStream_t s) {
    k_jobs_reset<R><<<(K + 255) / 256, 256, 0, s>>>(K, jc, st);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_jobs_check(int K, const JobCheck* jc, JobsState st, int iter, cudaStream_t s) {
    k_jobs_check<R><<<1, 1024, 0, s>>>(K, jc, st, iter);
    return cudaGetLastError();
}

template cudaError_t launch_jobs_reset<float>(int, const JobCheck*, JobsState, cudaStream_t);
template cudaError_t launch_jobs_reset<double>(int, const JobCheck*, JobsState, cudaStream_t);
template cudaError_t launch_jobs_check<float>(int, const JobCheck*, JobsState, int, cudaStream_t);
template cudaError_t launch_jobs_check<double>(int, const JobCheck*, JobsState, int, cudaStream_t);

template cudaError_t launch_fp_check<float>(const void*, FpCtl*, double, int, unsigned long long, cudaStream_t);
template cudaError_t launch_fp_check<double>(const void*, FpCtl*, double, int, unsigned long long, cudaStream_t);

}  // namespace pide
