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

#include <algorithm>

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
// multi-job time loop (one launch per kernel over all jobs of a chunk): the
// whole loop of a chunk is one CUDA graph -- an outer while-node over the
// theta steps (k_step_select picks the step's argument arrays, k_step_tally
// advances the step) around an inner while-node over the fixed-point
// iterations (k_jobs_check applies each job's stopping rule and ends the
// inner loop when no job iterates any more)
// ---------------------------------------------------------------------------
// start of a theta step's iterations: every job iterating again, and the inner
// loop's condition armed (a conditional handle keeps the value the previous
// theta step's last check left)
template <typename R>
__global__ void k_jobs_reset(int K, const JobCheck* jc, JobsState st, cudaGraphConditionalHandle inner) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < K; j += gridDim.x * blockDim.x) {
        st.conv[j] = 0;
        st.kconv[j] = 0;
        st.kcount[j] = 0;
        *(double*)jc[j].resid = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *st.iter = 0;
        cudaGraphSetConditional(inner, 1);
    }
}

__global__ void k_jobs_check(int K, const JobCheck* jc, JobsState st, int kmax_all, cudaGraphConditionalHandle h) {
    __shared__ int act;
    if (threadIdx.x == 0) act = 0;
    __syncthreads();
    const int iter = *st.iter + 1;
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
    if (threadIdx.x == 0) {
        *st.iter = iter;                    // read by the kernels after this one (JobsCtl::skip)
        *st.active = act;
        if (act == 0 || iter >= kmax_all) cudaGraphSetConditional(h, 0);
    }
}

__global__ void k_step_select(const uint4* __restrict__ blobs, size_t n16, JobsState st, uint4* __restrict__ dst) {
    const uint4* src = blobs + (size_t)(*st.step) * n16;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

__global__ void k_step_tally(int K, JobsState st, const int* step_end, int steps, cudaGraphConditionalHandle h) {
    const int t = *st.step;
    const int end = step_end[t];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < K; j += gridDim.x * blockDim.x) {
        const int k = st.kcount[j];
        st.it_total[j] += k;
        const int sk = st.it_step[j] + k;
        if (end) {
            if (sk > st.it_max[j]) st.it_max[j] = sk;
            st.it_step[j] = 0;
        } else {
            st.it_step[j] = sk;
        }
    }
    // one block: every thread has read *st.step before thread 0 advances it
    __syncthreads();
    if (threadIdx.x == 0) {
        *st.step = t + 1;
        if (t + 1 >= steps) cudaGraphSetConditional(h, 0);
    }
}

template <typename R>
cudaError_t launch_jobs_reset(int K, const JobCheck* jc, JobsState st, unsigned long long inner, cudaStream_t s) {
    k_jobs_reset<R><<<(K + 255) / 256, 256, 0, s>>>(K, jc, st, (cudaGraphConditionalHandle)inner);
    return cudaGetLastError();
}

cudaError_t launch_jobs_check(int K, const JobCheck* jc, JobsState st, int kmax_all, unsigned long long cond,
                              cudaStream_t s) {
    k_jobs_check<<<1, 1024, 0, s>>>(K, jc, st, kmax_all, (cudaGraphConditionalHandle)cond);
    return cudaGetLastError();
}

cudaError_t launch_step_select(const void* blobs, size_t bytes, JobsState st, void* dst, cudaStream_t s) {
    const size_t n16 = bytes / 16;
    const int blocks = (int)std::min<size_t>((n16 + 255) / 256, 1024);
    k_step_select<<<blocks, 256, 0, s>>>((const uint4*)blobs, n16, st, (uint4*)dst);
    return cudaGetLastError();
}

cudaError_t launch_step_tally(int K, JobsState st, const int* step_end, int steps, unsigned long long cond,
                              cudaStream_t s) {
    k_step_tally<<<1, 1024, 0, s>>>(K, st, step_end, steps, (cudaGraphConditionalHandle)cond);
    return cudaGetLastError();
}

template cudaError_t launch_jobs_reset<float>(int, const JobCheck*, JobsState, unsigned long long, cudaStream_t);
template cudaError_t launch_jobs_reset<double>(int, const JobCheck*, JobsState, unsigned long long, cudaStream_t);

template cudaError_t launch_fp_check<float>(const void*, FpCtl*, double, int, unsigned long long, cudaStream_t);
template cudaError_t launch_fp_check<double>(const void*, FpCtl*, double, int, unsigned long long, cudaStream_t);

}  // namespace pide
