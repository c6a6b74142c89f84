// double instantiation of the time-stepping kernels (sweep_impl.cuh).
#include "sweep_impl.cuh"

namespace pide {

#define PIDE_PREC double
#define PIDE_INSTANTIATE(R)                                                                         \
    template cudaError_t launch_row_forward<R>(const FwdArgs<R>&, cudaStream_t);                    \
    template cudaError_t launch_col<R>(const ColArgs<R>&, cudaStream_t);                            \
    template cudaError_t launch_row_inverse<R>(const InvArgs<R>&, cudaStream_t);                    \
    template cudaError_t launch_col_solve<R>(const ColSolveArgs<R>&, cudaStream_t);                     \
    template cudaError_t launch_dst_row<R>(const DstRowArgs<R>&, cudaStream_t);                     \
    template cudaError_t launch_prep<R>(const PrepArgs<R>&, cudaStream_t);                          \
    template cudaError_t launch_row_dst<R>(const Geometry&, const double*, R*, const void*, cudaStream_t); \
    template cudaError_t launch_corr_col<R>(const Geometry&, const void*, const void*, int, int, double*, \
                                            const void*, cudaStream_t);                             \
    template cudaError_t launch_corr_finish<R>(const Geometry&, double*, double*, const void*, cudaStream_t); \
    template cudaError_t launch_ps_tin<R>(int, int, int, const int*, const double*, const double*, R*, cudaStream_t); \
    template cudaError_t launch_ps_rows_fwd<R>(int, const R*, int, void*, const void*, cudaStream_t); \
    template cudaError_t launch_ps_col<R>(int, void*, const void*, int, int, const void*, cudaStream_t); \
    template cudaError_t launch_ps_rows_inv<R>(int, const void*, int, double*, int, const void*, cudaStream_t); \
    template cudaError_t launch_row_forward_jobs<R>(const FwdArgs<R>&, const FwdArgs<R>*, int, JobsCtl, int, cudaStream_t); \
    template cudaError_t launch_col_jobs<R>(const ColArgs<R>&, const ColArgs<R>*, int, JobsCtl, int, cudaStream_t); \
    template cudaError_t launch_row_inverse_jobs<R>(const InvArgs<R>&, const InvArgs<R>*, int, JobsCtl, int, cudaStream_t); \
    template cudaError_t launch_col_solve_jobs<R>(const ColSolveArgs<R>&, const ColSolveArgs<R>*, int, JobsCtl, int, cudaStream_t); \
    template cudaError_t launch_dst_row_jobs<R>(const DstRowArgs<R>&, const DstRowArgs<R>*, int, JobsCtl, int, cudaStream_t); \
    template cudaError_t launch_prep_jobs<R>(const PrepArgs<R>&, const PrepArgs<R>*, int, bool, cudaStream_t); \
    template cudaError_t launch_weights_col<R>(const Geometry&, const void*, void*, void*, const void*, \
                                               cudaStream_t);                                       \
    template cudaError_t launch_state_from_double<R>(const Geometry&, const double*, int, St<R>*,  \
                                                     cudaStream_t);                                 \
    template cudaError_t launch_greeks<R>(const Geometry&, const St<R>*, const double*, const double*, \
                                          double, int, double*, int, cudaStream_t);                 \
    template cudaError_t launch_state_to_double<R>(const Geometry&, const St<R>*, double*, int,    \
                                                   cudaStream_t);
PIDE_INSTANTIATE(PIDE_PREC)
#undef PIDE_INSTANTIATE

}  // namespace pide
