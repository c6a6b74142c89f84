// double instantiation of the time-stepping kernels (sweep_impl.cuh).
#include "sweep_impl.cuh"

namespace pide {

#define PIDE_PREC double
#define PIDE_INSTANTIATE(R)                                                                         \
    template cudaError_t launch_row_forward<R>(const FwdArgs<R>&, cudaStream_t);                    \
    template cudaError_t launch_col<R>(const ColArgs<R>&, cudaStream_t);                            \
    template cudaError_t launch_row_inverse<R>(const InvArgs<R>&, cudaStream_t);                    \
    template cudaError_t launch_dst_col<R>(const DstColArgs<R>&, cudaStream_t);                     \
    template cudaError_t launch_dst_row<R>(const DstRowArgs<R>&, cudaStream_t);                     \
    template cudaError_t launch_prep<R>(const PrepArgs<R>&, cudaStream_t);                          \
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
