// Grouped launches of the x1 passes, real-space eta and reductions in double (instantiations).
#define FFTLS_GROUPED_TU
#include "fftls_kernels_impl.cuh"

namespace fftls {

// instantiated in the x2 and x3 grouped units
extern template cudaError_t set_attrs_ygrp<double>(size_t);
extern template cudaError_t set_attrs_zgrp<double>(size_t);

template cudaError_t launch_fwd_x_grp<double>(const IterArgs<double>&, cudaStream_t);
template cudaError_t launch_eta_stencil_grp<double>(const IterArgs<double>&, cudaStream_t);
template cudaError_t launch_reduce_eta_grp<double>(const IterArgs<double>&, cudaStream_t);
template cudaError_t launch_inv_x_grp<double>(const IterArgs<double>&, cudaStream_t);
template cudaError_t launch_reduce_delta_grp<double>(const IterArgs<double>&, cudaStream_t);
template cudaError_t set_attrs_xgrp<double>(size_t);
template cudaError_t set_attrs_grp<double>(size_t);

}  // namespace fftls
