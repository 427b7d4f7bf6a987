// Grouped launches of the x1 passes, real-space eta and reductions in float (instantiations).
#define FFTLS_GROUPED_TU
#include "fftls_kernels_impl.cuh"

namespace fftls {

// instantiated in the x2 and x3 grouped units
extern template cudaError_t set_attrs_ygrp<float>(size_t);
extern template cudaError_t set_attrs_zgrp<float>(size_t);

template cudaError_t launch_fwd_x_grp<float>(const IterArgs<float>&, cudaStream_t);
template cudaError_t launch_eta_stencil_grp<float>(const IterArgs<float>&, cudaStream_t);
template cudaError_t launch_reduce_eta_grp<float>(const IterArgs<float>&, cudaStream_t);
template cudaError_t launch_inv_x_grp<float>(const IterArgs<float>&, cudaStream_t);
template cudaError_t launch_reduce_delta_grp<float>(const IterArgs<float>&, cudaStream_t);
template cudaError_t set_attrs_xgrp<float>(size_t);
template cudaError_t set_attrs_grp<float>(size_t);

}  // namespace fftls
