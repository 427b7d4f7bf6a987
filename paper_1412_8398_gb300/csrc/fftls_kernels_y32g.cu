// Grouped launches of the x2 pass in float (instantiations).
#define FFTLS_GROUPED_TU
#include "fftls_kernels_impl.cuh"

namespace fftls {

template cudaError_t launch_mid_y_grp<float>(const IterArgs<float>&, bool, cudaStream_t);
template cudaError_t set_attrs_ygrp<float>(size_t);

}  // namespace fftls
