// Grouped launches of the x2 pass in double (instantiations).
#define FFTLS_GROUPED_TU
#include "fftls_kernels_impl.cuh"

namespace fftls {

template cudaError_t launch_mid_y_grp<double>(const IterArgs<double>&, bool, cudaStream_t);
template cudaError_t set_attrs_ygrp<double>(size_t);

}  // namespace fftls
