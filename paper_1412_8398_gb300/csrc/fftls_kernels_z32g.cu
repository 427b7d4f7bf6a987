// Grouped launches of the x3 transform and Fourier-space pass in float (instantiations).
#define FFTLS_GROUPED_TU
#include "fftls_kernels_impl.cuh"

namespace fftls {

template cudaError_t launch_fourier_z_grp<float>(const IterArgs<float>&, cudaStream_t);
template cudaError_t set_attrs_zgrp<float>(size_t);

}  // namespace fftls
