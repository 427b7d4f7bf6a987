// Grouped launches of the x3 transform and Fourier-space pass in double (instantiations).
#define FFTLS_GROUPED_TU
#include "fftls_kernels_impl.cuh"

namespace fftls {

template cudaError_t launch_fourier_z_grp<double>(const IterArgs<double>&, cudaStream_t);
template cudaError_t set_attrs_zgrp<double>(size_t);

}  // namespace fftls
