// x3 transform and Fourier-space pass in double (instantiations).
#include "fftls_kernels_impl.cuh"

namespace fftls {

template cudaError_t launch_fourier_z<double>(const IterArgs<double>&, cudaStream_t);
template cudaError_t set_attrs_z<double>(size_t);

}  // namespace fftls
