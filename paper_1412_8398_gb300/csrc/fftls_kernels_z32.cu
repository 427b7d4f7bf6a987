// x3 transform and Fourier-space pass in float (instantiations).
#include "fftls_kernels_impl.cuh"

namespace fftls {

template cudaError_t launch_fourier_z<float>(const IterArgs<float>&, cudaStream_t);
template cudaError_t set_attrs_z<float>(size_t);

}  // namespace fftls
