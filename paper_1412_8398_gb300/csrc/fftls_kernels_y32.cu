// x2 pass in float (instantiations).
#include "fftls_kernels_impl.cuh"

namespace fftls {

template cudaError_t launch_mid_y<float>(const IterArgs<float>&, bool, cudaStream_t);
template cudaError_t set_attrs_y<float>(size_t);

}  // namespace fftls
