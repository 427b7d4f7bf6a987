// x2 pass in double (instantiations).
#include "fftls_kernels_impl.cuh"

namespace fftls {

template cudaError_t launch_mid_y<double>(const IterArgs<double>&, bool, cudaStream_t);
template cudaError_t set_attrs_y<double>(size_t);

}  // namespace fftls
