// x1 passes, real-space eta, reductions and elementwise helpers in float, the
// precision conversions and the untyped helpers (instantiations).
#define FFTLS_KERNELS_MAIN
#include "fftls_kernels_impl.cuh"

namespace fftls {

// instantiated in the x2 and x3 translation units
extern template cudaError_t set_attrs_y<float>(size_t);
extern template cudaError_t set_attrs_z<float>(size_t);

#define FFTLS_INST_X(T)                                                                                 \
  template cudaError_t launch_fwd_x<T>(const IterArgs<T>&, cudaStream_t);                              \
  template cudaError_t launch_eta_stencil<T>(const IterArgs<T>&, cudaStream_t);                        \
  template cudaError_t launch_reduce_eta<T>(const IterArgs<T>&, cudaStream_t);                         \
  template cudaError_t launch_inv_x<T>(const IterArgs<T>&, cudaStream_t);                              \
  template cudaError_t launch_reduce_delta<T>(const IterArgs<T>&, cudaStream_t);                       \
  template cudaError_t set_kernel_attributes<T>(const IterArgs<T>&, size_t);                            \
  template cudaError_t launch_fill_eps<T>(T*, int, long long, const double*, cudaStream_t);            \
  template cudaError_t launch_stress<T>(const T*, const uint8_t*, const T*, int, long long, double*,   \
                                        double*, int, cudaStream_t);
FFTLS_INST_X(float)
template cudaError_t launch_convert<double, float>(double*, const float*, long long, cudaStream_t);
template cudaError_t launch_convert<float, double>(float*, const double*, long long, cudaStream_t);
template cudaError_t launch_convert<double, double>(double*, const double*, long long, cudaStream_t);

}  // namespace fftls
