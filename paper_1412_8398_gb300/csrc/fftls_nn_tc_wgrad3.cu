// Tensor-core warm-start path: the weight gradients of the 3x3x3 convolutions (fftls_nn_tc.cuh).
#include "fftls_nn_tc.cuh"

namespace fftls_tc {

fftls_status launch_wgrad_k3(bool pool, int c, int mo, const WgradArgs& a, const int* n, int batch, int tv,
                             cudaStream_t s) {
  return pool ? launch_wgrad_c<3, true>(c, mo, a, n, batch, tv, s) : launch_wgrad_c<3, false>(c, mo, a, n, batch, tv, s);
}

}  // namespace fftls_tc
