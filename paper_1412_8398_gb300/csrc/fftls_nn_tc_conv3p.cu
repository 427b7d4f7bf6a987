// Tensor-core warm-start path: the 3x3x3 convolutions of the mean pooling of a fine grid (fftls_nn_tc.cuh).
#include "fftls_nn_tc.cuh"

namespace fftls_tc {

fftls_status launch_k3_pool(int c, int nt, const ConvArgs& a, const int* n, int batch, cudaStream_t s) {
  return launch_c<3, true>(c, nt, a, n, batch, s);
}

}  // namespace fftls_tc
