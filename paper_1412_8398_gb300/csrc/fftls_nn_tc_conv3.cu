// Tensor-core warm-start path: the 3x3x3 convolutions of a grid or of its upsampled coarse grid (fftls_nn_tc.cuh).
#include "fftls_nn_tc.cuh"

namespace fftls_tc {

fftls_status launch_k3(int c, int nt, const ConvArgs& a, const int* n, int batch, cudaStream_t s) {
  return launch_c<3, false>(c, nt, a, n, batch, s);
}

}  // namespace fftls_tc
