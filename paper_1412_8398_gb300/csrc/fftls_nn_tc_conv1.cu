// Tensor-core warm-start path: the 1x1x1 convolutions (fftls_nn_tc.cuh).
#include "fftls_nn_tc.cuh"

namespace fftls_tc {

fftls_status launch_k1(bool pool, int c, int nt, const ConvArgs& a, const int* n, int batch, cudaStream_t s) {
  return pool ? launch_c<1, true>(c, nt, a, n, batch, s) : launch_c<1, false>(c, nt, a, n, batch, s);
}

}  // namespace fftls_tc
