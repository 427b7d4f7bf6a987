// Kernel interfaces of the FFT Lippmann-Schwinger iteration (internal header).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fftls_fft.cuh"

namespace fftls {

// Solver states kept in device memory (Ctrl::state).  Every kernel of an
// iteration reads it on entry, so a captured chunk of iterations stops on the
// device without a host round trip.
enum State : int {
  kRunning = 0,
  kConverged = 1,   // eta test passed: no update this iteration
  kLast = 2,        // max_iter reached: run this iteration's update, then stop
  kStopped = 3,     // set one iteration after kLast
  kDiverged = 4,    // non-finite eta or eta > 1e4 eta_0
  kSwitch = 5,      // precision hand-over (FP32 -> FP64): no update
};

enum Green : int { kMS = 0, kCentered = 1, kWillot = 2, kRotated = 3 };
enum Update : int { kUpdDirectTau = 0, kUpdDirectSig = 1, kUpdAccel = 2 };

// Mutable solver control block (device memory, written by the host between
// phases, advanced by the reduction kernels).
struct Ctrl {
  int state;
  int it;            // eta evaluations so far (all phases)
  int max_it;        // cap on `it`
  int stop_rule;     // 0 = eta, 1 = max delta
  int switch_mode;   // 1: eta <= tol means hand over to FP64 (kSwitch) instead of kConverged
  int stall;         // iterations since the last 10 % improvement of eta
  int stall_window;  // 0 disables stall detection
  int mean_guard;    // 1: eta test also needs |<eps> - eps_bar| <= tol |eps_bar|
  double tol;
  double eta0;
  double best;
  double last_eta;
  double last_delta;
  double last_mean_err;
};

// Geometry of the grid and of the half spectrum [comp][n3][n2][P].
struct Geom {
  int n1, n2, n3;
  int H;          // n1 / 2 + 1 (half spectrum length along x1)
  int P;          // padded row stride of the half spectrum (complex elements)
  long long N;    // voxels
  long long CS;   // complex elements per spectrum component = n3 * n2 * P
};

// Per-axis wave-vector table entry for index m (signed s, q = 2 pi s / L):
// {q, sin q, cos q - 1, sin(q/2), cos(q/2), nyquist flag}; exact zeros at the
// special modes so that k(q) = 0 is detected exactly.
template <typename T>
struct KTab {
  T q, sn, cm1, sh, ch, nyq;
};

// Coefficients per phase (8 entries, T):
// [0] lambda, [1] 2 mu, [2] lambda - lambda0, [3] 2 (mu - mu0),
// [4] 2 a_mu, [5] 2 (a_kappa - a_mu) / d, [6], [7] unused,
// with a_kappa = kappa0 / (kappa + kappa0), a_mu = mu0 / (mu + mu0).
constexpr int kCoef = 8;

template <typename T>
struct IterArgs {
  Geom g;
  int dim;
  int green;
  int dual;          // 1: forward transform carries tau (comps 0..nc-1) and sigma (nc..2nc-1)
  int update;        // Update
  int want_delta;    // K5 computes max |d eps|, |d sigma|
  T* eps;            // nc x N
  const uint8_t* phase;
  const T* coef;     // n_phases x kCoef
  typename Cplx<T>::type* spec;
  const typename Cplx<T>::type* twx;
  const typename Cplx<T>::type* twy;
  const typename Cplx<T>::type* twz;
  const KTab<T>* kx;
  const KTab<T>* ky;
  const KTab<T>* kz;
  AxisPlan px, py, pz;
  double lam0, mu0;
  double eps_bar[6];
  Ctrl* ctrl;
  double* part_mean;   // [grid_x1][2 nc]: sums of sigma and eps per block
  double* part_eta;    // [grid_fz]: sums of |k*.sigma_hat|^2 per block
  double* part_delta;  // [grid_x5][2]: max |d eps|, max |d sigma| per block
  double* eta_hist;    // [max_it]
  double* ms_hist;     // [max_it][nc]
  // launch shapes (host-computed)
  int x_lines;         // lines per batch in the x kernels
  int x1_blocks, x5_blocks;
  int y_w, z_w;        // column tile widths of the y and z kernels
  int y_threads, z_threads, x1_threads, x5_threads;
  size_t x1_smem, x5_smem, y_smem, z_smem;
};

// Launchers (fftls_kernels.cu).  All return cudaGetLastError().
template <typename T> cudaError_t launch_fwd_x(const IterArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_mid_y(const IterArgs<T>& a, int ncomp, bool inv, cudaStream_t s);
template <typename T> cudaError_t launch_fourier_z(const IterArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_reduce_eta(const IterArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_inv_x(const IterArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_reduce_delta(const IterArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t set_kernel_attributes(const IterArgs<T>& a);
// Largest block size the register use of kernel `which` allows (0 fwd_x, 1 mid_y, 2 fourier_z, 3 inv_x).
template <typename T> int kernel_max_threads(int dim, int which);

// Elementwise helpers.
template <typename T> cudaError_t launch_fill_eps(T* eps, int nc, long long N, const double* eps_bar6, cudaStream_t s);
template <typename TO, typename TI> cudaError_t launch_convert(TO* out, const TI* in, long long n, cudaStream_t s);
// stress = C(x):eps as FP64 (optional), plus FP64 sums of sigma and eps into part[blocks][2 nc]
template <typename T> cudaError_t launch_stress(const T* eps, const uint8_t* phase, const T* coef, int dim,
                                                 long long N, double* stress_out, double* part, int blocks,
                                                 cudaStream_t s);
// largest phase id in the image (atomicMax into *out, zeroed first)
cudaError_t launch_phase_max(const uint8_t* phase, long long N, unsigned int* out, int blocks, cudaStream_t s);
cudaError_t launch_sum_parts(const double* part, int blocks, int width, double* out, cudaStream_t s);

}  // namespace fftls
