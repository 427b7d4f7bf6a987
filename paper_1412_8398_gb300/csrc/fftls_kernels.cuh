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
  kSwitch = 5,      // hand-over to the next precision phase: no update
};

enum Green : int { kMS = 0, kCentered = 1, kWillot = 2, kRotated = 3 };
// scheme update of the inverse x1 pass
enum Update : int {
  kUpdDirectTau = 0,  // eps <- e                        (eq. ds, tau form)
  kUpdDirectSig = 1,  // eps <- eps + e                  (eq. ds, sigma form)
  kUpdAccel = 2,      // eps <- eps + 2 M (e - eps)      (eq. as)
  kUpdResidual = 3,   // r <- e - eps (eps unchanged)    (defect of the current iterate)
  kUpdCorrDirect = 4, // delta <- r + e                  (correction, direct scheme)
  kUpdCorrAccel = 5,  // delta <- delta + 2 M (r + e - delta) (correction, accelerated)
};

// Mutable solver control block (device memory, written by the host between
// phases, advanced by the reduction kernels).
struct Ctrl {
  int state;
  int it;            // eta evaluations so far (all phases)
  int max_it;        // cap on `it`
  int stop_rule;     // 0 = eta, 1 = max delta
  int switch_mode;   // 1: eta <= tol means hand over (kSwitch) instead of kConverged
  int stall;         // iterations since the last 10 % improvement of eta
  int stall_window;  // 0 disables stall detection
  int mean_guard;    // 1: eta test also needs |<eps> - eps_bar| <= tol |eps_bar|
  int phase_it;      // iterations in the current phase
  int phase_max;     // cap on phase_it (0: none); reaching it hands over (kSwitch)
  double tol;
  double eta0;
  double best;
  double last_eta;
  double last_delta;
  double last_mean_err;
  double off_sig[6];   // added to <sigma> and <eps> (correction phases: the FP64 iterate's means)
  double off_eps[6];
  double last_ms[6];   // <sigma>, <eps> of the last eta evaluation (with offsets)
  double last_me[6];
  int fault;           // 1: a tile copy did not complete within its wait limit; the solve was stopped
};

// Geometry: grid n1 x n2 x n3, half spectrum of H = n1/2 + 1 modes along x1,
// stored array-of-structures [x3 pos][x2 pos][x1][component].
struct Geom {
  int n1, n2, n3;
  int H;
  long long N;      // voxels
  long long modes;  // n3 * n2 * H
};

// Per-axis wave-vector table entry for frequency index m (signed s,
// q = 2 pi s / L): {q, sin q, cos q - 1, sin(q/2), cos(q/2), nyquist flag};
// exact zeros at the special modes so that k(q) = 0 is detected exactly.
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
  typedef typename Cplx<T>::type T2;
  Geom g;
  int dim;
  int green;
  int dual;          // 1: forward transform carries tau (buffer A) and sigma (buffer B)
  int update;        // Update
  int corr;          // 1: correction phase (zero mean mode, eta adds d64)
  int want_delta;    // inverse x1 pass computes max |d eps|, |d sigma|
  int write_d64;     // store the FP64 iterate's divergence (FP32) for a later correction phase
  int eta_real;      // 1: eta from the real-space divergence stencil (G^C/W/R, 3D, k_eta_stencil);
                     //    the forward transform then carries tau only
  int tauform;       // 1: the transformed field is tau (mean mode = eps_bar); 0: sigma
  T* eps;            // n_c x N (the iterate, or the correction delta)
  const uint8_t* phase;
  const T* coef;     // 256 x kCoef
  T2* specA;         // AoS [modes][n_c]: tau_hat (dual) or sigma_hat
  T2* specB;         // AoS [modes][n_c]: sigma_hat (dual)
  const T2* tw[3];   // per axis: e^{-2 pi i t / L}
  const KTab<T>* kt[3];
  const T2* rd[3];     // per axis, by storage position: {a, b} with kr_i = a_i prod_{m != i} b_m
                       // (G^R: a = 2 sin(q/2), b = cos(q/2); G^C: a = sin q, b = 1; G: a = q, b = 1)
  const int* perm[3];  // per axis: storage position -> frequency index
  const int* pos[3];   // per axis: frequency index -> storage position
  AxisPlan pl[3];
  double lam0, mu0;
  double eps_bar[6];
  Ctrl* ctrl;
  double* part_mean;   // [x1_blocks][2 nc]: sums of sigma and eps per block
  double* part_eta;    // [z blocks or eta blocks]: sums of |k*.sigma_hat|^2 per block
  double* part_delta;  // [x5_blocks][2]: max |d eps|, max |d sigma| per block
  double* eta_hist;    // [max_it]
  double* ms_hist;     // [max_it][nc]
  float* rfield;       // n_c x N defect r (written by kUpdResidual, read by corrections)
  float2* d64;         // [modes][3] by frequency index: k*.sigma_hat of the FP64 iterate (phase-free form), or with
                       // eta_real [3][N] floats: its real-space divergence
  // grouped launches (fftls_solve_batched): nsmp samples of one 3D geometry share a
  // launch; sample s finds its fields at these element offsets times s (null fields:
  // offset 0) and its lambda0, mu0, eps_bar[6] at smp_par[8 s ..] (device memory).
  // Single solves have nsmp = 1 and use the values above.
  int nsmp;
  long long st_field, st_phase, st_spec, st_coef, st_pmean, st_peta, st_pdelta, st_hist, st_d64;
  const double* smp_par;
  // launch shapes (host-computed)
  int x1_lines, x1_blocks;  // forward x1 pass: lines per batch, blocks (grid-stride over batches)
  int x1_vb;                // forward x1 pass: voxels per thread loaded together (1, 2 or 4; 0: staged by bulk copies)
  int x5_lines, x5_blocks;  // inverse x1 pass
  int x5_vb;                // inverse x1 pass: 1 register loads of eps, 0 staged by bulk copies (FP32)
  int x_threads;
  int y_w, y_threads, z_w, z_threads;
  size_t x1_smem, x5_smem, y_smem, z_smem;
  int e_planes, e_blocks;  // real-space eta: x3-planes per block, blocks (tiles x slabs)
  size_t e_smem;
};

// Shared memory of the forward x1 pass: twiddles, the tile of G lines, and for the
// staged variant the batch's eps (n_c rows of G n1 floats) and phase ids, 16-byte aligned.
__host__ __device__ inline size_t fwd_x_stage_offset(size_t tw_and_tile) { return (tw_and_tile + 15) & ~(size_t)15; }
__host__ __device__ inline size_t fwd_x_stage_bytes(int G, int n1, int nc) {
  return (size_t)G * n1 * (nc * sizeof(float) + 1);
}

// Threads per block of the strided (x2 / x3) passes with W modes per tile: a
// compile-time count, so that every stage of the tile transforms has a fixed
// trip count.
__host__ __device__ constexpr int strided_threads(int W) { return W == 1 ? 128 : 256; }

// Grouped launches (GRP variants, fftls_kernels_{x,y,z}{32,64}g.cu): the same
// kernels over a.nsmp samples of one 3D geometry; 2D grids are not grouped.
template <typename T> cudaError_t launch_fwd_x_grp(const IterArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_eta_stencil_grp(const IterArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_mid_y_grp(const IterArgs<T>& a, bool inv, cudaStream_t s);
template <typename T> cudaError_t launch_fourier_z_grp(const IterArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_reduce_eta_grp(const IterArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_inv_x_grp(const IterArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_reduce_delta_grp(const IterArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t set_attrs_grp(size_t smax);
template <typename T> cudaError_t set_attrs_xgrp(size_t smax);
template <typename T> cudaError_t set_attrs_ygrp(size_t smax);
template <typename T> cudaError_t set_attrs_zgrp(size_t smax);

// Launchers (fftls_kernels.cu).  All return cudaGetLastError().
template <typename T> cudaError_t launch_fwd_x(const IterArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_eta_stencil(const IterArgs<T>& a, cudaStream_t s);
// tile of the real-space eta kernel (x1 columns x x2 rows) and its threads
constexpr int kEtaTileX = 64, kEtaTileY = 8;
template <typename T> cudaError_t launch_mid_y(const IterArgs<T>& a, bool inv, cudaStream_t s);
template <typename T> cudaError_t launch_fourier_z(const IterArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_reduce_eta(const IterArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_inv_x(const IterArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_reduce_delta(const IterArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t set_kernel_attributes(const IterArgs<T>& a, size_t smax);
// dynamic shared-memory limits of the x2 and x3 kernels (their own translation units)
template <typename T> cudaError_t set_attrs_y(size_t smax);
template <typename T> cudaError_t set_attrs_z(size_t smax);

// Elementwise helpers.
template <typename T> cudaError_t launch_fill_eps(T* eps, int nc, long long N, const double* eps_bar6, cudaStream_t s);
template <typename TO, typename TI> cudaError_t launch_convert(TO* out, const TI* in, long long n, cudaStream_t s);
// out += in (FP64 += FP32), n values
cudaError_t launch_add_correction(double* out, const float* in, long long n, cudaStream_t s);
// stress = C(x):eps as FP64 (optional), plus FP64 sums of sigma and eps into part[blocks][2 nc]
template <typename T> cudaError_t launch_stress(const T* eps, const uint8_t* phase, const T* coef, int dim,
                                                 long long N, double* stress_out, double* part, int blocks,
                                                 cudaStream_t s);
// largest phase id in the image (atomicMax into *out, zeroed first)
cudaError_t launch_phase_max(const uint8_t* phase, long long N, unsigned int* out, int blocks, cudaStream_t s);
cudaError_t launch_sum_parts(const double* part, int blocks, int width, double* out, cudaStream_t s);

}  // namespace fftls
