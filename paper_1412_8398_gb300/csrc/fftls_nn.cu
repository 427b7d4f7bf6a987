// Kernels of the learned warm start (include/fftls_nn.h): periodic 3D
// convolutions (forward, input gradient, weight gradient), 2x pooling and
// upsampling, and the small elementwise pieces of training (loss, Adam) and of
// turning a prediction into an initial strain field.  FP32 throughout, FP64
// for reductions across threads.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "fftls_nn.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCOB = 8;             // output channels per block of the convolution
constexpr int kMeanBlocks = 256;    // partial sums per component in fftls_nn_strain_init

__device__ __forceinline__ int wrap1(int t, int n) {
  if (t < 0) t += n;
  if (t >= n) t -= n;
  return t;
}

// out[b][o](v) = sum_i sum_k W(o, i, k) in[b][i](v + d(k)),  d(k) = (kz, ky, kx) - KS/2,
// W(o, i, k) = w[o][i][k] (forward) or w[i][o][K-1-k] (transposed: the input
// gradient, since d(K-1-k) = -d(k)).  A block owns 256 voxels and kCOB output
// channels; its weights sit in shared memory as ws[i][k][oo], so the kCOB
// weights of one tap are read with broadcast vector loads.
template <int KS>
__global__ void __launch_bounds__(kThreads) k_conv3d(const float* __restrict__ in, const float* __restrict__ w,
                                                     const float* __restrict__ bias, const float* __restrict__ skip,
                                                     float* __restrict__ out, int cin, int cout, int n1, int n2,
                                                     int n3, int relu, int transposed, int accumulate) {
  constexpr int K = KS * KS * KS;
  extern __shared__ __align__(16) float ws[];
  const int o0 = blockIdx.y * kCOB;
  const int b = blockIdx.z;
  for (int t = threadIdx.x; t < cin * K * kCOB; t += blockDim.x) {
    const int oo = t % kCOB, rest = t / kCOB;
    const int k = rest % K, i = rest / K;
    const int o = o0 + oo;
    float val = 0.f;
    if (o < cout) val = transposed ? w[((size_t)i * cout + o) * K + (K - 1 - k)] : w[((size_t)o * cin + i) * K + k];
    ws[t] = val;
  }
  __syncthreads();
  const long long N = (long long)n1 * n2 * n3;
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N) return;
  const int xq = (int)(v % n1);
  const long long r = v / n1;
  const int yq = (int)(r % n2), zq = (int)(r / n2);
  int xo[KS], yo[KS];
  long long zo[KS];
#pragma unroll
  for (int d = 0; d < KS; ++d) {
    const int s = d - KS / 2;
    xo[d] = wrap1(xq + s, n1);
    yo[d] = wrap1(yq + s, n2) * n1;
    zo[d] = (long long)wrap1(zq + s, n3) * n1 * n2;
  }
  float acc[kCOB];
#pragma unroll
  for (int oo = 0; oo < kCOB; ++oo) acc[oo] = 0.f;
  const float* xb = in + (size_t)b * cin * N;
  for (int i = 0; i < cin; ++i) {
    const float* xi = xb + (size_t)i * N;
    const float* wi = ws + i * K * kCOB;
#pragma unroll
    for (int kz = 0; kz < KS; ++kz)
#pragma unroll
      for (int ky = 0; ky < KS; ++ky)
#pragma unroll
        for (int kx = 0; kx < KS; ++kx) {
          const float val = __ldg(xi + zo[kz] + yo[ky] + xo[kx]);
          const float4* wk = reinterpret_cast<const float4*>(wi + ((kz * KS + ky) * KS + kx) * kCOB);
          const float4 w0 = wk[0], w1 = wk[1];
          acc[0] += w0.x * val;
          acc[1] += w0.y * val;
          acc[2] += w0.z * val;
          acc[3] += w0.w * val;
          acc[4] += w1.x * val;
          acc[5] += w1.y * val;
          acc[6] += w1.z * val;
          acc[7] += w1.w * val;
        }
  }
#pragma unroll
  for (int oo = 0; oo < kCOB; ++oo) {
    const int o = o0 + oo;
    if (o >= cout) break;
    const size_t at = ((size_t)b * cout + o) * N + v;
    float s = acc[oo];
    if (bias) s += bias[o];
    if (skip) s += skip[at];
    if (relu) s = fmaxf(s, 0.f);
    out[at] = accumulate ? out[at] + s : s;
  }
}

// Weight and bias gradients, stage 1: block (chunk, pair = o * cin + i) sums
// dy[b][o](v) in[b][i](v + d(k)) over its chunk of (b, v) for every tap k, and
// dy itself (the bias term, kept for i = 0), into part[chunk][pair][K + 1].
template <int KS>
__global__ void __launch_bounds__(kThreads) k_conv3d_wgrad(const float* __restrict__ in, const float* __restrict__ dy,
                                                           float* __restrict__ part, int cin, int cout, int n1, int n2,
                                                           int n3, int batch, long long chunk) {
  constexpr int K = KS * KS * KS;
  const int pair = blockIdx.y;
  const int o = pair / cin, i = pair % cin;
  const long long N = (long long)n1 * n2 * n3;
  const long long total = (long long)batch * N;
  const long long c0 = (long long)blockIdx.x * chunk;
  const long long c1 = c0 + chunk < total ? c0 + chunk : total;
  float acc[K + 1];
#pragma unroll
  for (int k = 0; k <= K; ++k) acc[k] = 0.f;
  for (long long t = c0 + threadIdx.x; t < c1; t += blockDim.x) {
    const long long b = t / N, v = t - b * N;
    const float g = dy[((size_t)b * cout + o) * N + v];
    const float* xi = in + ((size_t)b * cin + i) * N;
    const int xq = (int)(v % n1);
    const long long r = v / n1;
    const int yq = (int)(r % n2), zq = (int)(r / n2);
#pragma unroll
    for (int kz = 0; kz < KS; ++kz) {
      const long long zz = (long long)wrap1(zq + kz - KS / 2, n3) * n1 * n2;
#pragma unroll
      for (int ky = 0; ky < KS; ++ky) {
        const long long yy = zz + (long long)wrap1(yq + ky - KS / 2, n2) * n1;
#pragma unroll
        for (int kx = 0; kx < KS; ++kx) acc[(kz * KS + ky) * KS + kx] += g * __ldg(xi + yy + wrap1(xq + kx - KS / 2, n1));
      }
    }
    acc[K] += g;
  }
  __shared__ float red[kThreads / 32][K + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k <= K; ++k) {
    float s = acc[k];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) red[warp][k] = s;
  }
  __syncthreads();
  if (threadIdx.x <= K) {
    float s = 0.f;
    for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) s += red[wi][threadIdx.x];
    part[((size_t)blockIdx.x * gridDim.y + pair) * (K + 1) + threadIdx.x] = s;
  }
}

// Stage 2: fixed-order sum over the chunks; dw[o][i][k], db[o] from the i = 0 pairs.
__global__ void k_wgrad_sum(const float* __restrict__ part, float* __restrict__ dw, float* __restrict__ db, int pairs,
                            int K, int cin, int nchunks) {
  const long long M = (long long)pairs * (K + 1);
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += part[(size_t)c * M + m];
    const int pair = (int)(m / (K + 1)), k = (int)(m % (K + 1));
    if (k < K) dw[(size_t)pair * K + k] = (float)s;
    else if (db && pair % cin == 0) db[pair / cin] = (float)s;
  }
}

__global__ void k_relu_bwd(float* __restrict__ dy, const float* __restrict__ y, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    if (!(y[t] > 0.f)) dy[t] = 0.f;
}

__global__ void k_pool2(const float* __restrict__ x, float* __restrict__ y, int planes, int n1, int n2, int n3) {
  const int m1 = n1 / 2, m2 = n2 / 2, m3 = n3 / 2;
  const long long M = (long long)m1 * m2 * m3, total = M * planes;
  const long long N = (long long)n1 * n2 * n3;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long p = t / M, u = t - p * M;
    const int a = (int)(u % m1), bq = (int)((u / m1) % m2), c = (int)(u / ((long long)m1 * m2));
    const float* xp = x + p * N + ((long long)(2 * c) * n2 + 2 * bq) * n1 + 2 * a;
    float s = 0.f;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dyq = 0; dyq < 2; ++dyq)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) s += xp[((long long)dz * n2 + dyq) * n1 + dx];
    y[t] = 0.125f * s;
  }
}

__global__ void k_pool2_bwd(const float* __restrict__ dy, float* __restrict__ dx, int planes, int n1, int n2, int n3,
                            int accumulate) {
  const int m1 = n1 / 2, m2 = n2 / 2;
  const long long N = (long long)n1 * n2 * n3, M = N / 8, total = N * planes;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long p = t / N, v = t - p * N;
    const int x = (int)(v % n1), yq = (int)((v / n1) % n2), z = (int)(v / ((long long)n1 * n2));
    const float g = 0.125f * dy[p * M + ((long long)(z / 2) * m2 + yq / 2) * m1 + x / 2];
    dx[t] = accumulate ? dx[t] + g : g;
  }
}

__global__ void k_up2(const float* __restrict__ x, float* __restrict__ y, int planes, int m1, int m2, int m3) {
  const int n1 = 2 * m1, n2 = 2 * m2;
  const long long M = (long long)m1 * m2 * m3, N = 8 * M, total = N * planes;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long p = t / N, v = t - p * N;
    const int xq = (int)(v % n1), yq = (int)((v / n1) % n2), z = (int)(v / ((long long)n1 * n2));
    y[t] = x[p * M + ((long long)(z / 2) * m2 + yq / 2) * m1 + xq / 2];
  }
}

__global__ void k_up2_bwd(const float* __restrict__ dy, float* __restrict__ dx, int planes, int m1, int m2, int m3) {
  const int n1 = 2 * m1, n2 = 2 * m2;
  const long long M = (long long)m1 * m2 * m3, N = 8 * M, total = M * planes;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long p = t / M, u = t - p * M;
    const int a = (int)(u % m1), bq = (int)((u / m1) % m2), c = (int)(u / ((long long)m1 * m2));
    const float* g = dy + p * N + ((long long)(2 * c) * n2 + 2 * bq) * n1 + 2 * a;
    float s = 0.f;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dyq = 0; dyq < 2; ++dyq)
#pragma unroll
        for (int dxq = 0; dxq < 2; ++dxq) s += g[((long long)dz * n2 + dyq) * n1 + dxq];
    dx[t] = s;
  }
}

__global__ void k_add(float* __restrict__ y, const float* __restrict__ x, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    y[t] += x[t];
}

__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ tg, float* __restrict__ dy,
                      double* __restrict__ loss, long long n) {
  double s = 0.0;
  const float sc = 2.f / (float)n;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const float d = y[t] - tg[t];
    dy[t] = sc * d;
    s += (double)d * d;
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  __shared__ double red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tsum = 0.0;
    for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) tsum += red[wi];
    atomicAdd(loss, tsum / (double)n);
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const float gt = g[t];
    const float mt = b1 * m[t] + (1.f - b1) * gt;
    const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
  }
}

__global__ void k_features(const uint8_t* __restrict__ phase, float* __restrict__ x, long long N, float lc) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
    x[t] = phase[t] == 1 ? 1.f : 0.f;
    x[N + t] = lc;
  }
}

// partial sums of each of the 6 output components: part[c][block]; FP32 compensated (Kahan) sums per
// thread, FP64 across threads and blocks
__global__ void k_comp_sums(const float* __restrict__ y, double* __restrict__ part, long long N) {
  const int c = blockIdx.y;
  const float* yc = y + (size_t)c * N;
  const long long stride = (long long)gridDim.x * blockDim.x;
  float sum = 0.f, comp = 0.f;
  auto add = [&](float x) {
    const float v = x - comp;
    const float nxt = sum + v;
    comp = (nxt - sum) - v;
    sum = nxt;
  };
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; t + 3 * stride < N; t += 4 * stride) {  // four loads in flight per thread
    const float a0 = yc[t], a1 = yc[t + stride], a2 = yc[t + 2 * stride], a3 = yc[t + 3 * stride];
    add(a0);
    add(a1);
    add(a2);
    add(a3);
  }
  for (; t < N; t += stride) add(yc[t]);
  double s = (double)sum - (double)comp;
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  __shared__ double red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tsum = 0.0;
    for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) tsum += red[wi];
    part[(size_t)c * gridDim.x + blockIdx.x] = tsum;
  }
}

// exact widening of a finite normal (or zero) float by its IEEE-754 fields: the exponent rebiased
// from 127 to 1023, the 23 mantissa bits moved to the top of the 52; other values through the
// conversion instruction
__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (u & 0x7fffffffu) == 0u ? ((u >> 31) ? -0.0 : 0.0) : (double)f;
  const uint64_t bits = ((uint64_t)(u >> 31) << 63) | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

// eps = eps_bar + scale (y - <y>): the fluctuation in FP32 (an initial guess), widened exactly to FP64
__global__ void k_strain_init(const float* __restrict__ y, double* __restrict__ eps, const double* __restrict__ part,
                              int nparts, long long N, double e0, double e1, double e2, double e3, double e4, double e5,
                              float scale) {
  __shared__ float mean[6];
  if (threadIdx.x < 6) {
    double s = 0.0;
    for (int q = 0; q < nparts; ++q) s += part[(size_t)threadIdx.x * nparts + q];
    mean[threadIdx.x] = (float)(s / (double)N);
  }
  __syncthreads();
  const double eb[6] = {e0, e1, e2, e3, e4, e5};
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const double f = widen(scale * (y[(size_t)c * N + t] - mean[c]));
      eps[(size_t)c * N + t] = eb[c] == 0.0 ? f : eb[c] + f;
    }
}

__global__ void k_strain_target(const double* __restrict__ eps, float* __restrict__ t, long long N, double e0,
                                double e1, double e2, double e3, double e4, double e5) {
  const double eb[6] = {e0, e1, e2, e3, e4, e5};
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < 6; ++c) t[(size_t)c * N + v] = (float)(eps[(size_t)c * N + v] - eb[c]);
}

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + kThreads - 1) / kThreads, 152LL * 16)); }

bool dims_ok(const int* n) { return n && n[0] >= 1 && n[1] >= 1 && n[2] >= 1; }

long long vox(const int* n) { return (long long)n[0] * n[1] * n[2]; }

fftls_status launched() { return cudaGetLastError() == cudaSuccess ? FFTLS_OK : FFTLS_E_CUDA; }

fftls_status conv_launch(const float* in, const float* w, const float* bias, const float* skip, float* out, int batch,
                         int cin, int cout, const int* n, int ksize, int relu, int transposed, int accumulate,
                         cudaStream_t s) {
  const long long N = vox(n);
  const int K = ksize * ksize * ksize;
  const size_t smem = (size_t)cin * K * kCOB * sizeof(float);
  dim3 grid((unsigned)((N + kThreads - 1) / kThreads), (unsigned)((cout + kCOB - 1) / kCOB), (unsigned)batch);
  cudaError_t e;
  if (ksize == 3) {
    e = cudaFuncSetAttribute((const void*)k_conv3d<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return FFTLS_E_CUDA;
    k_conv3d<3><<<grid, kThreads, smem, s>>>(in, w, bias, skip, out, cin, cout, n[0], n[1], n[2], relu, transposed,
                                             accumulate);
  } else {
    k_conv3d<1><<<grid, kThreads, smem, s>>>(in, w, bias, skip, out, cin, cout, n[0], n[1], n[2], relu, transposed,
                                             accumulate);
  }
  return launched();
}

int wgrad_chunks(int batch, int c_in, int c_out, const int* n) {
  const long long total = (long long)batch * vox(n);
  const long long pairs = (long long)c_in * c_out;
  long long want = (2048 + pairs - 1) / pairs;
  want = std::min<long long>(want, (total + 1023) / 1024);
  return (int)std::max<long long>(1, want);
}

}  // namespace

extern "C" {

fftls_status fftls_nn_conv3d(const float* x, const float* w, const float* bias, const float* skip, float* y, int batch,
                             int c_in, int c_out, const int n[3], int ksize, int relu, void* stream) {
  if (!x || !w || !y || !dims_ok(n) || batch < 1 || c_in < 1 || c_out < 1 || c_in > FFTLS_NN_MAX_CHANNELS ||
      c_out > FFTLS_NN_MAX_CHANNELS || (ksize != 1 && ksize != 3) || x == y)
    return FFTLS_E_INVALID_ARG;
  return conv_launch(x, w, bias, skip, y, batch, c_in, c_out, n, ksize, relu ? 1 : 0, 0, 0, (cudaStream_t)stream);
}

fftls_status fftls_nn_conv3d_backward_data(const float* dy, const float* w, float* dx, int batch, int c_in, int c_out,
                                           const int n[3], int ksize, int accumulate, void* stream) {
  if (!dy || !w || !dx || !dims_ok(n) || batch < 1 || c_in < 1 || c_out < 1 || c_in > FFTLS_NN_MAX_CHANNELS ||
      c_out > FFTLS_NN_MAX_CHANNELS || (ksize != 1 && ksize != 3) || dx == dy)
    return FFTLS_E_INVALID_ARG;
  // a convolution from the c_out gradient channels to the c_in input channels with w transposed and flipped
  return conv_launch(dy, w, nullptr, nullptr, dx, batch, c_out, c_in, n, ksize, 0, 1, accumulate ? 1 : 0,
                     (cudaStream_t)stream);
}

size_t fftls_nn_wgrad_scratch(int batch, int c_in, int c_out, const int n[3], int ksize) {
  if (!dims_ok(n) || batch < 1 || c_in < 1 || c_out < 1) return 0;
  const int K = ksize * ksize * ksize;
  return (size_t)wgrad_chunks(batch, c_in, c_out, n) * c_in * c_out * (K + 1);
}

fftls_status fftls_nn_conv3d_backward_weights(const float* x, const float* dy, float* dw, float* db, int batch,
                                              int c_in, int c_out, const int n[3], int ksize, float* scratch,
                                              size_t scratch_floats, void* stream) {
  if (!x || !dy || !dw || !scratch || !dims_ok(n) || batch < 1 || c_in < 1 || c_out < 1 ||
      c_in > FFTLS_NN_MAX_CHANNELS || c_out > FFTLS_NN_MAX_CHANNELS || (ksize != 1 && ksize != 3))
    return FFTLS_E_INVALID_ARG;
  if (scratch_floats < fftls_nn_wgrad_scratch(batch, c_in, c_out, n, ksize)) return FFTLS_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int nch = wgrad_chunks(batch, c_in, c_out, n);
  const long long total = (long long)batch * vox(n);
  const long long chunk = (total + nch - 1) / nch;
  const int pairs = c_in * c_out;
  dim3 grid((unsigned)nch, (unsigned)pairs);
  if (ksize == 3)
    k_conv3d_wgrad<3><<<grid, kThreads, 0, s>>>(x, dy, scratch, c_in, c_out, n[0], n[1], n[2], batch, chunk);
  else
    k_conv3d_wgrad<1><<<grid, kThreads, 0, s>>>(x, dy, scratch, c_in, c_out, n[0], n[1], n[2], batch, chunk);
  if (cudaGetLastError() != cudaSuccess) return FFTLS_E_CUDA;
  const int K = ksize * ksize * ksize;
  k_wgrad_sum<<<grid_for((long long)pairs * (K + 1)), kThreads, 0, s>>>(scratch, dw, db, pairs, K, c_in, nch);
  return launched();
}

fftls_status fftls_nn_relu_backward(float* dy, const float* y, long long count, void* stream) {
  if (!dy || !y || count < 0) return FFTLS_E_INVALID_ARG;
  if (count == 0) return FFTLS_OK;
  k_relu_bwd<<<grid_for(count), kThreads, 0, (cudaStream_t)stream>>>(dy, y, count);
  return launched();
}

fftls_status fftls_nn_pool2(const float* x, float* y, int planes, const int n[3], void* stream) {
  if (!x || !y || planes < 1 || !dims_ok(n) || (n[0] | n[1] | n[2]) & 1) return FFTLS_E_INVALID_ARG;
  k_pool2<<<grid_for(planes * vox(n) / 8), kThreads, 0, (cudaStream_t)stream>>>(x, y, planes, n[0], n[1], n[2]);
  return launched();
}

fftls_status fftls_nn_pool2_backward(const float* dy, float* dx, int planes, const int n[3], int accumulate,
                                     void* stream) {
  if (!dy || !dx || planes < 1 || !dims_ok(n) || (n[0] | n[1] | n[2]) & 1) return FFTLS_E_INVALID_ARG;
  k_pool2_bwd<<<grid_for(planes * vox(n)), kThreads, 0, (cudaStream_t)stream>>>(dy, dx, planes, n[0], n[1], n[2],
                                                                              accumulate ? 1 : 0);
  return launched();
}

fftls_status fftls_nn_upsample2(const float* x, float* y, int planes, const int nc[3], void* stream) {
  if (!x || !y || planes < 1 || !dims_ok(nc)) return FFTLS_E_INVALID_ARG;
  k_up2<<<grid_for(8 * planes * vox(nc)), kThreads, 0, (cudaStream_t)stream>>>(x, y, planes, nc[0], nc[1], nc[2]);
  return launched();
}

fftls_status fftls_nn_upsample2_backward(const float* dy, float* dx, int planes, const int nc[3], void* stream) {
  if (!dy || !dx || planes < 1 || !dims_ok(nc)) return FFTLS_E_INVALID_ARG;
  k_up2_bwd<<<grid_for(planes * vox(nc)), kThreads, 0, (cudaStream_t)stream>>>(dy, dx, planes, nc[0], nc[1], nc[2]);
  return launched();
}

fftls_status fftls_nn_add(float* y, const float* x, long long count, void* stream) {
  if (!y || !x || count < 0) return FFTLS_E_INVALID_ARG;
  if (count == 0) return FFTLS_OK;
  k_add<<<grid_for(count), kThreads, 0, (cudaStream_t)stream>>>(y, x, count);
  return launched();
}

fftls_status fftls_nn_mse(const float* y, const float* t, float* dy, double* loss, long long count, void* stream) {
  if (!y || !t || !dy || !loss || count < 1) return FFTLS_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(loss, 0, sizeof(double), s) != cudaSuccess) return FFTLS_E_CUDA;
  k_mse<<<grid_for(count), kThreads, 0, s>>>(y, t, dy, loss, count);
  return launched();
}

fftls_status fftls_nn_adam(float* p, const float* g, float* m, float* v, long long count, float lr, float beta1,
                           float beta2, float eps, int step, void* stream) {
  if (!p || !g || !m || !v || count < 0 || step < 1 || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) ||
      !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return FFTLS_E_INVALID_ARG;
  if (count == 0) return FFTLS_OK;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adam<<<grid_for(count), kThreads, 0, (cudaStream_t)stream>>>(p, g, m, v, count, lr, beta1, beta2, eps, c1, c2);
  return launched();
}

fftls_status fftls_nn_features(const uint8_t* phase, float* x, const int n[3], float log_contrast, void* stream) {
  if (!phase || !x || !dims_ok(n)) return FFTLS_E_INVALID_ARG;
  k_features<<<grid_for(vox(n)), kThreads, 0, (cudaStream_t)stream>>>(phase, x, vox(n), log_contrast);
  return launched();
}

fftls_status fftls_nn_strain_init(const float* y, double* eps, const int n[3], const double eps_bar[6], double scale,
                                  double* scratch, void* stream) {
  if (!y || !eps || !eps_bar || !scratch || !dims_ok(n)) return FFTLS_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = vox(n);
  k_comp_sums<<<dim3(kMeanBlocks, 6), kThreads, 0, s>>>(y, scratch, N);
  if (cudaGetLastError() != cudaSuccess) return FFTLS_E_CUDA;
  k_strain_init<<<grid_for(N), kThreads, 0, s>>>(y, eps, scratch, kMeanBlocks, N, eps_bar[0], eps_bar[1], eps_bar[2],
                                                 eps_bar[3], eps_bar[4], eps_bar[5], (float)scale);
  return launched();
}

fftls_status fftls_nn_strain_target(const double* eps, float* t, const int n[3], const double eps_bar[6], void* stream) {
  if (!eps || !t || !eps_bar || !dims_ok(n)) return FFTLS_E_INVALID_ARG;
  k_strain_target<<<grid_for(vox(n)), kThreads, 0, (cudaStream_t)stream>>>(eps, t, vox(n), eps_bar[0], eps_bar[1],
                                                                           eps_bar[2], eps_bar[3], eps_bar[4],
                                                                           eps_bar[5]);
  return launched();
}

}  // extern "C"
