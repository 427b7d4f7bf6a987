// Tensor-core path of the learned warm start (include/fftls_nn.h, fftls_nn_tc_*):
// periodic 3D convolutions as implicit GEMMs with BF16 operands and FP32
// accumulation (mma.sync m16n8k16), activations stored channels-last in BF16.
// The convolution kernel itself is in fftls_nn_tc.cuh; this file holds the
// weight packing, the first layer and the C ABI.
#include <algorithm>

#include "fftls_nn_tc.cuh"

namespace fftls_tc {
namespace {

// B fragments of every k step: out[(s * NT + nt) * 32 + lane] = {B[k][n], B[k+1][n]}, {B[k+8][n], B[k+9][n]}
// with k = 16 s + 2 (lane % 4), n = 8 nt + lane / 4; B[k][n] = W(n, ch, tap), k = tap * C + ch.
__global__ void k_pack(const float* __restrict__ w, uint32_t* __restrict__ out, int cin, int cout, int C, int NT,
                       int KS, int transposed, int steps) {
  const int KT = KS * KS * KS;
  const long long total = (long long)steps * NT * 64;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int hf = (int)(idx & 1), lane = (int)((idx >> 1) & 31);
    const long long rest = idx >> 6;
    const int nt = (int)(rest % NT), s = (int)(rest / NT);
    const int n = nt * 8 + (lane >> 2);
    float val[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int k = s * 16 + 2 * (lane & 3) + hf * 8 + e;
      const int tap = k / C, ch = k % C;
      float v = 0.f;
      if (tap < KT && ch < cin && n < cout)
        v = transposed ? w[((size_t)ch * cout + n) * KT + (KT - 1 - tap)] : w[((size_t)n * cin + ch) * KT + tap];
      val[e] = v;
    }
    out[idx] = pack_bf16(val[0], val[1]);
  }
}

// First layer straight from the phase image: y = act(conv([1{phase = 1}, lc], w) + bias), w [cout][2][27],
// cout <= 8, on FP32 cores (one input channel carries information; the constant channel lc adds
// lc * sum_k w[o][1][k] to the bias).  Tile 32 x 8 x 8 voxels; a thread owns one x3 column of 8 voxels
// and, per (dy, dx), reads the column's 10 halo values once for its three dz taps.
constexpr int kPX = 32, kPY = 8, kPZ = 8;
__global__ void __launch_bounds__(kThreads) k_conv_phase(const uint8_t* __restrict__ ph, const float* __restrict__ w,
                                                         const float* __restrict__ bias, __nv_bfloat16* __restrict__ y,
                                                         int n1, int n2, int n3, int tiles1, int tiles2, int cout,
                                                         float lc, int relu) {
  __shared__ __align__(16) float sw[27][8];
  __shared__ float sb[8];
  __shared__ float sp[kPZ + 2][kPY + 2][kPX + 2];
  int t = blockIdx.x;
  const int i1 = t % tiles1;
  t /= tiles1;
  const int i2 = t % tiles2, i3 = t / tiles2;
  const int x0 = i1 * kPX, y0 = i2 * kPY, z0 = i3 * kPZ;
  for (int q = threadIdx.x; q < 27 * 8; q += kThreads) {
    const int o = q & 7, k = q >> 3;
    sw[k][o] = o < cout ? w[(o * 2) * 27 + k] : 0.f;
  }
  if (threadIdx.x < 8) {
    const int o = threadIdx.x;
    float s = 0.f;
    if (o < cout) {
      for (int k = 0; k < 27; ++k) s += w[(o * 2 + 1) * 27 + k];
      s = lc * s + (bias ? bias[o] : 0.f);
    }
    sb[o] = s;
  }
  constexpr int NP = (kPZ + 2) * (kPY + 2) * (kPX + 2);
  constexpr int NIT = (NP + kThreads - 1) / kThreads;
  uint8_t pv[NIT];
#pragma unroll
  for (int k = 0; k < NIT; ++k) {
    const int q = threadIdx.x + k * kThreads;
    pv[k] = 0;
    if (q < NP) {
      const int px = q % (kPX + 2), rq = q / (kPX + 2);
      const int py = rq % (kPY + 2), pz = rq / (kPY + 2);
      pv[k] = __ldg(ph + ((size_t)wrapn(z0 + pz - 1, n3) * n2 + wrapn(y0 + py - 1, n2)) * n1 + wrapn(x0 + px - 1, n1));
    }
  }
#pragma unroll
  for (int k = 0; k < NIT; ++k) {
    const int q = threadIdx.x + k * kThreads;
    if (q < NP) (&sp[0][0][0])[q] = pv[k] == 1 ? 1.f : 0.f;
  }
  __syncthreads();
  const int tx = threadIdx.x % kPX, ty = threadIdx.x / kPX;
  float acc[kPZ][8];
#pragma unroll
  for (int zz = 0; zz < kPZ; ++zz)
#pragma unroll
    for (int o = 0; o < 8; ++o) acc[zz][o] = sb[o];
#pragma unroll
  for (int dy = 0; dy < 3; ++dy)
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
      float col[kPZ + 2];
#pragma unroll
      for (int zz = 0; zz < kPZ + 2; ++zz) col[zz] = sp[zz][ty + dy][tx + dx];
#pragma unroll
      for (int dz = 0; dz < 3; ++dz) {
        const int k = (dz * 3 + dy) * 3 + dx;
        const float4 w0 = *reinterpret_cast<const float4*>(&sw[k][0]);
        const float4 w1 = *reinterpret_cast<const float4*>(&sw[k][4]);
#pragma unroll
        for (int zz = 0; zz < kPZ; ++zz) {
          const float f = col[zz + dz];
          acc[zz][0] += f * w0.x;
          acc[zz][1] += f * w0.y;
          acc[zz][2] += f * w0.z;
          acc[zz][3] += f * w0.w;
          acc[zz][4] += f * w1.x;
          acc[zz][5] += f * w1.y;
          acc[zz][6] += f * w1.z;
          acc[zz][7] += f * w1.w;
        }
      }
    }
  const int x = x0 + tx, yq = y0 + ty;
  if (x >= n1 || yq >= n2) return;
#pragma unroll
  for (int zz = 0; zz < kPZ; ++zz) {
    const int z = z0 + zz;
    if (z >= n3) break;
    float o[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) o[e] = e < cout ? (relu ? fmaxf(acc[zz][e], 0.f) : acc[zz][e]) : 0.f;
    uint4 u;
    u.x = pack_bf16(o[0], o[1]);
    u.y = pack_bf16(o[2], o[3]);
    u.z = pack_bf16(o[4], o[5]);
    u.w = pack_bf16(o[6], o[7]);
    *reinterpret_cast<uint4*>(y + (((size_t)z * n2 + yq) * n1 + x) * 8) = u;
  }
}

// dW[o][i][k] (FP32 layout of the layer, i < cin) and db[o] from the tiles' partial sums, summed in FP64
// in tile order
__global__ void k_wgrad_reduce(const float* __restrict__ part, const float* __restrict__ partb, float* __restrict__ dw,
                               float* __restrict__ db, int tiles, int cout, int cin, int C, int KT) {
  const int ncols = KT * C;
  const long long M = (long long)cout * cin * KT;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < M + cout; q += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    if (q < M) {
      const int k = (int)(q % KT);
      const long long r = q / KT;
      const int i = (int)(r % cin), o = (int)(r / cin);
      const size_t col = (size_t)o * ncols + (size_t)k * C + i;
      for (int t = 0; t < tiles; ++t) s += part[(size_t)t * cout * ncols + col];
      dw[q] = (float)s;
    } else {
      const int o = (int)(q - M);
      for (int t = 0; t < tiles; ++t) s += partb[(size_t)t * cout + o];
      if (db) db[o] = (float)s;
    }
  }
}

__device__ __forceinline__ void unpack8(const uint4& u, float (&f)[8]) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float2 v = __bfloat1622float2(h[e]);
    f[2 * e] = v.x;
    f[2 * e + 1] = v.y;
  }
}

__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
  uint4 u;
  u.x = pack_bf16(f[0], f[1]);
  u.y = pack_bf16(f[2], f[3]);
  u.z = pack_bf16(f[4], f[5]);
  u.w = pack_bf16(f[6], f[7]);
  return u;
}

// channels-last BF16 [b][v][cs] from planar FP32 [b][c][N] (channels c..cs-1 zero)
__global__ void k_cl_from_planar(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, int c, int cs, long long N,
                                 long long total8) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total8; t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t % (cs / 8));
    const long long bv = t / (cs / 8);
    const long long b = bv / N, v = bv - b * N;
    float f[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int ch = q * 8 + e;
      f[e] = ch < c ? x[((size_t)b * c + ch) * N + v] : 0.f;
    }
    reinterpret_cast<uint4*>(y)[t] = pack8(f);
  }
}

// dy = y > 0 ? dy : 0, eight values at a time
__global__ void k_cl_relu_bwd(__nv_bfloat16* __restrict__ dy, const __nv_bfloat16* __restrict__ y, long long total8) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total8; t += (long long)gridDim.x * blockDim.x) {
    float g[8], a[8];
    unpack8(reinterpret_cast<const uint4*>(dy)[t], g);
    unpack8(reinterpret_cast<const uint4*>(y)[t], a);
#pragma unroll
    for (int e = 0; e < 8; ++e) g[e] = a[e] > 0.f ? g[e] : 0.f;
    reinterpret_cast<uint4*>(dy)[t] = pack8(g);
  }
}

// coarse (grid m) = sum over each 2x2x2 block of fine (grid 2m): the adjoint of nearest upsampling
__global__ void k_cl_up2_bwd(const __nv_bfloat16* __restrict__ fine, __nv_bfloat16* __restrict__ coarse, int cs, int m1,
                             int m2, int m3, long long total8) {
  const int cq = cs / 8;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total8; t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t % cq);
    long long r = t / cq;
    const int a1 = (int)(r % m1);
    r /= m1;
    const int a2 = (int)(r % m2);
    r /= m2;
    const int a3 = (int)(r % m3);
    const long long b = r / m3;
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) {
      const size_t v = (((size_t)b * 2 * m3 + 2 * a3 + (c8 >> 2)) * 2 * m2 + 2 * a2 + ((c8 >> 1) & 1)) * 2 * m1 + 2 * a1 +
                       (c8 & 1);
      float f[8];
      unpack8(reinterpret_cast<const uint4*>(fine)[v * cq + q], f);
#pragma unroll
      for (int e = 0; e < 8; ++e) s[e] += f[e];
    }
    reinterpret_cast<uint4*>(coarse)[t] = pack8(s);
  }
}

// fine (grid 2m) (+)= coarse / 8 spread over each 2x2x2 block: the adjoint of mean pooling
__global__ void k_cl_pool2_bwd(const __nv_bfloat16* __restrict__ coarse, __nv_bfloat16* __restrict__ fine, int cs,
                               int m1, int m2, int m3, int accumulate, long long total8) {
  const int cq = cs / 8;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total8; t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t % cq);
    long long r = t / cq;
    const int f1 = (int)(r % (2 * m1));
    r /= 2 * m1;
    const int f2 = (int)(r % (2 * m2));
    r /= 2 * m2;
    const int f3 = (int)(r % (2 * m3));
    const long long b = r / (2 * m3);
    const size_t u = (((size_t)b * m3 + (f3 >> 1)) * m2 + (f2 >> 1)) * m1 + (f1 >> 1);
    float g[8];
    unpack8(reinterpret_cast<const uint4*>(coarse)[u * cq + q], g);
    if (accumulate) {
      float o[8];
      unpack8(reinterpret_cast<const uint4*>(fine)[t], o);
#pragma unroll
      for (int e = 0; e < 8; ++e) g[e] = o[e] + 0.125f * g[e];
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) g[e] *= 0.125f;
    }
    reinterpret_cast<uint4*>(fine)[t] = pack8(g);
  }
}

// y += x, eight values at a time
__global__ void k_cl_add(__nv_bfloat16* __restrict__ y, const __nv_bfloat16* __restrict__ x, long long total8) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total8; t += (long long)gridDim.x * blockDim.x) {
    float a[8], b[8];
    unpack8(reinterpret_cast<const uint4*>(y)[t], a);
    unpack8(reinterpret_cast<const uint4*>(x)[t], b);
#pragma unroll
    for (int e = 0; e < 8; ++e) a[e] += b[e];
    reinterpret_cast<uint4*>(y)[t] = pack8(a);
  }
}

// weight gradient of the first layer (fftls_nn_tc_conv_phase): part[tile][o][k] = sum over the tile's
// voxels of dy(v)[o] 1{phase(v + d(k)) = 1}, and part[tile][o][27] = sum of dy(v)[o].  A block stages the
// indicator of a 32 x 8 x 4 tile with its halo and the tile's dy in shared memory; thread (o, k) sums
// over the tile's voxels in FP32.
constexpr int kWX = 32, kWY = 8, kWZ = 4;
__global__ void __launch_bounds__(kThreads) k_wgrad_phase(const uint8_t* __restrict__ ph,
                                                          const __nv_bfloat16* __restrict__ dy, float* __restrict__ part,
                                                          int n1, int n2, int n3, int tiles1, int tiles2, int cout) {
  __shared__ float sp[kWZ + 2][kWY + 2][kWX + 2];
  __shared__ float sg[kWZ * kWY * kWX][8];
  int t = blockIdx.x;
  const int i1 = t % tiles1;
  t /= tiles1;
  const int i2 = t % tiles2, i3 = t / tiles2;
  const int x0 = i1 * kWX, y0 = i2 * kWY, z0 = i3 * kWZ;
  constexpr int NP = (kWZ + 2) * (kWY + 2) * (kWX + 2);
  for (int q = threadIdx.x; q < NP; q += kThreads) {
    const int px = q % (kWX + 2), rq = q / (kWX + 2);
    const int py = rq % (kWY + 2), pz = rq / (kWY + 2);
    (&sp[0][0][0])[q] =
        __ldg(ph + ((size_t)wrapn(z0 + pz - 1, n3) * n2 + wrapn(y0 + py - 1, n2)) * n1 + wrapn(x0 + px - 1, n1)) == 1
            ? 1.f
            : 0.f;
  }
  for (int m = threadIdx.x; m < kWZ * kWY * kWX; m += kThreads) {
    const int x = x0 + (m & 31), y = y0 + ((m >> 5) & 7), z = z0 + (m >> 8);
    float g[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (x < n1 && y < n2 && z < n3) unpack8(reinterpret_cast<const uint4*>(dy)[((size_t)z * n2 + y) * n1 + x], g);
#pragma unroll
    for (int e = 0; e < 8; ++e) sg[m][e] = g[e];
  }
  __syncthreads();
  const int q = threadIdx.x;
  if (q >= cout * 28) return;
  const int o = q / 28, k = q % 28;
  const int dz = k / 9, dyy = (k / 3) % 3, dx = k % 3;
  float s4[4] = {0.f, 0.f, 0.f, 0.f};
  for (int m = 0; m < kWZ * kWY * kWX; m += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int mm = m + u;
      const float f = k < 27 ? sp[(mm >> 8) + dz][((mm >> 5) & 7) + dyy][(mm & 31) + dx] : 1.f;
      s4[u] += f * sg[mm][o];
    }
  }
  part[((size_t)blockIdx.x * cout + o) * 28 + k] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
}

// dW of the first layer [cout][2][27] and db: channel 0 from the indicator sums, channel 1 = lc times
// the sum of dy (the constant input channel), summed over tiles in FP64
__global__ void k_wgrad_phase_reduce(const float* __restrict__ part, float* __restrict__ dw, float* __restrict__ db,
                                     int tiles, int cout, float lc) {
  for (int q = threadIdx.x; q < cout * 28; q += blockDim.x) {
    const int o = q / 28, k = q % 28;
    double s = 0.0;
    for (int t = 0; t < tiles; ++t) s += part[((size_t)t * cout + o) * 28 + k];
    if (k < 27) {
      dw[(o * 2) * 27 + k] = (float)s;
    } else {
      for (int kk = 0; kk < 27; ++kk) dw[(o * 2 + 1) * 27 + kk] = (float)(s * (double)lc);
      if (db) db[o] = (float)s;
    }
  }
}

bool dims_ok(const int* n) { return n && n[0] >= 1 && n[1] >= 1 && n[2] >= 1; }

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + kThreads - 1) / kThreads, 152LL * 16)); }

}  // namespace
}  // namespace fftls_tc

using namespace fftls_tc;

extern "C" {

size_t fftls_nn_tc_packed_bytes(int c_in, int c_out, int ksize, int transposed) {
  if (c_in < 1 || c_out < 1 || c_in > 64 || c_out > 64 || (ksize != 1 && ksize != 3)) return 0;
  const int ci = transposed ? c_out : c_in, co = transposed ? c_in : c_out;
  return (size_t)ksteps_of(stored_of(ci), ksize) * (stored_of(co) / 8) * 32 * sizeof(uint2);
}

fftls_status fftls_nn_tc_pack(const float* w, void* packed, int c_in, int c_out, int ksize, int transposed,
                              void* stream) {
  if (!w || !packed || !aligned16(packed) || fftls_nn_tc_packed_bytes(c_in, c_out, ksize, transposed) == 0)
    return FFTLS_E_INVALID_ARG;
  const int ci = transposed ? c_out : c_in, co = transposed ? c_in : c_out;
  const int C = stored_of(ci), NT = stored_of(co) / 8, steps = ksteps_of(C, ksize);
  const long long total = (long long)steps * NT * 64;
  k_pack<<<grid_for(total), kThreads, 0, (cudaStream_t)stream>>>(w, static_cast<uint32_t*>(packed), ci, co, C, NT,
                                                                 ksize, transposed ? 1 : 0, steps);
  return cudaGetLastError() == cudaSuccess ? FFTLS_OK : FFTLS_E_CUDA;
}

fftls_status fftls_nn_tc_conv3d(const void* x, const void* packed, const float* bias, const void* skip, void* y,
                                int batch, int c_in, int c_out, const int n[3], int ksize, int in_mode, int relu,
                                int out_planar, int accumulate, void* stream) {
  if (!x || !packed || !y || !dims_ok(n) || batch < 1 || c_in < 1 || c_out < 1 || c_in > 64 || c_out > 64 ||
      (ksize != 1 && ksize != 3) || in_mode < 0 || in_mode > 2 || x == y || !aligned16(x) || !aligned16(packed) ||
      !aligned16(y) || (skip && (!aligned16(skip) || skip == y)))
    return FFTLS_E_INVALID_ARG;
  if (in_mode == 1 && ((n[0] | n[1] | n[2]) & 1)) return FFTLS_E_INVALID_ARG;
  ConvArgs a{};
  a.x = static_cast<const __nv_bfloat16*>(x);
  a.w = static_cast<const uint2*>(packed);
  a.bias = bias;
  a.skip = static_cast<const __nv_bfloat16*>(skip);
  a.y = y;
  a.n1 = n[0];
  a.n2 = n[1];
  a.n3 = n[2];
  const int f = in_mode == 1 ? -1 : in_mode == 2 ? 1 : 0;
  a.m1 = f < 0 ? n[0] / 2 : n[0] << f;
  a.m2 = f < 0 ? n[1] / 2 : n[1] << f;
  a.m3 = f < 0 ? n[2] / 2 : n[2] << f;
  a.cout = c_out;
  a.relu = relu ? 1 : 0;
  a.mode = in_mode;
  a.planar = out_planar ? 1 : 0;
  a.accumulate = accumulate ? 1 : 0;
  const int C = stored_of(c_in), NT = stored_of(c_out) / 8;
  cudaStream_t s = (cudaStream_t)stream;
  if (ksize == 1) return launch_k1(in_mode == 2, C, NT, a, n, batch, s);
  return in_mode == 2 ? launch_k3_pool(C, NT, a, n, batch, s) : launch_k3(C, NT, a, n, batch, s);
}

fftls_status fftls_nn_tc_conv_phase(const uint8_t* phase, const float* w, const float* bias, void* y, const int n[3],
                                    int c_out, float log_contrast, int relu, void* stream) {
  if (!phase || !w || !y || !dims_ok(n) || c_out < 1 || c_out > 8 || !aligned16(y)) return FFTLS_E_INVALID_ARG;
  const int t1 = (n[0] + kPX - 1) / kPX, t2 = (n[1] + kPY - 1) / kPY, t3 = (n[2] + kPZ - 1) / kPZ;
  const long long tiles = (long long)t1 * t2 * t3;
  if (tiles > 0x7fffffffLL) return FFTLS_E_UNSUPPORTED_SIZE;
  k_conv_phase<<<(unsigned)tiles, kThreads, 0, (cudaStream_t)stream>>>(
      phase, w, bias, static_cast<__nv_bfloat16*>(y), n[0], n[1], n[2], t1, t2, c_out, log_contrast, relu ? 1 : 0);
  return cudaGetLastError() == cudaSuccess ? FFTLS_OK : FFTLS_E_CUDA;
}

size_t fftls_nn_tc_wgrad_scratch(int batch, int c_in, int c_out, const int n[3], int ksize) {
  if (!dims_ok(n) || batch < 1 || c_in < 1 || c_out < 1 || c_in > 64 || c_out > 64 || (ksize != 1 && ksize != 3))
    return 0;
  const int C = stored_of(c_in), MO = (c_out + 15) / 16 > 2 ? 4 : (c_out + 15) / 16;
  const long long tiles = wgrad_tiles(n, ksize, C, MO);
  if (tiles == 0) return 0;
  return (size_t)batch * tiles * c_out * ((size_t)ksize * ksize * ksize * C + 1);
}

fftls_status fftls_nn_tc_conv3d_backward_weights(const void* x, const void* dy, float* dw, float* db, int batch,
                                                 int c_in, int c_out, const int n[3], int ksize, int in_mode,
                                                 float* scratch, size_t scratch_floats, void* stream) {
  if (!x || !dy || !dw || !scratch || !dims_ok(n) || batch < 1 || c_in < 1 || c_out < 1 || c_in > 64 ||
      c_out > 64 || (ksize != 1 && ksize != 3) || in_mode < 0 || in_mode > 2 || !aligned16(x) || !aligned16(dy))
    return FFTLS_E_INVALID_ARG;
  if (in_mode == 1 && ((n[0] | n[1] | n[2]) & 1)) return FFTLS_E_INVALID_ARG;
  const size_t need = fftls_nn_tc_wgrad_scratch(batch, c_in, c_out, n, ksize);
  if (need == 0) return FFTLS_E_UNSUPPORTED_SIZE;
  if (scratch_floats < need) return FFTLS_E_INVALID_ARG;
  const int C = stored_of(c_in), MO = (c_out + 15) / 16 > 2 ? 4 : (c_out + 15) / 16;
  const int KT = ksize * ksize * ksize;
  WgradArgs a{};
  a.x = static_cast<const __nv_bfloat16*>(x);
  a.dy = static_cast<const __nv_bfloat16*>(dy);
  a.n1 = n[0];
  a.n2 = n[1];
  a.n3 = n[2];
  const int f = in_mode == 1 ? -1 : in_mode == 2 ? 1 : 0;
  a.m1 = f < 0 ? n[0] / 2 : n[0] << f;
  a.m2 = f < 0 ? n[1] / 2 : n[1] << f;
  a.m3 = f < 0 ? n[2] / 2 : n[2] << f;
  a.mode = in_mode;
  a.cout = c_out;
  a.cso = stored_of(c_out);
  a.ncols = KT * C;
  a.tiles = (int)wgrad_tiles(n, ksize, C, MO);
  a.part = scratch;
  a.partb = scratch + (size_t)batch * a.tiles * c_out * a.ncols;
  const int tv = wgrad_tile_voxels(n, ksize, C, MO);
  cudaStream_t s = (cudaStream_t)stream;
  const fftls_status st = ksize == 3 ? launch_wgrad_k3(in_mode == 2, C, MO, a, n, batch, tv, s)
                                     : launch_wgrad_k1(in_mode == 2, C, MO, a, n, batch, tv, s);
  if (st != FFTLS_OK) return st;
  const long long M = (long long)c_out * c_in * KT + c_out;
  k_wgrad_reduce<<<grid_for(M), kThreads, 0, s>>>(a.part, a.partb, dw, db, batch * a.tiles, c_out, c_in, C, KT);
  return cudaGetLastError() == cudaSuccess ? FFTLS_OK : FFTLS_E_CUDA;
}

size_t fftls_nn_tc_phase_wgrad_scratch(const int n[3]) {
  if (!dims_ok(n)) return 0;
  const long long tiles = (long long)((n[0] + kWX - 1) / kWX) * ((n[1] + kWY - 1) / kWY) * ((n[2] + kWZ - 1) / kWZ);
  return (size_t)tiles * 8 * 28;
}

fftls_status fftls_nn_tc_conv_phase_backward_weights(const uint8_t* phase, const void* dy, float* dw, float* db,
                                                     const int n[3], int c_out, float log_contrast, float* scratch,
                                                     size_t scratch_floats, void* stream) {
  if (!phase || !dy || !dw || !scratch || !dims_ok(n) || c_out < 1 || c_out > 8 || !aligned16(dy))
    return FFTLS_E_INVALID_ARG;
  if (scratch_floats < fftls_nn_tc_phase_wgrad_scratch(n)) return FFTLS_E_INVALID_ARG;
  const int t1 = (n[0] + kWX - 1) / kWX, t2 = (n[1] + kWY - 1) / kWY, t3 = (n[2] + kWZ - 1) / kWZ;
  const long long tiles = (long long)t1 * t2 * t3;
  if (tiles > 0x7fffffffLL) return FFTLS_E_UNSUPPORTED_SIZE;
  cudaStream_t s = (cudaStream_t)stream;
  k_wgrad_phase<<<(unsigned)tiles, kThreads, 0, s>>>(phase, static_cast<const __nv_bfloat16*>(dy), scratch, n[0], n[1],
                                                     n[2], t1, t2, c_out);
  if (cudaGetLastError() != cudaSuccess) return FFTLS_E_CUDA;
  k_wgrad_phase_reduce<<<1, kThreads, 0, s>>>(scratch, dw, db, (int)tiles, c_out, log_contrast);
  return cudaGetLastError() == cudaSuccess ? FFTLS_OK : FFTLS_E_CUDA;
}

fftls_status fftls_nn_tc_from_planar(const float* x, void* y, int batch, int channels, long long voxels, void* stream) {
  if (!x || !y || batch < 1 || channels < 1 || channels > 64 || voxels < 1 || !aligned16(y)) return FFTLS_E_INVALID_ARG;
  const int cs = stored_of(channels);
  const long long total8 = (long long)batch * voxels * (cs / 8);
  k_cl_from_planar<<<grid_for(total8), kThreads, 0, (cudaStream_t)stream>>>(x, static_cast<__nv_bfloat16*>(y), channels,
                                                                            cs, voxels, total8);
  return cudaGetLastError() == cudaSuccess ? FFTLS_OK : FFTLS_E_CUDA;
}

fftls_status fftls_nn_tc_relu_backward(void* dy, const void* y, long long count, void* stream) {
  if (!dy || !y || count < 0 || (count & 7) || !aligned16(dy) || !aligned16(y)) return FFTLS_E_INVALID_ARG;
  if (count == 0) return FFTLS_OK;
  k_cl_relu_bwd<<<grid_for(count / 8), kThreads, 0, (cudaStream_t)stream>>>(
      static_cast<__nv_bfloat16*>(dy), static_cast<const __nv_bfloat16*>(y), count / 8);
  return cudaGetLastError() == cudaSuccess ? FFTLS_OK : FFTLS_E_CUDA;
}

fftls_status fftls_nn_tc_upsample2_backward(const void* dy, void* dx, int batch, int channels, const int nc[3],
                                            void* stream) {
  if (!dy || !dx || batch < 1 || channels < 1 || channels > 64 || !dims_ok(nc) || !aligned16(dy) || !aligned16(dx) ||
      dy == dx)
    return FFTLS_E_INVALID_ARG;
  const int cs = stored_of(channels);
  const long long total8 = (long long)batch * nc[0] * nc[1] * nc[2] * (cs / 8);
  k_cl_up2_bwd<<<grid_for(total8), kThreads, 0, (cudaStream_t)stream>>>(
      static_cast<const __nv_bfloat16*>(dy), static_cast<__nv_bfloat16*>(dx), cs, nc[0], nc[1], nc[2], total8);
  return cudaGetLastError() == cudaSuccess ? FFTLS_OK : FFTLS_E_CUDA;
}

fftls_status fftls_nn_tc_pool2_backward(const void* dy, void* dx, int batch, int channels, const int nc[3],
                                        int accumulate, void* stream) {
  if (!dy || !dx || batch < 1 || channels < 1 || channels > 64 || !dims_ok(nc) || !aligned16(dy) || !aligned16(dx) ||
      dy == dx)
    return FFTLS_E_INVALID_ARG;
  const int cs = stored_of(channels);
  const long long total8 = (long long)batch * 8 * nc[0] * nc[1] * nc[2] * (cs / 8);
  k_cl_pool2_bwd<<<grid_for(total8), kThreads, 0, (cudaStream_t)stream>>>(
      static_cast<const __nv_bfloat16*>(dy), static_cast<__nv_bfloat16*>(dx), cs, nc[0], nc[1], nc[2],
      accumulate ? 1 : 0, total8);
  return cudaGetLastError() == cudaSuccess ? FFTLS_OK : FFTLS_E_CUDA;
}

fftls_status fftls_nn_tc_add(void* y, const void* x, long long count, void* stream) {
  if (!y || !x || count < 0 || (count & 7) || !aligned16(y) || !aligned16(x)) return FFTLS_E_INVALID_ARG;
  if (count == 0) return FFTLS_OK;
  k_cl_add<<<grid_for(count / 8), kThreads, 0, (cudaStream_t)stream>>>(static_cast<__nv_bfloat16*>(y),
                                                                       static_cast<const __nv_bfloat16*>(x), count / 8);
  return cudaGetLastError() == cudaSuccess ? FFTLS_OK : FFTLS_E_CUDA;
}

}  // extern "C"
