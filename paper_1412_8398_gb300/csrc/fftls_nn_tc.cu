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

}  // extern "C"
