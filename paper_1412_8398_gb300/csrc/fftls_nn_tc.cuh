// Implicit-GEMM convolution kernel of the tensor-core warm-start path, shared by
// the translation units that instantiate it (one per kernel size and input kind).
//
// GEMM view of one convolution: M = output voxels, N = output channels,
// K = taps x input channels (tap-major).  A block stages the input halo of its
// voxel tile in shared memory, channels innermost, so the A operand of every
// tap is the same staged tile shifted by the tap's offset; eight neighbouring
// voxels of one x row form one 8x8 ldmatrix operand.  The B operand (the
// weights) is packed once per layer into the register order of the mma
// fragments and read through the read-only cache, one k step ahead.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fftls_nn.h"

namespace fftls_tc {


constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kMaxSmem = 226 * 1024;  // dynamic shared memory of a block (the tap table is static)

// stored channels of a channels-last activation with c channels
__host__ __device__ constexpr int stored_of(int c) { return c <= 8 ? 8 : c <= 16 ? 16 : c <= 32 ? 32 : 64; }
// shared-memory elements per staged voxel: above 8 channels, 8 more so that the eight rows of one
// ldmatrix (eight neighbouring voxels) start in distinct quads of banks
__host__ __device__ constexpr int pitch_of(int c) { return c >= 16 ? c + 8 : c; }
// m16 tiles per warp for NT n8 tiles: 64 accumulators per thread when N >= 16
__host__ __device__ constexpr int mt_of(int nt) { return nt >= 8 ? 2 : nt == 4 ? 4 : 8; }
__host__ __device__ constexpr int ksteps_of(int c, int ks) { return (ks * ks * ks * c + 15) / 16; }

struct ConvArgs {
  const __nv_bfloat16* x;      // input [batch][m3][m2][m1][C]
  const uint2* w;              // packed B fragments [step][nt][lane]
  const float* bias;           // [c_out] or null
  const __nv_bfloat16* skip;   // [batch][n3][n2][n1][NT*8] or null
  void* y;                     // [batch][n3][n2][n1][NT*8] BF16, or [batch][c_out][n3][n2][n1] FP32
  int n1, n2, n3;              // output grid
  int m1, m2, m3;              // input grid (n, n/2 or 2n)
  int lx, ly, lz;              // voxel tile 2^lx x 2^ly x 2^lz
  int tiles1, tiles2;          // tiles along x1, x2
  int cout, relu, mode, planar, accumulate;
};

__device__ __forceinline__ int wrapn(int v, int n) {
  if (v < 0) v += n;
  if (v >= n) v %= n;
  return v;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Stage the input of an output tile with its halo in shared memory, channels innermost:
// smem[pos][pitch_of(C)], pos = (z * hy + y) * hx + x, the tile origin (x0, y0, z0) on the output grid n,
// the input x (channels-last, C stored channels) on the grid m = n (mode 0), n / 2 (mode 1: nearest
// upsampling) or 2 n (POOL: the 2x2x2 mean, rounded to BF16).  cp.async copies are committed but not waited for.
template <int C, int KS, bool POOL>
__device__ __forceinline__ void stage_halo(const __nv_bfloat16* __restrict__ x, int b, int n1, int n2, int n3, int m1,
                                           int m2, int m3, int mode, int x0, int y0, int z0, int hx, int hy, int hz,
                                           uint32_t sbase) {
  constexpr int P = pitch_of(C);
  constexpr int H = KS / 2;
  constexpr int CH = C / 8;  // 16-byte chunks per voxel
  constexpr int LCH = CH == 1 ? 0 : CH == 2 ? 1 : CH == 4 ? 2 : 3;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // stage the halo tile, one (z, y) row per warp at a time: smem[pos][P], pos = (z * hy + y) * hx + x
  const int rowlen = hx * CH;
  for (int row = warp; !POOL && row < hy * hz; row += kWarps) {
    const int pz = row / hy, py = row - pz * hy;
    const int gy = wrapn(y0 + py - H, n2), gz = wrapn(z0 + pz - H, n3);
    const uint32_t drow = sbase + (uint32_t)(row * hx * P) * 2u;
    for (int c = lane; c < rowlen; c += 32) {
      const int px = c >> LCH, q = c & (CH - 1);
      const int gx = wrapn(x0 + px - H, n1);
      const uint32_t dst = drow + (uint32_t)(px * P + q * 8) * 2u;
      if (mode == 0) {
        cp_async16(dst, x + ((((size_t)b * m3 + gz) * m2 + gy) * m1 + gx) * C + q * 8);
      } else {  // nearest upsampling of the coarse grid
        cp_async16(dst, x + ((((size_t)b * m3 + (gz >> 1)) * m2 + (gy >> 1)) * m1 + (gx >> 1)) * C + q * 8);
      }
    }
  }
  if constexpr (POOL) {  // mean over the 2x2x2 block of the fine grid: all eight loads of a chunk, and of the
                      // lane's next chunk, are issued before any is used
    const int nch = hy * hz * rowlen;
    for (int idx0 = threadIdx.x; idx0 < nch; idx0 += 2 * kThreads) {
      uint4 u[2][8];
      uint32_t dst[2];
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int idx = idx0 + h2 * kThreads;
        const int row = idx / rowlen, c = idx - row * rowlen;
        const int pz = row / hy, py = row - pz * hy;
        const int px = c >> LCH, q = c & (CH - 1);
        const int gx = wrapn(x0 + px - H, n1), gy = wrapn(y0 + py - H, n2), gz = wrapn(z0 + pz - H, n3);
        dst[h2] = sbase + (uint32_t)((row * hx + px) * P + q * 8) * 2u;
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) {
          const size_t v = (((size_t)b * m3 + 2 * gz + (c8 >> 2)) * m2 + 2 * gy + ((c8 >> 1) & 1)) * m1 +
                           2 * gx + (c8 & 1);
          u[h2][c8] = idx < nch ? __ldg(reinterpret_cast<const uint4*>(x + v * C + q * 8)) : make_uint4(0, 0, 0, 0);
        }
      }
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        if (idx0 + h2 * kThreads >= nch) break;
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) {
          const __nv_bfloat162* hv = reinterpret_cast<const __nv_bfloat162*>(&u[h2][c8]);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 f = __bfloat1622float2(hv[e]);
            s[2 * e] += f.x;
            s[2 * e + 1] += f.y;
          }
        }
        uint4 o;
        o.x = pack_bf16(0.125f * s[0], 0.125f * s[1]);
        o.y = pack_bf16(0.125f * s[2], 0.125f * s[3]);
        o.z = pack_bf16(0.125f * s[4], 0.125f * s[5]);
        o.w = pack_bf16(0.125f * s[6], 0.125f * s[7]);
        asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};\n" ::"r"(dst[h2]), "r"(o.x), "r"(o.y), "r"(o.z),
                     "r"(o.w));
      }
    }
  }
}

// y = act(conv(x, W) + bias + skip) for C input channels, NT*8 output channels, kernel size KS; POOL: the
// input is the 2x2x2 mean pooling of a grid twice as fine (else the grid itself or, mode 1, half as fine).
// Tile extents are powers of two, tx >= 8: the eight voxels g = 0..7 of a half m tile share one x row.
template <int C, int NT, int KS, bool POOL>
__global__ void __launch_bounds__(kThreads) k_conv_tc(const ConvArgs a) {
  constexpr int MT = mt_of(NT);
  constexpr int P = pitch_of(C);
  constexpr int H = KS / 2;
  constexpr int KT = KS * KS * KS;
  constexpr int S = ksteps_of(C, KS);
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t toff_tab[KT];
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
  const int b = blockIdx.y;
  int t = blockIdx.x;
  const int i1 = t % a.tiles1;
  t /= a.tiles1;
  const int i2 = t % a.tiles2, i3 = t / a.tiles2;
  const int tx_ = 1 << a.lx, ty_ = 1 << a.ly, tz_ = 1 << a.lz;
  const int x0 = i1 << a.lx, y0 = i2 << a.ly, z0 = i3 << a.lz;
  const int hx = tx_ + 2 * H, hy = ty_ + 2 * H, hz = tz_ + 2 * H;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < KT) {
    const int k = threadIdx.x;
    const int dz = k / (KS * KS), dy = (k / KS) % KS, dx = k % KS;
    toff_tab[k] = (uint32_t)(((dz * hy + dy) * hx + dx) * P) * 2u;
  }

  stage_halo<C, KS, POOL>(a.x, b, a.n1, a.n2, a.n3, a.m1, a.m2, a.m3, a.mode, x0, y0, z0, hx, hy, hz, sbase);
  // the skip values of the tile, after the halo: [m][CS]
  constexpr int CS = NT * 8;
  const uint32_t skbase = sbase + (uint32_t)(hx * hy * hz * P) * 2u;
  if (a.skip) {
    constexpr int SCH = CS / 8;
    constexpr int LSCH = SCH == 1 ? 0 : SCH == 2 ? 1 : SCH == 4 ? 2 : 3;
    const int total = (tx_ * ty_ * tz_) * SCH;
    for (int idx = threadIdx.x; idx < total; idx += kThreads) {
      const int m = idx >> LSCH, q = idx & (SCH - 1);
      const int tx = m & (tx_ - 1), qq = m >> a.lx;
      const int ty = qq & (ty_ - 1), tz = qq >> a.ly;
      const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
      if (x < a.n1 && y < a.n2 && z < a.n3)
        cp_async16(skbase + (uint32_t)(m * CS + q * 8) * 2u,
                   a.skip + ((((size_t)b * a.n3 + z) * a.n2 + y) * a.n1 + x) * CS + q * 8);
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();

  const int jm = lane >> 3, r8 = lane & 7;
  uint32_t arow[MT];
#pragma unroll
  for (int mt = 0; mt < MT; ++mt) {
    const int m = (warp * MT + mt) * 16 + (jm & 1) * 8 + r8;
    const int tx = m & (tx_ - 1), q = m >> a.lx;
    const int ty = q & (ty_ - 1), tz = q >> a.ly;
    arow[mt] = sbase + (uint32_t)(((tz * hy + ty) * hx + tx) * P) * 2u;
  }
  float acc[MT][NT][4];
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;
  // k step s: C >= 16: tap s / (C / 16), channels 16 (s % (C / 16)) + 8 (jm / 2); C = 8: tap 2 s + jm / 2
  const uint2* wp = a.w + lane;
  uint2 bcur[NT];
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) bcur[nt] = __ldg(wp + nt * 32);
#pragma unroll 2
  for (int s = 0; s < S; ++s) {
    uint2 bnext[NT];
    const int sn = s + 1 < S ? s + 1 : s;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) bnext[nt] = __ldg(wp + (sn * NT + nt) * 32);
    uint32_t toff;
    if constexpr (C >= 16) {
      constexpr int CB = C / 16;
      toff = toff_tab[s / CB] + (uint32_t)((s % CB) * 32 + (jm >> 1) * 16);
    } else {
      const int tap = 2 * s + (jm >> 1);
      toff = toff_tab[tap < KT ? tap : KT - 1];
    }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      uint32_t af[4];
      ldsm_x4(af, arow[mt] + toff);
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) mma_bf16(acc[mt][nt], af, bcur[nt]);
    }
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) bcur[nt] = bnext[nt];
  }

  // epilogue: thread holds voxels g and g + 8 of each m tile, channels 2 tq and 2 tq + 1 of each n tile
  const int g = lane >> 2, tq = lane & 3;
  const size_t N = (size_t)a.n1 * a.n2 * a.n3;
  float bias0[NT], bias1[NT];
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const int ch = nt * 8 + 2 * tq;
    bias0[nt] = a.bias && ch < a.cout ? __ldg(a.bias + ch) : 0.f;
    bias1[nt] = a.bias && ch + 1 < a.cout ? __ldg(a.bias + ch + 1) : 0.f;
  }
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      const int m = (warp * MT + mt) * 16 + g + hf * 8;
      const int tx = m & (tx_ - 1), q = m >> a.lx;
      const int ty = q & (ty_ - 1), tz = q >> a.ly;
      const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
      if (x >= a.n1 || y >= a.n2 || z >= a.n3) continue;
      const size_t vl = ((size_t)z * a.n2 + y) * a.n1 + x;
      const size_t v = (size_t)b * N + vl;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int ch = nt * 8 + 2 * tq;
        float v0 = acc[mt][nt][2 * hf] + bias0[nt], v1 = acc[mt][nt][2 * hf + 1] + bias1[nt];
        if (a.skip) {
          uint32_t u;
          asm volatile("ld.shared.u32 %0, [%1];\n" : "=r"(u) : "r"(skbase + (uint32_t)(m * CS + ch) * 2u));
          const float2 sk = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
          v0 += sk.x;
          v1 += sk.y;
        }
        if (a.relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        if (ch >= a.cout) v0 = 0.f;
        if (ch + 1 >= a.cout) v1 = 0.f;
        if (a.planar) {
          float* yp = static_cast<float*>(a.y) + (size_t)b * a.cout * N + vl;
          if (ch < a.cout) yp[(size_t)ch * N] = a.accumulate ? yp[(size_t)ch * N] + v0 : v0;
          if (ch + 1 < a.cout) yp[(size_t)(ch + 1) * N] = a.accumulate ? yp[(size_t)(ch + 1) * N] + v1 : v1;
        } else {
          __nv_bfloat162* yp = reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(a.y) + v * CS + ch);
          if (a.accumulate) {
            const float2 o = __bfloat1622float2(*yp);
            v0 += o.x;
            v1 += o.y;
          }
          *yp = __floats2bfloat162_rn(v0, v1);
        }
      }
    }
}

inline int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

struct Tile {
  int tx, ty, tz;
  size_t smem;
};

// The voxel tile of kWarps * MT * 16 voxels whose staged halo, summed over the grid's tiles, is smallest.
inline bool pick_tile(int voxels, const int* n, int ks, int c, size_t skip_bytes, Tile* out) {
  const int h2 = 2 * (ks / 2);
  // x extent: the grid's, rounded up to a power of two, at least 8 and at most 32 (256 without a halo)
  int tx = 8;
  while (tx < n[0] && tx < (ks == 1 ? 256 : 32) && tx < voxels) tx *= 2;
  bool found = false;
  double best = 0;
  for (int ty = 1; tx * ty <= voxels; ty *= 2) {
    const int tz = voxels / (tx * ty);
    if (tz < 1 || tx * ty * tz != voxels) continue;
    const size_t smem = (size_t)(tx + h2) * (ty + h2) * (tz + h2) * pitch_of(c) * 2 + skip_bytes;
    if (smem > (size_t)kMaxSmem) continue;
    const double tiles = (double)((n[0] + tx - 1) / tx) * ((n[1] + ty - 1) / ty) * ((n[2] + tz - 1) / tz);
    const double cost = tiles * (double)((tx + h2) * (ty + h2) * (tz + h2));
    if (!found || cost < best) {
      best = cost;
      *out = Tile{tx, ty, tz, smem};
      found = true;
    }
  }
  return found;
}

template <int C, int NT, int KS, bool POOL>
fftls_status launch_conv(const ConvArgs& a0, const int* n, int batch, cudaStream_t s) {
  Tile t;
  const int voxels = kWarps * mt_of(NT) * 16;
  if (!pick_tile(voxels, n, KS, C, a0.skip ? (size_t)voxels * NT * 16 : 0, &t)) return FFTLS_E_UNSUPPORTED_SIZE;
  ConvArgs a = a0;
  a.lx = ilog2(t.tx);
  a.ly = ilog2(t.ty);
  a.lz = ilog2(t.tz);
  a.tiles1 = (n[0] + t.tx - 1) / t.tx;
  a.tiles2 = (n[1] + t.ty - 1) / t.ty;
  const long long tiles = (long long)a.tiles1 * a.tiles2 * ((n[2] + t.tz - 1) / t.tz);
  if (tiles > 0x7fffffffLL || batch > 65535) return FFTLS_E_UNSUPPORTED_SIZE;
  if (cudaFuncSetAttribute((const void*)k_conv_tc<C, NT, KS, POOL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)t.smem) != cudaSuccess)
    return FFTLS_E_CUDA;
  k_conv_tc<C, NT, KS, POOL><<<dim3((unsigned)tiles, (unsigned)batch), kThreads, t.smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? FFTLS_OK : FFTLS_E_CUDA;
}

template <int C, int KS, bool POOL>
fftls_status launch_nt(int nt, const ConvArgs& a, const int* n, int batch, cudaStream_t s) {
  switch (nt) {
    case 1: return launch_conv<C, 1, KS, POOL>(a, n, batch, s);
    case 2: return launch_conv<C, 2, KS, POOL>(a, n, batch, s);
    case 4: return launch_conv<C, 4, KS, POOL>(a, n, batch, s);
    default: return launch_conv<C, 8, KS, POOL>(a, n, batch, s);
  }
}

// every (stored input channels, n tiles) of one kernel size and input kind
template <int KS, bool POOL>
fftls_status launch_c(int c, int nt, const ConvArgs& a, const int* n, int batch, cudaStream_t s) {
  switch (c) {
    case 8: return launch_nt<8, KS, POOL>(nt, a, n, batch, s);
    case 16: return launch_nt<16, KS, POOL>(nt, a, n, batch, s);
    case 32: return launch_nt<32, KS, POOL>(nt, a, n, batch, s);
    default: return launch_nt<64, KS, POOL>(nt, a, n, batch, s);
  }
}

// ---------------------------------------------------------------------------
// Weight gradient: dW[o][i][k] = sum over batch and output voxels v of dy(v)[o] x'(v + d(k))[i].
// GEMM view: M = output channels (MO m16 tiles), N = taps x input channels (n = k * C + i), K = voxels.
// A block stages the input halo of a voxel tile (stage_halo) and the tile's dy rows, then each warp
// accumulates its WB column blocks of 16 (all M tiles) over the tile's voxels, 16 at a time; both
// operands come from shared memory through ldmatrix.trans (dy rows are voxels with channels
// innermost: transposed they are the A operand; likewise the input rows for B).  Every block writes
// its partial sums to part[tile][o][n]; k_wgrad_reduce sums the tiles in a fixed order in FP64.
// ---------------------------------------------------------------------------
constexpr int kWB = 2;  // column blocks of 16 per warp

struct WgradArgs {
  const __nv_bfloat16* x;   // layer input, channels-last, C stored channels, grid m
  const __nv_bfloat16* dy;  // gradient at the layer output, channels-last, cso stored channels, grid n
  float* part;              // [tiles][cout][ncols]
  float* partb;             // [tiles][cout]
  int n1, n2, n3, m1, m2, m3, mode;
  int lx, ly, lz, tiles1, tiles2, tiles;  // voxel tile 2^lx x 2^ly x 2^lz; tiles per sample
  int cout, cso, ncols;                   // ncols = KS^3 * C
};

__host__ __device__ constexpr int dy_pitch(int mo) { return 16 * mo + 8; }

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

template <int C, int MO, int KS, bool POOL>
__global__ void __launch_bounds__(kThreads) k_wgrad_tc(const WgradArgs a) {
  constexpr int P = pitch_of(C);
  constexpr int PD = dy_pitch(MO);
  constexpr int H = KS / 2;
  constexpr int KT = KS * KS * KS;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t toff_tab[KT];
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
  const int b = blockIdx.z;
  int t = blockIdx.x;
  const int i1 = t % a.tiles1;
  t /= a.tiles1;
  const int i2 = t % a.tiles2, i3 = t / a.tiles2;
  const int tx_ = 1 << a.lx, ty_ = 1 << a.ly, tz_ = 1 << a.lz;
  const int TV = tx_ * ty_ * tz_;
  const int x0 = i1 << a.lx, y0 = i2 << a.ly, z0 = i3 << a.lz;
  const int hx = tx_ + 2 * H, hy = ty_ + 2 * H, hz = tz_ + 2 * H;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < KT) {
    const int k = threadIdx.x;
    const int dz = k / (KS * KS), dyy = (k / KS) % KS, dx = k % KS;
    toff_tab[k] = (uint32_t)(((dz * hy + dyy) * hx + dx) * P) * 2u;
  }
  stage_halo<C, KS, POOL>(a.x, b, a.n1, a.n2, a.n3, a.m1, a.m2, a.m3, a.mode, x0, y0, z0, hx, hy, hz, sbase);
  // dy rows of the tile after the halo: [m][PD], channels >= cso and voxels outside the grid zero
  const uint32_t dbase = sbase + (uint32_t)(hx * hy * hz * P) * 2u;
  {
    constexpr int DCH = 2 * MO;  // 16-byte chunks of the 16 MO channels a row holds
    const int csoc = a.cso / 8;
    for (int idx = threadIdx.x; idx < TV * DCH; idx += kThreads) {
      const int m = idx / DCH, q = idx - m * DCH;
      const int tx = m & (tx_ - 1), qq = m >> a.lx;
      const int ty = qq & (ty_ - 1), tz = qq >> a.ly;
      const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
      const uint32_t dst = dbase + (uint32_t)(m * PD + q * 8) * 2u;
      if (q < csoc && x < a.n1 && y < a.n2 && z < a.n3)
        cp_async16(dst, a.dy + ((((size_t)b * a.n3 + z) * a.n2 + y) * a.n1 + x) * a.cso + q * 8);
      else
        asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};\n" ::"r"(dst), "r"(0u));
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();

  // bias partial sums (first column group only): warp w sums the voxels m = w mod 8, lane o the channels
  // o and o + 32
  if (blockIdx.y == 0) {
    __shared__ float bsum[kWarps][64];
    for (int o = lane; o < 64; o += 32) {
      float sb = 0.f;
      if (o < a.cout)
        for (int m = warp; m < TV; m += kWarps) {
          unsigned short h;
          asm volatile("ld.shared.u16 %0, [%1];\n" : "=h"(h) : "r"(dbase + (uint32_t)(m * PD + o) * 2u));
          sb += __bfloat162float(__ushort_as_bfloat16(h));
        }
      bsum[warp][o] = sb;
    }
    __syncthreads();
    if (threadIdx.x < a.cout) {
      float sb = 0.f;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) sb += bsum[w][threadIdx.x];
      a.partb[((size_t)b * a.tiles + blockIdx.x) * a.cout + threadIdx.x] = sb;
    }
  }

  const int jm = lane >> 3, r8 = lane & 7;
  const int nblk = (a.ncols + 15) / 16;
  const int blk0 = (blockIdx.y * kWarps + warp) * kWB;
  if (blk0 >= nblk) return;
  // this lane's column offset (tap position and channel) in each of the warp's blocks: B rows are
  // voxels, matrices 2 and 3 of an x4 load the columns 8..15 of the block
  uint32_t coff[kWB];
#pragma unroll
  for (int w = 0; w < kWB; ++w) {
    int col = (blk0 + w) * 16 + (jm >> 1) * 8;
    if (col >= KT * C) col = KT * C - 8;   // a padding column: any valid address, its sums are dropped
    coff[w] = toff_tab[col / C] + (uint32_t)(col % C) * 2u;
  }
  float acc[MO][2 * kWB][4];
#pragma unroll
  for (int mo = 0; mo < MO; ++mo)
#pragma unroll
    for (int nt = 0; nt < 2 * kWB; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[mo][nt][e] = 0.f;
  for (int v0 = 0; v0 < TV; v0 += 16) {
    // A: dy^T, rows o, k = voxels v0..v0+15; matrix j: voxels v0 + 8 (j / 2) + r, channels 8 (j % 2)
    const int va = v0 + (jm >> 1) * 8 + r8;
    uint32_t af[MO][4];
#pragma unroll
    for (int mo = 0; mo < MO; ++mo) ldsm_x4_t(af[mo], dbase + (uint32_t)(va * PD + mo * 16 + (jm & 1) * 8) * 2u);
    // B: rows k = voxels v0 + 8 (j % 2) + r at their halo positions
    const int vb = v0 + (jm & 1) * 8 + r8;
    const int tx = vb & (tx_ - 1), qq = vb >> a.lx;
    const int ty = qq & (ty_ - 1), tz = qq >> a.ly;
    const uint32_t brow = sbase + (uint32_t)(((tz * hy + ty) * hx + tx) * P) * 2u;
#pragma unroll
    for (int w = 0; w < kWB; ++w) {
      uint32_t bf[4];
      ldsm_x4_t(bf, brow + coff[w]);
      const uint2 b0 = make_uint2(bf[0], bf[1]), b1 = make_uint2(bf[2], bf[3]);
#pragma unroll
      for (int mo = 0; mo < MO; ++mo) {
        mma_bf16(acc[mo][2 * w], af[mo], b0);
        mma_bf16(acc[mo][2 * w + 1], af[mo], b1);
      }
    }
  }
  // partial sums: thread holds rows o = 16 mo + g (+8), columns 8 nt + 2 tq (+1)
  const int g = lane >> 2, tq = lane & 3;
  float* dst = a.part + ((size_t)b * a.tiles + blockIdx.x) * a.cout * a.ncols;
#pragma unroll
  for (int mo = 0; mo < MO; ++mo)
#pragma unroll
    for (int nt = 0; nt < 2 * kWB; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int o = 16 * mo + g + (e >> 1) * 8;
        const int n = (blk0 + nt / 2) * 16 + (nt & 1) * 8 + 2 * tq + (e & 1);
        if (o < a.cout && n < a.ncols) dst[(size_t)o * a.ncols + n] = acc[mo][nt][e];
      }
}

template <int C, int MO, int KS, bool POOL>
fftls_status launch_wgrad(const WgradArgs& a0, const int* n, int batch, int tv, cudaStream_t s) {
  Tile t;
  const size_t dbytes = (size_t)tv * dy_pitch(MO) * 2;
  if (!pick_tile(tv, n, KS, C, dbytes, &t)) return FFTLS_E_UNSUPPORTED_SIZE;
  WgradArgs a = a0;
  a.lx = ilog2(t.tx);
  a.ly = ilog2(t.ty);
  a.lz = ilog2(t.tz);
  a.tiles1 = (n[0] + t.tx - 1) / t.tx;
  a.tiles2 = (n[1] + t.ty - 1) / t.ty;
  const long long tiles = (long long)a.tiles1 * a.tiles2 * ((n[2] + t.tz - 1) / t.tz);
  if (tiles != a.tiles) return FFTLS_E_INVALID_ARG;
  const int groups = ((a.ncols + 15) / 16 + kWarps * kWB - 1) / (kWarps * kWB);
  if (cudaFuncSetAttribute((const void*)k_wgrad_tc<C, MO, KS, POOL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)t.smem) != cudaSuccess)
    return FFTLS_E_CUDA;
  k_wgrad_tc<C, MO, KS, POOL><<<dim3((unsigned)tiles, (unsigned)groups, (unsigned)batch), kThreads, t.smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? FFTLS_OK : FFTLS_E_CUDA;
}

// The voxel tile of the weight gradient: 1024 voxels where the staged halo and dy rows fit, else 512, 256.
inline int wgrad_tile_voxels(const int* n, int ks, int c, int mo) {
  for (int tv = 1024; tv >= 256; tv /= 2) {
    Tile t;
    if (pick_tile(tv, n, ks, c, (size_t)tv * dy_pitch(mo) * 2, &t)) return tv;
  }
  return 0;
}

inline long long wgrad_tiles(const int* n, int ks, int c, int mo) {
  const int tv = wgrad_tile_voxels(n, ks, c, mo);
  Tile t;
  if (tv == 0 || !pick_tile(tv, n, ks, c, (size_t)tv * dy_pitch(mo) * 2, &t)) return 0;
  return (long long)((n[0] + t.tx - 1) / t.tx) * ((n[1] + t.ty - 1) / t.ty) * ((n[2] + t.tz - 1) / t.tz);
}

template <int KS, bool POOL>
fftls_status launch_wgrad_c(int c, int mo, const WgradArgs& a, const int* n, int batch, int tv, cudaStream_t s) {
#define FFTLS_WG(CC)                                                           \
  switch (mo) {                                                                \
    case 1: return launch_wgrad<CC, 1, KS, POOL>(a, n, batch, tv, s);          \
    case 2: return launch_wgrad<CC, 2, KS, POOL>(a, n, batch, tv, s);          \
    default: return launch_wgrad<CC, 4, KS, POOL>(a, n, batch, tv, s);         \
  }
  switch (c) {
    case 8: FFTLS_WG(8)
    case 16: FFTLS_WG(16)
    case 32: FFTLS_WG(32)
    default: FFTLS_WG(64)
  }
#undef FFTLS_WG
}

fftls_status launch_wgrad_k1(bool pool, int c, int mo, const WgradArgs& a, const int* n, int batch, int tv,
                             cudaStream_t s);
fftls_status launch_wgrad_k3(bool pool, int c, int mo, const WgradArgs& a, const int* n, int batch, int tv,
                             cudaStream_t s);

fftls_status launch_k1(bool pool, int c, int nt, const ConvArgs& a, const int* n, int batch, cudaStream_t s);
fftls_status launch_k3(int c, int nt, const ConvArgs& a, const int* n, int batch, cudaStream_t s);
fftls_status launch_k3_pool(int c, int nt, const ConvArgs& a, const int* n, int batch, cudaStream_t s);

}  // namespace fftls_tc
