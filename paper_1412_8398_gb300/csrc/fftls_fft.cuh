// Shared-memory mixed-radix Stockham FFT building blocks (sm_103a).
//
// Transforms follow the paper's DFT convention (Sec. 3, eq. ft2 / ft):
// forward X[m] = sum_n x[n] e^{-2 pi i m n / L} (unnormalised), inverse with
// the opposite sign and no scaling here (the 1/N of eq. ft is folded into the
// Fourier-space kernel).
//
// A batch of lines lives in shared memory.  Line l starts at
//   base(l) = (l / W) * SA + (l % W) * SB
// and its element e sits at base(l) + e * ES.  One Stockham stage of radix R
// with Ns = product of the radices already applied reads element j + r L/R,
// multiplies by the twiddle W_{Ns R}^{(j mod Ns) r}, runs an R-point DFT in
// registers and writes element (j / Ns) Ns R + (j mod Ns) + r Ns.  Every
// thread first loads all its butterflies, the block synchronises, then all
// threads store: the transform runs in place.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fftls {

constexpr int kMaxStages = 12;
constexpr int kMaxRadix = 8;
constexpr int kPer = 2;  // butterflies per thread per stage (host sizes blocks for this)

struct AxisPlan {
  int L;                    // transform length
  int nst;                  // number of stages
  int radix[kMaxStages];    // radix of each stage, applied in order
};

template <typename T> struct Cplx;
template <> struct Cplx<float> { typedef float2 type; };
template <> struct Cplx<double> { typedef double2 type; };

template <typename T2> __device__ __forceinline__ T2 cmk(decltype(T2::x) a, decltype(T2::x) b) { T2 r; r.x = a; r.y = b; return r; }
template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { return cmk<T2>(a.x + b.x, a.y + b.y); }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { return cmk<T2>(a.x - b.x, a.y - b.y); }
template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) { return cmk<T2>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename T2> __device__ __forceinline__ T2 cconj(T2 a) { return cmk<T2>(a.x, -a.y); }
template <typename T2> __device__ __forceinline__ T2 cscale(T2 a, decltype(T2::x) s) { return cmk<T2>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <typename T2> __device__ __forceinline__ T2 cmul_mi(T2 a, bool inv) { return inv ? cmk<T2>(-a.y, a.x) : cmk<T2>(a.y, -a.x); }

// R-point DFTs in registers. Sign of the exponent: -1 forward, +1 inverse.
template <typename T2>
__device__ __forceinline__ void dft2(T2* v) {
  T2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <typename T2>
__device__ __forceinline__ void dft4(T2* v, bool inv) {
  T2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
  T2 b0 = cadd(v[1], v[3]), b1 = cmul_mi(csub(v[1], v[3]), inv);
  v[0] = cadd(a0, b0);
  v[2] = csub(a0, b0);
  v[1] = cadd(a1, b1);
  v[3] = csub(a1, b1);
}

template <typename T2>
__device__ __forceinline__ void dft8(T2* v, bool inv) {
  typedef decltype(T2::x) T;
  const T h = (T)0.70710678118654752440084436210484903928;  // 1/sqrt(2)
  T2 e[4] = {v[0], v[2], v[4], v[6]};
  T2 o[4] = {v[1], v[3], v[5], v[7]};
  dft4(e, inv);
  dft4(o, inv);
  // twiddles w8^s, s = 0..3: 1, (1 -+ i)/sqrt2, -+i, (-1 -+ i)/sqrt2
  T2 t1 = inv ? cmk<T2>(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
              : cmk<T2>(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
  T2 t2 = cmul_mi(o[2], inv);
  T2 t3 = inv ? cmk<T2>(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
              : cmk<T2>(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
  v[0] = cadd(e[0], o[0]);
  v[4] = csub(e[0], o[0]);
  v[1] = cadd(e[1], t1);
  v[5] = csub(e[1], t1);
  v[2] = cadd(e[2], t2);
  v[6] = csub(e[2], t2);
  v[3] = cadd(e[3], t3);
  v[7] = csub(e[3], t3);
}

template <typename T2>
__device__ __forceinline__ void dft3(T2* v, bool inv) {
  typedef decltype(T2::x) T;
  const T s3 = (T)0.86602540378443864676372317075293618347;  // sin(2 pi / 3)
  T2 a = cadd(v[1], v[2]);
  T2 b = csub(v[1], v[2]);
  T2 y0 = cadd(v[0], a);
  T2 t = cmk<T2>(v[0].x - (T)0.5 * a.x, v[0].y - (T)0.5 * a.y);
  T2 u = cmul_mi(cscale(b, s3), inv);  // -i s3 b (forward)
  v[0] = y0;
  v[1] = cadd(t, u);
  v[2] = csub(t, u);
}

template <typename T2>
__device__ __forceinline__ void dft5(T2* v, bool inv) {
  typedef decltype(T2::x) T;
  const T c1 = (T)0.30901699437494742410229341718281905886;   // cos(2 pi/5)
  const T c2 = (T)-0.80901699437494742410229341718281905886;  // cos(4 pi/5)
  const T s1 = (T)0.95105651629515357211643933337938214340;   // sin(2 pi/5)
  const T s2 = (T)0.58778525229247312916870595463907276860;   // sin(4 pi/5)
  T2 a1 = cadd(v[1], v[4]), a2 = cadd(v[2], v[3]);
  T2 b1 = csub(v[1], v[4]), b2 = csub(v[2], v[3]);
  T2 y0 = cadd(v[0], cadd(a1, a2));
  T2 p1 = cmk<T2>(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
  T2 p2 = cmk<T2>(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
  T2 q1 = cmul_mi(cmk<T2>(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y), inv);
  T2 q2 = cmul_mi(cmk<T2>(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y), inv);
  v[0] = y0;
  v[1] = cadd(p1, q1);
  v[4] = csub(p1, q1);
  v[2] = cadd(p2, q2);
  v[3] = csub(p2, q2);
}

template <typename T2>
__device__ __forceinline__ void dft_r(T2* v, int R, bool inv) {
  switch (R) {
    case 2: dft2(v); break;
    case 3: dft3(v, inv); break;
    case 4: dft4(v, inv); break;
    case 5: dft5(v, inv); break;
    case 8: dft8(v, inv); break;
    default: break;
  }
}

// In-place batched FFT of `nlines` lines of length p.L held in shared memory.
// tw[t] = e^{-2 pi i t / L}, t = 0 .. L-1 (global memory, read through L1).
// Requires nlines * L / min_radix <= kPer * blockDim.x (checked on the host).
template <typename T2>
__device__ void smem_fft(T2* buf, const AxisPlan& p, int nlines, int W, int SA, int SB, int ES,
                         const T2* __restrict__ tw, bool inv) {
  const int L = p.L;
  const int nthr = blockDim.x;
  const int tid = threadIdx.x;
  int Ns = 1;
  for (int s = 0; s < p.nst; ++s) {
    const int R = p.radix[s];
    const int nb = L / R;
    const int total = nlines * nb;
    const int twstride = L / (Ns * R);
    T2 v[kPer][kMaxRadix];
    int dst[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int idx = tid + q * nthr;
      dst[q] = -1;
      if (idx < total) {
        const int line = idx / nb;
        const int j = idx - line * nb;
        const int base = (line / W) * SA + (line % W) * SB;
        const int k = j % Ns;
#pragma unroll
        for (int r = 0; r < kMaxRadix; ++r)
          if (r < R) v[q][r] = buf[base + (j + r * nb) * ES];
        if (Ns > 1) {
#pragma unroll
          for (int r = 1; r < kMaxRadix; ++r) {
            if (r < R) {
              T2 w = __ldg(&tw[k * r * twstride]);
              if (inv) w.y = -w.y;
              v[q][r] = cmul(v[q][r], w);
            }
          }
        }
        dft_r(v[q], R, inv);
        dst[q] = base + ((j / Ns) * Ns * R + k) * ES;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      if (dst[q] >= 0) {
#pragma unroll
        for (int r = 0; r < kMaxRadix; ++r)
          if (r < R) buf[dst[q] + r * Ns * ES] = v[q][r];
      }
    }
    __syncthreads();
    Ns *= R;
  }
}

}  // namespace fftls
