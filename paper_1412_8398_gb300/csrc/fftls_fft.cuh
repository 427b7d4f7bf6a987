// Shared-memory mixed-radix FFT building blocks (sm_103a).
//
// Transforms follow the paper's DFT convention (Sec. 3, eq. ft2 / ft):
// forward X[m] = sum_n x[n] e^{-2 pi i m n / L} (unnormalised), inverse with
// the opposite sign and no scaling here (the 1/N of eq. ft is folded into the
// Fourier-space kernel).
//
// Tiles live in shared memory as [block][row e][column c]: element (b, e, c)
// sits at b * BS + e * C + c; the transform runs along e (length L) for every
// column c < ncols of every block.  The forward transform is an in-place
// decimation in frequency: natural order in, digit-reversed order out (position
// p holds frequency perm(p), see AxisPlan).  The inverse is the matching
// decimation in time: digit-reversed in, natural order out.  Each butterfly
// reads and writes the same R locations, so a stage needs no buffering across
// threads and a block may loop over any number of butterflies; one
// __syncthreads() separates stages.  The spectrum is never reordered: the
// Fourier-space kernel maps positions to frequencies through per-axis tables.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fftls {

constexpr int kMaxStages = 12;
constexpr int kMaxRadix = 8;

// Stage s (s = 0 first in the forward transform) has radix radix[s] and acts on
// sub-sequences of length msize[s] = L / (radix[0] ... radix[s-1]).  Position
// p = s_0 L/R_0 + s_1 L/(R_0 R_1) + ... holds frequency s_0 + R_0 (s_1 + R_1 (...)).
struct AxisPlan {
  int L;
  int nst;
  int radix[kMaxStages];
  int msize[kMaxStages];
};

template <typename T> struct Cplx;
template <> struct Cplx<float> { typedef float2 type; };
template <> struct Cplx<double> { typedef double2 type; };

template <typename T2> __device__ __forceinline__ T2 cmk(decltype(T2::x) a, decltype(T2::x) b) { T2 r; r.x = a; r.y = b; return r; }
template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { return cmk<T2>(a.x + b.x, a.y + b.y); }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { return cmk<T2>(a.x - b.x, a.y - b.y); }
template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) { return cmk<T2>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// a * conj(b)
template <typename T2> __device__ __forceinline__ T2 cmulc(T2 a, T2 b) { return cmk<T2>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }
template <typename T2> __device__ __forceinline__ T2 cconj(T2 a) { return cmk<T2>(a.x, -a.y); }
template <typename T2> __device__ __forceinline__ T2 cscale(T2 a, decltype(T2::x) s) { return cmk<T2>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <typename T2> __device__ __forceinline__ T2 cmul_mi(T2 a, bool inv) { return inv ? cmk<T2>(-a.y, a.x) : cmk<T2>(a.y, -a.x); }

// R-point DFTs in registers, output in natural order.  Exponent sign -1
// forward, +1 inverse.
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
  // o[s] * w8^s, w8 = e^{-+ i pi / 4}
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
  T2 u = cmul_mi(cscale(b, s3), inv);
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

// In-place transform of a tile (see the file comment).  tw[t] = e^{-2 pi i t / L}
// (shared memory).  Ends with __syncthreads().
template <typename T2>
__device__ void tile_fft(T2* buf, int nblk, int BS, int C, int ncols, const AxisPlan& p, const T2* tw, bool inv) {
  const int L = p.L;
  for (int si = 0; si < p.nst; ++si) {
    const int s = inv ? p.nst - 1 - si : si;
    const int R = p.radix[s];
    const int M = p.msize[s];
    const int MR = M / R;
    const int tstr = L / M;
    const int nb = L / R;
    const int total = nblk * nb * ncols;
    const int rs = MR * C;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int c = idx % ncols;
      const int rest = idx / ncols;
      const int bf = rest % nb;
      const int blk = rest / nb;
      const int b = bf / MR, j = bf - b * MR;
      T2* base = buf + blk * BS + (b * M + j) * C + c;
      T2 v[kMaxRadix];
#pragma unroll
      for (int r = 0; r < kMaxRadix; ++r)
        if (r < R) v[r] = base[r * rs];
      if (!inv) {
        dft_r(v, R, false);
        if (j) {
#pragma unroll
          for (int r = 1; r < kMaxRadix; ++r)
            if (r < R) v[r] = cmul(v[r], tw[j * r * tstr]);
        }
      } else {
        if (j) {
#pragma unroll
          for (int r = 1; r < kMaxRadix; ++r)
            if (r < R) v[r] = cmulc(v[r], tw[j * r * tstr]);
        }
        dft_r(v, R, true);
      }
#pragma unroll
      for (int r = 0; r < kMaxRadix; ++r)
        if (r < R) base[r * rs] = v[r];
    }
    __syncthreads();
  }
}

}  // namespace fftls
