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
#include <type_traits>

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

// Tiles of x1-lines (few columns, an odd row stride) pad one row every 16 rows,
// so that the butterflies of the stages with rows 8 or 64 apart, the rows of
// voxels staged in order, and the digit-reversed partners of the real-to-complex
// untangling spread over the shared-memory banks (the period was chosen by
// replaying each phase's addresses per half-warp: at L = 512 one pad row per 8
// rows needs 42 % more wavefronts than conflict-free accesses would, one per 16
// rows 21 %, one per 32 rows 49 %).
constexpr int kPadShift = 4;
__host__ __device__ constexpr int pad_row(int e) { return e + (e >> kPadShift); }
__host__ __device__ constexpr int padded_rows(int n) { return n + ((n + (1 << kPadShift) - 1) >> kPadShift); }
__device__ __forceinline__ int prow(int e, int pad) { return pad ? pad_row(e) : e; }

// Division by a runtime divisor 1 <= d < 2^31 through a multiply-high and a
// shift (Granlund and Montgomery 1994), exact for 0 <= n < 2^31.
struct FastDiv {
  unsigned int m, s;
  int d;
};

__host__ __device__ inline FastDiv make_fastdiv(int d) {
  unsigned int l = 0;
  while ((1u << l) < (unsigned int)d) ++l;
  const unsigned long long m = ((1ull << 32) * ((1ull << l) - (unsigned long long)d)) / (unsigned long long)d + 1ull;
  FastDiv f;
  f.m = (unsigned int)m;
  f.s = l;
  f.d = d;
  return f;
}

__device__ __forceinline__ int fdiv(int n, const FastDiv& f) {
  return (int)((__umulhi((unsigned int)n, f.m) + (unsigned int)n) >> f.s);
}

// Radix plan of a power-of-two length, identical to the host plan: radix 8
// stages, led by one radix-4 stage (log2 L = 2 mod 3), two radix-4 stages
// (log2 L = 1 mod 3, L >= 16) or a single radix-2 stage (L = 2).
__host__ __device__ constexpr int p2_log(int L) { return L <= 1 ? 0 : 1 + p2_log(L / 2); }
__host__ __device__ constexpr int p2_nst(int L) {
  return p2_log(L) % 3 == 0 ? p2_log(L) / 3 : (p2_log(L) % 3 == 2 ? p2_log(L) / 3 + 1 : (p2_log(L) < 3 ? 1 : p2_log(L) / 3 + 1));
}
__host__ __device__ constexpr int p2_radix(int L, int s) {
  return p2_log(L) % 3 == 0 ? 8
       : p2_log(L) % 3 == 2 ? (s == 0 ? 4 : 8)
       : p2_log(L) < 3 ? 2
       : (s < 2 ? 4 : 8);
}
__host__ __device__ constexpr int p2_msize(int L, int s) { return s == 0 ? L : p2_msize(L, s - 1) / p2_radix(L, s - 1); }

// Lengths whose transforms run the compile-time stages (tile_fft_ct).
__host__ __device__ constexpr bool ct_length(int L) { return L == 64 || L == 128 || L == 256 || L == 512; }
// Radix-3 lengths whose strided (x2 / x3) transforms also run compile-time stages, with the host plan:
// the power-of-two plan of L / 3, then one radix-3 stage (48 = 4 4 3, 96 = 4 8 3).
__host__ __device__ constexpr bool r3_length(int L) { return L == 48 || L == 96; }
__host__ __device__ constexpr int ct_nst(int L) { return r3_length(L) ? p2_nst(L / 3) + 1 : p2_nst(L); }
__host__ __device__ constexpr int ct_radix(int L, int s) {
  return r3_length(L) ? (s < p2_nst(L / 3) ? p2_radix(L / 3, s) : 3) : p2_radix(L, s);
}
__host__ __device__ constexpr int ct_msize(int L, int s) { return s == 0 ? L : ct_msize(L, s - 1) / ct_radix(L, s - 1); }
// Twiddle table of a compile-time length, laid out by stage (read by the
// padded x1 tiles): stage s with MR = M / R > 1 (M = msize, R = radix) holds MR
// rows of R complex values, row j = {w^(j T), w^(2 j T), ..., w^((R-1) j T),
// unused} with w = e^{-2 pi i / L} and T = L / M, so a butterfly reads its R - 1
// twiddles as one contiguous 16-byte-aligned row.  stage_tw_offset(L, s) is the
// first entry of stage s; the stages without twiddles (MR = 1) take no rows.
__host__ __device__ constexpr int stage_tw_offset(int L, int s) {
  return s == 0 ? 0 : stage_tw_offset(L, s - 1) + (p2_msize(L, s - 1) > p2_radix(L, s - 1) ? p2_msize(L, s - 1) : 0);
}
// Twiddle-table layouts of an axis (shared memory): kTwPlain, tw[t] = w^t for
// t < L; kTwX1, the stage rows above (the padded x1 tiles of the compile-time
// lengths); kTwStrided, the same rows padded to srow(R) complex values (ten for
// radix 8), read by the x2 / x3 tiles, whose warps touch up to six consecutive
// rows of a stage at once: 80-byte rows put those on distinct banks (64-byte rows
// would place rows j and j + 2 on the same banks).
enum TwLayout : int { kTwPlain = 0, kTwX1 = 1, kTwStrided = 2 };
__host__ __device__ constexpr int srow(int R) { return R == 8 ? 10 : R; }
__host__ __device__ constexpr int strided_tw_offset(int L, int s) {
  return s == 0 ? 0
                : strided_tw_offset(L, s - 1) +
                      (ct_msize(L, s - 1) > ct_radix(L, s - 1)
                           ? (ct_msize(L, s - 1) / ct_radix(L, s - 1)) * srow(ct_radix(L, s - 1))
                           : 0);
}
// Complex entries of an axis's shared-memory twiddle table (even, so that the
// tile after it starts 16-byte aligned): the stage layouts for the compile-time
// lengths, else the plain table.  Written out as constants (checked below) so
// that a kernel pays no run-time recursion for it.
__host__ __device__ constexpr int tw_count(int L, int layout) {
  return layout == kTwX1 ? (L == 64 ? 64 : L == 128 ? 160 : L == 256 ? 320 : L == 512 ? 576 : ((L + 1) & ~1))
       : layout == kTwStrided ? (L == 48 ? 60 : L == 64 ? 80 : L == 96 ? 126 : L == 128 ? 160 : L == 256 ? 336
                                 : L == 512 ? 720 : ((L + 1) & ~1))
       : ((L + 1) & ~1);
}
static_assert(tw_count(64, kTwX1) == stage_tw_offset(64, p2_nst(64)) &&
                  tw_count(128, kTwX1) == stage_tw_offset(128, p2_nst(128)) &&
                  tw_count(256, kTwX1) == stage_tw_offset(256, p2_nst(256)) &&
                  tw_count(512, kTwX1) == stage_tw_offset(512, p2_nst(512)),
              "stage twiddle counts");
static_assert(tw_count(48, kTwStrided) == strided_tw_offset(48, ct_nst(48)) &&
                  tw_count(96, kTwStrided) == strided_tw_offset(96, ct_nst(96)) &&
                  tw_count(64, kTwStrided) == strided_tw_offset(64, p2_nst(64)) &&
                  tw_count(128, kTwStrided) == strided_tw_offset(128, p2_nst(128)) &&
                  tw_count(256, kTwStrided) == strided_tw_offset(256, p2_nst(256)) &&
                  tw_count(512, kTwStrided) == strided_tw_offset(512, p2_nst(512)),
              "strided twiddle counts");

template <int R, typename T2>
__device__ __forceinline__ void dft_fixed(T2* v, bool inv) {
  if (R == 2) dft2(v);
  else if (R == 3) dft3(v, inv);
  else if (R == 4) dft4(v, inv);
  else dft8(v, inv);
}

template <int L, int S, typename T2>
__device__ __forceinline__ void p2_stage(T2* buf, int nblk, int BS, int C, const FastDiv& fc, int ncols, const T2* tw,
                                         bool inv, int pad) {
  constexpr int R = p2_radix(L, S);
  constexpr int M = p2_msize(L, S);
  constexpr int MR = M / R;
  constexpr int NB = L / R;
  constexpr int TSTR = L / M;
  const int total = nblk * NB * ncols;
  const int rs = MR * C;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int rest = fdiv(idx, fc);
    const int c = idx - rest * ncols;
    const int bf = rest & (NB - 1);
    const int blk = rest / NB;
    const int b = bf / MR, j = bf & (MR - 1);
    T2* base = buf + blk * BS + c;
    const int e0 = b * M + j;
    int off[R];
#pragma unroll
    for (int r = 0; r < R; ++r) off[r] = pad ? prow(e0 + r * MR, 1) * C : (e0 * C + r * rs);
    T2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = base[off[r]];
    if (!inv) {
      dft_fixed<R>(v, false);
      if (MR > 1 && j) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[j * r * TSTR]);
      }
    } else {
      if (MR > 1 && j) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmulc(v[r], tw[j * r * TSTR]);
      }
      dft_fixed<R>(v, true);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) base[off[r]] = v[r];
  }
  __syncthreads();
}

template <int L, typename T2>
__device__ void tile_fft_p2(T2* buf, int nblk, int BS, int C, int ncols, const T2* tw, bool inv, int pad) {
  constexpr int NST = p2_nst(L);
  const FastDiv fc = make_fastdiv(ncols);
  if (!inv) {
    if constexpr (NST > 0) p2_stage<L, 0>(buf, nblk, BS, C, fc, ncols, tw, false, pad);
    if constexpr (NST > 1) p2_stage<L, 1>(buf, nblk, BS, C, fc, ncols, tw, false, pad);
    if constexpr (NST > 2) p2_stage<L, 2>(buf, nblk, BS, C, fc, ncols, tw, false, pad);
    if constexpr (NST > 3) p2_stage<L, 3>(buf, nblk, BS, C, fc, ncols, tw, false, pad);
  } else {
    if constexpr (NST > 3) p2_stage<L, 3>(buf, nblk, BS, C, fc, ncols, tw, true, pad);
    if constexpr (NST > 2) p2_stage<L, 2>(buf, nblk, BS, C, fc, ncols, tw, true, pad);
    if constexpr (NST > 1) p2_stage<L, 1>(buf, nblk, BS, C, fc, ncols, tw, true, pad);
    if constexpr (NST > 0) p2_stage<L, 0>(buf, nblk, BS, C, fc, ncols, tw, true, pad);
  }
}

// One twiddle row of the stage layout (R complex values, 16-byte aligned) into
// registers: 16-byte loads for FP32, one load per value for FP64.
template <int R>
__device__ __forceinline__ void load_tw_row(const float2* p, float2* w) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < R / 2; ++i) {
    const float4 t = q[i];
    w[2 * i] = make_float2(t.x, t.y);
    w[2 * i + 1] = make_float2(t.z, t.w);
  }
}
template <int R>
__device__ __forceinline__ void load_tw_row(const double2* p, double2* w) {
#pragma unroll
  for (int i = 0; i < R - 1; ++i) w[i] = p[i];
}

// The R - 1 twiddles w^(r j L / M), r = 1..R-1, of butterfly j of stage S:
// one row of the stage layout (STAGED), else gathered from the plain table.
template <int L, int S, bool STAGED, typename T2>
__device__ __forceinline__ void stage_twiddles(const T2* tw, int j, T2* w) {
  constexpr int R = p2_radix(L, S);
  constexpr int TSTR = L / p2_msize(L, S);
  if (STAGED) {
    load_tw_row<R>(tw + stage_tw_offset(L, S) + j * R, w);
  } else {
    const T2* tj = tw + j * TSTR;
#pragma unroll
    for (int r = 1; r < R; ++r) w[r - 1] = tj[(r - 1) * j * TSTR];
  }
}

// pad_row(e0 + r MR) == pad_row(e0) + r MR + (r MR >> kPadShift) for every butterfly
// (base row e0, leg r) of every stage of the plan of length L.
__host__ __device__ constexpr bool pad_offsets_hold(int L) {
  for (int s = 0; s < p2_nst(L); ++s) {
    const int R = p2_radix(L, s), M = p2_msize(L, s), MR = M / R;
    for (int bf = 0; bf < L / R; ++bf) {
      const int e0 = (bf / MR) * M + bf % MR;
      for (int r = 0; r < R; ++r)
        if (pad_row(e0 + r * MR) != pad_row(e0) + r * MR + ((r * MR) >> kPadShift)) return false;
    }
  }
  return true;
}
static_assert(pad_offsets_hold(64) && pad_offsets_hold(128) && pad_offsets_hold(256) && pad_offsets_hold(512),
              "padded butterfly offsets are compile-time constants");

// Stage S of the power-of-two plan of length L on tiles whose geometry is
// known at compile time: C complex values per row (row stride), the first
// NCOLS columns transformed, rows padded (PAD) or not.  Every butterfly of a
// stage then reads and writes at compile-time offsets from one base address:
// with rows e0 + r MR, the padded row index pad_row(e0 + r MR) equals
// pad_row(e0) + r MR + floor(r MR / 16) for every stage of the compile-time
// lengths (checked below: pad_offsets_hold).
template <int L, int S, int C, int NCOLS, bool PAD, bool INV, typename T2>
__device__ __forceinline__ void p2_stage_ct(T2* buf, int nblk, const T2* tw) {
  constexpr int R = p2_radix(L, S);
  constexpr int M = p2_msize(L, S);
  constexpr int MR = M / R;
  constexpr int NB = L / R;
  constexpr int BS = (PAD ? padded_rows(L) : L) * C;
  const int nbf = nblk * NB;
  const int total = nbf * NCOLS;
  // thread order: consecutive threads take consecutive columns, except in the last
  // stage of the padded x1 tiles (few columns, legs 1 row apart), where consecutive
  // butterflies of one column keep a half-warp on distinct shared-memory banks
  constexpr bool BF_ORDER = PAD && MR == 1;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    int c, rest;
    if (BF_ORDER) {  // c = idx / nbf by at most NCOLS - 1 subtractions (NCOLS is small)
      c = 0;
      rest = idx;
#pragma unroll
      for (int k = 1; k < NCOLS; ++k)
        if (rest >= nbf) {
          rest -= nbf;
          ++c;
        }
    } else {
      rest = idx / NCOLS;
      c = idx - rest * NCOLS;
    }
    const int bf = rest & (NB - 1);
    const int blk = rest / NB;
    const int b = bf / MR, j = bf & (MR - 1);
    const int e0 = b * M + j;
    T2* base = buf + blk * BS + (PAD ? prow(e0, 1) : e0) * C + c;
    T2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = base[(PAD ? r * MR + ((r * MR) >> kPadShift) : r * MR) * C];
    if (!INV) {
      dft_fixed<R>(v, false);
      if (MR > 1 && j) {
        T2 w[R];
        stage_twiddles<L, S, PAD>(tw, j, w);
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], w[r - 1]);
      }
    } else {
      if (MR > 1 && j) {
        T2 w[R];
        stage_twiddles<L, S, PAD>(tw, j, w);
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmulc(v[r], w[r - 1]);
      }
      dft_fixed<R>(v, true);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) base[(PAD ? r * MR + ((r * MR) >> kPadShift) : r * MR) * C] = v[r];
  }
  __syncthreads();
}

template <int L, int C, int NCOLS, bool PAD, typename T2>
__device__ __forceinline__ void tile_fft_p2_ct(T2* buf, int nblk, const T2* tw, bool inv) {
  constexpr int NST = p2_nst(L);
  if (!inv) {
    if constexpr (NST > 0) p2_stage_ct<L, 0, C, NCOLS, PAD, false>(buf, nblk, tw);
    if constexpr (NST > 1) p2_stage_ct<L, 1, C, NCOLS, PAD, false>(buf, nblk, tw);
    if constexpr (NST > 2) p2_stage_ct<L, 2, C, NCOLS, PAD, false>(buf, nblk, tw);
    if constexpr (NST > 3) p2_stage_ct<L, 3, C, NCOLS, PAD, false>(buf, nblk, tw);
  } else {
    if constexpr (NST > 3) p2_stage_ct<L, 3, C, NCOLS, PAD, true>(buf, nblk, tw);
    if constexpr (NST > 2) p2_stage_ct<L, 2, C, NCOLS, PAD, true>(buf, nblk, tw);
    if constexpr (NST > 1) p2_stage_ct<L, 1, C, NCOLS, PAD, true>(buf, nblk, tw);
    if constexpr (NST > 0) p2_stage_ct<L, 0, C, NCOLS, PAD, true>(buf, nblk, tw);
  }
}

// Mixed-radix transform for any supported length (runtime plan).
template <typename T2>
__device__ void tile_fft_generic(T2* buf, int nblk, int BS, int C, int ncols, const AxisPlan& p, const T2* tw, bool inv,
                                 int pad) {
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
      T2* base = buf + blk * BS + c;
      const int e0 = b * M + j;
      T2 v[kMaxRadix];
#pragma unroll
      for (int r = 0; r < kMaxRadix; ++r)
        if (r < R) v[r] = base[pad ? prow(e0 + r * MR, 1) * C : e0 * C + r * rs];
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
        if (r < R) base[pad ? prow(e0 + r * MR, 1) * C : e0 * C + r * rs] = v[r];
    }
    __syncthreads();
  }
}

// In-place transform of a tile (see the file comment) with a runtime tile
// geometry, for the lengths tile_fft_ct does not specialise: the short and the
// longest powers of two run their fixed plans, any other length the runtime
// plan.  tw[t] = e^{-2 pi i t / L} (shared memory).  Ends with __syncthreads()
// when the length has at least one stage.  pad = 1: row e of the tile is stored
// at prow(e) (x1-line tiles).
template <typename T2>
__device__ void tile_fft_rt(T2* buf, int nblk, int BS, int C, int ncols, const AxisPlan& p, const T2* tw, bool inv,
                            int pad) {
  switch (p.L) {
    case 1: return;
    case 2: tile_fft_p2<2>(buf, nblk, BS, C, ncols, tw, inv, pad); return;
    case 4: tile_fft_p2<4>(buf, nblk, BS, C, ncols, tw, inv, pad); return;
    case 8: tile_fft_p2<8>(buf, nblk, BS, C, ncols, tw, inv, pad); return;
    case 16: tile_fft_p2<16>(buf, nblk, BS, C, ncols, tw, inv, pad); return;
    case 32: tile_fft_p2<32>(buf, nblk, BS, C, ncols, tw, inv, pad); return;
    case 1024: tile_fft_p2<1024>(buf, nblk, BS, C, ncols, tw, inv, pad); return;
    default: tile_fft_generic(buf, nblk, BS, C, ncols, p, tw, inv, pad); return;
  }
}

// Stage S of the length-L transform on a strided tile (x2 / x3 passes): one
// block of L rows of C columns, row stride C, NT threads.  Item it = tid + k NT
// is butterfly it / C of column it % C; consecutive threads take consecutive
// columns, so a warp's loads and stores cover contiguous shared memory.  The
// trip count is a compile-time constant, and the butterfly j = 0 multiplies by
// the unit twiddles of its row instead of branching.
template <int L, int S, int C, int NT, bool INV, typename T2>
__device__ __forceinline__ void strided_stage(T2* __restrict__ buf, const T2* __restrict__ tw) {
  constexpr int R = ct_radix(L, S);
  constexpr int M = ct_msize(L, S);
  constexpr int MR = M / R;
  constexpr int NB = L / R;
  constexpr int ITEMS = NB * C;
  constexpr int K = (ITEMS + NT - 1) / NT;
  constexpr int TWO = strided_tw_offset(L, S);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int it = (int)threadIdx.x + k * NT;
    if ((ITEMS % NT) != 0 && it >= ITEMS) break;
    const int bf = it / C;
    const int c = it - bf * C;
    const int j = (int)((unsigned)bf % (unsigned)MR);  // MR compile-time: a mask or a multiply-shift
    T2* base = buf + ((int)((unsigned)bf / (unsigned)MR) * M + j) * C + c;
    T2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = base[r * MR * C];
    if (!INV) {
      dft_fixed<R>(v, false);
      if (MR > 1) {
        T2 w[R];
        load_tw_row<R>(tw + TWO + j * srow(R), w);
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], w[r - 1]);
      }
    } else {
      if (MR > 1) {
        T2 w[R];
        load_tw_row<R>(tw + TWO + j * srow(R), w);
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmulc(v[r], w[r - 1]);
      }
      dft_fixed<R>(v, true);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) base[r * MR * C] = v[r];
  }
  __syncthreads();
}

// The same stage for FP32 tiles of an even column count: item it is butterfly
// it / (C / 2) of the column pair (2 p, 2 p + 1), p = it % (C / 2).  A thread
// moves both columns of a leg with one 16-byte shared-memory access and shares
// the butterfly's twiddle row between them; each column goes through exactly
// the operations of strided_stage, so the results are the same bit for bit.
template <int L, int S, int C, int NT, bool INV>
__device__ __forceinline__ void strided_stage_pair(float2* __restrict__ buf, const float2* __restrict__ tw) {
  static_assert(C % 2 == 0, "column pairs");
  constexpr int R = ct_radix(L, S);
  constexpr int M = ct_msize(L, S);
  constexpr int MR = M / R;
  constexpr int NB = L / R;
  constexpr int CP = C / 2;
  constexpr int ITEMS = NB * CP;
  constexpr int K = (ITEMS + NT - 1) / NT;
  constexpr int TWO = strided_tw_offset(L, S);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int it = (int)threadIdx.x + k * NT;
    if ((ITEMS % NT) != 0 && it >= ITEMS) break;
    const int bf = it / CP;
    const int cp = it - bf * CP;
    const int j = (int)((unsigned)bf % (unsigned)MR);
    float4* base = reinterpret_cast<float4*>(buf + ((int)((unsigned)bf / (unsigned)MR) * M + j) * C) + cp;
    float2 v[R], u[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4 t = base[r * MR * CP];
      v[r] = make_float2(t.x, t.y);
      u[r] = make_float2(t.z, t.w);
    }
    if (!INV) {
      dft_fixed<R>(v, false);
      dft_fixed<R>(u, false);
      if (MR > 1) {
        float2 w[R];
        load_tw_row<R>(tw + TWO + j * srow(R), w);
#pragma unroll
        for (int r = 1; r < R; ++r) {
          v[r] = cmul(v[r], w[r - 1]);
          u[r] = cmul(u[r], w[r - 1]);
        }
      }
    } else {
      if (MR > 1) {
        float2 w[R];
        load_tw_row<R>(tw + TWO + j * srow(R), w);
#pragma unroll
        for (int r = 1; r < R; ++r) {
          v[r] = cmulc(v[r], w[r - 1]);
          u[r] = cmulc(u[r], w[r - 1]);
        }
      }
      dft_fixed<R>(v, true);
      dft_fixed<R>(u, true);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) base[r * MR * CP] = make_float4(v[r].x, v[r].y, u[r].x, u[r].y);
  }
  __syncthreads();
}

// One stage, by column pairs where asked for (PAIR) and the tile allows it (FP32, even C).
template <int L, int S, int C, int NT, bool INV, bool PAIR, typename T2>
__device__ __forceinline__ void strided_stage_any(T2* buf, const T2* tw) {
  if constexpr (PAIR && std::is_same<T2, float2>::value && C % 2 == 0) strided_stage_pair<L, S, C, NT, INV>(buf, tw);
  else strided_stage<L, S, C, NT, INV>(buf, tw);
}

template <int L, int C, int NT, bool INV, bool PAIR, typename T2>
__device__ __forceinline__ void strided_fft(T2* buf, const T2* tw) {
  constexpr int NST = ct_nst(L);
  if (!INV) {
    if constexpr (NST > 0) strided_stage_any<L, 0, C, NT, false, PAIR>(buf, tw);
    if constexpr (NST > 1) strided_stage_any<L, 1, C, NT, false, PAIR>(buf, tw);
    if constexpr (NST > 2) strided_stage_any<L, 2, C, NT, false, PAIR>(buf, tw);
    if constexpr (NST > 3) strided_stage_any<L, 3, C, NT, false, PAIR>(buf, tw);
  } else {
    if constexpr (NST > 3) strided_stage_any<L, 3, C, NT, true, PAIR>(buf, tw);
    if constexpr (NST > 2) strided_stage_any<L, 2, C, NT, true, PAIR>(buf, tw);
    if constexpr (NST > 1) strided_stage_any<L, 1, C, NT, true, PAIR>(buf, tw);
    if constexpr (NST > 0) strided_stage_any<L, 0, C, NT, true, PAIR>(buf, tw);
  }
}

// In-place transform of a strided tile (x2 / x3 passes): the compile-time
// lengths and the radix-3 lengths 48 and 96 run strided_fft (twiddles in the
// kTwStrided layout), any other length the run-time paths (plain table).  All C columns are transformed.
// PAIR: FP32 stages move column pairs (strided_stage_pair).  Measured at 512^3 (CUDA events, two
// runs each): the forward x2 pass 0.6 % faster, the inverse x2 pass 2 % and the x3 pass 0.4 % slower,
// so only the forward x2 pass takes them.
// A tile of L rows of C columns fits the 227 KB of shared memory of a block (the
// compile-time stages are generated only for tiles that can run).
template <typename T2>
__host__ __device__ constexpr bool strided_fits(int L, int C) { return (long long)L * C * (long long)sizeof(T2) <= 232448; }

template <int C, int NT, bool INV, bool PAIR, typename T2>
__device__ void tile_fft_strided(T2* buf, const AxisPlan& p, const T2* tw) {
  switch (p.L) {
    case 48: if constexpr (strided_fits<T2>(48, C)) { strided_fft<48, C, NT, INV, PAIR>(buf, tw); return; } break;
    case 64: if constexpr (strided_fits<T2>(64, C)) { strided_fft<64, C, NT, INV, PAIR>(buf, tw); return; } break;
    case 96: if constexpr (strided_fits<T2>(96, C)) { strided_fft<96, C, NT, INV, PAIR>(buf, tw); return; } break;
    case 128: if constexpr (strided_fits<T2>(128, C)) { strided_fft<128, C, NT, INV, PAIR>(buf, tw); return; } break;
    case 256: if constexpr (strided_fits<T2>(256, C)) { strided_fft<256, C, NT, INV, PAIR>(buf, tw); return; } break;
    case 512: if constexpr (strided_fits<T2>(512, C)) { strided_fft<512, C, NT, INV, PAIR>(buf, tw); return; } break;
    default: break;
  }
  tile_fft_rt(buf, 1, 0, C, C, p, tw, INV, 0);
}

// tile_fft with the tile geometry fixed at compile time (row stride C complex
// values, first NCOLS columns transformed, padded rows when PAD): the lengths
// 64..512 that are powers of two take the compile-time stages, any other
// length the runtime paths.  BS is the block stride of the general path.  tw
// holds tw_count(L, PAD) entries: the padded (x1) tiles of the compile-time
// lengths read the stage layout, every other transform the plain table.
template <int C, int NCOLS, bool PAD, typename T2>
__device__ void tile_fft_ct(T2* buf, int nblk, int BS, const AxisPlan& p, const T2* tw, bool inv) {
  static_assert(ct_length(64) && ct_length(128) && ct_length(256) && ct_length(512), "compile-time lengths");
  switch (p.L) {
    case 64: tile_fft_p2_ct<64, C, NCOLS, PAD>(buf, nblk, tw, inv); return;
    case 128: tile_fft_p2_ct<128, C, NCOLS, PAD>(buf, nblk, tw, inv); return;
    case 256: tile_fft_p2_ct<256, C, NCOLS, PAD>(buf, nblk, tw, inv); return;
    case 512: tile_fft_p2_ct<512, C, NCOLS, PAD>(buf, nblk, tw, inv); return;
    default: tile_fft_rt(buf, nblk, BS, C, NCOLS, p, tw, inv, PAD ? 1 : 0); return;
  }
}

}  // namespace fftls
