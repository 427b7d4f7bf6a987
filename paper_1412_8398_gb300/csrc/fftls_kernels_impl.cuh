#pragma once
// CUDA kernels of the FFT Lippmann-Schwinger iteration (Willot 2015), sm_103a.
// Implementation header: the kernel and launcher templates.  The translation
// units fftls_kernels_x32/_x64.cu (x1 passes, eta, reductions, helpers),
// _y32/_y64 (x2 pass) and _z32/_z64 (x3 + Fourier pass) each instantiate their
// share, so the library's kernels compile in parallel.
//
// One iteration is five passes over the fields in HBM:
//   K1 fwd_x     : sigma = C(x):eps (and tau = sigma - C0:eps) per voxel,
//                  fused with the x1 real-to-half-complex transform; FP64 sums
//                  of <sigma>, <eps>                          (eq. ls, a1)
//   K2 mid_y     : transform along x2 (forward)
//   K3 fourier_z : transform along x3, then per mode the equilibrium norm
//                  |k* . sigma_hat|^2 and e_hat = -G'(k):x_hat, the mean mode,
//                  the 1/N of eq. ft, then the inverse transform along x3
//                                                             (eq. discFour2, criterion)
//   R  reduce_eta: eta, <sigma> history and the stop decision (one block)
//   K2 mid_y     : inverse transform along x2
//   K5 inv_x     : half-complex-to-real along x1 fused with the scheme update
//                  (eq. ds or eq. as), optional max |delta| for the max-delta stop
// The half spectrum is array-of-structures [x3 pos][x2 pos][x1][component]: a
// strided pass reads rows of W modes x n_c components (192 contiguous bytes in
// FP32 with W = 4, n_c = 6).  Along x2 and x3 the spectrum is kept in the
// digit-reversed order of the in-place transforms (see fftls_fft.cuh).
#include <math.h>

#include "fftls_kernels.cuh"

namespace fftls {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
// The view of sample s of a grouped launch: its fields and parameters.
template <typename T>
__device__ __forceinline__ void at_sample(IterArgs<T>& a, int s) {
  a.eps += s * a.st_field;
  a.phase += s * a.st_phase;
  a.coef += s * a.st_coef;
  a.specA += s * a.st_spec;
  a.specB += s * a.st_spec;
  a.ctrl += s;
  a.part_mean += s * a.st_pmean;
  a.part_eta += s * a.st_peta;
  a.part_delta += s * a.st_pdelta;
  a.eta_hist += s * a.st_hist;
  a.ms_hist += s * a.st_hist * 6;
  a.rfield += s * a.st_field;
  a.d64 += s * a.st_d64;
  const double* p = a.smp_par + 8 * s;
  a.lam0 = p[0];
  a.mu0 = p[1];
#pragma unroll
  for (int i = 0; i < 6; ++i) a.eps_bar[i] = p[2 + i];
}

template <int DIM> struct Comp;
template <> struct Comp<3> {
  static constexpr int NC = 6;
  __device__ static constexpr int I(int c) { return c < 3 ? c : (c == 3 ? 1 : 0); }
  __device__ static constexpr int J(int c) { return c < 3 ? c : (c == 5 ? 1 : 2); }
};
template <> struct Comp<2> {
  static constexpr int NC = 3;
  __device__ static constexpr int I(int c) { return c < 2 ? c : 0; }
  __device__ static constexpr int J(int c) { return c < 2 ? c : 1; }
};

// Block-wide FP64 sum of W values per thread; result valid in thread 0.
template <int W>
__device__ void block_sum(double (&v)[W]) {
  __shared__ double red[32][W];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    double x = v[i];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    v[i] = x;
  }
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < W; ++i) red[warp][i] = v[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < W; ++i) {
      double x = lane < nw ? red[lane][i] : 0.0;
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[i] = x;
    }
  }
  __syncthreads();
}

template <int W>
__device__ void block_max(double (&v)[W]) {
  __shared__ double red[32][W];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    double x = v[i];
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    v[i] = x;
  }
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < W; ++i) red[warp][i] = v[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < W; ++i) {
      double x = lane < nw ? red[lane][i] : 0.0;
      for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
      v[i] = x;
    }
  }
  __syncthreads();
}

// Dynamic shared memory: twiddles of the transformed axis (tw_count(L, layout)
// entries: kTwX1 for the x1 tiles, kTwStrided for the x2 / x3 tiles), then the tile.
template <typename T2>
__device__ __forceinline__ T2* load_twiddles(const T2* __restrict__ tw, int L, int layout, T2** tile) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* tws = reinterpret_cast<T2*>(smem_raw);
  const int n = tw_count(L, layout);
  for (int t = threadIdx.x; t < n; t += blockDim.x) tws[t] = tw[t];
  *tile = tws + n;
  __syncthreads();
  return tws;
}

__host__ __device__ constexpr int odd_stride(int n) { return (n & 1) ? n : n + 1; }

// 16-byte asynchronous copy global -> shared (bypasses registers and L1), so a
// block keeps all loads of a tile in flight at once.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Bulk copies between global and shared memory (the copy engine of sm_90+: one instruction per
// contiguous run of bytes, 16-byte aligned, a multiple of 16 bytes long); completion of loads is
// counted in bytes on an mbarrier in shared memory.
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(src), "r"(bytes)
               : "memory");
}
// commit the thread's bulk stores and wait until they have read shared memory (the block may then
// exit; the global writes complete with the kernel)
__device__ __forceinline__ void bulk_commit_and_wait() {
  asm volatile("cp.async.bulk.commit_group;\ncp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// try_wait rounds before a tile load is declared lost (each round may suspend the thread for a while)
constexpr long long kBulkWaitRounds = 1LL << 16;

// L2 prefetch of the fields of voxels [v0, v0 + nvox) (n_c components of eps and the
// phase ids): one prefetch per 128-byte line, spread over the block's threads, so that
// loads issued later in the kernel hit L2 instead of waiting on DRAM.
template <typename T>
__device__ __forceinline__ void prefetch_voxels(const T* eps, const uint8_t* phase, long long N, int nc, long long v0,
                                                int nvox) {
  constexpr int PER = 128 / sizeof(T);
  const int lines = (nvox + PER - 1) / PER + 1;  // +1: the run need not start on a line
  for (int t = threadIdx.x; t < nc * lines; t += blockDim.x) {
    const int c = t / lines, l = t - c * lines;
    const long long v = min(v0 + (long long)l * PER, v0 + nvox - 1);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(eps + (long long)c * N + v));
  }
  for (int l = threadIdx.x; l <= nvox / 128; l += blockDim.x)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(phase + v0 + min((long long)l * 128, (long long)nvox - 1)));
}

// Copy `rows` rows of `cols` complex values between a tile (row stride C, a
// compile-time width) and global memory (row stride gstride, in complex values).
// Rows of whole 16-byte units with 16-byte aligned starts go through cp.async
// (loads) and 16-byte vector accesses; anything else element by element.  Full
// rows (cols == C) split the work with compile-time divisions; only a partial
// tile builds a run-time divider (a 64-bit division per thread).
// Whether a strided tile moves by bulk copies: every row of cols values starts 16-byte aligned in
// global and shared memory and is a multiple of 16 bytes long.
template <int C, typename T2>
__device__ __forceinline__ bool tile_bulk_ok(const T2* tile, const T2* g, long long gstride, int cols) {
  return ((C * sizeof(T2)) % 16 == 0) && ((cols * sizeof(T2)) % 16 == 0) && ((gstride * sizeof(T2)) % 16 == 0) &&
         (((size_t)g & 15) == 0) && (((size_t)tile & 15) == 0);
}

// rows x cols values from g (row stride gstride) into tile (row stride C), by bulk copies of whole
// rows (BULK, where tile_bulk_ok) or by 16-byte copies per thread.  Returns false, with the solve
// stopped (ctl->fault = 1, state kStopped) and nothing else done, when a bulk copy has not completed
// after kBulkWaitRounds waits; every thread of the block returns the same value.  (Measured at 512^3:
// the bulk copies speed up the x3 pass, whose transforms and G' overlap them, by 8 % and slow the
// memory-bound x2 pass by 7 %, so only the x3 pass takes them.)
template <int C, bool BULK, typename T2>
__device__ __forceinline__ bool tile_load(T2* tile, const T2* g, long long gstride, int rows, int cols, Ctrl* ctl) {
  if (BULK && tile_bulk_ok<C>(tile, g, gstride, cols)) {
    __shared__ __align__(8) unsigned long long bar_word;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&bar_word);
    const uint32_t row_bytes = (uint32_t)(cols * sizeof(T2));
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
      mbar_arrive_expect_tx(bar, row_bytes * (uint32_t)rows);
    }
    __syncthreads();
    const uint32_t t0 = (uint32_t)__cvta_generic_to_shared(tile);
    for (int r = threadIdx.x; r < rows; r += blockDim.x)
      bulk_load(t0 + (uint32_t)(r * C * sizeof(T2)), g + r * gstride, row_bytes, bar);
    bool done = false;
    for (long long k = 0; k < kBulkWaitRounds && !done; ++k) done = mbar_try_wait(bar, 0);
    const bool lost = __syncthreads_or(!done);
    if (lost) {
      if (threadIdx.x == 0) {
        ctl->fault = 1;
        ctl->state = kStopped;
      }
      // the block's own copies: one more bounded wait before the block gives up its shared memory
      for (long long k = 0; k < kBulkWaitRounds && !done; ++k) done = mbar_try_wait(bar, 0);
      return false;
    }
    return true;
  }
  constexpr int PER = 16 / sizeof(T2);
  const bool vec = (C % PER == 0) && (cols % PER == 0) && ((gstride * sizeof(T2)) % 16 == 0) &&
                   (((size_t)g & 15) == 0);
  if (vec) {
    constexpr int UC = C / PER;
    const bool full = cols == C;
    const int U = cols / PER;
    FastDiv fu = {0u, 0u, 1};
    if (!full) fu = make_fastdiv(U);
    for (int idx = threadIdx.x; idx < rows * U; idx += blockDim.x) {
      const int r = full ? (int)((unsigned)idx / UC) : fdiv(idx, fu), u = idx - r * U;
      cp_async16(tile + r * C + u * PER, g + r * gstride + u * PER);
    }
    cp_async_wait_all();
  } else {
    const FastDiv fc = make_fastdiv(cols);
    for (int idx = threadIdx.x; idx < rows * cols; idx += blockDim.x) {
      const int r = fdiv(idx, fc), cc = idx - r * cols;
      tile[r * C + cc] = g[r * gstride + cc];
    }
  }
  __syncthreads();
  return true;
}

template <int C, bool BULK, typename T2>
__device__ __forceinline__ void tile_store(const T2* tile, T2* g, long long gstride, int rows, int cols) {
  if (BULK && tile_bulk_ok<C>(tile, g, gstride, cols)) {
    // the tile was written through ordinary stores: order them before the copy engine reads it
    fence_async_shared();
    __syncthreads();
    const uint32_t t0 = (uint32_t)__cvta_generic_to_shared(tile);
    const uint32_t row_bytes = (uint32_t)(cols * sizeof(T2));
    bool issued = false;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
      bulk_store(g + r * gstride, t0 + (uint32_t)(r * C * sizeof(T2)), row_bytes);
      issued = true;
    }
    if (issued) bulk_commit_and_wait();
    return;
  }
  constexpr int PER = 16 / sizeof(T2);
  const bool vec = (C % PER == 0) && (cols % PER == 0) && ((gstride * sizeof(T2)) % 16 == 0) &&
                   (((size_t)g & 15) == 0);
  if (vec) {
    constexpr int UC = C / PER;
    const bool full = cols == C;
    const int U = cols / PER;
    FastDiv fu = {0u, 0u, 1};
    if (!full) fu = make_fastdiv(U);
    for (int idx = threadIdx.x; idx < rows * U; idx += blockDim.x) {
      const int r = full ? (int)((unsigned)idx / UC) : fdiv(idx, fu), u = idx - r * U;
      *reinterpret_cast<float4*>(g + r * gstride + u * PER) = *reinterpret_cast<const float4*>(tile + r * C + u * PER);
    }
  } else {
    const FastDiv fc = make_fastdiv(cols);
    for (int idx = threadIdx.x; idx < rows * cols; idx += blockDim.x) {
      const int r = fdiv(idx, fc), cc = idx - r * cols;
      g[r * gstride + cc] = tile[r * C + cc];
    }
  }
}

// two adjacent complex values (16-byte aligned in FP32: one vector store)
__device__ __forceinline__ void store_pair(float2* d, float2 a, float2 b) {
  *reinterpret_cast<float4*>(d) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void store_pair(double2* d, double2 a, double2 b) {
  d[0] = a;
  d[1] = b;
}
__device__ __forceinline__ void load_pair(const float2* d, float2& a, float2& b) {
  const float4 v = *reinterpret_cast<const float4*>(d);
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void load_pair(const double2* d, double2& a, double2& b) {
  a = d[0];
  b = d[1];
}

// ---------------------------------------------------------------------------
// K1: constitutive law + forward x1 transform (real -> half complex)
// ---------------------------------------------------------------------------
// VB: voxels per thread whose loads are issued together (a tuned trade of
// registers against loads in flight).
// One voxel of the forward x1 pass: sigma = C(x) : eps and the packed row of the
// transformed fields (tau, or sigma in the sigma form; tau and sigma for DUAL),
// two real components per complex column; the FP32 sums of sigma and eps gathered.
template <typename T, int DIM, bool DUAL>
__device__ __forceinline__ void fwd_x_voxel(const IterArgs<T>& a, const T (&e)[Comp<DIM>::NC], int ph,
                                            T (&accf)[2 * Comp<DIM>::NC], typename Cplx<T>::type* row) {
  typedef typename Cplx<T>::type T2;
  constexpr int NC = Comp<DIM>::NC;
  constexpr int nout = DUAL ? 2 * NC : NC;
  constexpr int NP = (nout + 1) / 2;
  const T* cf = a.coef + ph * kCoef;
  const T lam = cf[0], mu2 = cf[1], dlam = cf[2], dmu2 = cf[3];
  T tr = e[0] + e[1];
  if (DIM == 3) tr += e[2];
  T out[nout];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const bool diag = c < DIM;
    const T s = mu2 * e[c] + (diag ? lam * tr : (T)0);
    accf[c] += s;
    accf[NC + c] += e[c];
    if (DUAL) {
      out[c] = dmu2 * e[c] + (diag ? dlam * tr : (T)0);
      out[NC + c] = s;
    } else {
      out[c] = a.tauform ? dmu2 * e[c] + (diag ? dlam * tr : (T)0) : s;
    }
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    T2 w;
    w.x = out[2 * p];
    w.y = (2 * p + 1 < nout) ? out[2 * p + 1] : (T)0;
    row[p] = w;
  }
}

// The packed real transforms of a batch of nl lines (tile, line stride BS) untangled
// into the half spectrum of lines l0 ... l0 + nl - 1: one thread per mode k, every
// component of it.
template <typename T, int DIM, bool DUAL>
__device__ __forceinline__ void fwd_x_untangle(const IterArgs<T>& a, const typename Cplx<T>::type* tile, int nl,
                                               long long l0, int BS, const FastDiv& fH) {
  typedef typename Cplx<T>::type T2;
  constexpr int NC = Comp<DIM>::NC;
  constexpr int nout = DUAL ? 2 * NC : NC;
  constexpr int NP = (nout + 1) / 2;
  constexpr int CP = odd_stride(NP);
  const int L1 = a.g.n1, H = a.g.H;
  const int* __restrict__ pos = a.pos[0];
  for (int idx = threadIdx.x; idx < nl * H; idx += blockDim.x) {
    const int gl = fdiv(idx, fH), k = idx - gl * H;
    const T2* r0 = tile + gl * BS + prow(__ldg(&pos[k]), 1) * CP;
    const T2* r1 = tile + gl * BS + prow(__ldg(&pos[k == 0 ? 0 : L1 - k]), 1) * CP;
    const long long m = (l0 + gl) * (long long)H + k;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const T2 Z = r0[p], Zm = r1[p];
      T2 A, B;
      A.x = (T)0.5 * (Z.x + Zm.x);
      A.y = (T)0.5 * (Z.y - Zm.y);
      B.x = (T)0.5 * (Z.y + Zm.y);
      B.y = (T)-0.5 * (Z.x - Zm.x);
      const int o0 = 2 * p, o1 = 2 * p + 1;
      T2* d0 = (o0 < NC ? a.specA : a.specB) + m * NC + (o0 % NC);
      if (NC % 2 == 0 && o1 < nout && (o0 < NC) == (o1 < NC)) {
        store_pair(d0, A, B);  // components o0 (even), o1 adjacent in one spectrum: 16-byte aligned
      } else {
        *d0 = A;
        if (o1 < nout) (o1 < NC ? a.specA : a.specB)[m * NC + (o1 % NC)] = B;
      }
    }
  }
}

template <typename T, int DIM, bool DUAL, int VB>
__device__ __forceinline__ void k_fwd_x_body(const IterArgs<T>& a, const AxisPlan* pl) {
  typedef typename Cplx<T>::type T2;
  constexpr int NC = Comp<DIM>::NC;
  if (a.ctrl->state != kRunning) return;
  const Geom g = a.g;
  const int L1 = g.n1, H = g.H;
  T2* tile;
  const T2* tws = load_twiddles(a.tw[0], L1, kTwX1, &tile);
  constexpr int nout = DUAL ? 2 * NC : NC;
  constexpr int NP = (nout + 1) / 2;
  constexpr int CP = odd_stride(NP);
  const int BS = padded_rows(L1) * CP;
  const long long nlines = (long long)g.n2 * g.n3;
  const int G = a.x1_lines;
  // FP64 running sums of <sigma>, <eps> per warp (the FP32 sums of one batch are
  // reduced over the warp and added here by lane 0)
  __shared__ double wacc[8][2 * NC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < 8 * 2 * NC; i += blockDim.x) (&wacc[0][0])[i] = 0.0;

  const FastDiv fL = make_fastdiv(L1), fH = make_fastdiv(H);
  for (long long l0 = (long long)blockIdx.x * G; l0 < nlines; l0 += (long long)gridDim.x * G) {
    const int nl = (int)min((long long)G, nlines - l0);
    T accf[2 * NC];
#pragma unroll
    for (int c = 0; c < 2 * NC; ++c) accf[c] = (T)0;
    for (int ib = threadIdx.x; ib < nl * L1; ib += VB * blockDim.x) {
      T ev[VB][NC];
      int phv[VB];
#pragma unroll
      for (int v = 0; v < VB; ++v) {
        const int idx = ib + v * blockDim.x;
        if (idx < nl * L1) {
          const int gl = fdiv(idx, fL), x = idx - gl * L1;
          const long long vox = (l0 + gl) * (long long)L1 + x;
          phv[v] = a.phase[vox];
#pragma unroll
          for (int c = 0; c < NC; ++c) ev[v][c] = a.eps[(long long)c * g.N + vox];
        }
      }
#pragma unroll
      for (int v = 0; v < VB; ++v) {
      const int idx = ib + v * blockDim.x;
      if (idx >= nl * L1) break;
      const int gl = fdiv(idx, fL), x = idx - gl * L1;
      fwd_x_voxel<T, DIM, DUAL>(a, ev[v], phv[v], accf, tile + gl * BS + prow(x, 1) * CP);
      }
    }
#pragma unroll
    for (int c = 0; c < 2 * NC; ++c) {
      T x = accf[c];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) wacc[warp][c] += (double)x;
    }
    __syncthreads();
    {  // the next batch's eps and phase ids, while this batch is transformed
      const long long ln = l0 + (long long)gridDim.x * G;
      if (ln < nlines) prefetch_voxels<T>(a.eps, a.phase, g.N, NC, ln * L1, (int)min((long long)G, nlines - ln) * L1);
    }
    tile_fft_ct<CP, NP, true>(tile, nl, BS, pl[0], tws, false);
    fwd_x_untangle<T, DIM, DUAL>(a, tile, nl, l0, BS, fH);
    __syncthreads();
  }
  __syncthreads();
  if (threadIdx.x < 2 * NC) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wacc[w][threadIdx.x];
    a.part_mean[(size_t)blockIdx.x * 2 * NC + threadIdx.x] = t;
  }
}

// Whether the forward x1 pass may stage its batches by bulk copies (x1_vb == 0):
// FP32, every component row of a batch and its phase ids 16-byte aligned and a
// multiple of 16 bytes long (n1 a multiple of 16, aligned field starts).
template <typename T>
__host__ __device__ inline bool fwd_x_staged_ok(const IterArgs<T>& a) {
  return sizeof(T) == 4 && a.g.n1 % 16 == 0 && ((size_t)a.eps & 15) == 0 && ((size_t)a.phase & 15) == 0 &&
         (a.nsmp <= 1 || ((a.st_field * (long long)sizeof(T)) % 16 == 0 && a.st_phase % 16 == 0));
}

// The forward x1 pass with each batch's eps and phase ids moved into shared memory by bulk copies
// (one copy per component row of the batch, completion counted in bytes on an mbarrier).  The copies
// of the next batch start as soon as this batch has been read out of the staging area, so they run
// under its transform and untangling; the voxels, their order per thread and the arithmetic are
// those of the register-loading variant, so the transformed fields are the same bit for bit (the
// FP32 partial sums of <sigma> and <eps> agree to rounding: the compiler may contract them into
// fused multiply-adds differently).  A copy that has not completed after kBulkWaitRounds waits
// stops the solve (ctl->fault).
template <int DIM, bool DUAL>
__device__ __forceinline__ void k_fwd_x_staged_body(const IterArgs<float>& a, const AxisPlan* pl) {
  typedef float T;
  typedef float2 T2;
  constexpr int NC = Comp<DIM>::NC;
  constexpr int VB = 2;
  if (a.ctrl->state != kRunning) return;
  const Geom g = a.g;
  const int L1 = g.n1, H = g.H;
  T2* tile;
  const T2* tws = load_twiddles(a.tw[0], L1, kTwX1, &tile);
  constexpr int nout = DUAL ? 2 * NC : NC;
  constexpr int NP = (nout + 1) / 2;
  constexpr int CP = odd_stride(NP);
  const int BS = padded_rows(L1) * CP;
  const long long nlines = (long long)g.n2 * g.n3;
  const int G = a.x1_lines;
  const long long step = (long long)gridDim.x * G;
  __shared__ double wacc[8][2 * NC];
  __shared__ __align__(8) unsigned long long bar_word;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < 8 * 2 * NC; i += blockDim.x) (&wacc[0][0])[i] = 0.0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const size_t so = fwd_x_stage_offset((size_t)((const unsigned char*)(tile + G * BS) - smem_raw));
  const T* raw = reinterpret_cast<const T*>(smem_raw + so);
  const uint8_t* rph = smem_raw + so + (size_t)NC * G * L1 * sizeof(T);
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&bar_word);
  const uint32_t sraw = (uint32_t)__cvta_generic_to_shared(raw);
  const uint32_t sph = (uint32_t)__cvta_generic_to_shared(rph);
  const int cstride = G * L1;  // floats between the staged component rows
  auto issue = [&](long long l) {
    const int n = (int)min((long long)G, nlines - l) * L1;
    const uint32_t eb = (uint32_t)n * (uint32_t)sizeof(T);
    mbar_arrive_expect_tx(bar, NC * eb + (uint32_t)n);
#pragma unroll
    for (int c = 0; c < NC; ++c)
      bulk_load(sraw + (uint32_t)(c * cstride * sizeof(T)), a.eps + (long long)c * g.N + l * L1, eb, bar);
    bulk_load(sph, a.phase + l * L1, (uint32_t)n, bar);
  };
  long long l0 = (long long)blockIdx.x * G;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    if (l0 < nlines) issue(l0);
  }
  __syncthreads();

  const FastDiv fL = make_fastdiv(L1), fH = make_fastdiv(H);
  for (uint32_t parity = 0; l0 < nlines; l0 += step, parity ^= 1u) {
    const int nl = (int)min((long long)G, nlines - l0);
    bool done = false;
    for (long long k = 0; k < kBulkWaitRounds && !done; ++k) done = mbar_try_wait(bar, parity);
    if (__syncthreads_or(!done)) {
      if (threadIdx.x == 0) {
        a.ctrl->fault = 1;
        a.ctrl->state = kStopped;
      }
      // the block's own copies: one more bounded wait before it gives up its shared memory
      for (long long k = 0; k < kBulkWaitRounds && !done; ++k) done = mbar_try_wait(bar, parity);
      return;
    }
    T accf[2 * NC];
#pragma unroll
    for (int c = 0; c < 2 * NC; ++c) accf[c] = (T)0;
    for (int ib = threadIdx.x; ib < nl * L1; ib += VB * blockDim.x) {
      T ev[VB][NC];
      int phv[VB];
#pragma unroll
      for (int v = 0; v < VB; ++v) {
        const int idx = ib + v * blockDim.x;
        if (idx < nl * L1) {
          phv[v] = rph[idx];
#pragma unroll
          for (int c = 0; c < NC; ++c) ev[v][c] = raw[c * cstride + idx];
        }
      }
#pragma unroll
      for (int v = 0; v < VB; ++v) {
        const int idx = ib + v * blockDim.x;
        if (idx >= nl * L1) break;
        const int gl = fdiv(idx, fL), x = idx - gl * L1;
        fwd_x_voxel<T, DIM, DUAL>(a, ev[v], phv[v], accf, tile + gl * BS + prow(x, 1) * CP);
      }
    }
#pragma unroll
    for (int c = 0; c < 2 * NC; ++c) {
      T x = accf[c];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) wacc[warp][c] += (double)x;
    }
    __syncthreads();  // the staging area is read out: the next batch's copies may overwrite it
    if (threadIdx.x == 0 && l0 + step < nlines) {
      fence_async_shared();
      issue(l0 + step);
    }
    tile_fft_ct<CP, NP, true>(tile, nl, BS, pl[0], tws, false);
    fwd_x_untangle<T, DIM, DUAL>(a, tile, nl, l0, BS, fH);
    __syncthreads();
  }
  __syncthreads();
  if (threadIdx.x < 2 * NC) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wacc[w][threadIdx.x];
    a.part_mean[(size_t)blockIdx.x * 2 * NC + threadIdx.x] = t;
  }
}

// GRP: a grouped launch (fftls_solve_batched), every block working on its sample's view
// Register budgets: the FP32 four-voxel loads (taken with eight-line batches, two blocks per SM by
// shared memory) ask for one block per SM, which lets the compiler use 108 registers (its default
// choice, 80, ran 0.7 % slower at 512^3); every other variant keeps the compiler's default (0).
template <typename T, int DIM, bool DUAL, int VB, bool GRP>
__global__ void __launch_bounds__(256, (VB == 4 && sizeof(T) == 4) ? 1 : 0) k_fwd_x(const __grid_constant__ IterArgs<T> a_) {
  if constexpr (GRP) {
    IterArgs<T> a = a_;
    at_sample(a, blockIdx.y);
    k_fwd_x_body<T, DIM, DUAL, VB>(a, a_.pl);
  } else {
    k_fwd_x_body<T, DIM, DUAL, VB>(a_, a_.pl);
  }
}

// The staged variant (x1_vb == 0, FP32) as a kernel of its own: held to 64 registers (four blocks
// per SM), while the register-loading kernels keep the compiler's own allocation.
template <int DIM, bool DUAL, bool GRP>
__global__ void __launch_bounds__(256, 4) k_fwd_x_staged(const __grid_constant__ IterArgs<float> a_) {
  if constexpr (GRP) {
    IterArgs<float> a = a_;
    at_sample(a, blockIdx.y);
    k_fwd_x_staged_body<DIM, DUAL>(a, a_.pl);
  } else {
    k_fwd_x_staged_body<DIM, DUAL>(a_, a_.pl);
  }
}

// ---------------------------------------------------------------------------
// E (3D, G^C / G^W / G^R): the equilibrium norm from the real-space divergence
// ---------------------------------------------------------------------------
// For the finite-difference operators the divergence k*(q).sigma_hat(q) is the
// transform of a stencil applied to sigma on the grid (eq. mul1, wil071 and the
// rotated stencil of eq. disc3dsig, each scaled to match its k), so by Parseval
// sum_q |k*.sigma_hat|^2 = N sum_x |div sigma(x)|^2 (eq. criterion) and only tau
// has to go through the FFT.  A block owns a tile of kEX x1-columns by kEY
// x2-rows and marches over e_planes x3-planes: per plane it evaluates sigma on
// the tile and its halo into shared memory (double-buffered, one barrier per
// plane), then each thread forms the in-plane part U and the x3 part V of the
// divergence of its voxels and combines them with a per-voxel ring carried in
// registers from plane to plane:
//   W: div(z) = U(z) + V(z) - V(z-1)                  (backward differences)
//   R: div(z) = U(z) + V(z) + [U - V](z-1)             (backward differences averaged
//                                                       over the other two axes)
//   C: div(z-1) = U(z-1) + (V(z) - V(z-2)) / 2         (centred differences)
constexpr int kEX = kEtaTileX, kEY = kEtaTileY, kEThreads = 256;
constexpr int kERows = kEThreads / kEX;     // thread rows; each thread owns kEY / kERows voxels
constexpr int kEOwn = kEY / kERows;

template <typename T>
__device__ __forceinline__ void sigma_of(const T* __restrict__ eps, const uint8_t* __restrict__ phase,
                                         const T* __restrict__ coef, long long N, long long v, T* s) {
  const T* cf = coef + (int)phase[v] * kCoef;
  T e[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) e[c] = eps[(long long)c * N + v];
  const T tr = e[0] + e[1] + e[2];
#pragma unroll
  for (int c = 0; c < 6; ++c) s[c] = cf[1] * e[c] + (c < 3 ? cf[0] * tr : (T)0);
}

// Periodic index for i within a few periods of [0, n) (loops instead of a division).
__device__ __forceinline__ int wrap_index(int i, int n) {
  while (i < 0) i += n;
  while (i >= n) i -= n;
  return i;
}

template <typename T, bool CEN>
__device__ __forceinline__ void k_eta_stencil_body(const IterArgs<T>& a, const AxisPlan* pl) {
  if (a.ctrl->state != kRunning) return;
  const Geom g = a.g;
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3;
  const long long N = g.N;
  const int ntx = (n1 + kEX - 1) / kEX, nty = (n2 + kEY - 1) / kEY;
  const int bx = blockIdx.x % ntx, rest = blockIdx.x / ntx;
  const int by = rest % nty, bz = rest / nty;
  const int x0 = bx * kEX, y0 = by * kEY;
  const int z0 = bz * a.e_planes, z1 = min(n3, z0 + a.e_planes);
  // shared tile of sigma: [2 buffers][6][SY][SX]; tile voxel (xl, yl) at (yl + 1, xl + 1)
  constexpr int SX = kEX + 2, SY = kEY + 2;
  constexpr int HC = CEN ? SX : SX - 1, HR = CEN ? SY : SY - 1;  // filled halo: both sides (C) or -1 only
  constexpr int PL = SY * SX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sS = reinterpret_cast<T*>(smem_raw);
  const T* __restrict__ eps = a.eps;
  const uint8_t* __restrict__ phase = a.phase;
  const T* __restrict__ coef = a.coef;
  const int tx = threadIdx.x % kEX, ty = threadIdx.x / kEX;
  const int IDX[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
  // smem x offsets of the halo columns: column i of the tile is x0 - 1 + i (wrapped)
  T rg[kEOwn][CEN ? 9 : 3];
#pragma unroll
  for (int k = 0; k < kEOwn; ++k)
#pragma unroll
    for (int i = 0; i < (CEN ? 9 : 3); ++i) rg[k][i] = (T)0;
  double acce = 0.0;
  const int zstart = z0 - (CEN ? 2 : 1);
  const int zend = CEN ? z1 : z1 - 1;
  // a thread's (at most kEFill) halo-tile elements: their place in the shared tile and in an x3-plane,
  // the same for every plane of the march
  constexpr int kEFill = (HR * HC + kEThreads - 1) / kEThreads;
  int soff[kEFill], goff[kEFill];
#pragma unroll
  for (int u = 0; u < kEFill; ++u) {
    const int e = threadIdx.x + u * kEThreads;
    soff[u] = -1;
    goff[u] = 0;
    if (e < HR * HC) {
      const int r = e / HC, ci = e - r * HC;
      soff[u] = r * SX + ci;
      goff[u] = wrap_index(y0 - 1 + r, n2) * n1 + wrap_index(x0 - 1 + ci, n1);
    }
  }
  for (int zz = zstart; zz <= zend; ++zz) {
    const int z = wrap_index(zz, n3);
    T* S = sS + ((zz - zstart) & 1) * 6 * PL;
    const T* __restrict__ ez = eps + (long long)z * n2 * n1;
    const uint8_t* __restrict__ pz = phase + (long long)z * n2 * n1;
    // sigma on the tile and its halo; all of a thread's loads are issued before any is used
    T ev[kEFill][6];
    int pv[kEFill];
#pragma unroll
    for (int u = 0; u < kEFill; ++u) {
      if (soff[u] >= 0) {
        pv[u] = pz[goff[u]];
#pragma unroll
        for (int c = 0; c < 6; ++c) ev[u][c] = ez[(long long)c * N + goff[u]];
      }
    }
#pragma unroll
    for (int u = 0; u < kEFill; ++u) {
      if (soff[u] >= 0) {
        const T* cf = coef + pv[u] * kCoef;
        const T tr = ev[u][0] + ev[u][1] + ev[u][2];
#pragma unroll
        for (int c = 0; c < 6; ++c) S[c * PL + soff[u]] = cf[1] * ev[u][c] + (c < 3 ? cf[0] * tr : (T)0);
      }
    }
    __syncthreads();
    const bool valid = CEN ? (zz - 1 >= z0) : (zz >= z0);
    const int zdiv = CEN ? wrap_index(zz - 1, n3) : z;
    T se = (T)0;
#pragma unroll
    for (int k = 0; k < kEOwn; ++k) {
      const int yl = ty + k * kERows;
      const int x = x0 + tx, y = y0 + yl;
      const T* P = S + (yl + 1) * SX + (tx + 1);  // this voxel's sigma, component stride PL
      T d[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int c0 = IDX[0][j], c1 = IDX[1][j], c2 = IDX[2][j];
        if (CEN) {
          const T U = (T)0.5 * (P[c0 * PL + 1] - P[c0 * PL - 1]) + (T)0.5 * (P[c1 * PL + SX] - P[c1 * PL - SX]);
          const T V = P[c2 * PL];
          // ring: [j] U(z-1), [3 + j] V(z-1), [6 + j] V(z-2)
          d[j] = rg[k][j] + (T)0.5 * (V - rg[k][6 + j]);
          rg[k][6 + j] = rg[k][3 + j];
          rg[k][3 + j] = V;
          rg[k][j] = U;
        } else if (a.green == kWillot) {
          const T U = (P[c0 * PL] - P[c0 * PL - 1]) + (P[c1 * PL] - P[c1 * PL - SX]);
          const T V = P[c2 * PL];
          d[j] = U + V - rg[k][j];
          rg[k][j] = V;
        } else {
          const T s00 = P[c0 * PL], s0m = P[c0 * PL - 1], s0y = P[c0 * PL - SX], s0my = P[c0 * PL - SX - 1];
          const T s10 = P[c1 * PL], s1m = P[c1 * PL - 1], s1y = P[c1 * PL - SX], s1my = P[c1 * PL - SX - 1];
          const T U = (T)0.25 * ((s00 - s0m) + (s0y - s0my) + (s10 - s1y) + (s1m - s1my));
          const T V = (T)0.25 * (P[c2 * PL] + P[c2 * PL - 1] + P[c2 * PL - SX] + P[c2 * PL - SX - 1]);
          d[j] = U + V + rg[k][j];
          rg[k][j] = U - V;
        }
      }
      if (valid && x < n1 && y < n2) {
        const long long vdiv = ((long long)zdiv * n2 + y) * n1 + x;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          if (a.write_d64) reinterpret_cast<float*>(a.d64)[(long long)j * N + vdiv] = (float)d[j];
          if (a.corr) d[j] += (T)reinterpret_cast<const float*>(a.d64)[(long long)j * N + vdiv];
          se += d[j] * d[j];
        }
      }
    }
    acce += (double)se;
  }
  double e1[1] = {acce * (double)N};
  block_sum<1>(e1);
  if (threadIdx.x == 0) a.part_eta[blockIdx.x] = e1[0];
}

// GRP: a grouped launch (fftls_solve_batched), every block working on its sample's view
template <typename T, bool CEN, bool GRP>
__global__ void __launch_bounds__(kEThreads) k_eta_stencil(const __grid_constant__ IterArgs<T> a_) {
  if constexpr (GRP) {
    IterArgs<T> a = a_;
    at_sample(a, blockIdx.y);
    k_eta_stencil_body<T, CEN>(a, a_.pl);
  } else {
    k_eta_stencil_body<T, CEN>(a_, a_.pl);
  }
}

// ---------------------------------------------------------------------------
// K2: transform along x2, in place; tiles of y_w modes x n2 rows x n_c
// ---------------------------------------------------------------------------
// W: modes per tile (a compile-time tile geometry; the last tile along x1 may
// hold fewer modes, its other columns are transformed but never stored).
// Blocks of strided_threads(W) threads (a compile-time count for the stages).

template <typename T, int NC, int W>
__device__ __forceinline__ void k_mid_y_body(const IterArgs<T>& a, const AxisPlan* pl, int inv, int kind) {
  typedef typename Cplx<T>::type T2;
  constexpr int NT = strided_threads(W);
  const int st = a.ctrl->state;
  if (inv ? (st != kRunning && st != kLast) : (st != kRunning)) return;
  const Geom g = a.g;
  const int n2 = g.n2;
  T2* tile;
  const T2* tws = load_twiddles(a.tw[1], n2, kTwStrided, &tile);
  const int x0 = blockIdx.x * W;
  const int nx = min(W, g.H - x0);
  constexpr int C = W * NC;
  const int cols = nx * NC;
  T2* spec = kind ? a.specB : a.specA;
  const long long base = ((long long)blockIdx.y * n2 * g.H + x0) * NC;
  const long long rstride = (long long)g.H * NC;
  if (!tile_load<C, false>(tile, spec + base, rstride, n2, cols, a.ctrl)) return;
  if (inv) tile_fft_strided<C, NT, true, false>(tile, pl[1], tws);
  else tile_fft_strided<C, NT, false, true>(tile, pl[1], tws);
  tile_store<C, false>(tile, spec + base, rstride, n2, cols);
}

// GRP: a grouped launch (fftls_solve_batched), every block working on its sample's view
template <typename T, int NC, int W, bool GRP>
__global__ void __launch_bounds__(strided_threads(W)) k_mid_y(const __grid_constant__ IterArgs<T> a_, int inv) {
  if constexpr (GRP) {
    const int kinds = gridDim.z / a_.nsmp;
    IterArgs<T> a = a_;
    at_sample(a, blockIdx.z / kinds);
    k_mid_y_body<T, NC, W>(a, a_.pl, inv, (int)(blockIdx.z % kinds));
  } else {
    k_mid_y_body<T, NC, W>(a_, a_.pl, inv, (int)blockIdx.z);
  }
}

// ---------------------------------------------------------------------------
// K3: transform along x3 + Fourier-space work + inverse along x3
// ---------------------------------------------------------------------------
// Per mode with x_hat the tensor held by this block:
//   * eta: w_q |k* . x_hat|^2 (x_hat = sigma_hat), w_q = 2 for x1 modes with a
//     conjugate partner outside the half spectrum, else 1 (eq. criterion);
//   * e_hat = -G'(k) : x_hat / N at q != 0, with
//       MS/C/R (k = phase * i * kr, kr real): the continuum operator eq. green0b at
//       direction kr (the phase cancels),
//       W: the displacement form with a 2x2 solve in span{k, conj(k)},
//       MS with some q_i = pi (even L): G = C0^{-1} (eq. hfreq),
//       k = 0 at q != 0 (C, R): 0 (eq. mulfix, mysymgr, 3D rule);
//   * q = 0: e_hat = eps_bar (tau form: N eps_bar / N) or 0 (sigma form, corrections).
// The divergence is accumulated in a phase-free form: V = x_hat . kr for MS/C/R
// and b = conj(k) . x_hat for W; d64 holds that vector for the FP64 iterate.
template <typename T, int DIM>
__device__ __forceinline__ void fourier_mode(const IterArgs<T>& a, int x, int y, int z, long long mfreq,
                                             typename Cplx<T>::type* X, bool do_green, bool do_eta,
                                             T& eta_acc) {
  typedef typename Cplx<T>::type T2;
  typedef Comp<DIM> CM;
  constexpr int NC = CM::NC;
  const KTab<T> kt[3] = {a.kt[0][x], a.kt[1][y], a.kt[2][z]};
  const bool q0 = (x == 0 && y == 0 && z == 0);
  const T wq = (x == 0 || 2 * x == a.g.n1) ? (T)1 : (T)2;
  const T invN = (T)(1.0 / (double)a.g.N);
  const T mu0 = (T)a.mu0, lam0 = (T)a.lam0;
  T2 M[DIM][DIM];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    M[CM::I(c)][CM::J(c)] = X[c];
    M[CM::J(c)][CM::I(c)] = X[c];
  }
  T2 E[NC];
  if (a.green != kWillot) {
    T kr[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      if (a.green == kMS) kr[i] = kt[i].q;
      else if (a.green == kCentered) kr[i] = kt[i].sn;
      else {
        T v = (T)2 * kt[i].sh;
#pragma unroll
        for (int m = 0; m < DIM; ++m)
          if (m != i) v *= kt[m].ch;
        kr[i] = v;
      }
    }
    T2 V[DIM];
    T K2 = (T)0;
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      T2 s;
      s.x = (T)0; s.y = (T)0;
#pragma unroll
      for (int i = 0; i < DIM; ++i) { s.x += M[i][j].x * kr[i]; s.y += M[i][j].y * kr[i]; }
      V[j] = s;
      K2 += kr[j] * kr[j];
    }
    if (do_eta) {
      if (a.write_d64) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          float2 f;
          f.x = j < DIM ? (float)V[j].x : 0.f;
          f.y = j < DIM ? (float)V[j].y : 0.f;
          a.d64[mfreq * 3 + j] = f;
        }
      }
      T s = (T)0;
      if (a.corr) {
        // estimate for a correction phase: the stored FP64 divergence plus this one
        // (the conjugate-partner term of operator G below is left out here)
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
          const float2 f = a.d64[mfreq * 3 + j];
          const T vx = V[j].x + (T)f.x, vy = V[j].y + (T)f.y;
          s += vx * vx + vy * vy;
        }
        eta_acc += wq * s;
      } else {
#pragma unroll
        for (int j = 0; j < DIM; ++j) s += V[j].x * V[j].x + V[j].y * V[j].y;
        // operator G uses q_i = +pi at an even-L Nyquist index on both sides of the
        // spectrum, so the conjugate partner (-q) of a half-spectrum mode has k with
        // the Nyquist components of x2, x3 not negated: add its term explicitly.
        bool flip = false;
        if (a.green == kMS && wq == (T)2) {
#pragma unroll
          for (int i = 1; i < DIM; ++i) flip = flip || (kt[i].nyq != (T)0);
        }
        if (flip) {
          T sp = (T)0;
#pragma unroll
          for (int j = 0; j < DIM; ++j) {
            T2 u;
            u.x = (T)0; u.y = (T)0;
#pragma unroll
            for (int i = 0; i < DIM; ++i) {
              const T kk = (i > 0 && kt[i].nyq != (T)0) ? -kr[i] : kr[i];
              u.x += M[i][j].x * kk;
              u.y += M[i][j].y * kk;
            }
            sp += u.x * u.x + u.y * u.y;
          }
          eta_acc += s + sp;
        } else {
          eta_acc += wq * s;
        }
      }
    }
    if (!do_green) return;
    bool nyq = false;
    if (a.green == kMS) {
#pragma unroll
      for (int i = 0; i < DIM; ++i) nyq = nyq || (kt[i].nyq != (T)0);
    }
    if (q0) {
#pragma unroll
      for (int c = 0; c < NC; ++c) { E[c].x = (a.tauform && !a.corr) ? (T)a.eps_bar[c] : (T)0; E[c].y = (T)0; }
    } else if (nyq) {
      // -C0^{-1}:x / N,  C0^{-1} = I/(2 mu0) - lam0 / (2 mu0 (d lam0 + 2 mu0)) dd
      T2 tr;
      tr.x = (T)0; tr.y = (T)0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) { tr.x += X[c].x; tr.y += X[c].y; }
      const T a1 = (T)(0.5 / a.mu0);
      const T a2 = (T)(a.lam0 / (2.0 * a.mu0 * (DIM * a.lam0 + 2.0 * a.mu0)));
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const bool diag = c < DIM;
        E[c].x = -invN * (a1 * X[c].x - (diag ? a2 * tr.x : (T)0));
        E[c].y = -invN * (a1 * X[c].y - (diag ? a2 * tr.y : (T)0));
      }
    } else if (K2 == (T)0) {
#pragma unroll
      for (int c = 0; c < NC; ++c) { E[c].x = (T)0; E[c].y = (T)0; }
    } else {
      const T c0 = (lam0 + mu0) / (lam0 + (T)2 * mu0);
      T2 S;
      S.x = (T)0; S.y = (T)0;
#pragma unroll
      for (int j = 0; j < DIM; ++j) { S.x += kr[j] * V[j].x; S.y += kr[j] * V[j].y; }
      const T f = -invN / (mu0 * K2);
      const T h = c0 / K2;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int i = CM::I(c), j = CM::J(c);
        E[c].x = f * ((T)0.5 * (kr[i] * V[j].x + kr[j] * V[i].x) - h * kr[i] * kr[j] * S.x);
        E[c].y = f * ((T)0.5 * (kr[i] * V[j].y + kr[j] * V[i].y) - h * kr[i] * kr[j] * S.y);
      }
    }
  } else {
    // Willot-Pellegrini k_i = e^{i q_i} - 1 (complex)
    T2 k[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) { k[i].x = kt[i].cm1; k[i].y = kt[i].sn; }
    T2 b[DIM];  // b_j = sum_i conj(k_i) x_ij
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      T2 s;
      s.x = (T)0; s.y = (T)0;
#pragma unroll
      for (int i = 0; i < DIM; ++i) s = cadd(s, cmul(cconj(k[i]), M[i][j]));
      b[j] = s;
    }
    if (do_eta) {
      if (a.write_d64) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          float2 f;
          f.x = j < DIM ? (float)b[j].x : 0.f;
          f.y = j < DIM ? (float)b[j].y : 0.f;
          a.d64[mfreq * 3 + j] = f;
        }
      }
      T s = (T)0;
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        T bx = b[j].x, by = b[j].y;
        if (a.corr) {
          const float2 f = a.d64[mfreq * 3 + j];
          bx += (T)f.x;
          by += (T)f.y;
        }
        s += bx * bx + by * by;
      }
      eta_acc += wq * s;
    }
    if (!do_green) return;
    if (q0) {
#pragma unroll
      for (int c = 0; c < NC; ++c) { E[c].x = (a.tauform && !a.corr) ? (T)a.eps_bar[c] : (T)0; E[c].y = (T)0; }
    } else {
      T K = (T)0;
      T2 gk, p, r;
      gk.x = gk.y = p.x = p.y = r.x = r.y = (T)0;
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        K += k[i].x * k[i].x + k[i].y * k[i].y;
        gk = cadd(gk, cmul(k[i], k[i]));
        p = cadd(p, cmul(k[i], b[i]));
        r = cadd(r, cmul(cconj(k[i]), b[i]));
      }
      // (lam0 + mu0) K alpha + mu0 g beta = p ;  lam0 conj(g) alpha + 2 mu0 K beta = r
      const T det = (T)2 * mu0 * (lam0 + mu0) * K * K - lam0 * mu0 * (gk.x * gk.x + gk.y * gk.y);
      const T idet = (T)1 / det;
      T2 al = csub(cscale(p, (T)2 * mu0 * K), cscale(cmul(gk, r), mu0));
      T2 be = csub(cscale(r, (lam0 + mu0) * K), cscale(cmul(cconj(gk), p), lam0));
      al = cscale(al, idet);
      be = cscale(be, idet);
      const T iu = (T)1 / (mu0 * K);
      T2 u[DIM];
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        T2 t = csub(b[j], cscale(cmul(cconj(k[j]), al), lam0));
        t = csub(t, cscale(cmul(k[j], be), mu0));
        u[j] = cscale(t, iu);
      }
      const T f = (T)-0.5 * invN;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int i = CM::I(c), j = CM::J(c);
        E[c] = cscale(cadd(cmul(k[i], u[j]), cmul(k[j], u[i])), f);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) X[c] = E[c];
}

// Reciprocal of a positive scalar: correctly rounded in float (__frcp_rn), a
// plain division in double.
__device__ __forceinline__ float recip_pos(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip_pos(double x) { return 1.0 / x; }

// e_hat = -G'(k) : tau_hat / N at one mode of the real-direction operators
// G^C / G^R (3D), k = phase * i * kr with kr real (the phase cancels, eq. green0b
// at direction kr): with V_j = tau_ij kr_i, S = kr . V, K2 = |kr|^2,
// U_i = V_i - kr_i c0 S / K2 and f = -1 / (N mu0 K2),
//   e_ij = f (kr_i U_j + kr_j U_i) / 2,      c0 = (lambda0 + mu0) / (lambda0 + 2 mu0),
// and 0 where K2 = 0 (the modes of eq. mulfix and of the rule G^R = 0 where two
// q_i = pi; q = 0 is set by the caller).
template <typename T, typename T2>
__device__ __forceinline__ void green_rd_mode(T2 (&X)[6], T k0, T k1, T k2, T cf, T c0) {
  const T K2 = k0 * k0 + k1 * k1 + k2 * k2;
  const T iK2 = K2 > (T)0 ? recip_pos(K2) : (T)0;
  T2 V[3];
  V[0].x = X[0].x * k0 + X[5].x * k1 + X[4].x * k2;
  V[0].y = X[0].y * k0 + X[5].y * k1 + X[4].y * k2;
  V[1].x = X[5].x * k0 + X[1].x * k1 + X[3].x * k2;
  V[1].y = X[5].y * k0 + X[1].y * k1 + X[3].y * k2;
  V[2].x = X[4].x * k0 + X[3].x * k1 + X[2].x * k2;
  V[2].y = X[4].y * k0 + X[3].y * k1 + X[2].y * k2;
  const T hs = c0 * iK2;
  const T Sx = (k0 * V[0].x + k1 * V[1].x + k2 * V[2].x) * hs;
  const T Sy = (k0 * V[0].y + k1 * V[1].y + k2 * V[2].y) * hs;
  const T kr[3] = {k0, k1, k2};
  T2 U[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    U[i].x = V[i].x - kr[i] * Sx;
    U[i].y = V[i].y - kr[i] * Sy;
  }
  const T f = cf * iK2;
  const T fk[3] = {f * k0, f * k1, f * k2};
  const T h = (T)0.5;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    X[i].x = fk[i] * U[i].x;
    X[i].y = fk[i] * U[i].y;
  }
  X[3].x = h * (fk[1] * U[2].x + fk[2] * U[1].x);
  X[3].y = h * (fk[1] * U[2].y + fk[2] * U[1].y);
  X[4].x = h * (fk[0] * U[2].x + fk[2] * U[0].x);
  X[4].y = h * (fk[0] * U[2].y + fk[2] * U[0].y);
  X[5].x = h * (fk[0] * U[1].x + fk[1] * U[0].x);
  X[5].y = h * (fk[0] * U[1].y + fk[1] * U[0].y);
}

// Six complex values of one mode between registers and the tile (16-byte accesses;
// a mode starts on a 48-byte (float) or 96-byte (double) boundary).
__device__ __forceinline__ void load_mode6(const float2* p, float2 (&X)[6]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float4 t = q[i];
    X[2 * i] = make_float2(t.x, t.y);
    X[2 * i + 1] = make_float2(t.z, t.w);
  }
}
__device__ __forceinline__ void store_mode6(float2* p, const float2 (&X)[6]) {
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int i = 0; i < 3; ++i) q[i] = make_float4(X[2 * i].x, X[2 * i].y, X[2 * i + 1].x, X[2 * i + 1].y);
}
__device__ __forceinline__ void load_mode6(const double2* p, double2 (&X)[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) X[i] = p[i];
}
__device__ __forceinline__ void store_mode6(double2* p, const double2 (&X)[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) p[i] = X[i];
}

// FAST: 3D G^C / G^R with eta from the real-space stencil (only tau is
// transformed, no eta here): the modes take green_rd_mode with the per-axis
// factors of rd (by storage position), kr_1 = a_1 b_2 b_3, kr_2 = b_1 a_2 b_3,
// kr_3 = b_1 b_2 a_3.  Otherwise the general fourier_mode.
template <typename T, int DIM, int W, bool FAST>
__device__ __forceinline__ void k_fourier_z_body(const IterArgs<T>& a, const AxisPlan* pl, int kind) {
  typedef typename Cplx<T>::type T2;
  constexpr int NC = Comp<DIM>::NC;
  constexpr int NT = strided_threads(W);
  if (a.ctrl->state != kRunning) return;
  const Geom g = a.g;
  const int n3 = g.n3;
  T2* tile;
  const T2* tws = load_twiddles(a.tw[2], n3, kTwStrided, &tile);
  const int x0 = blockIdx.x * W;
  const int py = blockIdx.y;
  const bool do_green = kind == 0;
  const bool do_eta = !a.eta_real && (a.dual ? (kind == 1) : true);
  const int nx = min(W, g.H - x0);
  constexpr int C = W * NC;
  const int cols = nx * NC;
  T2* spec = kind ? a.specB : a.specA;
  const long long base = ((long long)py * g.H + x0) * NC;
  const long long zstride = (long long)g.n2 * g.H * NC;
  if (!tile_load<C, true>(tile, spec + base, zstride, n3, cols, a.ctrl)) return;
  tile_fft_strided<C, NT, false, false>(tile, pl[2], tws);
  T eta_acc = (T)0;
  if constexpr (FAST) {
    static_assert(DIM == 3 && NT % W == 0, "fast Fourier pass: 3D, whole modes per thread");
    const int xc = (int)threadIdx.x % W;
    if (xc < nx) {
      const T2 rx = a.rd[0][x0 + xc], ry = a.rd[1][py];
      const T cf = (T)(-1.0 / ((double)g.N * a.mu0));
      const T c0 = (T)((a.lam0 + a.mu0) / (a.lam0 + 2.0 * a.mu0));
      const T bxy = rx.y * ry.y, axy = rx.x * ry.y, bxay = rx.y * ry.x;
      const bool line0 = (x0 + xc == 0) && (py == 0);
      for (int pz = (int)threadIdx.x / W; pz < n3; pz += NT / W) {
        const T2 rz = __ldg(&a.rd[2][pz]);
        T2* mp = tile + pz * C + xc * NC;
        T2 X[6];
        load_mode6(mp, X);
        green_rd_mode<T>(X, axy * rz.y, bxay * rz.y, bxy * rz.x, cf, c0);
        if (line0 && pz == 0) {
#pragma unroll
          for (int c = 0; c < 6; ++c) { X[c].x = a.corr ? (T)0 : (T)a.eps_bar[c]; X[c].y = (T)0; }
        }
        store_mode6(mp, X);
      }
    }
  } else {
    FastDiv fnx = {0u, 0u, 1};  // full tiles (nx == W) divide by the compile-time width
    if (nx != W) fnx = make_fastdiv(nx);
    const int ym = __ldg(&a.perm[1][py]);
    for (int idx = threadIdx.x; idx < n3 * nx; idx += blockDim.x) {
      const int pz = nx == W ? (int)((unsigned)idx / W) : fdiv(idx, fnx), xc = idx - pz * nx;
      const int zm = __ldg(&a.perm[2][pz]);
      T2* mp = tile + pz * C + xc * NC;
      T2 X[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) X[c] = mp[c];
      // the FP64 divergence kept for correction phases is indexed by frequency, not by
      // storage position
      const long long mfreq = ((long long)zm * g.n2 + ym) * g.H + x0 + xc;
      fourier_mode<T, DIM>(a, x0 + xc, ym, zm, mfreq, X, do_green, do_eta, eta_acc);
      if (do_green)
#pragma unroll
        for (int c = 0; c < NC; ++c) mp[c] = X[c];
    }
  }
  __syncthreads();
  if (do_green) {
    tile_fft_strided<C, NT, true, false>(tile, pl[2], tws);
    tile_store<C, true>(tile, spec + base, zstride, n3, cols);
  }
  if (!a.eta_real) {  // with the real-space eta the x1 pass owns part_eta
    double e1[1] = {(double)eta_acc};
    block_sum<1>(e1);
    if (threadIdx.x == 0)
      a.part_eta[((size_t)kind * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = e1[0];
  }
}

// GRP: a grouped launch (fftls_solve_batched), every block working on its sample's view
template <typename T, int DIM, int W, bool FAST, bool GRP>
__global__ void __launch_bounds__(strided_threads(W)) k_fourier_z(const __grid_constant__ IterArgs<T> a_) {
  if constexpr (GRP) {
    const int kinds = gridDim.z / a_.nsmp;
    IterArgs<T> a = a_;
    at_sample(a, blockIdx.z / kinds);
    k_fourier_z_body<T, DIM, W, FAST>(a, a_.pl, (int)(blockIdx.z % kinds));
  } else {
    k_fourier_z_body<T, DIM, W, FAST>(a_, a_.pl, (int)blockIdx.z);
  }
}

// ---------------------------------------------------------------------------
// R: eta, <sigma>, history and stop decision (single block)
// ---------------------------------------------------------------------------
// Block sums of W values per thread for the kRedThreads threads of k_reduce_eta, returned to every
// thread: the values go through shared memory column by column, and warp w sums the columns w,
// w + 8, ... (8 FP64 additions per lane and a 5-level shuffle per column), so the block issues about
// 13 W warp-wide FP64 additions instead of the 5 W per warp of a shuffle tree in every warp (GB300's
// FP64 pipe takes about 16 cycles for one).
constexpr int kRedThreads = 256;
template <int W>
__device__ void block_sum_columns(double (&v)[W]) {
  __shared__ double col[W][kRedThreads];
  __shared__ double out[W];
#pragma unroll
  for (int i = 0; i < W; ++i) col[i][threadIdx.x] = v[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < W; i += kRedThreads / 32) {
    double x = 0.0;
#pragma unroll
    for (int k = 0; k < kRedThreads / 32; ++k) x += col[i][lane + 32 * k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) out[i] = x;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < W; ++i) v[i] = out[i];
}

template <typename T, int DIM>
__device__ __forceinline__ void k_reduce_eta_body(const IterArgs<T>& a, const AxisPlan* pl, int n_eta_parts, int n_mean_parts) {
  constexpr int NC = Comp<DIM>::NC;
  Ctrl* ctl = a.ctrl;
  const int st = ctl->state;
  if (st != kRunning || ctl->it >= ctl->max_it) {
    if (threadIdx.x == 0 && (st == kLast || st == kRunning)) ctl->state = kStopped;
    return;
  }
  double s[2 * NC + 1];
#pragma unroll
  for (int c = 0; c < 2 * NC + 1; ++c) s[c] = 0.0;
  for (int b = threadIdx.x; b < n_mean_parts; b += blockDim.x)
#pragma unroll
    for (int c = 0; c < 2 * NC; ++c) s[c] += a.part_mean[(size_t)b * 2 * NC + c];
  for (int b = threadIdx.x; b < n_eta_parts; b += blockDim.x) s[2 * NC] += a.part_eta[b];
  block_sum_columns<2 * NC + 1>(s);
  if (threadIdx.x != 0) return;
  const double N = (double)a.g.N, invN = 1.0 / N;
  double fro2 = 0.0, eb2 = 0.0, d2 = 0.0;
  const int it = ctl->it;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const double ms = ctl->off_sig[c] + s[c] * invN, me = ctl->off_eps[c] + s[NC + c] * invN;
    const double wgt = c < DIM ? 1.0 : 2.0;
    fro2 += wgt * ms * ms;
    eb2 += wgt * a.eps_bar[c] * a.eps_bar[c];
    d2 += wgt * (me - a.eps_bar[c]) * (me - a.eps_bar[c]);
    a.ms_hist[(size_t)it * NC + c] = ms;
    ctl->last_ms[c] = ms;
    ctl->last_me[c] = me;
  }
  const double num = sqrt(fmax(s[2 * NC], 0.0));
  const double den = N * sqrt(fro2);
  double eta;
  if (num == 0.0) eta = 0.0;
  else if (den == 0.0) eta = INFINITY;
  else eta = num / den;
  const double merr = eb2 > 0.0 ? sqrt(d2 / eb2) : sqrt(d2);
  a.eta_hist[it] = eta;
  ctl->it = it + 1;
  ctl->phase_it += 1;
  ctl->last_eta = eta;
  ctl->last_mean_err = merr;
  if (it == 0) { ctl->eta0 = eta; ctl->best = eta; }
  int ns = kRunning;
  if (!isfinite(eta) || (ctl->eta0 > 0.0 && eta > 1e4 * ctl->eta0)) {
    ns = kDiverged;
  } else if (ctl->stop_rule == 0 && eta <= ctl->tol && (!ctl->mean_guard || merr <= ctl->tol)) {
    ns = ctl->switch_mode ? kSwitch : kConverged;
  } else {
    if (ctl->stall_window > 0) {
      if (eta < 0.9 * ctl->best) { ctl->best = eta; ctl->stall = 0; }
      else if (++ctl->stall >= (ctl->best < 1e-3 ? ctl->stall_window : 8 * ctl->stall_window)) ns = kSwitch;
    }
    if (ns == kRunning && ctl->phase_max > 0 && ctl->phase_it >= ctl->phase_max) ns = kSwitch;
    if (ns == kRunning && it + 1 >= ctl->max_it) ns = kLast;
  }
  ctl->state = ns;
}

// GRP: a grouped launch (fftls_solve_batched), every block working on its sample's view
template <typename T, int DIM, bool GRP>
__global__ void k_reduce_eta(const __grid_constant__ IterArgs<T> a_, int n_eta_parts, int n_mean_parts) {
  if constexpr (GRP) {
    IterArgs<T> a = a_;
    at_sample(a, blockIdx.y);
    k_reduce_eta_body<T, DIM>(a, a_.pl, n_eta_parts, n_mean_parts);
  } else {
    k_reduce_eta_body<T, DIM>(a_, a_.pl, n_eta_parts, n_mean_parts);
  }
}

// ---------------------------------------------------------------------------
// K5: inverse x1 transform (half complex -> real) + scheme update
// ---------------------------------------------------------------------------
// STAGED (FP32): the batch's eps and phase ids move into shared memory by bulk copies issued before
// its packing and transform, so the update reads them from shared memory instead of waiting on L2
// (completion counted on an mbarrier; a copy lost after kBulkWaitRounds waits stops the solve with
// ctl->fault).  The arithmetic per voxel is the same: the fields are the same bit for bit.
template <typename T, int DIM, bool STAGED>
__device__ __forceinline__ void k_inv_x_body(const IterArgs<T>& a, const AxisPlan* pl) {
  typedef typename Cplx<T>::type T2;
  constexpr int NC = Comp<DIM>::NC;
  constexpr int NPI = (NC + 1) / 2;
  constexpr int CP = odd_stride(NPI);
  const int st = a.ctrl->state;
  if (st != kRunning && st != kLast) return;
  const Geom g = a.g;
  const int L1 = g.n1, H = g.H;
  T2* tile;
  const T2* tws = load_twiddles(a.tw[0], L1, kTwX1, &tile);
  const int BS = padded_rows(L1) * CP;
  const int* __restrict__ pos = a.pos[0];
  const long long nlines = (long long)g.n2 * g.n3;
  const int G = a.x5_lines;
  double dmax[2] = {0.0, 0.0};
  const FastDiv fL = make_fastdiv(L1), fH = make_fastdiv(H);
  // staging area after the tile: NC rows of G n1 values, then G n1 phase ids
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bar_word;
  const size_t so = fwd_x_stage_offset((size_t)((const unsigned char*)(tile + G * BS) - smem_raw));
  const T* raw = reinterpret_cast<const T*>(smem_raw + so);
  const uint8_t* rph = smem_raw + so + (size_t)NC * G * L1 * sizeof(T);
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&bar_word);
  const bool stage = STAGED && a.update != kUpdDirectTau;  // the tau form does not read eps
  if (STAGED) {
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
  }
  uint32_t parity = 0;
  for (long long l0 = (long long)blockIdx.x * G; l0 < nlines; l0 += (long long)gridDim.x * G) {
    const int nl = (int)min((long long)G, nlines - l0);
    if (stage) {
      if (threadIdx.x == 0) {  // the previous batch's update has read the staging area (barrier at loop end)
        fence_async_shared();
        const int n = nl * L1;
        const uint32_t eb = (uint32_t)n * (uint32_t)sizeof(T);
        const uint32_t sraw = (uint32_t)__cvta_generic_to_shared(raw);
        mbar_arrive_expect_tx(bar, NC * eb + (uint32_t)n);
#pragma unroll
        for (int c = 0; c < NC; ++c)
          bulk_load(sraw + (uint32_t)(c * G * L1 * sizeof(T)), a.eps + (long long)c * g.N + l0 * L1, eb, bar);
        bulk_load((uint32_t)__cvta_generic_to_shared(rph), a.phase + l0 * L1, (uint32_t)n, bar);
      }
    } else if (a.update != kUpdDirectTau) {
      // eps and the phase ids are read after the transform: bring them towards L2 now
      prefetch_voxels<T>(a.eps, a.phase, g.N, NC, l0 * L1, nl * L1);
    }
    // pack pairs of components into complex lines: one thread per mode k, every component of it
    for (int idx = threadIdx.x; idx < nl * H; idx += blockDim.x) {
      const int gl = fdiv(idx, fH), k = idx - gl * H;
      const long long m = (l0 + gl) * (long long)H + k;
      const bool edge = k == 0 || 2 * k == L1;
      const bool mirror = k > 0 && L1 - k >= H;
      T2* r0 = tile + gl * BS + prow(__ldg(&pos[k]), 1) * CP;
      T2* r1 = tile + gl * BS + prow(__ldg(&pos[mirror ? L1 - k : k]), 1) * CP;
#pragma unroll
      for (int p = 0; p < NPI; ++p) {
        T2 A, B;
        if (NC % 2 == 0) {
          load_pair(a.specA + m * NC + 2 * p, A, B);   // 16-byte aligned in FP32
        } else {
          A = a.specA[m * NC + 2 * p];
          if (2 * p + 1 < NC) B = a.specA[m * NC + 2 * p + 1];
          else { B.x = (T)0; B.y = (T)0; }
        }
        if (edge) { A.y = (T)0; B.y = (T)0; }
        T2 z;
        z.x = A.x - B.y;
        z.y = A.y + B.x;
        r0[p] = z;
        if (mirror) {
          T2 zm;
          zm.x = A.x + B.y;
          zm.y = B.x - A.y;
          r1[p] = zm;
        }
      }
    }
    __syncthreads();
    {  // the next batch's half spectrum (its lines are consecutive, so one contiguous run)
      const long long ln = l0 + (long long)gridDim.x * G;
      if (ln < nlines) {
        const int nn = (int)min((long long)G, nlines - ln);
        const T2* base = a.specA + ln * (long long)H * NC;
        const int bytes = nn * H * NC * (int)sizeof(T2);
        for (int off = threadIdx.x * 128; off < bytes; off += blockDim.x * 128)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char*>(base) + off));
      }
    }
    tile_fft_ct<CP, NPI, true>(tile, nl, BS, pl[0], tws, true);
    if (stage) {
      bool done = false;
      for (long long k = 0; k < kBulkWaitRounds && !done; ++k) done = mbar_try_wait(bar, parity);
      if (__syncthreads_or(!done)) {
        if (threadIdx.x == 0) {
          a.ctrl->fault = 1;
          a.ctrl->state = kStopped;
        }
        // the block's own copies: one more bounded wait before it gives up its shared memory
        for (long long k = 0; k < kBulkWaitRounds && !done; ++k) done = mbar_try_wait(bar, parity);
        return;
      }
      parity ^= 1u;
    }
    for (int idx = threadIdx.x; idx < nl * L1; idx += blockDim.x) {
      const int gl = fdiv(idx, fL), x = idx - gl * L1;
      const long long vox = (l0 + gl) * (long long)L1 + x;
      T e[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T2 v = tile[gl * BS + prow(x, 1) * CP + c / 2];
        e[c] = (c & 1) ? v.y : v.x;
      }
      T o[NC], n[NC];
      int ph;
      if (stage) {
#pragma unroll
        for (int c = 0; c < NC; ++c) o[c] = raw[c * G * L1 + idx];
        ph = rph[idx];
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) o[c] = a.eps[(long long)c * g.N + vox];
        ph = a.phase[vox];
      }
      const T* cf = a.coef + ph * kCoef;
      const int upd = a.update;
      if (upd == kUpdDirectTau) {
#pragma unroll
        for (int c = 0; c < NC; ++c) n[c] = e[c];
      } else if (upd == kUpdDirectSig) {
#pragma unroll
        for (int c = 0; c < NC; ++c) n[c] = o[c] + e[c];
      } else if (upd == kUpdResidual) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          a.rfield[(long long)c * g.N + vox] = (float)(e[c] - o[c]);
          n[c] = o[c];
        }
      } else if (upd == kUpdCorrDirect) {
#pragma unroll
        for (int c = 0; c < NC; ++c) n[c] = (T)a.rfield[(long long)c * g.N + vox] + e[c];
      } else {
        T d[NC];
        T trd = (T)0;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          d[c] = e[c] - o[c];
          if (upd == kUpdCorrAccel) d[c] += (T)a.rfield[(long long)c * g.N + vox];
          if (c < DIM) trd += d[c];
        }
        const T am = cf[4], av = cf[5];
#pragma unroll
        for (int c = 0; c < NC; ++c) n[c] = o[c] + am * d[c] + (c < DIM ? av * trd : (T)0);
      }
      if (upd != kUpdResidual) {
#pragma unroll
        for (int c = 0; c < NC; ++c) a.eps[(long long)c * g.N + vox] = n[c];
      }
      if (a.want_delta) {
        T dn[NC];
        T trn = (T)0;
#pragma unroll
        for (int c = 0; c < NC; ++c) { dn[c] = n[c] - o[c]; if (c < DIM) trn += dn[c]; }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const T ds = cf[1] * dn[c] + (c < DIM ? cf[0] * trn : (T)0);
          dmax[0] = fmax(dmax[0], (double)fabs(dn[c]));
          dmax[1] = fmax(dmax[1], (double)fabs(ds));
        }
      }
    }
    __syncthreads();
  }
  if (a.want_delta) {
    block_max<2>(dmax);
    if (threadIdx.x == 0) {
      a.part_delta[(size_t)blockIdx.x * 2] = dmax[0];
      a.part_delta[(size_t)blockIdx.x * 2 + 1] = dmax[1];
    }
  }
}

// GRP: a grouped launch (fftls_solve_batched), every block working on its sample's view
template <typename T, int DIM, bool GRP, bool STAGED>
__global__ void __launch_bounds__(256) k_inv_x(const __grid_constant__ IterArgs<T> a_) {
  if constexpr (GRP) {
    IterArgs<T> a = a_;
    at_sample(a, blockIdx.y);
    k_inv_x_body<T, DIM, STAGED>(a, a_.pl);
  } else {
    k_inv_x_body<T, DIM, STAGED>(a_, a_.pl);
  }
}

template <typename T>
__device__ __forceinline__ void k_reduce_delta_body(const IterArgs<T>& a, const AxisPlan* pl) {
  Ctrl* ctl = a.ctrl;
  const int st = ctl->state;
  if (st != kRunning && st != kLast) return;
  double m[2] = {0.0, 0.0};
  for (int b = threadIdx.x; b < a.x5_blocks; b += blockDim.x) {
    m[0] = fmax(m[0], a.part_delta[(size_t)b * 2]);
    m[1] = fmax(m[1], a.part_delta[(size_t)b * 2 + 1]);
  }
  block_max<2>(m);
  if (threadIdx.x == 0) {
    const double dl = fmax(m[0], m[1]);
    ctl->last_delta = dl;
    if (ctl->stop_rule == 1 && dl < ctl->tol) ctl->state = kConverged;
  }
}

// GRP: a grouped launch (fftls_solve_batched), every block working on its sample's view
template <typename T, bool GRP>
__global__ void k_reduce_delta(const __grid_constant__ IterArgs<T> a_) {
  if constexpr (GRP) {
    IterArgs<T> a = a_;
    at_sample(a, blockIdx.y);
    k_reduce_delta_body<T>(a, a_.pl);
  } else {
    k_reduce_delta_body<T>(a_, a_.pl);
  }
}

// ---------------------------------------------------------------------------
// elementwise helpers
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_fill_eps(T* eps, int nc, long long N, double e0, double e1, double e2, double e3, double e4,
                           double e5) {
  const double ev[6] = {e0, e1, e2, e3, e4, e5};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    for (int c = 0; c < nc; ++c) eps[(long long)c * N + i] = (T)ev[c];
}

template <typename TO, typename TI>
__global__ void k_convert(TO* out, const TI* in, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (TO)in[i];
}

#ifdef FFTLS_KERNELS_MAIN
__global__ void k_add_correction(double* out, const float* in, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] += (double)in[i];
}
#endif

template <typename T, int DIM>
__global__ void k_stress(const T* eps, const uint8_t* phase, const T* coef, long long N, double* stress,
                         double* part) {
  constexpr int NC = Comp<DIM>::NC;
  double acc[2 * NC];
#pragma unroll
  for (int c = 0; c < 2 * NC; ++c) acc[c] = 0.0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x) {
    const T* cf = coef + (int)phase[v] * kCoef;
    double e[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) e[c] = (double)eps[(long long)c * N + v];
    double tr = e[0] + e[1] + (DIM == 3 ? e[2] : 0.0);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double s = (double)cf[1] * e[c] + (c < DIM ? (double)cf[0] * tr : 0.0);
      if (stress) stress[(long long)c * N + v] = s;
      acc[c] += s;
      acc[NC + c] += e[c];
    }
  }
  block_sum<2 * NC>(acc);
  if (threadIdx.x == 0)
#pragma unroll
    for (int c = 0; c < 2 * NC; ++c) part[(size_t)blockIdx.x * 2 * NC + c] = acc[c];
}

#ifdef FFTLS_KERNELS_MAIN
__global__ void k_phase_max(const uint8_t* phase, long long N, unsigned int* out) {
  unsigned int m = 0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x)
    m = max(m, (unsigned int)phase[v]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}
#endif

#ifdef FFTLS_KERNELS_MAIN
__global__ void k_sum_parts(const double* part, int blocks, int width, double* out) {
  // one thread per output value, fixed order: deterministic
  const int c = threadIdx.x;
  if (c >= width) return;
  double s = 0.0;
  for (int b = 0; b < blocks; ++b) s += part[(size_t)b * width + c];
  out[c] = s;
}
#endif

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// Each launcher comes in two variants: GRP = false, a single solve (sample 0 of a
// group of one, the kernels read their parameters directly), and GRP = true, a
// grouped launch over a.nsmp samples of one 3D geometry (fftls_solve_batched): the
// 1D grids take the sample as blockIdx.y, the strided grids fold it into blockIdx.z.
// The public launchers pick the variant from a.nsmp; the grouped instantiations
// live in their own translation units (fftls_kernels_{x,y,z}{32,64}g.cu).
template <typename T, bool GRP>
cudaError_t launch_fwd_x_t(const IterArgs<T>& a, cudaStream_t s) {
  const dim3 grid(a.x1_blocks, GRP ? a.nsmp : 1);
#define FFTLS_FWD(D, U, V) k_fwd_x<T, D, U, V, GRP><<<grid, a.x_threads, a.x1_smem, s>>>(a)
#define FFTLS_FWD_ST(D, U) k_fwd_x_staged<D, U, GRP><<<grid, a.x_threads, a.x1_smem, s>>>(a)
// FP64 forward passes (the few certification passes of the ladder) load one voxel at a time
#define FFTLS_FWD_VB(D, U)                                                                              \
  if constexpr (sizeof(T) == 8) FFTLS_FWD(D, U, 1);                                                     \
  else if (a.x1_vb == 0 && fwd_x_staged_ok(a)) FFTLS_FWD_ST(D, U);                                      \
  else if (a.x1_vb >= 4 || a.x1_vb == 0) FFTLS_FWD(D, U, 4);                                            \
  else if (a.x1_vb == 2) FFTLS_FWD(D, U, 2);                                                            \
  else FFTLS_FWD(D, U, 1)
  if (a.dim == 3) {
    if (a.dual) { FFTLS_FWD_VB(3, true); }
    else { FFTLS_FWD_VB(3, false); }
  } else if constexpr (!GRP) {
    if (a.dual) { FFTLS_FWD_VB(2, true); }
    else { FFTLS_FWD_VB(2, false); }
  } else {
    return cudaErrorInvalidValue;
  }
#undef FFTLS_FWD_VB
#undef FFTLS_FWD_ST
#undef FFTLS_FWD
  return cudaGetLastError();
}

template <typename T, bool GRP>
cudaError_t launch_eta_stencil_t(const IterArgs<T>& a, cudaStream_t s) {
  const dim3 grid(a.e_blocks, GRP ? a.nsmp : 1);
  if (a.green == kCentered) k_eta_stencil<T, true, GRP><<<grid, kEThreads, a.e_smem, s>>>(a);
  else k_eta_stencil<T, false, GRP><<<grid, kEThreads, a.e_smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, bool GRP>
cudaError_t launch_mid_y_t(const IterArgs<T>& a, bool inv, cudaStream_t s) {
  if (a.g.n2 == 1) return cudaSuccess;
  dim3 grid((a.g.H + a.y_w - 1) / a.y_w, a.g.n3, ((!inv && a.dual && !a.eta_real) ? 2 : 1) * (GRP ? a.nsmp : 1));
#define FFTLS_MIDY(NCV, WV) k_mid_y<T, NCV, WV, GRP><<<grid, strided_threads(WV), a.y_smem, s>>>(a, inv ? 1 : 0)
#define FFTLS_MIDY_W(NCV)                                                                               \
  switch (a.y_w) {                                                                                      \
    case 1: FFTLS_MIDY(NCV, 1); break;                                                                  \
    case 2: FFTLS_MIDY(NCV, 2); break;                                                                  \
    case 4: FFTLS_MIDY(NCV, 4); break;                                                                  \
    case 8: FFTLS_MIDY(NCV, 8); break;                                                                  \
    case 16: FFTLS_MIDY(NCV, 16); break;                                                                \
    default: return cudaErrorInvalidValue;                                                              \
  }
  if (a.dim == 3) { FFTLS_MIDY_W(6) }
  else if constexpr (!GRP) { FFTLS_MIDY_W(3) }
  else return cudaErrorInvalidValue;
#undef FFTLS_MIDY_W
#undef FFTLS_MIDY
  return cudaGetLastError();
}

// The fast Fourier pass serves 3D G^C / G^R when eta comes from the real-space stencil.
template <typename T>
bool fourier_fast(const IterArgs<T>& a) {
  return a.dim == 3 && a.eta_real && (a.green == kCentered || a.green == kRotated);
}

template <typename T, bool GRP>
cudaError_t launch_fourier_z_t(const IterArgs<T>& a, cudaStream_t s) {
  dim3 grid((a.g.H + a.z_w - 1) / a.z_w, a.g.n2, ((a.dual && !a.eta_real) ? 2 : 1) * (GRP ? a.nsmp : 1));
#define FFTLS_FZ(D, WV, F) k_fourier_z<T, D, WV, F, GRP><<<grid, strided_threads(WV), a.z_smem, s>>>(a)
#define FFTLS_FZ_W(D, F)                                                                                \
  switch (a.z_w) {                                                                                      \
    case 1: FFTLS_FZ(D, 1, F); break;                                                                   \
    case 2: FFTLS_FZ(D, 2, F); break;                                                                   \
    case 4: FFTLS_FZ(D, 4, F); break;                                                                   \
    case 8: FFTLS_FZ(D, 8, F); break;                                                                   \
    case 16: FFTLS_FZ(D, 16, F); break;                                                                 \
    default: return cudaErrorInvalidValue;                                                              \
  }
  if (a.dim == 3) {
    if (fourier_fast(a)) { FFTLS_FZ_W(3, true) }
    else { FFTLS_FZ_W(3, false) }
  } else if constexpr (!GRP) {
    FFTLS_FZ_W(2, false)
  } else {
    return cudaErrorInvalidValue;
  }
#undef FFTLS_FZ_W
#undef FFTLS_FZ
  return cudaGetLastError();
}

template <typename T, bool GRP>
cudaError_t launch_reduce_eta_t(const IterArgs<T>& a, cudaStream_t s) {
  const int nparts = a.eta_real ? a.e_blocks : ((a.g.H + a.z_w - 1) / a.z_w) * a.g.n2 * (a.dual ? 2 : 1);
  const int mparts = a.x1_blocks;
  const dim3 grid(1, GRP ? a.nsmp : 1);
  if (a.dim == 3) k_reduce_eta<T, 3, GRP><<<grid, kRedThreads, 0, s>>>(a, nparts, mparts);
  else if constexpr (!GRP) k_reduce_eta<T, 2, GRP><<<grid, kRedThreads, 0, s>>>(a, nparts, mparts);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <typename T, bool GRP>
cudaError_t launch_inv_x_t(const IterArgs<T>& a, cudaStream_t s) {
  const dim3 grid(a.x5_blocks, GRP ? a.nsmp : 1);
  // the staged variant (x5_vb == 0, FP32) where the batch's rows are 16-byte aligned, else register loads
  const bool staged = sizeof(T) == 4 && a.x5_vb == 0 && fwd_x_staged_ok(a);
  if (a.dim == 3) {
    if (staged) k_inv_x<T, 3, GRP, sizeof(T) == 4><<<grid, a.x_threads, a.x5_smem, s>>>(a);
    else k_inv_x<T, 3, GRP, false><<<grid, a.x_threads, a.x5_smem, s>>>(a);
  } else if constexpr (!GRP) {
    if (staged) k_inv_x<T, 2, GRP, sizeof(T) == 4><<<grid, a.x_threads, a.x5_smem, s>>>(a);
    else k_inv_x<T, 2, GRP, false><<<grid, a.x_threads, a.x5_smem, s>>>(a);
  }
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <typename T, bool GRP>
cudaError_t launch_reduce_delta_t(const IterArgs<T>& a, cudaStream_t s) {
  k_reduce_delta<T, GRP><<<dim3(1, GRP ? a.nsmp : 1), 512, 0, s>>>(a);
  return cudaGetLastError();
}

#define FFTLS_PICK(fn, ...) (a.nsmp > 1 ? fn##_grp<T>(__VA_ARGS__) : fn##_t<T, false>(__VA_ARGS__))
template <typename T> cudaError_t launch_fwd_x(const IterArgs<T>& a, cudaStream_t s) { return FFTLS_PICK(launch_fwd_x, a, s); }
template <typename T> cudaError_t launch_eta_stencil(const IterArgs<T>& a, cudaStream_t s) { return FFTLS_PICK(launch_eta_stencil, a, s); }
template <typename T> cudaError_t launch_mid_y(const IterArgs<T>& a, bool inv, cudaStream_t s) { return FFTLS_PICK(launch_mid_y, a, inv, s); }
template <typename T> cudaError_t launch_fourier_z(const IterArgs<T>& a, cudaStream_t s) { return FFTLS_PICK(launch_fourier_z, a, s); }
template <typename T> cudaError_t launch_reduce_eta(const IterArgs<T>& a, cudaStream_t s) { return FFTLS_PICK(launch_reduce_eta, a, s); }
template <typename T> cudaError_t launch_inv_x(const IterArgs<T>& a, cudaStream_t s) { return FFTLS_PICK(launch_inv_x, a, s); }
template <typename T> cudaError_t launch_reduce_delta(const IterArgs<T>& a, cudaStream_t s) { return FFTLS_PICK(launch_reduce_delta, a, s); }
#undef FFTLS_PICK

// Every kernel of the iteration may take up to smax bytes of dynamic shared
// memory (any tile schedule the host picks stays below it).  One function per
// translation unit, each touching only the kernels that unit instantiates.
#define FFTLS_ATTR(fn)                                                                                          \
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);

template <typename T, bool GRP>
cudaError_t set_attrs_y_t(size_t smax) {
  cudaError_t e = cudaSuccess;
  FFTLS_ATTR((k_mid_y<T, 6, 1, GRP>));
  FFTLS_ATTR((k_mid_y<T, 6, 2, GRP>));
  FFTLS_ATTR((k_mid_y<T, 6, 4, GRP>));
  FFTLS_ATTR((k_mid_y<T, 6, 8, GRP>));
  FFTLS_ATTR((k_mid_y<T, 6, 16, GRP>));
  if constexpr (!GRP) {
    FFTLS_ATTR((k_mid_y<T, 3, 1, GRP>));
    FFTLS_ATTR((k_mid_y<T, 3, 2, GRP>));
    FFTLS_ATTR((k_mid_y<T, 3, 4, GRP>));
    FFTLS_ATTR((k_mid_y<T, 3, 8, GRP>));
    FFTLS_ATTR((k_mid_y<T, 3, 16, GRP>));
  }
  return e;
}

template <typename T, bool GRP>
cudaError_t set_attrs_z_t(size_t smax) {
  cudaError_t e = cudaSuccess;
  FFTLS_ATTR((k_fourier_z<T, 3, 1, false, GRP>));
  FFTLS_ATTR((k_fourier_z<T, 3, 2, false, GRP>));
  FFTLS_ATTR((k_fourier_z<T, 3, 4, false, GRP>));
  FFTLS_ATTR((k_fourier_z<T, 3, 8, false, GRP>));
  FFTLS_ATTR((k_fourier_z<T, 3, 16, false, GRP>));
  FFTLS_ATTR((k_fourier_z<T, 3, 1, true, GRP>));
  FFTLS_ATTR((k_fourier_z<T, 3, 2, true, GRP>));
  FFTLS_ATTR((k_fourier_z<T, 3, 4, true, GRP>));
  FFTLS_ATTR((k_fourier_z<T, 3, 8, true, GRP>));
  FFTLS_ATTR((k_fourier_z<T, 3, 16, true, GRP>));
  if constexpr (!GRP) {
    FFTLS_ATTR((k_fourier_z<T, 2, 1, false, GRP>));
    FFTLS_ATTR((k_fourier_z<T, 2, 2, false, GRP>));
    FFTLS_ATTR((k_fourier_z<T, 2, 4, false, GRP>));
    FFTLS_ATTR((k_fourier_z<T, 2, 8, false, GRP>));
    FFTLS_ATTR((k_fourier_z<T, 2, 16, false, GRP>));
  }
  return e;
}

template <typename T, bool GRP>
cudaError_t set_attrs_x_t(size_t smax) {
  cudaError_t e = cudaSuccess;
  FFTLS_ATTR((k_eta_stencil<T, true, GRP>));
  FFTLS_ATTR((k_eta_stencil<T, false, GRP>));
  FFTLS_ATTR((k_fwd_x<T, 3, true, 1, GRP>));
  FFTLS_ATTR((k_fwd_x<T, 3, false, 1, GRP>));
  if constexpr (!GRP) {
    FFTLS_ATTR((k_fwd_x<T, 2, true, 1, GRP>));
    FFTLS_ATTR((k_fwd_x<T, 2, false, 1, GRP>));
  }
  if constexpr (sizeof(T) == 4) {
    FFTLS_ATTR((k_fwd_x_staged<3, true, GRP>));
    FFTLS_ATTR((k_fwd_x_staged<3, false, GRP>));
    if constexpr (!GRP) {
      FFTLS_ATTR((k_fwd_x_staged<2, true, GRP>));
      FFTLS_ATTR((k_fwd_x_staged<2, false, GRP>));
    }
    FFTLS_ATTR((k_fwd_x<T, 3, true, 2, GRP>));
    FFTLS_ATTR((k_fwd_x<T, 3, true, 4, GRP>));
    FFTLS_ATTR((k_fwd_x<T, 3, false, 2, GRP>));
    FFTLS_ATTR((k_fwd_x<T, 3, false, 4, GRP>));
    if constexpr (!GRP) {
      FFTLS_ATTR((k_fwd_x<T, 2, true, 2, GRP>));
      FFTLS_ATTR((k_fwd_x<T, 2, true, 4, GRP>));
      FFTLS_ATTR((k_fwd_x<T, 2, false, 2, GRP>));
      FFTLS_ATTR((k_fwd_x<T, 2, false, 4, GRP>));
    }
  }
  FFTLS_ATTR((k_inv_x<T, 3, GRP, false>));
  if constexpr (!GRP) FFTLS_ATTR((k_inv_x<T, 2, GRP, false>));
  if constexpr (sizeof(T) == 4) {
    FFTLS_ATTR((k_inv_x<T, 3, GRP, true>));
    if constexpr (!GRP) FFTLS_ATTR((k_inv_x<T, 2, GRP, true>));
  }
  return e;
}
#ifdef FFTLS_GROUPED_TU
template <typename T> cudaError_t launch_fwd_x_grp(const IterArgs<T>& a, cudaStream_t s) { return launch_fwd_x_t<T, true>(a, s); }
template <typename T> cudaError_t launch_eta_stencil_grp(const IterArgs<T>& a, cudaStream_t s) { return launch_eta_stencil_t<T, true>(a, s); }
template <typename T> cudaError_t launch_mid_y_grp(const IterArgs<T>& a, bool inv, cudaStream_t s) { return launch_mid_y_t<T, true>(a, inv, s); }
template <typename T> cudaError_t launch_fourier_z_grp(const IterArgs<T>& a, cudaStream_t s) { return launch_fourier_z_t<T, true>(a, s); }
template <typename T> cudaError_t launch_reduce_eta_grp(const IterArgs<T>& a, cudaStream_t s) { return launch_reduce_eta_t<T, true>(a, s); }
template <typename T> cudaError_t launch_inv_x_grp(const IterArgs<T>& a, cudaStream_t s) { return launch_inv_x_t<T, true>(a, s); }
template <typename T> cudaError_t launch_reduce_delta_grp(const IterArgs<T>& a, cudaStream_t s) { return launch_reduce_delta_t<T, true>(a, s); }
template <typename T> cudaError_t set_attrs_xgrp(size_t smax) { return set_attrs_x_t<T, true>(smax); }
template <typename T> cudaError_t set_attrs_ygrp(size_t smax) { return set_attrs_y_t<T, true>(smax); }
template <typename T> cudaError_t set_attrs_zgrp(size_t smax) { return set_attrs_z_t<T, true>(smax); }
template <typename T>
cudaError_t set_attrs_grp(size_t smax) {
  cudaError_t e = set_attrs_xgrp<T>(smax);
  if (e == cudaSuccess) e = set_attrs_ygrp<T>(smax);
  if (e == cudaSuccess) e = set_attrs_zgrp<T>(smax);
  return e;
}
#endif
template <typename T> cudaError_t set_attrs_y(size_t smax) { return set_attrs_y_t<T, false>(smax); }
template <typename T> cudaError_t set_attrs_z(size_t smax) { return set_attrs_z_t<T, false>(smax); }

template <typename T>
cudaError_t set_kernel_attributes(const IterArgs<T>& a, size_t smax) {
  (void)a;
  cudaError_t e = set_attrs_x_t<T, false>(smax);
  if (e == cudaSuccess) e = set_attrs_y<T>(smax);
  if (e == cudaSuccess) e = set_attrs_z<T>(smax);
  if (e == cudaSuccess) e = set_attrs_grp<T>(smax);
  return e;
}
#undef FFTLS_ATTR

template <typename T>
cudaError_t launch_fill_eps(T* eps, int nc, long long N, const double* e, cudaStream_t s) {
  const int blocks = (int)min((N + 255) / 256, (long long)152 * 16);
  k_fill_eps<T><<<blocks, 256, 0, s>>>(eps, nc, N, e[0], e[1], e[2], e[3], e[4], e[5]);
  return cudaGetLastError();
}

template <typename TO, typename TI>
cudaError_t launch_convert(TO* out, const TI* in, long long n, cudaStream_t s) {
  const int blocks = (int)min((n + 255) / 256, (long long)152 * 16);
  k_convert<TO, TI><<<blocks, 256, 0, s>>>(out, in, n);
  return cudaGetLastError();
}

#ifdef FFTLS_KERNELS_MAIN
cudaError_t launch_add_correction(double* out, const float* in, long long n, cudaStream_t s) {
  const int blocks = (int)min((n + 255) / 256, (long long)152 * 16);
  k_add_correction<<<blocks, 256, 0, s>>>(out, in, n);
  return cudaGetLastError();
}
#endif

template <typename T>
cudaError_t launch_stress(const T* eps, const uint8_t* phase, const T* coef, int dim, long long N, double* stress_out,
                          double* part, int blocks, cudaStream_t s) {
  if (dim == 3) k_stress<T, 3><<<blocks, 256, 0, s>>>(eps, phase, coef, N, stress_out, part);
  else k_stress<T, 2><<<blocks, 256, 0, s>>>(eps, phase, coef, N, stress_out, part);
  return cudaGetLastError();
}

#ifdef FFTLS_KERNELS_MAIN
cudaError_t launch_phase_max(const uint8_t* phase, long long N, unsigned int* out, int blocks, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  k_phase_max<<<blocks, 256, 0, s>>>(phase, N, out);
  return cudaGetLastError();
}
#endif

#ifdef FFTLS_KERNELS_MAIN
cudaError_t launch_sum_parts(const double* part, int blocks, int width, double* out, cudaStream_t s) {
  k_sum_parts<<<1, 32, 0, s>>>(part, blocks, width, out);
  return cudaGetLastError();
}
#endif



}  // namespace fftls
