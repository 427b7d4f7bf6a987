// Host driver and C ABI of the FFT Lippmann-Schwinger solver (see include/fftls.h).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "fftls.h"
#include "fftls_kernels.cuh"

using namespace fftls;

namespace {

constexpr int kMaxL = 2048;
constexpr int kNumKinds = 8;
const char* const kKindNames[2][kNumKinds] = {
    {"fwd_x_f32", "mid_y_fwd_f32", "fourier_z_f32", "reduce_eta_f32", "mid_y_inv_f32", "inv_x_f32",
     "reduce_delta_f32", "eta_x_f32"},
    {"fwd_x_f64", "mid_y_fwd_f64", "fourier_z_f64", "reduce_eta_f64", "mid_y_inv_f64", "inv_x_f64",
     "reduce_delta_f64", "eta_x_f64"}};
constexpr int kMaxOuter = 8;  // FP64 residual evaluations of the refinement ladder
constexpr int kMaxWorkers = 64, kDefaultWorkers = 8;  // concurrent solves of fftls_solve_batched
// grouped launches of fftls_solve_batched: samples per group, and the device memory a
// group may take (about kGroupBytesPerVoxel bytes per voxel of every sample: both
// iterates, both spectra in FP64, the ladder's defect and divergence, the phase ids)
constexpr int kMaxGroup = 256;
constexpr long long kGroupBytes = 24LL << 30, kGroupBytesPerVoxel = 210;

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
    if (e == cudaSuccess) cap = bytes;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  std::vector<unsigned char> key;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    key.clear();
  }
};

bool factor_plan(int L, AxisPlan* p) {
  if (L < 1 || L > kMaxL) return false;
  int n = L, twos = 0, threes = 0, fives = 0;
  while (n % 2 == 0) { n /= 2; ++twos; }
  while (n % 3 == 0) { n /= 3; ++threes; }
  while (n % 5 == 0) { n /= 5; ++fives; }
  if (n != 1) return false;
  std::vector<int> r;
  int n8 = twos / 3, rem = twos % 3;
  if (rem == 1 && n8 > 0) { --n8; r.push_back(4); r.push_back(4); }
  else if (rem == 2) r.push_back(4);
  else if (rem == 1) r.push_back(2);
  for (int i = 0; i < n8; ++i) r.push_back(8);
  for (int i = 0; i < threes; ++i) r.push_back(3);
  for (int i = 0; i < fives; ++i) r.push_back(5);
  if ((int)r.size() > kMaxStages) return false;
  p->L = L;
  p->nst = (int)r.size();
  int M = L;
  for (int i = 0; i < kMaxStages; ++i) {
    p->radix[i] = i < p->nst ? r[i] : 1;
    p->msize[i] = i < p->nst ? M : 1;
    if (i < p->nst) M /= r[i];
  }
  return true;
}

// storage position -> frequency index of the in-place forward transform (fftls_fft.cuh)
void plan_permutation(const AxisPlan& p, int* perm, int* pos) {
  for (int q = 0; q < p.L; ++q) {
    int rem = q, k = 0, mult = 1, span = p.L;
    for (int s = 0; s < p.nst; ++s) {
      span /= p.radix[s];
      const int d = rem / span;
      rem %= span;
      k += d * mult;
      mult *= p.radix[s];
    }
    perm[q] = k;
    pos[k] = q;
  }
}

// Twiddles w^t = e^{-2 pi i t / L} (exact at multiples of pi/2) in the layout
// the tile transforms read (tw_count(L, layout) complex values: the plain table
// w^t by t, or rows per stage for the compile-time lengths, kTwX1 for the x1
// tiles and kTwStrided, with padded rows, for the x2 / x3 tiles), the
// wave-vector table {q, sin q, cos q - 1, sin q/2, cos q/2, nyquist} by frequency
// index, and the real-direction factors {a, b} of operator `green` by storage
// position p (frequency perm[p]; perm = NULL: natural order): kr_i = a_i prod_{m != i} b_m, with
// G^R: a = 2 sin(q/2), b = cos(q/2);  G^C: a = sin q, b = 1;  G: a = q, b = 1.
void axis_tables(int L, int layout, int green, const int* perm, double* tw, double* kt, double* rd) {
  static_assert(fftls::tw_count(512, fftls::kTwStrided) <= kMaxL + 2, "stage twiddle rows fit the plain table's bound");
  double plain[2 * kMaxL];
  for (int t = 0; t < L; ++t) {
    const double ang = -2.0 * M_PI * (double)t / (double)L;
    double cs = cos(ang), sn = sin(ang);
    if ((4 * t) % L == 0) {
      const int qd = (4 * t) / L;
      const double cq[4] = {1, 0, -1, 0}, sq[4] = {0, -1, 0, 1};
      cs = cq[qd % 4];
      sn = sq[qd % 4];
    }
    plain[2 * t] = cs;
    plain[2 * t + 1] = sn;
  }
  const int ntw = fftls::tw_count(L, layout);
  for (int t = 0; t < 2 * ntw; ++t) tw[t] = t < 2 * L ? plain[t] : 0.0;
  if ((layout != fftls::kTwPlain && fftls::ct_length(L)) || (layout == fftls::kTwStrided && fftls::r3_length(L))) {
    for (int t = 0; t < 2 * ntw; ++t) tw[t] = 0.0;
    for (int st = 0; st < fftls::ct_nst(L); ++st) {
      const int R = fftls::ct_radix(L, st), M = fftls::ct_msize(L, st), MR = M / R, T = L / M;
      if (MR == 1) continue;
      const int row = layout == fftls::kTwX1 ? R : fftls::srow(R);
      const size_t off = layout == fftls::kTwX1 ? (size_t)fftls::stage_tw_offset(L, st)
                                                : (size_t)fftls::strided_tw_offset(L, st);
      double* rows = tw + 2 * off;
      for (int j = 0; j < MR; ++j)
        for (int r = 1; r < R; ++r) {
          rows[2 * (j * row + r - 1)] = plain[2 * (r * j * T)];
          rows[2 * (j * row + r - 1) + 1] = plain[2 * (r * j * T) + 1];
        }
    }
  }
  for (int m = 0; m < L; ++m) {
    const int s = m <= L / 2 ? m : m - L;
    const double q = 2.0 * M_PI * s / L;
    double sn = sin(q), sh = sin(0.5 * q), ch = cos(0.5 * q);
    if ((2 * s) % L == 0) sn = 0.0;  // q = 0, pi
    if (s == 0) sh = 0.0;
    if (2 * s == L) ch = 0.0;  // q = pi
    if (4 * s == L) sn = 1.0;
    if (4 * s == -L) sn = -1.0;
    double* e = kt + 6 * (size_t)m;
    e[0] = q;
    e[1] = sn;
    e[2] = -2.0 * sh * sh;  // cos q - 1 without cancellation
    e[3] = sh;
    e[4] = ch;
    e[5] = (L % 2 == 0 && 2 * m == L) ? 1.0 : 0.0;
  }
  for (int p = 0; p < L; ++p) {
    const double* e = kt + 6 * (size_t)(perm ? perm[p] : p);
    double av = 0.0, bv = 1.0;
    if (green == FFTLS_GREEN_R) { av = 2.0 * e[3]; bv = e[4]; }
    else if (green == FFTLS_GREEN_C) av = e[1];
    else if (green == FFTLS_GREEN_MS) av = e[0];
    rd[2 * (size_t)p] = av;
    rd[2 * (size_t)p + 1] = bv;
  }
}

// Tile schedule of one iteration: lines per batch of the forward and inverse x1
// passes, modes per tile of the x2 and x3 passes, x3-planes per block of the
// real-space eta kernel.  Any schedule that fits shared memory gives the same
// arithmetic per line and per mode; only the partial-sum grouping of the
// reductions changes.
struct TilePlan {
  int x1_lines, x5_lines, y_w, z_w, e_planes, x1_vb;
  int x5_vb = 1;  // inverse x1 pass: 1 register loads of eps, 0 staged by bulk copies (FP32)
  int y_thr, z_thr;  // threads per block of the strided passes (0: by tile size)
  int tuned;  // 1: chosen by timing candidates on the device
};

struct PlanKey {
  int prec, n1, n2, n3, dim, green, real_eta;
  bool operator==(const PlanKey& o) const { return memcmp(this, &o, sizeof(PlanKey)) == 0; }
};

}  // namespace

struct fftls_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  size_t smem_optin = 0;
  int num_sms = 0;
  DevBuf phase, eps32, eps64, specA, specB, coef32, coef64, tab32, tab64, perms;
  DevBuf part_mean, part_eta, part_delta, sums, ctrl, eta_hist, ms_hist, scratch, rfield, d64;
  GraphCache graphs[2];
  Ctrl* h_ctrl = nullptr;  // pinned
  double* h_sums = nullptr;
  DevBuf gpar;             // per-sample lambda0, mu0, eps_bar of a grouped solve
  Ctrl* h_gctrl = nullptr;  // pinned control blocks of a grouped solve
  int h_gcap = 0;
  long long launches = 0;  // kernels launched (graph nodes counted one by one)
  long long graph_launches = 0;
  double prof_ms[2][kNumKinds];
  int prof_n[2][kNumKinds];
  std::vector<std::pair<PlanKey, TilePlan>> plans;  // tile schedules per grid and precision
  std::vector<fftls_ctx*> workers;  // child contexts of fftls_solve_batched
  struct ProfEv { cudaEvent_t a, b; int kind; };
  std::vector<ProfEv> ev;
};

namespace {

fftls_status set_err(fftls_ctx* c, fftls_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CUDA_TRY(ctx, ...)                                                                                      \
  do {                                                                                                          \
    cudaError_t e_ = (__VA_ARGS__);                                                                             \
    if (e_ != cudaSuccess)                                                                                      \
      return set_err(ctx, e_ == cudaErrorMemoryAllocation ? FFTLS_E_OOM : FFTLS_E_CUDA, "%s: %s (line %d)",      \
                     #__VA_ARGS__, cudaGetErrorString(e_), __LINE__);                                           \
  } while (0)

int ncomp(int dim) { return dim == 3 ? 6 : 3; }
int odd_up(int n) { return (n & 1) ? n : n + 1; }

bool default_medium(const fftls_problem* p, double* l0, double* m0) {
  const int d = p->dim;
  double kmin = INFINITY, kmax = -INFINITY, mmin = INFINITY, mmax = -INFINITY;
  for (int a = 0; a < p->n_phases; ++a) {
    const double k = p->lambda[a] + 2.0 / d * p->mu[a];
    kmin = std::min(kmin, k);
    kmax = std::max(kmax, k);
    mmin = std::min(mmin, p->mu[a]);
    mmax = std::max(mmax, p->mu[a]);
  }
  double k0, mu0;
  if (p->scheme == FFTLS_ACCELERATED) {
    k0 = sqrt(kmin * kmax);
    mu0 = sqrt(mmin * mmax);
  } else {
    k0 = 0.5 * (kmin + kmax);
    mu0 = 0.5 * (mmin + mmax);
  }
  *l0 = k0 - 2.0 / d * mu0;
  *m0 = mu0;
  return mu0 > 0.0 && k0 > 0.0 && isfinite(k0) && isfinite(mu0);
}

fftls_status validate(fftls_ctx* c, const fftls_problem* p, const fftls_options* o) {
  if (!p || !o) return set_err(c, FFTLS_E_INVALID_ARG, "null problem or options");
  if (p->dim != 2 && p->dim != 3) return set_err(c, FFTLS_E_INVALID_ARG, "dim must be 2 or 3 (got %d)", p->dim);
  for (int i = 0; i < 3; ++i)
    if (p->n[i] < 1) return set_err(c, FFTLS_E_INVALID_ARG, "n[%d] = %d must be >= 1", i, p->n[i]);
  if (p->dim == 2 && p->n[2] != 1) return set_err(c, FFTLS_E_INVALID_ARG, "dim 2 needs n[2] == 1");
  for (int i = 0; i < 3; ++i) {
    AxisPlan ap;
    if (!factor_plan(p->n[i], &ap))
      return set_err(c, FFTLS_E_UNSUPPORTED_SIZE, "n[%d] = %d: lengths must be <= %d with prime factors 2, 3, 5", i,
                     p->n[i], kMaxL);
  }
  if (!p->phase) return set_err(c, FFTLS_E_INVALID_ARG, "phase is null");
  if (p->n_phases < 1 || p->n_phases > 256) return set_err(c, FFTLS_E_INVALID_ARG, "n_phases must be 1..256");
  if (!p->lambda || !p->mu) return set_err(c, FFTLS_E_INVALID_ARG, "lambda / mu are null");
  for (int a = 0; a < p->n_phases; ++a) {
    const double l = p->lambda[a], m = p->mu[a];
    if (!isfinite(l) || !isfinite(m) || m < 0.0 || l + 2.0 / p->dim * m < 0.0)
      return set_err(c, FFTLS_E_INVALID_ARG, "phase %d: need finite mu >= 0 and kappa >= 0", a);
  }
  if (p->green < 0 || p->green > 3) return set_err(c, FFTLS_E_INVALID_ARG, "unknown green %d", p->green);
  if (p->scheme != FFTLS_DIRECT && p->scheme != FFTLS_ACCELERATED)
    return set_err(c, FFTLS_E_INVALID_ARG, "unknown scheme %d", p->scheme);
  for (int i = 0; i < ncomp(p->dim); ++i)
    if (!isfinite(p->eps_bar[i])) return set_err(c, FFTLS_E_INVALID_ARG, "eps_bar[%d] not finite", i);
  const bool l0nan = isnan(p->lambda0), m0nan = isnan(p->mu0);
  if (l0nan != m0nan) return set_err(c, FFTLS_E_INVALID_ARG, "lambda0 and mu0 must both be NaN or both set");
  if (!l0nan) {
    if (!(p->mu0 > 0.0) || !(p->lambda0 + 2.0 / p->dim * p->mu0 > 0.0) || !isfinite(p->lambda0) || !isfinite(p->mu0))
      return set_err(c, FFTLS_E_INVALID_ARG, "reference medium must be positive definite (mu0 > 0, kappa0 > 0)");
  } else {
    double l0, m0;
    if (!default_medium(p, &l0, &m0))
      return set_err(c, FFTLS_E_INVALID_ARG,
                     "default reference medium degenerates (a phase with mu = 0 or kappa = 0): pass lambda0, mu0");
  }
  if (!(o->tol >= 0.0) || !isfinite(o->tol)) return set_err(c, FFTLS_E_INVALID_ARG, "tol must be finite and >= 0");
  if (o->stop != FFTLS_STOP_ETA && o->stop != FFTLS_STOP_MAXDELTA)
    return set_err(c, FFTLS_E_INVALID_ARG, "unknown stop rule %d", o->stop);
  if (o->max_iter < 1) return set_err(c, FFTLS_E_INVALID_ARG, "max_iter must be >= 1");
  if (o->precision < 0 || o->precision > 2) return set_err(c, FFTLS_E_INVALID_ARG, "unknown precision %d", o->precision);
  if (o->precision == FFTLS_FP32_REFINE64 && o->stop != FFTLS_STOP_ETA)
    return set_err(c, FFTLS_E_INVALID_ARG, "FP32_REFINE64 refines on eta: use FFTLS_STOP_ETA");
  return FFTLS_OK;
}

template <typename T> struct Prec;
template <> struct Prec<float> { static constexpr int idx = 0; };
template <> struct Prec<double> { static constexpr int idx = 1; };

struct Setup {
  int dim, nc;
  Geom g;
  AxisPlan pl[3];
  double lam0, mu0;
  double eps_bar[6];
  int green, scheme;
  const uint8_t* d_phase;
  cudaStream_t s;
  bool profile, graphs;
  int smem_optin, num_sms;
};

void setup_geometry(Setup& S, const fftls_problem* p) {
  const int d = p->dim, nc = ncomp(d);
  S.dim = d;
  S.nc = nc;
  S.green = p->green;
  S.scheme = p->scheme;
  S.g.n1 = p->n[0];
  S.g.n2 = p->n[1];
  S.g.n3 = p->n[2];
  S.g.H = p->n[0] / 2 + 1;
  S.g.N = (long long)p->n[0] * p->n[1] * p->n[2];
  S.g.modes = (long long)S.g.n3 * S.g.n2 * S.g.H;
  for (int ax = 0; ax < 3; ++ax) factor_plan(p->n[ax], &S.pl[ax]);
  if (isnan(p->lambda0)) default_medium(p, &S.lam0, &S.mu0);
  else { S.lam0 = p->lambda0; S.mu0 = p->mu0; }
  for (int i = 0; i < 6; ++i) S.eps_bar[i] = i < nc ? p->eps_bar[i] : 0.0;
}

// Phase coefficient table (256 entries: ids >= n_phases read NaN, never out of bounds).
void coef_table(const Setup& S, const fftls_problem* p, double* cf) {
  const int d = S.dim;
  for (int i = 0; i < 256 * kCoef; ++i) cf[i] = NAN;
  const double k0 = S.lam0 + 2.0 / d * S.mu0;
  for (int a = 0; a < p->n_phases; ++a) {
    const double l = p->lambda[a], m = p->mu[a];
    const double k = l + 2.0 / d * m;
    const double ak = k0 / (k + k0), am = S.mu0 / (m + S.mu0);
    double* e = cf + (size_t)a * kCoef;
    e[0] = l;
    e[1] = 2.0 * m;
    e[2] = l - S.lam0;
    e[3] = 2.0 * (m - S.mu0);
    e[4] = 2.0 * am;
    e[5] = 2.0 * (ak - am) / d;
    e[6] = e[7] = 0.0;
  }
}

// Table block per precision: per axis twiddles (tw_count(L, tw_layout(ax))
// complex), the k table (L x 6) and the real-direction factors (L x 2).
int tw_layout(int ax) { return ax == 0 ? fftls::kTwX1 : fftls::kTwStrided; }
size_t axis_table_count(int L, int ax) { return 2 * (size_t)fftls::tw_count(L, tw_layout(ax)) + 8 * (size_t)L; }
size_t table_offset_tw(const Setup& S, int ax) {
  size_t off = 0;
  for (int a = 0; a < ax; ++a) off += axis_table_count(S.pl[a].L, a);
  return off;
}
size_t table_offset_kt(const Setup& S, int ax) {
  return table_offset_tw(S, ax) + 2 * (size_t)fftls::tw_count(S.pl[ax].L, tw_layout(ax));
}
size_t table_offset_rd(const Setup& S, int ax) { return table_offset_kt(S, ax) + 6 * (size_t)S.pl[ax].L; }
size_t table_count(const Setup& S) { return table_offset_tw(S, 3); }

// Fill the table block (tab) and the per-axis permutations (perms: storage position ->
// frequency, then frequency -> position, per axis).  No heap allocation (the
// allocation-free entry point stages its tables through here).
void fill_tables(const Setup& S, double* tab, int* perms) {
  size_t po = 0;
  for (int ax = 0; ax < 3; ++ax) {
    const int L = S.pl[ax].L;
    plan_permutation(S.pl[ax], &perms[po], &perms[po + L]);
    // x1: the half spectrum is stored in natural order (the rd table is by frequency)
    axis_tables(L, tw_layout(ax), S.green, ax == 0 ? nullptr : &perms[po], &tab[table_offset_tw(S, ax)],
                &tab[table_offset_kt(S, ax)], &tab[table_offset_rd(S, ax)]);
    po += 2 * (size_t)L;
  }
}

void build_tables(const Setup& S, std::vector<double>& tab, std::vector<int>& perms) {
  tab.assign(table_count(S), 0.0);
  perms.assign(2 * (size_t)(S.pl[0].L + S.pl[1].L + S.pl[2].L), 0);
  fill_tables(S, tab.data(), perms.data());
}

// Launch shapes for precision T; false if a size does not fit in shared memory.
// real_eta: 3D G^C/W/R take eta from the real-space stencil and the forward x1
// pass carries tau alone (rows half as wide); dual: the forward pass carries tau
// and sigma (no real-space eta, accelerated scheme).
struct PlanGeom {
  size_t cb, lim, twx, line1, line5;
  long long nlines, tiles;
};

PlanGeom plan_geom(const Setup& S, size_t cb, bool real_eta) {
  PlanGeom G;
  const int nc = S.nc;
  G.cb = cb;
  G.lim = (size_t)S.smem_optin - 4096;  // static reduction arrays
  G.twx = (size_t)fftls::tw_count(S.g.n1, fftls::kTwX1) * cb;
  G.line1 = (size_t)padded_rows(S.g.n1) * odd_up(real_eta ? (nc + 1) / 2 : nc) * cb;
  G.line5 = (size_t)padded_rows(S.g.n1) * odd_up((nc + 1) / 2) * cb;
  G.nlines = (long long)S.g.n2 * S.g.n3;
  G.tiles = (long long)((S.g.n1 + kEtaTileX - 1) / kEtaTileX) * ((S.g.n2 + kEtaTileY - 1) / kEtaTileY);
  return G;
}

size_t strided_smem(int L, int w, int nc, size_t cb) {
  return (size_t)fftls::tw_count(L, fftls::kTwStrided) * cb + (size_t)L * w * nc * cb;
}

// Built-in schedule: x1 tiles of about 32 KB (64 KB for the two-field forward
// tile), x2/x3 tiles of at most 16 modes and about 100 KB, eta slabs of up to 32
// planes with enough slabs for several waves of blocks.
TilePlan default_plan(const Setup& S, size_t cb, bool real_eta) {
  const PlanGeom G = plan_geom(S, cb, real_eta);
  TilePlan P;
  P.tuned = 0;
  P.x1_lines = (int)std::max<size_t>(1, (real_eta ? 32 * 1024 : 64 * 1024) / G.line1);
  P.x5_lines = (int)std::max<size_t>(1, (32 * 1024) / G.line5);
  P.x1_vb = cb == 16 ? 1 : 4;  // double precision loads one voxel at a time
  P.y_thr = P.z_thr = 0;
  auto pick_w = [&](int L) {
    int w = 16;
    while (w > 1 && strided_smem(L, w, S.nc, cb) > std::min<size_t>(G.lim, 100 * 1024)) w /= 2;
    while (w > 1 && w / 2 >= S.g.H) w /= 2;
    return w;
  };
  P.y_w = pick_w(S.g.n2);
  P.z_w = pick_w(S.g.n3);
  const long long want_slabs = std::max<long long>(1, (8LL * S.num_sms + G.tiles - 1) / G.tiles);
  int Z = (int)((S.g.n3 + want_slabs - 1) / want_slabs);
  P.e_planes = std::max(std::min(Z, 32), std::min(4, S.g.n3));
  return P;
}

// Derive launch shapes and shared-memory sizes from a schedule; false when it
// does not fit.
template <typename T>
bool apply_plan(const Setup& S, IterArgs<T>& a, bool real_eta, const TilePlan& P) {
  typedef typename Cplx<T>::type T2;
  const PlanGeom G = plan_geom(S, sizeof(T2), real_eta);
  const Geom& g = S.g;
  if (P.x1_lines < 1 || P.x5_lines < 1 || P.y_w < 1 || P.z_w < 1) return false;
  const int G1 = (int)std::min<long long>(P.x1_lines, G.nlines);
  const int G5 = (int)std::min<long long>(P.x5_lines, G.nlines);
  if (G.twx + G1 * G.line1 > G.lim || G.twx + G5 * G.line5 > G.lim) return false;
  a.x1_lines = G1;
  a.x5_lines = G5;
  a.x1_vb = P.x1_vb >= 4 ? 4 : P.x1_vb == 2 ? 2 : P.x1_vb == 0 ? 0 : 1;
  a.x1_smem = G.twx + G1 * G.line1;
  if (a.x1_vb == 0) {  // staged batches (FP32): the staging area after the tile
    if (sizeof(T) != 4 || g.n1 % 16 != 0) return false;
    a.x1_smem = fwd_x_stage_offset(a.x1_smem) + fwd_x_stage_bytes(G1, g.n1, S.nc);
    if (a.x1_smem > G.lim) return false;
  }
  a.x5_vb = P.x5_vb == 0 ? 0 : 1;
  a.x5_smem = G.twx + G5 * G.line5;
  if (a.x5_vb == 0) {
    if (sizeof(T) != 4 || g.n1 % 16 != 0) return false;
    a.x5_smem = fwd_x_stage_offset(a.x5_smem) + fwd_x_stage_bytes(G5, g.n1, S.nc);
    if (a.x5_smem > G.lim) return false;
  }
  a.x_threads = 256;
  a.x1_blocks = (int)std::min<long long>((G.nlines + G1 - 1) / G1, (long long)S.num_sms * 8);
  a.x5_blocks = (int)std::min<long long>((G.nlines + G5 - 1) / G5, (long long)S.num_sms * 8);
  a.y_smem = strided_smem(g.n2, P.y_w, S.nc, sizeof(T2));
  a.z_smem = strided_smem(g.n3, P.z_w, S.nc, sizeof(T2));
  if (a.y_smem > G.lim || a.z_smem > G.lim) return false;
  a.y_w = P.y_w;
  a.z_w = P.z_w;
  a.y_threads = fftls::strided_threads(a.y_w);
  a.z_threads = fftls::strided_threads(a.z_w);
  a.e_planes = a.e_blocks = 0;
  a.e_smem = 0;
  if (real_eta) {
    const int Z = std::max(1, std::min(P.e_planes, g.n3));
    a.e_planes = Z;
    a.e_blocks = (int)(G.tiles * ((g.n3 + Z - 1) / Z));
    a.e_smem = (size_t)2 * 6 * (kEtaTileY + 2) * (kEtaTileX + 2) * sizeof(T);
  }
  return true;
}

// Largest block counts over every schedule apply_plan accepts (partial-sum buffers).
size_t max_x_blocks(const Setup& S) {
  return (size_t)std::min<long long>((long long)S.g.n2 * S.g.n3, (long long)S.num_sms * 8);
}
size_t max_eta_parts(const Setup& S) {
  const PlanGeom G = plan_geom(S, 8, true);
  return std::max<size_t>((size_t)S.g.H * S.g.n2 * 2, (size_t)(G.tiles * S.g.n3));
}

template <typename T>
struct Runner {
  fftls_ctx* c;
  const Setup& S;
  IterArgs<T> a;
  bool capturing = false;
  int ns = 1;          // samples of the group (a single solve: 1)
  Ctrl* hctl;          // their control blocks on the host (pinned), read after every chunk
  Runner(fftls_ctx* c_, const Setup& S_) : c(c_), S(S_), hctl(c_->h_ctrl) { memset(&a, 0, sizeof(a)); }

  int kernels_per_iter() const { return 4 + (S.g.n2 > 1 ? 2 : 0) + (a.want_delta ? 1 : 0) + (a.eta_real ? 1 : 0); }

  fftls_status launch(int kind, cudaError_t (*fn)(Runner*, cudaStream_t), bool prof) {
    const int pi = Prec<T>::idx;
    if (!capturing) c->launches += (kind == 1 || kind == 4) ? (S.g.n2 > 1) : 1;
    if (prof) {
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, S.s);
      cudaError_t e = fn(this, S.s);
      cudaEventRecord(e1, S.s);
      if (e != cudaSuccess) return set_err(c, FFTLS_E_CUDA, "kernel %s: %s", kKindNames[pi][kind], cudaGetErrorString(e));
      c->ev.push_back({e0, e1, pi * kNumKinds + kind});
      return FFTLS_OK;
    }
    cudaError_t e = fn(this, S.s);
    if (e != cudaSuccess) return set_err(c, FFTLS_E_CUDA, "kernel %s: %s", kKindNames[pi][kind], cudaGetErrorString(e));
    return FFTLS_OK;
  }

  fftls_status iteration(bool dual, int update, bool prof) {
    a.dual = (dual && !a.eta_real) ? 1 : 0;
    a.tauform = (a.dual || a.eta_real) ? 1 : 0;
    a.update = update;
    fftls_status st;
    if (a.eta_real)
      if ((st = launch(7, [](Runner* r, cudaStream_t s) { return launch_eta_stencil<T>(r->a, s); }, prof))) return st;
    if ((st = launch(0, [](Runner* r, cudaStream_t s) { return launch_fwd_x<T>(r->a, s); }, prof))) return st;
    if ((st = launch(1, [](Runner* r, cudaStream_t s) { return launch_mid_y<T>(r->a, false, s); }, prof))) return st;
    if ((st = launch(2, [](Runner* r, cudaStream_t s) { return launch_fourier_z<T>(r->a, s); }, prof))) return st;
    if ((st = launch(3, [](Runner* r, cudaStream_t s) { return launch_reduce_eta<T>(r->a, s); }, prof))) return st;
    if ((st = launch(4, [](Runner* r, cudaStream_t s) { return launch_mid_y<T>(r->a, true, s); }, prof))) return st;
    if ((st = launch(5, [](Runner* r, cudaStream_t s) { return launch_inv_x<T>(r->a, s); }, prof))) return st;
    if (a.want_delta)
      if ((st = launch(6, [](Runner* r, cudaStream_t s) { return launch_reduce_delta<T>(r->a, s); }, prof)))
        return st;
    return FFTLS_OK;
  }

  fftls_status collect_profile() {
    if (c->ev.empty()) return FFTLS_OK;
    CUDA_TRY(c, cudaStreamSynchronize(S.s));
    for (auto& e : c->ev) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e.a, e.b);
      c->prof_ms[e.kind / kNumKinds][e.kind % kNumKinds] += ms;
      c->prof_n[e.kind / kNumKinds][e.kind % kNumKinds] += 1;
      cudaEventDestroy(e.a);
      cudaEventDestroy(e.b);
    }
    c->ev.clear();
    return FFTLS_OK;
  }

  fftls_status read_ctrl() {
    CUDA_TRY(c, cudaMemcpyAsync(hctl, a.ctrl, (size_t)ns * sizeof(Ctrl), cudaMemcpyDeviceToHost, S.s));
    CUDA_TRY(c, cudaStreamSynchronize(S.s));
    for (int i = 0; i < ns; ++i)
      if (hctl[i].fault)
        return set_err(c, FFTLS_E_TIMEOUT, "%s",
                       "a shared-memory tile copy did not complete within its wait limit; the solve was stopped");
    return FFTLS_OK;
  }
  fftls_status put_ctrl(const Ctrl* init) {
    memcpy(hctl, init, (size_t)ns * sizeof(Ctrl));
    CUDA_TRY(c, cudaMemcpyAsync(a.ctrl, hctl, (size_t)ns * sizeof(Ctrl), cudaMemcpyHostToDevice, S.s));
    return FFTLS_OK;
  }
  bool running() const {
    for (int i = 0; i < ns; ++i)
      if (hctl[i].state == kRunning) return true;
    return false;
  }

  // One iteration launched directly (no graph); the states after it are in hctl.
  fftls_status single(const Ctrl* init, bool dual, int update) {
    fftls_status st;
    if ((st = put_ctrl(init))) return st;
    if ((st = iteration(dual, update, S.profile))) return st;
    if ((st = collect_profile())) return st;
    return read_ctrl();
  }

  // eta of the current iterate without the transforms (3D G^C/G^W/G^R): the real-space
  // stencil, the means of sigma and eps, and the reduction's stop decision (no update).
  fftls_status certify(const Ctrl* init) {
    fftls_status st;
    if ((st = put_ctrl(init))) return st;
    if ((st = launch(7, [](Runner* r, cudaStream_t s) { return launch_eta_stencil<T>(r->a, s); }, S.profile)))
      return st;
    for (int i = 0; i < ns; ++i) {
      CUDA_TRY(c, launch_stress<T>(a.eps + i * a.st_field, a.phase + i * a.st_phase, a.coef + i * a.st_coef, a.dim,
                                   a.g.N, nullptr, a.part_mean + i * a.st_pmean, a.x1_blocks, S.s));
      c->launches += 1;
    }
    if ((st = launch(3, [](Runner* r, cudaStream_t s) { return launch_reduce_eta<T>(r->a, s); }, S.profile)))
      return st;
    if ((st = collect_profile())) return st;
    return read_ctrl();
  }

  // Run iterations until no sample's state is kRunning (states in hctl).
  fftls_status run(const Ctrl* init, bool first_dual, bool dual, int update) {
    fftls_status st;
    if ((st = put_ctrl(init))) return st;
    if (first_dual && !dual) {
      if ((st = iteration(true, kUpdDirectTau, S.profile))) return st;
      if ((st = collect_profile())) return st;
      if ((st = read_ctrl())) return st;
      if (!running()) return FFTLS_OK;
    }
    const long long N = S.g.N * ns;
    const int chunk = (int)std::max<long long>(1, std::min<long long>(32, 40000000LL / std::max<long long>(N, 1)));
    cudaGraphExec_t exec = nullptr;
    if (S.graphs && !S.profile) {
      a.dual = (dual && !a.eta_real) ? 1 : 0;
      a.tauform = (a.dual || a.eta_real) ? 1 : 0;
      a.update = update;
      GraphCache& gc = c->graphs[Prec<T>::idx];
      std::vector<unsigned char> key(sizeof(a) + sizeof(int));
      memcpy(key.data(), &a, sizeof(a));
      memcpy(key.data() + sizeof(a), &chunk, sizeof(int));
      if (gc.exec && gc.key == key) {
        exec = gc.exec;
      } else {
        gc.release();
        cudaGraph_t graph;
        CUDA_TRY(c, cudaStreamBeginCapture(S.s, cudaStreamCaptureModeThreadLocal));
        fftls_status cs = FFTLS_OK;
        capturing = true;
        for (int i = 0; i < chunk && cs == FFTLS_OK; ++i) cs = iteration(dual, update, false);
        capturing = false;
        cudaError_t ce = cudaStreamEndCapture(S.s, &graph);
        if (cs) return cs;
        CUDA_TRY(c, ce);
        ce = cudaGraphInstantiate(&gc.exec, graph, 0);
        cudaGraphDestroy(graph);
        CUDA_TRY(c, ce);
        gc.key = key;
        exec = gc.exec;
      }
    }
    for (;;) {
      if (exec) {
        CUDA_TRY(c, cudaGraphLaunch(exec, S.s));
        c->graph_launches += 1;
        c->launches += (long long)chunk * kernels_per_iter();
      } else {
        for (int i = 0; i < chunk; ++i)
          if ((st = iteration(dual, update, S.profile))) return st;
        if ((st = collect_profile())) return st;
      }
      if ((st = read_ctrl())) return st;
      if (!running()) break;
    }
    return FFTLS_OK;
  }
};

// Autotuner: time the candidate schedules of each kernel on the live buffers and
// keep the fastest, one kernel at a time (the kernels of an iteration are
// separate launches, so their schedules are independent).  It runs before the
// first iteration: the forward passes and the eta kernel only read the iterate,
// the strided passes work in place on the spectrum, and the inverse x1 pass
// writes its update into specB (unused at that point) instead of the iterate.
template <typename T>
fftls_status tune_plan(fftls_ctx* c, const Setup& S, IterArgs<T>& a, bool real_eta, TilePlan& P) {
  typedef cudaError_t (*LaunchFn)(const IterArgs<T>&, cudaStream_t);
  const IterArgs<T> keep = a;
  cudaStream_t s = S.s;
  Ctrl run;
  memset(&run, 0, sizeof(run));
  run.state = kRunning;
  CUDA_TRY(c, cudaMemcpyAsync(a.ctrl, &run, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
  a.dual = (!real_eta && S.scheme == FFTLS_ACCELERATED) ? 1 : 0;
  a.tauform = (a.dual || real_eta) ? 1 : 0;
  a.update = kUpdAccel;
  a.want_delta = a.write_d64 = a.corr = 0;
  cudaEvent_t e0, e1;
  CUDA_TRY(c, cudaEventCreate(&e0));
  CUDA_TRY(c, cudaEventCreate(&e1));
  constexpr int kReps = 2;
  auto timed = [&](LaunchFn fn, float* ms) -> cudaError_t {
    cudaError_t e = fn(a, s);  // warm-up
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecord(e0, s)) != cudaSuccess) return e;
    for (int r = 0; r < kReps; ++r)
      if ((e = fn(a, s)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(e1, s)) != cudaSuccess) return e;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
    return cudaEventElapsedTime(ms, e0, e1);
  };
  cudaError_t err = cudaSuccess;
  auto search = [&](int TilePlan::*field, const std::vector<int>& cands, LaunchFn fn) {
    float best = INFINITY;
    int bestv = P.*field;
    for (int v : cands) {
      if (err != cudaSuccess) return;
      TilePlan Q = P;
      Q.*field = v;
      if (!apply_plan<T>(S, a, real_eta, Q)) continue;
      float ms = 0.f;
      err = timed(fn, &ms);
      c->launches += 1 + kReps;
      if (ms < best) {
        best = ms;
        bestv = v;
      }
    }
    P.*field = bestv;
    apply_plan<T>(S, a, real_eta, P);
  };
  // tile widths of the strided passes: powers of two up to 16 modes, no wider than the half spectrum needs
  std::vector<int> widths;
  for (int w = 1; w <= 16; w *= 2)
    if (w == 1 || w / 2 < S.g.H) widths.push_back(w);
  // forward x1 pass: lines per batch and voxels loaded together, searched jointly
  {
    float best = INFINITY;
    int bl = P.x1_lines, bv = P.x1_vb;
    // (vb = 0: the batches staged in shared memory by bulk copies, FP32)
    const std::vector<int> vbs = sizeof(T) == 8 ? std::vector<int>{1} : std::vector<int>{1, 2, 4, 0};
    for (int lines : {1, 2, 4, 8})
      for (int vb : vbs) {
        if (err != cudaSuccess) break;
        TilePlan Q = P;
        Q.x1_lines = lines;
        Q.x1_vb = vb;
        if (!apply_plan<T>(S, a, real_eta, Q)) continue;
        float ms = 0.f;
        err = timed([](const IterArgs<T>& x, cudaStream_t st) { return launch_fwd_x<T>(x, st); }, &ms);
        c->launches += 1 + kReps;
        if (ms < best) {
          best = ms;
          bl = lines;
          bv = vb;
        }
      }
    P.x1_lines = bl;
    P.x1_vb = bv;
    apply_plan<T>(S, a, real_eta, P);
  }
  // strided passes: tile width (the block size follows from it, strided_threads)
  auto search_wt = [&](int TilePlan::*wf, int TilePlan::*tf, LaunchFn fn) {
    float best = INFINITY;
    int bw = P.*wf, bt = P.*tf;
    for (int w : widths)
      for (int thr : {fftls::strided_threads(w)}) {
        if (err != cudaSuccess) return;
        TilePlan Q = P;
        Q.*wf = w;
        Q.*tf = thr;
        if (!apply_plan<T>(S, a, real_eta, Q)) continue;
        float ms = 0.f;
        err = timed(fn, &ms);
        c->launches += 1 + kReps;
        if (ms < best) {
          best = ms;
          bw = w;
          bt = thr;
        }
      }
    P.*wf = bw;
    P.*tf = bt;
    apply_plan<T>(S, a, real_eta, P);
  };
  if (S.g.n2 > 1)
    search_wt(&TilePlan::y_w, &TilePlan::y_thr,
              [](const IterArgs<T>& x, cudaStream_t st) { return launch_mid_y<T>(x, false, st); });
  search_wt(&TilePlan::z_w, &TilePlan::z_thr,
            [](const IterArgs<T>& x, cudaStream_t st) { return launch_fourier_z<T>(x, st); });
  a.eps = (T*)c->specB.p;  // scratch target of the inverse pass's update
  // inverse x1 pass: lines per batch and (FP32) eps loaded by the threads or staged by bulk copies, jointly
  {
    float best = INFINITY;
    int bl = P.x5_lines, bv = P.x5_vb;
    const std::vector<int> vbs = sizeof(T) == 8 ? std::vector<int>{1} : std::vector<int>{1, 0};
    for (int lines : {1, 2, 4, 8})
      for (int vb : vbs) {
        if (err != cudaSuccess) break;
        TilePlan Q = P;
        Q.x5_lines = lines;
        Q.x5_vb = vb;
        if (!apply_plan<T>(S, a, real_eta, Q)) continue;
        float ms = 0.f;
        err = timed([](const IterArgs<T>& x, cudaStream_t st) { return launch_inv_x<T>(x, st); }, &ms);
        c->launches += 1 + kReps;
        if (ms < best) {
          best = ms;
          bl = lines;
          bv = vb;
        }
      }
    P.x5_lines = bl;
    P.x5_vb = bv;
    apply_plan<T>(S, a, real_eta, P);
  }
  a.eps = keep.eps;
  if (real_eta)
    search(&TilePlan::e_planes, {4, 8, 16, 32, 64},
           [](const IterArgs<T>& x, cudaStream_t st) { return launch_eta_stencil<T>(x, st); });
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return set_err(c, FFTLS_E_CUDA, "autotune: %s", cudaGetErrorString(err));
  P.tuned = 1;
  a = keep;
  apply_plan<T>(S, a, real_eta, P);
  return FFTLS_OK;
}

template <typename T>
fftls_status prepare(fftls_ctx* c, const Setup& S, const fftls_problem* p, const fftls_options* o, Runner<T>& R,
                     T* eps, const std::vector<double>& tab, const int* d_perms) {
  typedef typename Cplx<T>::type T2;
  IterArgs<T>& a = R.a;
  a.g = S.g;
  a.dim = S.dim;
  a.green = S.green;
  for (int ax = 0; ax < 3; ++ax) a.pl[ax] = S.pl[ax];
  a.lam0 = S.lam0;
  a.mu0 = S.mu0;
  for (int i = 0; i < 6; ++i) a.eps_bar[i] = S.eps_bar[i];
  const bool real_eta = S.dim == 3 && S.green != kMS;
  const PlanKey key{Prec<T>::idx, S.g.n1, S.g.n2, S.g.n3, S.dim, S.green, real_eta ? 1 : 0};
  int cached = -1;
  for (size_t i = 0; i < c->plans.size(); ++i)
    if (c->plans[i].first == key) cached = (int)i;
  TilePlan P = cached >= 0 ? c->plans[cached].second : default_plan(S, sizeof(T2), real_eta);
  if (!apply_plan<T>(S, a, real_eta, P))
    return set_err(c, FFTLS_E_UNSUPPORTED_SIZE, "grid %dx%dx%d does not fit the shared-memory tiles", S.g.n1, S.g.n2,
                   S.g.n3);
  // coefficients and tables in precision T
  std::vector<double> cf(256 * kCoef);
  coef_table(S, p, cf.data());
  std::vector<T> cfT(cf.begin(), cf.end()), tabT(tab.begin(), tab.end());
  DevBuf& cb = Prec<T>::idx ? c->coef64 : c->coef32;
  DevBuf& tb = Prec<T>::idx ? c->tab64 : c->tab32;
  CUDA_TRY(c, cb.ensure(cfT.size() * sizeof(T)));
  CUDA_TRY(c, tb.ensure(tabT.size() * sizeof(T)));
  CUDA_TRY(c, cudaMemcpyAsync(cb.p, cfT.data(), cfT.size() * sizeof(T), cudaMemcpyHostToDevice, S.s));
  CUDA_TRY(c, cudaMemcpyAsync(tb.p, tabT.data(), tabT.size() * sizeof(T), cudaMemcpyHostToDevice, S.s));
  CUDA_TRY(c, cudaStreamSynchronize(S.s));  // the host vectors go out of scope
  a.coef = (const T*)cb.p;
  size_t po = 0;
  for (int ax = 0; ax < 3; ++ax) {
    a.tw[ax] = (const T2*)((const T*)tb.p + table_offset_tw(S, ax));
    a.kt[ax] = (const KTab<T>*)((const T*)tb.p + table_offset_kt(S, ax));
    a.rd[ax] = (const T2*)((const T*)tb.p + table_offset_rd(S, ax));
    a.perm[ax] = d_perms + po;
    a.pos[ax] = d_perms + po + S.pl[ax].L;
    po += 2 * (size_t)S.pl[ax].L;
  }
  a.eps = eps;
  a.phase = S.d_phase;
  a.specA = (T2*)c->specA.p;
  a.specB = (T2*)c->specB.p;
  a.ctrl = (Ctrl*)c->ctrl.p;
  a.eta_hist = (double*)c->eta_hist.p;
  a.ms_hist = (double*)c->ms_hist.p;
  a.want_delta = o->stop == FFTLS_STOP_MAXDELTA ? 1 : 0;
  a.eta_real = real_eta ? 1 : 0;
  // partial-sum buffers sized for every schedule the tuner may pick
  CUDA_TRY(c, c->part_mean.ensure(max_x_blocks(S) * 2 * S.nc * sizeof(double)));
  CUDA_TRY(c, c->part_eta.ensure(max_eta_parts(S) * sizeof(double)));
  CUDA_TRY(c, c->part_delta.ensure(max_x_blocks(S) * 2 * sizeof(double)));
  a.part_mean = (double*)c->part_mean.p;
  a.part_eta = (double*)c->part_eta.p;
  a.part_delta = (double*)c->part_delta.p;
  a.rfield = (float*)c->rfield.p;
  a.d64 = (float2*)c->d64.p;
  CUDA_TRY(c, set_kernel_attributes<T>(a, (size_t)S.smem_optin - 4096));
  if (o->autotune && !P.tuned) {
    fftls_status st = tune_plan<T>(c, S, a, real_eta, P);
    if (st) return st;
  }
  if (cached >= 0) c->plans[cached].second = P;
  else c->plans.push_back({key, P});
  return FFTLS_OK;
}

void mandel_unit(int dim, int J, double* e) {
  for (int i = 0; i < 6; ++i) e[i] = 0.0;
  e[J] = J < dim ? 1.0 : 1.0 / sqrt(2.0);
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void fftls_default_options(fftls_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->tol = 1e-8;
  o->stop = FFTLS_STOP_ETA;
  o->max_iter = 1000;
  o->precision = FFTLS_FP64;
  o->refine_switch = 0.0;
  o->use_graphs = 1;
  o->autotune = 1;
}

fftls_status fftls_tile_plans(const fftls_ctx* c, int* rows, int* count) {
  if (!c || !count || *count < 0 || (*count > 0 && !rows)) return FFTLS_E_INVALID_ARG;
  const int held = (int)c->plans.size();
  for (int i = 0; i < std::min(*count, held); ++i) {
    const PlanKey& k = c->plans[i].first;
    const TilePlan& P = c->plans[i].second;
    const int row[FFTLS_PLAN_FIELDS] = {k.prec,     k.n1,  k.n2,  k.n3, k.green, P.x1_lines, P.x1_vb,
                                        P.x5_lines, P.y_w, P.z_w, k.real_eta ? P.e_planes : 0, P.tuned,
                                        P.y_thr,    P.z_thr, P.x5_vb};
    memcpy(rows + (size_t)i * FFTLS_PLAN_FIELDS, row, sizeof(row));
  }
  *count = held;
  return FFTLS_OK;
}

fftls_status fftls_set_tile_plans(fftls_ctx* c, const int* rows, int count) {
  if (!c || count < 0 || (count > 0 && !rows)) return FFTLS_E_INVALID_ARG;
  std::vector<std::pair<PlanKey, TilePlan>> add;
  for (int i = 0; i < count; ++i) {
    const int* r = rows + (size_t)i * FFTLS_PLAN_FIELDS;
    const int prec = r[0], n1 = r[1], n2 = r[2], n3 = r[3], green = r[4];
    TilePlan P;
    P.x1_lines = r[5];
    P.x1_vb = r[6];
    P.x5_lines = r[7];
    P.y_w = r[8];
    P.z_w = r[9];
    P.e_planes = r[10];
    P.y_thr = r[12];
    P.z_thr = r[13];
    P.x5_vb = r[14];
    P.tuned = 1;  // imported schedules are used as they are, never re-tuned
    auto pow2_16 = [](int w) { return w == 1 || w == 2 || w == 4 || w == 8 || w == 16; };
    auto thr_ok = [](int t, int w) { return t == 0 || t == fftls::strided_threads(w); };
    const bool ok = (prec == 0 || prec == 1) && n1 >= 1 && n2 >= 1 && n3 >= 1 && green >= kMS && green <= kRotated &&
                    P.x1_lines >= 1 && P.x1_lines <= 8 && P.x5_lines >= 1 && P.x5_lines <= 8 &&
                    (P.x1_vb == 1 || P.x1_vb == 2 || P.x1_vb == 4 || (P.x1_vb == 0 && prec == 0 && n1 % 16 == 0)) &&
                    (prec == 0 || P.x1_vb == 1) && (P.x5_vb == 1 || (P.x5_vb == 0 && prec == 0 && n1 % 16 == 0)) &&
                    pow2_16(P.y_w) && pow2_16(P.z_w) && P.e_planes >= 0 &&
                    P.e_planes <= n3 && thr_ok(P.y_thr, P.y_w) && thr_ok(P.z_thr, P.z_w);
    if (!ok) return set_err(c, FFTLS_E_INVALID_ARG, "tile plan row %d is not a valid schedule", i);
    // a row names the grid, not the dimension: it serves the 3D problem on it and, with n3 = 1, the 2D one
    for (int dim = 2; dim <= 3; ++dim) {
      if (dim == 2 && n3 != 1) continue;
      const bool real_eta = dim == 3 && green != kMS;
      if (real_eta && P.e_planes < 1) continue;
      add.push_back({PlanKey{prec, n1, n2, n3, dim, green, real_eta ? 1 : 0}, P});
    }
  }
  for (auto& kv : add) {
    bool have = false;
    for (auto& mine : c->plans)
      if (mine.first == kv.first) {
        mine.second = kv.second;
        have = true;
      }
    if (!have) c->plans.push_back(kv);
  }
  return FFTLS_OK;
}

fftls_status fftls_create(fftls_ctx** out, int device) {
  if (!out) return FFTLS_E_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FFTLS_E_CUDA;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return FFTLS_E_CUDA;
  fftls_ctx* c = new fftls_ctx();
  c->device = device;
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, device);
  c->smem_optin = prop.sharedMemPerBlockOptin;
  c->num_sms = prop.multiProcessorCount;
  bool ok = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMallocHost((void**)&c->h_ctrl, sizeof(Ctrl)) == cudaSuccess &&
            cudaMallocHost((void**)&c->h_sums, 64 * sizeof(double)) == cudaSuccess &&
            c->ctrl.ensure(sizeof(Ctrl)) == cudaSuccess && c->sums.ensure(64 * sizeof(double)) == cudaSuccess;
  memset(c->prof_ms, 0, sizeof(c->prof_ms));
  memset(c->prof_n, 0, sizeof(c->prof_n));
  cudaSetDevice(prev);
  if (!ok) {
    fftls_destroy(c);
    return FFTLS_E_CUDA;
  }
  *out = c;
  return FFTLS_OK;
}

void fftls_destroy(fftls_ctx* c) {
  if (!c) return;
  for (fftls_ctx* w : c->workers) fftls_destroy(w);
  c->workers.clear();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  for (auto& g : c->graphs) g.release();
  DevBuf* bufs[] = {&c->phase, &c->eps32, &c->eps64, &c->specA, &c->specB, &c->coef32, &c->coef64, &c->tab32,
                    &c->tab64, &c->perms, &c->part_mean, &c->part_eta, &c->part_delta, &c->sums, &c->ctrl,
                    &c->eta_hist, &c->ms_hist, &c->scratch, &c->rfield, &c->d64};
  for (DevBuf* b : bufs) b->release();
  for (auto& e : c->ev) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  if (c->h_ctrl) cudaFreeHost(c->h_ctrl);
  if (c->h_gctrl) cudaFreeHost(c->h_gctrl);
  c->gpar.release();
  if (c->h_sums) cudaFreeHost(c->h_sums);
  if (c->stream) cudaStreamDestroy(c->stream);
  cudaSetDevice(prev);
  delete c;
}

const char* fftls_last_error(const fftls_ctx* c) { return c ? c->err.c_str() : ""; }

fftls_status fftls_counters(const fftls_ctx* c, long long* kernel_launches, long long* graph_launches) {
  if (!c) return FFTLS_E_INVALID_ARG;
  if (kernel_launches) *kernel_launches = c->launches;
  if (graph_launches) *graph_launches = c->graph_launches;
  return FFTLS_OK;
}

const char* fftls_status_string(fftls_status s) {
  switch (s) {
    case FFTLS_OK: return "FFTLS_OK";
    case FFTLS_E_INVALID_ARG: return "FFTLS_E_INVALID_ARG";
    case FFTLS_E_UNSUPPORTED_SIZE: return "FFTLS_E_UNSUPPORTED_SIZE";
    case FFTLS_E_OOM: return "FFTLS_E_OOM";
    case FFTLS_E_CUDA: return "FFTLS_E_CUDA";
    case FFTLS_E_NOT_CONVERGED: return "FFTLS_E_NOT_CONVERGED";
    case FFTLS_E_DIVERGED: return "FFTLS_E_DIVERGED";
    case FFTLS_E_TIMEOUT: return "FFTLS_E_TIMEOUT";
  }
  return "unknown";
}

fftls_status fftls_supported_length(int L) {
  AxisPlan p;
  return factor_plan(L, &p) ? FFTLS_OK : FFTLS_E_UNSUPPORTED_SIZE;
}

fftls_status fftls_reference_medium(const fftls_problem* p, double* l0, double* m0) {
  if (!p || !l0 || !m0 || (p->dim != 2 && p->dim != 3) || p->n_phases < 1 || !p->lambda || !p->mu)
    return FFTLS_E_INVALID_ARG;
  return default_medium(p, l0, m0) ? FFTLS_OK : FFTLS_E_INVALID_ARG;
}

fftls_status fftls_profile(const fftls_ctx* c, const char** names, double* total_ms, int* launches, int* count) {
  if (!c || !count) return FFTLS_E_INVALID_ARG;
  int n = 0;
  for (int p = 0; p < 2; ++p)
    for (int k = 0; k < kNumKinds; ++k) {
      if (!c->prof_n[p][k]) continue;
      if (n < *count) {
        if (names) names[n] = kKindNames[p][k];
        if (total_ms) total_ms[n] = c->prof_ms[p][k];
        if (launches) launches[n] = c->prof_n[p][k];
      }
      ++n;
    }
  *count = n;
  return FFTLS_OK;
}

// Solve ns problems that share one grid, dimension, operator and scheme (a single
// solve is ns = 1; ns > 1 runs every kernel of the iteration as one grouped launch
// over the samples, 3D only, and every sample follows exactly the path it would
// take alone: its own control block, stop decisions, precision ladder and
// history).  Per-sample statuses go to stat[]; the return value is the first
// error that stopped the whole group (FFTLS_OK otherwise).
static fftls_status solve_core(fftls_ctx* c, const fftls_problem* const* P, int ns, const fftls_options* o,
                               fftls_result* const* R, fftls_status* stat) {
  const fftls_problem* p = P[0];
  for (int i = 0; i < ns; ++i) {
    fftls_status st = validate(c, P[i], o);
    if (st) return st;
    if (!R[i]) return set_err(c, FFTLS_E_INVALID_ARG, "null result");
  }
  if (ns > 1 && o->eps_init) return set_err(c, FFTLS_E_INVALID_ARG, "grouped solve: eps_init must be NULL");
  Setup S;
  memset(&S, 0, sizeof(S));
  setup_geometry(S, p);
  const int d = S.dim, nc = S.nc;
  if (ns > 1 && d != 3) return set_err(c, FFTLS_E_INVALID_ARG, "grouped solve: 3D grids only");
  std::vector<Setup> Ss(ns);
  for (int i = 0; i < ns; ++i) {
    memset(&Ss[i], 0, sizeof(Setup));
    setup_geometry(Ss[i], P[i]);
  }
  S.s = o->stream ? (cudaStream_t)o->stream : c->stream;
  S.profile = o->profile != 0;
  S.graphs = o->use_graphs != 0;
  S.smem_optin = (int)c->smem_optin;
  S.num_sms = c->num_sms;
  const long long N = S.g.N;
  if (S.profile) {
    memset(c->prof_ms, 0, sizeof(c->prof_ms));
    memset(c->prof_n, 0, sizeof(c->prof_n));
  }
  // phase images on the device (one slice per sample), ids checked there (< n_phases)
  if (ns == 1 && p->phase_on_device) {
    S.d_phase = p->phase;
  } else {
    CUDA_TRY(c, c->phase.ensure((size_t)N * ns));
    for (int i = 0; i < ns; ++i)
      CUDA_TRY(c, cudaMemcpyAsync((uint8_t*)c->phase.p + (size_t)i * N, P[i]->phase, (size_t)N,
                                  P[i]->phase_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, S.s));
    S.d_phase = (const uint8_t*)c->phase.p;
  }
  {
    CUDA_TRY(c, c->sums.ensure(std::max<size_t>(64 * sizeof(double), (size_t)ns * sizeof(unsigned int))));
    const int pb = (int)std::min<long long>((N + 255) / 256, (long long)c->num_sms * 8);
    for (int i = 0; i < ns; ++i) {
      CUDA_TRY(c, launch_phase_max(S.d_phase + (size_t)i * N, N, (unsigned int*)c->sums.p + i, pb, S.s));
      c->launches += 1;
    }
    std::vector<unsigned int> pmax(ns);
    CUDA_TRY(c, cudaMemcpyAsync(pmax.data(), c->sums.p, (size_t)ns * sizeof(unsigned int), cudaMemcpyDeviceToHost, S.s));
    CUDA_TRY(c, cudaStreamSynchronize(S.s));
    for (int i = 0; i < ns; ++i)
      if ((int)pmax[i] >= P[i]->n_phases)
        return set_err(c, FFTLS_E_INVALID_ARG, "%sphase image holds id %u >= n_phases = %d",
                       ns > 1 ? "sample of the group: " : "", pmax[i], P[i]->n_phases);
  }
  const bool use32 = o->precision != FFTLS_FP64;
  const bool use64 = o->precision != FFTLS_FP32;
  const bool ladder = o->precision == FFTLS_FP32_REFINE64;
  const size_t spec_bytes = (size_t)S.g.modes * nc * (use64 ? 16 : 8);
  CUDA_TRY(c, c->specA.ensure(spec_bytes * ns));
  CUDA_TRY(c, c->specB.ensure(spec_bytes * ns));
  if (use32) CUDA_TRY(c, c->eps32.ensure((size_t)nc * N * sizeof(float) * ns));
  if (use64 || o->eps_init) CUDA_TRY(c, c->eps64.ensure((size_t)nc * N * sizeof(double) * ns));
  const size_t d64_elems = std::max<size_t>((size_t)S.g.modes * 3, (size_t)(3 * N + 1) / 2);  // float2 units
  if (ladder) {
    CUDA_TRY(c, c->rfield.ensure((size_t)nc * N * sizeof(float) * ns));
    CUDA_TRY(c, c->d64.ensure(d64_elems * sizeof(float2) * ns));
  }
  CUDA_TRY(c, c->eta_hist.ensure((size_t)o->max_iter * sizeof(double) * ns));
  CUDA_TRY(c, c->ms_hist.ensure((size_t)o->max_iter * 6 * sizeof(double) * ns));
  CUDA_TRY(c, c->ctrl.ensure(sizeof(Ctrl) * ns));
  Ctrl* hctl = c->h_ctrl;
  if (ns > 1) {
    if (c->h_gcap < ns) {
      if (c->h_gctrl) cudaFreeHost(c->h_gctrl);
      c->h_gctrl = nullptr;
      c->h_gcap = 0;
      CUDA_TRY(c, cudaMallocHost((void**)&c->h_gctrl, sizeof(Ctrl) * ns));
      c->h_gcap = ns;
    }
    hctl = c->h_gctrl;
  }
  // tables shared by both precisions
  std::vector<double> tab;
  std::vector<int> perms;
  build_tables(S, tab, perms);
  CUDA_TRY(c, c->perms.ensure(perms.size() * sizeof(int)));
  CUDA_TRY(c, cudaMemcpyAsync(c->perms.p, perms.data(), perms.size() * sizeof(int), cudaMemcpyHostToDevice, S.s));
  const int* d_perms = (const int*)c->perms.p;
  // initial fields
  const bool warm = o->eps_init != nullptr;
  if (warm) {
    CUDA_TRY(c, cudaMemcpyAsync(c->eps64.p, o->eps_init, (size_t)nc * N * sizeof(double),
                                o->eps_init_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, S.s));
    if (use32) {
      CUDA_TRY(c, launch_convert<float, double>((float*)c->eps32.p, (const double*)c->eps64.p, (long long)nc * N, S.s));
      c->launches += 1;
    }
  } else {
    for (int i = 0; i < ns; ++i) {
      if (o->precision == FFTLS_FP64)
        CUDA_TRY(c, launch_fill_eps<double>((double*)c->eps64.p + (size_t)i * nc * N, nc, N, Ss[i].eps_bar, S.s));
      else
        CUDA_TRY(c, launch_fill_eps<float>((float*)c->eps32.p + (size_t)i * nc * N, nc, N, Ss[i].eps_bar, S.s));
      c->launches += 1;
    }
  }
  const bool direct = p->scheme == FFTLS_DIRECT;
  // G^C / G^W / G^R in 3D take eta from the real-space stencil and transform tau
  // only (tau form for both schemes); otherwise AS transforms tau and sigma and
  // DS uses the sigma form while its iterate is compatible.
  auto upd_of = [&](bool er) { return direct ? (er ? (int)kUpdDirectTau : (int)kUpdDirectSig) : (int)kUpdAccel; };
  const bool dual_steady = !direct;
  // a group's per-sample views: coefficient tables, parameters, partial sums, strides
  auto group_view = [&](auto& Rn) -> fftls_status {
    typedef typename std::remove_reference<decltype(Rn.a)>::type ArgsT;
    typedef typename std::remove_pointer<decltype(Rn.a.eps)>::type T;
    ArgsT& a = Rn.a;
    Rn.ns = ns;
    Rn.hctl = hctl;
    if (ns == 1) return FFTLS_OK;
    std::vector<double> cf((size_t)ns * 256 * kCoef), par((size_t)ns * 8);
    for (int i = 0; i < ns; ++i) {
      coef_table(Ss[i], P[i], &cf[(size_t)i * 256 * kCoef]);
      par[8 * (size_t)i] = Ss[i].lam0;
      par[8 * (size_t)i + 1] = Ss[i].mu0;
      for (int k = 0; k < 6; ++k) par[8 * (size_t)i + 2 + k] = Ss[i].eps_bar[k];
    }
    std::vector<T> cfT(cf.begin(), cf.end());
    DevBuf& cb = Prec<T>::idx ? c->coef64 : c->coef32;
    CUDA_TRY(c, cb.ensure(cfT.size() * sizeof(T)));
    CUDA_TRY(c, c->gpar.ensure(par.size() * sizeof(double)));
    CUDA_TRY(c, cudaMemcpyAsync(cb.p, cfT.data(), cfT.size() * sizeof(T), cudaMemcpyHostToDevice, S.s));
    CUDA_TRY(c, cudaMemcpyAsync(c->gpar.p, par.data(), par.size() * sizeof(double), cudaMemcpyHostToDevice, S.s));
    CUDA_TRY(c, cudaStreamSynchronize(S.s));  // the host vectors go out of scope
    const size_t pm = max_x_blocks(S) * 2 * nc, pe = max_eta_parts(S), pd = max_x_blocks(S) * 2;
    CUDA_TRY(c, c->part_mean.ensure(pm * sizeof(double) * ns));
    CUDA_TRY(c, c->part_eta.ensure(pe * sizeof(double) * ns));
    CUDA_TRY(c, c->part_delta.ensure(pd * sizeof(double) * ns));
    a.coef = (const T*)cb.p;
    a.part_mean = (double*)c->part_mean.p;
    a.part_eta = (double*)c->part_eta.p;
    a.part_delta = (double*)c->part_delta.p;
    a.nsmp = ns;
    a.st_field = (long long)nc * N;
    a.st_phase = N;
    a.st_spec = (long long)S.g.modes * nc;
    a.st_coef = 256 * kCoef;
    a.st_pmean = (long long)pm;
    a.st_peta = (long long)pe;
    a.st_pdelta = (long long)pd;
    a.st_hist = o->max_iter;
    a.st_d64 = a.d64 ? (long long)d64_elems : 0;
    a.smp_par = (const double*)c->gpar.p;
    return FFTLS_OK;
  };
  Ctrl ctl0;
  memset(&ctl0, 0, sizeof(ctl0));
  ctl0.state = kRunning;
  ctl0.max_it = o->max_iter;
  ctl0.mean_guard = (direct || o->eta_only) ? 0 : 1;
  ctl0.best = INFINITY;
  ctl0.stop_rule = o->stop;
  ctl0.tol = o->tol;
  std::vector<Ctrl> ctl(ns, ctl0), init(ns);
  std::vector<int> state(ns, kRunning), it32(ns, 0);
  std::vector<char> final64(ns, o->precision == FFTLS_FP64 ? 1 : 0);  // the returned field is the FP64 iterate
  fftls_status st;
  auto take = [&](int i) { ctl[i] = hctl[i]; state[i] = hctl[i].state; };
  if (o->precision == FFTLS_FP64) {
    Runner<double> R64(c, S);
    if ((st = prepare<double>(c, S, p, o, R64, (double*)c->eps64.p, tab, d_perms))) return st;
    if ((st = group_view(R64))) return st;
    const bool er = R64.a.eta_real;
    if ((st = R64.run(ctl.data(), direct && warm && !er, dual_steady, upd_of(er)))) return st;
    for (int i = 0; i < ns; ++i) take(i);
  } else if (o->precision == FFTLS_FP32) {
    Runner<float> R32(c, S);
    if ((st = prepare<float>(c, S, p, o, R32, (float*)c->eps32.p, tab, d_perms))) return st;
    if ((st = group_view(R32))) return st;
    const bool er = R32.a.eta_real;
    if ((st = R32.run(ctl.data(), direct && warm && !er, dual_steady, upd_of(er)))) return st;
    for (int i = 0; i < ns; ++i) {
      take(i);
      it32[i] = ctl[i].it;
    }
  } else {
    // Ladder.  A: plain FP32 iterations until eta <= refine_switch (or a stall).
    Runner<float> R32(c, S);
    if ((st = prepare<float>(c, S, p, o, R32, (float*)c->eps32.p, tab, d_perms))) return st;
    Runner<double> R64(c, S);
    if ((st = prepare<double>(c, S, p, o, R64, (double*)c->eps64.p, tab, d_perms))) return st;
    if ((st = group_view(R32))) return st;
    if ((st = group_view(R64))) return st;
    // both precisions must measure eta the same way (the FP64 divergence feeds the FP32 estimate)
    if (R32.a.eta_real != R64.a.eta_real)
      return set_err(c, FFTLS_E_CUDA, "internal: FP32 and FP64 plans measure eta differently");
    for (int i = 0; i < ns; ++i) {
      init[i] = ctl0;
      init[i].stop_rule = 0;
      init[i].tol = o->refine_switch > 0.0 ? o->refine_switch : std::max(o->tol, 3e-5);
      init[i].switch_mode = 1;
      init[i].stall_window = 32;
    }
    R32.a.want_delta = 0;
    const bool er = R32.a.eta_real;
    if ((st = R32.run(init.data(), direct && warm && !er, dual_steady, upd_of(er)))) return st;
    std::vector<char> active(ns, 0);
    bool any = false;
    for (int i = 0; i < ns; ++i) {
      take(i);
      it32[i] = ctl[i].it;
      active[i] = state[i] == kSwitch;
      any = any || active[i];
    }
    for (int i = 0; i < ns; ++i) final64[i] = active[i];
    if (any) {
      CUDA_TRY(c, launch_convert<double, float>((double*)c->eps64.p, (const float*)c->eps32.p, (long long)nc * N * ns, S.s));
      c->launches += 1;
      // B / C: FP64 defect of the iterate (and its exact eta), then an FP32
      // correction solve for delta, eps64 += delta; until the FP64 eta passes.
      R64.a.write_d64 = 1;
      R32.a.corr = 1;
      for (int i = 0; i < ns; ++i)
        if (active[i]) state[i] = kRunning;
      Ctrl idle;
      memset(&idle, 0, sizeof(idle));
      idle.state = kStopped;  // samples that take no part: every kernel of theirs exits at once
      for (int outer = 0; outer < kMaxOuter && any; ++outer) {
        for (int i = 0; i < ns; ++i) {
          init[i] = idle;
          if (!active[i]) continue;
          if (ctl[i].it >= o->max_iter) {
            state[i] = kStopped;
            active[i] = 0;
            continue;
          }
          Ctrl cb = ctl[i];
          cb.state = kRunning;
          cb.stop_rule = 0;
          cb.tol = o->tol;
          cb.switch_mode = 0;
          cb.stall_window = 0;
          cb.phase_max = 0;
          cb.max_it = ctl[i].it + 1;  // exactly one evaluation; kLast runs the residual update
          for (int k = 0; k < 6; ++k) cb.off_sig[k] = cb.off_eps[k] = 0.0;
          init[i] = cb;
        }
        if (outer > 0 && R64.a.eta_real) {
          // after a correction: certify eta of eps64 first; the full FP64 pass (defect and eta)
          // only runs if the certificate fails, and then its own eta evaluation counts instead
          if ((st = R64.certify(init.data()))) return st;
          for (int i = 0; i < ns; ++i) {
            if (!active[i]) continue;
            if (hctl[i].state == kConverged || hctl[i].state == kDiverged) {
              take(i);
              ctl[i].max_it = o->max_iter;
              active[i] = 0;
              init[i] = idle;
            }
          }
        }
        if ((st = R64.single(init.data(), true, kUpdResidual))) return st;
        any = false;
        for (int i = 0; i < ns; ++i) {
          if (!active[i]) {
            init[i] = idle;
            continue;
          }
          take(i);
          ctl[i].max_it = o->max_iter;
          init[i] = idle;
          if (state[i] == kConverged || state[i] == kDiverged) {
            active[i] = 0;
            continue;
          }
          if (ctl[i].it >= o->max_iter) {
            state[i] = kStopped;
            active[i] = 0;
            continue;
          }
          // C: correction delta from 0 with the defect r as source
          CUDA_TRY(c, cudaMemsetAsync((float*)c->eps32.p + (size_t)i * nc * N, 0, (size_t)nc * N * sizeof(float), S.s));
          Ctrl cc = ctl[i];
          cc.state = kRunning;
          cc.stop_rule = 0;
          cc.tol = 0.5 * o->tol;  // the estimate's FP32 error stays well below tol / 2 (FP64 certifies)
          cc.switch_mode = 1;
          cc.stall_window = 32;
          cc.stall = 0;
          cc.best = INFINITY;
          cc.phase_it = 0;
          cc.phase_max = 0;
          for (int k = 0; k < 6; ++k) {
            cc.off_sig[k] = ctl[i].last_ms[k];
            cc.off_eps[k] = ctl[i].last_me[k];
          }
          init[i] = cc;
          any = true;
        }
        if (!any) break;
        if ((st = R32.run(init.data(), false, true, direct ? kUpdCorrDirect : kUpdCorrAccel))) return st;
        any = false;
        for (int i = 0; i < ns; ++i) {
          if (!active[i]) continue;
          it32[i] += hctl[i].it - ctl[i].it;
          take(i);
          CUDA_TRY(c, launch_add_correction((double*)c->eps64.p + (size_t)i * nc * N,
                                            (const float*)c->eps32.p + (size_t)i * nc * N, (long long)nc * N, S.s));
          c->launches += 1;
          if (state[i] == kDiverged) { active[i] = 0; continue; }
          if (state[i] != kSwitch) { state[i] = kStopped; active[i] = 0; continue; }  // max_iter inside the correction
          state[i] = kRunning;
          any = true;
        }
      }
      for (int i = 0; i < ns; ++i)
        if (state[i] == kRunning) state[i] = kStopped;
    }
  }
  // outputs from the final fields
  const int sblocks = (int)std::min<long long>((N + 255) / 256, (long long)c->num_sms * 8);
  CUDA_TRY(c, c->part_mean.ensure((size_t)sblocks * 2 * nc * sizeof(double)));
  CUDA_TRY(c, c->sums.ensure((size_t)std::max(ns, 1) * 2 * nc * sizeof(double)));
  std::vector<double> hs((size_t)ns * 2 * nc);
  fftls_status worst = FFTLS_OK;
  for (int i = 0; i < ns; ++i) {
    fftls_result* r = R[i];
    const Ctrl fin = ctl[i];
    const bool o64 = final64[i];  // else the FP32 field (FP32, or a ladder sample stopped in its FP32 phase)
    const void* epsf = o64 ? (const void*)((const double*)c->eps64.p + (size_t)i * nc * N)
                           : (const void*)((const float*)c->eps32.p + (size_t)i * nc * N);
    const uint8_t* ph = S.d_phase + (size_t)i * N;
    double* stress_dev = nullptr;
    if (r->stress) {
      if (o->fields_on_device) stress_dev = r->stress;
      else {
        CUDA_TRY(c, c->scratch.ensure((size_t)nc * N * sizeof(double)));
        stress_dev = (double*)c->scratch.p;
      }
    }
    if (o64)
      CUDA_TRY(c, launch_stress<double>((const double*)epsf, ph, (const double*)c->coef64.p + (size_t)(ns > 1 ? i : 0) * 256 * kCoef,
                                        d, N, stress_dev, (double*)c->part_mean.p, sblocks, S.s));
    else
      CUDA_TRY(c, launch_stress<float>((const float*)epsf, ph, (const float*)c->coef32.p + (size_t)(ns > 1 ? i : 0) * 256 * kCoef,
                                       d, N, stress_dev, (double*)c->part_mean.p, sblocks, S.s));
    CUDA_TRY(c, launch_sum_parts((const double*)c->part_mean.p, sblocks, 2 * nc, (double*)c->sums.p + (size_t)i * 2 * nc, S.s));
    c->launches += 2;
    if (r->stress && !o->fields_on_device)
      CUDA_TRY(c, cudaMemcpyAsync(r->stress, stress_dev, (size_t)nc * N * sizeof(double), cudaMemcpyDeviceToHost, S.s));
    if (r->strain) {
      const cudaMemcpyKind kind = o->fields_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
      if (o64) {
        CUDA_TRY(c, cudaMemcpyAsync(r->strain, epsf, (size_t)nc * N * sizeof(double), kind, S.s));
      } else if (o->fields_on_device) {
        CUDA_TRY(c, launch_convert<double, float>(r->strain, (const float*)epsf, (long long)nc * N, S.s));
      } else {
        CUDA_TRY(c, c->scratch.ensure((size_t)nc * N * sizeof(double)));
        CUDA_TRY(c, launch_convert<double, float>((double*)c->scratch.p, (const float*)epsf, (long long)nc * N, S.s));
        CUDA_TRY(c, cudaMemcpyAsync(r->strain, c->scratch.p, (size_t)nc * N * sizeof(double), kind, S.s));
      }
    }
    const int hl = std::min(fin.it, r->history_capacity);
    if (r->eta_history && hl > 0)
      CUDA_TRY(c, cudaMemcpyAsync(r->eta_history, (const double*)c->eta_hist.p + (size_t)i * o->max_iter,
                                  (size_t)hl * sizeof(double), cudaMemcpyDeviceToHost, S.s));
    if (r->mean_stress_history && hl > 0) {
      // one sample's history: [it][nc] at its slice (per-sample stride max_iter x 6 in a group)
      const double* src = (const double*)c->ms_hist.p + (size_t)i * o->max_iter * (ns > 1 ? 6 : nc);
      CUDA_TRY(c, cudaMemcpyAsync(r->mean_stress_history, src, (size_t)hl * nc * sizeof(double), cudaMemcpyDeviceToHost, S.s));
    }
    CUDA_TRY(c, cudaStreamSynchronize(S.s));  // scratch is reused by the next sample
    r->iterations = fin.it;
    r->iterations_fp32 = it32[i];
    r->final_eta = fin.last_eta;
    r->final_delta = fin.last_delta;
    r->history_len = hl;
    stat[i] = state[i] == kConverged ? FFTLS_OK : state[i] == kDiverged ? FFTLS_E_DIVERGED : FFTLS_E_NOT_CONVERGED;
    if (stat[i] != FFTLS_OK && worst == FFTLS_OK) worst = stat[i];
  }
  CUDA_TRY(c, cudaMemcpyAsync(hs.data(), c->sums.p, hs.size() * sizeof(double), cudaMemcpyDeviceToHost, S.s));
  CUDA_TRY(c, cudaStreamSynchronize(S.s));
  for (int i = 0; i < ns; ++i)
    for (int k = 0; k < 6; ++k) {
      R[i]->mean_stress[k] = k < nc ? hs[(size_t)i * 2 * nc + k] / (double)N : 0.0;
      R[i]->mean_strain[k] = k < nc ? hs[(size_t)i * 2 * nc + nc + k] / (double)N : 0.0;
    }
  return FFTLS_OK;
}

static fftls_status solve_impl(fftls_ctx* c, const fftls_problem* p, const fftls_options* o, fftls_result* r) {
  fftls_status st = FFTLS_OK;
  const fftls_status e = solve_core(c, &p, 1, o, &r, &st);
  if (e != FFTLS_OK) return e;
  const Ctrl fin = c->h_ctrl[0];
  (void)fin;
  if (st == FFTLS_OK) return FFTLS_OK;
  if (st == FFTLS_E_DIVERGED)
    return set_err(c, FFTLS_E_DIVERGED, "diverged: eta = %g after %d iterations", r->final_eta, r->iterations);
  return set_err(c, FFTLS_E_NOT_CONVERGED, "not converged after %d iterations (eta = %g)", r->iterations, r->final_eta);
}

fftls_status fftls_solve(fftls_ctx* c, const fftls_problem* p, const fftls_options* o, fftls_result* r) {
  if (!c) return FFTLS_E_INVALID_ARG;
  c->err.clear();
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(c->device) != cudaSuccess) return set_err(c, FFTLS_E_CUDA, "cannot select device %d", c->device);
  fftls_status s = solve_impl(c, p, o, r);
  cudaSetDevice(prev);
  return s;
}

fftls_status fftls_solve_batched(fftls_ctx* c, const fftls_problem* probs, int count, const fftls_options* o,
                                 fftls_result* results, fftls_status* statuses, int concurrency) {
  if (!c) return FFTLS_E_INVALID_ARG;
  c->err.clear();
  if (count < 0 || (count > 0 && (!probs || !o || !results)))
    return set_err(c, FFTLS_E_INVALID_ARG, "batched solve: null arrays or negative count");
  if (count == 0) return FFTLS_OK;
  if (o->eps_init) return set_err(c, FFTLS_E_INVALID_ARG, "batched solve: eps_init must be NULL");
  if (concurrency < 0 || concurrency > kMaxWorkers)
    return set_err(c, FFTLS_E_INVALID_ARG, "batched solve: concurrency must be in 0..%d", kMaxWorkers);
  const int nw = std::min(concurrency > 0 ? concurrency : kDefaultWorkers, count);
  while ((int)c->workers.size() < nw) {
    fftls_ctx* w = nullptr;
    const fftls_status s = fftls_create(&w, c->device);
    if (s != FFTLS_OK) return set_err(c, s, "batched solve: cannot create worker context");
    w->plans = c->plans;
    c->workers.push_back(w);
  }
  if (o->stream) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    const cudaError_t e = cudaStreamSynchronize((cudaStream_t)o->stream);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return set_err(c, FFTLS_E_CUDA, "batched solve: %s", cudaGetErrorString(e));
  }
  // Tasks: 3D samples that share a grid, operator and scheme form groups solved by
  // grouped launches (solve_core, at most kGroupBytes of device memory per group);
  // every other sample is a task of its own.  Largest tasks first (longest-
  // processing-time order balances the workers).
  std::vector<std::vector<int>> tasks;
  std::vector<fftls_status> st(count, FFTLS_OK);
  std::vector<std::string> msg(count);
  {
    std::vector<int> order;
    for (int i = 0; i < count; ++i) {  // invalid samples are reported, never grouped or run
      fftls_ctx vc;
      const fftls_status vs = validate(&vc, &probs[i], o);
      if (vs != FFTLS_OK) {
        st[i] = vs;
        msg[i] = vc.err;
      } else {
        order.push_back(i);
      }
    }
    const int nvalid = (int)order.size();
    auto key_less = [&](int x, int y) {
      const fftls_problem &a = probs[x], &b = probs[y];
      if (a.dim != b.dim) return a.dim < b.dim;
      for (int k = 0; k < 3; ++k)
        if (a.n[k] != b.n[k]) return a.n[k] < b.n[k];
      if (a.green != b.green) return a.green < b.green;
      return a.scheme < b.scheme;
    };
    std::stable_sort(order.begin(), order.end(), key_less);
    for (int k = 0; k < nvalid;) {
      int e = k + 1;
      while (e < nvalid && !key_less(order[k], order[e]) && !key_less(order[e], order[k])) ++e;
      const fftls_problem& q = probs[order[k]];
      const long long vox = (long long)q.n[0] * q.n[1] * q.n[2];
      const int per = q.dim == 3 ? (int)std::max<long long>(1, std::min<long long>(kMaxGroup, kGroupBytes / (kGroupBytesPerVoxel * vox))) : 1;
      for (int b = k; b < e; b += per) tasks.emplace_back(order.begin() + b, order.begin() + std::min(e, b + per));
      k = e;
    }
    auto work_of = [&](const std::vector<int>& t) {
      return (long long)t.size() * probs[t[0]].n[0] * probs[t[0]].n[1] * probs[t[0]].n[2];
    };
    std::stable_sort(tasks.begin(), tasks.end(), [&](const std::vector<int>& x, const std::vector<int>& y) {
      return work_of(x) > work_of(y);
    });
  }
  fftls_options wo = *o;
  wo.stream = nullptr;  // each worker runs on its own stream
  std::atomic<int> next(0);
  std::vector<long long> k0(nw), g0(nw);
  for (int t = 0; t < nw; ++t) {
    k0[t] = c->workers[t]->launches;
    g0[t] = c->workers[t]->graph_launches;
  }
  const int ntask = (int)tasks.size();
  auto work = [&](fftls_ctx* w) {
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= ntask) break;
      const std::vector<int>& t = tasks[k];
      if (t.size() == 1) {
        const int i = t[0];
        st[i] = fftls_solve(w, &probs[i], &wo, &results[i]);
        if (st[i] != FFTLS_OK) msg[i] = w->err;
        continue;
      }
      std::vector<const fftls_problem*> P(t.size());
      std::vector<fftls_result*> Rp(t.size());
      std::vector<fftls_status> sst(t.size(), FFTLS_OK);
      for (size_t j = 0; j < t.size(); ++j) {
        P[j] = &probs[t[j]];
        Rp[j] = &results[t[j]];
      }
      int prev = 0;
      cudaGetDevice(&prev);
      cudaSetDevice(w->device);
      w->err.clear();
      const fftls_status e = solve_core(w, P.data(), (int)t.size(), &wo, Rp.data(), sst.data());
      cudaSetDevice(prev);
      for (size_t j = 0; j < t.size(); ++j) {
        st[t[j]] = e != FFTLS_OK ? e : sst[j];
        if (st[t[j]] != FFTLS_OK)
          msg[t[j]] = e != FFTLS_OK ? w->err : std::string(sst[j] == FFTLS_E_DIVERGED ? "diverged" : "not converged");
      }
    }
  };
  std::vector<std::thread> pool;
  pool.reserve(nw);
  for (int t = 0; t < nw; ++t) pool.emplace_back(work, c->workers[t]);
  for (auto& t : pool) t.join();
  for (int t = 0; t < nw; ++t) {
    fftls_ctx* w = c->workers[t];
    c->launches += w->launches - k0[t];
    c->graph_launches += w->graph_launches - g0[t];
    for (auto& kv : w->plans) {
      bool have = false;
      for (auto& mine : c->plans)
        if (mine.first == kv.first) {
          have = true;
          if (kv.second.tuned && !mine.second.tuned) mine.second = kv.second;
        }
      if (!have) c->plans.push_back(kv);
    }
  }
  fftls_status worst = FFTLS_OK;
  for (int i = 0; i < count; ++i) {
    if (statuses) statuses[i] = st[i];
    if (st[i] != FFTLS_OK && worst == FFTLS_OK) {
      worst = st[i];
      set_err(c, worst, "sample %d: %s", i, msg[i].c_str());
    }
  }
  return worst;
}

fftls_status fftls_effective_stiffness(fftls_ctx* c, const fftls_problem* p, const fftls_options* o, double* C_eff,
                                       int* iterations) {
  if (!c || !p || !o || !C_eff) return set_err(c, FFTLS_E_INVALID_ARG, "null argument");
  if (p->dim != 2 && p->dim != 3) return set_err(c, FFTLS_E_INVALID_ARG, "dim must be 2 or 3");
  const int nc = ncomp(p->dim);
  fftls_problem q = *p;
  fftls_status worst = FFTLS_OK;
  for (int J = 0; J < nc; ++J) {
    mandel_unit(p->dim, J, q.eps_bar);
    fftls_result r;
    memset(&r, 0, sizeof(r));
    fftls_status s = fftls_solve(c, &q, o, &r);
    if (s != FFTLS_OK && s != FFTLS_E_NOT_CONVERGED && s != FFTLS_E_DIVERGED) return s;
    if (s != FFTLS_OK && worst == FFTLS_OK) worst = s;
    for (int I = 0; I < nc; ++I) C_eff[I * nc + J] = r.mean_stress[I] * (I < p->dim ? 1.0 : sqrt(2.0));
    if (iterations) iterations[J] = r.iterations;
  }
  return worst;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free solve (fftls_solve_noalloc).  The paper has no counterpart:
// this serves callers that cannot call cudaMalloc (applications whose device
// memory is reserved up front and handed out by their own allocator).  All
// scratch lives in one file-scope device array.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;  // 16 MiB, held by every device that loads the library
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
constexpr int kNoAllocMaxDevices = 64;
void* g_noalloc_base[kNoAllocMaxDevices];  // device address of g_noalloc_scratch per device (set up on first call)

// host staging for the tables (fixed size: no heap allocation), shared by every
// device: g_na_lock serialises building them and issuing their copies (a
// cudaMemcpyAsync from pageable memory returns once the source has been staged,
// so the arrays are free again when the lock is released)
std::mutex g_na_lock;
double g_na_coef[256 * kCoef];
double g_na_tab[3 * (2 * (kMaxL + 2) + 8 * kMaxL)];
int g_na_perm[6 * kMaxL];

size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" fftls_status fftls_solve_noalloc(const fftls_problem* p, const fftls_options* o, fftls_result* r) {
#define NA_TRY(...)                                        \
  do {                                                     \
    if ((__VA_ARGS__) != cudaSuccess) return FFTLS_E_CUDA; \
  } while (0)
  fftls_status st = validate(nullptr, p, o);
  if (st) return st;
  if (!r || !r->strain || !o->fields_on_device || o->precision != FFTLS_FP64) return FFTLS_E_INVALID_ARG;
  int dev = 0;
  NA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return FFTLS_E_CUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_lock);
    if (!g_noalloc_base[dev]) {  // set-up, once per device, with that device current
      void* b = nullptr;
      NA_TRY(cudaGetSymbolAddress(&b, g_noalloc_scratch));
      g_noalloc_base[dev] = b;
    }
    base = (unsigned char*)g_noalloc_base[dev];
  }
  Setup S;
  memset(&S, 0, sizeof(S));
  setup_geometry(S, p);
  const int d = S.dim, nc = S.nc;
  S.s = (cudaStream_t)o->stream;
  const long long N = S.g.N;
  int v = 0;
  NA_TRY(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  S.smem_optin = v;
  NA_TRY(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
  S.num_sms = v;
  IterArgs<double> a;
  memset(&a, 0, sizeof(a));
  if (!apply_plan<double>(S, a, false, default_plan(S, sizeof(double2), false))) return FFTLS_E_UNSUPPORTED_SIZE;
  // scratch layout
  const int ntz = (S.g.H + a.z_w - 1) / a.z_w;
  const int sblocks = (int)std::min<long long>((N + 255) / 256, (long long)S.num_sms * 8);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t at = off; off = na_align(off + bytes); return at; };
  const size_t o_specA = take((size_t)S.g.modes * nc * 16);
  const size_t o_specB = take((size_t)S.g.modes * nc * 16);
  const size_t o_pmean = take((size_t)std::max(a.x1_blocks, sblocks) * 2 * nc * 8);
  const size_t o_peta = take((size_t)ntz * S.g.n2 * 2 * 8);
  const size_t o_pdelta = take((size_t)a.x5_blocks * 2 * 8);
  const size_t o_sums = take(64 * 8);
  const size_t o_ctrl = take(sizeof(Ctrl));
  const size_t o_eh = take((size_t)o->max_iter * 8);
  const size_t o_mh = take((size_t)o->max_iter * nc * 8);
  const size_t o_coef = take(256 * kCoef * 8);
  const size_t ntab = table_count(S);
  const size_t o_tab = take(ntab * 8);
  const size_t nperm = 2 * (size_t)(S.g.n1 + S.g.n2 + S.g.n3);
  const size_t o_perm = take(nperm * sizeof(int));
  const size_t o_phase = p->phase_on_device ? 0 : take((size_t)N);
  if (off > kNoAllocScratchBytes) return FFTLS_E_UNSUPPORTED_SIZE;  // grid too large for the fixed scratch
  // tables (host staging arrays, no heap), built and copied under the staging lock
  size_t po = 0;
  {
    std::lock_guard<std::mutex> lk(g_na_lock);
    coef_table(S, p, g_na_coef);
    NA_TRY(cudaMemcpyAsync(base + o_coef, g_na_coef, sizeof(g_na_coef), cudaMemcpyHostToDevice, S.s));
    fill_tables(S, g_na_tab, g_na_perm);
    NA_TRY(cudaMemcpyAsync(base + o_tab, g_na_tab, ntab * 8, cudaMemcpyHostToDevice, S.s));
    NA_TRY(cudaMemcpyAsync(base + o_perm, g_na_perm, nperm * sizeof(int), cudaMemcpyHostToDevice, S.s));
  }
  // phase image (copied into the scratch when it is on the host) and its id check
  const uint8_t* d_phase = p->phase;
  if (!p->phase_on_device) {
    NA_TRY(cudaMemcpyAsync(base + o_phase, p->phase, (size_t)N, cudaMemcpyHostToDevice, S.s));
    d_phase = base + o_phase;
  }
  S.d_phase = d_phase;
  unsigned int pmax = 0;
  NA_TRY(launch_phase_max(d_phase, N, (unsigned int*)(base + o_sums), sblocks, S.s));
  NA_TRY(cudaMemcpyAsync(&pmax, base + o_sums, sizeof(pmax), cudaMemcpyDeviceToHost, S.s));
  NA_TRY(cudaStreamSynchronize(S.s));
  if ((int)pmax >= p->n_phases) return FFTLS_E_INVALID_ARG;
  // the iterate lives in the caller's strain buffer
  double* eps = r->strain;
  if (o->eps_init)
    NA_TRY(cudaMemcpyAsync(eps, o->eps_init, (size_t)nc * N * 8,
                           o->eps_init_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, S.s));
  else
    NA_TRY(launch_fill_eps<double>(eps, nc, N, S.eps_bar, S.s));
  a.g = S.g;
  a.dim = d;
  a.green = S.green;
  for (int ax = 0; ax < 3; ++ax) a.pl[ax] = S.pl[ax];
  a.lam0 = S.lam0;
  a.mu0 = S.mu0;
  for (int i = 0; i < 6; ++i) a.eps_bar[i] = S.eps_bar[i];
  a.eps = eps;
  a.phase = d_phase;
  a.coef = (const double*)(base + o_coef);
  a.specA = (double2*)(base + o_specA);
  a.specB = (double2*)(base + o_specB);
  po = 0;
  for (int ax = 0; ax < 3; ++ax) {
    a.tw[ax] = (const double2*)((const double*)(base + o_tab) + table_offset_tw(S, ax));
    a.kt[ax] = (const KTab<double>*)((const double*)(base + o_tab) + table_offset_kt(S, ax));
    a.rd[ax] = (const double2*)((const double*)(base + o_tab) + table_offset_rd(S, ax));
    a.perm[ax] = (const int*)(base + o_perm) + po;
    a.pos[ax] = (const int*)(base + o_perm) + po + S.pl[ax].L;
    po += 2 * (size_t)S.pl[ax].L;
  }
  a.ctrl = (Ctrl*)(base + o_ctrl);
  a.part_mean = (double*)(base + o_pmean);
  a.part_eta = (double*)(base + o_peta);
  a.part_delta = (double*)(base + o_pdelta);
  a.eta_hist = (double*)(base + o_eh);
  a.ms_hist = (double*)(base + o_mh);
  a.want_delta = o->stop == FFTLS_STOP_MAXDELTA ? 1 : 0;
  NA_TRY(set_kernel_attributes<double>(a, (size_t)S.smem_optin - 4096));
  const bool direct = p->scheme == FFTLS_DIRECT;
  Ctrl ctl;
  memset(&ctl, 0, sizeof(ctl));
  ctl.state = kRunning;
  ctl.max_it = o->max_iter;
  ctl.stop_rule = o->stop;
  ctl.tol = o->tol;
  ctl.mean_guard = (direct || o->eta_only) ? 0 : 1;
  ctl.best = INFINITY;
  NA_TRY(cudaMemcpyAsync(a.ctrl, &ctl, sizeof(Ctrl), cudaMemcpyHostToDevice, S.s));
  auto iteration = [&](bool dual, int update) -> cudaError_t {
    a.dual = dual ? 1 : 0;
    a.tauform = a.dual;
    a.update = update;
    cudaError_t e;
    if ((e = launch_fwd_x<double>(a, S.s)) != cudaSuccess) return e;
    if ((e = launch_mid_y<double>(a, false, S.s)) != cudaSuccess) return e;
    if ((e = launch_fourier_z<double>(a, S.s)) != cudaSuccess) return e;
    if ((e = launch_reduce_eta<double>(a, S.s)) != cudaSuccess) return e;
    if ((e = launch_mid_y<double>(a, true, S.s)) != cudaSuccess) return e;
    if ((e = launch_inv_x<double>(a, S.s)) != cudaSuccess) return e;
    if (a.want_delta && (e = launch_reduce_delta<double>(a, S.s)) != cudaSuccess) return e;
    return cudaSuccess;
  };
  const bool dual = !direct;
  const int upd = direct ? kUpdDirectSig : kUpdAccel;
  if (direct && o->eps_init) NA_TRY(iteration(true, kUpdDirectTau));
  const int chunk = (int)std::max<long long>(1, std::min<long long>(32, 40000000LL / std::max<long long>(N, 1)));
  for (;;) {
    NA_TRY(cudaMemcpyAsync(&ctl, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, S.s));
    NA_TRY(cudaStreamSynchronize(S.s));
    if (ctl.fault) return FFTLS_E_TIMEOUT;  // a tile copy did not complete within its wait limit
    if (ctl.state != kRunning) break;
    for (int i = 0; i < chunk; ++i) NA_TRY(iteration(dual, upd));
  }
  // outputs
  double* part = (double*)(base + o_pmean);
  double* sums = (double*)(base + o_sums);
  NA_TRY(launch_stress<double>(eps, d_phase, a.coef, d, N, r->stress, part, sblocks, S.s));
  NA_TRY(launch_sum_parts(part, sblocks, 2 * nc, sums, S.s));
  double hs[12];
  NA_TRY(cudaMemcpyAsync(hs, sums, 2 * nc * sizeof(double), cudaMemcpyDeviceToHost, S.s));
  const int hl = std::min(ctl.it, r->history_capacity);
  if (r->eta_history && hl > 0)
    NA_TRY(cudaMemcpyAsync(r->eta_history, a.eta_hist, (size_t)hl * 8, cudaMemcpyDeviceToHost, S.s));
  if (r->mean_stress_history && hl > 0)
    NA_TRY(cudaMemcpyAsync(r->mean_stress_history, a.ms_hist, (size_t)hl * nc * 8, cudaMemcpyDeviceToHost, S.s));
  NA_TRY(cudaStreamSynchronize(S.s));
  for (int i = 0; i < 6; ++i) {
    r->mean_stress[i] = i < nc ? hs[i] / (double)N : 0.0;
    r->mean_strain[i] = i < nc ? hs[nc + i] / (double)N : 0.0;
  }
  r->iterations = ctl.it;
  r->iterations_fp32 = 0;
  r->final_eta = ctl.last_eta;
  r->final_delta = ctl.last_delta;
  r->history_len = hl;
  if (ctl.state == kConverged) return FFTLS_OK;
  if (ctl.state == kDiverged) return FFTLS_E_DIVERGED;
  return FFTLS_E_NOT_CONVERGED;
#undef NA_TRY
}
