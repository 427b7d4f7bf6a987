/*
 * fftls.h - C ABI of the GB300 (sm_103a) FFT Lippmann-Schwinger solver for
 * periodic 2D/3D voxel composites in linear elasticity, after
 * F. Willot, "Fourier-based schemes for computing the mechanical response of
 * composites with accurate local fields" (arXiv:1412.8398).
 *
 * Problem (Sec. 2, eq. a1-a2): on a periodic grid of n1 x n2 x n3 voxels
 * (n3 = 1 in 2D), each voxel holds a phase id; each phase is isotropic with
 * Lame coefficients (lambda, mu), C = lambda dd + mu (dd + dd).  Given the
 * macroscopic strain eps_bar, find the strain eps(x) with <eps> = eps_bar,
 * discrete compatibility and equilibrium (Sec. 4, eq. discFour) under one of
 * four discrete Green operators:
 *   FFTLS_GREEN_MS : G of Moulinec and Suquet, k = i q (eq. green0b) with the
 *                    even-L rule G = C0^{-1} at q_i = pi (eq. hfreq);
 *   FFTLS_GREEN_C  : centered differences, k_i = i sin q_i (eq. mul2, mulfix);
 *   FFTLS_GREEN_W  : forward/backward differences, k_i = e^{iq_i} - 1 (eq. wil072);
 *   FFTLS_GREEN_R  : the paper's rotated scheme, k^R of eq. wil14 (2D) /
 *                    wil14b (3D), G^R = 0 where k^R = 0 (eq. mysymgr).
 * Schemes: FFTLS_DIRECT (eq. ds) and FFTLS_ACCELERATED (eq. as), iterated
 * until the equilibrium norm eta of eq. criterion is <= tol.
 *
 * Conventions
 *  - Fields are structure-of-arrays, component-major: component c of voxel
 *    v = x1 + n1 (x2 + n2 x3) is at [c * N + v], N = n1 n2 n3.  Components
 *    are tensor components (not engineering shear) in the order
 *    11, 22, 33, 23, 13, 12 (3D) or 11, 22, 12 (2D): n_c = 6 or 3.
 *  - eta = sqrt(sum_q |k*(q) . sigma_hat(q)|^2) / (N ||<sigma>||_F), with the
 *    unnormalised DFT of eq. ft2, ||.||_F counting off-diagonal entries twice,
 *    0/0 = 0.  Under FFTLS_ACCELERATED the eta test also requires
 *    |<eps> - eps_bar|_F <= tol |eps_bar|_F (accelerated iterates need not
 *    have the prescribed mean).
 *  - `iterations` counts evaluations of eta, i.e. stresses sigma^k computed.
 *    A homogeneous medium returns 1.
 *  - All buffers are owned by the caller.  The context owns its device
 *    workspaces and reuses them across calls.  Calls on one context must not
 *    overlap; each call is synchronous with respect to the host.
 *  - No C++ exception crosses the ABI.  On error the call returns a status
 *    and fftls_last_error() holds a message for that context.
 */
#ifndef FFTLS_H
#define FFTLS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fftls_ctx fftls_ctx;

typedef enum {
  FFTLS_OK = 0,
  FFTLS_E_INVALID_ARG = 1,      /* bad dimension, size, moduli, enum or pointer */
  FFTLS_E_UNSUPPORTED_SIZE = 2, /* a length with a prime factor other than 2, 3, 5, or > 2048; tiles too large */
  FFTLS_E_OOM = 3,              /* device allocation failed */
  FFTLS_E_CUDA = 4,             /* a CUDA runtime call failed (message in fftls_last_error) */
  FFTLS_E_NOT_CONVERGED = 5,    /* max_iter reached; outputs hold the last iterate */
  FFTLS_E_DIVERGED = 6,         /* eta non-finite or > 1e4 eta_0; outputs hold the last iterate */
  FFTLS_E_TIMEOUT = 7           /* a bounded device wait ran out (a shared-memory tile copy that did not
                                   complete): the kernels stopped the solve; the context stays usable */
} fftls_status;

enum { FFTLS_GREEN_MS = 0, FFTLS_GREEN_C = 1, FFTLS_GREEN_W = 2, FFTLS_GREEN_R = 3 };
enum { FFTLS_DIRECT = 0, FFTLS_ACCELERATED = 1 };
/* FP64: every pass in double.  FP32_REFINE64: FFT passes, G' and the
 * constitutive update in float with FP64 reductions until eta <= refine_switch
 * (or eta stalls), then double until eta <= tol.  FP32: float only. */
enum { FFTLS_FP64 = 0, FFTLS_FP32_REFINE64 = 1, FFTLS_FP32 = 2 };
/* ETA: eq. criterion.  MAXDELTA: max over voxels and components of
 * |eps^{k+1} - eps^k| and |sigma^{k+1} - sigma^k| below tol (Sec. 5.1, 5.3);
 * the field returned is eps^{k+1} and `iterations` = k + 1. */
enum { FFTLS_STOP_ETA = 0, FFTLS_STOP_MAXDELTA = 1 };

typedef struct {
  int dim;                  /* 2 or 3 */
  int n[3];                 /* n1 (x1, fastest), n2, n3; n3 = 1 when dim == 2; each in 1..2048, factors 2,3,5.
                               The tiles must also fit in shared memory: in FP64 (and the ladder's FP64
                               passes) a 3D grid needs n2, n3 <= 2000 and, for G, n1 <= 1600 (so 2048 fits
                               in 2D and along x1 of 3D G^C/W/R only); else FFTLS_E_UNSUPPORTED_SIZE */
  const uint8_t* phase;     /* N phase ids in 0..n_phases-1, x1 fastest */
  int phase_on_device;      /* 1: `phase` is a device pointer on the context's device */
  int n_phases;             /* 1..256 */
  const double* lambda;     /* host, [n_phases]; 2D uses these (plane strain) values directly */
  const double* mu;         /* host, [n_phases]; mu >= 0, lambda + (2/d) mu >= 0 */
  double lambda0, mu0;      /* reference medium; NaN selects the default (fftls_reference_medium) */
  int green;                /* FFTLS_GREEN_* */
  int scheme;               /* FFTLS_DIRECT or FFTLS_ACCELERATED */
  double eps_bar[6];        /* macroscopic strain, tensor components in field order */
} fftls_problem;

typedef struct {
  double tol;               /* eta (or max-delta) tolerance, >= 0 */
  int stop;                 /* FFTLS_STOP_* */
  int max_iter;             /* >= 1; caps `iterations` over all precision phases */
  int precision;            /* FFTLS_FP64, FFTLS_FP32_REFINE64, FFTLS_FP32 */
  double refine_switch;     /* FP32_REFINE64: eta at which float hands over to double; <= 0 selects max(tol, 3e-5) */
  const double* eps_init;   /* optional initial strain (n_c x N, FP64); NULL starts from eps_bar */
  int eps_init_on_device;   /* 1: eps_init is a device pointer */
  int fields_on_device;     /* 1: result->strain / stress are device pointers */
  void* stream;             /* cudaStream_t to run on; NULL uses the context's own stream */
  int use_graphs;           /* 1 (default): capture chunks of iterations as CUDA graphs */
  int profile;              /* 1: time every kernel with CUDA events (no graphs); see fftls_profile */
  int autotune;             /* 1 (default): on the first solve of a grid, operator and precision on this
                               context, time candidate tile schedules of every kernel on the device and keep
                               the fastest (see fftls_tile_plans); 0: built-in schedule.  The schedule changes
                               no per-line or per-mode arithmetic, only the grouping of partial sums. */
  int eta_only;             /* 0 (default): the accelerated scheme's eta test also requires
                               |<eps> - eps_bar|_F <= tol |eps_bar|_F (its iterates need not have mean
                               eps_bar); 1: eta <= tol alone, the paper's criterion (eq. criterion) */
} fftls_options;

typedef struct {
  double* strain;               /* optional out, n_c x N FP64 (host or device, see fields_on_device) */
  double* stress;               /* optional out, n_c x N FP64 */
  double mean_stress[6];        /* <sigma> of the returned field */
  double mean_strain[6];        /* <eps> of the returned field */
  int iterations;               /* eta evaluations, all phases */
  int iterations_fp32;          /* of which in float */
  double final_eta;             /* last eta evaluated */
  double final_delta;           /* last max |delta| (MAXDELTA stop), else 0 */
  double* eta_history;          /* optional out (host), [history_capacity] */
  double* mean_stress_history;  /* optional out (host), [history_capacity x n_c] */
  int history_capacity;         /* entries available in the two histories */
  int history_len;              /* entries written (= iterations, capped by capacity) */
} fftls_result;

/* Fill *opt with defaults: tol 1e-8, STOP_ETA, max_iter 1000, FP64, graphs on. */
void fftls_default_options(fftls_options* opt);

/* Create a context on CUDA device `device`.  Returns FFTLS_E_CUDA if the
 * device cannot be used. */
fftls_status fftls_create(fftls_ctx** ctx, int device);

/* Free every device workspace and graph of the context.  NULL is ignored. */
void fftls_destroy(fftls_ctx* ctx);

/* Solve one load case (Sec. 3, eq. ds / eq. as with the chosen operator of Sec. 4).
 * Returns FFTLS_OK, FFTLS_E_NOT_CONVERGED or FFTLS_E_DIVERGED with the outputs
 * filled, or an error status with the outputs untouched (FFTLS_E_TIMEOUT when a
 * kernel's bounded wait for a tile copy ran out). */
fftls_status fftls_solve(fftls_ctx* ctx, const fftls_problem* prob, const fftls_options* opt, fftls_result* res);

/* Effective stiffness C~ from <sigma> = C~ eps_bar (Sec. 2), as a symmetric
 * Mandel matrix (shear rows and columns scaled by sqrt 2), n_c x n_c row-major
 * in the first n_c^2 entries of C_eff.  Runs n_c unit Mandel loads; prob->eps_bar
 * is ignored.  iterations[n_c] (optional) receives each solve's count. */
fftls_status fftls_effective_stiffness(fftls_ctx* ctx, const fftls_problem* prob, const fftls_options* opt,
                                       double* C_eff, int* iterations);

/* Allocation-free solve.  The paper has no counterpart: this entry point is
 * for callers that must not allocate device memory, typically an application
 * that reserves its GPU memory once at start-up and hands it out from its own
 * fixed pools (a long-running service with a hard memory budget, or a host
 * framework whose plug-ins may not call cudaMalloc behind its allocator's
 * back).  It makes no cudaMalloc / cudaFree call, creates no context, stream,
 * event or graph, and needs no fftls_ctx.
 *  - Scratch (spectrum, partial sums, control block, tables, histories and a
 *    copy of a host phase image) lives in one file-scope device array of
 *    16 MiB, which every GPU that loads the library holds until the process
 *    exits.  A problem that needs more (2 n_c complex doubles per half-spectrum
 *    mode dominate: about 40^3 voxels in 3D, 256^2 in 2D) is rejected with
 *    FFTLS_E_UNSUPPORTED_SIZE before anything runs.
 *  - Runs on the caller's current device and on opt->stream (NULL: the legacy
 *    default stream).  The first call on a device looks up the array's device
 *    address (cudaGetSymbolAddress) with that device current.
 *  - The call blocks the host: it copies a host phase image and the tables in
 *    with cudaMemcpyAsync, synchronises opt->stream after every chunk of
 *    iterations to read the solver's control block back, and copies the mean
 *    fields and the histories to the host before it returns.
 *  - FP64 only (opt->precision must be FFTLS_FP64); no profiling.
 *  - opt->fields_on_device must be 1 and res->strain a device buffer of
 *    n_c x N doubles: the iterate lives there.  res->stress (device) and the
 *    host histories are optional.
 *  - Every call on a device shares that device's array and leaves its
 *    contents behind; calls that overlap on one GPU (two host threads, or two
 *    streams) race and give wrong results.  Calls on different GPUs use
 *    different arrays; the host-side staging of their tables is serialised by
 *    a lock, so they may run from different host threads.  Returns the
 *    statuses of fftls_solve; no error message is kept (there is no context). */
fftls_status fftls_solve_noalloc(const fftls_problem* prob, const fftls_options* opt, fftls_result* res);

/* Default reference medium (lambda0, mu0) for prob->scheme: eq. refAcc for the
 * accelerated scheme (kappa0 = sqrt(k_min k_max), mu0 = sqrt(mu_min mu_max)),
 * eq. ref with beta = 1/2 for the direct scheme; kappa = lambda + (2/d) mu.
 * FFTLS_E_INVALID_ARG if the default degenerates (mu0 <= 0 or kappa0 <= 0). */
fftls_status fftls_reference_medium(const fftls_problem* prob, double* lambda0, double* mu0);

/* FFTLS_OK if the GPU transforms support a grid length L. */
fftls_status fftls_supported_length(int L);

/* Per-kernel device time of the last fftls_solve run with opt->profile = 1.
 * names[i] (static strings), total_ms[i], launches[i] for i < *count;
 * *count is the capacity on entry and the number of kernels on return. */
fftls_status fftls_profile(const fftls_ctx* ctx, const char** names, double* total_ms, int* launches, int* count);

/* Solves `count` independent problems (any mix of supported grid sizes, each
 * with its own phases, moduli, reference medium, operator, scheme and eps_bar)
 * under the shared options `opt`.  opt->eps_init must be NULL; opt->stream, if
 * set, is synchronised before the work starts.  3D samples that share a grid,
 * an operator and a scheme are solved together: every kernel of the iteration
 * runs as one grouped launch over them (a sample's blocks read its own control
 * block, so each stops, switches precision and diverges on its own), in groups
 * of at most 256 samples and about 24 GB of device memory; every other sample
 * runs as fftls_solve.  The groups and single samples are spread over
 * `concurrency` worker contexts (0 selects 8, at most 64), each with its own
 * stream, device buffers, CUDA graphs and tile schedules, largest task first.
 * results[i] (caller-owned buffers as in fftls_solve) and statuses[i] (may be
 * NULL) are what fftls_solve would give: the same status, iteration counts and
 * fields (bit for bit with opt->autotune = 0), the eta and <sigma> histories to
 * within one unit in the last place.  Invalid samples are reported with their
 * own status and never run.  Returns FFTLS_OK when every sample converged, else
 * the first failing status in sample order, with the sample named in
 * fftls_last_error.  Blocks until all samples are done.  The paper solves one
 * problem at a time; batching serves many-sample studies (its Boolean-model
 * statistics). */
fftls_status fftls_solve_batched(fftls_ctx* ctx, const fftls_problem* probs, int count, const fftls_options* opt,
                                 fftls_result* results, fftls_status* statuses, int concurrency);

/* Tile schedules held by this context, one row of FFTLS_PLAN_FIELDS ints per grid,
 * operator and precision: {precision (0 float, 1 double), n1, n2, n3, green,
 * lines per batch of the forward x1 pass, voxels per thread it loads together
 * (0: each batch staged in shared memory by bulk copies, FP32 only),
 * lines per batch of the inverse x1 pass, modes per tile of the x2 pass, of the
 * x3 pass, x3-planes per block of the real-space eta kernel (0: not used),
 * 1 if tuned on the device else 0, threads per block of the x2 pass and of
 * the x3 pass (0: chosen from the tile size), how the inverse x1 pass reads eps
 * (1: loaded by the threads, 0: staged in shared memory by bulk copies, FP32)}.  Copies min(*count, held) rows into
 * `rows` (may be NULL when *count is 0) and returns the number held in *count.
 * The paper has no counterpart (an implementation detail of the GPU path). */
#define FFTLS_PLAN_FIELDS 15
fftls_status fftls_tile_plans(const fftls_ctx* ctx, int* rows, int* count);

/* Imports `count` rows in the layout of fftls_tile_plans (host memory, copied;
 * the caller keeps ownership): later solves on this context use each row's
 * schedule for its grid, operator and precision as it is, without tuning (a
 * row with n3 = 1 also serves the 2D problem on n1 x n2; a row with 0 planes
 * for the real-space eta kernel serves only the operators that do not use it).
 * Rows replace schedules held for the same key.  FFTLS_E_INVALID_ARG, with
 * nothing imported, for a row outside the values the tuner can choose (lines
 * 1..8, voxels per load 1, 2 or 4, or 0 for FP32 with n1 a multiple of 16,
 * inverse loads 1, or 0 on the same terms; widths 1..16, powers of two;
 * thread counts 0 or those of the width); a schedule that does not fit shared
 * memory makes the solve that would use it fail with FFTLS_E_UNSUPPORTED_SIZE.
 * Lets a caller reuse the schedules tuned once on another context (the
 * arithmetic of a solve does not depend on its schedule beyond the grouping
 * of partial sums). */
fftls_status fftls_set_tile_plans(fftls_ctx* ctx, const int* rows, int count);

/* Kernels launched on this context since creation (nodes of CUDA graphs
 * counted one by one, including kernels that exit early once the solve has
 * stopped) and the number of graph launches. */
fftls_status fftls_counters(const fftls_ctx* ctx, long long* kernel_launches, long long* graph_launches);

/* Message of the last error on this context ("" if none). */
const char* fftls_last_error(const fftls_ctx* ctx);

/* Static name of a status code. */
const char* fftls_status_string(fftls_status s);

#ifdef __cplusplus
}
#endif

#endif /* FFTLS_H */
