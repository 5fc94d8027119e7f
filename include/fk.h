/*
 * fk.h -- C-ABI of the B300 (sm_103a) path for Fourier-represented kernel
 * regression (arXiv 2509.02649, "Fast kernel methods: Sobolev, physics-informed,
 * and additive models").
 *
 * What the library computes (paper notation, frequency scale pi/(2L) = 1, so
 * points are radians and a caller with data in [-L, L]^d passes x * pi/(2L)):
 *
 *   modes     K = { k in Z^d : |k|_inf <= m },  D = (2m+1)^d           (Sec. 2.2)
 *   moments   T_j = (1/n) sum_i exp(-i <j, X_i>),   |j|_inf <= 2m      (Sec. 2.3,
 *             covariance matrix: Phi^*Phi/n is d-level block Toeplitz with
 *             entries T_{k-k'})
 *   rhs       b_k = (1/n) sum_i Y_i exp(-i <k, X_i>), |k|_inf <= m      (Sec. 2.3,
 *             covariance vector)
 *   estimator theta = (Toep(T) + diag W)^{-1} b                         (Eq. 2)
 *   penalty   W_k = lambda (c0 + |k|_2^{2s})        Sobolev, M = S     (Sec. 3.1)
 *             W_k = lambda                           low bias, M = I    (Sec. 3.2)
 *             W_k += mu |P(ik)|^2                    physics-informed  (Sec. 4,
 *             tractable domain on the full period, where the Fourier matrix C
 *             of the domain is the identity)
 *   additive  block Gram of Prop. 5.1 (+ lambda I), blocks off the diagonal are
 *             2-D type-1 transforms of ones at (X_l1, -X_l2)            (Sec. 5)
 *   predict   f(x) = Re sum_k theta_k exp(+i <k, x>)                    (Eq. 1)
 *
 * Sums over points run through a type-1 non-uniform FFT (exponential-of-
 * semicircle spreading, FFT on an upsampled grid, deconvolution); prediction
 * through the type-2 transform (deconvolution, inverse FFT, interpolation).
 * eps is the requested relative l2 error of each transformed vector.
 *
 * Conventions shared by every entry point
 *  - Mode vectors are lexicographic over k in K with the LAST dimension
 *    fastest; flat index sum_l (k_l + m) (2m+1)^{d-1-l}.  Complex arrays are
 *    interleaved (re, im) doubles.
 *  - Points are structure-of-arrays, x[l * n + i] = coordinate l of point i.
 *    precision FK_MIXED: x and y are float32; FK_FP64: float64.  Points must
 *    lie in [-3 pi, 3 pi); they are folded onto [-pi, pi) (exact for integer
 *    modes by periodicity).  A point outside that range makes the call return
 *    FK_ERANGE.
 *  - Array arguments documented as "device" are device pointers owned by the
 *    caller; "host" arrays are read before the call returns.  The library never
 *    frees caller memory.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  Calls that return a status depending on device results (range
 *    flag, Cholesky pivots, CG convergence) synchronise `stream` before they
 *    return; fk_type1 / fk_type2 / fk_penalty_weights do not synchronise.
 *  - Scratch memory is allocated stream-ordered (cudaMallocAsync) on `stream`
 *    and released on it before return.
 *  - On error the outputs are unspecified and fk_last_error() describes the
 *    failure (thread-local string, valid until the next call on the thread).
 *    Argument errors are detected on the host before any launch.
 */
#ifndef FK_H_
#define FK_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FK_API __attribute__((visibility("default")))
#else
#define FK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FK_OK = 0,
  FK_EINVAL = 1,     /* invalid argument (detected on the host, nothing launched) */
  FK_ERANGE = 2,     /* a point outside [-3 pi, 3 pi) */
  FK_ENOMEM = 3,     /* device allocation failed */
  FK_ECUDA = 4,      /* a CUDA runtime call failed */
  FK_ENOTPD = 5,     /* Cholesky met a non-positive pivot (system not positive definite) */
  FK_ENOCONV = 6,    /* conjugate gradients did not reach cg_tol within cg_maxit */
  FK_ETIMEOUT = 7,   /* a bounded device-side wait gave up */
  FK_EINTERNAL = 8   /* internal consistency check failed */
} fk_status;

typedef enum { FK_FP64 = 0, FK_MIXED = 1 } fk_precision;
typedef enum { FK_PEN_SOBOLEV = 0, FK_PEN_LOWBIAS = 1 } fk_penalty;
/* EIG: the eigen route for sweeps over lambda (Sec. 5 grid search): one FP64 Hermitian
   eigendecomposition (parallel cyclic Jacobi) of S^-1 A0 S^-1 serves every penalty of the
   form lambda_l S^2, then O(D^2) per lambda and right-hand side.  Used by fk_fit_sobolev
   (Sobolev with c0 > 0, or low-bias) and fk_fit_additive; D <= 8192; not capturable. */
typedef enum { FK_SOLVER_AUTO = 0, FK_SOLVER_CHOL = 1, FK_SOLVER_CG = 2, FK_SOLVER_EIG = 3 } fk_solver;
/* Spreading methods of the mixed path: ATOMIC = fp64 global atomics per tap; BINNED =
   2-D partition + register accumulation (d = 2, ones and/or one strength channel);
   FIXED = 1-D integer fixed-point sums in shared memory (d = 1, any channel count,
   bitwise reproducible). */
typedef enum {
  FK_SPREAD_AUTO = 0,
  FK_SPREAD_ATOMIC = 1,
  FK_SPREAD_BINNED = 2,
  FK_SPREAD_FIXED = 3,        /* d = 1: integer (fixed-point) sums in shared memory; small grids are kept as
                                 32 lane copies per CTA, so that each lane's atomics go to its own bank */
  FK_SPREAD_FIXED_SHARED = 4  /* FIXED with one copy of each grid per CTA (no lane copies); the same sums
                                 bit for bit, since integer sums do not depend on the order of the adds */
} fk_spread;

/* Options; pass NULL for defaults (fk_default_opts). */
typedef struct {
  int solver;         /* fk_solver; AUTO = Cholesky for D <= 1024, else CG; EIG for lambda sweeps */
  double cg_tol;      /* relative residual target of CG (default 1e-13) */
  int cg_maxit;       /* CG iteration cap (default 1000) */
  int refine_steps;   /* iterative-refinement steps after a Cholesky solve (default 1) */
  double sobolev_c0;  /* c0 in lambda (c0 + |k|^{2s}); the paper's value is 1 (default 1) */
  double upsampfac;   /* minimum fine-grid oversampling sigma (default 1.9; grids are powers of 2) */
  int spread;         /* fk_spread: AUTO = BINNED (d = 2) or FIXED (d = 1) for FK_MIXED where the
                         shape allows, else ATOMIC; FK_FP64 always spreads with ATOMIC; FIXED_SHARED
                         as FIXED without lane copies */
  int deterministic;  /* 1: run-to-run identical type-1 sums (T, b, and the additive blocks): every
                         contribution is rounded to a 64-bit fixed-point integer (scale 2^(61-e)
                         with n max|strength| <= 2^e) and summed with integer atomics, for d = 1,
                         2, 3 and both precisions (the 1-D mixed fixed-point spreader is used
                         where it applies: its sums are order-independent already).  Slower than
                         the default register accumulation; the solvers' own reductions are not
                         covered (default 0) */
  int autotune;       /* 1: the first call of a problem class times the kernels' tunable shapes
                         (partition tile, cells per owner, round quota) on the call's own data,
                         keeps the fastest in a process-wide table and uses it from then on;
                         that first call runs the spreading several times (default 0) */
  long long wait_cycles; /* bound, in SM clock cycles, of each grid-barrier wait of the single-
                         launch conjugate-gradient solver; a wait that runs out makes the call
                         return FK_ETIMEOUT (default 0 = about 2 s at the maximum clock) */
} fk_opts;

/* Filled when a non-NULL pointer is passed (the call then synchronises `stream`). */
typedef struct {
  double ms_spread;     /* spreading (type-1) */
  double ms_fft;        /* FFT + deconvolution */
  double ms_solve;      /* penalty, assembly and solve */
  double ms_total;
  int cg_iters;         /* largest CG iteration count over the batch (0 for Cholesky) */
  double rel_residual;  /* largest |b - A theta| / |b| over the batch, FP64 */
  int64_t n_used;       /* points consumed */
  int fine_grid;        /* upsampled grid size per dimension */
  int kernel_width;     /* ES kernel width w (taps per dimension) */
  double ms_kernel;     /* the spreading step's main kernel alone (register accumulation or atomics) */
} fk_report;

FK_API void fk_default_opts(fk_opts* opts);

/* Workspace: every call takes its scratch from a library-owned stream-ordered memory
 * pool of the current device (created at first use) that keeps freed blocks, so that
 * repeated calls of the same shape reuse device memory.  fk_release_workspace returns
 * the pool's unused memory of the current device to the system (synchronises the
 * device). */
FK_API fk_status fk_release_workspace(void);

/* Autotuning table: fk_autotune_table writes one line per tuned problem class (device,
 * kernel, class, the timings tried and the winner) into buf (at most cap bytes, NUL
 * terminated) and returns the size it needs; fk_autotune_clear empties the table. */
FK_API size_t fk_autotune_table(char* buf, size_t cap);
FK_API void fk_autotune_clear(void);

/* Sobolev / low-bias estimator (Eq. 2 with Sec. 3.1 or 3.2 penalty) for a batch of
 * n_lambda regularisation values and n_targets response vectors.
 *   d in {1, 2, 3}; n >= 1; m >= 0; s >= 0; eps in [1e-14, 1e-1]; lambdas > 0.
 *   x: device, d x n;  y: device, n_targets x n;  lambdas: host, n_lambda.
 *   theta: device, [n_lambda][n_targets][D] complex (2 doubles each). */
FK_API fk_status fk_fit_sobolev(int d, int64_t n, const void* x, const void* y, int n_targets,
                         int m, double s, int penalty, const double* lambdas, int n_lambda,
                         double eps, int precision, const fk_opts* opts,
                         double* theta, void* stream, fk_report* rep);

/* Sweep over pairs (s_i, lambda_i) of the Sobolev or low-bias estimator from one
 * spreading pass (Sec. 3 experiments sweep s and lambda): penalty row i is
 * lambda_i (c0 + |k|^{2 s_i}) (or lambda_i for FK_PEN_LOWBIAS), and all n_pairs x
 * n_targets systems share T and b and are solved in one batch.
 *   s_values, lambdas: host, n_pairs;  theta: device, [n_pairs][n_targets][D] complex.
 *   Other arguments as fk_fit_sobolev. */
FK_API fk_status fk_fit_sobolev_pairs(int d, int64_t n, const void* x, const void* y, int n_targets, int m,
                                      const double* s_values, const double* lambdas, int n_pairs, int penalty,
                                      double eps, int precision, const fk_opts* opts, double* theta,
                                      void* stream, fk_report* rep);

/* Physics-informed estimator (Sec. 4, tractable domain = full period):
 *   W_k = lambda (c0 + |k|^{2s}) + mu |P(ik)|^2,  P(ik) = sum_t a_t prod_l (i k_l)^{alpha_t,l}.
 *   alpha: host, n_terms x d non-negative ints; a: host, n_terms reals.
 *   theta: device, [n_targets][D] complex.  Other arguments as fk_fit_sobolev. */
FK_API fk_status fk_fit_pik(int d, int64_t n, const void* x, const void* y, int n_targets,
                     int m, double s, double lambda, double mu, int n_terms,
                     const int* alpha, const double* a, double eps, int precision,
                     const fk_opts* opts, double* theta, void* stream, fk_report* rep);

/* Physics-informed estimator on a sub-domain or with collocation points (Sec. 4,
 * tractable and intractable domains): the penalty is lambda (c0 + |k|^{2s}) on the
 * diagonal plus mu D^* C D with D = diag P(ik) and the Hermitian Toeplitz C_{k,k'} =
 * c_{k-k'}, so the system is solved with conjugate gradients (two circulant products
 * per iteration) or, for D <= 1024, a dense Cholesky factorisation.
 *   c_moments: device complex (4m+1)^d, c_j = (2 pi)^{-d} int_Omega e^{-i<j,x>} dx for a
 *     domain Omega (fk_box_moments gives a box in closed form), or (1/n_r) sum_r
 *     e^{-i<j, X_r>} for collocation points X_r (the T output of fk_build_system on them).
 *     The full period has c_j = delta_j, where fk_fit_pik is the diagonal special case.
 *   Other arguments as fk_fit_pik (n_terms >= 1). */
FK_API fk_status fk_fit_pik_general(int d, int64_t n, const void* x, const void* y, int n_targets, int m,
                                    double s, double lambda, double mu, int n_terms, const int* alpha,
                                    const double* a, const double* c_moments, double eps, int precision,
                                    const fk_opts* opts, double* theta, void* stream, fk_report* rep);

/* Moments c_j (|j|_inf <= 2m) of the normalised Lebesgue measure of the box
 * prod_l [lo_l, hi_l] (host arrays, -3 pi <= lo_l < hi_l <= 3 pi):
 *   c_j = prod_l (e^{-i j_l hi_l} - e^{-i j_l lo_l}) / (-2 pi i j_l)  ((hi_l - lo_l)/(2 pi) at j_l = 0).
 *   c_moments: device complex (4m+1)^d, lexicographic. */
FK_API fk_status fk_box_moments(int d, int m, const double* lo, const double* hi, double* c_moments,
                                void* stream);

/* Low-bias additive estimator (Prop. 5.1): theta = (Sigma + lambda I)^{-1} (Phi_l^*Y/n)_l.
 *   d in [2, 16] coordinates; theta: device, [n_lambda][n_targets][d][2m+1] complex.
 *   The mixed path forks part of its work onto non-blocking streams of its own (one set
 *   per device and host thread: the pair transforms' accumulations and the 1-D
 *   transforms), ordered after the work already on `stream` by events and joined back
 *   into `stream` before the call returns, on error paths too; to the caller the work is
 *   ordered as if it were all on `stream`, and a capture on `stream` takes it in. */
FK_API fk_status fk_fit_additive(int d, int64_t n, const void* x, const void* y, int n_targets,
                          int m, const double* lambdas, int n_lambda, double eps,
                          int precision, const fk_opts* opts, double* theta, void* stream,
                          fk_report* rep);

/* Prediction f(x) = Re sum_k theta_k e^{+i<k,x>} (Eq. 1), or for additive != 0 the
 * additive form sum_l Re sum_k theta_{l,k} e^{i k x_l} (Sec. 5).
 *   theta: device, n_sets coefficient vectors (layout of the fit outputs);
 *   xq: device, d x n_q (precision as above);  f: device, [n_sets][n_q] doubles. */
FK_API fk_status fk_predict(int additive, int d, int m, const double* theta, int n_sets, int64_t n_q,
                     const void* xq, double eps, int precision, double* f, void* stream);

/* Building blocks (also the pieces of the autograd backward). */

/* Unnormalised type-1 sums out[c][k] = sum_i c_i exp(-i<k, x_i>), |k|_inf <= kmax.
 *   c: device, n_ch x n real strengths (precision of x);  out: device complex
 *   [n_ch][(2kmax+1)^d]. */
FK_API fk_status fk_type1(int d, int64_t n, const void* x, const void* c, int n_ch, int kmax,
                   double eps, int precision, double* out, void* stream);

/* Type-2 real parts out[s][i] = Re sum_k coef_{s,k} exp(+i<k, x_i>), |k|_inf <= kmax.
 *   coef: device complex [n_sets][(2kmax+1)^d];  out: device doubles [n_sets][n]. */
FK_API fk_status fk_type2(int d, int kmax, const double* coef, int n_sets, int64_t n, const void* x,
                   double eps, int precision, double* out, void* stream);

/* Type-1 sums as fk_type1, for callers that cannot allocate device memory at call
 * time (a process whose device memory is wholly reserved by its own pool allocator,
 * or a service that forbids device allocation after start-up).  The paper has no
 * counterpart to this entry point.
 *   All scratch comes from one built-in device array of FK_NOALLOC_SCRATCH_BYTES;
 *   no cudaMalloc / cudaMallocAsync / cudaFree is called.  Shapes whose scratch would
 *   exceed it (d = 2 needs about 16 N^2 n_ch bytes, N the upsampled grid) return
 *   FK_EINVAL with the required size in fk_last_error().
 *   The first call on a device does a one-time set-up with that device current: it
 *   looks up the array's device address (which, under the CUDA runtime's lazy module
 *   loading, is when the array is placed in device memory), loads the kernels later
 *   calls launch, and computes the quadrature nodes of the correction factors.  That
 *   call needs about FK_NOALLOC_SCRATCH_BYTES of free device memory plus the code, and
 *   returns FK_ECUDA if it cannot get them: make it at start-up, before device memory
 *   is reserved elsewhere, and before any stream capture.  The array is then held by
 *   that device until the process exits.
 *   Calls share the array and it keeps the last call's contents (the grid and the flag
 *   word are cleared each call; tables of the last call's plan are reused).  Calls
 *   whose work overlaps on the GPU (other streams, other host threads) race on it.
 *   The call synchronises `stream`.  Spreading uses the atomic form for both
 *   precisions.  Arguments and argument checks as fk_type1, with d in {1, 2}. */
#define FK_NOALLOC_SCRATCH_BYTES (16u << 20)
FK_API fk_status fk_type1_noalloc(int d, int64_t n, const void* x, const void* c, int n_ch, int kmax,
                                  double eps, int precision, double* out, void* stream);

/* Streaming sums.  T_j and b_k (Sec. 2.3) are sums over points, so a sample larger
 * than device memory (the 1-D sweep of 1e10 points) is added chunk by chunk onto
 * upsampled grids held by an accumulator; transform, penalty and solve run once.
 *   fk_accum_create: d in {1, 2}, m, n_targets in [0, 1024], eps and precision as in
 *     fk_fit_sobolev; allocates the grids ((1 + n_targets) N^d doubles) with cudaMalloc.
 *   fk_accum_add: adds n points (x: device d x n, y: device n_targets x n, precision as
 *     created).  y_absmax (device, n_targets float bit patterns of max|y_t| over this
 *     chunk, e.g. from fk_generate_sweep_1d) may be NULL; it sets the fixed-point scale
 *     of the 1-D mixed spreader, which otherwise reads y once more to find it.
 *     Asynchronous: inputs must stay valid until `stream` passes the call.
 *     Range errors surface at the next fk_accum_system / fk_accum_fit_sobolev.
 *   fk_accum_add_host: as fk_accum_add, with x (d x n) and y (n_targets x n) in HOST
 *     memory, row-major (coordinate l of point j at x[l n + j]).  The points go to the
 *     device in chunks of `chunk` points (0: FK_HOST_CHUNK_DEFAULT) through two
 *     device staging buffers owned by the accumulator (allocated by the first call,
 *     reallocated for a larger chunk, freed by fk_accum_destroy).  Each chunk is copied
 *     row by row on the accumulator's own copy stream and spread on `stream` once it
 *     has landed, so the copy of chunk i + 1 overlaps the spreading of chunk i.
 *     Page-locked host memory (cudaHostAlloc, cudaHostRegister) gets the link's full
 *     rate; pageable memory works, with the copies staged by the CUDA driver.  The call
 *     returns once the copies and spreads are enqueued: the host arrays must stay valid
 *     and unchanged until `stream` passes the call.  y_absmax is not taken (the 1-D
 *     fixed-point spreader finds each chunk's scale on the device).
 *     Errors: FK_EINVAL (null accumulator or arrays, n or chunk < 0), FK_ENOMEM
 *     (staging), FK_ECUDA; range errors as fk_accum_add.
 *   fk_accum_system: T (device complex (4m+1)^d) and b (device complex [n_targets][D]),
 *     each divided by the total point count; either may be NULL.  Synchronises.
 *   fk_accum_fit_sobolev: theta [n_lambda][n_targets][D] as fk_fit_sobolev.
 *   fk_accum_reset: clears the sums.  fk_accum_destroy: frees (NULL is allowed).
 * One accumulator is not safe for concurrent use from several host threads. */
typedef struct fk_accum fk_accum;
FK_API fk_status fk_accum_create(int d, int m, int n_targets, double eps, int precision,
                                 const fk_opts* opts, fk_accum** out, void* stream);
FK_API fk_status fk_accum_add(fk_accum* acc, int64_t n, const void* x, const void* y,
                              const unsigned* y_absmax, void* stream);
#define FK_HOST_CHUNK_DEFAULT (((int64_t)1) << 22)
FK_API fk_status fk_accum_add_host(fk_accum* acc, int64_t n, const void* x, const void* y, int64_t chunk,
                                   void* stream);
FK_API fk_status fk_accum_system(fk_accum* acc, double* T, double* b, int64_t* n_total, void* stream);
FK_API fk_status fk_accum_fit_sobolev(fk_accum* acc, double s, int penalty, const double* lambdas,
                                      int n_lambda, double* theta, void* stream, fk_report* rep);
FK_API fk_status fk_accum_reset(fk_accum* acc, void* stream);
FK_API fk_status fk_accum_destroy(fk_accum* acc);

/* Accumulator state on the host: checkpoint / resume of a chunked run, and the
 * reduction of shards.  The sums of Sec. 2.3 are additive over points, so a run can
 * stop after any chunk and resume from its saved sums, and shards of the points spread
 * by separate accumulators (other streams, devices or processes) combine by adding
 * their sums; fk_accum_system then divides by the total point count.
 *   fk_accum_state_bytes: size of the state (a 64-byte header, then the fp64 grids
 *     [1 + n_targets][N^d] as stored).
 *   fk_accum_save: writes the state (point count, device flags, grids) into buf (host,
 *     cap bytes); synchronises `stream`.
 *   fk_accum_load: replaces the accumulator's sums by a saved state of an accumulator
 *     of the same (d, m, n_targets, eps, precision, options), else FK_EINVAL.
 *   fk_accum_add_state: adds a saved state's sums, point count and flags to the
 *     accumulator (the shard reduction); synchronises `stream`.
 * The 1-D fixed-point path adds each chunk's sums to the fp64 grids in chunk order, so
 * a run resumed from a state saved after chunk k gives the same bits as the run that
 * was not interrupted. */
FK_API size_t fk_accum_state_bytes(const fk_accum* acc);
FK_API fk_status fk_accum_save(fk_accum* acc, void* buf, size_t cap, void* stream);
FK_API fk_status fk_accum_load(fk_accum* acc, const void* buf, size_t len, void* stream);
FK_API fk_status fk_accum_add_state(fk_accum* acc, const void* buf, size_t len, void* stream);

/* Capture of calls into one CUDA graph (no counterpart in the paper; the batching
 * form of the fits: a whole fit, e.g. the additive model's 8 + 28 transforms, Gram
 * assembly and dense solve, replayed with one graph launch).
 *   fk_capture_begin: starts capturing the calling host thread's library calls made
 *     on `stream` (a created stream, not the legacy default stream).  Until
 *     fk_capture_end the calls only record work: they return FK_OK without running
 *     it, and their outputs are written when the graph is launched.  Calls whose path
 *     needs a host round trip return FK_EINVAL and nothing of them is recorded:
 *     conjugate-gradient solves other than the 2-D single-launch solver (use
 *     FK_SOLVER_CHOL, D <= 8192, for the others), fk_hypergrad,
 *     fk_penalty_grads, fk_accum_*, fk_type1_noalloc, any call given a report, and
 *     fits with more than 256 lambdas.  Autotuning is off during a capture (stored
 *     shapes are used).
 *   fk_capture_end: ends the capture and returns the instantiated graph in *graph; if
 *     any call failed during the capture the graph is discarded (FK_EINVAL).
 *   fk_graph_launch: runs the recorded work on `stream` against the same buffers, so
 *     new data written into the inputs give new outputs.  Scratch memory is allocated
 *     and freed inside the graph.
 *   fk_graph_status: waits for the last launch, then returns the device-side condition
 *     of that run (FK_ERANGE, FK_ENOTPD, FK_ETIMEOUT, FK_ENOCONV) or FK_OK.
 *   fk_graph_destroy: waits for the last launch and frees the graph (NULL allowed).
 * Host arrays passed to captured calls (lambdas, PDE terms, box corners) are read at
 * capture time; device buffers must stay valid while the graph is used. */
typedef struct fk_graph fk_graph;
FK_API fk_status fk_capture_begin(void* stream);
FK_API fk_status fk_capture_end(void* stream, fk_graph** graph);
FK_API fk_status fk_graph_launch(fk_graph* graph, void* stream);
FK_API fk_status fk_graph_status(fk_graph* graph);
FK_API fk_status fk_graph_destroy(fk_graph* graph);
/* Time (ms) of the main spreading kernel (the 2-D binned accumulation, the 1-D
 * fixed-point spreader or the atomic spreader) in the last launch of the graph, from
 * event record nodes placed around it at capture (the last such kernel if the capture
 * holds several).  Waits for that launch. */
FK_API fk_status fk_graph_kernel_ms(fk_graph* graph, float* ms);

/* Synthetic 1-D sweep sample generated on the device (the paper's experiments are on
 * synthetic data; this one is too large to pass from the host).  Points first ..
 * first + n - 1 of the sample keyed by (seed, workload):
 *   X_i ~ Uniform(-pi, pi) (fp32), Y_ti = sign(X_i)|X_i|^0.7 + 0.2 z_ti, z ~ N(0, 1),
 * drawn with Philox4x32-10 counters so that any chunk can be made on its own.
 *   first: multiple of 4;  x: device float[n];  y: device float[n_targets][n];
 *   y_absmax: device unsigned[n_targets] (max |Y_t| of the chunk as float bits) or NULL. */
FK_API fk_status fk_generate_sweep_1d(uint64_t seed, int workload, int64_t first, int64_t n, int n_targets,
                                      float* x, float* y, unsigned* y_absmax, void* stream);

/* Moments and right-hand sides: T (device complex, (4m+1)^d) and
 * b (device complex, [n_targets][D]), each divided by n (Sec. 2.3). */
FK_API fk_status fk_build_system(int d, int64_t n, const void* x, const void* y, int n_targets, int m,
                          double eps, int precision, const fk_opts* opts, double* T, double* b,
                          void* stream, fk_report* rep);

/* Penalty diagonals W (device doubles, [n_lambda][D]) of Sec. 3.1 / 3.2 / 4:
 *   W = lambda (c0 + |k|^{2s}) (+ mu |P(ik)|^2 when n_terms > 0); penalty selects
 *   FK_PEN_SOBOLEV or FK_PEN_LOWBIAS (then W = lambda, s and c0 ignored). */
FK_API fk_status fk_penalty_weights(int d, int m, int penalty, double s, double c0,
                             const double* lambdas, int n_lambda, double mu, int n_terms,
                             const int* alpha, const double* a, double* W, void* stream);

/* Solve (Toep(T) + diag W_l) sol_{l,r} = rhs_r for every penalty l and right-hand side r.
 *   T: device complex (4m+1)^d;  W: device doubles [n_w][D];  rhs: device complex
 *   [n_rhs][D];  sol: device complex [n_w][n_rhs][D]. */
FK_API fk_status fk_solve(int d, int m, const double* T, const double* W, int n_w, const double* rhs,
                   int n_rhs, const fk_opts* opts, double* sol, void* stream, fk_report* rep);

/* Held-out-loss hypergradient (not in the paper; adjoint of Eq. 2).  Given the fit
 * theta for one (W, Y) pair and validation data (xv, yv):
 *   r = f(xv) - yv,  L = mean(r^2),  g = type1(xv, r) / n_v,  z = A^{-1} g,
 *   dW_k = -2 Re(conj(z_k) theta_k),  dY_i = (2/n) Re sum_k z_k e^{+i<k, X_i>}.
 *   T: device complex (4m+1)^d of the training points; W: device D; theta: device D
 *   complex; xv/yv: device (precision of x); outputs: loss (host double), dW (device
 *   D doubles), dY (device n doubles, may be NULL to skip). */
FK_API fk_status fk_hypergrad(int d, int64_t n, const void* x, int64_t n_v, const void* xv,
                       const void* yv, int m, const double* T, const double* W,
                       const double* theta, double eps, int precision, const fk_opts* opts,
                       double* loss, double* dW, double* dY, void* stream);

/* The same hypergradient in two halves, the forward and backward passes of the autograd
 * form (not in the paper):
 *   fk_heldout_loss: r = f(xv) - yv with f(x) = Re sum_k theta_k e^{+i<k,x>} (Eq. 1) and
 *     L = mean(r^2).  theta: device D complex; xv, yv: device (precision of x); loss: host;
 *     r: device n_v values in the precision of x.  Synchronises `stream`.
 *   fk_adjoint: g = type1(xv, r) / n_v, z = A^{-1} g with A = Toep(T) + diag W (the fit's
 *     matrix: T of the training points), dW_k = -2 Re(conj(z_k) theta_k), and, when zy is
 *     not NULL, zy = zscale z (device D complex).  With zscale = 2 c / n, the type-2 sums
 *     fk_type2(zy, X) give c dL/dY at any chunk X of the n training points, so the points
 *     can be produced chunk by chunk instead of stored.  Synchronises `stream`. */
FK_API fk_status fk_heldout_loss(int d, int m, const double* theta, int64_t n_v, const void* xv, const void* yv,
                                 double eps, int precision, const fk_opts* opts, double* loss, void* r,
                                 void* stream);
FK_API fk_status fk_adjoint(int d, int m, int64_t n_v, const void* xv, const void* r, const double* T,
                            const double* W, const double* theta, double eps, int precision, const fk_opts* opts,
                            double zscale, double* dW, double* zy, void* stream);

/* Chain rule from dL/dW (device, D doubles) to the penalty's parameters of
 *   W_k = lambda (c0 + |k|^{2s}) + mu |P(ik)|^2   (Sec. 3.1 and Sec. 4):
 *   out (host, 3 + n_terms doubles) = [dL/dlambda, dL/ds, dL/dmu, dL/da_0 .. dL/da_{n_terms-1}],
 *   dL/ds summing dW_k lambda |k|^{2s} ln|k|^2 over k != 0.  Synchronises `stream`. */
FK_API fk_status fk_penalty_grads(int d, int m, double s, double c0, double lambda, double mu, int n_terms,
                                  const int* alpha, const double* a, const double* dW, double* out,
                                  void* stream);

/* Thread-local description of the last failure on this thread ("" after success). */
FK_API const char* fk_last_error(void);

/* Upper bound of the scratch bytes one fit with these sizes allocates. */
FK_API size_t fk_workspace_bytes(int d, int m, int64_t n, int n_ch, double eps, int precision);

/* Number of CUDA kernels this library has launched in the process so far
 * (monotonic; a caller takes differences around a region of interest). */
FK_API int64_t fk_launch_count(void);

/* Measurement helper (no counterpart in the paper): the FP32 FMA throughput of the
 * current device, the peak the spreading kernels' flop rates are reported against.
 * One kernel of independent FMA chains (2048 threads per SM) is launched four times on
 * `stream` and timed with CUDA events; *tflops (host) receives the best of the last
 * three, at 2 flop per FMA, and *sm_count (host, may be NULL) the device's
 * multiprocessor count.  Synchronises `stream`; not capturable. */
FK_API fk_status fk_peak_fp32(double* tflops, int* sm_count, void* stream);

/* Measurement helper (no counterpart in the paper): the throughput of 32-bit integer
 * shared-memory atomic adds with a returned old value (the 1-D fixed-point spreader's
 * operation), in 1e9 lane operations per second, the peak its atomic rate is reported
 * against.  Two 1024-thread CTAs per SM each add into windows of 7 consecutive words of
 * a 98 KB array: *gops_distinct (host) when the 32 lanes of every warp instruction hit 32
 * different banks, *gops_random (host) for random windows.  Each is the best of three
 * launches after one warm-up on `stream`.  Synchronises `stream`; not capturable. */
FK_API fk_status fk_peak_smem_atomics(double* gops_distinct, double* gops_random, void* stream);

/* Library version string. */
FK_API const char* fk_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FK_H_ */
