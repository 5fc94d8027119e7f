// Internal declarations shared by the CUDA translation units of libfk.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/fk.h"

namespace fk {

// ------------------------------------------------------------------ errors
fk_status set_error(fk_status st, const char* fmt, ...);
void clear_error();
// Host-side checks shared by the entry points: d in {1, 2, 3}, n >= 1, m >= 0,
// eps in [1e-14, 1e-1], a known precision (FK_EINVAL with a message otherwise).
fk_status check_common(int d, int64_t n, int m, double eps, int precision);
// Process-wide count of kernels this library has launched (fk_launch_count).
void note_launch();

// Optional timing of the spreading step's main kernel for fk_report.ms_kernel:
// when `on`, the spreader records `start`/`stop` on its stream around that launch.
struct KernelTimer {
  bool on = false;
  bool recorded = false;
  cudaEvent_t start = nullptr, stop = nullptr;
  unsigned rec_flags = 0;  // cudaEventRecordExternal during a capture (event record nodes)
};
KernelTimer* kernel_timer();  // thread-local

// Named range around a host-side stage of a call (spreading, transform, solve, ...),
// shown on profilers' timelines; NVTX calls cost nothing when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  void next(const char* name) {  // ends this range and starts the next stage's
    nvtxRangePop();
    nvtxRangePushA(name);
  }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

#define FK_CUDA(call)                                                          \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess)                                                     \
      return ::fk::set_error(FK_ECUDA, "%s failed: %s (%s:%d)", #call,         \
                             cudaGetErrorString(e_), __FILE__, __LINE__);      \
  } while (0)

#define FK_TRY(expr)                    \
  do {                                  \
    fk_status s_ = (expr);              \
    if (s_ != FK_OK) return s_;         \
  } while (0)

// Device-side error flags (bits), read back by the host after a call.
enum : unsigned {
  FLAG_RANGE = 1u,      // a point outside [-3 pi, 3 pi)
  FLAG_NOTPD = 2u,      // Cholesky pivot <= 0
  FLAG_INTERNAL = 4u,   // an index check failed
  FLAG_TIMEOUT = 8u,    // a bounded wait gave up
  FLAG_NOCONV = 16u,    // conjugate gradients did not converge
};

// ------------------------------------------------------------------ complex
struct cd { double x, y; };
__host__ __device__ inline cd cmk(double a, double b) { return cd{a, b}; }
__host__ __device__ inline cd cadd(cd a, cd b) { return cd{a.x + b.x, a.y + b.y}; }
__host__ __device__ inline cd csub(cd a, cd b) { return cd{a.x - b.x, a.y - b.y}; }
__host__ __device__ inline cd cmul(cd a, cd b) { return cd{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__host__ __device__ inline cd cconjmul(cd a, cd b) { return cd{a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x}; }  // conj(a)*b
__host__ __device__ inline cd cscale(cd a, double s) { return cd{a.x * s, a.y * s}; }
__host__ __device__ inline cd cconj(cd a) { return cd{a.x, -a.y}; }
// acc + a b, acc + a conj(b), acc + conj(a) b: four FMAs each
__host__ __device__ inline cd cfma(cd a, cd b, cd acc) {
  return cd{fma(-a.y, b.y, fma(a.x, b.x, acc.x)), fma(a.y, b.x, fma(a.x, b.y, acc.y))};
}
__host__ __device__ inline cd cfma_cj(cd a, cd b, cd acc) {
  return cd{fma(a.y, b.y, fma(a.x, b.x, acc.x)), fma(-a.x, b.y, fma(a.y, b.x, acc.y))};
}
__host__ __device__ inline cd cjfma(cd a, cd b, cd acc) {
  return cd{fma(a.y, b.y, fma(a.x, b.x, acc.x)), fma(-a.y, b.x, fma(a.x, b.y, acc.y))};
}

template <typename R> struct cplx { R x, y; };

// ------------------------------------------------------------------ kernel plan
// Exponential-of-semicircle kernel phi(z) = exp(beta (sqrt(1 - z^2) - 1)), |z| < 1,
// spread over w grid nodes of spacing h = 2 pi / N (support radius w h / 2).
struct EsPlan {
  int d = 1;
  int N = 0;         // fine grid nodes per dimension (power of two)
  int w = 0;         // taps per dimension
  double beta = 0;   // ES shape
  double sigma = 0;  // N / (2 kmax + 1)
  int kmax = 0;      // largest |k| extracted per dimension
};

// Chooses N (power of two >= upsampfac * (2 kmax + 1), at least 2 w) and w, beta
// for the requested tolerance.
fk_status make_es_plan(int d, int kmax, double eps, double upsampfac, EsPlan* p);

// ------------------------------------------------------------------ workspace
// Library-owned stream-ordered memory pool of the current device.  It keeps freed
// blocks (release threshold unlimited), so repeated calls reuse the same device
// memory instead of mapping it again; fk_release_workspace() trims it.
cudaMemPool_t workspace_pool();

// Active capture of this host thread's library calls into a CUDA graph (capture.cu).
struct CaptureCtx {
  cudaStream_t st = nullptr;
  unsigned* flags = nullptr;  // the graph's flag word
  bool failed = false;        // a call returned an error during the capture
  cudaEvent_t kstart = nullptr, kstop = nullptr;  // main spreading kernel of the captured calls
  bool timed = false;                             // recorded as event nodes at least once
};
CaptureCtx* capture_ctx();
// FK_EINVAL when a capture is active and the call cannot be recorded (another stream,
// a report, or a host round trip on its path)
fk_status capture_check(cudaStream_t st, bool capturable, bool wants_report, const char* what);
// status of a device flag word
fk_status flags_status(unsigned h);

// Stream-ordered scratch allocation tracked for release at scope exit (during a
// capture: graph allocation nodes from the capturing stream).
struct Scratch {
  cudaStream_t st;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t s) : st(s) {}
  ~Scratch() { release(); }
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  void release() {
    for (size_t i = ptrs.size(); i-- > 0;) cudaFreeAsync(ptrs[i], st);
    ptrs.clear();
  }
  template <typename T>
  fk_status alloc(T** p, size_t elems) {
    size_t bytes = elems * sizeof(T);
    if (bytes == 0) bytes = 16;
    void* q = nullptr;
    cudaMemPool_t pool = capture_ctx() ? nullptr : workspace_pool();
    cudaError_t e = pool ? cudaMallocFromPoolAsync(&q, bytes, pool, st) : cudaMallocAsync(&q, bytes, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(FK_ENOMEM, "stream-ordered allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    ptrs.push_back(q);
    *p = static_cast<T*>(q);
    return FK_OK;
  }
};

int sm_count();  // multiprocessors of the current device (0 on error)

inline int grid_for(int64_t work, int block, int cap = 148 * 32) {
  int64_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return static_cast<int>(g);
}

// ------------------------------------------------------------------ component entry points
// (host functions enqueueing kernels on `st`; all pointers device)

// ES Fourier-transform correction factors corr[j + kmax] = (-1)^j h / Psi_hat(j),
// j = -kmax..kmax, in fp64 (Gauss-Legendre quadrature on the device).
fk_status es_correction(const EsPlan& p, double* corr, cudaStream_t st);

// Spreading: grid[c][node] += sum_i str_c(i) * prod_l psi(node_l - u_l(i)),
// ones channel optional (c = 0 when with_ones).  grid: fp64, n_ch x N^d, zeroed inside.
// R = float (FK_MIXED inputs) or double (FK_FP64 inputs).
template <typename R>
fk_status spread_atomic(const EsPlan& p, int64_t n, const R* x, const R* y, int n_y,
                        bool with_ones, double* grid, unsigned* flags, cudaStream_t st);

// Deterministic form (fk_opts.deterministic): 64-bit fixed-point integer sums, scaled
// back into the fp64 grid (zeroed inside); bitwise reproducible for d = 1, 2, 3.
template <typename R>
fk_status spread_deterministic(const EsPlan& p, int64_t n, const R* x, const R* y, int n_y, bool with_ones,
                               double* grid, unsigned* flags, cudaStream_t st, Scratch& scr);

// ------------------------------------------------------------------ autotuning
// Tunables of the kernels whose best shape depends on the problem; a process-wide
// table keyed by the problem's class holds the measured winners (autotune.cu).
struct BinCfg {       // 2-D binned spreading
  int half = 1;       // 1: partition blocks of 512 threads, two per SM (half tiles)
  int per = 7;        // points per thread and tile of the partition scatter (5..7)
  int cells = 0;      // cells per owner CTA (0: the kernel's maximum)
  float qmul = 0.5f;  // per-round quota = mean + qmul sqrt(mean)
};
enum TuneKind { TUNE_SPREAD2D = 1, TUNE_SPREAD1D = 2, TUNE_CG2D = 3 };
struct TuneKey {
  int kind, a, b, c, d;  // kind-specific class (grid size, width, channels, log2 n ...)
};
bool tune_lookup(const TuneKey& k, BinCfg* out);           // on the current device
void tune_store(const TuneKey& k, const BinCfg& v, const std::string& log);
bool tune_lookup_int(const TuneKey& k, int* out);
void tune_store_int(const TuneKey& k, int v, const std::string& log);

// Binned register-accumulation spreading (fp32, d = 2, ones and/or one strength channel).
// autotune: on the first call of a problem class, time the tunables and keep the best.
fk_status spread_binned(const EsPlan& p, int64_t n, const float* x, const float* y, int n_y,
                        bool with_ones, double* grid, unsigned* flags, cudaStream_t st,
                        Scratch& scratch, bool autotune = false);
bool spread_binned_supported(const EsPlan& p, int n_y, bool with_ones);
// As spread_binned with the two coordinates as separate rows, the second taken times s1.
fk_status spread_binned_xy(const EsPlan& p, int64_t n, const float* x0, const float* x1, float s1, const float* y,
                           int n_y, bool with_ones, double* grid, unsigned* flags, cudaStream_t st,
                           Scratch& scratch, bool autotune = false);

// Pair grids of the additive model (Sec. 5): for l1 < d - 1, the N x N grids of ones at
// (X_l1, -X_l2) for the partners l2 = l1 + 1 .. d - 1, from one partition of the points
// by the rows of coordinate l1 (mixed path, N <= 256, 4 <= w <= 8).  begin allocates the
// record streams in scr (two sets), counts every coordinate's row owners and computes
// the partners' code words once; part(l1) must follow for l1 = 0, 1, .. in order on one
// stream and writes record set l1 & 1; acc(l1), on any stream ordered after part(l1),
// reads that set and writes the d - 1 - l1 grids [partner][N^2] (zeroed inside).  So
// part(l1 + 2) must be ordered after acc(l1), and acc(l1) may overlap part(l1 + 1) and
// acc(l1 + 1).
struct AddPairState {
  EsPlan p;
  int d = 0, G = 0;
  int64_t n = 0, stride = 0;
  const float* x = nullptr;     // SoA rows [d][n]
  int* cnt = nullptr;           // [d + 1][G]: counts of each coordinate's row owners, then reservations
  unsigned* o1[2] = {};         // per record set: [stride] row words
  unsigned* code[2] = {};       // per record set: [d - 1][stride] code words
  unsigned* codes = nullptr;    // [d - 1][n] code words of -X_1 .. -X_(d-1), unbucketed
};
bool additive_pairs_supported(const EsPlan& p, int d, int64_t n);
fk_status additive_pairs_begin(const EsPlan& p, int d, int64_t n, const float* x, unsigned* flags, cudaStream_t st,
                               Scratch& scr, AddPairState* S);
fk_status additive_pairs_part(AddPairState& S, int l1, unsigned* flags, cudaStream_t st);
fk_status additive_pairs_acc(AddPairState& S, int l1, double* grids, unsigned* flags, cudaStream_t st);

// 1-D fixed-point shared-memory spreading (fp32 inputs, any channel count).  y_absmax:
// device array of max|y_c| bit patterns for the n_y strength channels, or null to
// compute it here.  accumulate: add into grid instead of overwriting it.
// Spread (ones channel if with_ones, then n_y strength channels) onto the fine grid with
// the spreader the options and the shape select (binned or fixed-point for the mixed path
// where they apply, fp64 atomics for FK_FP64, deterministic sums when asked), as the
// fits do.  x, y: device arrays of the precision's type.
fk_status spread_any(const EsPlan& p, int precision, const fk_opts& o, int64_t n, const void* x, const void* y,
                     int n_y, bool with_ones, double* grid, unsigned* flags, cudaStream_t st, Scratch& scr);

bool spread1d_fixed_supported(const EsPlan& p, int n_y, bool with_ones);
fk_status spread1d_fixed(const EsPlan& p, int64_t n, const float* x, const float* y, int n_y, bool with_ones,
                         const unsigned* y_absmax, double* grid, bool accumulate, unsigned* flags, cudaStream_t st,
                         Scratch& scratch, bool autotune = false, bool lane_copies = true);
// amax[c] = bit pattern of max_i |y[c][i]| (amax zeroed here first)
fk_status absmax_channels(int64_t n, const float* y, int n_y, unsigned* amax, cudaStream_t st);

// Forward transform of real fp64 grids + deconvolution + extraction of the modes
// |k|_inf <= kout (kout <= p.kmax) for channels [c0, c0 + nc), scaled by `scale`.
// out: complex [nc][(2 kout + 1)^d].  FFT arithmetic in R.
template <typename R>
fk_status grid_to_modes(const EsPlan& p, const double* grid, int c0, int nc, int kout,
                        const double* corr, double scale, double* out, cudaStream_t st,
                        Scratch& scratch);

// Type-2: coef [n_sets][(2 kmax_c + 1)^d] complex -> out [n_sets][n] = Re f(x_i).
template <typename R>
fk_status type2_eval(const EsPlan& p, int kmax_c, const double* coef, int n_sets, int64_t n,
                     const R* x, const double* corr, double* out, unsigned* flags,
                     cudaStream_t st, Scratch& scratch);

// Penalty diagonals.
fk_status penalty_weights(int d, int m, int penalty, double s, double c0, const double* lambdas,
                          int n_lambda, double mu, int n_terms, const int* alpha, const double* a,
                          double* W, cudaStream_t st);

// Extra penalty mu D^* C D of §4 with a non-diagonal Fourier matrix C_{k,k'} = c_{k-k'}
// (a sub-domain, or collocation points) and D = diag P(ik).
struct PenOp {
  const double* c = nullptr;  // (4m+1)^d complex moments, device
  const double* P = nullptr;  // (2m+1)^d complex symbol, device
  double mu = 0.0;
};
fk_status pde_symbol_vec(int d, int m, int n_terms, const int* alpha, const double* a, double* P, cudaStream_t st);
fk_status box_moments(int d, int m, const double* lo, const double* hi, double* c, cudaStream_t st);

// Dense / CG solves of (Toep(T) + diag W_l [+ mu D^* Toep(c) D]) X = B.
fk_status solve_system(int d, int m, const double* T, const double* W, int n_w, const double* rhs,
                       int n_rhs, const fk_opts& o, double* sol, cudaStream_t st,
                       Scratch& scratch, unsigned* flags, int* cg_iters, double* rel_res,
                       const PenOp* op = nullptr);

// Variants with caller-supplied scratch (used by the entry point that allocates nothing).
// es_gl_nodes_into writes the 2 es_gl_nodes() quadrature nodes and weights that
// es_correction_from_nodes reads.
fk_status es_gl_nodes_into(double* gl, cudaStream_t st);
fk_status es_correction_from_nodes(const EsPlan& p, double* corr, const double* gl, cudaStream_t st);
int es_gl_nodes();
// Force the lazy loading of the kernels the entry point without allocation launches
// (the ES tables, the atomic spreaders, the twiddles and the type-1 mode extraction),
// so that its later calls need no device memory for code.
fk_status preload_es_kernels();
fk_status preload_spread_atomic_kernels();
fk_status preload_modes_kernels();
template <typename R>
fk_status grid_to_modes_into(const EsPlan& p, const double* grid, int c0, int nc, int kout, const double* corr,
                             double scale, double* out, cudaStream_t st, double* tw, cplx<R>* H);

// Eigen route (eig.cu): Hermitian eigendecomposition by parallel cyclic Jacobi (A, D x D
// complex row-major, is overwritten; U gets the eigenvectors as columns, ev the
// eigenvalues), and the sweep solve theta[l][rhs] = S^-1 U (ev + lambda_l)^-1 U^H S^-1 b[rhs]
// (sinv = 1/S, or null for S = I; lambdas on the host).
fk_status eig_hermitian(int64_t D, double* A, double* U, double* ev, cudaStream_t st, Scratch& scr, int* sweeps);
fk_status eig_sweep_solve(int64_t D, const double* U, const double* ev, const double* sinv, const double* b,
                          int n_rhs, const double* lambdas, int n_lambda, double* sol, cudaStream_t st, Scratch& scr);
fk_status eig_scale_sym(int64_t D, const double* sinv, double* A, cudaStream_t st);
// Toep(T) + diag W as a dense D x D complex matrix (W: D doubles on the device)
fk_status assemble_toeplitz(int d, int m, const double* T, const double* W, double* A, cudaStream_t st);
// 1 / sqrt(w) elementwise
fk_status inv_sqrt(int64_t n, const double* w, double* out, cudaStream_t st);

// Dense Hermitian positive definite solve (A row-major complex, kept); X: B in, solution out.
fk_status solve_dense(const double* A, int64_t D, double* X, int n_rhs, int refine, cudaStream_t st, Scratch& scr,
                      unsigned* flags);

// Additive model (Prop. 5.1): theta [n_lambda][nt][d][2m+1]; prediction f [n_sets][nq].
fk_status fit_additive(int d, int64_t n, const void* x, const void* y, int nt, int m, const double* lambdas,
                       int n_lambda, double eps, int precision, const fk_opts& o, double* theta, cudaStream_t st,
                       fk_report* rep);
fk_status predict_additive(int d, int m, const double* theta, int n_sets, int64_t nq, const void* xq, double eps,
                           int precision, double* f, cudaStream_t st);

// FFT primitives (complex, in place on contiguous lines of length N, batched).
template <typename R>
fk_status fft_lines(cplx<R>* data, int N, int64_t n_lines, int64_t line_stride, int64_t elem_stride,
                    int sign, const double* tw, cudaStream_t st);
fk_status fft_twiddles(int N, double* tw, cudaStream_t st);  // tw[2t..2t+1] = e^{-2 pi i t / N}
// the same table, computed once per device and N and cached (*out stays valid)
fk_status twiddle_table(int N, cudaStream_t st, const double** out);

}  // namespace fk
