// C-ABI entry points of libfk (declared in include/fk.h): argument checks on the
// host, scratch management, and the order of the device stages of each call.
#include "fk_internal.cuh"

#include <atomic>
#include <cstring>
#include <mutex>
#include <chrono>
#include <vector>

namespace fk {

static thread_local std::string g_err;
static std::atomic<int64_t> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static thread_local KernelTimer g_ktimer;
KernelTimer* kernel_timer() { return &g_ktimer; }

// Arms the main-kernel timer for one call when a report is requested.
// During a capture the timer records the capture's own events as event record nodes,
// read after a replay by fk_graph_kernel_ms.
struct KernelTimerScope {
  KernelTimer* t;
  cudaEvent_t own_start = nullptr, own_stop = nullptr;
  CaptureCtx* cap;
  explicit KernelTimerScope(bool enabled) : t(kernel_timer()), cap(capture_ctx()) {
    t->recorded = false;
    t->rec_flags = 0;
    if (cap) {
      own_start = t->start;
      own_stop = t->stop;
      t->start = cap->kstart;
      t->stop = cap->kstop;
      t->rec_flags = cudaEventRecordExternal;
      t->on = cap->kstart != nullptr;
      return;
    }
    t->on = enabled;
    if (enabled && !t->start) {
      cudaEventCreate(&t->start);
      cudaEventCreate(&t->stop);
    }
  }
  double ms() {
    if (cap || !t->on || !t->recorded) return 0.0;
    float v = 0.f;
    cudaEventSynchronize(t->stop);
    cudaEventElapsedTime(&v, t->start, t->stop);
    return v;
  }
  ~KernelTimerScope() {
    if (cap) {
      if (t->recorded) cap->timed = true;
      t->start = own_start;
      t->stop = own_stop;
      t->rec_flags = 0;
    }
    t->on = false;
  }
};

static std::mutex g_pool_mutex;
static cudaMemPool_t g_pools[64] = {};

cudaMemPool_t workspace_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  if (!g_pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
  }
  return g_pools[dev];
}

fk_status set_error(fk_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  if (CaptureCtx* c = capture_ctx()) c->failed = true;
  return st;
}

fk_status flags_status(unsigned h) {
  if (h & FLAG_RANGE) return set_error(FK_ERANGE, "a point lies outside [-3 pi, 3 pi)");
  if (h & FLAG_NOTPD) return set_error(FK_ENOTPD, "Cholesky met a non-positive pivot");
  if (h & FLAG_TIMEOUT) return set_error(FK_ETIMEOUT, "a bounded device wait gave up");
  if (h & FLAG_INTERNAL) return set_error(FK_EINTERNAL, "device index check failed");
  if (h & FLAG_NOCONV) return set_error(FK_ENOCONV, "conjugate gradients did not converge");
  if (h) return set_error(FK_EINTERNAL, "device flag 0x%x", h);
  return FK_OK;
}

void clear_error() { g_err.clear(); }

static fk_opts resolve_opts(const fk_opts* o) {
  fk_opts r;
  fk_default_opts(&r);
  if (o) r = *o;
  if (r.cg_tol <= 0) r.cg_tol = 1e-13;
  if (r.cg_maxit <= 0) r.cg_maxit = 1000;
  if (r.refine_steps < 0) r.refine_steps = 0;
  if (r.upsampfac <= 1.0) r.upsampfac = 1.9;
  if (r.wait_cycles < 0) r.wait_cycles = 0;
  if (capture_ctx()) r.autotune = 0;  // tuning times kernels on the host clock
  return r;
}

fk_status check_common(int d, int64_t n, int m, double eps, int precision) {
  if (d < 1 || d > 3) return set_error(FK_EINVAL, "d = %d: transforms are built for d in {1, 2, 3}", d);
  if (n < 1) return set_error(FK_EINVAL, "n = %lld < 1", (long long)n);
  if (m < 0) return set_error(FK_EINVAL, "m = %d < 0", m);
  if (!(eps >= 1e-14 && eps <= 1e-1)) return set_error(FK_EINVAL, "eps = %g outside [1e-14, 1e-1]", eps);
  if (precision != FK_FP64 && precision != FK_MIXED) return set_error(FK_EINVAL, "unknown precision %d", precision);
  return FK_OK;
}

static int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// Flags word that lives for one call.
struct Flags {
  unsigned* dev = nullptr;
  cudaStream_t st;
  explicit Flags(cudaStream_t s) : st(s) {}
  // during a capture the graph's flag word, read by fk_graph_status after a replay
  fk_status init(Scratch& scr) {
    if (CaptureCtx* c = capture_ctx()) {
      dev = c->flags;
      return FK_OK;
    }
    FK_TRY(scr.alloc(&dev, 1));
    FK_CUDA(cudaMemsetAsync(dev, 0, sizeof(unsigned), st));
    return FK_OK;
  }
  fk_status check() {
    if (capture_ctx()) return FK_OK;
    unsigned h = 0;
    FK_CUDA(cudaMemcpyAsync(&h, dev, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    FK_CUDA(cudaStreamSynchronize(st));
    return flags_status(h);
  }
};

// Stage timer of one call; its events are created once per host thread and reused.
struct Timer {
  cudaStream_t st;
  bool on;
  cudaEvent_t* ev;
  int n = 0;
  Timer(cudaStream_t s, bool enabled) : st(s), on(enabled) {
    static thread_local cudaEvent_t pool[8] = {};
    static thread_local bool made = false;
    if (on && !made) {
      for (int i = 0; i < 8; ++i) cudaEventCreate(&pool[i]);
      made = true;
    }
    ev = pool;
  }
  void mark() {
    if (!on || n >= 8) return;
    cudaEventRecord(ev[n], st);
    ++n;
  }
  double ms(int a, int b) {
    if (!on || b >= n) return 0.0;
    cudaEventSynchronize(ev[b]);
    float t = 0.f;
    cudaEventElapsedTime(&t, ev[a], ev[b]);
    return t;
  }
};

// Spread (ones channel if with_ones, then n_y strength channels) onto the fine grid.
fk_status spread_any(const EsPlan& p, int precision, const fk_opts& o, int64_t n, const void* x,
                            const void* y, int n_y, bool with_ones, double* grid, unsigned* flags,
                            cudaStream_t st, Scratch& scr) {
  // deterministic sums: the 1-D fixed-point spreader (order-independent already) where it
  // applies, else 64-bit fixed-point global sums
  const bool fixed1d = precision == FK_MIXED && p.d == 1 && o.spread != FK_SPREAD_ATOMIC &&
                       spread1d_fixed_supported(p, n_y, with_ones);
  if (o.deterministic && !fixed1d) {
    if (precision == FK_FP64)
      return spread_deterministic<double>(p, n, static_cast<const double*>(x), static_cast<const double*>(y), n_y,
                                          with_ones, grid, flags, st, scr);
    return spread_deterministic<float>(p, n, static_cast<const float*>(x), static_cast<const float*>(y), n_y,
                                       with_ones, grid, flags, st, scr);
  }
  if (precision == FK_FP64)
    return spread_atomic<double>(p, n, static_cast<const double*>(x), static_cast<const double*>(y), n_y,
                                 with_ones, grid, flags, st);
  const int nc = n_y + (with_ones ? 1 : 0);
  const bool fixed_req = o.spread == FK_SPREAD_FIXED || o.spread == FK_SPREAD_FIXED_SHARED;
  if (p.d == 1 && (fixed_req || (o.spread == FK_SPREAD_AUTO && spread1d_fixed_supported(p, n_y, with_ones)))) {
    if (!spread1d_fixed_supported(p, n_y, with_ones))
      return set_error(FK_EINVAL, "fixed-point spreading does not support N=%d w=%d channels=%d", p.N, p.w, nc);
    return spread1d_fixed(p, n, static_cast<const float*>(x), static_cast<const float*>(y), n_y, with_ones, nullptr,
                          grid, false, flags, st, scr, o.autotune != 0, o.spread != FK_SPREAD_FIXED_SHARED);
  }
  if (fixed_req) return set_error(FK_EINVAL, "fixed-point spreading is built for d = 1");
  const bool binned = (o.spread == FK_SPREAD_BINNED) ||
                      (o.spread == FK_SPREAD_AUTO && spread_binned_supported(p, n_y, with_ones));
  if (binned) {
    if (!spread_binned_supported(p, n_y, with_ones))
      return set_error(FK_EINVAL, "binned spreading does not support d=%d w=%d channels=%d", p.d, p.w, nc);
    return spread_binned(p, n, static_cast<const float*>(x), static_cast<const float*>(y), n_y, with_ones, grid,
                         flags, st, scr, o.autotune != 0);
  }
  return spread_atomic<float>(p, n, static_cast<const float*>(x), static_cast<const float*>(y), n_y, with_ones,
                              grid, flags, st);
}

static fk_status modes_any(const EsPlan& p, int precision, const double* grid, int c0, int nc, int kout,
                           const double* corr, double scale, double* out, cudaStream_t st, Scratch& scr) {
  if (precision == FK_FP64) return grid_to_modes<double>(p, grid, c0, nc, kout, corr, scale, out, st, scr);
  return grid_to_modes<float>(p, grid, c0, nc, kout, corr, scale, out, st, scr);
}

// T (doubled range, divided by n) and b (n_targets channels, divided by n).
static fk_status build_system(int d, int64_t n, const void* x, const void* y, int n_targets, int m, double eps,
                              int precision, const fk_opts& o, double* T, double* b, cudaStream_t st,
                              Scratch& scr, unsigned* flags, EsPlan* plan_out, Timer* tm) {
  EsPlan p;
  FK_TRY(make_es_plan(d, 2 * m, eps, o.upsampfac, &p));
  if (plan_out) *plan_out = p;
  const int nc = 1 + n_targets;
  const int64_t G = ipow(p.N, d);
  double *grid = nullptr, *corr = nullptr;
  FK_TRY(scr.alloc(&grid, G * nc));
  FK_TRY(scr.alloc(&corr, 2 * static_cast<size_t>(p.kmax) + 1));
  FK_TRY(es_correction(p, corr, st));
  if (tm) tm->mark();
  {
    NvtxRange r("fk spread");
    FK_TRY(spread_any(p, precision, o, n, x, y, n_targets, true, grid, flags, st, scr));
  }
  if (tm) tm->mark();
  {
    NvtxRange r("fk transform");
    const double inv_n = 1.0 / static_cast<double>(n);
    FK_TRY(modes_any(p, precision, grid, 0, 1, 2 * m, corr, inv_n, T, st, scr));
    if (n_targets > 0) FK_TRY(modes_any(p, precision, grid, 1, n_targets, m, corr, inv_n, b, st, scr));
  }
  if (tm) tm->mark();
  return FK_OK;
}

}  // namespace fk

using namespace fk;

extern "C" {

void fk_default_opts(fk_opts* o) {
  if (!o) return;
  o->solver = FK_SOLVER_AUTO;
  o->cg_tol = 1e-13;
  o->cg_maxit = 1000;
  o->refine_steps = 1;
  o->sobolev_c0 = 1.0;
  o->upsampfac = 1.9;
  o->spread = FK_SPREAD_AUTO;
  o->deterministic = 0;
  o->autotune = 0;
  o->wait_cycles = 0;
}

const char* fk_last_error(void) { return g_err.c_str(); }

fk_status fk_release_workspace(void) {
  clear_error();
  cudaMemPool_t pool = workspace_pool();
  if (!pool) return set_error(FK_ECUDA, "no workspace pool on this device");
  FK_CUDA(cudaDeviceSynchronize());
  FK_CUDA(cudaMemPoolTrimTo(pool, 0));
  return FK_OK;
}

const char* fk_version(void) { return "fk 0.1 (sm_103a)"; }

int64_t fk_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

size_t fk_workspace_bytes(int d, int m, int64_t n, int n_ch, double eps, int precision) {
  (void)n;
  (void)precision;
  EsPlan p;
  if (make_es_plan(d, 2 * m, eps, 1.9, &p) != FK_OK) return 0;
  const int64_t G = ipow(p.N, d);
  const int64_t D = ipow(2 * m + 1, d);
  size_t bytes = sizeof(double) * G * (n_ch + 1);          // grids
  bytes += sizeof(double) * 2 * G * (n_ch + 1);            // FFT intermediates (upper bound)
  bytes += sizeof(double) * 2 * ipow(4 * m + 1, d);        // T
  bytes += sizeof(double) * 2 * D * D;                     // dense system (Cholesky route)
  bytes += sizeof(double) * 2 * D * 8 * (n_ch + 1);        // CG vectors
  bytes += 64u << 20;                                      // binning buffers
  return bytes;
}

fk_status fk_type1(int d, int64_t n, const void* x, const void* c, int n_ch, int kmax, double eps, int precision,
                   double* out, void* stream) {
  clear_error();
  FK_TRY(check_common(d, n, 0, eps, precision));
  if (kmax < 0 || n_ch < 1 || !x || !c || !out) return set_error(FK_EINVAL, "bad type-1 arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, true, false, "fk_type1"));
  const fk_opts o = resolve_opts(nullptr);
  Scratch scr(st);
  Flags fl(st);
  FK_TRY(fl.init(scr));
  EsPlan p;
  FK_TRY(make_es_plan(d, kmax, eps, o.upsampfac, &p));
  double *grid = nullptr, *corr = nullptr;
  FK_TRY(scr.alloc(&grid, ipow(p.N, d) * n_ch));
  FK_TRY(scr.alloc(&corr, 2 * static_cast<size_t>(kmax) + 1));
  FK_TRY(es_correction(p, corr, st));
  FK_TRY(spread_any(p, precision, o, n, x, c, n_ch, false, grid, fl.dev, st, scr));
  FK_TRY(modes_any(p, precision, grid, 0, n_ch, kmax, corr, 1.0, out, st, scr));
  return fl.check();
}

fk_status fk_type2(int d, int kmax, const double* coef, int n_sets, int64_t n, const void* x, double eps,
                   int precision, double* out, void* stream) {
  clear_error();
  FK_TRY(check_common(d, n, 0, eps, precision));
  if (kmax < 0 || n_sets < 1 || !x || !coef || !out) return set_error(FK_EINVAL, "bad type-2 arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, true, false, "fk_type2"));
  const fk_opts o = resolve_opts(nullptr);
  Scratch scr(st);
  Flags fl(st);
  FK_TRY(fl.init(scr));
  EsPlan p;
  FK_TRY(make_es_plan(d, kmax, eps, o.upsampfac, &p));
  double* corr = nullptr;
  FK_TRY(scr.alloc(&corr, 2 * static_cast<size_t>(kmax) + 1));
  FK_TRY(es_correction(p, corr, st));
  if (precision == FK_FP64)
    FK_TRY(type2_eval<double>(p, kmax, coef, n_sets, n, static_cast<const double*>(x), corr, out, fl.dev, st, scr));
  else
    FK_TRY(type2_eval<float>(p, kmax, coef, n_sets, n, static_cast<const float*>(x), corr, out, fl.dev, st, scr));
  return fl.check();
}

fk_status fk_build_system(int d, int64_t n, const void* x, const void* y, int n_targets, int m, double eps,
                          int precision, const fk_opts* opts, double* T, double* b, void* stream, fk_report* rep) {
  clear_error();
  FK_TRY(check_common(d, n, m, eps, precision));
  if (!x || !T || (n_targets > 0 && (!y || !b)) || n_targets < 0)
    return set_error(FK_EINVAL, "bad build_system arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, true, rep != nullptr, "fk_build_system"));
  const fk_opts o = resolve_opts(opts);
  Scratch scr(st);
  Flags fl(st);
  FK_TRY(fl.init(scr));
  Timer tm(st, rep != nullptr);
  KernelTimerScope kts(rep != nullptr);
  tm.mark();
  EsPlan p;
  FK_TRY(build_system(d, n, x, y, n_targets, m, eps, precision, o, T, b, st, scr, fl.dev, &p, &tm));
  FK_TRY(fl.check());
  if (rep) {
    *rep = fk_report{};
    rep->ms_spread = tm.ms(1, 2);
    rep->ms_fft = tm.ms(2, 3);
    rep->ms_total = tm.ms(0, 3);
    rep->n_used = n;
    rep->fine_grid = p.N;
    rep->kernel_width = p.w;
    rep->ms_kernel = kts.ms();
  }
  return FK_OK;
}

fk_status fk_penalty_weights(int d, int m, int penalty, double s, double c0, const double* lambdas, int n_lambda,
                             double mu, int n_terms, const int* alpha, const double* a, double* W, void* stream) {
  clear_error();
  if (d < 1 || d > 3 || m < 0 || n_lambda < 1 || !lambdas || !W) return set_error(FK_EINVAL, "bad penalty arguments");
  if (n_terms > 0 && (!alpha || !a)) return set_error(FK_EINVAL, "PDE terms need alpha and a");
  if (penalty != FK_PEN_SOBOLEV && penalty != FK_PEN_LOWBIAS) return set_error(FK_EINVAL, "unknown penalty");
  if (s < 0) return set_error(FK_EINVAL, "s < 0");
  return penalty_weights(d, m, penalty, s, c0, lambdas, n_lambda, mu, n_terms, alpha, a, W,
                         static_cast<cudaStream_t>(stream));
}

fk_status fk_solve(int d, int m, const double* T, const double* W, int n_w, const double* rhs, int n_rhs,
                   const fk_opts* opts, double* sol, void* stream, fk_report* rep) {
  clear_error();
  if (d < 1 || d > 3 || m < 0 || n_w < 1 || n_rhs < 1 || !T || !W || !rhs || !sol)
    return set_error(FK_EINVAL, "bad solve arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, true, rep != nullptr, "fk_solve"));
  const fk_opts o = resolve_opts(opts);
  Scratch scr(st);
  Flags fl(st);
  FK_TRY(fl.init(scr));
  int iters = 0;
  double rr = 0;
  FK_TRY(solve_system(d, m, T, W, n_w, rhs, n_rhs, o, sol, st, scr, fl.dev, &iters, rep ? &rr : nullptr));
  FK_TRY(fl.check());
  if (rep) {
    *rep = fk_report{};
    rep->cg_iters = iters;
    rep->rel_residual = rr;
  }
  return FK_OK;
}

static fk_status fit_common(int d, int64_t n, const void* x, const void* y, int n_targets, int m,
                            int penalty, double s, const double* lambdas, int n_lambda, double mu, int n_terms,
                            const int* alpha, const double* a, double eps, int precision, const fk_opts* opts,
                            double* theta, void* stream, fk_report* rep, const double* cmom = nullptr) {
  FK_TRY(check_common(d, n, m, eps, precision));
  if (!x || !y || !theta || !lambdas || n_targets < 1 || n_lambda < 1)
    return set_error(FK_EINVAL, "bad fit arguments");
  for (int i = 0; i < n_lambda; ++i)
    if (!(lambdas[i] >= 0.0)) return set_error(FK_EINVAL, "lambda[%d] = %g < 0", i, lambdas[i]);
  if (s < 0) return set_error(FK_EINVAL, "s < 0");
  if (mu < 0) return set_error(FK_EINVAL, "mu < 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, true, rep != nullptr, "the fit"));
  const fk_opts o = resolve_opts(opts);
  Scratch scr(st);
  Flags fl(st);
  FK_TRY(fl.init(scr));
  Timer tm(st, rep != nullptr);
  KernelTimerScope kts(rep != nullptr);
  tm.mark();
  const int64_t D = ipow(2 * m + 1, d), M2 = ipow(4 * m + 1, d);
  double *T = nullptr, *b = nullptr, *W = nullptr;
  FK_TRY(scr.alloc(&T, 2 * M2));
  FK_TRY(scr.alloc(&b, 2 * D * n_targets));
  FK_TRY(scr.alloc(&W, D * n_lambda));
  EsPlan p;
  FK_TRY(build_system(d, n, x, y, n_targets, m, eps, precision, o, T, b, st, scr, fl.dev, &p, &tm));
  if (o.solver == FK_SOLVER_EIG) {
    // eigen route: every penalty is lambda_l S^2 with S^2 the weights at lambda = 1
    if (cmom || mu != 0.0 || n_terms > 0)
      return set_error(FK_EINVAL, "the eigen route needs penalties lambda S^2 (no physics-informed term)");
    if (penalty == FK_PEN_SOBOLEV && !(o.sobolev_c0 > 0.0))
      return set_error(FK_EINVAL, "the eigen route needs c0 > 0 (S^2 = c0 + |k|^{2s} invertible)");
    if (D > 8192) return set_error(FK_EINVAL, "the eigen route is limited to D <= 8192 (D = %lld)", (long long)D);
    if (capture_ctx()) return set_error(FK_EINVAL, "the eigen route tests convergence on the host: not capturable");
    NvtxRange r("fk solve (eigen route)");
    const double one = 1.0;
    double *S2 = nullptr, *sinv = nullptr, *zero = nullptr, *A = nullptr, *U = nullptr, *ev = nullptr;
    FK_TRY(scr.alloc(&S2, D));
    FK_TRY(scr.alloc(&sinv, D));
    FK_TRY(scr.alloc(&zero, D));
    FK_TRY(scr.alloc(&A, 2 * D * D));
    FK_TRY(scr.alloc(&U, 2 * D * D));
    FK_TRY(scr.alloc(&ev, D));
    FK_TRY(penalty_weights(d, m, penalty, s, o.sobolev_c0, &one, 1, 0.0, 0, nullptr, nullptr, S2, st));
    FK_TRY(inv_sqrt(D, S2, sinv, st));
    FK_CUDA(cudaMemsetAsync(zero, 0, sizeof(double) * D, st));
    FK_TRY(assemble_toeplitz(d, m, T, zero, A, st));
    FK_TRY(eig_scale_sym(D, sinv, A, st));
    int sweeps = 0;
    FK_TRY(eig_hermitian(D, A, U, ev, st, scr, &sweeps));
    FK_TRY(eig_sweep_solve(D, U, ev, sinv, b, n_targets, lambdas, n_lambda, theta, st, scr));
    tm.mark();
    FK_TRY(fl.check());
    if (rep) {
      *rep = fk_report{};
      rep->ms_spread = tm.ms(1, 2);
      rep->ms_fft = tm.ms(2, 3);
      rep->ms_solve = tm.ms(3, 4);
      rep->ms_total = tm.ms(0, 4);
      rep->n_used = n;
      rep->fine_grid = p.N;
      rep->kernel_width = p.w;
      rep->ms_kernel = kts.ms();
    }
    return FK_OK;
  }
  PenOp op;
  if (cmom) {
    // sub-domain / collocation penalty: W keeps the Sobolev part, mu D^* C D is an operator
    double* P = nullptr;
    FK_TRY(scr.alloc(&P, 2 * D));
    FK_TRY(pde_symbol_vec(d, m, n_terms, alpha, a, P, st));
    FK_TRY(penalty_weights(d, m, penalty, s, o.sobolev_c0, lambdas, n_lambda, 0.0, 0, nullptr, nullptr, W, st));
    op.c = cmom;
    op.P = P;
    op.mu = mu;
  } else {
    FK_TRY(penalty_weights(d, m, penalty, s, o.sobolev_c0, lambdas, n_lambda, mu, n_terms, alpha, a, W, st));
  }
  int iters = 0;
  double rr = 0;
  {
    NvtxRange r("fk solve");
    FK_TRY(solve_system(d, m, T, W, n_lambda, b, n_targets, o, theta, st, scr, fl.dev, &iters, rep ? &rr : nullptr,
                        cmom ? &op : nullptr));
  }
  tm.mark();
  FK_TRY(fl.check());
  if (rep) {
    *rep = fk_report{};
    rep->ms_spread = tm.ms(1, 2);
    rep->ms_fft = tm.ms(2, 3);
    rep->ms_solve = tm.ms(3, 4);
    rep->ms_total = tm.ms(0, 4);
    rep->cg_iters = iters;
    rep->rel_residual = rr;
    rep->n_used = n;
    rep->fine_grid = p.N;
    rep->kernel_width = p.w;
    rep->ms_kernel = kts.ms();
  }
  return FK_OK;
}

fk_status fk_fit_sobolev(int d, int64_t n, const void* x, const void* y, int n_targets, int m, double s,
                         int penalty, const double* lambdas, int n_lambda, double eps, int precision,
                         const fk_opts* opts, double* theta, void* stream, fk_report* rep) {
  clear_error();
  if (penalty != FK_PEN_SOBOLEV && penalty != FK_PEN_LOWBIAS) return set_error(FK_EINVAL, "unknown penalty");
  return fit_common(d, n, x, y, n_targets, m, penalty, s, lambdas, n_lambda, 0.0, 0, nullptr, nullptr, eps,
                    precision, opts, theta, stream, rep);
}

fk_status fk_fit_pik(int d, int64_t n, const void* x, const void* y, int n_targets, int m, double s, double lambda,
                     double mu, int n_terms, const int* alpha, const double* a, double eps, int precision,
                     const fk_opts* opts, double* theta, void* stream, fk_report* rep) {
  clear_error();
  if (n_terms < 0 || n_terms > 16 || (n_terms > 0 && (!alpha || !a)))
    return set_error(FK_EINVAL, "bad PDE operator arguments");
  return fit_common(d, n, x, y, n_targets, m, FK_PEN_SOBOLEV, s, &lambda, 1, mu, n_terms, alpha, a, eps, precision,
                    opts, theta, stream, rep);
}

fk_status fk_fit_sobolev_pairs(int d, int64_t n, const void* x, const void* y, int n_targets, int m,
                               const double* s_values, const double* lambdas, int n_pairs, int penalty, double eps,
                               int precision, const fk_opts* opts, double* theta, void* stream, fk_report* rep) {
  clear_error();
  FK_TRY(check_common(d, n, m, eps, precision));
  if (!x || !y || !theta || !s_values || !lambdas || n_targets < 1 || n_pairs < 1)
    return set_error(FK_EINVAL, "bad fit arguments");
  if (penalty != FK_PEN_SOBOLEV && penalty != FK_PEN_LOWBIAS) return set_error(FK_EINVAL, "unknown penalty");
  for (int i = 0; i < n_pairs; ++i) {
    if (!(lambdas[i] >= 0.0)) return set_error(FK_EINVAL, "lambda[%d] = %g < 0", i, lambdas[i]);
    if (!(s_values[i] >= 0.0)) return set_error(FK_EINVAL, "s[%d] = %g < 0", i, s_values[i]);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, true, rep != nullptr, "fk_fit_sobolev_pairs"));
  const fk_opts o = resolve_opts(opts);
  Scratch scr(st);
  Flags fl(st);
  FK_TRY(fl.init(scr));
  Timer tm(st, rep != nullptr);
  KernelTimerScope kts(rep != nullptr);
  tm.mark();
  const int64_t D = ipow(2 * m + 1, d), M2 = ipow(4 * m + 1, d);
  double *T = nullptr, *b = nullptr, *W = nullptr;
  FK_TRY(scr.alloc(&T, 2 * M2));
  FK_TRY(scr.alloc(&b, 2 * D * n_targets));
  FK_TRY(scr.alloc(&W, D * n_pairs));
  EsPlan p;
  FK_TRY(build_system(d, n, x, y, n_targets, m, eps, precision, o, T, b, st, scr, fl.dev, &p, &tm));
  if (o.solver == FK_SOLVER_EIG)
    return set_error(FK_EINVAL, "the eigen route needs one penalty shape lambda S^2 for the whole sweep");
  // one penalty row per (s, lambda) pair; all rows share T and b (one spreading pass)
  for (int i = 0; i < n_pairs; ++i)
    FK_TRY(penalty_weights(d, m, penalty, s_values[i], o.sobolev_c0, lambdas + i, 1, 0.0, 0, nullptr, nullptr,
                           W + static_cast<int64_t>(i) * D, st));
  int iters = 0;
  double rr = 0;
  FK_TRY(solve_system(d, m, T, W, n_pairs, b, n_targets, o, theta, st, scr, fl.dev, &iters, rep ? &rr : nullptr));
  tm.mark();
  FK_TRY(fl.check());
  if (rep) {
    *rep = fk_report{};
    rep->ms_spread = tm.ms(1, 2);
    rep->ms_fft = tm.ms(2, 3);
    rep->ms_solve = tm.ms(3, 4);
    rep->ms_total = tm.ms(0, 4);
    rep->cg_iters = iters;
    rep->rel_residual = rr;
    rep->n_used = n;
    rep->fine_grid = p.N;
    rep->kernel_width = p.w;
    rep->ms_kernel = kts.ms();
  }
  return FK_OK;
}

fk_status fk_fit_pik_general(int d, int64_t n, const void* x, const void* y, int n_targets, int m, double s,
                             double lambda, double mu, int n_terms, const int* alpha, const double* a,
                             const double* c_moments, double eps, int precision, const fk_opts* opts, double* theta,
                             void* stream, fk_report* rep) {
  clear_error();
  if (!c_moments) return set_error(FK_EINVAL, "c_moments is null (use fk_fit_pik for the full period)");
  if (n_terms < 1 || n_terms > 16 || !alpha || !a) return set_error(FK_EINVAL, "bad PDE operator arguments");
  return fit_common(d, n, x, y, n_targets, m, FK_PEN_SOBOLEV, s, &lambda, 1, mu, n_terms, alpha, a, eps, precision,
                    opts, theta, stream, rep, c_moments);
}

fk_status fk_box_moments(int d, int m, const double* lo, const double* hi, double* c_moments, void* stream) {
  clear_error();
  if (d < 1 || d > 3 || m < 0 || !lo || !hi || !c_moments) return set_error(FK_EINVAL, "bad box moment arguments");
  return box_moments(d, m, lo, hi, c_moments, static_cast<cudaStream_t>(stream));
}

fk_status fk_fit_additive(int d, int64_t n, const void* x, const void* y, int n_targets, int m,
                          const double* lambdas, int n_lambda, double eps, int precision, const fk_opts* opts,
                          double* theta, void* stream, fk_report* rep) {
  clear_error();
  if (d < 2 || d > 16) return set_error(FK_EINVAL, "additive model: d = %d outside [2, 16]", d);
  if (n < 1) return set_error(FK_EINVAL, "n = %lld < 1", (long long)n);
  if (m < 0) return set_error(FK_EINVAL, "m = %d < 0", m);
  if (!(eps >= 1e-14 && eps <= 1e-1)) return set_error(FK_EINVAL, "eps = %g outside [1e-14, 1e-1]", eps);
  if (precision != FK_FP64 && precision != FK_MIXED) return set_error(FK_EINVAL, "unknown precision %d", precision);
  if (!x || !y || !theta || !lambdas || n_targets < 1 || n_lambda < 1) return set_error(FK_EINVAL, "bad fit arguments");
  for (int i = 0; i < n_lambda; ++i)
    if (!(lambdas[i] > 0.0)) return set_error(FK_EINVAL, "lambda[%d] = %g must be > 0 (Sigma is singular)", i, lambdas[i]);
  if (static_cast<int64_t>(d) * (2 * m + 1) > 8192) return set_error(FK_EINVAL, "d (2m + 1) > 8192");
  FK_TRY(capture_check(static_cast<cudaStream_t>(stream), true, rep != nullptr, "fk_fit_additive"));
  return fit_additive(d, n, x, y, n_targets, m, lambdas, n_lambda, eps, precision, resolve_opts(opts), theta,
                      static_cast<cudaStream_t>(stream), rep);
}

fk_status fk_predict(int additive, int d, int m, const double* theta, int n_sets, int64_t n_q, const void* xq,
                     double eps, int precision, double* f, void* stream) {
  clear_error();
  if (additive) {
    if (d < 2 || d > 16 || m < 0 || n_sets < 1 || n_q < 1 || !theta || !xq || !f)
      return set_error(FK_EINVAL, "bad additive prediction arguments");
    if (!(eps >= 1e-14 && eps <= 1e-1)) return set_error(FK_EINVAL, "eps = %g outside [1e-14, 1e-1]", eps);
    if (precision != FK_FP64 && precision != FK_MIXED) return set_error(FK_EINVAL, "unknown precision %d", precision);
    FK_TRY(capture_check(static_cast<cudaStream_t>(stream), true, false, "fk_predict"));
    return predict_additive(d, m, theta, n_sets, n_q, xq, eps, precision, f, static_cast<cudaStream_t>(stream));
  }
  return fk_type2(d, m, theta, n_sets, n_q, xq, eps, precision, f, stream);
}

}  // extern "C"

// ---------------------------------------------------------------- streaming sums
// The moments T_j and right-hand sides b_k of Sec. 2.3 are sums over points, so a
// sample larger than device memory is spread chunk by chunk onto fine grids that
// live between calls; the transform, penalty and solve then run once.
struct fk_accum {
  int d = 1, m = 0, nt = 0, precision = FK_MIXED;
  double eps = 1e-6;
  fk_opts o{};
  fk::EsPlan p;
  int64_t n_total = 0;
  double* grid = nullptr;    // [1 + nt][N^d], fp64
  double* corr = nullptr;    // [2 kmax + 1]
  unsigned* flags = nullptr;
  int device = 0;
  // fk_accum_add_host: two device staging buffers of stage_pts points each ((d + nt)
  // rows), the stream their copies run on, and per buffer the event of its copy's
  // arrival and the event after which its last spread no longer reads it
  void* stage[2] = {nullptr, nullptr};
  int64_t stage_pts = 0;
  cudaStream_t copy_st = nullptr;
  cudaEvent_t landed[2] = {nullptr, nullptr};
  cudaEvent_t freed[2] = {nullptr, nullptr};
};

namespace fk {

__global__ void k_add_grid(int64_t total, const double* src, double* dst) {
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dst[t] += src[t];
}

static fk_status accum_flags(fk_accum* a, cudaStream_t st) {
  unsigned h = 0;
  FK_CUDA(cudaMemcpyAsync(&h, a->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  FK_CUDA(cudaStreamSynchronize(st));
  if (h & FLAG_RANGE) return set_error(FK_ERANGE, "a point lies outside [-3 pi, 3 pi)");
  if (h & FLAG_TIMEOUT) return set_error(FK_ETIMEOUT, "a bounded device wait gave up");
  if (h) return set_error(FK_EINTERNAL, "device flag 0x%x", h);
  return FK_OK;
}

}  // namespace fk

extern "C" {

fk_status fk_accum_create(int d, int m, int n_targets, double eps, int precision, const fk_opts* opts,
                          fk_accum** out, void* stream) {
  clear_error();
  if (!out) return set_error(FK_EINVAL, "null output handle");
  *out = nullptr;
  FK_TRY(check_common(d, 1, m, eps, precision));
  if (n_targets < 0 || n_targets > 1024) return set_error(FK_EINVAL, "n_targets = %d outside [0, 1024]", n_targets);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, false, false, "fk_accum_create"));
  fk_accum* a = new fk_accum();
  a->d = d;
  a->m = m;
  a->nt = n_targets;
  a->precision = precision;
  a->eps = eps;
  a->o = resolve_opts(opts);
  cudaGetDevice(&a->device);
  fk_status rc = make_es_plan(d, 2 * m, eps, a->o.upsampfac, &a->p);
  const int64_t G = ipow(a->p.N, d) * (1 + n_targets);
  if (rc == FK_OK && cudaMalloc(&a->grid, sizeof(double) * G) != cudaSuccess)
    rc = set_error(FK_ENOMEM, "accumulator grids (%lld doubles)", (long long)G);
  if (rc == FK_OK && cudaMalloc(&a->corr, sizeof(double) * (2 * static_cast<size_t>(a->p.kmax) + 1)) != cudaSuccess)
    rc = set_error(FK_ENOMEM, "correction factors");
  if (rc == FK_OK && cudaMalloc(&a->flags, sizeof(unsigned)) != cudaSuccess) rc = set_error(FK_ENOMEM, "flags");
  if (rc == FK_OK) rc = es_correction(a->p, a->corr, st);
  if (rc == FK_OK && cudaMemsetAsync(a->grid, 0, sizeof(double) * G, st) != cudaSuccess)
    rc = set_error(FK_ECUDA, "memset");
  if (rc == FK_OK && cudaMemsetAsync(a->flags, 0, sizeof(unsigned), st) != cudaSuccess)
    rc = set_error(FK_ECUDA, "memset");
  if (rc != FK_OK) {
    cudaGetLastError();
    cudaFree(a->grid);
    cudaFree(a->corr);
    cudaFree(a->flags);
    delete a;
    return rc;
  }
  *out = a;
  return FK_OK;
}

fk_status fk_accum_add(fk_accum* a, int64_t n, const void* x, const void* y, const unsigned* y_absmax, void* stream) {
  clear_error();
  if (!a) return set_error(FK_EINVAL, "null accumulator");
  if (n < 0) return set_error(FK_EINVAL, "n = %lld < 0", (long long)n);
  if (n == 0) return FK_OK;
  if (!x || (a->nt > 0 && !y)) return set_error(FK_EINVAL, "null points or targets");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, false, false, "fk_accum_add"));
  NvtxRange range("fk accum add");
  Scratch scr(st);
  const EsPlan& p = a->p;
  if (a->precision == FK_MIXED && a->d == 1 && a->o.spread != FK_SPREAD_ATOMIC &&
      spread1d_fixed_supported(p, a->nt, true)) {
    FK_TRY(spread1d_fixed(p, n, static_cast<const float*>(x), static_cast<const float*>(y), a->nt, true, y_absmax,
                          a->grid, true, a->flags, st, scr, a->o.autotune != 0,
                          a->o.spread != FK_SPREAD_FIXED_SHARED));
  } else {
    const int64_t G = ipow(p.N, a->d) * (1 + a->nt);
    double* tmp = nullptr;
    FK_TRY(scr.alloc(&tmp, G));
    FK_TRY(spread_any(p, a->precision, a->o, n, x, y, a->nt, true, tmp, a->flags, st, scr));
    k_add_grid<<<grid_for(G, 256), 256, 0, st>>>(G, tmp, a->grid); note_launch();
    FK_CUDA(cudaGetLastError());
  }
  a->n_total += n;
  return FK_OK;
}

fk_status fk_accum_add_host(fk_accum* a, int64_t n, const void* x, const void* y, int64_t chunk, void* stream) {
  clear_error();
  if (!a) return set_error(FK_EINVAL, "null accumulator");
  if (n < 0) return set_error(FK_EINVAL, "n = %lld < 0", (long long)n);
  if (chunk < 0) return set_error(FK_EINVAL, "chunk = %lld < 0", (long long)chunk);
  if (n == 0) return FK_OK;
  if (!x || (a->nt > 0 && !y)) return set_error(FK_EINVAL, "null points or targets");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, false, false, "fk_accum_add_host"));
  NvtxRange range("fk accum add host");
  const int64_t C = std::min(n, chunk > 0 ? chunk : FK_HOST_CHUNK_DEFAULT);
  const size_t es = a->precision == FK_FP64 ? sizeof(double) : sizeof(float);
  const int rows = a->d + a->nt;
  if (!a->copy_st) {
    FK_CUDA(cudaStreamCreateWithFlags(&a->copy_st, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
      FK_CUDA(cudaEventCreateWithFlags(&a->landed[b], cudaEventDisableTiming));
      FK_CUDA(cudaEventCreateWithFlags(&a->freed[b], cudaEventDisableTiming));
    }
  }
  if (a->stage_pts < C) {
    // earlier spreads may still read the old buffers
    for (int b = 0; b < 2; ++b) FK_CUDA(cudaEventSynchronize(a->freed[b]));
    for (int b = 0; b < 2; ++b) {
      cudaFree(a->stage[b]);
      a->stage[b] = nullptr;
    }
    a->stage_pts = 0;
    for (int b = 0; b < 2; ++b)
      if (cudaMalloc(&a->stage[b], es * rows * static_cast<size_t>(C)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(a->stage[0]);
        a->stage[0] = nullptr;
        return set_error(FK_ENOMEM, "staging buffers (2 x %lld points)", (long long)C);
      }
    a->stage_pts = C;
  }
  const char* xh = static_cast<const char*>(x);
  const char* yh = static_cast<const char*>(y);
  for (int64_t i = 0, p0 = 0; p0 < n; ++i, p0 += C) {
    const int b = static_cast<int>(i & 1);
    const int64_t cnt = std::min(C, n - p0);
    char* dst = static_cast<char*>(a->stage[b]);
    // one copy per row of the chunk (coordinates, then targets), each landing contiguous
    FK_CUDA(cudaStreamWaitEvent(a->copy_st, a->freed[b], 0));
    for (int r = 0; r < rows; ++r) {
      const char* src = r < a->d ? xh + es * (static_cast<size_t>(r) * n + p0)
                                 : yh + es * (static_cast<size_t>(r - a->d) * n + p0);
      FK_CUDA(cudaMemcpyAsync(dst + es * static_cast<size_t>(r) * cnt, src, es * cnt, cudaMemcpyHostToDevice,
                              a->copy_st));
    }
    FK_CUDA(cudaEventRecord(a->landed[b], a->copy_st));
    FK_CUDA(cudaStreamWaitEvent(st, a->landed[b], 0));
    FK_TRY(fk_accum_add(a, cnt, dst, a->nt ? dst + es * static_cast<size_t>(a->d) * cnt : nullptr, nullptr, stream));
    FK_CUDA(cudaEventRecord(a->freed[b], st));
  }
  return FK_OK;
}

fk_status fk_accum_system(fk_accum* a, double* T, double* b, int64_t* n_total, void* stream) {
  clear_error();
  if (!a) return set_error(FK_EINVAL, "null accumulator");
  if (a->n_total < 1) return set_error(FK_EINVAL, "no points added");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, false, false, "fk_accum_system"));
  Scratch scr(st);
  const double inv_n = 1.0 / static_cast<double>(a->n_total);
  if (T) FK_TRY(modes_any(a->p, a->precision, a->grid, 0, 1, 2 * a->m, a->corr, inv_n, T, st, scr));
  if (b && a->nt > 0) FK_TRY(modes_any(a->p, a->precision, a->grid, 1, a->nt, a->m, a->corr, inv_n, b, st, scr));
  if (n_total) *n_total = a->n_total;
  return accum_flags(a, st);
}

fk_status fk_accum_fit_sobolev(fk_accum* a, double s, int penalty, const double* lambdas, int n_lambda,
                               double* theta, void* stream, fk_report* rep) {
  clear_error();
  if (!a || !theta || !lambdas || n_lambda < 1 || a->nt < 1) return set_error(FK_EINVAL, "bad accumulator fit arguments");
  if (penalty != FK_PEN_SOBOLEV && penalty != FK_PEN_LOWBIAS) return set_error(FK_EINVAL, "unknown penalty");
  if (s < 0) return set_error(FK_EINVAL, "s < 0");
  for (int i = 0; i < n_lambda; ++i)
    if (!(lambdas[i] >= 0.0)) return set_error(FK_EINVAL, "lambda[%d] = %g < 0", i, lambdas[i]);
  if (a->n_total < 1) return set_error(FK_EINVAL, "no points added");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, false, false, "fk_accum_fit_sobolev"));
  Scratch scr(st);
  Flags fl(st);
  FK_TRY(fl.init(scr));
  Timer tm(st, rep != nullptr);
  tm.mark();
  const int d = a->d, m = a->m;
  const int64_t D = ipow(2 * m + 1, d), M2 = ipow(4 * m + 1, d);
  double *T = nullptr, *b = nullptr, *W = nullptr;
  FK_TRY(scr.alloc(&T, 2 * M2));
  FK_TRY(scr.alloc(&b, 2 * D * a->nt));
  FK_TRY(scr.alloc(&W, D * n_lambda));
  const double inv_n = 1.0 / static_cast<double>(a->n_total);
  FK_TRY(modes_any(a->p, a->precision, a->grid, 0, 1, 2 * m, a->corr, inv_n, T, st, scr));
  FK_TRY(modes_any(a->p, a->precision, a->grid, 1, a->nt, m, a->corr, inv_n, b, st, scr));
  tm.mark();
  FK_TRY(penalty_weights(d, m, penalty, s, a->o.sobolev_c0, lambdas, n_lambda, 0.0, 0, nullptr, nullptr, W, st));
  int iters = 0;
  double rr = 0;
  FK_TRY(solve_system(d, m, T, W, n_lambda, b, a->nt, a->o, theta, st, scr, fl.dev, &iters, rep ? &rr : nullptr));
  tm.mark();
  FK_TRY(fl.check());
  FK_TRY(accum_flags(a, st));
  if (rep) {
    *rep = fk_report{};
    rep->ms_fft = tm.ms(0, 1);
    rep->ms_solve = tm.ms(1, 2);
    rep->ms_total = tm.ms(0, 2);
    rep->cg_iters = iters;
    rep->rel_residual = rr;
    rep->n_used = a->n_total;
    rep->fine_grid = a->p.N;
    rep->kernel_width = a->p.w;
  }
  return FK_OK;
}

fk_status fk_accum_reset(fk_accum* a, void* stream) {
  clear_error();
  if (!a) return set_error(FK_EINVAL, "null accumulator");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, false, false, "fk_accum_reset"));
  const int64_t G = ipow(a->p.N, a->d) * (1 + a->nt);
  FK_CUDA(cudaMemsetAsync(a->grid, 0, sizeof(double) * G, st));
  FK_CUDA(cudaMemsetAsync(a->flags, 0, sizeof(unsigned), st));
  a->n_total = 0;
  return FK_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- accumulator state
// Host image of an accumulator: a fixed header, then the fp64 grids [1 + n_targets][N^d]
// as stored on the device.
namespace fk {
namespace {
struct AccumHeader {
  char magic[8];  // "FKACCUM1"
  int32_t d, m, n_targets, precision, N, w;
  double eps;
  int64_t n_total;
  uint32_t flags, reserved;
  int64_t grid_doubles;
};
static_assert(sizeof(AccumHeader) == 64, "header layout");
const char kAccumMagic[8] = {'F', 'K', 'A', 'C', 'C', 'U', 'M', '1'};

int64_t accum_grid_doubles(const fk_accum* a) { return ipow(a->p.N, a->d) * (1 + a->nt); }

fk_status accum_check_state(const fk_accum* a, const void* buf, size_t len, const AccumHeader** out) {
  if (!buf || len < sizeof(AccumHeader)) return set_error(FK_EINVAL, "state buffer too short");
  const AccumHeader* h = static_cast<const AccumHeader*>(buf);
  if (std::memcmp(h->magic, kAccumMagic, 8) != 0) return set_error(FK_EINVAL, "not an accumulator state");
  if (h->d != a->d || h->m != a->m || h->n_targets != a->nt || h->precision != a->precision || h->N != a->p.N ||
      h->w != a->p.w || h->eps != a->eps)
    return set_error(FK_EINVAL, "state of another accumulator shape (d=%d m=%d targets=%d precision=%d eps=%g)", h->d,
                     h->m, h->n_targets, h->precision, h->eps);
  if (h->grid_doubles != accum_grid_doubles(a) ||
      len < sizeof(AccumHeader) + sizeof(double) * static_cast<size_t>(h->grid_doubles))
    return set_error(FK_EINVAL, "state buffer holds %zu bytes, the grids need more", len);
  *out = h;
  return FK_OK;
}

__global__ void k_or_flag(unsigned* flags, unsigned v) { atomicOr(flags, v); }
}  // namespace
}  // namespace fk

extern "C" {

size_t fk_accum_state_bytes(const fk_accum* a) {
  if (!a) return 0;
  return sizeof(AccumHeader) + sizeof(double) * static_cast<size_t>(accum_grid_doubles(a));
}

fk_status fk_accum_save(fk_accum* a, void* buf, size_t cap, void* stream) {
  clear_error();
  if (!a || !buf) return set_error(FK_EINVAL, "null accumulator or buffer");
  if (cap < fk_accum_state_bytes(a)) return set_error(FK_EINVAL, "state needs %zu bytes, buffer has %zu",
                                                      fk_accum_state_bytes(a), cap);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, false, false, "fk_accum_save"));
  AccumHeader h{};
  std::memcpy(h.magic, kAccumMagic, 8);
  h.d = a->d;
  h.m = a->m;
  h.n_targets = a->nt;
  h.precision = a->precision;
  h.N = a->p.N;
  h.w = a->p.w;
  h.eps = a->eps;
  h.n_total = a->n_total;
  h.grid_doubles = accum_grid_doubles(a);
  unsigned char* out = static_cast<unsigned char*>(buf);
  FK_CUDA(cudaMemcpyAsync(&h.flags, a->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  FK_CUDA(cudaMemcpyAsync(out + sizeof(AccumHeader), a->grid, sizeof(double) * h.grid_doubles,
                          cudaMemcpyDeviceToHost, st));
  FK_CUDA(cudaStreamSynchronize(st));
  std::memcpy(out, &h, sizeof(h));
  return FK_OK;
}

fk_status fk_accum_load(fk_accum* a, const void* buf, size_t len, void* stream) {
  clear_error();
  if (!a) return set_error(FK_EINVAL, "null accumulator");
  const AccumHeader* h = nullptr;
  FK_TRY(accum_check_state(a, buf, len, &h));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, false, false, "fk_accum_load"));
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  FK_CUDA(cudaMemcpyAsync(a->grid, in + sizeof(AccumHeader), sizeof(double) * h->grid_doubles,
                          cudaMemcpyHostToDevice, st));
  const unsigned fl = h->flags;
  FK_CUDA(cudaMemcpyAsync(a->flags, &fl, sizeof(unsigned), cudaMemcpyHostToDevice, st));
  FK_CUDA(cudaStreamSynchronize(st));
  a->n_total = h->n_total;
  return FK_OK;
}

fk_status fk_accum_add_state(fk_accum* a, const void* buf, size_t len, void* stream) {
  clear_error();
  if (!a) return set_error(FK_EINVAL, "null accumulator");
  const AccumHeader* h = nullptr;
  FK_TRY(accum_check_state(a, buf, len, &h));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, false, false, "fk_accum_add_state"));
  Scratch scr(st);
  double* tmp = nullptr;
  FK_TRY(scr.alloc(&tmp, static_cast<size_t>(h->grid_doubles)));
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  FK_CUDA(cudaMemcpyAsync(tmp, in + sizeof(AccumHeader), sizeof(double) * h->grid_doubles, cudaMemcpyHostToDevice,
                          st));
  k_add_grid<<<grid_for(h->grid_doubles, 256), 256, 0, st>>>(h->grid_doubles, tmp, a->grid); note_launch();
  FK_CUDA(cudaGetLastError());
  if (h->flags) {
    k_or_flag<<<1, 1, 0, st>>>(a->flags, h->flags); note_launch();
    FK_CUDA(cudaGetLastError());
  }
  FK_CUDA(cudaStreamSynchronize(st));  // the host buffer is read before return
  a->n_total += h->n_total;
  return FK_OK;
}

fk_status fk_accum_destroy(fk_accum* a) {
  clear_error();
  if (!a) return FK_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != a->device) cudaSetDevice(a->device);
  cudaFree(a->grid);
  cudaFree(a->corr);
  cudaFree(a->flags);
  if (a->copy_st) {
    for (int b = 0; b < 2; ++b) cudaEventSynchronize(a->freed[b]);
    cudaStreamSynchronize(a->copy_st);
    for (int b = 0; b < 2; ++b) {
      cudaFree(a->stage[b]);
      cudaEventDestroy(a->landed[b]);
      cudaEventDestroy(a->freed[b]);
    }
    cudaStreamDestroy(a->copy_st);
  }
  if (cur != a->device) cudaSetDevice(cur);
  delete a;
  return FK_OK;
}

}  // extern "C"
