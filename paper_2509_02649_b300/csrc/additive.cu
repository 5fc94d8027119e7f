// Low-bias additive model (Prop. 5.1, Sec. 5): block Gram, right-hand side, solve and
// additive prediction.
//
// Blocks of Sigma (each (2m+1) x (2m+1), k in -m..m):
//   (l, l)    Toeplitz in the 1-D moments T^(l)_j = (1/n) sum_i e^{-i j X_il}, |j| <= 2m
//   (l1, l2)  (1/n) sum_i e^{-i k1 X_il1} e^{+i k2 X_il2}: a 2-D type-1 transform of ones at
//             the points (X_l1, -X_l2) (Sec. 5, Complexity); (l2, l1) is its conjugate
//             transpose
// right-hand side b_l[k] = (1/n) sum_i Y_i e^{-i k X_il}, and theta = (Sigma + lambda I)^{-1} b
// by a dense FP64 Cholesky solve of size d(2m+1) with one refinement step.
#include <functional>

#include "fk_internal.cuh"

namespace fk {
namespace {

template <typename R>
__global__ void k_pair_points(int64_t n, const R* x, int l1, int l2, R* out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    out[i] = x[l1 * n + i];
    out[n + i] = -x[l2 * n + i];
  }
}

// A[(l1,k1),(l2,k2)], row-major, D = d K, plus lambda on the diagonal
__global__ void k_additive_gram(int d, int m, const double* T1, const double* Bp, double lambda, double* A) {
  const int K = 2 * m + 1, M2 = 4 * m + 1;
  const int64_t D = static_cast<int64_t>(d) * K;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < D * D;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t row = t / D, col = t - (t / D) * D;
    const int l1 = static_cast<int>(row / K), k1 = static_cast<int>(row % K);
    const int l2 = static_cast<int>(col / K), k2 = static_cast<int>(col % K);
    double re, im;
    if (l1 == l2) {
      const int j = k1 - k2 + 2 * m;  // moment index of k1 - k2
      re = T1[2 * (static_cast<int64_t>(l1) * M2 + j)];
      im = T1[2 * (static_cast<int64_t>(l1) * M2 + j) + 1];
      if (k1 == k2) re += lambda;
    } else {
      const int a = l1 < l2 ? l1 : l2, b = l1 < l2 ? l2 : l1;
      const int64_t pair = static_cast<int64_t>(a) * d - static_cast<int64_t>(a) * (a + 1) / 2 + (b - a - 1);
      const double* blk = Bp + 2 * pair * K * K;
      if (l1 < l2) {
        re = blk[2 * (static_cast<int64_t>(k1) * K + k2)];
        im = blk[2 * (static_cast<int64_t>(k1) * K + k2) + 1];
      } else {  // conjugate transpose of block (l2, l1)
        re = blk[2 * (static_cast<int64_t>(k2) * K + k1)];
        im = -blk[2 * (static_cast<int64_t>(k2) * K + k1) + 1];
      }
    }
    A[2 * t] = re;
    A[2 * t + 1] = im;
  }
}

__global__ void k_add_into(int64_t n, const double* a, double* acc) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    acc[i] += a[i];
}

// Non-blocking streams per device and host thread for work forked off the caller's
// stream (joined back before the call returns), created on first use and kept: a stream
// that joined a capture must outlive it, and per-thread streams keep one thread's
// capture from taking in another thread's work.
constexpr int NSIDE = 3;
fk_status side_streams(cudaStream_t out[NSIDE]) {
  constexpr int MAXD = 64;
  thread_local cudaStream_t tab[MAXD][NSIDE] = {};
  int dev = 0;
  FK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAXD) return set_error(FK_EINTERNAL, "side streams: device %d", dev);
  for (int k = 0; k < NSIDE; ++k) {
    if (!tab[dev][k]) FK_CUDA(cudaStreamCreateWithFlags(&tab[dev][k], cudaStreamNonBlocking));
    out[k] = tab[dev][k];
  }
  return FK_OK;
}

template <typename R>
fk_status fit_additive_impl(int d, int64_t n, const R* x, const R* y, int nt, int m, const double* lambdas,
                            int n_lambda, double eps, int precision, const fk_opts& o, double* theta,
                            cudaStream_t st, fk_report* rep) {
  Scratch scr(st);
  CaptureCtx* cap = capture_ctx();
  unsigned* flags = nullptr;
  if (cap) {
    flags = cap->flags;
  } else {
    FK_TRY(scr.alloc(&flags, 1));
    FK_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned), st));
  }
  const int K = 2 * m + 1, M2 = 4 * m + 1;
  const int64_t Dall = static_cast<int64_t>(d) * K;
  const int npairs = d * (d - 1) / 2;
  cudaEvent_t ev[4] = {};
  if (rep)
    for (int i = 0; i < 4; ++i) cudaEventCreate(&ev[i]);
  if (rep) cudaEventRecord(ev[0], st);

  // 1-D moments and right-hand sides per coordinate
  EsPlan p1;
  FK_TRY(make_es_plan(1, 2 * m, eps, o.upsampfac, &p1));
  double *corr1 = nullptr, *grid1 = nullptr, *T1 = nullptr, *bt = nullptr, *rhs = nullptr;
  FK_TRY(scr.alloc(&corr1, 2 * static_cast<size_t>(p1.kmax) + 1));
  FK_TRY(scr.alloc(&grid1, static_cast<size_t>(p1.N) * (1 + nt)));
  FK_TRY(scr.alloc(&T1, 2 * static_cast<size_t>(d) * M2));
  FK_TRY(scr.alloc(&bt, 2 * static_cast<size_t>(nt) * K));
  FK_TRY(scr.alloc(&rhs, 2 * static_cast<size_t>(nt) * Dall));
  FK_TRY(es_correction(p1, corr1, st));
  const double inv_n = 1.0 / static_cast<double>(n);
  const bool fixed1d = (precision == FK_MIXED) && o.spread != FK_SPREAD_ATOMIC && spread1d_fixed_supported(p1, nt, true);
  // deterministic sums (fk_opts.deterministic): 64-bit fixed-point spreading wherever the
  // 1-D fixed-point spreader does not apply
  const bool det = o.deterministic != 0;
  unsigned* amax = nullptr;
  if (fixed1d) {
    FK_TRY(scr.alloc(&amax, static_cast<size_t>(nt)));
    FK_TRY(absmax_channels(n, reinterpret_cast<const float*>(y), nt, amax, st));
  }
  NvtxRange stage_range("fk additive 1-D");
  // The 1-D transforms run on side stream 2, forked here and joined after the pair
  // transforms (which they do not touch), so that their short launches (FFT,
  // extraction, copies) overlap the pairs' long ones.  Every exit after the fork joins
  // first: the scratch memory they use is released on the caller's stream.
  cudaStream_t side[NSIDE];
  FK_TRY(side_streams(side));
  cudaEvent_t ev_fork = nullptr, ev_1d = nullptr;
  FK_CUDA(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
  FK_CUDA(cudaEventCreateWithFlags(&ev_1d, cudaEventDisableTiming));
  struct EvGuard {
    cudaEvent_t* e[2];
    ~EvGuard() {
      for (cudaEvent_t* p : e) cudaEventDestroy(*p);
    }
  } ev_guard{{&ev_fork, &ev_1d}};
  FK_CUDA(cudaEventRecord(ev_fork, st));
  FK_CUDA(cudaStreamWaitEvent(side[2], ev_fork, 0));
  auto run1d = [&](cudaStream_t s1) -> fk_status {
    for (int l = 0; l < d; ++l) {
      Scratch inner(s1);  // released (stream-ordered) after each coordinate
      if (fixed1d)
        FK_TRY(spread1d_fixed(p1, n, reinterpret_cast<const float*>(x + static_cast<int64_t>(l) * n),
                              reinterpret_cast<const float*>(y), nt, true, amax, grid1, false, flags, s1, inner,
                              o.autotune != 0, o.spread != FK_SPREAD_FIXED_SHARED));
      else if (det)
        FK_TRY(spread_deterministic<R>(p1, n, x + static_cast<int64_t>(l) * n, y, nt, true, grid1, flags, s1, inner));
      else
        FK_TRY(spread_atomic<R>(p1, n, x + static_cast<int64_t>(l) * n, y, nt, true, grid1, flags, s1));
      if (precision == FK_FP64) {
        FK_TRY(grid_to_modes<double>(p1, grid1, 0, 1, 2 * m, corr1, inv_n, T1 + 2 * static_cast<int64_t>(l) * M2, s1, inner));
        FK_TRY(grid_to_modes<double>(p1, grid1, 1, nt, m, corr1, inv_n, bt, s1, inner));
      } else {
        FK_TRY(grid_to_modes<float>(p1, grid1, 0, 1, 2 * m, corr1, inv_n, T1 + 2 * static_cast<int64_t>(l) * M2, s1, inner));
        FK_TRY(grid_to_modes<float>(p1, grid1, 1, nt, m, corr1, inv_n, bt, s1, inner));
      }
      // rhs[t][l K + k] = bt[t][k]
      FK_CUDA(cudaMemcpy2DAsync(rhs + 2 * static_cast<int64_t>(l) * K, sizeof(double) * 2 * Dall, bt,
                                sizeof(double) * 2 * K, sizeof(double) * 2 * K, nt, cudaMemcpyDeviceToDevice, s1));
    }
    return FK_OK;
  };
  {
    const fk_status rc1 = run1d(side[2]);
    const cudaError_t e1 = cudaEventRecord(ev_1d, side[2]);
    if (rc1 != FK_OK || e1 != cudaSuccess) {
      if (e1 == cudaSuccess) cudaStreamWaitEvent(st, ev_1d, 0);
      else cudaStreamSynchronize(side[2]);
      if (rc1 != FK_OK) return rc1;
      FK_CUDA(e1);
    }
  }
  // from here every return joins side stream 2 first
  auto join1d = [&]() { cudaStreamWaitEvent(st, ev_1d, 0); };
  struct Join {
    std::function<void()> f;
    bool done = false;
    void operator()() {
      if (!done) f();
      done = true;
    }
    ~Join() { (*this)(); }
  } join{join1d};
  // 2-D blocks of ones at (X_l1, -X_l2)
  EsPlan p2;
  FK_TRY(make_es_plan(2, m, eps, o.upsampfac, &p2));
  double *corr2 = nullptr, *grid2 = nullptr, *Bp = nullptr;
  R* pts = nullptr;
  FK_TRY(scr.alloc(&corr2, 2 * static_cast<size_t>(p2.kmax) + 1));
  FK_TRY(scr.alloc(&grid2, static_cast<size_t>(p2.N) * p2.N));
  FK_TRY(scr.alloc(&Bp, 2 * static_cast<size_t>(npairs > 0 ? npairs : 1) * K * K));
  // mixed path: one partition per first coordinate l1 serves all its partners (row
  // owners), or else one partition per pair reading X_l1 and X_l2 in place; otherwise
  // the pair's points are gathered into (X_l1, -X_l2) rows first
  const bool mixed_binned = precision == FK_MIXED && o.spread != FK_SPREAD_ATOMIC && !det;
  const bool rowpairs = mixed_binned && additive_pairs_supported(p2, d, n);
  const bool binned2 = mixed_binned && !rowpairs && spread_binned_supported(p2, 0, true);
  if (!binned2 && !rowpairs) FK_TRY(scr.alloc(&pts, 2 * static_cast<size_t>(n)));
  FK_TRY(es_correction(p2, corr2, st));
  stage_range.next("fk additive pairs");
  if (rowpairs) {
    // Partitions on the caller's stream, in order; accumulation l1 on side stream l1 & 1
    // (record set l1 & 1), so that the next partition and accumulation fill the SMs that
    // an accumulation's last wave leaves idle (128 owners x P partners of one-SM CTAs),
    // instead of each launch ending in a part-filled wave.  Partition l1 + 2 waits for
    // accumulation l1, which reads the same record set.
    const int64_t NN = static_cast<int64_t>(p2.N) * p2.N;
    AddPairState S;
    double* pg = nullptr;
    FK_TRY(scr.alloc(&pg, static_cast<size_t>(npairs) * NN));
    FK_TRY(additive_pairs_begin(p2, d, n, reinterpret_cast<const float*>(x), flags, st, scr, &S));
    cudaEvent_t ev_part = nullptr, ev_done[2] = {};
    FK_CUDA(cudaEventCreateWithFlags(&ev_part, cudaEventDisableTiming));
    FK_CUDA(cudaEventCreateWithFlags(&ev_done[0], cudaEventDisableTiming));
    FK_CUDA(cudaEventCreateWithFlags(&ev_done[1], cudaEventDisableTiming));
    bool used[2] = {false, false};
    fk_status rc = FK_OK;
    // a failed call inside the fork ends the loop (no early return: the side streams are
    // joined below first)
    auto ck = [&](cudaError_t e, const char* what) {
      if (e != cudaSuccess && rc == FK_OK)
        rc = set_error(FK_ECUDA, "additive pairs: %s failed: %s", what, cudaGetErrorString(e));
      return rc == FK_OK;
    };
    int pair0 = 0;
    for (int l1 = 0; l1 + 1 < d && rc == FK_OK; ++l1) {
      const int s = l1 & 1;
      if (used[s] && !ck(cudaStreamWaitEvent(st, ev_done[s], 0), "cudaStreamWaitEvent")) break;
      rc = additive_pairs_part(S, l1, flags, st);
      if (rc != FK_OK) break;
      if (!ck(cudaEventRecord(ev_part, st), "cudaEventRecord")) break;
      if (!ck(cudaStreamWaitEvent(side[s], ev_part, 0), "cudaStreamWaitEvent")) break;
      rc = additive_pairs_acc(S, l1, pg + pair0 * NN, flags, side[s]);
      // the pair blocks of l1 from their grids, on the same side stream
      for (int l2 = l1 + 1; l2 < d && rc == FK_OK; ++l2) {
        Scratch inner(side[s]);
        const int pair = pair0 + (l2 - l1 - 1);
        rc = grid_to_modes<float>(p2, pg + pair * NN, 0, 1, m, corr2, inv_n,
                                  Bp + 2 * static_cast<int64_t>(pair) * K * K, side[s], inner);
      }
      if (cudaEventRecord(ev_done[s], side[s]) != cudaSuccess) {
        cudaStreamSynchronize(side[s]);  // cannot be joined by an event: wait for it here
        ck(cudaErrorUnknown, "cudaEventRecord");
        break;
      }
      used[s] = true;
      pair0 += d - 1 - l1;
    }
    // join the side streams (also after an error, so that nothing is left forked)
    for (int s = 0; s < 2; ++s)
      if (used[s] && cudaStreamWaitEvent(st, ev_done[s], 0) != cudaSuccess) {
        cudaStreamSynchronize(side[s]);
        ck(cudaErrorUnknown, "cudaStreamWaitEvent");
      }
    cudaEventDestroy(ev_part);
    cudaEventDestroy(ev_done[0]);
    cudaEventDestroy(ev_done[1]);
    FK_TRY(rc);
  }
  int pair = 0;
  for (int l1 = 0; l1 < d && !rowpairs; ++l1)
    for (int l2 = l1 + 1; l2 < d; ++l2, ++pair) {
      Scratch inner(st);  // released (stream-ordered) after each pair
      if (!binned2) {
        k_pair_points<R><<<grid_for(n, 256), 256, 0, st>>>(n, x, l1, l2, pts); note_launch();
        FK_CUDA(cudaGetLastError());
      }
      double* blk = Bp + 2 * static_cast<int64_t>(pair) * K * K;
      if (det) {
        FK_TRY(spread_deterministic<R>(p2, n, pts, nullptr, 0, true, grid2, flags, st, inner));
        if (precision == FK_FP64)
          FK_TRY(grid_to_modes<double>(p2, grid2, 0, 1, m, corr2, inv_n, blk, st, inner));
        else
          FK_TRY(grid_to_modes<float>(p2, grid2, 0, 1, m, corr2, inv_n, blk, st, inner));
      } else if (precision == FK_FP64) {
        FK_TRY(spread_atomic<double>(p2, n, reinterpret_cast<const double*>(pts), nullptr, 0, true, grid2, flags, st));
        FK_TRY(grid_to_modes<double>(p2, grid2, 0, 1, m, corr2, inv_n, blk, st, inner));
      } else if (binned2) {
        const float* xf = reinterpret_cast<const float*>(x);
        FK_TRY(spread_binned_xy(p2, n, xf + static_cast<int64_t>(l1) * n, xf + static_cast<int64_t>(l2) * n, -1.0f,
                                nullptr, 0, true, grid2, flags, st, inner, o.autotune != 0));
        FK_TRY(grid_to_modes<float>(p2, grid2, 0, 1, m, corr2, inv_n, blk, st, inner));
      } else {
        const float* fp = reinterpret_cast<const float*>(pts);
        FK_TRY(spread_atomic<float>(p2, n, fp, nullptr, 0, true, grid2, flags, st));
        FK_TRY(grid_to_modes<float>(p2, grid2, 0, 1, m, corr2, inv_n, blk, st, inner));
      }
    }
  join();  // the 1-D transforms
  if (rep) cudaEventRecord(ev[1], st);
  // block Gram + lambda I, dense solve per lambda (or one eigendecomposition for all)
  stage_range.next("fk additive solve");
  double* A = nullptr;
  FK_TRY(scr.alloc(&A, 2 * Dall * Dall));
  if (o.solver == FK_SOLVER_EIG) {
    if (cap) return set_error(FK_EINVAL, "the eigen route tests convergence on the host: not capturable");
    double *U = nullptr, *ev = nullptr;
    FK_TRY(scr.alloc(&U, 2 * Dall * Dall));
    FK_TRY(scr.alloc(&ev, Dall));
    k_additive_gram<<<grid_for(Dall * Dall, 256), 256, 0, st>>>(d, m, T1, Bp, 0.0, A); note_launch();
    FK_CUDA(cudaGetLastError());
    int sweeps = 0;
    FK_TRY(eig_hermitian(Dall, A, U, ev, st, scr, &sweeps));
    FK_TRY(eig_sweep_solve(Dall, U, ev, nullptr, rhs, nt, lambdas, n_lambda, theta, st, scr));
  }
  for (int li = 0; li < n_lambda && o.solver != FK_SOLVER_EIG; ++li) {
    k_additive_gram<<<grid_for(Dall * Dall, 256), 256, 0, st>>>(d, m, T1, Bp, lambdas[li], A); note_launch();
    FK_CUDA(cudaGetLastError());
    double* X = theta + 2 * static_cast<int64_t>(li) * nt * Dall;
    FK_CUDA(cudaMemcpyAsync(X, rhs, sizeof(double) * 2 * nt * Dall, cudaMemcpyDeviceToDevice, st));
    Scratch inner(st);
    FK_TRY(solve_dense(A, Dall, X, nt, o.refine_steps, st, inner, flags));
  }
  if (cap) return FK_OK;  // the graph's flag word is read by fk_graph_status
  if (rep) cudaEventRecord(ev[2], st);
  unsigned h = 0;
  FK_CUDA(cudaMemcpyAsync(&h, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  FK_CUDA(cudaStreamSynchronize(st));
  if (rep) {
    *rep = fk_report{};
    float a = 0.f, b2 = 0.f;
    cudaEventElapsedTime(&a, ev[0], ev[1]);
    cudaEventElapsedTime(&b2, ev[1], ev[2]);
    rep->ms_spread = a;
    rep->ms_solve = b2;
    rep->ms_total = a + b2;
    rep->n_used = n;
    rep->fine_grid = p2.N;
    rep->kernel_width = p2.w;
  }
  if (rep)
    for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
  return flags_status(h);
}

template <typename R>
fk_status predict_additive_impl(int d, int m, const double* theta, int n_sets, int64_t nq, const R* xq, double eps,
                                double* f, cudaStream_t st) {
  Scratch scr(st);
  CaptureCtx* cap = capture_ctx();
  unsigned* flags = nullptr;
  if (cap) {
    flags = cap->flags;
  } else {
    FK_TRY(scr.alloc(&flags, 1));
    FK_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned), st));
  }
  const int K = 2 * m + 1;
  EsPlan p;
  FK_TRY(make_es_plan(1, m, eps, 1.9, &p));
  double *corr = nullptr, *coef = nullptr, *part = nullptr;
  FK_TRY(scr.alloc(&corr, 2 * static_cast<size_t>(m) + 1));
  FK_TRY(scr.alloc(&coef, 2 * static_cast<size_t>(n_sets) * K));
  FK_TRY(scr.alloc(&part, static_cast<size_t>(n_sets) * nq));
  FK_TRY(es_correction(p, corr, st));
  FK_CUDA(cudaMemsetAsync(f, 0, sizeof(double) * n_sets * nq, st));
  for (int l = 0; l < d; ++l) {
    FK_CUDA(cudaMemcpy2DAsync(coef, sizeof(double) * 2 * K, theta + 2 * static_cast<int64_t>(l) * K,
                              sizeof(double) * 2 * d * K, sizeof(double) * 2 * K, n_sets, cudaMemcpyDeviceToDevice, st));
    FK_TRY(type2_eval<R>(p, m, coef, n_sets, nq, xq + static_cast<int64_t>(l) * nq, corr, part, flags, st, scr));
    k_add_into<<<grid_for(static_cast<int64_t>(n_sets) * nq, 256), 256, 0, st>>>(static_cast<int64_t>(n_sets) * nq,
                                                                                   part, f); note_launch();
    FK_CUDA(cudaGetLastError());
  }
  if (cap) return FK_OK;
  unsigned h = 0;
  FK_CUDA(cudaMemcpyAsync(&h, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  FK_CUDA(cudaStreamSynchronize(st));
  return flags_status(h);
}

}  // namespace

fk_status fit_additive(int d, int64_t n, const void* x, const void* y, int nt, int m, const double* lambdas,
                       int n_lambda, double eps, int precision, const fk_opts& o, double* theta, cudaStream_t st,
                       fk_report* rep) {
  if (precision == FK_FP64)
    return fit_additive_impl<double>(d, n, static_cast<const double*>(x), static_cast<const double*>(y), nt, m, lambdas,
                                     n_lambda, eps, precision, o, theta, st, rep);
  return fit_additive_impl<float>(d, n, static_cast<const float*>(x), static_cast<const float*>(y), nt, m, lambdas,
                                  n_lambda, eps, precision, o, theta, st, rep);
}

fk_status predict_additive(int d, int m, const double* theta, int n_sets, int64_t nq, const void* xq, double eps,
                           int precision, double* f, cudaStream_t st) {
  if (precision == FK_FP64)
    return predict_additive_impl<double>(d, m, theta, n_sets, nq, static_cast<const double*>(xq), eps, f, st);
  return predict_additive_impl<float>(d, m, theta, n_sets, nq, static_cast<const float*>(xq), eps, f, st);
}

}  // namespace fk
