// Held-out-loss hypergradient by the adjoint of Eq. 2 (not in the paper).
//
// With A = Toep(T) + diag W, theta = A^{-1} b and residual r = f(x^v) - y^v:
//   L = mean(r^2)
//   g_k = (1/n_v) sum_i r_i e^{-i<k, x^v_i>}      (type-1 of the residuals)
//   z = A^{-1} g                                  (adjoint solve; A is Hermitian)
//   dL/dW_k = -2 Re(conj(z_k) theta_k)
//   dL/dY_i = (2/n) Re sum_k z_k e^{+i<k, X_i>}    (type-2 of z at the training points)
// and the chain rule from dL/dW to the penalty's parameters
//   W_k = lambda (c0 + |k|^{2s}) + mu |P(ik)|^2,  P(ik) = sum_t a_t prod_l (i k_l)^{alpha_tl}.
#include "fk_internal.cuh"

#include <vector>

namespace fk {
namespace {

template <typename R>
__global__ void k_residual(int64_t n, const double* f, const R* yv, R* r, double* sum) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double e = f[i] - static_cast<double>(yv[i]);
    r[i] = static_cast<R>(e);
    acc += e * e;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(sum, s);
  }
}

__global__ void k_dW(int64_t D, const double* z, const double* theta, double* dW) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < D;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dW[k] = -2.0 * (z[2 * k] * theta[2 * k] + z[2 * k + 1] * theta[2 * k + 1]);
}

__global__ void k_scale(int64_t n, double s, double* v) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    v[i] *= s;
}

struct PdeTermsG {
  int n_terms;
  int alpha[16][3];
  double a[16];
};

// out[0] = dL/dlambda, out[1] = dL/ds, out[2] = dL/dmu, out[3 + t] = dL/da_t (one CTA, fp64)
__global__ void k_penalty_grads(int d, int m, double s, double c0, double lambda, double mu, PdeTermsG pde,
                                const double* dW, double* out) {
  const int K = 2 * m + 1;
  int64_t D = 1;
  for (int l = 0; l < d; ++l) D *= K;
  const int nout = 3 + pde.n_terms;
  double acc[3 + 16];
  for (int j = 0; j < nout; ++j) acc[j] = 0.0;
  for (int64_t q = threadIdx.x; q < D; q += blockDim.x) {
    int k[3] = {0, 0, 0};
    int64_t qq = q;
    for (int l = d - 1; l >= 0; --l) {
      k[l] = static_cast<int>(qq % K) - m;
      qq /= K;
    }
    double r2 = 0.0;
    for (int l = 0; l < d; ++l) r2 += static_cast<double>(k[l]) * k[l];
    const double pw = r2 > 0.0 ? pow(r2, s) : 0.0;
    const double g = dW[q];
    acc[0] += g * (c0 + pw);
    acc[1] += (r2 > 0.0) ? g * lambda * pw * log(r2) : 0.0;
    if (pde.n_terms > 0) {
      double pre = 0.0, pim = 0.0;
      double mre[16], mim[16];
      for (int t = 0; t < pde.n_terms; ++t) {
        double tre = 1.0, tim = 0.0;
        for (int l = 0; l < d; ++l)
          for (int e = 0; e < pde.alpha[t][l]; ++e) {  // multiply by i k_l
            const double nre = -tim * k[l], nim = tre * k[l];
            tre = nre;
            tim = nim;
          }
        mre[t] = tre;
        mim[t] = tim;
        pre += pde.a[t] * tre;
        pim += pde.a[t] * tim;
      }
      acc[2] += g * (pre * pre + pim * pim);
      for (int t = 0; t < pde.n_terms; ++t) acc[3 + t] += g * 2.0 * mu * (pre * mre[t] + pim * mim[t]);
    }
  }
  __shared__ double red[3 + 16][32];
  for (int j = 0; j < nout; ++j) {
    double v = acc[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[j][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < nout) {
    double v = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
    out[threadIdx.x] = v;
  }
}

template <typename R>
fk_status hypergrad_impl(int d, int64_t n, const R* x, int64_t n_v, const R* xv, const R* yv, int m, const double* T,
                         const double* W, const double* theta, double eps, int precision, const fk_opts& o,
                         double* loss, double* dW, double* dY, cudaStream_t st) {
  Scratch scr(st);
  unsigned* flags = nullptr;
  FK_TRY(scr.alloc(&flags, 1));
  FK_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned), st));
  EsPlan p;
  FK_TRY(make_es_plan(d, m, eps, o.upsampfac, &p));
  double* corr = nullptr;
  FK_TRY(scr.alloc(&corr, 2 * static_cast<size_t>(m) + 1));
  FK_TRY(es_correction(p, corr, st));
  int64_t D = 1, G = 1;
  for (int l = 0; l < d; ++l) {
    D *= (2 * m + 1);
    G *= p.N;
  }
  // predictions at the validation points and residuals
  double *f = nullptr, *sum = nullptr, *g = nullptr, *z = nullptr, *grid = nullptr;
  R* r = nullptr;
  FK_TRY(scr.alloc(&f, static_cast<size_t>(n_v)));
  FK_TRY(scr.alloc(&r, static_cast<size_t>(n_v)));
  FK_TRY(scr.alloc(&sum, 1));
  FK_TRY(scr.alloc(&g, 2 * static_cast<size_t>(D)));
  FK_TRY(scr.alloc(&z, 2 * static_cast<size_t>(D)));
  FK_TRY(scr.alloc(&grid, static_cast<size_t>(G)));
  FK_TRY(type2_eval<R>(p, m, theta, 1, n_v, xv, corr, f, flags, st, scr));
  FK_CUDA(cudaMemsetAsync(sum, 0, sizeof(double), st));
  k_residual<R><<<grid_for(n_v, 256, 148 * 8), 256, 0, st>>>(n_v, f, yv, r, sum); note_launch();
  FK_CUDA(cudaGetLastError());
  // g = type1(xv, r) / n_v, with the fits' spreader (binned for the mixed path in 2-D)
  FK_TRY(spread_any(p, precision, o, n_v, xv, r, 1, false, grid, flags, st, scr));
  if (precision == FK_FP64)
    FK_TRY(grid_to_modes<double>(p, grid, 0, 1, m, corr, 1.0 / static_cast<double>(n_v), g, st, scr));
  else
    FK_TRY(grid_to_modes<float>(p, grid, 0, 1, m, corr, 1.0 / static_cast<double>(n_v), g, st, scr));
  // adjoint solve
  int iters = 0;
  double rr = 0.0;
  FK_TRY(solve_system(d, m, T, W, 1, g, 1, o, z, st, scr, flags, &iters, &rr));
  k_dW<<<grid_for(D, 256), 256, 0, st>>>(D, z, theta, dW); note_launch();
  FK_CUDA(cudaGetLastError());
  if (dY) {
    FK_TRY(type2_eval<R>(p, m, z, 1, n, x, corr, dY, flags, st, scr));
    k_scale<<<grid_for(n, 256), 256, 0, st>>>(n, 2.0 / static_cast<double>(n), dY); note_launch();
    FK_CUDA(cudaGetLastError());
  }
  double hsum = 0.0;
  unsigned hflags = 0;
  FK_CUDA(cudaMemcpyAsync(&hsum, sum, sizeof(double), cudaMemcpyDeviceToHost, st));
  FK_CUDA(cudaMemcpyAsync(&hflags, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  FK_CUDA(cudaStreamSynchronize(st));
  if (hflags & FLAG_RANGE) return set_error(FK_ERANGE, "a point lies outside [-3 pi, 3 pi)");
  if (hflags & FLAG_NOTPD) return set_error(FK_ENOTPD, "Cholesky met a non-positive pivot");
  if (hflags) return set_error(FK_EINTERNAL, "device flag 0x%x", hflags);
  *loss = hsum / static_cast<double>(n_v);
  return FK_OK;
}

// forward half: predictions at the validation points, residual r (precision R) and the loss
template <typename R>
fk_status heldout_loss_impl(int d, int m, const double* theta, int64_t n_v, const R* xv, const R* yv, double eps,
                            const fk_opts& o, double* loss, R* r, cudaStream_t st) {
  Scratch scr(st);
  unsigned* flags = nullptr;
  FK_TRY(scr.alloc(&flags, 1));
  FK_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned), st));
  EsPlan p;
  FK_TRY(make_es_plan(d, m, eps, o.upsampfac, &p));
  double *corr = nullptr, *f = nullptr, *sum = nullptr;
  FK_TRY(scr.alloc(&corr, 2 * static_cast<size_t>(m) + 1));
  FK_TRY(es_correction(p, corr, st));
  FK_TRY(scr.alloc(&f, static_cast<size_t>(n_v)));
  FK_TRY(scr.alloc(&sum, 1));
  FK_TRY(type2_eval<R>(p, m, theta, 1, n_v, xv, corr, f, flags, st, scr));
  FK_CUDA(cudaMemsetAsync(sum, 0, sizeof(double), st));
  k_residual<R><<<grid_for(n_v, 256, 148 * 8), 256, 0, st>>>(n_v, f, yv, r, sum); note_launch();
  FK_CUDA(cudaGetLastError());
  double hsum = 0.0;
  unsigned hflags = 0;
  FK_CUDA(cudaMemcpyAsync(&hsum, sum, sizeof(double), cudaMemcpyDeviceToHost, st));
  FK_CUDA(cudaMemcpyAsync(&hflags, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  FK_CUDA(cudaStreamSynchronize(st));
  FK_TRY(flags_status(hflags));
  *loss = hsum / static_cast<double>(n_v);
  return FK_OK;
}

// backward half: g = type1(xv, r) / n_v, z = A^{-1} g, dW = -2 Re(conj(z) theta), zy = zscale z
template <typename R>
fk_status adjoint_impl(int d, int m, int64_t n_v, const R* xv, const R* r, const double* T, const double* W,
                       const double* theta, double eps, int precision, const fk_opts& o, double zscale, double* dW,
                       double* zy, cudaStream_t st) {
  Scratch scr(st);
  unsigned* flags = nullptr;
  FK_TRY(scr.alloc(&flags, 1));
  FK_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned), st));
  EsPlan p;
  FK_TRY(make_es_plan(d, m, eps, o.upsampfac, &p));
  int64_t D = 1, G = 1;
  for (int l = 0; l < d; ++l) {
    D *= (2 * m + 1);
    G *= p.N;
  }
  double *corr = nullptr, *g = nullptr, *z = nullptr, *grid = nullptr;
  FK_TRY(scr.alloc(&corr, 2 * static_cast<size_t>(m) + 1));
  FK_TRY(es_correction(p, corr, st));
  FK_TRY(scr.alloc(&g, 2 * static_cast<size_t>(D)));
  FK_TRY(scr.alloc(&z, 2 * static_cast<size_t>(D)));
  FK_TRY(scr.alloc(&grid, static_cast<size_t>(G)));
  // g = type1(xv, r) / n_v, with the fits' spreader (binned for the mixed path in 2-D)
  FK_TRY(spread_any(p, precision, o, n_v, xv, r, 1, false, grid, flags, st, scr));
  if (precision == FK_FP64)
    FK_TRY(grid_to_modes<double>(p, grid, 0, 1, m, corr, 1.0 / static_cast<double>(n_v), g, st, scr));
  else
    FK_TRY(grid_to_modes<float>(p, grid, 0, 1, m, corr, 1.0 / static_cast<double>(n_v), g, st, scr));
  int iters = 0;
  double rr = 0.0;
  FK_TRY(solve_system(d, m, T, W, 1, g, 1, o, z, st, scr, flags, &iters, &rr));
  k_dW<<<grid_for(D, 256), 256, 0, st>>>(D, z, theta, dW); note_launch();
  FK_CUDA(cudaGetLastError());
  if (zy) {
    FK_CUDA(cudaMemcpyAsync(zy, z, sizeof(double) * 2 * D, cudaMemcpyDeviceToDevice, st));
    k_scale<<<grid_for(2 * D, 256), 256, 0, st>>>(2 * D, zscale, zy); note_launch();
    FK_CUDA(cudaGetLastError());
  }
  unsigned hflags = 0;
  FK_CUDA(cudaMemcpyAsync(&hflags, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  FK_CUDA(cudaStreamSynchronize(st));
  return flags_status(hflags);
}

fk_opts hyper_opts(const fk_opts* opts) {
  fk_opts o;
  fk_default_opts(&o);
  if (opts) o = *opts;
  if (o.cg_tol <= 0) o.cg_tol = 1e-13;
  if (o.cg_maxit <= 0) o.cg_maxit = 1000;
  if (o.upsampfac <= 1.0) o.upsampfac = 1.9;
  return o;
}

}  // namespace
}  // namespace fk

using namespace fk;

extern "C" {

fk_status fk_heldout_loss(int d, int m, const double* theta, int64_t n_v, const void* xv, const void* yv, double eps,
                          int precision, const fk_opts* opts, double* loss, void* r, void* stream) {
  clear_error();
  FK_TRY(check_common(d, n_v, m, eps, precision));
  if (!theta || !xv || !yv || !loss || !r) return set_error(FK_EINVAL, "null pointer argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, false, false, "fk_heldout_loss"));
  const fk_opts o = hyper_opts(opts);
  if (precision == FK_FP64)
    return heldout_loss_impl<double>(d, m, theta, n_v, static_cast<const double*>(xv), static_cast<const double*>(yv),
                                     eps, o, loss, static_cast<double*>(r), st);
  return heldout_loss_impl<float>(d, m, theta, n_v, static_cast<const float*>(xv), static_cast<const float*>(yv), eps,
                                  o, loss, static_cast<float*>(r), st);
}

fk_status fk_adjoint(int d, int m, int64_t n_v, const void* xv, const void* r, const double* T, const double* W,
                     const double* theta, double eps, int precision, const fk_opts* opts, double zscale, double* dW,
                     double* zy, void* stream) {
  clear_error();
  FK_TRY(check_common(d, n_v, m, eps, precision));
  if (!xv || !r || !T || !W || !theta || !dW) return set_error(FK_EINVAL, "null pointer argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, false, false, "fk_adjoint"));
  const fk_opts o = hyper_opts(opts);
  if (precision == FK_FP64)
    return adjoint_impl<double>(d, m, n_v, static_cast<const double*>(xv), static_cast<const double*>(r), T, W, theta,
                                eps, precision, o, zscale, dW, zy, st);
  return adjoint_impl<float>(d, m, n_v, static_cast<const float*>(xv), static_cast<const float*>(r), T, W, theta, eps,
                             precision, o, zscale, dW, zy, st);
}

fk_status fk_hypergrad(int d, int64_t n, const void* x, int64_t n_v, const void* xv, const void* yv, int m,
                       const double* T, const double* W, const double* theta, double eps, int precision,
                       const fk_opts* opts, double* loss, double* dW, double* dY, void* stream) {
  clear_error();
  if (d < 1 || d > 3) return set_error(FK_EINVAL, "d = %d: transforms are built for d in {1, 2, 3}", d);
  if (n < 1 || n_v < 1 || m < 0) return set_error(FK_EINVAL, "bad sizes n=%lld n_v=%lld m=%d", (long long)n,
                                                 (long long)n_v, m);
  if (!(eps >= 1e-14 && eps <= 1e-1)) return set_error(FK_EINVAL, "eps = %g outside [1e-14, 1e-1]", eps);
  if (!x || !xv || !yv || !T || !W || !theta || !loss || !dW) return set_error(FK_EINVAL, "null pointer argument");
  fk_opts o;
  fk_default_opts(&o);
  if (opts) o = *opts;
  if (o.cg_tol <= 0) o.cg_tol = 1e-13;
  if (o.cg_maxit <= 0) o.cg_maxit = 1000;
  if (o.upsampfac <= 1.0) o.upsampfac = 1.9;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, false, false, "fk_hypergrad"));
  if (precision == FK_FP64)
    return hypergrad_impl<double>(d, n, static_cast<const double*>(x), n_v, static_cast<const double*>(xv),
                                  static_cast<const double*>(yv), m, T, W, theta, eps, precision, o, loss, dW, dY, st);
  if (precision == FK_MIXED)
    return hypergrad_impl<float>(d, n, static_cast<const float*>(x), n_v, static_cast<const float*>(xv),
                                 static_cast<const float*>(yv), m, T, W, theta, eps, precision, o, loss, dW, dY, st);
  return set_error(FK_EINVAL, "unknown precision %d", precision);
}

fk_status fk_penalty_grads(int d, int m, double s, double c0, double lambda, double mu, int n_terms, const int* alpha,
                           const double* a, const double* dW, double* out, void* stream) {
  clear_error();
  if (d < 1 || d > 3 || m < 0 || !dW || !out) return set_error(FK_EINVAL, "bad penalty-gradient arguments");
  if (n_terms < 0 || n_terms > 16 || (n_terms > 0 && (!alpha || !a))) return set_error(FK_EINVAL, "bad PDE terms");
  PdeTermsG pde{};
  pde.n_terms = n_terms;
  for (int t = 0; t < n_terms; ++t) {
    pde.a[t] = a[t];
    for (int l = 0; l < d; ++l) {
      if (alpha[t * d + l] < 0 || alpha[t * d + l] > 32) return set_error(FK_EINVAL, "alpha out of range");
      pde.alpha[t][l] = alpha[t * d + l];
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, false, false, "fk_penalty_grads"));
  double* dout = nullptr;
  FK_CUDA(cudaMallocAsync(&dout, sizeof(double) * (3 + n_terms), st));
  k_penalty_grads<<<1, 256, 0, st>>>(d, m, s, c0, lambda, mu, pde, dW, dout); note_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof(double) * (3 + n_terms), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(dout, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(FK_ECUDA, "penalty gradients: %s", cudaGetErrorString(e));
  return FK_OK;
}

}  // extern "C"
