// Exponential-of-semicircle (ES) kernel plan and its Fourier-transform correction.
//
// The type-1 sums of Sec. 2.3 are evaluated as a non-uniform FFT: strengths are
// spread onto an upsampled periodic grid with psi(x) = phi(x / alpha),
// phi(z) = exp(beta (sqrt(1 - z^2) - 1)), alpha = w h / 2, h = 2 pi / N; the grid
// is Fourier transformed and each mode divided by the kernel's transform
//   Psi_hat(j) = alpha * int_{-1}^{1} phi(z) cos(j alpha z) dz,
// so that sum_i c_i e^{-i j x_i} ~= (-1)^j h / Psi_hat(j) * DFT(g)[j mod N]
// (Poisson summation; grid node l sits at x_l = -pi + l h).  The integral is
// evaluated by Gauss-Legendre quadrature whose nodes come from Newton's method on
// the Legendre recurrence, all in fp64 on the device.
#include "fk_internal.cuh"
#include "es_poly.cuh"

#include <map>
#include <mutex>
#include <tuple>

namespace fk {

static int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

fk_status make_es_plan(int d, int kmax, double eps, double upsampfac, EsPlan* p) {
  if (kmax < 0) return set_error(FK_EINVAL, "kmax < 0");
  const int K = 2 * kmax + 1;
  if (upsampfac <= 1.0) upsampfac = 1.9;
  int N = next_pow2(static_cast<int>(std::ceil(upsampfac * K)));
  if (N < 16) N = 16;
  // width from the ES error estimate exp(-pi w sqrt(1 - 1/sigma)), with half a tap of
  // margin: measured relative l2 errors then stay within ~2 eps over sigma in [2, 5]
  int w = 0;
  for (int iter = 0; iter < 4; ++iter) {
    const double sigma = static_cast<double>(N) / K;
    w = static_cast<int>(std::ceil(std::log(1.0 / eps) / (M_PI * std::sqrt(1.0 - 1.0 / sigma)) + 0.5));
    if (w < 2) w = 2;
    if (w > 16) w = 16;
    if (N >= 2 * w) break;
    N *= 2;
  }
  const double sigma = static_cast<double>(N) / K;
  p->d = d;
  p->N = N;
  p->w = w;
  p->sigma = sigma;
  p->kmax = kmax;
  p->beta = 0.97 * M_PI * (1.0 - 0.5 / sigma) * w;
  return FK_OK;
}

constexpr int GL_Q = 128;  // quadrature nodes on [-1, 1]

// Gauss-Legendre nodes and weights: one thread per root.
__global__ void k_gauss_legendre(double* nodes, double* weights) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= GL_Q) return;
  const int q = GL_Q;
  double x = cos(M_PI * (i + 0.75) / (q + 0.5));
  double dp = 1.0;
  for (int it = 0; it < 30; ++it) {
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= q; ++k) {
      const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    // p1 = P_q(x), p0 = P_{q-1}(x);  P_q'(x) = q (x P_q - P_{q-1}) / (x^2 - 1)
    dp = q * (x * p1 - p0) / (x * x - 1.0);
    const double dx = p1 / dp;
    x -= dx;
    if (fabs(dx) < 1e-14) break;  // quadratic convergence: the last step already polished x
  }
  {
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= q; ++k) {
      const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = q * (x * p1 - p0) / (x * x - 1.0);
  }
  nodes[i] = x;
  weights[i] = 2.0 / ((1.0 - x * x) * dp * dp);
}

__global__ void k_es_correction(int kmax, int N, int w, double beta, const double* nodes,
                                const double* weights, double* corr) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t > 2 * kmax) return;
  const int j = t - kmax;
  const double h = 2.0 * M_PI / N;
  const double alpha = 0.5 * w * h;
  double acc = 0.0;
  for (int q = 0; q < GL_Q; ++q) {
    const double z = nodes[q];
    const double phi = exp(beta * (sqrt(1.0 - z * z) - 1.0));
    acc += weights[q] * phi * cos(j * alpha * z);
  }
  const double psi_hat = alpha * acc;
  const double sgn = (j & 1) ? -1.0 : 1.0;
  corr[t] = sgn * h / psi_hat;
}

static fk_status es_correction_compute(const EsPlan& p, double* corr, cudaStream_t st) {
  double* nw = nullptr;
  FK_CUDA(cudaMallocAsync(&nw, 2 * GL_Q * sizeof(double), st));
  k_gauss_legendre<<<1, GL_Q, 0, st>>>(nw, nw + GL_Q); note_launch();
  const int K = 2 * p.kmax + 1;
  k_es_correction<<<(K + 127) / 128, 128, 0, st>>>(p.kmax, p.N, p.w, p.beta, nw, nw + GL_Q, corr); note_launch();
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(nw, st);
  if (e != cudaSuccess) return set_error(FK_ECUDA, "es_correction launch: %s", cudaGetErrorString(e));
  return FK_OK;
}

// Correction factors depend only on (kmax, N, w, beta): computed once per device and
// plan, kept for the life of the process, and copied into the caller's buffer.
fk_status es_correction(const EsPlan& p, double* corr, cudaStream_t st) {
  int dev = 0;
  FK_CUDA(cudaGetDevice(&dev));
  const size_t bytes = sizeof(double) * (2 * static_cast<size_t>(p.kmax) + 1);
  const auto key = std::make_tuple(dev, p.kmax, p.N, p.w, p.beta);
  static std::mutex mtx;
  static std::map<std::tuple<int, int, int, int, double>, double*> cache;
  double* src = nullptr;
  {
    std::lock_guard<std::mutex> lock(mtx);
    auto it = cache.find(key);
    if (it != cache.end()) {
      src = it->second;
    } else {
      FK_CUDA(cudaMalloc(&src, bytes));
      // during a capture the table is made on a stream of its own, outside the graph
      cudaStream_t cs = st;
      if (capture_ctx() && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(src);
        return set_error(FK_ECUDA, "es_correction stream");
      }
      fk_status stt = es_correction_compute(p, src, cs);
      if (stt == FK_OK && cudaStreamSynchronize(cs) != cudaSuccess) stt = set_error(FK_ECUDA, "es_correction sync");
      if (cs != st) cudaStreamDestroy(cs);
      if (stt != FK_OK) {
        cudaFree(src);
        return stt;
      }
      cache.emplace(key, src);
    }
  }
  FK_CUDA(cudaMemcpyAsync(corr, src, bytes, cudaMemcpyDeviceToDevice, st));
  return FK_OK;
}

}  // namespace fk

namespace fk {

fk_status es_gl_nodes_into(double* gl, cudaStream_t st) {
  k_gauss_legendre<<<1, GL_Q, 0, st>>>(gl, gl + GL_Q); note_launch();
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}

// As es_correction, from quadrature nodes already in device memory (es_gl_nodes_into).
fk_status es_correction_from_nodes(const EsPlan& p, double* corr, const double* gl, cudaStream_t st) {
  const int K = 2 * p.kmax + 1;
  k_es_correction<<<(K + 127) / 128, 128, 0, st>>>(p.kmax, p.N, p.w, p.beta, gl, gl + GL_Q, corr); note_launch();
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}

fk_status preload_es_kernels() {
  cudaFuncAttributes fa;
  FK_CUDA(cudaFuncGetAttributes(&fa, k_gauss_legendre));
  FK_CUDA(cudaFuncGetAttributes(&fa, k_es_correction));
  return FK_OK;
}

int es_gl_nodes() { return GL_Q; }

}  // namespace fk

namespace fk {

// Chebyshev interpolation of each tap at the 9 Chebyshev points of (-1/2, 1/2), then
// the change of basis to powers of g (T_0 = 1, T_1 = u, T_{k+1} = 2 u T_k - T_{k-1},
// u = 2 g), in fp64.
EsPoly es_poly(int w, double beta) {
  constexpr int PMAX = 8;
  const int P = es_poly_deg(w), NP = P + 1;
  EsPoly out{};
  const double c = 0.5 * (w - 1);
  auto phi = [&](double z) {
    const double t = 1.0 - z * z;
    return t > 0.0 ? std::exp(beta * (std::sqrt(t) - 1.0)) : 0.0;
  };
  // monomial coefficients of T_k(u), k = 0..P
  double Tm[PMAX + 1][PMAX + 1] = {};
  Tm[0][0] = 1.0;
  Tm[1][1] = 1.0;
  for (int k = 1; k + 1 < NP; ++k)
    for (int j = 0; j < NP; ++j) Tm[k + 1][j] = (j > 0 ? 2.0 * Tm[k][j - 1] : 0.0) - Tm[k - 1][j];
  for (int a = 0; a < (w + 1) / 2 && a < ES_POLY_MAXW / 2; ++a) {
    double v[PMAX + 1], ch[PMAX + 1], mono[PMAX + 1] = {};
    for (int j = 0; j < NP; ++j) {
      const double u = std::cos(M_PI * (j + 0.5) / NP);
      v[j] = phi((a - c - 0.5 * u) * 2.0 / w);
    }
    for (int k = 0; k < NP; ++k) {
      double s = 0.0;
      for (int j = 0; j < NP; ++j) s += v[j] * std::cos(M_PI * k * (j + 0.5) / NP);
      ch[k] = (k == 0 ? 1.0 : 2.0) * s / NP;
    }
    for (int k = 0; k < NP; ++k)
      for (int j = 0; j < NP; ++j) mono[j] += ch[k] * Tm[k][j];
    // powers of u = 2 g  ->  powers of g
    for (int j = 0; j < NP; ++j) mono[j] *= std::ldexp(1.0, j);
    for (int j = 0; 2 * j < NP; ++j) out.e[a][j] = static_cast<float>(mono[2 * j]);
    for (int j = 0; 2 * j + 1 < NP; ++j) out.o[a][j] = static_cast<float>(mono[2 * j + 1]);
    for (int j = 0; j < 4; ++j) out.eo[a][j] = make_float2(out.e[a][j], out.o[a][j]);
  }
  return out;
}

}  // namespace fk
