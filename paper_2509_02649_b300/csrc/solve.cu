// Penalty diagonals, Toeplitz assembly and the FP64 solves of
//   (Toep(T) + diag W) theta = b                                   (Eq. 2, Sec. 2.3)
// Dense route: blocked right-looking complex Cholesky A = L L^H (non-positive
// pivot -> FLAG_NOTPD), triangular solves, iterative refinement.
// Iterative route: Jacobi-preconditioned conjugate gradients whose Toeplitz
// matvec runs through a circulant embedding and FFTs (Sec. 2.3, matvec via FFT),
// batched over every (penalty, right-hand side) pair.
#include "fk_internal.cuh"

#include <cstring>
#include "fft_device.cuh"

#include <map>
#include <mutex>
#include <vector>

namespace fk {

// ---------------------------------------------------------------- penalty (Sec. 3.1, 3.2, 4)
struct PdeTerms {
  int n_terms;
  int alpha[16][3];
  double a[16];
};

__device__ inline void mode_of(int64_t q, int d, int m, int* k) {
  const int K = 2 * m + 1;
  for (int l = d - 1; l >= 0; --l) {
    k[l] = static_cast<int>(q % K) - m;
    q /= K;
  }
}

// lambdas by value (a captured graph keeps launch parameters, not host memory)
constexpr int LAM_INLINE = 256;
struct LamList {
  double v[LAM_INLINE];
};

__global__ void k_penalty(int d, int m, int penalty, double s, double c0, const double* lambdas, LamList lin,
                          int n_lambda, double mu, PdeTerms pde, double* W) {
  const int K = 2 * m + 1;
  int64_t D = 1;
  for (int l = 0; l < d; ++l) D *= K;
  const int64_t total = D * n_lambda;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int li = static_cast<int>(t / D);
    const int64_t q = t - li * D;
    int k[3] = {0, 0, 0};
    mode_of(q, d, m, k);
    const double lam = lambdas ? lambdas[li] : lin.v[li];
    double wv;
    if (penalty == FK_PEN_LOWBIAS) {
      wv = lam;
    } else {
      double r2 = 0.0;
      for (int l = 0; l < d; ++l) r2 += static_cast<double>(k[l]) * k[l];
      const double pw = (r2 > 0.0) ? pow(r2, s) : 0.0;
      wv = lam * (c0 + pw);
    }
    if (pde.n_terms > 0) {
      // P(ik) = sum_t a_t prod_l (i k_l)^alpha_tl
      double pre = 0.0, pim = 0.0;
      for (int tt = 0; tt < pde.n_terms; ++tt) {
        double tre = pde.a[tt], tim = 0.0;
        for (int l = 0; l < d; ++l) {
          for (int e = 0; e < pde.alpha[tt][l]; ++e) {  // multiply by i k_l
            const double nre = -tim * k[l];
            const double nim = tre * k[l];
            tre = nre;
            tim = nim;
          }
        }
        pre += tre;
        pim += tim;
      }
      wv += mu * (pre * pre + pim * pim);
    }
    W[t] = wv;
  }
}

fk_status penalty_weights(int d, int m, int penalty, double s, double c0, const double* lambdas, int n_lambda,
                          double mu, int n_terms, const int* alpha, const double* a, double* W, cudaStream_t st) {
  if (n_terms < 0 || n_terms > 16) return set_error(FK_EINVAL, "n_terms must be in [0, 16]");
  if (d < 1 || d > 3) return set_error(FK_EINVAL, "d must be 1..3");
  PdeTerms pde{};
  pde.n_terms = n_terms;
  for (int t = 0; t < n_terms; ++t) {
    pde.a[t] = a[t];
    for (int l = 0; l < d; ++l) {
      if (alpha[t * d + l] < 0 || alpha[t * d + l] > 32) return set_error(FK_EINVAL, "alpha out of range");
      pde.alpha[t][l] = alpha[t * d + l];
    }
  }
  int64_t D = 1;
  for (int l = 0; l < d; ++l) D *= (2 * m + 1);
  LamList lin{};
  if (n_lambda <= LAM_INLINE) {
    for (int i = 0; i < n_lambda; ++i) lin.v[i] = lambdas[i];
    k_penalty<<<grid_for(D * n_lambda, 256), 256, 0, st>>>(d, m, penalty, s, c0, nullptr, lin, n_lambda, mu, pde, W);
    note_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
  }
  if (capture_ctx()) return set_error(FK_EINVAL, "more than %d lambdas in one captured call", LAM_INLINE);
  double* dl = nullptr;
  FK_CUDA(cudaMallocAsync(&dl, sizeof(double) * n_lambda, st));
  cudaError_t e = cudaMemcpyAsync(dl, lambdas, sizeof(double) * n_lambda, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_penalty<<<grid_for(D * n_lambda, 256), 256, 0, st>>>(d, m, penalty, s, c0, dl, lin, n_lambda, mu, pde, W);
    note_launch();
    e = cudaGetLastError();
  }
  cudaFreeAsync(dl, st);
  if (e != cudaSuccess) return set_error(FK_ECUDA, "penalty: %s", cudaGetErrorString(e));
  return FK_OK;
}

// ---------------------------------------------------------------- dense assembly
// A[r][c] = T_{k_r - k_c} + delta_rc W[r]
// P(ik) = sum_t a_t prod_l (i k_l)^alpha_tl for every mode (complex, interleaved)
__global__ void k_pde_symbol(int d, int m, PdeTerms pde, double* P) {
  const int K = 2 * m + 1;
  int64_t D = 1;
  for (int l = 0; l < d; ++l) D *= K;
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < D;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int k[3] = {0, 0, 0};
    mode_of(q, d, m, k);
    double pre = 0.0, pim = 0.0;
    for (int tt = 0; tt < pde.n_terms; ++tt) {
      double tre = pde.a[tt], tim = 0.0;
      for (int l = 0; l < d; ++l)
        for (int e = 0; e < pde.alpha[tt][l]; ++e) {
          const double nre = -tim * k[l];
          tim = tre * k[l];
          tre = nre;
        }
      pre += tre;
      pim += tim;
    }
    P[2 * q] = pre;
    P[2 * q + 1] = pim;
  }
}

// c_j = (2 pi)^{-d} int_box e^{-i<j,x>} dx for |j|_inf <= 2m (box in [-3 pi, 3 pi)^d)
struct Box {
  double lo[3], hi[3];
};
__global__ void k_box_moments(int d, int m, Box bx, double* c) {
  const int K2 = 4 * m + 1;
  int64_t M2 = 1;
  for (int l = 0; l < d; ++l) M2 *= K2;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < M2;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int64_t q = t;
    double re = 1.0, im = 0.0;
    for (int l = d - 1; l >= 0; --l) {
      const int j = static_cast<int>(q % K2) - 2 * m;
      q /= K2;
      double fr, fi;
      if (j == 0) {
        fr = bx.hi[l] - bx.lo[l];
        fi = 0.0;
      } else {
        // (e^{-i j hi} - e^{-i j lo}) / (-i j) = (sin(j hi) - sin(j lo)) / j + i (cos(j hi) - cos(j lo)) / j
        double sh, ch, sl, cl;
        sincos(j * bx.hi[l], &sh, &ch);
        sincos(j * bx.lo[l], &sl, &cl);
        fr = (sh - sl) / j;
        fi = (ch - cl) / j;
      }
      fr *= 0.15915494309189535;  // 1 / (2 pi)
      fi *= 0.15915494309189535;
      const double nr = re * fr - im * fi, ni = re * fi + im * fr;
      re = nr;
      im = ni;
    }
    c[2 * t] = re;
    c[2 * t + 1] = im;
  }
}

fk_status pde_symbol_vec(int d, int m, int n_terms, const int* alpha, const double* a, double* P, cudaStream_t st) {
  if (n_terms < 0 || n_terms > 16) return set_error(FK_EINVAL, "n_terms must be in [0, 16]");
  PdeTerms pde{};
  pde.n_terms = n_terms;
  for (int t = 0; t < n_terms; ++t) {
    pde.a[t] = a[t];
    for (int l = 0; l < d; ++l) {
      if (alpha[t * d + l] < 0 || alpha[t * d + l] > 32) return set_error(FK_EINVAL, "alpha out of range");
      pde.alpha[t][l] = alpha[t * d + l];
    }
  }
  int64_t D = 1;
  for (int l = 0; l < d; ++l) D *= (2 * m + 1);
  k_pde_symbol<<<grid_for(D, 256), 256, 0, st>>>(d, m, pde, P); note_launch();
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}

fk_status box_moments(int d, int m, const double* lo, const double* hi, double* c, cudaStream_t st) {
  if (d < 1 || d > 3) return set_error(FK_EINVAL, "box moments: d = %d", d);
  Box bx{};
  for (int l = 0; l < d; ++l) {
    if (!(lo[l] < hi[l]) || !(lo[l] >= -3.0 * M_PI) || !(hi[l] <= 3.0 * M_PI))
      return set_error(FK_EINVAL, "box side %d: need -3 pi <= lo < hi <= 3 pi", l);
    bx.lo[l] = lo[l];
    bx.hi[l] = hi[l];
  }
  int64_t M2 = 1;
  for (int l = 0; l < d; ++l) M2 *= (4 * m + 1);
  k_box_moments<<<grid_for(M2, 256), 256, 0, st>>>(d, m, bx, c); note_launch();
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}

// dense operator part: A[k][k'] += mu conj(P_k) c_{k-k'} P_k'
__global__ void k_assemble_op(int d, int m, const double* c, const double* P, double mu, double* A) {
  const int K = 2 * m + 1, K2 = 4 * m + 1;
  int64_t D = 1;
  for (int l = 0; l < d; ++l) D *= K;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < D * D;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = t / D, cc = t - r * D;
    int kr[3] = {0, 0, 0}, kc[3] = {0, 0, 0};
    mode_of(r, d, m, kr);
    mode_of(cc, d, m, kc);
    int64_t jidx = 0;
    for (int l = 0; l < d; ++l) jidx = jidx * K2 + (kr[l] - kc[l] + 2 * m);
    const double cr = c[2 * jidx], ci = c[2 * jidx + 1];
    const double pr = P[2 * r], pi = -P[2 * r + 1];  // conj(P_k)
    const double qr = P[2 * cc], qi = P[2 * cc + 1];
    // conj(P_k) c P_k'
    const double ar = pr * cr - pi * ci, ai = pr * ci + pi * cr;
    A[2 * t] += mu * (ar * qr - ai * qi);
    A[2 * t + 1] += mu * (ar * qi + ai * qr);
  }
}

// Jacobi diagonal of the operator form: W_k + mu |P_k|^2 Re c_0
__global__ void k_op_diag(int64_t D, int n_w, const double* W, const double* P, const double* c0, double mu,
                          double* Wd) {
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < D * n_w;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t q = t % D;
    Wd[t] = W[t] + mu * (P[2 * q] * P[2 * q] + P[2 * q + 1] * P[2 * q + 1]) * c0[0];
  }
}

__global__ void k_assemble(int d, int m, const double* T, const double* W, double* A) {
  const int K = 2 * m + 1, K2 = 4 * m + 1;
  int64_t D = 1;
  for (int l = 0; l < d; ++l) D *= K;
  const int64_t total = D * D;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = t / D, c = t - (t / D) * D;
    int kr[3] = {0, 0, 0}, kc[3] = {0, 0, 0};
    mode_of(r, d, m, kr);
    mode_of(c, d, m, kc);
    int64_t idx = 0;
    for (int l = 0; l < d; ++l) idx = idx * K2 + (kr[l] - kc[l] + 2 * m);
    double re = T[2 * idx], im = T[2 * idx + 1];
    if (r == c) re += W[r];
    A[2 * t] = re;
    A[2 * t + 1] = im;
  }
}


__global__ void k_inv_sqrt(int64_t n, const double* w, double* out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[i] = 1.0 / sqrt(w[i]);
}

fk_status assemble_toeplitz(int d, int m, const double* T, const double* W, double* A, cudaStream_t st) {
  int64_t D = 1;
  for (int l = 0; l < d; ++l) D *= (2 * m + 1);
  k_assemble<<<grid_for(D * D, 256), 256, 0, st>>>(d, m, T, W, A); note_launch();
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}

fk_status inv_sqrt(int64_t n, const double* w, double* out, cudaStream_t st) {
  k_inv_sqrt<<<grid_for(n, 256), 256, 0, st>>>(n, w, out); note_launch();
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}

// ---------------------------------------------------------------- Cholesky
constexpr int NB = 32;

// Factor the nb x nb diagonal block in place (one CTA).  Step j takes the pivot, scales
// column j and updates the trailing lower triangle; the entries (i, k), k > j, i >= k,
// listed with k descending, make step j's active set a prefix of one table, so only
// warps with work issue (this part's FP64 pipe costs the same per warp instruction
// whatever the number of active lanes).
__global__ void k_chol_diag(double* A, int64_t D, int kb, int nb, unsigned* flags) {
  __shared__ cd s[NB][NB + 1];
  __shared__ double rdiag[NB];                  // 1 / L_jj: one FP64 division per pivot
  __shared__ unsigned short tab[NB * (NB + 1) / 2];  // (i << 8) | k
  const int tid = threadIdx.x;
  for (int t = tid; t < nb * nb; t += blockDim.x) {
    const int i = t / nb, j = t % nb;
    const double* p = A + 2 * ((kb + i) * D + (kb + j));
    s[i][j] = cd{p[0], p[1]};
  }
  for (int t = tid; t < (nb - 1) * nb / 2; t += blockDim.x) {
    int k = nb - 1, before = 0;  // group k holds the nb - k entries (k .. nb - 1, k)
    while (t >= before + (nb - k)) {
      before += nb - k;
      --k;
    }
    tab[t] = static_cast<unsigned short>(((k + t - before) << 8) | k);
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {
      double piv = s[j][j].x;
      if (!(piv > 0.0)) {
        atomicOr(flags, FLAG_NOTPD);
        piv = 1.0;
      }
      const double r = rsqrt(piv);  // one FP64 sequence for both the pivot and its inverse
      s[j][j] = cd{piv * r, 0.0};
      rdiag[j] = r;
    }
    __syncthreads();
    const double inv = rdiag[j];
    for (int i = j + 1 + tid; i < nb; i += blockDim.x) s[i][j] = cscale(s[i][j], inv);
    __syncthreads();
    const int act = (nb - 1 - j) * (nb - j) / 2;  // entries with k > j
    for (int t = tid; t < act; t += blockDim.x) {
      const int i = tab[t] >> 8, k = tab[t] & 0xFF;
      s[i][k] = cfma_cj(cd{-s[i][j].x, -s[i][j].y}, s[k][j], s[i][k]);
    }
    __syncthreads();
  }
  for (int t = tid; t < nb * nb; t += blockDim.x) {
    const int i = t / nb, j = t % nb;
    double* p = A + 2 * ((kb + i) * D + (kb + j));
    if (j <= i) {
      p[0] = s[i][j].x;
      p[1] = s[i][j].y;
    } else {
      p[0] = 0.0;
      p[1] = 0.0;
    }
  }
}

// Inverse of the factored diagonal block, one column per CTA (one warp) so that the
// FP64 work spreads over nb SMs: L v = e_c by right-looking substitution, lane i
// holding v_i; after v_p is known every lane i > p takes away L_ip v_p.
// Linv: [NB][NB] complex, zero above the diagonal and beyond nb.
static_assert(NB == 32, "one lane per row of a diagonal block");
__global__ void k_chol_inv(const double* A, int64_t D, int kb, int nb, double* Linv) {
  __shared__ cd s[NB][NB + 1];
  const int c = blockIdx.x, lane = threadIdx.x;
  for (int t = lane; t < nb * nb; t += 32) {
    const int i = t / nb, j = t % nb;
    const double* p = A + 2 * ((kb + i) * D + (kb + j));
    s[i][j] = (j <= i) ? cd{p[0], p[1]} : cd{0.0, 0.0};
  }
  __syncwarp();
  const double rd = (lane < nb) ? 1.0 / s[lane][lane].x : 0.0;
  cd acc = cd{(lane == c) ? 1.0 : 0.0, 0.0};
  cd v = cd{0.0, 0.0};
  for (int p = c; p < nb; ++p) {
    if (lane == p) v = cscale(acc, rd);
    const cd vp = cd{__shfl_sync(0xffffffffu, v.x, p), __shfl_sync(0xffffffffu, v.y, p)};
    if (lane > p && lane < nb) acc = cfma(cd{-s[lane][p].x, -s[lane][p].y}, vp, acc);
  }
  // column c of the inverse: rows lane >= c
  const cd val = (lane < nb && lane >= c) ? v : cd{0.0, 0.0};
  Linv[2 * (lane * NB + c)] = val.x;
  Linv[2 * (lane * NB + c) + 1] = val.y;
}

// columns c >= nb of the inverse are zero
__global__ void k_chol_inv_pad(int nb, double* Linv) {
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x)
    if (t % NB >= nb) {
      Linv[2 * t] = 0.0;
      Linv[2 * t + 1] = 0.0;
    }
}

// A22[i][j] -= sum_p L21[i][p] conj(L21[j][p]),  lower triangle, TT x TT tiles
template <int TT>
__global__ void __launch_bounds__(256) k_chol_update(double* A, int64_t D, int kb, int nb) {
  const int64_t base = kb + nb;
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (tj > ti) return;
  const int64_t i0 = base + static_cast<int64_t>(ti) * TT, j0 = base + static_cast<int64_t>(tj) * TT;
  __shared__ cd Li[TT][NB + 1], Lj[TT][NB + 1];
  for (int t = threadIdx.x; t < TT * nb; t += blockDim.x) {
    const int r = t / nb, p = t % nb;
    const int64_t gi = i0 + r, gj = j0 + r;
    Li[r][p] = (gi < D) ? cd{A[2 * (gi * D + kb + p)], A[2 * (gi * D + kb + p) + 1]} : cd{0, 0};
    Lj[r][p] = (gj < D) ? cd{A[2 * (gj * D + kb + p)], A[2 * (gj * D + kb + p) + 1]} : cd{0, 0};
  }
  __syncthreads();
  for (int t = threadIdx.x; t < TT * TT; t += blockDim.x) {
    const int r = t / TT, c = t % TT;
    const int64_t gi = i0 + r, gj = j0 + c;
    if (gi >= D || gj >= D || gj > gi) continue;
    cd a0 = cd{0, 0}, a1 = cd{0, 0};
    int p = 0;
    for (; p + 1 < nb; p += 2) {
      a0 = cfma_cj(Li[r][p], Lj[c][p], a0);
      a1 = cfma_cj(Li[r][p + 1], Lj[c][p + 1], a1);
    }
    if (p < nb) a0 = cfma_cj(Li[r][p], Lj[c][p], a0);
    double* q = A + 2 * (gi * D + gj);
    q[0] -= a0.x + a1.x;
    q[1] -= a0.y + a1.y;
  }
}

// panel rows i >= kb + nb: L21 = A21 (L11^{-1})^H, i.e. x_j = sum_p a_p conj(Linv[j][p]);
// one CTA per 32 rows, the 32 x 32 inverse and the row tile in shared memory
constexpr int PANEL_ROWS = 8;  // rows per CTA: spreads the FP64 work over more SMs
__global__ void k_chol_panel_mm(double* A, int64_t D, int kb, int nb, const double* Linv) {
  __shared__ cd Li[NB][NB + 1], At[PANEL_ROWS][NB + 1];
  const int64_t r0 = kb + nb + static_cast<int64_t>(blockIdx.x) * PANEL_ROWS;
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int i = t / NB, j = t % NB;
    Li[i][j] = cd{Linv[2 * t], Linv[2 * t + 1]};
  }
  for (int t = threadIdx.x; t < PANEL_ROWS * NB; t += blockDim.x) {
    const int i = t / NB, j = t % NB;
    const int64_t row = r0 + i;
    At[i][j] = (row < D && j < nb) ? cd{A[2 * (row * D + kb + j)], A[2 * (row * D + kb + j) + 1]} : cd{0, 0};
  }
  __syncthreads();
  for (int t = threadIdx.x; t < PANEL_ROWS * NB; t += blockDim.x) {
    const int r = t / NB, j = t % NB;
    const int64_t row = r0 + r;
    if (row >= D || j >= nb) continue;
    cd acc = cd{0, 0};
    for (int p = 0; p <= j; ++p) acc = cfma_cj(At[r][p], Li[j][p], acc);
    A[2 * (row * D + kb + j)] = acc.x;
    A[2 * (row * D + kb + j) + 1] = acc.y;
  }
}

// Blocked right-looking Cholesky A = L L^H in place (lower triangle; the strict upper
// triangle is zeroed).  linv: [ceil(D / NB)][NB][NB] complex, receives the inverse of
// every diagonal block (zero-padded); the panel update and the triangular solves use
// them as products.
static int64_t linv_blocks(int64_t D) { return (D + NB - 1) / NB; }

static fk_status cholesky(double* A, int64_t D, unsigned* flags, cudaStream_t st, double* linv) {
  int sms = 0, dev = 0;
  FK_CUDA(cudaGetDevice(&dev));
  FK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  for (int kb = 0; kb < D; kb += NB) {
    const int nb = static_cast<int>(std::min<int64_t>(NB, D - kb));
    const int64_t rest = D - kb - nb;
    double* li = linv + 2 * static_cast<int64_t>(kb / NB) * NB * NB;
    k_chol_diag<<<1, 256, 0, st>>>(A, D, kb, nb, flags); note_launch();
    if (nb < NB) {
      k_chol_inv_pad<<<1, 256, 0, st>>>(nb, li); note_launch();
    }
    k_chol_inv<<<nb, 32, 0, st>>>(A, D, kb, nb, li); note_launch();
    if (rest > 0) {
      k_chol_panel_mm<<<static_cast<int>((rest + PANEL_ROWS - 1) / PANEL_ROWS), 256, 0, st>>>(A, D, kb, nb, li);
      note_launch();
      // 32 x 32 tiles while they fill the SMs twice over, else 16 x 16 (each tile's FP64
      // work sits on one SM, so the late, small updates need more, smaller tiles)
      const int64_t n32 = (rest + 31) / 32;
      if (n32 * (n32 + 1) / 2 >= 2 * static_cast<int64_t>(sms)) {
        k_chol_update<32><<<dim3(static_cast<unsigned>(n32), static_cast<unsigned>(n32)), 256, 0, st>>>(A, D, kb, nb);
      } else {
        const int64_t n16 = (rest + 15) / 16;
        k_chol_update<16><<<dim3(static_cast<unsigned>(n16), static_cast<unsigned>(n16)), 256, 0, st>>>(A, D, kb, nb);
      }
      note_launch();
    }
    FK_CUDA(cudaGetLastError());
  }
  return FK_OK;
}

// R = B - A X  (dense Hermitian A given by T, W) for refinement; one CTA per (rhs, row block)
// Blocked triangular solves L L^H x = b for one right-hand side per CTA (blockIdx.x):
// the vector lives in shared memory; each 32 x 32 diagonal block is staged in shared
// memory and solved by one warp; the off-diagonal updates give every thread one row
// (forward) or one column (backward) and 32 independent loads.  L: row-major complex
// lower triangle (the Cholesky factor), X: B on entry, solution on exit.
constexpr int TS_NB = 32;
static_assert(TS_NB == NB, "the triangular solves use the Cholesky's diagonal-block inverses");
constexpr int TS_THREADS = 512;

__global__ void __launch_bounds__(TS_THREADS) k_trisolve_blk(const double* __restrict__ L, int D, double* X) {
  extern __shared__ __align__(16) unsigned char smem_ts[];
  cd* ys = reinterpret_cast<cd*>(smem_ts);               // [D]
  cd* dg = ys + D;                                       // [TS_NB][TS_NB + 1]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* xs = X + 2 * static_cast<int64_t>(blockIdx.x) * D;
  for (int i = tid; i < D; i += TS_THREADS) ys[i] = cd{xs[2 * i], xs[2 * i + 1]};
  auto Lat = [&](int r, int c) { return cd{__ldg(L + 2 * (static_cast<int64_t>(r) * D + c)),
                                           __ldg(L + 2 * (static_cast<int64_t>(r) * D + c) + 1)}; };
  auto stage_diag = [&](int kb, int nb) {
    for (int t = tid; t < TS_NB * TS_NB; t += TS_THREADS) {
      const int r = t / TS_NB, c = t - r * TS_NB;
      dg[r * (TS_NB + 1) + c] = (r < nb && c <= r) ? Lat(kb + r, kb + c) : cd{0, 0};
    }
  };
  __syncthreads();
  // forward: L y = b
  for (int kb = 0; kb < D; kb += TS_NB) {
    const int nb = min(TS_NB, D - kb);
    stage_diag(kb, nb);
    __syncthreads();
    if (warp == 0) {
      for (int i = 0; i < nb; ++i) {
        cd t = (lane < i) ? cmul(dg[i * (TS_NB + 1) + lane], ys[kb + lane]) : cd{0, 0};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
          t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
        }
        if (lane == 0) {
          const double lii = dg[i * (TS_NB + 1) + i].x;
          ys[kb + i] = cd{(ys[kb + i].x - t.x) / lii, (ys[kb + i].y - t.y) / lii};
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int r = kb + nb + tid; r < D; r += TS_THREADS) {
      cd acc = cd{0, 0};
#pragma unroll 8
      for (int j = 0; j < nb; ++j) acc = cadd(acc, cmul(Lat(r, kb + j), ys[kb + j]));
      ys[r] = cd{ys[r].x - acc.x, ys[r].y - acc.y};
    }
    __syncthreads();
  }
  // backward: L^H x = y
  const int nblocks = (D + TS_NB - 1) / TS_NB;
  for (int bi = nblocks - 1; bi >= 0; --bi) {
    const int kb = bi * TS_NB, nb = min(TS_NB, D - kb);
    stage_diag(kb, nb);
    __syncthreads();
    if (warp == 0) {
      for (int i = nb - 1; i >= 0; --i) {
        // x_i = (y_i - sum_{j > i} conj(L[j][i]) x_j) / L[i][i]
        cd t = (lane > i && lane < nb) ? cconjmul(dg[lane * (TS_NB + 1) + i], ys[kb + lane]) : cd{0, 0};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
          t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
        }
        if (lane == 0) {
          const double lii = dg[i * (TS_NB + 1) + i].x;
          ys[kb + i] = cd{(ys[kb + i].x - t.x) / lii, (ys[kb + i].y - t.y) / lii};
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int c = tid; c < kb; c += TS_THREADS) {
      cd acc = cd{0, 0};
#pragma unroll 8
      for (int j = 0; j < nb; ++j) acc = cadd(acc, cconjmul(Lat(kb + j, c), ys[kb + j]));
      ys[c] = cd{ys[c].x - acc.x, ys[c].y - acc.y};
    }
    __syncthreads();
  }
  for (int i = tid; i < D; i += TS_THREADS) {
    xs[2 * i] = ys[i].x;
    xs[2 * i + 1] = ys[i].y;
  }
}

fk_status trisolve_coop(const double* L, const double* Linv, int64_t D, double* X, int n_rhs, cudaStream_t st,
                        Scratch& scr, unsigned* flags, bool* handled);

// The cooperative form spreads the FP64 updates over every SM (this part's FP64 rate
// makes one SM the bottleneck at D ~ 1000); the one-CTA blocked form is the fallback.
static fk_status trisolve(const double* L, int64_t D, double* X, int n_rhs, cudaStream_t st, Scratch* scr = nullptr,
                          unsigned* flags = nullptr, const double* Linv = nullptr) {
  if (scr && flags) {
    bool handled = false;
    FK_TRY(trisolve_coop(L, Linv, D, X, n_rhs, st, *scr, flags, &handled));
    if (handled) return FK_OK;
  }
  // D <= 8192 (the dense route's limit): the vector fits in shared memory
  const size_t smem = sizeof(cd) * (static_cast<size_t>(D) + TS_NB * (TS_NB + 1));
  if (smem > 200 * 1024) return set_error(FK_EINVAL, "triangular solve: D = %lld too large", (long long)D);
  FK_CUDA(cudaFuncSetAttribute(k_trisolve_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  k_trisolve_blk<<<n_rhs, TS_THREADS, smem, st>>>(L, static_cast<int>(D), X); note_launch();
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}

__global__ void k_residual_dense(int d, int m, const double* T, const double* W, const double* X,
                                 const double* B, double* R, int n_rhs) {
  const int K = 2 * m + 1, K2 = 4 * m + 1;
  int64_t D = 1;
  for (int l = 0; l < d; ++l) D *= K;
  const int64_t total = D * n_rhs;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t rr = t / D, row = t - (t / D) * D;
    int kr[3] = {0, 0, 0};
    mode_of(row, d, m, kr);
    cd acc = cd{B[2 * t], B[2 * t + 1]};
    const double* x = X + 2 * rr * D;
    for (int64_t c = 0; c < D; ++c) {
      int kc[3] = {0, 0, 0};
      mode_of(c, d, m, kc);
      int64_t idx = 0;
      for (int l = 0; l < d; ++l) idx = idx * K2 + (kr[l] - kc[l] + 2 * m);
      cd a = cd{T[2 * idx], T[2 * idx + 1]};
      if (c == row) a.x += W[row];
      acc = csub(acc, cmul(a, cd{x[2 * c], x[2 * c + 1]}));
    }
    R[2 * t] = acc.x;
    R[2 * t + 1] = acc.y;
  }
}

__global__ void k_axpy_c(int64_t n2, const double* dx, double* x) {
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < n2;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x)
    x[t] += dx[t];
}

// ---------------------------------------------------------------- CG with FFT Toeplitz matvec
// Circulant of side Lc >= 4m + 1: c[(j mod Lc)] = T_j for |j|_inf <= 2m.
__global__ void k_circ_embed(int d, int m, int Lc, const double* T, cplx<double>* c) {
  const int K2 = 4 * m + 1;
  int64_t M2 = 1;
  for (int l = 0; l < d; ++l) M2 *= K2;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < M2;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int64_t q = t, node = 0, mul = 1;
    int jj[3];
    bool aliased = false;  // Lc = 4m: the lag -2m shares its node with +2m, which keeps it
    for (int l = d - 1; l >= 0; --l) {
      jj[l] = static_cast<int>(q % K2) - 2 * m;
      aliased |= Lc < K2 && jj[l] == -2 * m;
      q /= K2;
    }
    if (aliased) continue;
    for (int l = d - 1; l >= 0; --l) {
      node += mul * ((jj[l] + Lc) % Lc);
      mul *= Lc;
    }
    c[node].x = T[2 * t];
    c[node].y = T[2 * t + 1];
  }
}

// pad: buf[s][node(q)] = v[s][q] (q over D modes at node q_l = k_l + m), zeros elsewhere (buffer pre-zeroed)
__global__ void k_pad(int d, int m, int Lc, int nsys, const double* v, cplx<double>* buf) {
  const int K = 2 * m + 1;
  int64_t D = 1, LL = 1;
  for (int l = 0; l < d; ++l) { D *= K; LL *= Lc; }
  const int64_t total = D * nsys;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t s = t / D;
    int64_t q = t - s * D, node = 0, mul = 1;
    for (int l = d - 1; l >= 0; --l) {
      node += mul * (q % K);
      q /= K;
      mul *= Lc;
    }
    buf[s * LL + node].x = v[2 * t];
    buf[s * LL + node].y = v[2 * t + 1];
  }
}

__global__ void k_pointwise(int64_t LL, int nsys, const cplx<double>* ch, cplx<double>* buf) {
  const int64_t total = LL * nsys;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const cplx<double> a = ch[t % LL], b = buf[t];
    buf[t].x = a.x * b.x - a.y * b.y;
    buf[t].y = a.x * b.y + a.y * b.x;
  }
}

// q[s] = extract(buf[s]) / LL + W[l(s)] * p[s];  systems s = l * n_rhs + r
__global__ void k_extract_addw(int d, int m, int Lc, int nsys, int n_rhs, const cplx<double>* buf, const double* W,
                               const double* p, double* q) {
  const int K = 2 * m + 1;
  int64_t D = 1, LL = 1;
  for (int l = 0; l < d; ++l) { D *= K; LL *= Lc; }
  const double inv = 1.0 / static_cast<double>(LL);
  const int64_t total = D * nsys;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t s = t / D;
    const int64_t qi = t - s * D;
    int64_t qq = qi, node = 0, mul = 1;
    for (int l = d - 1; l >= 0; --l) {
      node += mul * (qq % K);
      qq /= K;
      mul *= Lc;
    }
    const double w = W[(s / n_rhs) * D + qi];
    const cplx<double> v = buf[s * LL + node];
    q[2 * t] = v.x * inv + w * p[2 * t];
    q[2 * t + 1] = v.y * inv + w * p[2 * t + 1];
  }
}

// per-system reductions: out[s] = sum_k Re(conj(a_k) b_k)  (optionally scaled by invdiag)
__global__ void k_dot(int64_t D, const double* a, const double* b, double* out) {
  const int s = blockIdx.x;
  const double* pa = a + 2 * s * D;
  const double* pb = b + 2 * s * D;
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < D; k += blockDim.x) acc += pa[2 * k] * pb[2 * k] + pa[2 * k + 1] * pb[2 * k + 1];
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) out[s] = acc;
  }
}

struct CgState {
  double* rz;     // <r, z>
  double* pq;     // <p, A p>
  double* rr;     // <r, r>
  double* bb;     // <b, b>
  int* active;    // 1 while not converged
};

// x += alpha p; r -= alpha q; z = r / diag ; per-system alpha = rz / pq
__global__ void k_cg_update_xr(int64_t D, int n_rhs, const double* W, double T0, CgState cs, const double* p,
                               const double* q, double* x, double* r, double* z) {
  const int s = blockIdx.y;
  if (!cs.active[s]) return;
  const double alpha = cs.rz[s] / cs.pq[s];
  const int l = s / n_rhs;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < D;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t o = 2 * (s * D + k);
    x[o] += alpha * p[o];
    x[o + 1] += alpha * p[o + 1];
    r[o] -= alpha * q[o];
    r[o + 1] -= alpha * q[o + 1];
    const double inv = 1.0 / (T0 + W[l * D + k]);
    z[o] = r[o] * inv;
    z[o + 1] = r[o + 1] * inv;
  }
}

// beta = rz_new / rz_old ; p = z + beta p ; update rz, convergence flags
__global__ void k_cg_beta(int nsys, double tol2, CgState cs, double* rz_new) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys || !cs.active[s]) return;
  if (cs.rr[s] <= tol2 * cs.bb[s]) {
    cs.active[s] = 0;
    return;
  }
  const double beta = rz_new[s] / cs.rz[s];
  cs.rz[s] = rz_new[s];
  rz_new[s] = beta;  // reuse as beta
}

__global__ void k_cg_update_p(int64_t D, CgState cs, const double* beta, const double* z, double* p) {
  const int s = blockIdx.y;
  if (!cs.active[s]) return;
  const double b = beta[s];
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < D;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t o = 2 * (s * D + k);
    p[o] = z[o] + b * p[o];
    p[o + 1] = z[o + 1] + b * p[o + 1];
  }
}

__global__ void k_cg_init(int64_t D, int n_rhs, int nsys, const double* W, double T0, const double* b, double* x,
                          double* r, double* z, double* p) {
  const int s = blockIdx.y;
  const int l = s / n_rhs, rr = s % n_rhs;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < D;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t o = 2 * (s * D + k), ob = 2 * (rr * D + k);
    x[o] = 0.0;
    x[o + 1] = 0.0;
    r[o] = b[ob];
    r[o + 1] = b[ob + 1];
    const double inv = 1.0 / (T0 + W[l * D + k]);
    z[o] = b[ob] * inv;
    z[o + 1] = b[ob + 1] * inv;
    p[o] = z[o];
    p[o + 1] = z[o + 1];
  }
}

__global__ void k_set_active(int nsys, int* active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nsys) active[s] = 1;
}

__global__ void k_count_active(int nsys, const int* active, int* count) {
  __shared__ int c;
  if (threadIdx.x == 0) c = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < nsys; s += blockDim.x)
    if (active[s]) atomicAdd(&c, 1);
  __syncthreads();
  if (threadIdx.x == 0) *count = c;
}

static int next_pow2i(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Toeplitz matvec q = Toep(T) v + W v for all systems (v, q: [nsys][D]).
struct Circ {
  int d, m, Lc;
  int64_t LL, D;
  cplx<double>* ch;   // FFT of the circulant
  cplx<double>* buf;  // nsys * LL
  const double* tw;
};

static fk_status fft_nd(const Circ& c, int nsys, int sign, cudaStream_t st) {
  if (c.d == 1) return fft_lines<double>(c.buf, c.Lc, nsys, c.Lc, 1, sign, c.tw, st);
  if (c.d == 2) {
    FK_TRY(fft_lines<double>(c.buf, c.Lc, static_cast<int64_t>(nsys) * c.Lc, c.Lc, 1, sign, c.tw, st));  // rows
    for (int s = 0; s < nsys; ++s)
      FK_TRY(fft_lines<double>(c.buf + s * c.LL, c.Lc, c.Lc, 1, c.Lc, sign, c.tw, st));  // columns
    return FK_OK;
  }
  if (c.d == 3) {
    const int64_t L2 = static_cast<int64_t>(c.Lc) * c.Lc;
    FK_TRY(fft_lines<double>(c.buf, c.Lc, static_cast<int64_t>(nsys) * L2, c.Lc, 1, sign, c.tw, st));
    for (int64_t q = 0; q < static_cast<int64_t>(nsys) * c.Lc; ++q)
      FK_TRY(fft_lines<double>(c.buf + q * L2, c.Lc, c.Lc, 1, c.Lc, sign, c.tw, st));
    for (int s = 0; s < nsys; ++s) FK_TRY(fft_lines<double>(c.buf + s * c.LL, c.Lc, L2, 1, L2, sign, c.tw, st));
    return FK_OK;
  }
  return set_error(FK_EINVAL, "CG: d = %d not built", c.d);
}

static fk_status matvec(const Circ& c, int nsys, int n_rhs, const double* W, const double* v, double* q,
                        cudaStream_t st) {
  FK_CUDA(cudaMemsetAsync(c.buf, 0, sizeof(cplx<double>) * c.LL * nsys, st));
  k_pad<<<grid_for(c.D * nsys, 256), 256, 0, st>>>(c.d, c.m, c.Lc, nsys, v, c.buf); note_launch();
  FK_TRY(fft_nd(c, nsys, -1, st));
  k_pointwise<<<grid_for(c.LL * nsys, 256), 256, 0, st>>>(c.LL, nsys, c.ch, c.buf); note_launch();
  FK_TRY(fft_nd(c, nsys, +1, st));
  k_extract_addw<<<grid_for(c.D * nsys, 256), 256, 0, st>>>(c.d, c.m, c.Lc, nsys, n_rhs, c.buf, W, v, q); note_launch();
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}

// per system s: rr[s] = |b_{s % n_rhs} - q_s|^2, bb[s] = |b_{s % n_rhs}|^2
__global__ void k_resid_norm(int64_t D, int n_rhs, const double* b, const double* q, double* rr, double* bb) {
  const int s = blockIdx.x;
  const double* pb = b + 2 * (s % n_rhs) * D;
  const double* pq = q + 2 * s * D;
  double a0 = 0.0, a1 = 0.0;
  for (int64_t k = threadIdx.x; k < D; k += blockDim.x) {
    const double er = pb[2 * k] - pq[2 * k], ei = pb[2 * k + 1] - pq[2 * k + 1];
    a0 += er * er + ei * ei;
    a1 += pb[2 * k] * pb[2 * k] + pb[2 * k + 1] * pb[2 * k + 1];
  }
  __shared__ double red[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_down_sync(0xffffffffu, a0, o);
    a1 += __shfl_down_sync(0xffffffffu, a1, o);
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = a0; red[1][threadIdx.x >> 5] = a1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { s0 += red[0][w]; s1 += red[1][w]; }
    rr[s] = s0;
    bb[s] = s1;
  }
}

static fk_status cg_solve(int d, int m, const double* T, const double* W, int n_w, const double* rhs, int n_rhs,
                          const fk_opts& o, double* sol, cudaStream_t st, Scratch& scr, int* iters_out,
                          double* relres_out) {
  Circ c;
  c.d = d;
  c.m = m;
  c.Lc = next_pow2i(4 * m + 1);
  if (c.Lc < 2) c.Lc = 2;
  c.LL = 1;
  c.D = 1;
  for (int l = 0; l < d; ++l) {
    c.LL *= c.Lc;
    c.D *= (2 * m + 1);
  }
  const int nsys = n_w * n_rhs;
  const int64_t D = c.D;
  FK_TRY(scr.alloc(&c.ch, c.LL));
  FK_TRY(scr.alloc(&c.buf, c.LL * nsys));
  FK_TRY(twiddle_table(c.Lc, st, &c.tw));
  FK_CUDA(cudaMemsetAsync(c.ch, 0, sizeof(cplx<double>) * c.LL, st));
  int64_t M2 = 1;
  for (int l = 0; l < d; ++l) M2 *= (4 * m + 1);
  k_circ_embed<<<grid_for(M2, 256), 256, 0, st>>>(d, m, c.Lc, T, c.ch); note_launch();
  FK_CUDA(cudaGetLastError());
  {
    Circ c1 = c;
    c1.buf = c.ch;
    FK_TRY(fft_nd(c1, 1, -1, st));
  }
  // T_0 (real part of the centre moment) for the Jacobi preconditioner
  int64_t centre = 0;
  for (int l = 0; l < d; ++l) centre = centre * (4 * m + 1) + 2 * m;
  double T0 = 1.0;
  FK_CUDA(cudaMemcpyAsync(&T0, T + 2 * centre, sizeof(double), cudaMemcpyDeviceToHost, st));
  FK_CUDA(cudaStreamSynchronize(st));
  if (!(T0 > 0.0)) T0 = 1.0;

  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *scal = nullptr;
  int *active = nullptr, *cnt = nullptr;
  FK_TRY(scr.alloc(&r, 2 * D * nsys));
  FK_TRY(scr.alloc(&z, 2 * D * nsys));
  FK_TRY(scr.alloc(&p, 2 * D * nsys));
  FK_TRY(scr.alloc(&q, 2 * D * nsys));
  FK_TRY(scr.alloc(&scal, 5 * static_cast<size_t>(nsys)));
  FK_TRY(scr.alloc(&active, nsys));
  FK_TRY(scr.alloc(&cnt, 1));
  CgState cs{scal, scal + nsys, scal + 2 * nsys, scal + 3 * nsys, active};
  double* rznew = scal + 4 * nsys;
  double* x = sol;
  const dim3 g2(static_cast<unsigned>(std::min<int64_t>((D + 255) / 256, 64)), nsys);
  k_cg_init<<<g2, 256, 0, st>>>(D, n_rhs, nsys, W, T0, rhs, x, r, z, p); note_launch();
  k_set_active<<<(nsys + 255) / 256, 256, 0, st>>>(nsys, active); note_launch();
  k_dot<<<nsys, 256, 0, st>>>(D, r, z, cs.rz); note_launch();
  // |b|^2 per system: b of system s is rhs[s % n_rhs] = r at init
  k_dot<<<nsys, 256, 0, st>>>(D, r, r, cs.bb); note_launch();
  FK_CUDA(cudaGetLastError());
  const double tol2 = o.cg_tol * o.cg_tol;
  int it = 0;
  int host_active = nsys;
  for (it = 0; it < o.cg_maxit; ++it) {
    FK_TRY(matvec(c, nsys, n_rhs, W, p, q, st));
    k_dot<<<nsys, 256, 0, st>>>(D, p, q, cs.pq); note_launch();
    k_cg_update_xr<<<g2, 256, 0, st>>>(D, n_rhs, W, T0, cs, p, q, x, r, z); note_launch();
    k_dot<<<nsys, 256, 0, st>>>(D, r, z, rznew); note_launch();
    k_dot<<<nsys, 256, 0, st>>>(D, r, r, cs.rr); note_launch();
    k_cg_beta<<<(nsys + 255) / 256, 256, 0, st>>>(nsys, tol2, cs, rznew); note_launch();
    k_cg_update_p<<<g2, 256, 0, st>>>(D, cs, rznew, z, p); note_launch();
    FK_CUDA(cudaGetLastError());
    if ((it & 3) == 3 || it + 1 == o.cg_maxit) {
      k_count_active<<<1, 256, 0, st>>>(nsys, active, cnt); note_launch();
      FK_CUDA(cudaMemcpyAsync(&host_active, cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
      FK_CUDA(cudaStreamSynchronize(st));
      if (host_active == 0) break;
    }
  }
  if (iters_out) *iters_out = it + 1;
  // final relative residual from a fresh matvec: |b - A x| / |b| per system
  FK_TRY(matvec(c, nsys, n_rhs, W, x, q, st));
  k_resid_norm<<<nsys, 256, 0, st>>>(D, n_rhs, rhs, q, cs.rr, cs.bb); note_launch();
  FK_CUDA(cudaGetLastError());
  {
    std::vector<double> rr(nsys), bb(nsys);
    FK_CUDA(cudaMemcpyAsync(rr.data(), cs.rr, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st));
    FK_CUDA(cudaMemcpyAsync(bb.data(), cs.bb, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st));
    FK_CUDA(cudaStreamSynchronize(st));
    double worst = 0.0;
    for (int s = 0; s < nsys; ++s) worst = std::max(worst, bb[s] > 0 ? std::sqrt(rr[s] / bb[s]) : std::sqrt(rr[s]));
    if (relres_out) *relres_out = worst;
  }
  if (host_active != 0) return set_error(FK_ENOCONV, "CG did not converge in %d iterations", o.cg_maxit);
  return FK_OK;
}

// ---------------------------------------------------------------- fused CG (d = 1, 2)
// Scalars per system s (double): PQ = <p, Ap>, RZ0 / RZ1 = <r, z> (ping-pong by
// iteration parity), RR = |r|^2, BB = |b|^2.  A matvec q = Toep(T) v + W v goes through
// the circulant of side Lc >= 4m + 1: only the K = 2m + 1 nonzero rows of the padded
// input are transformed, and only K output rows are kept.
struct CgScal {
  double *pq, *rz0, *rz1, *rr, *bb;
  int* active;
};

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += red[w];
  __syncthreads();
  return t;  // valid in thread 0
}

// 2-D, step 1: forward FFT of the nonzero rows r < K of the padded input v
__global__ void k_cgf_rows_fwd(int K, int Lc, int logLc, const double* v, cplx<double>* buf, const double* tw,
                               CgScal sc, int zero_scalars, int cur) {
  extern __shared__ unsigned char smem_raw[];
  cplx<double>* sl = reinterpret_cast<cplx<double>*>(smem_raw);
  const int r = blockIdx.x, s = blockIdx.y;
  if (!sc.active[s]) return;
  if (zero_scalars && r == 0 && threadIdx.x == 0) {
    sc.pq[s] = 0.0;
    sc.rr[s] = 0.0;
    (cur ? sc.rz0 : sc.rz1)[s] = 0.0;  // the next <r, z>
  }
  const int64_t D = static_cast<int64_t>(K) * K;
  const double* vs = v + 2 * (s * D + static_cast<int64_t>(r) * K);
  for (int i = threadIdx.x; i < Lc; i += blockDim.x) {
    cplx<double> e;
    e.x = (i < K) ? vs[2 * i] : 0.0;
    e.y = (i < K) ? vs[2 * i + 1] : 0.0;
    sl[bitrev(i, logLc)] = e;
  }
  __syncthreads();
  fft_smem<double>(sl, Lc, -1, tw);
  cplx<double>* o = buf + (static_cast<int64_t>(s) * K + r) * Lc;
  for (int i = threadIdx.x; i < Lc; i += blockDim.x) o[i] = sl[i];
}

// 2-D, step 2: per column c: FFT over rows (K nonzero), times the circulant spectrum,
// inverse FFT, keep rows < K
__global__ void k_cgf_cols(int K, int Lc, int logLc, cplx<double>* buf, const cplx<double>* ch, const double* tw,
                           CgScal sc) {
  extern __shared__ unsigned char smem_raw[];
  cplx<double>* sl = reinterpret_cast<cplx<double>*>(smem_raw);
  const int c = blockIdx.x, s = blockIdx.y;
  if (!sc.active[s]) return;
  cplx<double>* b = buf + static_cast<int64_t>(s) * K * Lc + c;
  for (int i = threadIdx.x; i < Lc; i += blockDim.x) {
    cplx<double> e;
    if (i < K) e = b[static_cast<int64_t>(i) * Lc];
    else e.x = e.y = 0.0;
    sl[bitrev(i, logLc)] = e;
  }
  __syncthreads();
  fft_smem<double>(sl, Lc, -1, tw);
  for (int i = threadIdx.x; i < Lc; i += blockDim.x) {
    const cplx<double> a = ch[static_cast<int64_t>(i) * Lc + c], e = sl[i];
    cplx<double> t;
    t.x = a.x * e.x - a.y * e.y;
    t.y = a.x * e.y + a.y * e.x;
    sl[i] = t;
  }
  __syncthreads();
  bitrev_permute<double>(sl, Lc, logLc);
  fft_smem<double>(sl, Lc, +1, tw);
  for (int i = threadIdx.x; i < K; i += blockDim.x) b[static_cast<int64_t>(i) * Lc] = sl[i];
}

// 2-D, step 3: inverse FFT of rows r < K, q = (.)/Lc^2 + W v, and <v, q>
__global__ void k_cgf_rows_inv(int K, int Lc, int logLc, int n_rhs, const cplx<double>* buf, const double* W,
                               const double* v, double* q, const double* tw, CgScal sc, int want_dot) {
  extern __shared__ unsigned char smem_raw[];
  cplx<double>* sl = reinterpret_cast<cplx<double>*>(smem_raw);
  __shared__ double red[32];
  const int r = blockIdx.x, s = blockIdx.y;
  if (!sc.active[s]) return;
  const cplx<double>* b = buf + (static_cast<int64_t>(s) * K + r) * Lc;
  for (int i = threadIdx.x; i < Lc; i += blockDim.x) sl[bitrev(i, logLc)] = b[i];
  __syncthreads();
  fft_smem<double>(sl, Lc, +1, tw);
  const int64_t D = static_cast<int64_t>(K) * K;
  const double inv = 1.0 / (static_cast<double>(Lc) * Lc);
  const double* Ws = W + (s / n_rhs) * D + static_cast<int64_t>(r) * K;
  const double* vs = v + 2 * (s * D + static_cast<int64_t>(r) * K);
  double* qs = q + 2 * (s * D + static_cast<int64_t>(r) * K);
  double acc = 0.0;
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    const double qr = sl[i].x * inv + Ws[i] * vs[2 * i];
    const double qi = sl[i].y * inv + Ws[i] * vs[2 * i + 1];
    qs[2 * i] = qr;
    qs[2 * i + 1] = qi;
    acc += vs[2 * i] * qr + vs[2 * i + 1] * qi;
  }
  if (want_dot) {
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) atomicAdd(sc.pq + s, t);
  }
}

// 1-D: the whole matvec of one system per CTA; with ch2 != null the operator term
// mu conj(P) Toep(c) (P v) of a sub-domain / collocation penalty is added (second
// circulant product on the same shared line)
__global__ void k_cgf_1d(int K, int Lc, int logLc, int n_rhs, const cplx<double>* ch, const double* W, const double* v,
                         double* q, const double* tw, CgScal sc, int zero_scalars, int cur, int want_dot,
                         const cplx<double>* ch2, const double* P, double mu) {
  extern __shared__ unsigned char smem_raw[];
  cplx<double>* sl = reinterpret_cast<cplx<double>*>(smem_raw);
  __shared__ double red[32];
  const int s = blockIdx.x;
  if (!sc.active[s]) return;
  if (zero_scalars && threadIdx.x == 0) {
    sc.rr[s] = 0.0;
    (cur ? sc.rz0 : sc.rz1)[s] = 0.0;
  }
  const double* vs = v + 2 * static_cast<int64_t>(s) * K;
  const double inv = 1.0 / static_cast<double>(Lc);
  const double* Ws = W + static_cast<int64_t>(s / n_rhs) * K;
  double* qs = q + 2 * static_cast<int64_t>(s) * K;
  for (int pass = 0; pass < (ch2 ? 2 : 1); ++pass) {
    const cplx<double>* spec = pass ? ch2 : ch;
    for (int i = threadIdx.x; i < Lc; i += blockDim.x) {
      cplx<double> e;
      e.x = (i < K) ? vs[2 * i] : 0.0;
      e.y = (i < K) ? vs[2 * i + 1] : 0.0;
      if (pass && i < K) {  // P v
        const double pr = P[2 * i], pi = P[2 * i + 1];
        const double ex = pr * e.x - pi * e.y, ey = pr * e.y + pi * e.x;
        e.x = ex;
        e.y = ey;
      }
      sl[bitrev(i, logLc)] = e;
    }
    __syncthreads();
    fft_smem<double>(sl, Lc, -1, tw);
    for (int i = threadIdx.x; i < Lc; i += blockDim.x) {
      const cplx<double> a = spec[i], e = sl[i];
      cplx<double> t;
      t.x = a.x * e.x - a.y * e.y;
      t.y = a.x * e.y + a.y * e.x;
      sl[i] = t;
    }
    __syncthreads();
    bitrev_permute<double>(sl, Lc, logLc);
    fft_smem<double>(sl, Lc, +1, tw);
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
      if (pass == 0) {
        qs[2 * i] = sl[i].x * inv + Ws[i] * vs[2 * i];
        qs[2 * i + 1] = sl[i].y * inv + Ws[i] * vs[2 * i + 1];
      } else {  // + mu conj(P) (.)
        const double pr = P[2 * i], pi = -P[2 * i + 1];
        const double tr = sl[i].x * inv, ti = sl[i].y * inv;
        qs[2 * i] += mu * (pr * tr - pi * ti);
        qs[2 * i + 1] += mu * (pr * ti + pi * tr);
      }
    }
    __syncthreads();
  }
  double acc = 0.0;
  for (int i = threadIdx.x; i < K; i += blockDim.x) acc += vs[2 * i] * qs[2 * i] + vs[2 * i + 1] * qs[2 * i + 1];
  if (want_dot) {
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) sc.pq[s] = t;
  }
}

// x += alpha p; r -= alpha q; z = r / diag; <r, z> and |r|^2 into the next slots
__global__ void k_cgf_update(int64_t D, int n_rhs, const double* W, double T0, CgScal sc, int cur, const double* p,
                             const double* q, double* x, double* r, double* z) {
  __shared__ double red[32];
  const int s = blockIdx.y;
  if (!sc.active[s]) return;
  const double alpha = (cur ? sc.rz1 : sc.rz0)[s] / sc.pq[s];
  const double* Ws = W + static_cast<int64_t>(s / n_rhs) * D;
  double arz = 0.0, arr = 0.0;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < D;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t o = 2 * (s * D + k);
    x[o] += alpha * p[o];
    x[o + 1] += alpha * p[o + 1];
    const double rr0 = r[o] - alpha * q[o], rr1 = r[o + 1] - alpha * q[o + 1];
    r[o] = rr0;
    r[o + 1] = rr1;
    const double inv = 1.0 / (T0 + Ws[k]);
    z[o] = rr0 * inv;
    z[o + 1] = rr1 * inv;
    arz += (rr0 * rr0 + rr1 * rr1) * inv;
    arr += rr0 * rr0 + rr1 * rr1;
  }
  const double t1 = block_sum(arz, red);
  const double t2 = block_sum(arr, red);
  if (threadIdx.x == 0) {
    atomicAdd((cur ? sc.rz0 : sc.rz1) + s, t1);
    atomicAdd(sc.rr + s, t2);
  }
}

// convergence test and p = z + beta p
__global__ void k_cgf_direction(int64_t D, double tol2, CgScal sc, int cur, const double* z, double* p) {
  const int s = blockIdx.y;
  if (!sc.active[s]) return;
  if (sc.rr[s] <= tol2 * sc.bb[s]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) sc.active[s] = 0;
    return;
  }
  const double beta = (cur ? sc.rz0 : sc.rz1)[s] / (cur ? sc.rz1 : sc.rz0)[s];
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < D;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t o = 2 * (s * D + k);
    p[o] = z[o] + beta * p[o];
    p[o + 1] = z[o + 1] + beta * p[o + 1];
  }
}

// x = 0, r = b, z = r / diag, p = z; <r, z> -> rz0, |b|^2 -> bb and rr
__global__ void k_cgf_init(int64_t D, int n_rhs, const double* W, double T0, const double* b, double* x, double* r,
                           double* z, double* p, CgScal sc) {
  __shared__ double red[32];
  const int s = blockIdx.y;
  const double* bs = b + 2 * static_cast<int64_t>(s % n_rhs) * D;
  const double* Ws = W + static_cast<int64_t>(s / n_rhs) * D;
  double arz = 0.0, abb = 0.0;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < D;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t o = 2 * (s * D + k);
    const double b0 = bs[2 * k], b1 = bs[2 * k + 1];
    const double inv = 1.0 / (T0 + Ws[k]);
    x[o] = 0.0;
    x[o + 1] = 0.0;
    r[o] = b0;
    r[o + 1] = b1;
    z[o] = b0 * inv;
    z[o + 1] = b1 * inv;
    p[o] = b0 * inv;
    p[o + 1] = b1 * inv;
    arz += (b0 * b0 + b1 * b1) * inv;
    abb += b0 * b0 + b1 * b1;
  }
  const double t1 = block_sum(arz, red);
  const double t2 = block_sum(abb, red);
  if (threadIdx.x == 0) {
    atomicAdd(sc.rz0 + s, t1);
    atomicAdd(sc.bb + s, t2);
    atomicAdd(sc.rr + s, t2);
  }
}

static fk_status cg_solve_fused(int d, int m, const double* T, const double* W, int n_w, const double* rhs, int n_rhs,
                                const fk_opts& o, double* sol, cudaStream_t st, Scratch& scr, int* iters_out,
                                double* relres_out, const PenOp* op = nullptr) {
  if (op && d != 1) return set_error(FK_EINVAL, "operator penalty: the multi-launch CG is built for d = 1");
  const int K = 2 * m + 1;
  int Lc = next_pow2i(4 * m + 1);
  if (Lc < 2) Lc = 2;
  int logLc = 0;
  while ((1 << logLc) < Lc) ++logLc;
  const size_t line_sm = sizeof(cplx<double>) * Lc;
  if (line_sm > 200 * 1024) return set_error(FK_EINVAL, "CG: circulant side %d too long", Lc);
  const int nsys = n_w * n_rhs;
  const int64_t D = (d == 1) ? K : static_cast<int64_t>(K) * K;
  const int64_t LL = (d == 1) ? Lc : static_cast<int64_t>(Lc) * Lc;
  cplx<double>* ch = nullptr;
  const double* tw = nullptr;
  FK_TRY(scr.alloc(&ch, LL));
  FK_TRY(twiddle_table(Lc, st, &tw));
  FK_CUDA(cudaMemsetAsync(ch, 0, sizeof(cplx<double>) * LL, st));
  int64_t M2 = 1;
  for (int l = 0; l < d; ++l) M2 *= (4 * m + 1);
  k_circ_embed<<<grid_for(M2, 256), 256, 0, st>>>(d, m, Lc, T, ch); note_launch();
  FK_CUDA(cudaGetLastError());
  if (d == 1) {
    FK_TRY(fft_lines<double>(ch, Lc, 1, Lc, 1, -1, tw, st));
  } else {
    FK_TRY(fft_lines<double>(ch, Lc, Lc, Lc, 1, -1, tw, st));
    FK_TRY(fft_lines<double>(ch, Lc, Lc, 1, Lc, -1, tw, st));
  }
  int64_t centre = 0;
  for (int l = 0; l < d; ++l) centre = centre * (4 * m + 1) + 2 * m;
  double T0 = 1.0;
  FK_CUDA(cudaMemcpyAsync(&T0, T + 2 * centre, sizeof(double), cudaMemcpyDeviceToHost, st));
  FK_CUDA(cudaStreamSynchronize(st));
  if (!(T0 > 0.0)) T0 = 1.0;

  // operator penalty: its circulant spectrum, and W + mu |P|^2 c_0 as the Jacobi diagonal
  cplx<double>* ch2 = nullptr;
  const double* Wd = W;
  if (op) {
    FK_TRY(scr.alloc(&ch2, LL));
    FK_CUDA(cudaMemsetAsync(ch2, 0, sizeof(cplx<double>) * LL, st));
    k_circ_embed<<<grid_for(M2, 256), 256, 0, st>>>(d, m, Lc, op->c, ch2); note_launch();
    FK_TRY(fft_lines<double>(ch2, Lc, 1, Lc, 1, -1, tw, st));
    double* wd = nullptr;
    FK_TRY(scr.alloc(&wd, D * n_w));
    k_op_diag<<<grid_for(D * n_w, 256), 256, 0, st>>>(D, n_w, W, op->P, op->c + 2 * centre, op->mu, wd); note_launch();
    FK_CUDA(cudaGetLastError());
    Wd = wd;
  }

  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *scal = nullptr;
  int *active = nullptr, *cnt = nullptr;
  cplx<double>* buf = nullptr;
  FK_TRY(scr.alloc(&r, 2 * D * nsys));
  FK_TRY(scr.alloc(&z, 2 * D * nsys));
  FK_TRY(scr.alloc(&p, 2 * D * nsys));
  FK_TRY(scr.alloc(&q, 2 * D * nsys));
  FK_TRY(scr.alloc(&scal, 5 * static_cast<size_t>(nsys)));
  FK_TRY(scr.alloc(&active, nsys));
  FK_TRY(scr.alloc(&cnt, 1));
  if (d == 2) FK_TRY(scr.alloc(&buf, static_cast<size_t>(nsys) * K * Lc));
  CgScal sc{scal, scal + nsys, scal + 2 * nsys, scal + 3 * nsys, scal + 4 * nsys, active};
  FK_CUDA(cudaMemsetAsync(scal, 0, sizeof(double) * 5 * nsys, st));
  k_set_active<<<(nsys + 255) / 256, 256, 0, st>>>(nsys, active); note_launch();
  double* x = sol;
  const dim3 gv(static_cast<unsigned>(std::min<int64_t>((D + 255) / 256, 64)), nsys);
  k_cgf_init<<<gv, 256, 0, st>>>(D, n_rhs, Wd, T0, rhs, x, r, z, p, sc); note_launch();
  FK_CUDA(cudaGetLastError());
  const int thr = Lc >= 256 ? 256 : (Lc >= 64 ? Lc / 2 : 32);
  if (line_sm > 48 * 1024) {
    FK_CUDA(cudaFuncSetAttribute(k_cgf_rows_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)line_sm));
    FK_CUDA(cudaFuncSetAttribute(k_cgf_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)line_sm));
    FK_CUDA(cudaFuncSetAttribute(k_cgf_rows_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)line_sm));
    FK_CUDA(cudaFuncSetAttribute(k_cgf_1d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)line_sm));
  }
  auto matvec = [&](const double* v, double* out, int zero, int cur, int dot) -> fk_status {
    if (d == 1) {
      k_cgf_1d<<<nsys, thr, line_sm, st>>>(K, Lc, logLc, n_rhs, ch, W, v, out, tw, sc, zero, cur, dot, ch2,
                                           op ? op->P : nullptr, op ? op->mu : 0.0);
      note_launch();
    } else {
      k_cgf_rows_fwd<<<dim3(K, nsys), thr, line_sm, st>>>(K, Lc, logLc, v, buf, tw, sc, zero, cur); note_launch();
      k_cgf_cols<<<dim3(Lc, nsys), thr, line_sm, st>>>(K, Lc, logLc, buf, ch, tw, sc); note_launch();
      k_cgf_rows_inv<<<dim3(K, nsys), thr, line_sm, st>>>(K, Lc, logLc, n_rhs, buf, W, v, out, tw, sc, dot);
      note_launch();
    }
    FK_CUDA(cudaGetLastError());
    return FK_OK;
  };
  const double tol2 = o.cg_tol * o.cg_tol;
  int it = 0, host_active = nsys;
  for (it = 0; it < o.cg_maxit; ++it) {
    const int cur = it & 1;
    FK_TRY(matvec(p, q, 1, cur, 1));
    k_cgf_update<<<gv, 256, 0, st>>>(D, n_rhs, Wd, T0, sc, cur, p, q, x, r, z); note_launch();
    k_cgf_direction<<<gv, 256, 0, st>>>(D, tol2, sc, cur, z, p); note_launch();
    FK_CUDA(cudaGetLastError());
    if ((it & 3) == 3 || it + 1 == o.cg_maxit) {
      k_count_active<<<1, 256, 0, st>>>(nsys, active, cnt); note_launch();
      FK_CUDA(cudaMemcpyAsync(&host_active, cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
      FK_CUDA(cudaStreamSynchronize(st));
      if (host_active == 0) break;
    }
  }
  if (iters_out) *iters_out = it + 1;
  // true relative residual from a fresh matvec
  k_set_active<<<(nsys + 255) / 256, 256, 0, st>>>(nsys, active); note_launch();
  FK_TRY(matvec(x, q, 0, 0, 0));
  k_resid_norm<<<nsys, 256, 0, st>>>(D, n_rhs, rhs, q, sc.rr, sc.bb); note_launch();
  FK_CUDA(cudaGetLastError());
  {
    std::vector<double> rr(nsys), bb(nsys);
    FK_CUDA(cudaMemcpyAsync(rr.data(), sc.rr, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st));
    FK_CUDA(cudaMemcpyAsync(bb.data(), sc.bb, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st));
    FK_CUDA(cudaStreamSynchronize(st));
    double worst = 0.0;
    for (int s2 = 0; s2 < nsys; ++s2) worst = std::max(worst, bb[s2] > 0 ? std::sqrt(rr[s2] / bb[s2]) : std::sqrt(rr[s2]));
    if (relres_out) *relres_out = worst;
  }
  if (host_active != 0) return set_error(FK_ENOCONV, "CG did not converge in %d iterations", o.cg_maxit);
  return FK_OK;
}

// ---------------------------------------------------------------- dispatcher
fk_status cg_solve_persistent(int m, const double* T, const double* W, int n_w, const double* rhs, int n_rhs,
                              const fk_opts& o, double* sol, cudaStream_t st, Scratch& scr, unsigned* flags,
                              int* iters_out, double* relres_out, bool* handled, const PenOp* op);
__global__ void k_dense_residual(const double* A, int64_t D, const double* X, const double* B, double* R, int n_rhs);

fk_status solve_system(int d, int m, const double* T, const double* W, int n_w, const double* rhs, int n_rhs,
                       const fk_opts& o, double* sol, cudaStream_t st, Scratch& scratch, unsigned* flags,
                       int* cg_iters, double* rel_res, const PenOp* op) {
  int64_t D = 1;
  for (int l = 0; l < d; ++l) D *= (2 * m + 1);
  const bool with_op = op && op->c && op->P && op->mu != 0.0;
  int solver = o.solver;
  if (solver == FK_SOLVER_AUTO) solver = (D <= 1024) ? FK_SOLVER_CHOL : FK_SOLVER_CG;
  if (solver == FK_SOLVER_EIG)
    return set_error(FK_EINVAL, "the eigen route serves whole sweeps of penalties lambda S^2: use it through "
                                "fk_fit_sobolev or fk_fit_additive");
  if (cg_iters) *cg_iters = 0;
  if (rel_res) *rel_res = 0.0;
  if (solver == FK_SOLVER_CG) {
    if (d == 2) {
      bool handled = false;
      const fk_status rc = cg_solve_persistent(m, T, W, n_w, rhs, n_rhs, o, sol, st, scratch, flags, cg_iters, rel_res,
                                               &handled, with_op ? op : nullptr);
      if (handled || rc != FK_OK) return rc;
      if (with_op) return set_error(FK_EINVAL, "the operator penalty's CG needs a cooperative launch");
    }
    if (capture_ctx())
      return set_error(FK_EINVAL, "this conjugate-gradient path tests convergence on the host: not capturable "
                                  "(the 2-D single-launch CG and the Cholesky solver are)");
    if (d <= 2) return cg_solve_fused(d, m, T, W, n_w, rhs, n_rhs, o, sol, st, scratch, cg_iters, rel_res,
                                      with_op ? op : nullptr);
    if (with_op) return set_error(FK_EINVAL, "the operator penalty is built for d <= 2");
    return cg_solve(d, m, T, W, n_w, rhs, n_rhs, o, sol, st, scratch, cg_iters, rel_res);
  }
  if (D > 8192) return set_error(FK_EINVAL, "dense Cholesky limited to D <= 8192 (D = %lld)", (long long)D);
  double *A = nullptr, *R = nullptr, *A0 = nullptr;
  FK_TRY(scratch.alloc(&A, 2 * D * D));
  FK_TRY(scratch.alloc(&R, 2 * D * n_rhs));
  if (with_op) FK_TRY(scratch.alloc(&A0, 2 * D * D));  // the assembled matrix, for the refinement residual
  for (int l = 0; l < n_w; ++l) {
    const double* Wl = W + l * D;
    double* X = sol + 2 * static_cast<int64_t>(l) * n_rhs * D;
    k_assemble<<<grid_for(D * D, 256), 256, 0, st>>>(d, m, T, Wl, A); note_launch();
    if (with_op) {
      k_assemble_op<<<grid_for(D * D, 256), 256, 0, st>>>(d, m, op->c, op->P, op->mu, A); note_launch();
      FK_CUDA(cudaMemcpyAsync(A0, A, sizeof(double) * 2 * D * D, cudaMemcpyDeviceToDevice, st));
    }
    FK_CUDA(cudaGetLastError());
    double* linv = nullptr;
    FK_TRY(scratch.alloc(&linv, 2 * linv_blocks(D) * NB * NB));
    FK_TRY(cholesky(A, D, flags, st, linv));
    FK_CUDA(cudaMemcpyAsync(X, rhs, sizeof(double) * 2 * D * n_rhs, cudaMemcpyDeviceToDevice, st));
    FK_TRY(trisolve(A, D, X, n_rhs, st, &scratch, flags, linv));
    FK_CUDA(cudaGetLastError());
    for (int it = 0; it < o.refine_steps; ++it) {
      if (with_op) {
        k_dense_residual<<<grid_for(D * n_rhs, 128), 128, 0, st>>>(A0, D, X, rhs, R, n_rhs); note_launch();
      } else {
        k_residual_dense<<<grid_for(D * n_rhs, 128), 128, 0, st>>>(d, m, T, Wl, X, rhs, R, n_rhs); note_launch();
      }
      FK_TRY(trisolve(A, D, R, n_rhs, st, &scratch, flags, linv));
      k_axpy_c<<<grid_for(2 * D * n_rhs, 256), 256, 0, st>>>(2 * D * n_rhs, R, X); note_launch();
      FK_CUDA(cudaGetLastError());
    }
  }
  return FK_OK;
}

}  // namespace fk

namespace fk {

// R = B - A X for a dense row-major complex A (D x D); X, B, R: [n_rhs][D]
__global__ void k_dense_residual(const double* A, int64_t D, const double* X, const double* B, double* R, int n_rhs) {
  const int64_t total = D * n_rhs;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t rr = t / D, row = t - (t / D) * D;
    const double* a = A + 2 * row * D;
    const double* x = X + 2 * rr * D;
    cd acc = cd{B[2 * t], B[2 * t + 1]};
    for (int64_t c = 0; c < D; ++c) acc = csub(acc, cmul(cd{a[2 * c], a[2 * c + 1]}, cd{x[2 * c], x[2 * c + 1]}));
    R[2 * t] = acc.x;
    R[2 * t + 1] = acc.y;
  }
}

// Solve A X = B for a dense Hermitian positive definite A (row-major complex, unchanged):
// Cholesky of a copy, triangular solves, `refine` steps of iterative refinement against A.
// X holds B on entry and the solution on exit.
fk_status solve_dense(const double* A, int64_t D, double* X, int n_rhs, int refine, cudaStream_t st, Scratch& scr,
                      unsigned* flags) {
  double *L = nullptr, *B = nullptr, *R = nullptr;
  FK_TRY(scr.alloc(&L, 2 * D * D));
  FK_TRY(scr.alloc(&B, 2 * D * n_rhs));
  FK_TRY(scr.alloc(&R, 2 * D * n_rhs));
  FK_CUDA(cudaMemcpyAsync(L, A, sizeof(double) * 2 * D * D, cudaMemcpyDeviceToDevice, st));
  FK_CUDA(cudaMemcpyAsync(B, X, sizeof(double) * 2 * D * n_rhs, cudaMemcpyDeviceToDevice, st));
  double* linv = nullptr;
  FK_TRY(scr.alloc(&linv, 2 * linv_blocks(D) * NB * NB));
  FK_TRY(cholesky(L, D, flags, st, linv));
  FK_TRY(trisolve(L, D, X, n_rhs, st, &scr, flags, linv));
  FK_CUDA(cudaGetLastError());
  for (int it = 0; it < refine; ++it) {
    k_dense_residual<<<grid_for(D * n_rhs, 128), 128, 0, st>>>(A, D, X, B, R, n_rhs); note_launch();
    FK_TRY(trisolve(L, D, R, n_rhs, st, &scr, flags, linv));
    k_axpy_c<<<grid_for(2 * D * n_rhs, 256), 256, 0, st>>>(2 * D * n_rhs, R, X); note_launch();
    FK_CUDA(cudaGetLastError());
  }
  return FK_OK;
}

}  // namespace fk

namespace fk {

// ---------------------------------------------------------------- CG in one cooperative launch
// The fused CG above costs five dependent launches per iteration (2-D) and a host
// round trip every four; at the workloads' sizes (D = 65^2, Lc = 128) each launch does
// microseconds of work.  Here all iterations run in one cooperative launch whose CTAs
// meet at a grid barrier between the three phases of an iteration:
//   P1 rows:    p = z + beta p (p = z at the first iteration) for one row of modes,
//               zero-padded to Lc and transformed along the row; sum W |p|^2;
//   P2 columns: transform along the column, times the circulant spectrum, inverse;
//               sum |p^|^2 c^ / Lc^2, the circulant's part of <p, A p> (Parseval);
//   P3 rows:    inverse transform, q = (.) / Lc^2 + W p, and, since <p, A p> is
//               complete, the row's update x += alpha p, r -= alpha q, z = r / diag
//               with its parts of <r, z> and |r|^2.
// <p, A p> from the spectrum instead of <p, q> after P3 saves a fourth phase and its
// barrier; x and r stay consistent whatever rounding alpha carries (both take the same
// alpha).  Scalars that an iteration reads and the next one accumulates are kept in two
// copies selected by the iteration's parity, so every CTA sees the same values within
// an iteration without an extra barrier.  After convergence one more matvec of x gives
// the true residual |b - A x|.  The barrier's wait is bounded (FK_ETIMEOUT).
namespace {

constexpr long long BAR_WAIT_CYCLES = 4000000000LL;  // default bound of a barrier wait: ~2 s at 2 GHz

struct GridBar {
  unsigned count, unused;  // count: arrivals since the launch (zeroed before it)
};

struct CgP {
  int K, Lc, logLc, n_rhs, nsys, maxit;
  int64_t D;
  double tol2;
  const double* T0p;  // &Re T_0
  const cplx<double>* ch;
  const double* W;
  const double* b;
  const double* tw;
  double *x, *r, *z, *p, *q;
  cplx<double>* buf;
  double *rz, *rr, *pq, *bb, *rres;  // rz, rr, pq: [2][nsys] by iteration parity
  GridBar* bar;
  unsigned* flags;
  int* info;  // [0] iterations, [1] systems not converged
  // operator penalty mu conj(P) Toep(c) (P v) (ch2 null: none); Wd: the Jacobi diagonal
  const cplx<double>* ch2;
  const double* P;
  double mu;
  const double* Wd;
  cplx<double>* buf2;
  double* idg;         // [n_w][D] inverse Jacobi diagonal 1 / (T_0 + Wd), set by the init phase
  int final_residual;  // one more matvec for |b - A x| (reports only)
  // Lc = 4m (alias): the circulant cannot tell the lags -2m and +2m apart and holds
  // +2m; the terms of lag -2m in either coordinate are added from the Toeplitz
  // entries themselves (Tc, and Cc for the operator penalty) into corr
  // [nsys][4][K]: 0/1 the moment matrix's row-0 / column-0 corrections, 2/3 the
  // operator's.
  int alias;
  const double* Tc;
  const double* Cc;
  cplx<double>* corr;
  long long wait;  // bound of each grid-barrier wait in SM cycles (0: BAR_WAIT_CYCLES)
};

// all CTAs of the launch; false when the wait gave up (the caller returns)
// The arrival counter only grows: a CTA's arrival returns the count before it, which
// names its barrier, and the CTA waits until the count reaches that barrier's last
// arrival.  The CTA barrier orders the block's writes before thread 0's releasing
// arrival, and thread 0's acquiring loads order the later barrier's reads after every
// other CTA's arrival, so no thread needs a separate fence.
__device__ bool grid_sync(GridBar* gb, unsigned* flags, long long wait) {
  const long long limit = wait > 0 ? wait : BAR_WAIT_CYCLES;
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(&gb->count) : "memory");
    const unsigned target = (old / gridDim.x + 1) * gridDim.x;
    const long long t0 = clock64();
    while (true) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(&gb->count) : "memory");
      if (static_cast<int>(v - target) >= 0) break;
      if (*reinterpret_cast<volatile unsigned*>(flags) & FLAG_TIMEOUT) {
        ok = 0;
        break;
      }
      if (clock64() - t0 > limit) {
        atomicOr(flags, FLAG_TIMEOUT);
        ok = 0;
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ bool cg_active(const CgP& A, int it, int s) {
  return __ldcg(A.rr + (it & 1) * A.nsys + s) > A.tol2 * __ldcg(A.bb + s);
}

__device__ __forceinline__ double block_sum_all(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += red[w];
  __syncthreads();
  return t;  // valid in thread 0
}

// P1: p = z + beta p and the row's transform (final: the rows of x); the penalty's
// part of <p, A p>, sum W |p|^2, goes into pq
__device__ void cgp_rows_fwd(const CgP& A, cplx<double>* sl, double* red, int it, bool final_pass) {
  const int K = A.K, Lc = A.Lc;
  for (int item = blockIdx.x; item < A.nsys * K; item += gridDim.x) {
    const int s = item / K, row = item - s * K;
    if (!final_pass && !cg_active(A, it, s)) continue;
    const int64_t o = 2 * (s * A.D + static_cast<int64_t>(row) * K);
    const double* Ws = A.W + static_cast<int64_t>(s / A.n_rhs) * A.D + static_cast<int64_t>(row) * K;
    double beta = 0.0;
    if (!final_pass && it > 0)
      beta = __ldcg(A.rz + (it & 1) * A.nsys + s) / __ldcg(A.rz + ((it + 1) & 1) * A.nsys + s);
    double pw = 0.0;
    for (int i = threadIdx.x; i < Lc; i += blockDim.x) {
      cplx<double> e;
      e.x = e.y = 0.0;
      if (i < K) {
        if (final_pass) {
          e.x = __ldcg(A.x + o + 2 * i);
          e.y = __ldcg(A.x + o + 2 * i + 1);
        } else {
          e.x = __ldcg(A.z + o + 2 * i);
          e.y = __ldcg(A.z + o + 2 * i + 1);
          if (it > 0) {
            e.x += beta * __ldcg(A.p + o + 2 * i);
            e.y += beta * __ldcg(A.p + o + 2 * i + 1);
          }
          A.p[o + 2 * i] = e.x;
          A.p[o + 2 * i + 1] = e.y;
          pw += Ws[i] * (e.x * e.x + e.y * e.y);
        }
      }
      sl[bitrev(i, A.logLc)] = e;
    }
    if (!final_pass) {
      const double t = block_sum_all(pw, red);
      if (threadIdx.x == 0) atomicAdd(A.pq + (it & 1) * A.nsys + s, t);
    }
    __syncthreads();
    fft_smem<double>(sl, Lc, -1, A.tw);
    cplx<double>* ob = A.buf + (static_cast<int64_t>(s) * K + row) * Lc;
    for (int i = threadIdx.x; i < Lc; i += blockDim.x) ob[i] = sl[i];
    __syncthreads();
    if (A.ch2) {
      // the same row times P, for the operator penalty (this thread's own writes of p)
      const double* v = final_pass ? A.x : A.p;
      for (int i = threadIdx.x; i < Lc; i += blockDim.x) {
        cplx<double> e;
        e.x = e.y = 0.0;
        if (i < K) {
          const double vr = final_pass ? __ldcg(v + o + 2 * i) : v[o + 2 * i];
          const double vi = final_pass ? __ldcg(v + o + 2 * i + 1) : v[o + 2 * i + 1];
          const int64_t pk = static_cast<int64_t>(row) * K + i;
          const double pr = A.P[2 * pk], pim = A.P[2 * pk + 1];
          e.x = pr * vr - pim * vi;
          e.y = pr * vi + pim * vr;
        }
        sl[bitrev(i, A.logLc)] = e;
      }
      __syncthreads();
      fft_smem<double>(sl, Lc, -1, A.tw);
      cplx<double>* ob2 = A.buf2 + (static_cast<int64_t>(s) * K + row) * Lc;
      for (int i = threadIdx.x; i < Lc; i += blockDim.x) ob2[i] = sl[i];
      __syncthreads();
    }
  }
}

// corrections per system: one warp per output, 8 outputs per task, for the row-0 and
// column-0 parts of each aliased product
__host__ __device__ __forceinline__ int cg_alias_tasks(int K, bool op) { return (op ? 4 : 2) * ((K + 7) / 8); }

// Lag -2m terms of the Toeplitz product for one task.  With modes indexed 0..K-1
// (j = index - m), lag (d1, d2) = j - k, and Lc = 4m, the circulant applied the
// entry at lag alias(d) (each -2m coordinate replaced by +2m) where the product wants
// T[d].  The differences are nonzero only where d1 = -2m (outputs of row 0, inputs
// from row K-1) or d2 = -2m (outputs of column 0, inputs from column K-1); the second
// set leaves out d1 = -2m, which the first already holds.
__device__ void cgp_alias_task(const CgP& A, int t, int it, bool final_pass) {
  const int K = A.K, m = (K - 1) / 2, K2 = 4 * m + 1;
  const int ngrp = (K + 7) / 8, per = cg_alias_tasks(K, A.ch2 != nullptr);
  const int s = t / per, r = t - s * per;
  const int kind = r / ngrp, g = r - kind * ngrp;
  if (!final_pass && !cg_active(A, it, s)) return;
  const int e = g * 8 + static_cast<int>(threadIdx.x >> 5);
  if (e >= K) return;
  const int lane = threadIdx.x & 31;
  const double* Tm = kind >= 2 ? A.Cc : A.Tc;
  const bool col0 = kind & 1;
  const double* v = (final_pass ? A.x : A.p) + 2 * static_cast<int64_t>(s) * A.D;
  double sr = 0.0, si = 0.0;
  for (int k = lane; k < K; k += 32) {
    const int dd = e - k + 2 * m;  // lag along the convolved coordinate, + 2m
    int64_t ia, ib;                // T entries of the true and of the applied lag
    if (!col0) {
      ia = dd;
      ib = static_cast<int64_t>(4 * m) * K2 + (dd == 0 ? 4 * m : dd);
    } else {
      if (dd == 0) continue;
      ia = static_cast<int64_t>(dd) * K2;
      ib = ia + 4 * m;
    }
    const int64_t pk = col0 ? static_cast<int64_t>(k) * K + (K - 1) : static_cast<int64_t>(K - 1) * K + k;
    double vr = __ldcg(v + 2 * pk), vi = __ldcg(v + 2 * pk + 1);
    if (kind >= 2) {
      const double pr = A.P[2 * pk], pim = A.P[2 * pk + 1];
      const double ur = pr * vr - pim * vi;
      vi = pr * vi + pim * vr;
      vr = ur;
    }
    const double dr = __ldg(Tm + 2 * ia) - __ldg(Tm + 2 * ib);
    const double di = __ldg(Tm + 2 * ia + 1) - __ldg(Tm + 2 * ib + 1);
    sr += dr * vr - di * vi;
    si += dr * vi + di * vr;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, o);
    si += __shfl_down_sync(0xffffffffu, si, o);
  }
  if (lane == 0) {
    cplx<double>& c = A.corr[(static_cast<int64_t>(s) * 4 + kind) * K + e];
    c.x = sr;
    c.y = si;
    if (!final_pass) {
      // its part of <p, A p>: Re(conj(v_j) c_j) at the output mode j (v = P p for the
      // operator's corrections, which rows_inv multiplies by mu conj(P_j))
      const int64_t pj = col0 ? static_cast<int64_t>(e) * K : static_cast<int64_t>(e);
      double vr = __ldcg(v + 2 * pj), vi = __ldcg(v + 2 * pj + 1);
      if (kind >= 2) {
        const double pr = A.P[2 * pj], pim = A.P[2 * pj + 1];
        const double ur = pr * vr - pim * vi;
        vi = pr * vi + pim * vr;
        vr = ur;
      }
      atomicAdd(A.pq + (it & 1) * A.nsys + s, (kind >= 2 ? A.mu : 1.0) * (vr * sr + vi * si));
    }
  }
}

// the correction of output (row, i): row 0 takes task 0 (2), column 0 task 1 (3)
__device__ __forceinline__ cplx<double> cg_alias_corr(const CgP& A, int s, int row, int i, int base) {
  cplx<double> c;
  c.x = c.y = 0.0;
  if (!A.alias) return c;
  const cplx<double>* cs = A.corr + static_cast<int64_t>(s) * 4 * A.K;
  if (row == 0) {
    const double2 a = __ldcg(reinterpret_cast<const double2*>(cs + base * A.K + i));
    c.x += a.x;
    c.y += a.y;
  }
  if (i == 0) {
    const double2 b = __ldcg(reinterpret_cast<const double2*>(cs + (base + 1) * A.K + row));
    c.x += b.x;
    c.y += b.y;
  }
  return c;
}

// P2 (and the alias corrections, on the CTAs past the columns)
__device__ void cgp_cols(const CgP& A, cplx<double>* sl, double* red, int it, bool final_pass) {
  const int K = A.K, Lc = A.Lc;
  const int nitems = A.nsys * Lc * (A.ch2 ? 2 : 1);
  const int ntot = nitems + (A.alias ? A.nsys * cg_alias_tasks(K, A.ch2 != nullptr) : 0);
  for (int item2 = blockIdx.x; item2 < ntot; item2 += gridDim.x) {
    if (item2 >= nitems) {
      cgp_alias_task(A, item2 - nitems, it, final_pass);
      continue;
    }
    const bool second = item2 >= A.nsys * Lc;  // the operator penalty's product
    const int item = second ? item2 - A.nsys * Lc : item2;
    const cplx<double>* spec = second ? A.ch2 : A.ch;
    cplx<double>* base = second ? A.buf2 : A.buf;
    const int s = item / Lc, c = item - s * Lc;
    if (!second && !final_pass && c == 0 && threadIdx.x == 0) {
      // next iteration's accumulators; a finished system carries its values over so
      // that it stays finished
      const bool act = cg_active(A, it, s);
      const int cur = (it & 1) * A.nsys + s, nxt = ((it + 1) & 1) * A.nsys + s;
      A.rz[nxt] = act ? 0.0 : __ldcg(A.rz + cur);
      A.rr[nxt] = act ? 0.0 : __ldcg(A.rr + cur);
      A.pq[nxt] = 0.0;
    }
    if (!final_pass && !cg_active(A, it, s)) continue;
    cplx<double>* bcol = base + static_cast<int64_t>(s) * K * Lc + c;
    for (int i = threadIdx.x; i < Lc; i += blockDim.x) {
      cplx<double> e;
      e.x = e.y = 0.0;
      if (i < K) {
        const double2 v = __ldcg(reinterpret_cast<const double2*>(bcol + static_cast<int64_t>(i) * Lc));
        e.x = v.x;
        e.y = v.y;
      }
      sl[bitrev(i, A.logLc)] = e;
    }
    __syncthreads();
    fft_smem<double>(sl, Lc, -1, A.tw);
    // <u, C u> = sum |u^|^2 c^ / Lc^2 (Parseval) for this column's spectrum: the
    // circulant product's part of <p, A p>
    double pc = 0.0;
    for (int i = threadIdx.x; i < Lc; i += blockDim.x) {
      const cplx<double> a = spec[static_cast<int64_t>(i) * Lc + c], e = sl[i];
      pc += a.x * (e.x * e.x + e.y * e.y);
      cplx<double> t;
      t.x = a.x * e.x - a.y * e.y;
      t.y = a.x * e.y + a.y * e.x;
      sl[i] = t;
    }
    if (!final_pass) {
      const double t = block_sum_all(pc, red);
      if (threadIdx.x == 0)
        atomicAdd(A.pq + (it & 1) * A.nsys + s, (second ? A.mu : 1.0) * t / (static_cast<double>(Lc) * Lc));
    }
    __syncthreads();
    bitrev_permute<double>(sl, Lc, A.logLc);
    fft_smem<double>(sl, Lc, +1, A.tw);
    for (int i = threadIdx.x; i < K; i += blockDim.x) bcol[static_cast<int64_t>(i) * Lc] = sl[i];
    __syncthreads();
  }
}

// P3: q = A v for v = p (or x in the final pass) and <p, q>
__device__ void cgp_rows_inv(const CgP& A, cplx<double>* sl, double* red, int it, bool final_pass) {
  const int K = A.K, Lc = A.Lc;
  const double inv = 1.0 / (static_cast<double>(Lc) * Lc);
  for (int item = blockIdx.x; item < A.nsys * K; item += gridDim.x) {
    const int s = item / K, row = item - s * K;
    if (!final_pass && !cg_active(A, it, s)) continue;
    const cplx<double>* bb = A.buf + (static_cast<int64_t>(s) * K + row) * Lc;
    for (int i = threadIdx.x; i < Lc; i += blockDim.x) {
      const double2 v = __ldcg(reinterpret_cast<const double2*>(bb + i));
      cplx<double> e;
      e.x = v.x;
      e.y = v.y;
      sl[bitrev(i, A.logLc)] = e;
    }
    __syncthreads();
    fft_smem<double>(sl, Lc, +1, A.tw);
    const int64_t o = 2 * (s * A.D + static_cast<int64_t>(row) * K);
    const double* Ws = A.W + static_cast<int64_t>(s / A.n_rhs) * A.D + static_cast<int64_t>(row) * K;
    const double* v = final_pass ? A.x : A.p;
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
      const double vr = __ldcg(v + o + 2 * i), vi = __ldcg(v + o + 2 * i + 1);
      const cplx<double> c = cg_alias_corr(A, s, row, i, 0);
      A.q[o + 2 * i] = sl[i].x * inv + c.x + Ws[i] * vr;
      A.q[o + 2 * i + 1] = sl[i].y * inv + c.y + Ws[i] * vi;
    }
    if (A.ch2) {
      __syncthreads();
      const cplx<double>* bb2 = A.buf2 + (static_cast<int64_t>(s) * K + row) * Lc;
      for (int i = threadIdx.x; i < Lc; i += blockDim.x) {
        const double2 w2 = __ldcg(reinterpret_cast<const double2*>(bb2 + i));
        cplx<double> e;
        e.x = w2.x;
        e.y = w2.y;
        sl[bitrev(i, A.logLc)] = e;
      }
      __syncthreads();
      fft_smem<double>(sl, Lc, +1, A.tw);
      for (int i = threadIdx.x; i < K; i += blockDim.x) {
        const int64_t pk = static_cast<int64_t>(row) * K + i;
        const double pr = A.P[2 * pk], pim = -A.P[2 * pk + 1];  // conj(P)
        const cplx<double> c = cg_alias_corr(A, s, row, i, 2);
        const double tr = sl[i].x * inv + c.x, ti = sl[i].y * inv + c.y;
        A.q[o + 2 * i] += A.mu * (pr * tr - pim * ti);
        A.q[o + 2 * i + 1] += A.mu * (pr * ti + pim * tr);
      }
    }
    // this row's update (the same threads wrote its q above): alpha = rho / <p, A p>,
    // <p, A p> complete since the column phase; x += alpha p, r -= alpha q,
    // z = r / diag, and the row's parts of <r, z> and |r|^2 for the next iteration
    // (final pass: |b - A x|^2)
    const int cur = (it & 1) * A.nsys + s, nxt = ((it + 1) & 1) * A.nsys + s;
    const double alpha = final_pass ? 0.0 : __ldcg(A.rz + cur) / __ldcg(A.pq + cur);
    const double* idg = A.idg + static_cast<int64_t>(s / A.n_rhs) * A.D + static_cast<int64_t>(row) * K;
    const double* bs = A.b + 2 * (static_cast<int64_t>(s % A.n_rhs) * A.D + static_cast<int64_t>(row) * K);
    double a1 = 0.0, a2 = 0.0;
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
      const double q0 = A.q[o + 2 * i], q1 = A.q[o + 2 * i + 1];
      if (final_pass) {
        const double e0 = bs[2 * i] - q0, e1 = bs[2 * i + 1] - q1;
        a1 += e0 * e0 + e1 * e1;
        continue;
      }
      const double p0 = __ldcg(A.p + o + 2 * i), p1 = __ldcg(A.p + o + 2 * i + 1);
      A.x[o + 2 * i] = __ldcg(A.x + o + 2 * i) + alpha * p0;
      A.x[o + 2 * i + 1] = __ldcg(A.x + o + 2 * i + 1) + alpha * p1;
      const double r0 = __ldcg(A.r + o + 2 * i) - alpha * q0, r1 = __ldcg(A.r + o + 2 * i + 1) - alpha * q1;
      A.r[o + 2 * i] = r0;
      A.r[o + 2 * i + 1] = r1;
      const double id = __ldcg(idg + i);
      A.z[o + 2 * i] = r0 * id;
      A.z[o + 2 * i + 1] = r1 * id;
      a1 += (r0 * r0 + r1 * r1) * id;
      a2 += r0 * r0 + r1 * r1;
    }
    const double t1 = block_sum_all(a1, red);
    const double t2 = final_pass ? 0.0 : block_sum_all(a2, red);
    if (threadIdx.x == 0) {
      if (final_pass) {
        atomicAdd(A.rres + s, t1);
      } else {
        atomicAdd(A.rz + nxt, t1);
        atomicAdd(A.rr + nxt, t2);
      }
    }
    __syncthreads();
  }
}

// x = 0, r = b, z = b / diag; <r, z> -> rz[0], |b|^2 -> bb and rr[0]
__device__ void cgp_init(const CgP& A, double* red, double T0) {
  const int64_t D = A.D;
  const int chunk = 4 * blockDim.x;
  const int nch = static_cast<int>((D + chunk - 1) / chunk);
  for (int item = blockIdx.x; item < A.nsys * nch; item += gridDim.x) {
    const int s = item / nch, cb = item - s * nch;
    const double* Ws = A.Wd + static_cast<int64_t>(s / A.n_rhs) * D;
    const double* bs = A.b + 2 * static_cast<int64_t>(s % A.n_rhs) * D;
    double a1 = 0.0, a2 = 0.0;
    for (int64_t k = static_cast<int64_t>(cb) * chunk + threadIdx.x; k < min(D, static_cast<int64_t>(cb + 1) * chunk);
         k += blockDim.x) {
      const int64_t o = 2 * (s * D + k);
      const double b0 = bs[2 * k], b1 = bs[2 * k + 1];
      const double id = 1.0 / (T0 + Ws[k]);
      if (s % A.n_rhs == 0) A.idg[static_cast<int64_t>(s / A.n_rhs) * D + k] = id;
      A.x[o] = 0.0;
      A.x[o + 1] = 0.0;
      A.r[o] = b0;
      A.r[o + 1] = b1;
      A.z[o] = b0 * id;
      A.z[o + 1] = b1 * id;
      a1 += (b0 * b0 + b1 * b1) * id;
      a2 += b0 * b0 + b1 * b1;
    }
    const double t1 = block_sum_all(a1, red);
    const double t2 = block_sum_all(a2, red);
    if (threadIdx.x == 0) {
      atomicAdd(A.rz + s, t1);
      atomicAdd(A.bb + s, t2);
      atomicAdd(A.rr + s, t2);
    }
  }
}

__global__ void __launch_bounds__(256) k_cg_persist2d(CgP A) {
  extern __shared__ unsigned char smem_raw[];
  cplx<double>* sl = reinterpret_cast<cplx<double>*>(smem_raw);
  __shared__ double red[32];
  double T0 = __ldg(A.T0p);
  if (!(T0 > 0.0)) T0 = 1.0;
  cgp_init(A, red, T0);
  if (!grid_sync(A.bar, A.flags, A.wait)) return;
  int it = 0;
  for (; it < A.maxit; ++it) {
    bool any = false;
    for (int s = 0; s < A.nsys && !any; ++s) any = cg_active(A, it, s);
    if (!any) break;
    cgp_rows_fwd(A, sl, red, it, false);
    if (!grid_sync(A.bar, A.flags, A.wait)) return;
    cgp_cols(A, sl, red, it, false);
    if (!grid_sync(A.bar, A.flags, A.wait)) return;
    cgp_rows_inv(A, sl, red, it, false);
    if (!grid_sync(A.bar, A.flags, A.wait)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int left = 0;
    for (int s = 0; s < A.nsys; ++s) left += cg_active(A, it, s) ? 1 : 0;
    A.info[0] = it;
    A.info[1] = left;
    if (left) atomicOr(A.flags, FLAG_NOCONV);
  }
  if (!A.final_residual) return;
  // true residual of the result
  cgp_rows_fwd(A, sl, red, it, true);
  if (!grid_sync(A.bar, A.flags, A.wait)) return;
  cgp_cols(A, sl, red, it, true);
  if (!grid_sync(A.bar, A.flags, A.wait)) return;
  cgp_rows_inv(A, sl, red, it, true);
}

}  // namespace

fk_status cg_solve_persistent(int m, const double* T, const double* W, int n_w, const double* rhs, int n_rhs,
                              const fk_opts& o, double* sol, cudaStream_t st, Scratch& scr, unsigned* flags,
                              int* iters_out, double* relres_out, bool* handled, const PenOp* op) {
  *handled = false;
  int dev = 0, coop = 0, sms = 0;
  FK_CUDA(cudaGetDevice(&dev));
  FK_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  FK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int K = 2 * m + 1;
  // the lags span 4m + 1 values; where 4m is a power of two the circulant takes
  // length 4m and the lag -2m is added separately (a quarter of the FFT work of 8m)
  const bool alias = m >= 1 && next_pow2i(4 * m) == 4 * m;
  int Lc = alias ? 4 * m : next_pow2i(4 * m + 1);
  if (Lc < 2) Lc = 2;
  int logLc = 0;
  while ((1 << logLc) < Lc) ++logLc;
  const size_t smem = sizeof(cplx<double>) * Lc;
  if (!coop || smem > 48 * 1024) return FK_OK;  // not handled: the caller uses the multi-launch form
  const int threads = 256;
  // resident CTAs per SM for this shared-memory size (cached per device)
  static std::mutex occ_mu;
  static std::map<std::pair<int, size_t>, int> occ_cache;
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lock(occ_mu);
    auto it = occ_cache.find({dev, smem});
    if (it != occ_cache.end()) {
      per_sm = it->second;
    } else {
      FK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_persist2d, threads, smem));
      occ_cache[{dev, smem}] = per_sm;
    }
  }
  if (per_sm < 1) return FK_OK;
  const int nsys = n_w * n_rhs;
  const int64_t D = static_cast<int64_t>(K) * K;
  const int64_t want = std::max<int64_t>(
      static_cast<int64_t>(nsys) * (Lc * (op ? 2 : 1) + (alias ? cg_alias_tasks(K, op != nullptr) : 0)), 1);
  const int nb = static_cast<int>(std::min<int64_t>(want, static_cast<int64_t>(std::min(per_sm, 2)) * sms));

  CgP A{};
  A.K = K;
  A.Lc = Lc;
  A.logLc = logLc;
  A.n_rhs = n_rhs;
  A.nsys = nsys;
  A.maxit = o.cg_maxit;
  A.D = D;
  A.tol2 = o.cg_tol * o.cg_tol;
  A.W = W;
  A.b = rhs;
  A.x = sol;
  int64_t centre = 2 * static_cast<int64_t>(4 * m + 1) * m + 2 * m;  // index of T_(0,0)
  A.T0p = T + 2 * centre;
  cplx<double>* ch = nullptr;
  const double* tw = nullptr;
  FK_TRY(scr.alloc(&ch, static_cast<int64_t>(Lc) * Lc));
  FK_TRY(twiddle_table(Lc, st, &tw));
  FK_CUDA(cudaMemsetAsync(ch, 0, sizeof(cplx<double>) * Lc * Lc, st));
  const int64_t M2 = static_cast<int64_t>(4 * m + 1) * (4 * m + 1);
  k_circ_embed<<<grid_for(M2, 256), 256, 0, st>>>(2, m, Lc, T, ch); note_launch();
  FK_CUDA(cudaGetLastError());
  FK_TRY(fft_lines<double>(ch, Lc, Lc, Lc, 1, -1, tw, st));
  FK_TRY(fft_lines<double>(ch, Lc, Lc, 1, Lc, -1, tw, st));
  A.ch = ch;
  A.tw = tw;
  A.Wd = W;
  if (op) {
    cplx<double>* ch2 = nullptr;
    FK_TRY(scr.alloc(&ch2, static_cast<int64_t>(Lc) * Lc));
    FK_CUDA(cudaMemsetAsync(ch2, 0, sizeof(cplx<double>) * Lc * Lc, st));
    k_circ_embed<<<grid_for(M2, 256), 256, 0, st>>>(2, m, Lc, op->c, ch2); note_launch();
    FK_CUDA(cudaGetLastError());
    FK_TRY(fft_lines<double>(ch2, Lc, Lc, Lc, 1, -1, tw, st));
    FK_TRY(fft_lines<double>(ch2, Lc, Lc, 1, Lc, -1, tw, st));
    double* wd = nullptr;
    FK_TRY(scr.alloc(&wd, D * n_w));
    k_op_diag<<<grid_for(D * n_w, 256), 256, 0, st>>>(D, n_w, W, op->P, op->c + 2 * centre, op->mu, wd); note_launch();
    FK_CUDA(cudaGetLastError());
    A.ch2 = ch2;
    A.P = op->P;
    A.mu = op->mu;
    A.Wd = wd;
    FK_TRY(scr.alloc(&A.buf2, static_cast<size_t>(nsys) * K * Lc));
  }
  A.alias = alias ? 1 : 0;
  A.Tc = T;
  A.Cc = op ? op->c : nullptr;
  if (alias) FK_TRY(scr.alloc(&A.corr, static_cast<size_t>(nsys) * 4 * K));
  FK_TRY(scr.alloc(&A.r, 2 * D * nsys));
  FK_TRY(scr.alloc(&A.idg, D * n_w));
  A.final_residual = relres_out != nullptr;
  A.wait = o.wait_cycles;
  FK_TRY(scr.alloc(&A.z, 2 * D * nsys));
  FK_TRY(scr.alloc(&A.p, 2 * D * nsys));
  FK_TRY(scr.alloc(&A.q, 2 * D * nsys));
  FK_TRY(scr.alloc(&A.buf, static_cast<size_t>(nsys) * K * Lc));
  // scalars [rz 2n | rr 2n | pq 2n | bb n | rres n | info], then the barrier: one memset,
  // and bb, rres and info come back in one copy
  double* scal = nullptr;
  FK_TRY(scr.alloc(&scal, 8 * static_cast<size_t>(nsys) + 1 + 8));
  FK_CUDA(cudaMemsetAsync(scal, 0, sizeof(double) * (8 * nsys + 1 + 8), st));
  A.rz = scal;
  A.rr = scal + 2 * nsys;
  A.pq = scal + 4 * nsys;
  A.bb = scal + 6 * nsys;
  A.rres = scal + 7 * nsys;
  A.info = reinterpret_cast<int*>(scal + 8 * nsys);
  A.bar = reinterpret_cast<GridBar*>(scal + 8 * nsys + 1);
  A.flags = flags;
  void* args[] = {&A};
  FK_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_cg_persist2d), dim3(nb), dim3(threads), args, smem,
                                      st));
  note_launch();
  if (capture_ctx()) {
    // recorded, not run: no read-back; non-convergence reaches the graph's flag word
    *handled = true;
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    return FK_OK;
  }
  std::vector<double> back(2 * static_cast<size_t>(nsys) + 1);  // bb, rres, info
  FK_CUDA(cudaMemcpyAsync(back.data(), A.bb, sizeof(double) * back.size(), cudaMemcpyDeviceToHost, st));
  FK_CUDA(cudaStreamSynchronize(st));
  *handled = true;
  const double* bb = back.data();
  const double* rres = bb + nsys;
  int info[2];
  std::memcpy(info, bb + 2 * nsys, sizeof(info));
  // a barrier that gave up sets FK_ETIMEOUT in the flag word, which the caller checks
  double worst = 0.0;
  if (relres_out)
    for (int s = 0; s < nsys; ++s) worst = std::max(worst, bb[s] > 0 ? std::sqrt(rres[s] / bb[s]) : std::sqrt(rres[s]));
  if (iters_out) *iters_out = info[0];
  if (relres_out) *relres_out = worst;
  if (info[1] != 0) return set_error(FK_ENOCONV, "CG did not converge in %d iterations", o.cg_maxit);
  return FK_OK;
}

}  // namespace fk

namespace fk {
namespace {

// Triangular solves L L^H x = b for one right-hand side in one cooperative launch.
// Forward: per 32-row block k, CTA 0 solves the diagonal block (its rows already
// carry every earlier block's update), then after one grid barrier all CTAs subtract
// block k's contribution from the rows below, CTA 0 taking block k + 1's rows first
// so that it can solve that block while the others update the rest.  Backward is the
// same on columns with conj(L)^T.  Updates of one row from different blocks are
// separated by barriers; within a phase each row has one writer.
struct TsP {
  const double* L;
  const double* Linv;  // [blocks][TS_NB][TS_NB] inverses of the diagonal blocks, or null
  int D;
  double* x;      // [D] complex, b in / solution out
  GridBar* bar;
  unsigned* flags;
  long long wait;  // bound of each grid-barrier wait in SM cycles (0: BAR_WAIT_CYCLES)
};

// all threads of CTA 0: stage the diagonal block, or its inverse (independent loads in
// flight)
__device__ void ts_stage(const TsP& A, int kb, int nb, cd* dg) {
  if (A.Linv) {
    const double* li = A.Linv + 2 * static_cast<int64_t>(kb / TS_NB) * TS_NB * TS_NB;
    for (int t = threadIdx.x; t < TS_NB * TS_NB; t += blockDim.x) {
      const int r = t / TS_NB, c = t - r * TS_NB;
      dg[r * (TS_NB + 1) + c] = cd{__ldg(li + 2 * t), __ldg(li + 2 * t + 1)};
    }
    return;
  }
  for (int t = threadIdx.x; t < TS_NB * TS_NB; t += blockDim.x) {
    const int r = t / TS_NB, c = t - r * TS_NB;
    dg[r * (TS_NB + 1) + c] = (r < nb && c <= r)
        ? cd{__ldg(A.L + 2 * (static_cast<int64_t>(kb + r) * A.D + kb + c)),
             __ldg(A.L + 2 * (static_cast<int64_t>(kb + r) * A.D + kb + c) + 1)}
        : cd{0, 0};
  }
}

// one warp of CTA 0, after ts_stage and a CTA barrier
__device__ void ts_diag(const TsP& A, int kb, int nb, bool fwd, cd* dg) {
  const int lane = threadIdx.x & 31;
  cd yv = (lane < nb) ? cd{__ldcg(A.x + 2 * (kb + lane)), __ldcg(A.x + 2 * (kb + lane) + 1)} : cd{0, 0};
  if (A.Linv) {
    // y = Linv r (forward) or Linv^H r (backward): one output per lane, two partial sums
    __shared__ cd rv[TS_NB];
    rv[lane] = yv;
    __syncwarp();
    // the inverse blocks are zero above the diagonal (and beyond nb), so full sums
    cd s0 = cd{0, 0}, s1 = cd{0, 0};
    if (fwd) {
#pragma unroll 4
      for (int j = 0; j < TS_NB; j += 2) {
        s0 = cfma(dg[lane * (TS_NB + 1) + j], rv[j], s0);
        s1 = cfma(dg[lane * (TS_NB + 1) + j + 1], rv[j + 1], s1);
      }
    } else {
#pragma unroll 4
      for (int j = 0; j < TS_NB; j += 2) {
        s0 = cjfma(dg[j * (TS_NB + 1) + lane], rv[j], s0);
        s1 = cjfma(dg[(j + 1) * (TS_NB + 1) + lane], rv[j + 1], s1);
      }
    }
    __syncwarp();
    if (lane < nb) {
      const cd v = cadd(s0, s1);
      A.x[2 * (kb + lane)] = v.x;
      A.x[2 * (kb + lane) + 1] = v.y;
    }
    return;
  }
  for (int s = 0; s < nb; ++s) {
    const int i = fwd ? s : nb - 1 - s;
    cd t = cd{0, 0};
    if (fwd && lane < i) t = cmul(dg[i * (TS_NB + 1) + lane], yv);
    if (!fwd && lane > i && lane < nb) t = cconjmul(dg[lane * (TS_NB + 1) + i], yv);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
      t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
    }
    if (lane == i) {
      const double inv = 1.0 / dg[i * (TS_NB + 1) + i].x;
      yv = cd{(yv.x - t.x) * inv, (yv.y - t.y) * inv};
    }
    __syncwarp();
  }
  if (lane < nb) {
    A.x[2 * (kb + lane)] = yv.x;
    A.x[2 * (kb + lane) + 1] = yv.y;
  }
}

__global__ void __launch_bounds__(256) k_trisolve_coop(TsP A) {
  __shared__ cd dg[TS_NB * (TS_NB + 1)];
  __shared__ cd yb[TS_NB];
  const int D = A.D;
  const int nblocks = (D + TS_NB - 1) / TS_NB;
  const int64_t gth = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int pass = 0; pass < 2; ++pass) {
    const bool fwd = (pass == 0);
    // first diagonal block of the pass
    if (blockIdx.x == 0) {
      const int kb0 = fwd ? 0 : (nblocks - 1) * TS_NB, nb0 = fwd ? min(TS_NB, D) : D - (nblocks - 1) * TS_NB;
      ts_stage(A, kb0, nb0, dg);
      __syncthreads();
      if (threadIdx.x < 32) ts_diag(A, kb0, nb0, fwd, dg);
    }
    if (!grid_sync(A.bar, A.flags, A.wait)) return;
    for (int s = 0; s < nblocks; ++s) {
      const int bi = fwd ? s : nblocks - 1 - s;
      const int kb = bi * TS_NB, nb = min(TS_NB, D - kb);
      for (int j = threadIdx.x; j < nb; j += blockDim.x)
        yb[j] = cd{__ldcg(A.x + 2 * (kb + j)), __ldcg(A.x + 2 * (kb + j) + 1)};
      __syncthreads();
      // rows (forward) or columns (backward) still to update: [lo, hi)
      const int lo = fwd ? kb + nb : 0, hi = fwd ? D : kb;
      const bool has_next = fwd ? (s + 1 < nblocks) : (bi > 0);
      const int nkb = fwd ? kb + nb : kb - TS_NB;  // next block start
      const int nnb = has_next ? min(TS_NB, D - nkb) : 0;
      auto update = [&](int r) {
        cd a0 = cd{0, 0}, a1 = cd{0, 0};
        if (fwd) {
          const double* lr = A.L + 2 * (static_cast<int64_t>(r) * D + kb);
#pragma unroll 8
          for (int j = 0; j < nb; j += 2) {
            a0 = cfma(cd{__ldg(lr + 2 * j), __ldg(lr + 2 * j + 1)}, yb[j], a0);
            if (j + 1 < nb) a1 = cfma(cd{__ldg(lr + 2 * j + 2), __ldg(lr + 2 * j + 3)}, yb[j + 1], a1);
          }
        } else {
#pragma unroll 8
          for (int j = 0; j < nb; j += 2) {
            const double* l0 = A.L + 2 * (static_cast<int64_t>(kb + j) * D + r);
            a0 = cjfma(cd{__ldg(l0), __ldg(l0 + 1)}, yb[j], a0);
            if (j + 1 < nb) a1 = cjfma(cd{__ldg(l0 + 2 * D), __ldg(l0 + 2 * D + 1)}, yb[j + 1], a1);
          }
        }
        A.x[2 * r] = __ldcg(A.x + 2 * r) - (a0.x + a1.x);
        A.x[2 * r + 1] = __ldcg(A.x + 2 * r + 1) - (a0.y + a1.y);
      };
      if (blockIdx.x == 0) {
        // the next block's rows, then its diagonal solve
        if (has_next) {
          ts_stage(A, nkb, nnb, dg);
          for (int r = nkb + threadIdx.x; r < nkb + nnb; r += blockDim.x) update(r);
          __threadfence_block();
          __syncthreads();
          if (threadIdx.x < 32) ts_diag(A, nkb, nnb, fwd, dg);
        }
      } else {
        // the rest, spread over CTAs 1 ..
        const int64_t t = static_cast<int64_t>(blockIdx.x - 1) * blockDim.x + threadIdx.x;
        const int64_t stride = gth - blockDim.x;
        for (int64_t r = t; r < hi - lo; r += stride) {
          const int rr = static_cast<int>(fwd ? lo + r : r);
          if (has_next && rr >= nkb && rr < nkb + nnb) continue;  // CTA 0's rows
          update(rr);
        }
      }
      if (!grid_sync(A.bar, A.flags, A.wait)) return;
    }
  }
}

}  // namespace

// nullptr-free launcher: returns false in *handled when a cooperative launch is not possible
fk_status trisolve_coop(const double* L, const double* Linv, int64_t D, double* X, int n_rhs, cudaStream_t st,
                        Scratch& scr, unsigned* flags, bool* handled) {
  *handled = false;
  int dev = 0, coop = 0, sms = 0;
  FK_CUDA(cudaGetDevice(&dev));
  FK_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  FK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (!coop || D < 2 * TS_NB || D > (1 << 30)) return FK_OK;
  unsigned char* misc = nullptr;
  FK_TRY(scr.alloc(&misc, 16 * static_cast<size_t>(n_rhs)));
  FK_CUDA(cudaMemsetAsync(misc, 0, 16 * static_cast<size_t>(n_rhs), st));
  for (int r = 0; r < n_rhs; ++r) {
    TsP A{L, Linv, static_cast<int>(D), X + 2 * static_cast<int64_t>(r) * D,
          reinterpret_cast<GridBar*>(misc + 16 * r), flags};
    void* args[] = {&A};
    FK_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_trisolve_coop), dim3(sms), dim3(256), args, 0,
                                        st));
    note_launch();
  }
  *handled = true;
  return FK_OK;
}

}  // namespace fk
