// Eigen route for sweeps over lambda (Sec. 5, the grid search reuses one transform pass).
//
// When every penalty of a sweep is lambda times one fixed diagonal, W_l = lambda_l S^2
// (Sobolev with a common s, low-bias with S = I, the additive model's lambda I), the
// systems (A0 + lambda_l S^2) theta = b share one Hermitian eigendecomposition
//   S^-1 A0 S^-1 = U Lambda U^H,   theta_l = S^-1 U (Lambda + lambda_l)^-1 U^H S^-1 b,
// so after one O(D^3) factorisation each lambda costs O(D^2) per right-hand side: one
// projection c = U^H S^-1 b and one product U (c / (Lambda + lambda)) for all (lambda,
// right-hand side) columns together.
//
// The decomposition is the cyclic Jacobi method in FP64 with the round-robin ordering:
// each step rotates D/2 disjoint index pairs (p, q) at once, so that one sweep of D - 1
// steps meets every pair once.  The rotation of a pair annihilates the 2 x 2 block
// [[a, h], [conj h, b]] (a, b real, h = |h| e^{i phi}):
//   G = [[c, s e^{i phi}], [-s e^{-i phi}, c]],  t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
//   tau = (b - a) / (2 |h|),  c = 1 / sqrt(1 + t^2),  s = t c,
// and A <- G^H A G, U <- U G.  A step first updates rows p and q of every pair (one CTA
// per pair, contiguous rows), then the columns, by rows: one CTA holds a row of A (or of
// U) in shared memory and applies every pair's rotation to it, so all accesses are
// coalesced.  Sweeps stop when the off-diagonal Frobenius norm falls below 1e-13 of
// the matrix's, or stops falling once below 1e-10 (checked on the host after each sweep).
#include "fk_internal.cuh"

#include <algorithm>
#include <vector>

namespace fk {
namespace {

struct Rot {
  double c, s, er, ei;  // G = [[c, s e], [-s conj(e), c]], e = er + i ei
};

// pair k of step r of the round-robin schedule over Dp (even) positions: position Dp - 1
// stays, the others turn; p < q
__device__ __forceinline__ void rr_pair(int Dp, int r, int k, int* p, int* q) {
  int a, b;
  if (k == 0) {
    a = r;
    b = Dp - 1;
  } else {
    a = (r + k) % (Dp - 1);
    b = (r - k + (Dp - 1)) % (Dp - 1);
  }
  *p = a < b ? a : b;
  *q = a < b ? b : a;
}

// rotations of step r, and the update of rows p and q of A (G^H A): one CTA per pair
__global__ void k_jac_rows(int D, int Dp, int r, double* A, Rot* rot) {
  const int k = blockIdx.x;
  int p, q;
  rr_pair(Dp, r, k, &p, &q);
  __shared__ Rot g;
  if (threadIdx.x == 0) {
    Rot R{1.0, 0.0, 1.0, 0.0};
    if (q < D) {
      const double a = A[2 * (static_cast<int64_t>(p) * D + p)];
      const double b = A[2 * (static_cast<int64_t>(q) * D + q)];
      const double hr = A[2 * (static_cast<int64_t>(p) * D + q)], hi = A[2 * (static_cast<int64_t>(p) * D + q) + 1];
      const double h = hypot(hr, hi);
      // rotate unless |h| is negligible against the diagonal (or zero)
      if (h > 1e-300 && h > 1e-18 * (fabs(a) + fabs(b))) {
        const double tau = (b - a) / (2.0 * h);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t);
        R = Rot{c, t * c, hr / h, hi / h};
      }
    }
    g = R;
    rot[k] = R;
  }
  __syncthreads();
  if (q >= D || g.s == 0.0) return;
  double* Ap = A + 2 * static_cast<int64_t>(p) * D;
  double* Aq = A + 2 * static_cast<int64_t>(q) * D;
  for (int j = threadIdx.x; j < D; j += blockDim.x) {
    const double pr = Ap[2 * j], pi = Ap[2 * j + 1], qr = Aq[2 * j], qi = Aq[2 * j + 1];
    // row p: c A_p - s e A_q;  row q: s conj(e) A_p + c A_q
    Ap[2 * j] = g.c * pr - g.s * (g.er * qr - g.ei * qi);
    Ap[2 * j + 1] = g.c * pi - g.s * (g.er * qi + g.ei * qr);
    Aq[2 * j] = g.s * (g.er * pr + g.ei * pi) + g.c * qr;
    Aq[2 * j + 1] = g.s * (g.er * pi - g.ei * pr) + g.c * qi;
  }
}

// columns p, q of every pair (M G), row by row: CTA i < D takes row i of A, CTA D + i
// row i of U; the row sits in shared memory while all pairs' rotations apply
__global__ void k_jac_cols(int D, int Dp, int r, double* A, double* U, const Rot* rot) {
  extern __shared__ double row[];  // [2 D]
  const int which = blockIdx.x >= D;
  const int i = blockIdx.x - which * D;
  double* M = (which ? U : A) + 2 * static_cast<int64_t>(i) * D;
  for (int j = threadIdx.x; j < 2 * D; j += blockDim.x) row[j] = M[j];
  __syncthreads();
  for (int k = threadIdx.x; k < Dp / 2; k += blockDim.x) {
    int p, q;
    rr_pair(Dp, r, k, &p, &q);
    if (q >= D) continue;
    const Rot g = rot[k];
    if (g.s == 0.0) continue;
    const double pr = row[2 * p], pi = row[2 * p + 1], qr = row[2 * q], qi = row[2 * q + 1];
    // column p: c M_p - s conj(e) M_q;  column q: s e M_p + c M_q
    row[2 * p] = g.c * pr - g.s * (g.er * qr + g.ei * qi);
    row[2 * p + 1] = g.c * pi - g.s * (g.er * qi - g.ei * qr);
    row[2 * q] = g.s * (g.er * pr - g.ei * pi) + g.c * qr;
    row[2 * q + 1] = g.s * (g.er * pi + g.ei * pr) + g.c * qi;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < 2 * D; j += blockDim.x) M[j] = row[j];
}

// out[0] += sum of |A_ij|^2 off the diagonal, out[1] += sum over all entries
__global__ void k_jac_norms(int D, const double* A, double* out) {
  double off = 0.0, all = 0.0;
  const int64_t total = static_cast<int64_t>(D) * D;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double v = A[2 * t] * A[2 * t] + A[2 * t + 1] * A[2 * t + 1];
    all += v;
    if (t / D != t % D) off += v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    off += __shfl_down_sync(0xffffffffu, off, o);
    all += __shfl_down_sync(0xffffffffu, all, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out, off);
    atomicAdd(out + 1, all);
  }
}

__global__ void k_eye(int D, double* U) {
  const int64_t total = static_cast<int64_t>(D) * D;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    U[2 * t] = (t / D == t % D) ? 1.0 : 0.0;
    U[2 * t + 1] = 0.0;
  }
}

__global__ void k_diag_real(int D, const double* A, double* ev) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < D; i += gridDim.x * blockDim.x)
    ev[i] = A[2 * (static_cast<int64_t>(i) * D + i)];
}

// A[r][c] *= sinv[r] sinv[c]
__global__ void k_scale_sym(int D, const double* sinv, double* A) {
  const int64_t total = static_cast<int64_t>(D) * D;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double f = sinv[t / D] * sinv[t % D];
    A[2 * t] *= f;
    A[2 * t + 1] *= f;
  }
}

// c[rhs][j] = sum_i conj(U[i][j]) sinv_i b[rhs][i]: one CTA per (j, rhs)
__global__ void k_eig_project(int D, const double* U, const double* sinv, const double* b, double* c) {
  const int j = blockIdx.x, rhs = blockIdx.y;
  const double* br = b + 2 * static_cast<int64_t>(rhs) * D;
  double sr = 0.0, si = 0.0;
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    const double ur = U[2 * (static_cast<int64_t>(i) * D + j)], ui = U[2 * (static_cast<int64_t>(i) * D + j) + 1];
    const double f = sinv ? sinv[i] : 1.0;
    const double xr = br[2 * i] * f, xi = br[2 * i + 1] * f;
    sr += ur * xr + ui * xi;
    si += ur * xi - ui * xr;
  }
  __shared__ double red[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, o);
    si += __shfl_down_sync(0xffffffffu, si, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sr;
    red[1][threadIdx.x >> 5] = si;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, bb = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
      a += red[0][w];
      bb += red[1][w];
    }
    c[2 * (static_cast<int64_t>(rhs) * D + j)] = a;
    c[2 * (static_cast<int64_t>(rhs) * D + j) + 1] = bb;
  }
}

struct LamArr {
  double v[256];
};

// sol[l][rhs][i] = sinv_i sum_j U[i][j] c[rhs][j] / (ev_j + lambda_l), 16 x 16 output
// tiles (16 rows i by 16 columns (l, rhs)) with shared-memory tiles of U and of the
// scaled projections
constexpr int ET = 16;
__global__ void k_eig_back(int D, int n_rhs, int n_lam, LamArr lam, const double* U, const double* sinv,
                           const double* ev, const double* c, double* sol) {
  __shared__ double ut[ET][ET][2];
  __shared__ double yt[ET][ET][2];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.y * ET + ty;      // output row
  const int col = blockIdx.x * ET + tx;    // output column (l, rhs)
  const int ncol = n_lam * n_rhs;
  double ar = 0.0, ai = 0.0;
  for (int j0 = 0; j0 < D; j0 += ET) {
    // U[i][j0 + tx]
    {
      const int j = j0 + tx;
      const bool ok = i < D && j < D;
      ut[ty][tx][0] = ok ? U[2 * (static_cast<int64_t>(i) * D + j)] : 0.0;
      ut[ty][tx][1] = ok ? U[2 * (static_cast<int64_t>(i) * D + j) + 1] : 0.0;
    }
    // y[j0 + ty][col] = c[rhs][j] / (ev_j + lambda_l)
    {
      const int j = j0 + ty;
      const int cc = blockIdx.x * ET + tx;
      double yr = 0.0, yi = 0.0;
      if (j < D && cc < ncol) {
        const int l = cc / n_rhs, rhs = cc - l * n_rhs;
        const double den = 1.0 / (ev[j] + lam.v[l]);
        yr = c[2 * (static_cast<int64_t>(rhs) * D + j)] * den;
        yi = c[2 * (static_cast<int64_t>(rhs) * D + j) + 1] * den;
      }
      yt[ty][tx][0] = yr;
      yt[ty][tx][1] = yi;
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < ET; ++jj) {
      const double ur = ut[ty][jj][0], ui = ut[ty][jj][1];
      const double yr = yt[jj][tx][0], yi = yt[jj][tx][1];
      ar = fma(ur, yr, fma(-ui, yi, ar));
      ai = fma(ur, yi, fma(ui, yr, ai));
    }
    __syncthreads();
  }
  if (i < D && col < ncol) {
    const double f = sinv ? sinv[i] : 1.0;
    sol[2 * (static_cast<int64_t>(col) * D + i)] = ar * f;
    sol[2 * (static_cast<int64_t>(col) * D + i) + 1] = ai * f;
  }
}

}  // namespace

// Hermitian eigendecomposition of A (D x D complex, row-major; overwritten): U (D x D,
// columns are eigenvectors) and ev (D eigenvalues, unsorted).
fk_status eig_hermitian(int64_t D64, double* A, double* U, double* ev, cudaStream_t st, Scratch& scr, int* sweeps_out) {
  if (D64 < 1 || D64 > 16384) return set_error(FK_EINVAL, "eigendecomposition: D = %lld outside [1, 16384]",
                                               static_cast<long long>(D64));
  const int D = static_cast<int>(D64);
  const int Dp = D + (D & 1);
  Rot* rot = nullptr;
  double* nrm = nullptr;
  FK_TRY(scr.alloc(&rot, static_cast<size_t>(Dp / 2)));
  FK_TRY(scr.alloc(&nrm, 2));
  k_eye<<<grid_for(D64 * D64, 256), 256, 0, st>>>(D, U); note_launch();
  FK_CUDA(cudaGetLastError());
  const size_t row_smem = sizeof(double) * 2 * D;
  if (row_smem > 48 * 1024)
    FK_CUDA(cudaFuncSetAttribute(k_jac_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(row_smem)));
  int sweep = 0;
  double prev = 0.0;
  for (; sweep < 40; ++sweep) {
    FK_CUDA(cudaMemsetAsync(nrm, 0, 2 * sizeof(double), st));
    k_jac_norms<<<grid_for(D64 * D64, 256, 148 * 4), 256, 0, st>>>(D, A, nrm); note_launch();
    double h[2] = {0.0, 0.0};
    FK_CUDA(cudaMemcpyAsync(h, nrm, sizeof(h), cudaMemcpyDeviceToHost, st));
    FK_CUDA(cudaStreamSynchronize(st));
    // converged: off-diagonal norm below 1e-13 of the matrix's, or no longer halving once
    // below 1e-10 (the rounding floor, about D eps, has been reached)
    if (!(h[0] > 1e-26 * h[1])) break;
    if (sweep > 0 && h[0] > 0.25 * prev && h[0] <= 1e-20 * h[1]) break;
    prev = h[0];
    for (int r = 0; r < Dp - 1; ++r) {
      k_jac_rows<<<Dp / 2, 256, 0, st>>>(D, Dp, r, A, rot); note_launch();
      k_jac_cols<<<2 * D, 256, row_smem, st>>>(D, Dp, r, A, U, rot); note_launch();
    }
    FK_CUDA(cudaGetLastError());
  }
  if (sweep == 40) return set_error(FK_ENOCONV, "Jacobi eigendecomposition did not converge in 40 sweeps");
  k_diag_real<<<grid_for(D, 256), 256, 0, st>>>(D, A, ev); note_launch();
  FK_CUDA(cudaGetLastError());
  if (sweeps_out) *sweeps_out = sweep;
  return FK_OK;
}

// theta[l][rhs] = S^-1 U (ev + lambda_l)^-1 U^H S^-1 b[rhs] for the decomposition of
// S^-1 A0 S^-1 (sinv = 1/S, or null for S = I).
fk_status eig_sweep_solve(int64_t D, const double* U, const double* ev, const double* sinv, const double* b,
                          int n_rhs, const double* lambdas, int n_lambda, double* sol, cudaStream_t st, Scratch& scr) {
  // each system must be positive definite: smallest eigenvalue + lambda > 0 (as the
  // Cholesky route's pivots)
  std::vector<double> evh(static_cast<size_t>(D));
  FK_CUDA(cudaMemcpyAsync(evh.data(), ev, sizeof(double) * D, cudaMemcpyDeviceToHost, st));
  FK_CUDA(cudaStreamSynchronize(st));
  double emin = evh[0];
  for (double v : evh) emin = std::min(emin, v);
  for (int l = 0; l < n_lambda; ++l)
    if (!(emin + lambdas[l] > 0.0))
      return set_error(FK_ENOTPD, "eigen route: smallest eigenvalue %.3g + lambda %.3g is not positive", emin,
                       lambdas[l]);
  double* c = nullptr;
  FK_TRY(scr.alloc(&c, 2 * static_cast<size_t>(D) * n_rhs));
  k_eig_project<<<dim3(static_cast<unsigned>(D), n_rhs), 256, 0, st>>>(static_cast<int>(D), U, sinv, b, c);
  note_launch();
  FK_CUDA(cudaGetLastError());
  for (int l0 = 0; l0 < n_lambda; l0 += 256) {
    const int nl = std::min(256, n_lambda - l0);
    LamArr la{};
    for (int l = 0; l < nl; ++l) la.v[l] = lambdas[l0 + l];
    const int ncol = nl * n_rhs;
    k_eig_back<<<dim3((ncol + ET - 1) / ET, static_cast<unsigned>((D + ET - 1) / ET)), dim3(ET, ET), 0, st>>>(
        static_cast<int>(D), n_rhs, nl, la, U, sinv, ev, c, sol + 2 * static_cast<int64_t>(l0) * n_rhs * D);
    note_launch();
    FK_CUDA(cudaGetLastError());
  }
  return FK_OK;
}

fk_status eig_scale_sym(int64_t D, const double* sinv, double* A, cudaStream_t st) {
  k_scale_sym<<<grid_for(D * D, 256), 256, 0, st>>>(static_cast<int>(D), sinv, A); note_launch();
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}

}  // namespace fk
