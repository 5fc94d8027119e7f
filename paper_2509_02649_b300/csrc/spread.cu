// Spreading (type-1) and interpolation (type-2) with the ES kernel, atomic form.
//
// Point i with coordinate x sits at grid position u = (x + pi) / h, h = 2 pi / N.
// Its window is the w nodes l = l0 .. l0 + w - 1 with l0 = ceil(u - w/2), and node l
// receives the weight phi(z) with z = (l - u) * 2 / w in [-1, 1),
// phi(z) = exp(beta (sqrt(1-z^2) - 1)).  Indices wrap modulo N (the grid is periodic);
// window.cuh computes l0 and the offset u - l0.
//
// This file holds the straightforward form: one thread per point, fp64 global
// atomics into the grid.  It is the FP64 path's spreader and the fallback of the
// mixed path; the register-accumulating binned spreader lives in spread_binned.cu.
#include "fk_internal.cuh"
#include "window.cuh"
#include "es_poly.cuh"

namespace fk {

constexpr int MAXW = 16;

// Window start l0 and offset f of one coordinate (window.cuh); false outside [-3 pi, 3 pi).
template <typename R> struct Win;
template <> struct Win<double> {
  int N, W;
  __device__ __forceinline__ bool operator()(double x, int* l0, double* f) const { return window_f64(x, N, W, l0, f); }
};
template <> struct Win<float> {
  int N, W;
  float c_hi, c_lo;
  __device__ __forceinline__ bool operator()(float x, int* l0, float* f) const {
    return window_f32(x, N, c_hi, c_lo, W, l0, f);
  }
};

template <typename R>
Win<R> make_win(int N, int W);
template <> Win<double> make_win<double>(int N, int W) { return Win<double>{N, W}; }
template <> Win<float> make_win<float>(int N, int W) {
  const CoordConst c = coord_const(N);
  return Win<float>{N, W, c.hi, c.lo};
}

template <typename R>
__device__ __forceinline__ R es_phi(R z, R beta);
template <> __device__ __forceinline__ double es_phi<double>(double z, double beta) {
  return exp(beta * (sqrt(1.0 - z * z) - 1.0));
}
template <> __device__ __forceinline__ float es_phi<float>(float z, float beta) {
  return expf(beta * (sqrtf(fmaxf(1.0f - z * z, 0.0f)) - 1.0f));
}

// Weights ker[a] = psi((a - f) 2 / w), a = 0..w-1.
template <typename R>
__device__ __forceinline__ void es_weights(R f, int w, R beta, R* ker) {
  const R sc = R(2) / w;
#pragma unroll
  for (int a = 0; a < MAXW; ++a)
    if (a < w) ker[a] = es_phi<R>((a - f) * sc, beta);
}

template <typename R>
__global__ void k_spread_atomic(int d, Win<R> win, R beta, int64_t n, const R* __restrict__ x,
                                const R* __restrict__ y, int n_y, int with_ones, double* grid,
                                unsigned* flags) {
  const int N = win.N, w = win.W;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t G = (d == 1) ? N : (d == 2 ? static_cast<int64_t>(N) * N : static_cast<int64_t>(N) * N * N);
  const int nc = n_y + with_ones;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    R ker[3][MAXW];
    int l0[3];
    bool ok = true;
    for (int l = 0; l < d; ++l) {
      R f;
      if (!win(x[l * n + i], &l0[l], &f)) { ok = false; break; }
      es_weights<R>(f, w, beta, ker[l]);
    }
    if (!ok) { atomicOr(flags, FLAG_RANGE); continue; }
    for (int c = 0; c < nc; ++c) {
      const double str = (with_ones && c == 0) ? 1.0 : static_cast<double>(y[(c - with_ones) * n + i]);
      double* g = grid + c * G;
      if (d == 1) {
        for (int a = 0; a < w; ++a) {
          const int idx = wrap_node(l0[0] + a, N);
          atomicAdd(g + idx, str * static_cast<double>(ker[0][a]));
        }
      } else if (d == 2) {
        for (int a = 0; a < w; ++a) {
          const int r = wrap_node(l0[0] + a, N);
          const double sa = str * static_cast<double>(ker[0][a]);
          for (int b = 0; b < w; ++b) {
            const int cidx = wrap_node(l0[1] + b, N);
            atomicAdd(g + static_cast<int64_t>(r) * N + cidx, sa * static_cast<double>(ker[1][b]));
          }
        }
      } else {
        for (int a = 0; a < w; ++a) {
          const int64_t r = wrap_node(l0[0] + a, N);
          const double sa = str * static_cast<double>(ker[0][a]);
          for (int b = 0; b < w; ++b) {
            const int64_t rb = r * N + wrap_node(l0[1] + b, N);
            const double sb = sa * static_cast<double>(ker[1][b]);
            for (int c = 0; c < w; ++c)
              atomicAdd(g + rb * N + wrap_node(l0[2] + c, N), sb * static_cast<double>(ker[2][c]));
          }
        }
      }
    }
  }
}

template <typename R>
fk_status spread_atomic(const EsPlan& p, int64_t n, const R* x, const R* y, int n_y, bool with_ones,
                        double* grid, unsigned* flags, cudaStream_t st) {
  if (p.d < 1 || p.d > 3) return set_error(FK_EINVAL, "spread: d = %d not built", p.d);
  if (p.w > MAXW) return set_error(FK_EINTERNAL, "w > %d", MAXW);
  const int nc = n_y + (with_ones ? 1 : 0);
  int64_t G = 1;
  for (int l = 0; l < p.d; ++l) G *= p.N;
  FK_CUDA(cudaMemsetAsync(grid, 0, sizeof(double) * G * nc, st));
  if (n == 0) return FK_OK;
  const int block = 256;
  KernelTimer* kt = kernel_timer();
  if (kt->on) cudaEventRecordWithFlags(kt->start, st, kt->rec_flags);
  k_spread_atomic<R><<<grid_for(n, block, 148 * 16), block, 0, st>>>(
      p.d, make_win<R>(p.N, p.w), static_cast<R>(p.beta), n, x, y, n_y, with_ones ? 1 : 0, grid, flags); note_launch();
  if (kt->on) {
    cudaEventRecordWithFlags(kt->stop, st, kt->rec_flags);
    kt->recorded = true;
  }
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}
// ---------------------------------------------------------------- deterministic form
// Each contribution str * prod psi is rounded to a 64-bit fixed-point integer and added
// with integer atomics, whose sums do not depend on the order of the additions; the
// integer sums are then scaled back into the fp64 grid, so repeated runs give the same
// bits.  Scale of channel c: S_c = 2^(61 - e_c) with n max|str_c| <= 2^e_c (ones: max 1);
// every |product| <= max|str_c| (the ES weights are <= 1), so every partial sum stays
// below 2^61 + n in magnitude, and each contribution is rounded to the nearest multiple
// of 2^(e_c - 61), a relative error of at most n 2^-62 of the channel's largest possible
// sum.

template <typename R>
__global__ void k_absmax_det(int64_t n, const R* __restrict__ y, int n_y, unsigned long long* amax) {
  const int c = blockIdx.y;
  const R* yc = y + static_cast<int64_t>(c) * n;
  double m = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double a = fabs(static_cast<double>(yc[i]));
    m = (a > m) ? a : m;  // NaN inputs are left out
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  // non-negative doubles order as their bit patterns
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(amax + c, static_cast<unsigned long long>(__double_as_longlong(m)));
}

// scale[c] = 2^(61 - e_c), inv[c] = 2^(e_c - 61), n max|str_c| <= 2^e_c
__global__ void k_det_scale(int nc, int with_ones, int64_t n, const unsigned long long* amax, double* scale,
                            double* inv) {
  const int c = threadIdx.x;
  if (c >= nc) return;
  const double m = (with_ones && c == 0) ? 1.0 : __longlong_as_double(static_cast<long long>(amax[c - with_ones]));
  const double tot = m * static_cast<double>(n);
  int e = 0;
  if (tot > 0.0) {
    const double fr = frexp(tot, &e);  // tot = fr 2^e, fr in [0.5, 1): tot <= 2^e
    (void)fr;
  }
  scale[c] = ldexp(1.0, 61 - e);
  inv[c] = ldexp(1.0, e - 61);
}

template <typename R>
__global__ void k_spread_det(int d, Win<R> win, R beta, int64_t n, const R* __restrict__ x, const R* __restrict__ y,
                             int n_y, int with_ones, const double* __restrict__ scale, unsigned long long* acc,
                             unsigned* flags) {
  const int N = win.N, w = win.W;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t G = (d == 1) ? N : (d == 2 ? static_cast<int64_t>(N) * N : static_cast<int64_t>(N) * N * N);
  const int nc = n_y + with_ones;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    R ker[3][MAXW];
    int l0[3];
    bool ok = true;
    for (int l = 0; l < d; ++l) {
      R f;
      if (!win(x[l * n + i], &l0[l], &f)) { ok = false; break; }
      es_weights<R>(f, w, beta, ker[l]);
    }
    if (!ok) { atomicOr(flags, FLAG_RANGE); continue; }
    for (int c = 0; c < nc; ++c) {
      const double str = ((with_ones && c == 0) ? 1.0 : static_cast<double>(y[(c - with_ones) * n + i])) * scale[c];
      unsigned long long* g = acc + c * G;
      if (d == 1) {
        for (int a = 0; a < w; ++a)
          atomicAdd(g + wrap_node(l0[0] + a, N),
                    static_cast<unsigned long long>(__double2ll_rn(str * static_cast<double>(ker[0][a]))));
      } else if (d == 2) {
        for (int a = 0; a < w; ++a) {
          const int64_t r = wrap_node(l0[0] + a, N);
          const double sa = str * static_cast<double>(ker[0][a]);
          for (int b = 0; b < w; ++b)
            atomicAdd(g + r * N + wrap_node(l0[1] + b, N),
                      static_cast<unsigned long long>(__double2ll_rn(sa * static_cast<double>(ker[1][b]))));
        }
      } else {
        for (int a = 0; a < w; ++a) {
          const int64_t r = wrap_node(l0[0] + a, N);
          const double sa = str * static_cast<double>(ker[0][a]);
          for (int b = 0; b < w; ++b) {
            const int64_t rb = r * N + wrap_node(l0[1] + b, N);
            const double sb = sa * static_cast<double>(ker[1][b]);
            for (int cc = 0; cc < w; ++cc)
              atomicAdd(g + rb * N + wrap_node(l0[2] + cc, N),
                        static_cast<unsigned long long>(__double2ll_rn(sb * static_cast<double>(ker[2][cc]))));
          }
        }
      }
    }
  }
}

__global__ void k_det_to_grid(int64_t total, int64_t G, const double* inv, const unsigned long long* acc,
                              double* grid) {
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x)
    grid[t] = static_cast<double>(static_cast<long long>(acc[t])) * inv[t / G];
}

template <typename R>
fk_status spread_deterministic(const EsPlan& p, int64_t n, const R* x, const R* y, int n_y, bool with_ones,
                               double* grid, unsigned* flags, cudaStream_t st, Scratch& scr) {
  if (p.d < 1 || p.d > 3) return set_error(FK_EINVAL, "spread: d = %d not built", p.d);
  if (p.w > MAXW) return set_error(FK_EINTERNAL, "w > %d", MAXW);
  const int nc = n_y + (with_ones ? 1 : 0);
  if (nc < 1 || nc > 1024) return set_error(FK_EINVAL, "deterministic spreading: %d channels", nc);
  int64_t G = 1;
  for (int l = 0; l < p.d; ++l) G *= p.N;
  unsigned long long *acc = nullptr, *amax = nullptr;
  double* sc = nullptr;
  FK_TRY(scr.alloc(&acc, static_cast<size_t>(G) * nc));
  FK_TRY(scr.alloc(&amax, static_cast<size_t>(n_y > 0 ? n_y : 1)));
  FK_TRY(scr.alloc(&sc, 2 * static_cast<size_t>(nc)));
  FK_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * G * nc, st));
  FK_CUDA(cudaMemsetAsync(amax, 0, sizeof(unsigned long long) * (n_y > 0 ? n_y : 1), st));
  if (n_y > 0 && n > 0) {
    if (n_y > 65535) return set_error(FK_EINVAL, "deterministic spreading: %d channels", n_y);
    k_absmax_det<R><<<dim3(grid_for(n, 256, 148 * 8), n_y), 256, 0, st>>>(n, y, n_y, amax); note_launch();
    FK_CUDA(cudaGetLastError());
  }
  k_det_scale<<<1, 1024, 0, st>>>(nc, with_ones ? 1 : 0, n, amax, sc, sc + nc); note_launch();
  FK_CUDA(cudaGetLastError());
  if (n > 0) {
    KernelTimer* kt = kernel_timer();
    if (kt->on) cudaEventRecordWithFlags(kt->start, st, kt->rec_flags);
    k_spread_det<R><<<grid_for(n, 256, 148 * 16), 256, 0, st>>>(p.d, make_win<R>(p.N, p.w), static_cast<R>(p.beta), n,
                                                                   x, y, n_y, with_ones ? 1 : 0, sc, acc, flags);
    note_launch();
    if (kt->on) {
      cudaEventRecordWithFlags(kt->stop, st, kt->rec_flags);
      kt->recorded = true;
    }
    FK_CUDA(cudaGetLastError());
  }
  const int64_t total = G * nc;
  k_det_to_grid<<<grid_for(total, 256), 256, 0, st>>>(total, G, sc + nc, acc, grid); note_launch();
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}
template fk_status spread_deterministic<float>(const EsPlan&, int64_t, const float*, const float*, int, bool, double*,
                                               unsigned*, cudaStream_t, Scratch&);
template fk_status spread_deterministic<double>(const EsPlan&, int64_t, const double*, const double*, int, bool,
                                                double*, unsigned*, cudaStream_t, Scratch&);

fk_status preload_spread_atomic_kernels() {
  cudaFuncAttributes fa;
  FK_CUDA(cudaFuncGetAttributes(&fa, k_spread_atomic<float>));
  FK_CUDA(cudaFuncGetAttributes(&fa, k_spread_atomic<double>));
  return FK_OK;
}

template fk_status spread_atomic<float>(const EsPlan&, int64_t, const float*, const float*, int, bool, double*,
                                        unsigned*, cudaStream_t);
template fk_status spread_atomic<double>(const EsPlan&, int64_t, const double*, const double*, int, bool,
                                         double*, unsigned*, cudaStream_t);

// ---------------------------------------------------------------- type 2
// Place coef'_k = coef_k * corr(k) at node (k mod N) of a zeroed complex grid,
// inverse-transform (sign +1) and keep the real part; then interpolate.
template <typename R>
__global__ void k_t2_place(int d, int N, int kc, int corr_off, const double* coef, int n_sets,
                           const double* corr, cplx<R>* G) {
  const int K = 2 * kc + 1;
  int64_t D = 1, GN = 1;
  for (int l = 0; l < d; ++l) {
    D *= K;
    GN *= N;
  }
  const int64_t total = D * n_sets;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int sidx = static_cast<int>(t / D);
    const int64_t q = t - sidx * D;
    double f;
    int64_t node;
    if (d == 1) {
      const int k = static_cast<int>(q) - kc;
      f = corr[q + corr_off];
      node = (k + N) & (N - 1);
    } else if (d == 2) {
      const int a = static_cast<int>(q / K), b = static_cast<int>(q - static_cast<int64_t>(a) * K);
      f = corr[a + corr_off] * corr[b + corr_off];
      node = static_cast<int64_t>((a - kc + N) & (N - 1)) * N + ((b - kc + N) & (N - 1));
    } else {
      const int a = static_cast<int>(q / (static_cast<int64_t>(K) * K));
      const int64_t rem = q - static_cast<int64_t>(a) * K * K;
      const int b = static_cast<int>(rem / K), c = static_cast<int>(rem - static_cast<int64_t>(b) * K);
      f = corr[a + corr_off] * corr[b + corr_off] * corr[c + corr_off];
      node = (static_cast<int64_t>((a - kc + N) & (N - 1)) * N + ((b - kc + N) & (N - 1))) * N +
             ((c - kc + N) & (N - 1));
    }
    cplx<R> v;
    v.x = static_cast<R>(coef[2 * t] * f);
    v.y = static_cast<R>(coef[2 * t + 1] * f);
    G[sidx * GN + node] = v;
  }
}

template <typename R>
__global__ void k_t2_interp(int d, Win<R> win, R beta, int64_t n, const R* __restrict__ x, int n_sets,
                            const cplx<R>* __restrict__ G, double* out, unsigned* flags) {
  const int N = win.N, w = win.W;
  int64_t GN = 1;
  for (int l = 0; l < d; ++l) GN *= N;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    R ker[3][MAXW];
    int l0[3];
    bool ok = true;
    for (int l = 0; l < d; ++l) {
      R f;
      if (!win(x[l * n + i], &l0[l], &f)) { ok = false; break; }
      es_weights<R>(f, w, beta, ker[l]);
    }
    if (!ok) {
      atomicOr(flags, FLAG_RANGE);
      for (int s = 0; s < n_sets; ++s) out[s * n + i] = 0.0;
      continue;
    }
    for (int s = 0; s < n_sets; ++s) {
      const cplx<R>* g = G + s * GN;
      double acc = 0.0;
      if (d == 1) {
        for (int a = 0; a < w; ++a) acc += static_cast<double>(ker[0][a]) * static_cast<double>(g[wrap_node(l0[0] + a, N)].x);
      } else if (d == 2) {
        for (int a = 0; a < w; ++a) {
          const int r = wrap_node(l0[0] + a, N);
          R row = R(0);
          for (int b = 0; b < w; ++b) row += ker[1][b] * g[static_cast<int64_t>(r) * N + (wrap_node(l0[1] + b, N))].x;
          acc += static_cast<double>(ker[0][a]) * static_cast<double>(row);
        }
      } else {
        for (int a = 0; a < w; ++a) {
          const int64_t r = wrap_node(l0[0] + a, N);
          R plane = R(0);
          for (int b = 0; b < w; ++b) {
            const int64_t rb = r * N + wrap_node(l0[1] + b, N);
            R row = R(0);
            for (int c = 0; c < w; ++c) row += ker[2][c] * g[rb * N + wrap_node(l0[2] + c, N)].x;
            plane += ker[1][b] * row;
          }
          acc += static_cast<double>(ker[0][a]) * static_cast<double>(plane);
        }
      }
      out[s * n + i] = acc;
    }
  }
}

// Interpolation in 2-D, fp32, fine grids of at most T2S_MAXN^2 nodes: each CTA stages the
// real parts of the grid (the only part Re f needs) in shared memory once, rows padded
// by W - 1 columns that repeat the first ones (so a window's columns are contiguous),
// and takes the W taps of each coordinate from the tap polynomials.  Row sums in fp32;
// the W row terms are summed with error-free transformations (two-product, two-sum),
// so the outer sum is as accurate as a double one without FP64 instructions.
constexpr int T2S_MAXN = 128;
template <int W>
__global__ void __launch_bounds__(256) k_t2_interp2d_smem(Win<float> win, EsPoly poly, int64_t n,
                                                          const float* __restrict__ x, int n_sets,
                                                          const cplx<float>* __restrict__ G, double* out,
                                                          unsigned* flags) {
  extern __shared__ float gr[];  // [N][N + W - 1]
  const int N = win.N, ld = N + W - 1;
  const float gc = 0.5f * static_cast<float>(W - 1);
  for (int s = 0; s < n_sets; ++s) {
    const cplx<float>* g = G + static_cast<int64_t>(s) * N * N;
    __syncthreads();  // the previous set's reads are done
    for (int t = threadIdx.x; t < N * ld; t += blockDim.x) {
      const int r = t / ld, c = t - r * ld;
      gr[t] = g[r * N + (c & (N - 1))].x;
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
      int l0, l1;
      float f0, f1;
      if (!win(x[i], &l0, &f0) || !win(x[n + i], &l1, &f1)) {
        if (s == 0) atomicOr(flags, FLAG_RANGE);
        out[static_cast<int64_t>(s) * n + i] = 0.0;
        continue;
      }
      float k0[W], k1[W];
      es_taps_poly<W>(f0 - gc, poly, k0);
      es_taps_poly<W>(f1 - gc, poly, k1);
      const int r0 = wrap_node(l0, N);
      const float* col = gr + wrap_node(l1, N);
      float hi = 0.f, lo = 0.f;  // outer sum as hi + lo
#pragma unroll
      for (int a = 0; a < W; ++a) {
        const float* row = col + ((r0 + a) & (N - 1)) * ld;
        float rs = 0.f;
#pragma unroll
        for (int b = 0; b < W; ++b) rs = fmaf(k1[b], row[b], rs);
        // two-product: k0 rs = p + e exactly; two-sum: hi + p = u + v exactly (explicitly
        // rounded operations, so that none is contracted into an FMA)
        const float pr = __fmul_rn(k0[a], rs);
        const float e = fmaf(k0[a], rs, -pr);
        const float u = __fadd_rn(hi, pr);
        const float bb = __fsub_rn(u, hi);
        const float v = __fadd_rn(__fsub_rn(hi, __fsub_rn(u, bb)), __fsub_rn(pr, bb));
        hi = u;
        lo += e + v;
      }
      out[static_cast<int64_t>(s) * n + i] = static_cast<double>(hi) + static_cast<double>(lo);
    }
  }
}

template <int W>
fk_status launch_t2_smem(const EsPlan& p, int n_sets, int64_t n, const float* x, const cplx<float>* G, double* out,
                         unsigned* flags, cudaStream_t st) {
  const size_t sm = sizeof(float) * static_cast<size_t>(p.N) * (p.N + W - 1);
  FK_CUDA(cudaFuncSetAttribute(k_t2_interp2d_smem<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm)));
  int per_sm = 1;
  FK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_t2_interp2d_smem<W>, 256, sm));
  const int blocks = grid_for(n, 256, std::max(1, per_sm) * std::max(1, sm_count()));
  k_t2_interp2d_smem<W><<<blocks, 256, sm, st>>>(make_win<float>(p.N, p.w), es_poly(p.w, p.beta), n, x, n_sets, G, out,
                                                 flags);
  note_launch();
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}

// the shared-memory interpolation where it applies (2-D, fp32, N <= T2S_MAXN, 4 <= w <= 8)
template <typename R>
bool t2_smem_launch(const EsPlan&, int, int64_t, const R*, const cplx<R>*, double*, unsigned*, cudaStream_t,
                    fk_status*) {
  return false;
}
template <>
bool t2_smem_launch<float>(const EsPlan& p, int n_sets, int64_t n, const float* x, const cplx<float>* G, double* out,
                           unsigned* flags, cudaStream_t st, fk_status* rc) {
  if (p.d != 2 || p.N > T2S_MAXN || p.N < 16) return false;
  switch (p.w) {
    case 4: *rc = launch_t2_smem<4>(p, n_sets, n, x, G, out, flags, st); return true;
    case 5: *rc = launch_t2_smem<5>(p, n_sets, n, x, G, out, flags, st); return true;
    case 6: *rc = launch_t2_smem<6>(p, n_sets, n, x, G, out, flags, st); return true;
    case 7: *rc = launch_t2_smem<7>(p, n_sets, n, x, G, out, flags, st); return true;
    case 8: *rc = launch_t2_smem<8>(p, n_sets, n, x, G, out, flags, st); return true;
    default: return false;
  }
}

template <typename R>
fk_status type2_eval(const EsPlan& p, int kmax_c, const double* coef, int n_sets, int64_t n, const R* x,
                     const double* corr, double* out, unsigned* flags, cudaStream_t st, Scratch& scratch) {
  if (p.d < 1 || p.d > 3) return set_error(FK_EINVAL, "type 2: d = %d not built", p.d);
  if (kmax_c > p.kmax) return set_error(FK_EINTERNAL, "type 2: kmax_c > plan kmax");
  const int N = p.N;
  int64_t GN = 1;
  for (int l = 0; l < p.d; ++l) GN *= N;
  cplx<R>* G = nullptr;
  const double* tw = nullptr;
  FK_TRY(scratch.alloc(&G, GN * n_sets));
  FK_TRY(twiddle_table(N, st, &tw));
  FK_CUDA(cudaMemsetAsync(G, 0, sizeof(cplx<R>) * GN * n_sets, st));
  const int K = 2 * kmax_c + 1;
  int64_t D = 1;
  for (int l = 0; l < p.d; ++l) D *= K;
  k_t2_place<R><<<grid_for(D * n_sets, 256), 256, 0, st>>>(p.d, N, kmax_c, p.kmax - kmax_c, coef, n_sets, corr, G); note_launch();
  FK_CUDA(cudaGetLastError());
  if (p.d == 1) {
    FK_TRY(fft_lines<R>(G, N, n_sets, N, 1, +1, tw, st));
  } else if (p.d == 3) {
    // every line of each dimension: last, middle (one call per first index), first
    const int64_t NN = static_cast<int64_t>(N) * N;
    FK_TRY(fft_lines<R>(G, N, static_cast<int64_t>(n_sets) * NN, N, 1, +1, tw, st));
    for (int64_t s2 = 0; s2 < static_cast<int64_t>(n_sets) * N; ++s2)
      FK_TRY(fft_lines<R>(G + s2 * NN, N, N, 1, N, +1, tw, st));
    for (int sidx = 0; sidx < n_sets; ++sidx) FK_TRY(fft_lines<R>(G + sidx * GN, N, NN, 1, NN, +1, tw, st));
  } else {
    // columns first (only the K nonzero ones per set), then every row
    for (int s = 0; s < n_sets; ++s) {
      cplx<R>* Gs = G + s * GN;
      // columns with index (b - kc) mod N for b = 0..K-1: two contiguous ranges
      const int lo_cnt = kmax_c + 1;  // columns 0..kc
      FK_TRY(fft_lines<R>(Gs, N, lo_cnt, 1, N, +1, tw, st));
      if (kmax_c > 0) FK_TRY(fft_lines<R>(Gs + (N - kmax_c), N, kmax_c, 1, N, +1, tw, st));
    }
    FK_TRY(fft_lines<R>(G, N, static_cast<int64_t>(n_sets) * N, N, 1, +1, tw, st));
  }
  if (n > 0) {
    fk_status rc = FK_OK;
    if (t2_smem_launch<R>(p, n_sets, n, x, G, out, flags, st, &rc)) return rc;
    k_t2_interp<R><<<grid_for(n, 256, 148 * 16), 256, 0, st>>>(p.d, make_win<R>(N, p.w), static_cast<R>(p.beta), n, x, n_sets,
                                                               G, out, flags); note_launch();
    FK_CUDA(cudaGetLastError());
  }
  return FK_OK;
}
template fk_status type2_eval<float>(const EsPlan&, int, const double*, int, int64_t, const float*, const double*,
                                     double*, unsigned*, cudaStream_t, Scratch&);
template fk_status type2_eval<double>(const EsPlan&, int, const double*, int, int64_t, const double*,
                                      const double*, double*, unsigned*, cudaStream_t, Scratch&);

}  // namespace fk
