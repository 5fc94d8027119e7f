// Power-of-two complex FFTs of short lines held in shared memory, plus the
// fused "transform the upsampled grid, deconvolve, extract the wanted modes"
// kernels of the type-1 path and the "place corrected modes, inverse transform"
// kernels of the type-2 path.
//
// One CTA transforms one line (N <= 8192 for fp64, <= 16384 for fp32): the line
// is loaded in bit-reversed order, then log2 N radix-2 decimation-in-time stages
// run in place in shared memory.  Twiddles e^{-2 pi i t / N} come from an fp64
// table built once per plan with sincospi.
#include "fk_internal.cuh"

#include <map>
#include <mutex>
#include <utility>
#include "fft_device.cuh"

namespace fk {

__global__ void k_twiddles(int N, double* tw) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  double s, c;
  sincospi(-2.0 * t / N, &s, &c);
  tw[2 * t] = c;
  tw[2 * t + 1] = s;
}

fk_status fft_twiddles(int N, double* tw, cudaStream_t st) {
  k_twiddles<<<(N + 255) / 256, 256, 0, st>>>(N, tw); note_launch();
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}

// Twiddle tables depend only on N: computed once per device and N, kept for the
// life of the process (during a stream capture the first computation runs on a
// stream of its own, outside the graph).
fk_status twiddle_table(int N, cudaStream_t st, const double** out) {
  int dev = 0;
  FK_CUDA(cudaGetDevice(&dev));
  static std::mutex mtx;
  static std::map<std::pair<int, int>, double*> cache;
  std::lock_guard<std::mutex> lock(mtx);
  const auto key = std::make_pair(dev, N);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *out = it->second;
    return FK_OK;
  }
  double* tw = nullptr;
  FK_CUDA(cudaMalloc(&tw, sizeof(double) * 2 * static_cast<size_t>(N)));
  cudaStream_t cs = st;
  if (capture_ctx() && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(tw);
    return set_error(FK_ECUDA, "twiddle stream");
  }
  fk_status rc = fft_twiddles(N, tw, cs);
  if (rc == FK_OK && cudaStreamSynchronize(cs) != cudaSuccess) rc = set_error(FK_ECUDA, "twiddle table");
  if (cs != st) cudaStreamDestroy(cs);
  if (rc != FK_OK) {
    cudaFree(tw);
    return rc;
  }
  cache.emplace(key, tw);
  *out = tw;
  return FK_OK;
}

// ---------------------------------------------------------------- generic lines
template <typename R>
__global__ void k_fft_lines(cplx<R>* data, int N, int logN, int64_t line_stride, int64_t elem_stride,
                            int sign, const double* tw) {
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* s = reinterpret_cast<cplx<R>*>(smem_raw);
  cplx<R>* line = data + static_cast<int64_t>(blockIdx.x) * line_stride;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s[bitrev(i, logN)] = line[i * elem_stride];
  __syncthreads();
  fft_smem<R>(s, N, sign, tw);
  for (int i = threadIdx.x; i < N; i += blockDim.x) line[i * elem_stride] = s[i];
}

static int ilog2(int N) {
  int l = 0;
  while ((1 << l) < N) ++l;
  return l;
}

template <typename R>
fk_status fft_lines(cplx<R>* data, int N, int64_t n_lines, int64_t line_stride, int64_t elem_stride,
                    int sign, const double* tw, cudaStream_t st) {
  const size_t sm = static_cast<size_t>(N) * sizeof(cplx<R>);
  if (sm > 200 * 1024) return set_error(FK_EINVAL, "FFT line of %d too long", N);
  if (sm > 48 * 1024) FK_CUDA(cudaFuncSetAttribute(k_fft_lines<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  for (int64_t l0 = 0; l0 < n_lines; l0 += 65535) {
    const int nl = static_cast<int>(std::min<int64_t>(65535, n_lines - l0));
    k_fft_lines<R><<<nl, 256, sm, st>>>(data + l0 * line_stride, N, ilog2(N), line_stride, elem_stride, sign, tw); note_launch();
    FK_CUDA(cudaGetLastError());
  }
  return FK_OK;
}
template fk_status fft_lines<float>(cplx<float>*, int, int64_t, int64_t, int64_t, int, const double*, cudaStream_t);
template fk_status fft_lines<double>(cplx<double>*, int, int64_t, int64_t, int64_t, int, const double*, cudaStream_t);

// ---------------------------------------------------------------- type-1 side
// 1-D: line c of the real grid -> modes |j| <= kout, times corr and scale.
template <typename R>
__global__ void k_t1_1d(const double* grid, int N, int logN, int c0, int kout, const double* corr,
                        int corr_off, double scale, const double* tw, double* out) {
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* s = reinterpret_cast<cplx<R>*>(smem_raw);
  const int c = blockIdx.x;
  const double* g = grid + static_cast<int64_t>(c0 + c) * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    cplx<R> v;
    v.x = static_cast<R>(g[i]);
    v.y = R(0);
    s[bitrev(i, logN)] = v;
  }
  __syncthreads();
  fft_smem<R>(s, N, -1, tw);
  const int K = 2 * kout + 1;
  double* o = out + static_cast<int64_t>(c) * 2 * K;
  for (int t = threadIdx.x; t < K; t += blockDim.x) {
    const int j = t - kout;
    const cplx<R> v = s[(j + N) & (N - 1)];
    const double f = corr[t + corr_off] * scale;
    o[2 * t] = static_cast<double>(v.x) * f;
    o[2 * t + 1] = static_cast<double>(v.y) * f;
  }
}

// 2-D step 1: rows (dim 1) of the real grid -> H[c][l0][jj], jj = j1 + kout.
template <typename R>
__global__ void k_t1_2d_rows(const double* grid, int N, int logN, int c0, int kout, const double* tw,
                             cplx<R>* H) {
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* s = reinterpret_cast<cplx<R>*>(smem_raw);
  const int64_t line = blockIdx.x;  // = c * N + l0
  const double* g = grid + (static_cast<int64_t>(c0) * N + line) * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    cplx<R> v;
    v.x = static_cast<R>(g[i]);
    v.y = R(0);
    s[bitrev(i, logN)] = v;
  }
  __syncthreads();
  fft_smem<R>(s, N, -1, tw);
  const int K = 2 * kout + 1;
  cplx<R>* h = H + line * K;
  for (int t = threadIdx.x; t < K; t += blockDim.x) h[t] = s[(t - kout + N) & (N - 1)];
}

// 2-D step 2: columns of H -> out[c][(j0 + kout) K + jj] with corr(j0) corr(j1) scale.
template <typename R>
__global__ void k_t1_2d_cols(const cplx<R>* H, int N, int logN, int kout, const double* corr, int corr_off,
                             double scale, const double* tw, double* out) {
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* s = reinterpret_cast<cplx<R>*>(smem_raw);
  const int K = 2 * kout + 1;
  const int c = blockIdx.x / K;
  const int jj = blockIdx.x - c * K;
  const cplx<R>* h = H + static_cast<int64_t>(c) * N * K + jj;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s[bitrev(i, logN)] = h[static_cast<int64_t>(i) * K];
  __syncthreads();
  fft_smem<R>(s, N, -1, tw);
  double* o = out + static_cast<int64_t>(c) * 2 * K * K;
  const double fj1 = corr[jj + corr_off] * scale;
  for (int t = threadIdx.x; t < K; t += blockDim.x) {
    const int j0 = t - kout;
    const cplx<R> v = s[(j0 + N) & (N - 1)];
    const double f = corr[t + corr_off] * fj1;
    const int64_t idx = static_cast<int64_t>(t) * K + jj;
    o[2 * idx] = static_cast<double>(v.x) * f;
    o[2 * idx + 1] = static_cast<double>(v.y) * f;
  }
}

// 3-D: lines of dimension 2 (contiguous, real grid) -> H1[line][jj2], then lines of
// dimension 1 -> H2[c][i0][jj1][jj2], then dimension 0 with corr and scale.
template <typename R>
__global__ void k_t1_3d_a(const double* grid, int N, int logN, int c0, int kout, const double* tw, cplx<R>* H1) {
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* s = reinterpret_cast<cplx<R>*>(smem_raw);
  const int64_t line = blockIdx.x;  // (c N + i0) N + i1
  const double* g = grid + (static_cast<int64_t>(c0) * N * N + line) * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    cplx<R> v;
    v.x = static_cast<R>(g[i]);
    v.y = R(0);
    s[bitrev(i, logN)] = v;
  }
  __syncthreads();
  fft_smem<R>(s, N, -1, tw);
  const int K = 2 * kout + 1;
  for (int t = threadIdx.x; t < K; t += blockDim.x) H1[line * K + t] = s[(t - kout + N) & (N - 1)];
}

template <typename R>
__global__ void k_t1_3d_b(const cplx<R>* H1, int N, int logN, int kout, const double* tw, cplx<R>* H2) {
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* s = reinterpret_cast<cplx<R>*>(smem_raw);
  const int K = 2 * kout + 1;
  const int64_t b = blockIdx.x;  // (c N + i0) K + jj2
  const int64_t ci0 = b / K;
  const int jj2 = static_cast<int>(b - ci0 * K);
  const cplx<R>* h = H1 + ci0 * N * K + jj2;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s[bitrev(i, logN)] = h[static_cast<int64_t>(i) * K];
  __syncthreads();
  fft_smem<R>(s, N, -1, tw);
  for (int t = threadIdx.x; t < K; t += blockDim.x) H2[(ci0 * K + t) * K + jj2] = s[(t - kout + N) & (N - 1)];
}

template <typename R>
__global__ void k_t1_3d_c(const cplx<R>* H2, int N, int logN, int kout, const double* corr, int corr_off,
                          double scale, const double* tw, double* out) {
  extern __shared__ unsigned char smem_raw[];
  cplx<R>* s = reinterpret_cast<cplx<R>*>(smem_raw);
  const int K = 2 * kout + 1;
  const int64_t KK = static_cast<int64_t>(K) * K;
  const int64_t b = blockIdx.x;  // c K K + jj1 K + jj2
  const int64_t c = b / KK;
  const int64_t rem = b - c * KK;
  const int jj1 = static_cast<int>(rem / K), jj2 = static_cast<int>(rem - static_cast<int64_t>(jj1) * K);
  const cplx<R>* h = H2 + c * N * KK + rem;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s[bitrev(i, logN)] = h[static_cast<int64_t>(i) * KK];
  __syncthreads();
  fft_smem<R>(s, N, -1, tw);
  double* o = out + c * 2 * KK * K;
  const double f12 = corr[jj1 + corr_off] * corr[jj2 + corr_off] * scale;
  for (int t = threadIdx.x; t < K; t += blockDim.x) {
    const cplx<R> v = s[(t - kout + N) & (N - 1)];
    const double f = corr[t + corr_off] * f12;
    const int64_t idx = static_cast<int64_t>(t) * KK + rem;
    o[2 * idx] = static_cast<double>(v.x) * f;
    o[2 * idx + 1] = static_cast<double>(v.y) * f;
  }
}

template <typename R>
static fk_status set_smem(const void* fn, size_t sm) {
  if (sm > 48 * 1024) FK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  return FK_OK;
}

template <typename R>
fk_status grid_to_modes(const EsPlan& p, const double* grid, int c0, int nc, int kout,
                        const double* corr, double scale, double* out, cudaStream_t st,
                        Scratch& scratch) {
  if (kout > p.kmax) return set_error(FK_EINTERNAL, "kout %d > kmax %d", kout, p.kmax);
  const int N = p.N, logN = ilog2(N);
  const size_t sm = static_cast<size_t>(N) * sizeof(cplx<R>);
  if (sm > 200 * 1024) return set_error(FK_EINVAL, "fine grid %d too long for one CTA", N);
  const int corr_off = p.kmax - kout;
  const double* tw = nullptr;
  FK_TRY(twiddle_table(N, st, &tw));
  const int K = 2 * kout + 1;
  if (p.d == 1) {
    FK_TRY(set_smem<R>((const void*)k_t1_1d<R>, sm));
    k_t1_1d<R><<<nc, 256, sm, st>>>(grid, N, logN, c0, kout, corr, corr_off, scale, tw, out); note_launch();
    FK_CUDA(cudaGetLastError());
  } else if (p.d == 2) {
    cplx<R>* H = nullptr;
    FK_TRY(scratch.alloc(&H, static_cast<size_t>(nc) * N * K));
    FK_TRY(set_smem<R>((const void*)k_t1_2d_rows<R>, sm));
    FK_TRY(set_smem<R>((const void*)k_t1_2d_cols<R>, sm));
    k_t1_2d_rows<R><<<nc * N, 256, sm, st>>>(grid, N, logN, c0, kout, tw, H); note_launch();
    FK_CUDA(cudaGetLastError());
    k_t1_2d_cols<R><<<nc * K, 256, sm, st>>>(H, N, logN, kout, corr, corr_off, scale, tw, out); note_launch();
    FK_CUDA(cudaGetLastError());
  } else if (p.d == 3) {
    cplx<R>* H1 = nullptr;
    cplx<R>* H2 = nullptr;
    FK_TRY(scratch.alloc(&H1, static_cast<size_t>(nc) * N * N * K));
    FK_TRY(scratch.alloc(&H2, static_cast<size_t>(nc) * N * K * K));
    FK_TRY(set_smem<R>((const void*)k_t1_3d_a<R>, sm));
    FK_TRY(set_smem<R>((const void*)k_t1_3d_b<R>, sm));
    FK_TRY(set_smem<R>((const void*)k_t1_3d_c<R>, sm));
    k_t1_3d_a<R><<<static_cast<unsigned>(static_cast<int64_t>(nc) * N * N), 256, sm, st>>>(grid, N, logN, c0, kout, tw,
                                                                                           H1);
    note_launch();
    k_t1_3d_b<R><<<static_cast<unsigned>(static_cast<int64_t>(nc) * N * K), 256, sm, st>>>(H1, N, logN, kout, tw, H2);
    note_launch();
    k_t1_3d_c<R><<<static_cast<unsigned>(static_cast<int64_t>(nc) * K * K), 256, sm, st>>>(H2, N, logN, kout, corr,
                                                                                           corr_off, scale, tw, out);
    note_launch();
    FK_CUDA(cudaGetLastError());
  } else {
    return set_error(FK_EINVAL, "d = %d transforms are not built", p.d);
  }
  return FK_OK;
}
template fk_status grid_to_modes<float>(const EsPlan&, const double*, int, int, int, const double*, double,
                                        double*, cudaStream_t, Scratch&);
template fk_status grid_to_modes<double>(const EsPlan&, const double*, int, int, int, const double*, double,
                                         double*, cudaStream_t, Scratch&);

}  // namespace fk

namespace fk {

// Same as grid_to_modes, with the twiddle table (2 N doubles, filled by fft_twiddles)
// and, for d = 2, the row-transform intermediate (nc * N * (2 kout + 1) complex values)
// supplied by the caller instead of allocated.
template <typename R>
fk_status grid_to_modes_into(const EsPlan& p, const double* grid, int c0, int nc, int kout, const double* corr,
                             double scale, double* out, cudaStream_t st, double* tw, cplx<R>* H) {
  if (kout > p.kmax) return set_error(FK_EINTERNAL, "kout %d > kmax %d", kout, p.kmax);
  const int N = p.N, logN = ilog2(N);
  const size_t sm = static_cast<size_t>(N) * sizeof(cplx<R>);
  if (sm > 200 * 1024) return set_error(FK_EINVAL, "fine grid %d too long for one CTA", N);
  const int corr_off = p.kmax - kout;
  const int K = 2 * kout + 1;
  if (p.d == 1) {
    FK_TRY(set_smem<R>((const void*)k_t1_1d<R>, sm));
    k_t1_1d<R><<<nc, 256, sm, st>>>(grid, N, logN, c0, kout, corr, corr_off, scale, tw, out); note_launch();
    FK_CUDA(cudaGetLastError());
  } else if (p.d == 2) {
    FK_TRY(set_smem<R>((const void*)k_t1_2d_rows<R>, sm));
    FK_TRY(set_smem<R>((const void*)k_t1_2d_cols<R>, sm));
    k_t1_2d_rows<R><<<nc * N, 256, sm, st>>>(grid, N, logN, c0, kout, tw, H); note_launch();
    FK_CUDA(cudaGetLastError());
    k_t1_2d_cols<R><<<nc * K, 256, sm, st>>>(H, N, logN, kout, corr, corr_off, scale, tw, out); note_launch();
    FK_CUDA(cudaGetLastError());
  } else {
    return set_error(FK_EINVAL, "d = %d transforms are not built", p.d);
  }
  return FK_OK;
}
fk_status preload_modes_kernels() {
  cudaFuncAttributes fa;
  FK_CUDA(cudaFuncGetAttributes(&fa, k_twiddles));
  FK_CUDA(cudaFuncGetAttributes(&fa, k_t1_1d<float>));
  FK_CUDA(cudaFuncGetAttributes(&fa, k_t1_1d<double>));
  FK_CUDA(cudaFuncGetAttributes(&fa, k_t1_2d_rows<float>));
  FK_CUDA(cudaFuncGetAttributes(&fa, k_t1_2d_rows<double>));
  FK_CUDA(cudaFuncGetAttributes(&fa, k_t1_2d_cols<float>));
  FK_CUDA(cudaFuncGetAttributes(&fa, k_t1_2d_cols<double>));
  return FK_OK;
}

template fk_status grid_to_modes_into<float>(const EsPlan&, const double*, int, int, int, const double*, double,
                                             double*, cudaStream_t, double*, cplx<float>*);
template fk_status grid_to_modes_into<double>(const EsPlan&, const double*, int, int, int, const double*, double,
                                              double*, cudaStream_t, double*, cplx<double>*);

}  // namespace fk
