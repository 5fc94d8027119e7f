// Measurement helpers (no counterpart in the paper): the peaks the kernels' rates are
// reported against.
// * FP32 FMA throughput: one launch of 2048 threads per SM (four 512-thread CTAs), each
//   thread running eight independent FMA chains (a = a b + c, which stays bounded).
// * 32-bit shared-memory atomic adds with a returned value: two 1024-thread CTAs per
//   SM, each thread adding into windows of 7 consecutive words (the 1-D spreader's
//   access), with the 32 lanes of a warp instruction on 32 different banks or at
//   random.
// Each is timed with CUDA events on the caller's stream: the best of three launches
// after one warm-up.
#include "fk_internal.cuh"

namespace fk {
namespace {

constexpr int PROBE_THREADS = 512;
constexpr int PROBE_CTAS_PER_SM = 4;
constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_UNROLL = 8;
constexpr int PROBE_ITERS = 4096;

__global__ void __launch_bounds__(PROBE_THREADS, PROBE_CTAS_PER_SM) k_ffma_probe(float b, float c, float* sink,
                                                                                int keep) {
  float a[PROBE_CHAINS];
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = static_cast<float>(threadIdx.x + k) * 1e-3f;
  for (int it = 0; it < PROBE_ITERS; ++it) {
#pragma unroll
    for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
      for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
  if (keep) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keep (never taken: keep = 0)
}

constexpr int ATOM_THREADS = 1024;
constexpr int ATOM_CTAS_PER_SM = 2;
constexpr int ATOM_WORDS = 3 * 8208;  // three 8192-node grids with their 16-node halos
constexpr int ATOM_ITERS = 2048;
constexpr int ATOM_TAPS = 7;

__device__ __forceinline__ unsigned probe_hash(unsigned x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

// window starts: lane + 32 r for a random row r (every lane on its own bank, for each of
// the 7 taps), or uniformly random; all windows inside the array
template <bool RANDOM>
__global__ void __launch_bounds__(ATOM_THREADS, ATOM_CTAS_PER_SM) k_atom_probe(unsigned* sink, int keep) {
  extern __shared__ unsigned words[];
  for (int i = threadIdx.x; i < ATOM_WORDS; i += blockDim.x) words[i] = 0u;
  __syncthreads();
  const unsigned lane = threadIdx.x & 31u;
  unsigned h = probe_hash(threadIdx.x + 7919u * blockIdx.x);
  unsigned acc = 0u;
  for (int it = 0; it < ATOM_ITERS; ++it) {
    h = probe_hash(h + static_cast<unsigned>(it));
    // (h & 511) 32 + 31 + 6 < ATOM_WORDS, and h % (ATOM_WORDS - 8) + 6 < ATOM_WORDS
    const unsigned base = RANDOM ? h % static_cast<unsigned>(ATOM_WORDS - 8) : (h & 511u) * 32u + lane;
#pragma unroll
    for (int a = 0; a < ATOM_TAPS; ++a) acc += atomicAdd(&words[base + a], h & 0xFFu);
  }
  __syncthreads();
  if (keep) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc + words[threadIdx.x];  // never taken
}

// best of three timed launches after a warm-up, in ms
template <typename F>
fk_status best_ms(cudaStream_t st, F launch, float* out) {
  cudaEvent_t e0, e1;
  FK_CUDA(cudaEventCreate(&e0));
  FK_CUDA(cudaEventCreate(&e1));
  float best = 0.f;
  fk_status rc = FK_OK;
  for (int rep = 0; rep < 4 && rc == FK_OK; ++rep) {
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      rc = set_error(FK_ECUDA, "probe: %s", cudaGetErrorString(e));
      break;
    }
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;  // launch 0 warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  FK_TRY(rc);
  *out = best;
  return FK_OK;
}

}  // namespace
}  // namespace fk

using namespace fk;

extern "C" fk_status fk_peak_smem_atomics(double* gops_distinct, double* gops_random, void* stream) {
  clear_error();
  if (!gops_distinct || !gops_random) return set_error(FK_EINVAL, "null output");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, false, false, "fk_peak_smem_atomics"));
  const int sms = sm_count();
  if (sms <= 0) return set_error(FK_ECUDA, "no multiprocessor count for the current device");
  const int grid = sms * ATOM_CTAS_PER_SM;
  const size_t smem = sizeof(unsigned) * ATOM_WORDS;
  FK_CUDA(cudaFuncSetAttribute(k_atom_probe<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  FK_CUDA(cudaFuncSetAttribute(k_atom_probe<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  float ms_d = 0.f, ms_r = 0.f;
  FK_TRY(best_ms(st, [&] { k_atom_probe<false><<<grid, ATOM_THREADS, smem, st>>>(nullptr, 0); note_launch(); }, &ms_d));
  FK_TRY(best_ms(st, [&] { k_atom_probe<true><<<grid, ATOM_THREADS, smem, st>>>(nullptr, 0); note_launch(); }, &ms_r));
  const double ops = static_cast<double>(grid) * ATOM_THREADS * ATOM_ITERS * ATOM_TAPS;
  *gops_distinct = ops / (ms_d * 1e-3) / 1e9;
  *gops_random = ops / (ms_r * 1e-3) / 1e9;
  return FK_OK;
}

extern "C" fk_status fk_peak_fp32(double* tflops, int* sms_out, void* stream) {
  clear_error();
  if (!tflops) return set_error(FK_EINVAL, "null output");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, false, false, "fk_peak_fp32"));
  const int sms = sm_count();
  if (sms <= 0) return set_error(FK_ECUDA, "no multiprocessor count for the current device");
  const int grid = sms * PROBE_CTAS_PER_SM;
  cudaEvent_t e0, e1;
  FK_CUDA(cudaEventCreate(&e0));
  FK_CUDA(cudaEventCreate(&e1));
  float best = 0.f;
  fk_status rc = FK_OK;
  for (int rep = 0; rep < 4 && rc == FK_OK; ++rep) {
    cudaEventRecord(e0, st);
    k_ffma_probe<<<grid, PROBE_THREADS, 0, st>>>(0.9999999f, 1e-7f, nullptr, 0); note_launch();
    cudaEventRecord(e1, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      rc = set_error(FK_ECUDA, "FMA probe: %s", cudaGetErrorString(e));
      break;
    }
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;  // launch 0 warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  FK_TRY(rc);
  const double fmas = static_cast<double>(grid) * PROBE_THREADS * PROBE_ITERS * PROBE_UNROLL * PROBE_CHAINS;
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  if (sms_out) *sms_out = sms;
  return FK_OK;
}
