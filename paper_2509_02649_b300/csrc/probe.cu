// Measurement helper: the FP32 FMA throughput of the current device, the peak against
// which the spreading kernels' flop rates are reported (no counterpart in the paper).
//
// One launch of 2048 threads per SM (four 512-thread CTAs), each thread running eight
// independent FMA chains (a = a b + c, which stays bounded), timed with CUDA events
// on the caller's stream: the best of three launches after one warm-up.
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

}  // namespace
}  // namespace fk

using namespace fk;

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
