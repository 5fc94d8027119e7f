// On-device generation of the 1-D sweep workload at scale (points and targets drawn
// from a counter-based generator, so any chunk of the sample can be made on its own
// and the host can reproduce it).
//
// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC 2011): a ten-round bijection of a
// 128-bit counter under a 64-bit key; each round multiplies counter words 0 and 2 by
// 0xD2511F53 and 0xCD9E8D57, mixes the high halves with words 1 and 3 and the key,
// and the key is bumped by 0x9E3779B9 / 0xBB67AE85 between rounds.
//
// Draws for point i (j = i / 4, r = i mod 4), key (seed mod 2^32, workload):
//   X_i   = fp32(u 2pi_f - pi_f), u = (word_r >> 9 + 1/2) 2^-23 of counter (j, 0, 0);
//   z_ti  = Box-Muller of words (2p, 2p+1), p = r / 2, of counter (j, 1 + t, 0):
//           sqrt(-2 ln u1) cos(2 pi u2) for even r, sin(2 pi u2) for odd r;
//   Y_ti  = sign(X_i) |X_i|^0.7 + 0.2 z_ti.
// Max |Y_t| of the chunk is returned as well (it sets the fixed-point scale of the
// 1-D spreader without another pass over Y).
#include "fk_internal.cuh"

namespace fk {

namespace {

struct U4 {
  unsigned a, b, c, d;
};

__device__ __forceinline__ U4 philox4x32_10(U4 ctr, unsigned k0, unsigned k1) {
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const unsigned lo0 = 0xD2511F53u * ctr.a, hi0 = __umulhi(0xD2511F53u, ctr.a);
    const unsigned lo1 = 0xCD9E8D57u * ctr.c, hi1 = __umulhi(0xCD9E8D57u, ctr.c);
    ctr = U4{hi1 ^ ctr.b ^ k0, lo1, hi0 ^ ctr.d ^ k1, lo0};
  }
  return ctr;
}

__device__ __forceinline__ float unit_f32(unsigned w) {
  return fmaf(static_cast<float>(w >> 9), 1.0f / 8388608.0f, 1.0f / 16777216.0f);
}

__device__ __forceinline__ unsigned word(const U4& v, int r) {
  return r == 0 ? v.a : (r == 1 ? v.b : (r == 2 ? v.c : v.d));
}

__global__ void k_gen_sweep(unsigned k0, unsigned k1, int64_t first, int64_t n, int n_t, float* __restrict__ x,
                            float* __restrict__ y, unsigned* amax) {
  const int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;  // quad of points
  const int64_t i0 = 4 * q;                                                        // offset in the chunk
  const bool live = i0 < n;
  const uint64_t j = static_cast<uint64_t>(first) / 4 + static_cast<uint64_t>(q);
  const unsigned jlo = static_cast<unsigned>(j), jhi = static_cast<unsigned>(j >> 32);
  const float twopi_f = 6.28318548202514648f, pi_f = 3.14159274101257324f;
  float xv[4], fs[4];
  if (live) {
    const U4 w = philox4x32_10(U4{jlo, jhi, 0u, 0u}, k0, k1);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      xv[r] = fmaf(unit_f32(word(w, r)), twopi_f, -pi_f);
      fs[r] = copysignf(powf(fabsf(xv[r]), 0.7f), xv[r]);
    }
    if (i0 + 3 < n && (reinterpret_cast<uintptr_t>(x + i0) & 15) == 0) {
      *reinterpret_cast<float4*>(x + i0) = make_float4(xv[0], xv[1], xv[2], xv[3]);
    } else {
      for (int r = 0; r < 4; ++r)
        if (i0 + r < n) x[i0 + r] = xv[r];
    }
  }
  // four targets per trip: independent Philox / Box-Muller chains interleave
#pragma unroll 4
  for (int t = 0; t < n_t; ++t) {
    float m = 0.f;
    if (live) {
      const U4 w = philox4x32_10(U4{jlo, jhi, 1u + static_cast<unsigned>(t), 0u}, k0, k1);
      float yv[4];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const float u1 = unit_f32(word(w, 2 * p)), u2 = unit_f32(word(w, 2 * p + 1));
        const float rad = sqrtf(-2.0f * logf(u1));
        float s, c;
        sincospif(2.0f * u2, &s, &c);
        yv[2 * p] = fmaf(0.2f, rad * c, fs[2 * p]);
        yv[2 * p + 1] = fmaf(0.2f, rad * s, fs[2 * p + 1]);
      }
      float* yt = y + static_cast<int64_t>(t) * n;
      if (i0 + 3 < n && (reinterpret_cast<uintptr_t>(yt + i0) & 15) == 0) {
        *reinterpret_cast<float4*>(yt + i0) = make_float4(yv[0], yv[1], yv[2], yv[3]);
      } else {
        for (int r = 0; r < 4; ++r)
          if (i0 + r < n) yt[i0 + r] = yv[r];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (i0 + r < n) m = fmaxf(m, fabsf(yv[r]));
    }
    if (amax) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(amax + t, __float_as_uint(m));
    }
  }
}

}  // namespace

}  // namespace fk

using namespace fk;

extern "C" fk_status fk_generate_sweep_1d(uint64_t seed, int workload, int64_t first, int64_t n, int n_targets,
                                          float* x, float* y, unsigned* y_absmax, void* stream) {
  clear_error();
  if (n < 0 || first < 0 || (first & 3) != 0) return set_error(FK_EINVAL, "first = %lld must be >= 0 and a multiple of 4", (long long)first);
  if (n_targets < 0 || n_targets > 1024) return set_error(FK_EINVAL, "n_targets = %d outside [0, 1024]", n_targets);
  if (n > 0 && (!x || (n_targets > 0 && !y))) return set_error(FK_EINVAL, "null output");
  if (workload < 0) return set_error(FK_EINVAL, "workload < 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FK_TRY(capture_check(st, true, false, "fk_generate_sweep_1d"));
  if (y_absmax && n_targets > 0) FK_CUDA(cudaMemsetAsync(y_absmax, 0, sizeof(unsigned) * n_targets, st));
  if (n == 0) return FK_OK;
  const int64_t quads = (n + 3) / 4;
  const int block = 256;
  const int64_t blocks = (quads + block - 1) / block;
  if (blocks > 0x7fffffffLL) return set_error(FK_EINVAL, "n too large for one call");
  k_gen_sweep<<<static_cast<unsigned>(blocks), block, 0, st>>>(static_cast<unsigned>(seed & 0xFFFFFFFFu),
                                                                static_cast<unsigned>(workload), first, n, n_targets,
                                                                x, y, y_absmax);
  note_launch();
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}
