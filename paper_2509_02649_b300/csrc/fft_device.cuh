// Shared-memory FFT device helpers (power-of-two lengths, radix-2 decimation in time).
#pragma once

#include "fk_internal.cuh"

namespace fk {

__device__ __forceinline__ unsigned bitrev(unsigned v, int bits) { return __brev(v) >> (32 - bits); }

template <typename R>
__device__ __forceinline__ cplx<R> tw_get(const double* tw, int idx, int sign) {
  // e^{sign * 2 pi i idx / N}; the table holds e^{-2 pi i t / N}
  cplx<R> r;
  r.x = static_cast<R>(__ldg(tw + 2 * idx));
  const R im = static_cast<R>(__ldg(tw + 2 * idx + 1));
  r.y = sign < 0 ? im : -im;
  return r;
}

// In-place radix-2 DIT over s[0..N) (already in bit-reversed order).  The first two
// stages have the twiddles 1 and e^{sign i pi/2} = sign i: no multiplications.
template <typename R>
__device__ void fft_smem(cplx<R>* s, int N, int sign, const double* tw) {
  if (N >= 4) {
    // stages len = 2 and 4 together: each thread a group of four
    for (int g = threadIdx.x; g < (N >> 2); g += blockDim.x) {
      cplx<R>* q = s + 4 * g;
      const cplx<R> a0 = q[0], a1 = q[1], a2 = q[2], a3 = q[3];
      const cplx<R> b0{a0.x + a1.x, a0.y + a1.y}, b1{a0.x - a1.x, a0.y - a1.y};
      const cplx<R> b2{a2.x + a3.x, a2.y + a3.y}, b3{a2.x - a3.x, a2.y - a3.y};
      // b3 times sign i
      const cplx<R> t3{sign < 0 ? b3.y : -b3.y, sign < 0 ? -b3.x : b3.x};
      q[0] = cplx<R>{b0.x + b2.x, b0.y + b2.y};
      q[2] = cplx<R>{b0.x - b2.x, b0.y - b2.y};
      q[1] = cplx<R>{b1.x + t3.x, b1.y + t3.y};
      q[3] = cplx<R>{b1.x - t3.x, b1.y - t3.y};
    }
    __syncthreads();
  }
  for (int len = (N >= 4 ? 8 : 2); len <= N; len <<= 1) {
    const int half = len >> 1;
    const int tstep = N / len;
    for (int b = threadIdx.x; b < (N >> 1); b += blockDim.x) {
      const int grp = b / half;
      const int k = b - grp * half;
      const int i0 = grp * len + k;
      const int i1 = i0 + half;
      const cplx<R> w = tw_get<R>(tw, k * tstep, sign);
      const cplx<R> a = s[i0];
      const cplx<R> v = s[i1];
      cplx<R> bw;
      bw.x = v.x * w.x - v.y * w.y;
      bw.y = v.x * w.y + v.y * w.x;
      s[i0].x = a.x + bw.x;
      s[i0].y = a.y + bw.y;
      s[i1].x = a.x - bw.x;
      s[i1].y = a.y - bw.y;
    }
    __syncthreads();
  }
}

// In-place bit-reversal permutation of s[0..N) (natural <-> bit-reversed order).
template <typename R>
__device__ void bitrev_permute(cplx<R>* s, int N, int logN) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int j = static_cast<int>(bitrev(static_cast<unsigned>(i), logN));
    if (i < j) {
      const cplx<R> t = s[i];
      s[i] = s[j];
      s[j] = t;
    }
  }
  __syncthreads();
}

}  // namespace fk
