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

template <typename R>
__device__ __forceinline__ cplx<R> cmul_tw(const cplx<R>& w, const cplx<R>& v) {
  cplx<R> r;
  r.x = v.x * w.x - v.y * w.y;
  r.y = v.x * w.y + v.y * w.x;
  return r;
}

// In-place decimation-in-time FFT over s[0..N) (already in bit-reversed order), radix
// 4 with one radix-2 stage last when log2 N is odd.  With bit-reversed input, the
// four consecutive size-q blocks that a radix-4 stage combines hold the DFTs of the
// subsequences of index residue 0, 2, 1, 3 (mod 4) of the size-4q subsequence being
// formed; output m of the size-4q DFT at k + m q is
//   sum_r (sign i)^(r m) w^(r k) D_r[k],  w = e^{sign 2 pi i / (4q)}.
// The first stage (q = 1) has the twiddles 1: no multiplications.
template <typename R>
__device__ void fft_smem(cplx<R>* s, int N, int sign, const double* tw) {
  // (x + i y) times sign i
  auto rot = [sign](const cplx<R>& v) {
    cplx<R> r;
    r.x = sign < 0 ? v.y : -v.y;
    r.y = sign < 0 ? -v.x : v.x;
    return r;
  };
  int q = 1;
  if (N >= 4) {
    for (int g = threadIdx.x; g < (N >> 2); g += blockDim.x) {
      cplx<R>* p = s + 4 * g;
      const cplx<R> a0 = p[0], a1 = p[1], a2 = p[2], a3 = p[3];
      const cplx<R> b0{a0.x + a1.x, a0.y + a1.y}, b1{a0.x - a1.x, a0.y - a1.y};
      const cplx<R> b2{a2.x + a3.x, a2.y + a3.y};
      const cplx<R> t3 = rot(cplx<R>{a2.x - a3.x, a2.y - a3.y});
      p[0] = cplx<R>{b0.x + b2.x, b0.y + b2.y};
      p[2] = cplx<R>{b0.x - b2.x, b0.y - b2.y};
      p[1] = cplx<R>{b1.x + t3.x, b1.y + t3.y};
      p[3] = cplx<R>{b1.x - t3.x, b1.y - t3.y};
    }
    __syncthreads();
    q = 4;
  }
  for (; 4 * q <= N; q *= 4) {
    const int tstep = N / (4 * q);
    for (int b = threadIdx.x; b < (N >> 2); b += blockDim.x) {
      const int grp = b / q;
      const int k = b - grp * q;
      cplx<R>* p = s + grp * 4 * q + k;
      const cplx<R> t0 = p[0];
      const cplx<R> t2 = cmul_tw(tw_get<R>(tw, 2 * k * tstep, sign), p[q]);      // residue 2
      const cplx<R> t1 = cmul_tw(tw_get<R>(tw, k * tstep, sign), p[2 * q]);      // residue 1
      const cplx<R> t3 = cmul_tw(tw_get<R>(tw, 3 * k * tstep, sign), p[3 * q]);  // residue 3
      const cplx<R> a{t0.x + t2.x, t0.y + t2.y}, bb{t0.x - t2.x, t0.y - t2.y};
      const cplx<R> c{t1.x + t3.x, t1.y + t3.y};
      const cplx<R> d = rot(cplx<R>{t1.x - t3.x, t1.y - t3.y});
      p[0] = cplx<R>{a.x + c.x, a.y + c.y};
      p[q] = cplx<R>{bb.x + d.x, bb.y + d.y};
      p[2 * q] = cplx<R>{a.x - c.x, a.y - c.y};
      p[3 * q] = cplx<R>{bb.x - d.x, bb.y - d.y};
    }
    __syncthreads();
  }
  if (q < N) {  // 2 q == N: the even- and odd-index halves
    for (int k = threadIdx.x; k < q; k += blockDim.x) {
      const cplx<R> a = s[k];
      const cplx<R> v = cmul_tw(tw_get<R>(tw, k, sign), s[k + q]);
      s[k] = cplx<R>{a.x + v.x, a.y + v.y};
      s[k + q] = cplx<R>{a.x - v.x, a.y - v.y};
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
