// Window of a point on the upsampled grid (Sec. 2.3: ES kernel of width W on N nodes
// with spacing h = 2 pi / N, node l at -pi + l h).
//
// u = x N / (2 pi) + N / 2 is the point's position in grid units; its window is the
// W nodes l0 .. l0 + W - 1 with l0 = ceil(u - W/2), and node l0 + a gets the weight
// psi((a - f) 2 / W) with f = u - l0 in (W/2 - 1, W/2].
//
// No folding of x: for x in [-3 pi, 3 pi) the position u lies in [-N, 2N) and the
// periodicity is applied to node indices, (l0 + a + 2N) mod N, which is exact.
//
// fp32: the product x N / (2 pi) is carried as an unevaluated sum (the constant as a
// float pair, the product's rounding error recovered with an FMA), so f is accurate
// to a few ulps of f itself; u as one fp32 number would carry an error of up to
// ulp(N) / 2, i.e. a phase error of pi |k| ulp(N) / N at mode k.
#pragma once

namespace fk {

// false when x is outside [-3 pi, 3 pi) or NaN
__device__ __forceinline__ bool window_f32(float x, int N, float c_hi, float c_lo, int W, int* l0, float* f) {
  const float lim = 9.42477796076938f;  // 3 pi rounded down
  if (!(x >= -lim && x < lim)) return false;
  // explicitly rounded operations (never contracted into FMAs), so that every kernel
  // computes the same window for the same x: partitions count points in one kernel and
  // place them in another
  const float p = __fmul_rn(x, c_hi);
  const float t = fmaf(x, c_lo, fmaf(x, c_hi, -p));  // x c_lo + (x c_hi - p)
  const float hN = 0.5f * static_cast<float>(N);
  const float hW = 0.5f * static_cast<float>(W);
  float l = ceilf(__fsub_rn(__fadd_rn(__fadd_rn(hN, p), t), hW));
  float fr = __fadd_rn(__fadd_rn(__fsub_rn(hN, l), p), t);
  if (fr > hW) {
    l = __fadd_rn(l, 1.0f);
    fr = __fsub_rn(fr, 1.0f);
  } else if (fr <= hW - 1.0f) {
    l = __fsub_rn(l, 1.0f);
    fr = __fadd_rn(fr, 1.0f);
  }
  *l0 = static_cast<int>(l);
  *f = fr;
  return true;
}

__device__ __forceinline__ bool window_f64(double x, int N, int W, int* l0, double* f) {
  if (!(x >= -3.0 * M_PI && x < 3.0 * M_PI)) return false;
  const double u = fma(x, N / (2.0 * M_PI), 0.5 * N);
  const double l = ceil(u - 0.5 * W);
  *l0 = static_cast<int>(l);
  *f = u - l;
  return true;
}

// float pair for N / (2 pi)
struct CoordConst {
  float hi, lo;
};
inline CoordConst coord_const(int N) {
  const double c = N / (2.0 * M_PI);
  CoordConst r;
  r.hi = static_cast<float>(c);
  r.lo = static_cast<float>(c - static_cast<double>(r.hi));
  return r;
}

__host__ __device__ __forceinline__ int wrap_node(int l, int N) { return (l + 2 * N) & (N - 1); }

}  // namespace fk
