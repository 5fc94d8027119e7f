// ES kernel weights of one coordinate by a piecewise polynomial (the FP32 spreaders).
//
// Tap a of a window weighs phi((a - f) 2 / w) with f = c + g, c = (w - 1) / 2 and the
// offset g in (-1/2, 1/2] (Sec. 2.3 kernel, window convention of window.cuh).  As a
// function of g each tap is smooth on that interval, so it is replaced by a polynomial
// of degree 7 (w <= 7) or 8 (Chebyshev interpolation, converted to powers of g).  phi is
// even, so tap w - 1 - a is tap a at -g: with h_a(g) = E_a(g^2) + g O_a(g^2), the pair
// costs one Horner chain for each part and two FMAs, and no transcendental function
// (the piecewise-polynomial evaluation of Barnett, Magland and af Klinteberg, 2019).
// Largest error against phi, fp32 evaluation included, for sigma ~ 2: 2.2e-7 at w = 7
// (eps = 1e-6), 6.9e-7 at w = 6 (1e-5), 6.0e-6 at w = 5 (1e-4), 5.5e-5 at w = 4 (1e-3),
// and ~1e-7 (the fp32 rounding floor) for w = 8 .. 16: each below the tolerance that
// chose the width, or at the precision fp32 inputs carry.
#pragma once

namespace fk {

constexpr int ES_POLY_MAXW = 16;

// polynomial degree for width w: 7 up to w = 7 (error 2.2e-7 at w = 7, eps = 1e-6),
// 8 beyond
__host__ __device__ constexpr int es_poly_deg(int w) { return w <= 7 ? 7 : 8; }

struct EsPoly {
  float e[ES_POLY_MAXW / 2][5];  // even part of tap a, coefficients of g^0, g^2, .., g^(2 ne - 2)
  float o[ES_POLY_MAXW / 2][4];  // odd part / g, coefficients of g^0, g^2, .., g^(2 no - 2)
  float2 eo[ES_POLY_MAXW / 2][4];  // (e[a][j], o[a][j]): both Horner chains in one packed FMA per step
};

// E_a(g^2) and O_a(g^2) of tap pair a as (E, O), the two Horner chains advanced together
// by packed FMAs (fma.rn.f32x2): the same operations, in the same order, as two scalar
// chains, so the values are identical
template <int NE, int NO>
__device__ __forceinline__ float2 es_eo(const EsPoly& P, int a, float g2) {
  static_assert(NE == NO || NE == NO + 1, "coefficient counts");
  const float2 g22 = make_float2(g2, g2);
  float2 eo;
  if constexpr (NE == NO) eo = P.eo[a][NO - 1];
  else eo = make_float2(fmaf(P.e[a][NE - 1], g2, P.e[a][NE - 2]), P.o[a][NO - 1]);
#pragma unroll
  for (int j = NO - 2; j >= 0; --j) eo = __ffma2_rn(eo, g22, P.eo[a][j]);
  return eo;
}

// weights of taps 0 .. W - 1 at offset g = f - (W - 1) / 2.  PH: advance the even and
// odd Horner chains of a tap pair together with packed FMAs (same values; which form
// schedules better depends on the caller's register pressure, so callers choose)
template <int W, bool PH = false>
__device__ __forceinline__ void es_taps_poly(float g, const EsPoly& P, float* out) {
  static_assert(W <= ES_POLY_MAXW, "width");
  constexpr int DEG = es_poly_deg(W);
  constexpr int NE = DEG / 2 + 1, NO = (DEG + 1) / 2;  // even and odd coefficient counts
  const float g2 = g * g;
#pragma unroll
  for (int a = 0; a < W / 2; ++a) {
    float E, O;
    if constexpr (PH) {
      const float2 eo = es_eo<NE, NO>(P, a, g2);
      E = eo.x;
      O = eo.y;
    } else {
      E = P.e[a][NE - 1];
#pragma unroll
      for (int j = NE - 2; j >= 0; --j) E = fmaf(E, g2, P.e[a][j]);
      O = P.o[a][NO - 1];
#pragma unroll
      for (int j = NO - 2; j >= 0; --j) O = fmaf(O, g2, P.o[a][j]);
    }
    out[a] = fmaf(g, O, E);
    out[W - 1 - a] = fmaf(-g, O, E);
  }
  if (W & 1) {
    constexpr int a = W / 2;
    float E = P.e[a][NE - 1];
#pragma unroll
    for (int j = NE - 2; j >= 0; --j) E = fmaf(E, g2, P.e[a][j]);
    out[a] = E;
  }
}

// the same weights as mirrored pairs: pr[a] = (tap a, tap W - 1 - a) for a < W / 2 and,
// for odd W, *mid = tap W / 2 (each value computed by the same operations as above)
template <int W>
__device__ __forceinline__ void es_taps_poly_pairs(float g, const EsPoly& P, float2* pr, float* mid) {
  static_assert(W <= ES_POLY_MAXW, "width");
  constexpr int DEG = es_poly_deg(W);
  constexpr int NE = DEG / 2 + 1, NO = (DEG + 1) / 2;
  const float g2 = g * g;
#pragma unroll
  for (int a = 0; a < W / 2; ++a) {
    float E = P.e[a][NE - 1];
#pragma unroll
    for (int j = NE - 2; j >= 0; --j) E = fmaf(E, g2, P.e[a][j]);
    float O = P.o[a][NO - 1];
#pragma unroll
    for (int j = NO - 2; j >= 0; --j) O = fmaf(O, g2, P.o[a][j]);
    pr[a] = make_float2(fmaf(g, O, E), fmaf(-g, O, E));
  }
  if (W & 1) {
    constexpr int a = W / 2;
    float E = P.e[a][NE - 1];
#pragma unroll
    for (int j = NE - 2; j >= 0; --j) E = fmaf(E, g2, P.e[a][j]);
    *mid = E;
  }
}

// coefficients for a plan's width and shape (host, fp64 arithmetic)
EsPoly es_poly(int w, double beta);

}  // namespace fk
