// ES kernel weights of one coordinate by a piecewise polynomial (the FP32 spreaders).
//
// Tap a of a window weighs phi((a - f) 2 / w) with f = c + g, c = (w - 1) / 2 and the
// offset g in (-1/2, 1/2] (Sec. 2.3 kernel, window convention of window.cuh).  As a
// function of g each tap is smooth on that interval, so it is replaced by a degree-8
// polynomial (Chebyshev interpolation at 9 nodes, converted to powers of g).  phi is
// even, so tap w - 1 - a is tap a at -g: with h_a(g) = E_a(g^2) + g O_a(g^2), the pair
// costs one Horner chain for each part and two FMAs, and no transcendental function
// (the piecewise-polynomial evaluation of Barnett, Magland and af Klinteberg, 2019).
// Largest error against phi, fp32 evaluation included, for sigma in [1.9, 2.5]:
// 1.1e-7 at w = 7 (eps = 1e-6), 7.6e-7 at w = 6 (1e-5), 6e-5 at w = 4 (1e-3), 5e-4
// at w = 3 (1e-2), and ~1e-7 (the fp32 rounding floor) for w = 8 .. 16: each below
// the tolerance that chose the width, or at the precision fp32 inputs carry.
#pragma once

namespace fk {

constexpr int ES_POLY_MAXW = 16;
constexpr int ES_POLY_DEG = 8;

struct EsPoly {
  float e[ES_POLY_MAXW / 2][5];  // even part of tap a, coefficients of g^0, g^2, .., g^8
  float o[ES_POLY_MAXW / 2][4];  // odd part / g, coefficients of g^0, g^2, g^4, g^6
};

// weights of taps 0 .. W - 1 at offset g = f - (W - 1) / 2
template <int W>
__device__ __forceinline__ void es_taps_poly(float g, const EsPoly& P, float* out) {
  static_assert(W <= ES_POLY_MAXW, "width");
  const float g2 = g * g;
#pragma unroll
  for (int a = 0; a < W / 2; ++a) {
    float E = fmaf(P.e[a][4], g2, P.e[a][3]);
    E = fmaf(E, g2, P.e[a][2]);
    E = fmaf(E, g2, P.e[a][1]);
    E = fmaf(E, g2, P.e[a][0]);
    float O = fmaf(P.o[a][3], g2, P.o[a][2]);
    O = fmaf(O, g2, P.o[a][1]);
    O = fmaf(O, g2, P.o[a][0]);
    out[a] = fmaf(g, O, E);
    out[W - 1 - a] = fmaf(-g, O, E);
  }
  if (W & 1) {
    constexpr int a = W / 2;
    float E = fmaf(P.e[a][4], g2, P.e[a][3]);
    E = fmaf(E, g2, P.e[a][2]);
    E = fmaf(E, g2, P.e[a][1]);
    out[a] = fmaf(E, g2, P.e[a][0]);
  }
}

// coefficients for a plan's width and shape (host, fp64 arithmetic)
EsPoly es_poly(int w, double beta);

}  // namespace fk
