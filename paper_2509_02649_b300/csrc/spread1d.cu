// One-dimensional spreading of many channels with integer (fixed-point) sums in
// shared memory (mixed path, fp32 inputs).
//
// The 1-D fine grids are short (N <= 8192 at the mode counts of §3 sweeps), so a
// CTA can hold whole grids of several channels in shared memory; points are taken
// in input order and every window tap is one shared-memory atomic.  On this part
// 32-bit integer shared atomics are native while fp32 and 64-bit ones are compare-
// and-swap loops, so each contribution psi_a * y is rounded to a fixed-point
// integer q = round(psi_a * y * S) and added to a 64-bit sum split in two: the low
// 32-bit word in shared memory takes an atomic add whose returned old value gives the
// carry, and the high part, in the global int64 accumulator, gets +-2^32 only when the
// low word wraps (rare: the low words start at 2^31).
//
// Scale: per channel S = 2^(21 - e) with max|y| <= 2^e (ones: e = 1), so every
// |q| <= 2^21 and q is formed with one FFMA against the constant 1.5 * 2^23 (the
// product psi_a * (y S) is exact inside the FMA and rounded once to an integer).
// The rounding error of a contribution is at most 2^-22 max|y|; it does not grow
// with the accumulated magnitude, unlike an fp32 running sum.  Integer sums do not
// depend on the order of the additions, so the result is bitwise reproducible.
//
// Layout: channel groups of at most `cmax` channels share a CTA (cmax N 4 bytes of
// shared memory); the CTAs of a group split the points into contiguous ranges; at
// the end each CTA adds its low words into the global int64 accumulator, which a
// last kernel scales back into the fp64 grid.
//
// Lane replicas (small grids, REP): the 32 lanes' windows start at unrelated nodes, so
// one warp's atomics land on ~3.6 words of the same bank on average and the shared-
// memory pipe serialises them.  When 32 copies of the group's grids fit in shared
// memory they are stored node-major with the lane index fastest (word (c, node) of
// lane L at ((c stride + node) 32 + L)): every lane adds into its own copy, which is
// its own bank, so each atomic instruction is one wavefront.  The copies are summed
// (as integers, so the result is the same bit for bit) when the CTA flushes.
#include "fk_internal.cuh"
#include "window.cuh"
#include "es_poly.cuh"
#include "checked.cuh"

namespace fk {

namespace {

constexpr int MAXGRP = 64;                      // channel groups per call
constexpr int CG = 6;                           // channels per CTA at most
constexpr int HALO = 16;                        // padding nodes after each grid (>= max W - 1)
constexpr int THREADS = 1024;
constexpr size_t SMEM_BUDGET = 220 * 1024;      // bytes of integer grids per CTA
constexpr float MAGIC = 12582912.0f;            // 1.5 * 2^23
constexpr int MAGIC_BITS = 0x4B400000;
constexpr unsigned WRAP_MARGIN = 1u << 22;      // > max |q| = 2^21 (+1)

struct Fx1dArgs {
  int64_t n;
  const float* x;
  const float* y;     // [n_y][n]
  int n_y;
  int with_ones;
  int N;
  float c_hi, c_lo;   // N / (2 pi) as a float pair
  EsPoly poly;        // tap polynomials of the plan's width
  int ngrp;
  int grp_c0[MAXGRP];  // first channel of each group (channel 0 = ones when with_ones)
  int grp_nc[MAXGRP];
  int grp_b0[MAXGRP + 1];  // first CTA of each group; grp_b0[ngrp] = total CTAs
  int vec;                 // x and every y row 16-byte aligned (four points per load)
  const unsigned* amax;    // [n_y] bit patterns of max |y_c| (non-negative floats)
  unsigned long long* acc; // [nc][N] int64 accumulators
  unsigned* flags;
};

// hi-word change of one low-word add: qsign + carry out of (old + q), where qsign is
// the sign extension (0 or -1) of q
__device__ __forceinline__ int carry_delta(unsigned old, unsigned q, int qsign) {
  int dh;
  asm("{\n\t.reg .u32 t;\n\tadd.cc.u32 t, %1, %2;\n\taddc.u32 %0, %3, 0;\n\t}" : "=r"(dh) : "r"(old), "r"(q), "r"(qsign));
  return dh;
}

// exponent e with |v| <= 2^e for the channel scale (v = 0 gives e = 0)
__device__ __forceinline__ int scale_exp(float v) {
  int e = 0;
  frexpf(v, &e);
  return e;
}

template <int W, bool REP>
__global__ void __launch_bounds__(THREADS) k_spread1d_fx(Fx1dArgs A) {
  extern __shared__ unsigned smem_fx[];
  const int b = blockIdx.x;
  int g = 0;
  while (g + 1 < A.ngrp && A.grp_b0[g + 1] <= b) ++g;
  const int c0 = A.grp_c0[g], nc = A.grp_nc[g];
  const int nblk = A.grp_b0[g + 1] - A.grp_b0[g];
  const int lb = b - A.grp_b0[g];
  const int N = A.N;
  // [nc][N + HALO] low words: a window starting at node b < N ends before N + HALO,
  // and the halo is added into nodes 0 .. HALO - 1 at the end.  The high words live in
  // the global int64 accumulator: a wrap of a low word adds +-2^32 there directly.
  // The low words start at 2^31 (the sums at that bias), so a signed sum hovering
  // around zero never wraps and the carry branch stays cold.
  const int stride = N + HALO;
  // REP: word (c, node) of lane L at ((c stride + node) << 5) | L (lane L's own bank)
  const int lane = threadIdx.x & 31;
  unsigned* lo = smem_fx + (REP ? lane : 0);
  constexpr int SH = REP ? 5 : 0;
  const int words = (nc * stride) << SH;
  for (int i = threadIdx.x; i < words; i += blockDim.x) smem_fx[i] = 0x80000000u;

  // per-channel scales
  float S[CG];
#pragma unroll
  for (int c = 0; c < CG; ++c) {
    S[c] = 0.f;
    if (c < nc) {
      const int ch = c0 + c;
      const float m = (A.with_ones && ch == 0) ? 1.0f : __uint_as_float(A.amax[ch - A.with_ones]);
      S[c] = ldexpf(1.0f, 21 - scale_exp(m));
    }
  }
  __syncthreads();

  // one point: window, W weights, then per channel W low-word adds in flight before
  // the (rare) carries are settled
  auto one = [&](float xv, const float* yv) {
    int l0;
    float f;
    if (!window_f32(xv, N, A.c_hi, A.c_lo, W, &l0, &f)) {
      atomicOr(A.flags, FLAG_RANGE);
      return;
    }
    float psi[W];
    es_taps_poly<W>(f - 0.5f * static_cast<float>(W - 1), A.poly, psi);
    const int b = wrap_node(l0, N);
    if (!fk_check(b >= 0 && b < N, A.flags)) return;
#pragma unroll
    for (int c = 0; c < CG; ++c) {
      if (c >= nc) break;
      const float v = yv[c] * S[c];
      unsigned* lc = lo + ((c * stride + b) << SH);
      unsigned old[W];
      int qv[W];
#pragma unroll
      for (int a = 0; a < W; ++a) {
        qv[a] = __float_as_int(fmaf(psi[a], v, MAGIC)) - MAGIC_BITS;
        old[a] = atomicAdd(lc + (a << SH), static_cast<unsigned>(qv[a]));
      }
      // a low word can wrap only if it was within |q| <= 2^21 (+1 for a tap rounding
      // above 1) of 0 mod 2^32 before the add: one unsigned min over the taps screens
      // for that, and the exact high-word changes (sign extension of q plus the carry
      // out of the add) are taken only then (rare: the words start at 2^31)
      unsigned near = 0xFFFFFFFFu;
#pragma unroll
      for (int a = 0; a < W; ++a) near = min(near, old[a] + WRAP_MARGIN);
      if (near < 2u * WRAP_MARGIN) {
        unsigned long long* hc = A.acc + static_cast<int64_t>(c0 + c) * N;
#pragma unroll
        for (int a = 0; a < W; ++a) {
          const int dh = carry_delta(old[a], static_cast<unsigned>(qv[a]), qv[a] >> 31);
          if (dh) atomicAdd(hc + ((b + a) & (N - 1)), static_cast<unsigned long long>(static_cast<long long>(dh) << 32));
        }
      }
    }
  };
  // strength of channel c at point i (ones channel: 1)
  const float* yrow[CG];
#pragma unroll
  for (int c = 0; c < CG; ++c) {
    const int ch = c0 + c;
    yrow[c] = (c < nc && !(A.with_ones && ch == 0)) ? A.y + static_cast<int64_t>(ch - A.with_ones) * A.n : nullptr;
  }

  const int64_t per = ((A.n + nblk - 1) / nblk + 3) & ~static_cast<int64_t>(3);
  const int64_t s0 = static_cast<int64_t>(lb) * per;
  const int64_t s1 = min(A.n, s0 + per);
  if (A.vec) {
    // four consecutive points per thread: one 16-byte load per array, all issued
    // before the first point is processed
    for (int64_t i = s0 + 4 * static_cast<int64_t>(threadIdx.x); i < s1; i += 4 * static_cast<int64_t>(blockDim.x)) {
      if (i + 3 < s1) {
        const float4 xq = __ldg(reinterpret_cast<const float4*>(A.x + i));
        float4 yq[CG];
#pragma unroll
        for (int c = 0; c < CG; ++c)
          yq[c] = yrow[c] ? __ldg(reinterpret_cast<const float4*>(yrow[c] + i)) : make_float4(1.f, 1.f, 1.f, 1.f);
        float yv[CG];
#pragma unroll
        for (int c = 0; c < CG; ++c) yv[c] = yq[c].x;
        one(xq.x, yv);
#pragma unroll
        for (int c = 0; c < CG; ++c) yv[c] = yq[c].y;
        one(xq.y, yv);
#pragma unroll
        for (int c = 0; c < CG; ++c) yv[c] = yq[c].z;
        one(xq.z, yv);
#pragma unroll
        for (int c = 0; c < CG; ++c) yv[c] = yq[c].w;
        one(xq.w, yv);
      } else {
        for (int64_t j2 = i; j2 < s1; ++j2) {
          float yv[CG];
#pragma unroll
          for (int c = 0; c < CG; ++c) yv[c] = yrow[c] ? yrow[c][j2] : 1.0f;
          one(A.x[j2], yv);
        }
      }
    }
  } else {
    for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
      float yv[CG];
#pragma unroll
      for (int c = 0; c < CG; ++c) yv[c] = yrow[c] ? yrow[c][i] : 1.0f;
      one(A.x[i], yv);
    }
  }
  __syncthreads();
  // add the CTA's integer grids (halo folded onto nodes 0 .. HALO - 1) into the
  // global accumulators
  for (int t = threadIdx.x; t < nc * stride; t += blockDim.x) {
    long long v;
    if constexpr (REP) {
      // the 32 lane copies of word t, read from bank (r + lane) at step r: conflict free
      const unsigned* row = smem_fx + (t << 5);
      v = 0;
#pragma unroll 8
      for (int r = 0; r < 32; ++r) v += static_cast<long long>(row[(r + lane) & 31]) - 0x80000000LL;
    } else {
      v = static_cast<long long>(lo[t]) - 0x80000000LL;
    }
    if (v != 0) {
      const int c = t / stride, node = (t - c * stride) & (N - 1);
      atomicAdd(A.acc + static_cast<int64_t>(c0 + c) * N + node, static_cast<unsigned long long>(v));
    }
  }
}

// max |y_c| per channel as float bit patterns (non-negative floats order like their bits)
__global__ void k_absmax(int64_t n, const float* __restrict__ y, int n_y, unsigned* amax) {
  const int c = blockIdx.y;
  const float* yc = y + static_cast<int64_t>(c) * n;
  float m = 0.f;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float a = fabsf(yc[i]);
    m = (a > m) ? a : m;  // NaN inputs are left out
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(amax + c, __float_as_uint(m));
}

// grid[c][node] (+)= acc[c][node] / S_c
__global__ void k_fx_to_grid(int64_t total, int N, int with_ones, const unsigned* amax,
                             const unsigned long long* acc, double* grid, int accumulate) {
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int ch = static_cast<int>(t / N);
    const float m = (with_ones && ch == 0) ? 1.0f : __uint_as_float(amax[ch - with_ones]);
    const double inv = ldexp(1.0, scale_exp(m) - 21);
    const double v = static_cast<double>(static_cast<long long>(acc[t])) * inv;
    grid[t] = accumulate ? grid[t] + v : v;
  }
}

using FxFn = void (*)(Fx1dArgs);

template <int W>
FxFn fx_fn(bool rep) {
  return rep ? k_spread1d_fx<W, true> : k_spread1d_fx<W, false>;
}

FxFn pick_fx(int w, bool rep) {
  switch (w) {
    case 2: return fx_fn<2>(rep);
    case 3: return fx_fn<3>(rep);
    case 4: return fx_fn<4>(rep);
    case 5: return fx_fn<5>(rep);
    case 6: return fx_fn<6>(rep);
    case 7: return fx_fn<7>(rep);
    case 8: return fx_fn<8>(rep);
    case 9: return fx_fn<9>(rep);
    case 10: return fx_fn<10>(rep);
    case 11: return fx_fn<11>(rep);
    case 12: return fx_fn<12>(rep);
    case 13: return fx_fn<13>(rep);
    case 14: return fx_fn<14>(rep);
    case 15: return fx_fn<15>(rep);
    case 16: return fx_fn<16>(rep);
    default: return nullptr;
  }
}

}  // namespace

fk_status absmax_channels(int64_t n, const float* y, int n_y, unsigned* amax, cudaStream_t st) {
  if (n_y < 1) return FK_OK;
  if (n_y > 65535) return set_error(FK_EINVAL, "absmax: %d channels", n_y);
  FK_CUDA(cudaMemsetAsync(amax, 0, sizeof(unsigned) * n_y, st));
  if (n == 0) return FK_OK;
  k_absmax<<<dim3(grid_for(n, 256, 148 * 8), n_y), 256, 0, st>>>(n, y, n_y, amax); note_launch();
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}

bool spread1d_fixed_supported(const EsPlan& p, int n_y, bool with_ones) {
  const int nc = n_y + (with_ones ? 1 : 0);
  if (p.d != 1 || nc < 1 || p.w < 2 || p.w > 16) return false;
  const int64_t cmax = static_cast<int64_t>(SMEM_BUDGET / (4 * static_cast<size_t>(p.N + HALO)));
  if (cmax < 1) return false;
  const int64_t c = std::min<int64_t>(cmax, CG);
  return (nc + c - 1) / c <= MAXGRP;
}

namespace {

// channels per CTA at most for this grid size (shared-memory budget and CG); rep: with
// 32 lane copies of each grid
int channel_cap(int N, bool rep = false) {
  const size_t per = 4 * static_cast<size_t>(N + HALO) * (rep ? 32 : 1);
  return static_cast<int>(std::min<size_t>(CG, SMEM_BUDGET / per));
}

// shape of a launch: channels per CTA (0: default) and lane copies; the autotuner's
// table holds it as one int, channels + 1000 with lane copies
struct Fx1dShape {
  int cmax;
  bool rep;
};
inline int shape_code(Fx1dShape s) { return s.cmax + (s.rep ? 1000 : 0); }
inline Fx1dShape shape_of(int v) { return Fx1dShape{v % 1000, v >= 1000}; }

fk_status spread1d_run(const EsPlan& p, int64_t n, const float* x, const float* y, int n_y, bool with_ones,
                       const unsigned* y_absmax, double* grid, bool accumulate, unsigned* flags, cudaStream_t st,
                       Scratch& scr, Fx1dShape shape) {
  const int nc = n_y + (with_ones ? 1 : 0);
  const int N = p.N;
  if (!accumulate) FK_CUDA(cudaMemsetAsync(grid, 0, sizeof(double) * N * nc, st));
  if (n == 0) return FK_OK;

  // default (cmax 0): with lane copies (where 32 copies of one channel fit: small
  // grids), as many channels per CTA as fit; without, half the shared-memory cap, so
  // that two 1024-thread CTAs share an SM (the fastest measured shape at N = 8192, 17
  // channels)
  const int cmax_req = shape.cmax;
  const int rcap = channel_cap(N, true);
  const bool rep = shape.rep && rcap >= 1 && (nc + rcap - 1) / rcap <= MAXGRP;
  int cmax = channel_cap(N, rep);
  if (cmax_req > 0 && cmax_req < cmax) cmax = cmax_req;
  else if (cmax_req <= 0 && !rep) cmax = (cmax + 1) / 2;
  if ((nc + cmax - 1) / cmax > MAXGRP) cmax = (nc + MAXGRP - 1) / MAXGRP;
  const int ngrp = (nc + cmax - 1) / cmax;
  Fx1dArgs A{};
  A.n = n;
  A.x = x;
  A.y = y;
  A.n_y = n_y;
  A.with_ones = with_ones ? 1 : 0;
  A.N = N;
  const CoordConst cc = coord_const(N);
  A.c_hi = cc.hi;
  A.c_lo = cc.lo;
  A.poly = es_poly(p.w, p.beta);
  A.ngrp = ngrp;
  A.flags = flags;
  A.vec = ((reinterpret_cast<uintptr_t>(x) & 15) == 0 && (n & 3) == 0 &&
           (n_y == 0 || (reinterpret_cast<uintptr_t>(y) & 15) == 0)) ? 1 : 0;
  // balanced groups: sizes differ by at most one channel
  int c = 0;
  size_t smem_max = 0;
  for (int g = 0; g < ngrp; ++g) {
    const int sz = nc / ngrp + (g < nc % ngrp ? 1 : 0);
    A.grp_c0[g] = c;
    A.grp_nc[g] = sz;
    c += sz;
    smem_max = std::max(smem_max, sizeof(unsigned) * static_cast<size_t>(sz) * (N + HALO) * (rep ? 32 : 1));
  }
  // CTAs: as many as fit on the device at once, shared out by channel count, and no
  // more than one per 4096 points, 32768 with lane copies (each CTA zeroes and flushes
  // whole grids)
  const int sms = std::max(1, sm_count());
  const int per_sm = std::max(1, std::min<int>(2, static_cast<int>((228 * 1024) / (smem_max + 1024))));
  const int64_t total_ctas = static_cast<int64_t>(sms) * per_sm;
  const int64_t per_cta = rep ? 32768 : 4096;  // lane copies: 32 times the grid words to zero and flush
  const int64_t by_n = std::max<int64_t>(1, (n + per_cta - 1) / per_cta);
  A.grp_b0[0] = 0;
  for (int g = 0; g < ngrp; ++g) {
    int64_t k = (total_ctas * A.grp_nc[g] + nc - 1) / nc;
    k = std::max<int64_t>(1, std::min(k, by_n));
    A.grp_b0[g + 1] = A.grp_b0[g] + static_cast<int>(k);
  }
  const int nblocks = A.grp_b0[ngrp];

  unsigned* amax = nullptr;
  if (n_y > 0) {
    if (y_absmax) {
      amax = const_cast<unsigned*>(y_absmax);
    } else {
      FK_TRY(scr.alloc(&amax, static_cast<size_t>(n_y)));
      FK_TRY(absmax_channels(n, y, n_y, amax, st));
    }
  }
  A.amax = amax;
  FK_TRY(scr.alloc(&A.acc, static_cast<size_t>(nc) * N));
  FK_CUDA(cudaMemsetAsync(A.acc, 0, sizeof(unsigned long long) * nc * N, st));

  const FxFn fn = pick_fx(p.w, rep);
  if (!fn) return set_error(FK_EINVAL, "1-D fixed-point spreading: w = %d not built", p.w);
  FK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem_max)));
  KernelTimer* kt = kernel_timer();
  if (kt->on) cudaEventRecordWithFlags(kt->start, st, kt->rec_flags);
  fn<<<nblocks, THREADS, smem_max, st>>>(A); note_launch();
  if (kt->on) {
    cudaEventRecordWithFlags(kt->stop, st, kt->rec_flags);
    kt->recorded = true;
  }
  FK_CUDA(cudaGetLastError());
  const int64_t total = static_cast<int64_t>(nc) * N;
  k_fx_to_grid<<<grid_for(total, 256), 256, 0, st>>>(total, N, A.with_ones, amax, A.acc, grid, accumulate ? 1 : 0);
  note_launch();
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}

}  // namespace

fk_status spread1d_fixed(const EsPlan& p, int64_t n, const float* x, const float* y, int n_y, bool with_ones,
                         const unsigned* y_absmax, double* grid, bool accumulate, unsigned* flags, cudaStream_t st,
                         Scratch& scr, bool autotune, bool lane_copies) {
  if (!spread1d_fixed_supported(p, n_y, with_ones))
    return set_error(FK_EINVAL, "1-D fixed-point spreading: unsupported shape (N = %d, w = %d)", p.N, p.w);
  const int nc = n_y + (with_ones ? 1 : 0);
  int lg = 0;
  while ((static_cast<int64_t>(1) << (lg + 1)) <= n) ++lg;
  // without lane copies: the default shape without them (not tuned)
  if (!lane_copies)
    return spread1d_run(p, n, x, y, n_y, with_ones, y_absmax, grid, accumulate, flags, st, scr, Fx1dShape{0, false});
  const TuneKey key{TUNE_SPREAD1D, p.N, p.w, nc, lg};
  int cm = 0;
  if (tune_lookup_int(key, &cm) || !autotune || n < (1 << 20))
    return spread1d_run(p, n, x, y, n_y, with_ones, y_absmax, grid, accumulate, flags, st, scr,
                        cm > 0 ? shape_of(cm) : Fx1dShape{0, true});
  // trials write a scratch grid when the call adds into the caller's grid
  double* tgrid = grid;
  if (accumulate) FK_TRY(scr.alloc(&tgrid, static_cast<size_t>(p.N) * nc));
  // channels per CTA: more channels share each point's weights, fewer let more CTAs
  // reside per SM; with or without lane copies where they fit; time each on this
  // call's data (the grid is rewritten each time)
  const int cap = channel_cap(p.N), rcap = channel_cap(p.N, true);
  std::vector<int> opts;
  for (int c = rcap; c >= 1 && opts.size() < 3; --c) opts.push_back(shape_code(Fx1dShape{c, true}));
  for (int c = cap; c >= 1 && opts.size() < 8; --c) opts.push_back(shape_code(Fx1dShape{c, false}));
  cudaEvent_t e0, e1;
  FK_CUDA(cudaEventCreate(&e0));
  FK_CUDA(cudaEventCreate(&e1));
  int best = opts[0];
  float best_ms = 1e30f;
  std::string log;
  fk_status rc = FK_OK;
  for (size_t i = 0; i <= opts.size() && rc == FK_OK; ++i) {
    const int c = opts[i == 0 ? 0 : i - 1];  // the first option twice: warm-up, then timed
    cudaEventRecord(e0, st);
    {
      Scratch inner(st);
      rc = spread1d_run(p, n, x, y, n_y, with_ones, y_absmax, tgrid, false, flags, st, inner, shape_of(c));
    }
    cudaEventRecord(e1, st);
    if (rc != FK_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (i == 0) continue;
    char line[64];
    snprintf(line, sizeof(line), "%schannels/CTA=%d%s %.3f ms", log.empty() ? "" : "; ", c % 1000,
             c >= 1000 ? " lane copies" : "", ms);
    log += line;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  FK_TRY(rc);
  char line[64];
  snprintf(line, sizeof(line), "  ->  channels/CTA=%d%s (%.3f ms)", best % 1000, best >= 1000 ? " lane copies" : "",
           best_ms);
  tune_store_int(key, best, log + line);
  return spread1d_run(p, n, x, y, n_y, with_ones, y_absmax, grid, accumulate, flags, st, scr, shape_of(best));
}

}  // namespace fk
