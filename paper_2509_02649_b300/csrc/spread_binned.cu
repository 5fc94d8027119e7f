// Binned spreading with register accumulation (mixed path, fp32 arithmetic, d = 2).
//
// The type-1 sums of Sec. 2.3 are spread onto the upsampled grid.  A point's window
// starts at node l0 = ceil(u - w/2) in each dimension; points sharing that start
// node (a "cell") touch exactly the same w x w nodes.  Lanes of the accumulation
// kernel own cells and keep the cell's w x w partial sums in registers for the
// whole call, so its hot loop is FFMA work on register operands: no atomics and no
// shared-memory read-modify-write.  With the ones channel (moments T) and one
// strength channel (right-hand side b) two lanes share a cell, one per channel;
// each lane evaluates the ES weights of one coordinate and the pair swaps them
// with one shuffle, so every weight is computed once.
//
// Owner o holds cells [o cpc, (o+1) cpc), cpc <= 448 (224 in pair mode, so that each
// lane keeps its w x w window in registers without spilling).
//   k_bin_scatter1 (one block per SM, one pass) recomputes each point's cell and
//                 fractional offsets, sorts a tile by owner in shared memory, reserves
//                 room in the owner buckets (fixed capacity: mean load + 2 % + 4096)
//                 with one global atomic per (tile, owner) and writes the tile's runs
//                 as contiguous records: 8 bytes (local cell and fixed-point window
//                 offsets), with the strengths in a parallel stream of floats;
//   k_bin_accumulate (one CTA per owner) streams its owner's bucket with double-
//                 buffered TMA bulk copies and links each round's records into per-cell
//                 lists in shared memory.  A record whose rank in its cell reaches the
//                 round's quota (the mean load plus a fraction of a standard deviation)
//                 moves to the next round's buffer instead, which keeps the warps' trip
//                 counts even.  A lane adds its register window into the fp64 grid
//                 every 2048 points, every 256 in a crowded round, and at the end.
// A bucket that would overflow (crowded points) sets a device flag; the exact
// partition (k_bin_count, k_bin_scan, k_bin_scatter2 or k_bin_scatter, then
// k_bin_accumulate on its 16-byte records) is always enqueued after and runs only when
// that flag is set, so there is no host round trip.
#include "fk_internal.cuh"
#include "window.cuh"
#include "es_poly.cuh"
#include "checked.cuh"

#include <type_traits>

namespace fk {

namespace {

constexpr int MAX_G = 511;  // owners (< partition block size, for the block-wide scans)
constexpr long long WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz
constexpr int THREADS_ACC = 448;                 // accumulation CTA size (one CTA per SM)

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------- async copies
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// returns false when the bounded wait gives up
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned* flags) {
  const long long t0 = clock64();
  while (true) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicOr(flags, FLAG_TIMEOUT);
      return false;
    }
  }
}
// After a wait gave up (the flag is set): wait once more, with the same bound, for the
// bulk copy that the phase still expects, so that the CTA does not exit while a copy
// into its shared memory is in flight.  Each kernel here has at most one copy in
// flight when it waits (the next one is issued after the wait succeeds), so this is
// the last wait before the CTA returns; its result is ignored.
__device__ __forceinline__ void mbar_drain(uint64_t* bar, unsigned parity) {
  const long long t0 = clock64();
  while (true) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done || clock64() - t0 > WAIT_CYCLES) return;
  }
}
// global -> shared bulk copy (TMA), completion counted in bytes on `bar`
__device__ __forceinline__ void bulk_g2s(void* sdst, const void* gsrc, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(sdst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

constexpr int P_THREADS = 1024;  // count kernel
constexpr int P_NWARPS = P_THREADS / 32;
constexpr int P_TILE = 4096;     // points per partition block, at least
constexpr int FLUSH_PTS = 2048;  // points per fp32 register run before an fp64 flush
// a lane whose round holds more than CROWD_RUN records (a crowded cell: the mean load
// per round is 16-45) flushes after every CROWD_RUN of them, since a crowded cell's
// points are often near-equal and their fp32 rounding errors then add up in one sign
// (a run of L equal terms is off by up to L 2^-25 of its sum)
constexpr int CROWD_RUN = 256;
constexpr long long NO_ROOM = -(1ll << 62);  // one-pass partition: the owner's bucket is full

// cells per owner: one lane per cell, or two (one per channel) in pair mode, whose
// CTAs have 16 warps (four per scheduler)
template <bool PAIR>
struct Cfg {
  static constexpr int THREADS = PAIR ? 512 : THREADS_ACC;
  static constexpr int CELLS = PAIR ? 256 : THREADS_ACC;
};

// Cells of owner o: nb "big" owners of cb cells, then owners of cs cells.  Two sizes
// let a grid of ~two waves give each wave whole multiples of four warps per SM (16
// then 12 in pair mode), so that no scheduler of an SM carries more warps than another.
struct OwnerMap {
  int nb, cb, cs;
  // ceil(2^32 / cells): k / cells = (k m) >> 32 exactly for k < 2^18 and cells <= 2^9
  // (the error k (m - 2^32 / cells) / 2^32 < 2^-14 stays below the gap 1 / cells)
  unsigned long long mb, ms;
  __host__ __device__ int first(int o) const { return o < nb ? o * cb : nb * cb + (o - nb) * cs; }
  __host__ __device__ int cells(int o) const { return o < nb ? cb : cs; }
  // owner of cell `key` and the cell's index inside it
  __device__ __forceinline__ int owner(int key, int* local) const {
    const int kb = nb * cb;
    const bool big = key < kb;
    const unsigned k = static_cast<unsigned>(big ? key : key - kb);
    const int q = static_cast<int>((static_cast<unsigned long long>(k) * (big ? mb : ms)) >> 32);
    *local = static_cast<int>(k) - q * (big ? cb : cs);
    return (big ? 0 : nb) + q;
  }
};
__host__ inline unsigned long long owner_magic(int cells) {
  return ((1ull << 32) + static_cast<unsigned long long>(cells) - 1) / static_cast<unsigned long long>(cells);
}

struct PartArgs {
  int N, W, G;
  OwnerMap om;
  int64_t n;
  const float* x;    // first coordinate (row)
  const float* x1;   // second coordinate (row), taken times s1 (the additive model's
  float s1;          // pair transforms use (X_l1, -X_l2))
  const float* y;
  int has_y;
  int vec_ok;       // x (both rows) and y 16-byte aligned: float4 loads
  int nblk;         // partition blocks
  int64_t range;    // points per partition block
  int* cnt;         // [nblk][G]
  int* off;         // [nblk][G] offset of the block's run inside its owner's bucket
  int* tot;         // [G]
  uint4* rec;       // records, bucketed by owner
  float* ybuf;      // strengths of 8-byte records with a strength, same indices
  unsigned* flags;
  float c_hi, c_lo;
  // one-pass partition: owner o's bucket is rec[bucket_base(o), + bucket_cap(o)) (cap
  // for the big owners, cap_s for the others), filled through atomic reservations on
  // fill[o]; ovf is set when a bucket would overflow, and the exact kernels (count,
  // scan, scatter) then run instead (guarded = 1: they return at once when ovf is clear)
  int* fill;
  int cap, cap_s;
  unsigned* ovf;
  int guarded;
};

__host__ __device__ __forceinline__ int64_t bucket_base(const OwnerMap& om, int cap, int cap_s, int o) {
  return o < om.nb ? static_cast<int64_t>(o) * cap
                   : static_cast<int64_t>(om.nb) * cap + static_cast<int64_t>(o - om.nb) * cap_s;
}
__host__ __device__ __forceinline__ int bucket_cap(const OwnerMap& om, int cap, int cap_s, int o) {
  return o < om.nb ? cap : cap_s;
}

__device__ __forceinline__ bool skip_guarded(const PartArgs& A) {
  return A.guarded && *reinterpret_cast<const volatile unsigned*>(A.ovf) == 0u;
}

// owner and packed key of one point; returns false for a point out of range
// Partition records.  Rec16 {owner << 16 | local cell, f0, f1, y} (fp32 bits) carries a
// strength; Rec8 is the ones-only form of the one-pass partition, half the bytes and
// twice the records per accumulation round:
//   lo = v0 | v1 << 24,  hi = v1 >> 8 | local cell << 16,
//   v = (w/2 - f) 2^24 in [0, 2^24): exact, since f in (w/2 - 1, w/2] is a multiple
//   of 2^-24 for w >= 3 (fp32 spacing below 4), so g = f - (w - 1)/2 = 1/2 - v 2^-24
//   decodes to the same fp32 value.
struct Rec16 {
  using T = uint4;
  static constexpr bool HAS_Y = true, SPLIT_Y = false;
  static constexpr int NP_THREADS = THREADS_ACC;  // CTA size (= cells) without pair mode
  // records come from partitions that write only cells of their owner (checked bucket
  // capacities), so linking does not re-check them
  static constexpr bool CHECK_CELL = false;
  static constexpr int CAPR = 4096, CARRY = 2048;
  __device__ static int cell(const uint4& r) { return static_cast<int>(r.x & 0xFFFFu); }
  __device__ static float g0(const uint4& r, float gc) { return __uint_as_float(r.y) - gc; }
  __device__ static float g1(const uint4& r, float gc) { return __uint_as_float(r.z) - gc; }
  __device__ static float y(const uint4& r) { return __uint_as_float(r.w); }
  // first coordinate's offset given the parallel stream (unused by this type)
  __device__ static float g0x(const uint4& r, const float*, int, float gc) { return g0(r, gc); }
};
struct Rec8 {
  using T = uint2;
  static constexpr bool HAS_Y = false, SPLIT_Y = false;
  static constexpr int NP_THREADS = THREADS_ACC;
  static constexpr bool CHECK_CELL = false;
  static constexpr int CAPR = 10240, CARRY = 2048;
  __device__ static int cell(const uint2& r) { return static_cast<int>(r.y >> 16); }
  __device__ static float g0(const uint2& r, float) {
    return fmaf(static_cast<float>(r.x & 0xFFFFFFu), -5.9604644775390625e-8f, 0.5f);
  }
  __device__ static float g1(const uint2& r, float) {
    return fmaf(static_cast<float>(__funnelshift_r(r.x, r.y, 24) & 0xFFFFFFu), -5.9604644775390625e-8f, 0.5f);
  }
  __device__ static float y(const uint2&) { return 1.0f; }
  __device__ static float g0x(const uint2& r, const float*, int, float gc) { return g0(r, gc); }
};
// Rec8 records with the strengths in a parallel stream of floats (same indices):
// 12 bytes per point, 8192 records per round (and up to 512 deferred ones in front)
struct Rec8Y : Rec8 {
  static constexpr bool HAS_Y = true, SPLIT_Y = true;
  static constexpr int CAPR = 8192, CARRY = 512;
};
// Additive-model pair records (owners of two grid rows).  The record is the column
// coordinate's code word  r << 31 | c2 << 23 | v2  (r: the row inside the owner's two
// rows, c2: the window-start column, v2 = (w/2 - f2) 2^23) and the parallel stream holds
// the row coordinate's word  o1 = c1 << 24 | v1  (c1: window-start row, v1 = (w/2 - f1)
// 2^23, bit 23 clear).  f in (w/2 - 1, w/2] is a multiple of 2^-23 for f >= 1 (fp32
// spacing), so both offsets are exact for w >= 4, and g = f - (w-1)/2 = 1.5 - (1 + v 2^-23)
// decodes with one OR and one (exact) subtraction.
struct RecAdd {
  using T = unsigned;
  static constexpr bool HAS_Y = false, SPLIT_Y = true;
  static constexpr int NP_THREADS = 512;  // one lane per cell of two 256-node rows
  // linking checks each record's cell against the owner's cells (2N may be < 512)
  static constexpr bool CHECK_CELL = true;
  static constexpr int CAPR = 10752, CARRY = 512;
  __device__ static int cell(unsigned r) { return static_cast<int>(r >> 23); }
  // (no g0 or y: the row coordinate's offset comes from the parallel stream, g0x, and
  // the pair transforms carry no strength)
  __device__ static float g1(unsigned r, float) { return 1.5f - __uint_as_float(0x3F800000u | (r & 0x7FFFFFu)); }
  __device__ static float g0x(unsigned, const float* par, int i, float) {
    return 1.5f - __uint_as_float(0x3F800000u | (__float_as_uint(par[i]) & 0x7FFFFFu));
  }
};
// Rec8 of a Rec16 {key, f0, f1, -} built by the partition (w: kernel width)
__device__ __forceinline__ uint2 pack_rec8(const uint4& r, float half_w) {
  const unsigned v0 = static_cast<unsigned>((half_w - __uint_as_float(r.y)) * 16777216.0f);
  const unsigned v1 = static_cast<unsigned>((half_w - __uint_as_float(r.z)) * 16777216.0f);
  return make_uint2(v0 | (v1 << 24), (v1 >> 8) | ((r.x & 0xFFFFu) << 16));
}

__device__ __forceinline__ bool point_key(float x0, float x1, const PartArgs& A, float* f0, float* f1,
                                          uint32_t* packed) {
  int la, lb;
  if (!window_f32(x0, A.N, A.c_hi, A.c_lo, A.W, &la, f0)) return false;
  if (!window_f32(A.s1 * x1, A.N, A.c_hi, A.c_lo, A.W, &lb, f1)) return false;
  const int N = A.N;
  const int key = wrap_node(la, N) * N + wrap_node(lb, N);
  int local;
  const int o = A.om.owner(key, &local);
  *packed = (static_cast<uint32_t>(o) << 16) | static_cast<uint32_t>(local);
  return true;
}

__global__ void __launch_bounds__(P_THREADS) k_bin_count(PartArgs A) {
  if (skip_guarded(A)) return;
  extern __shared__ int whist[];  // [P_NWARPS][G]
  const int tid = threadIdx.x, warp = tid >> 5;
  const int G = A.G;
  for (int o = tid; o < P_NWARPS * G; o += P_THREADS) whist[o] = 0;
  __syncthreads();
  const int64_t s = static_cast<int64_t>(blockIdx.x) * A.range;
  const int64_t e = min(A.n, s + A.range);
  int* wh = whist + warp * G;
  auto one = [&](float a0, float a1) {
    float f0, f1;
    uint32_t k;
    if (point_key(a0, a1, A, &f0, &f1, &k)) atomicAdd(&wh[k >> 16], 1);
    else atomicOr(A.flags, FLAG_RANGE);
  };
  if (A.vec_ok) {
    // four points per thread and iteration (float4 loads keep more bytes in flight)
    for (int64_t i = s + 4 * tid; i < e; i += 4 * P_THREADS) {
      if (i + 3 < e) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(A.x + i));
        const float4 c = __ldg(reinterpret_cast<const float4*>(A.x1 + i));
        one(a.x, c.x);
        one(a.y, c.y);
        one(a.z, c.z);
        one(a.w, c.w);
      } else {
        for (int64_t j = i; j < e; ++j) one(__ldg(A.x + j), __ldg(A.x1 + j));
      }
    }
  } else {
    for (int64_t i = s + tid; i < e; i += P_THREADS) one(__ldg(A.x + i), __ldg(A.x1 + i));
  }
  __syncthreads();
  for (int o = tid; o < G; o += P_THREADS) {
    int c = 0;
    for (int w = 0; w < P_NWARPS; ++w) c += whist[w * G + o];
    A.cnt[static_cast<size_t>(blockIdx.x) * G + o] = c;
  }
}

// one CTA per owner: exclusive scan over partition blocks
__global__ void k_bin_scan(PartArgs A) {
  if (skip_guarded(A)) return;
  __shared__ int wsum[32];
  const int o = blockIdx.x, G = A.G;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int carry = 0;
  for (int b0 = 0; b0 < A.nblk; b0 += blockDim.x) {
    const int bb = b0 + tid;
    // runs are padded to whole 128-byte lines (8 records) so that no line is shared by
    // two blocks' runs; the padding holds sentinel records
    const int v = (bb < A.nblk) ? ((A.cnt[static_cast<size_t>(bb) * G + o] + 7) & ~7) : 0;
    int incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int wpre = 0, total = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
      if (w < warp) wpre += wsum[w];
      total += wsum[w];
    }
    if (bb < A.nblk) A.off[static_cast<size_t>(bb) * G + o] = carry + wpre + incl - v;
    carry += total;
    __syncthreads();
  }
  if (tid == 0) A.tot[o] = carry;
}

// exclusive scan of tot[0..G) into base[0..G] by the whole block (G < blockDim.x);
// every total is loaded once, in parallel.  wsum: 32 ints of shared scratch.
__device__ __forceinline__ void owner_bases(const int* tot, int G, int* base, int* wsum) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int v = (tid < G) ? __ldg(tot + tid) : 0;
  int incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  int pre = 0;
  for (int w = 0; w < warp; ++w) pre += wsum[w];
  if (tid <= G) base[tid] = pre + incl - v;
  __syncthreads();
}

// Scatter in tiles of S_TILE points per block (one block per SM): the tile is sorted
// by owner in shared memory and copied out with coalesced stores, so each owner's run
// from a tile (S_TILE / G records on average) lands as one contiguous write; scattered
// 16-byte writes would run at a small fraction of the write bandwidth.
constexpr int S_THREADS = 1024;
constexpr int S_TILE = 12288;

__global__ void __launch_bounds__(S_THREADS, 1) k_bin_scatter(PartArgs A) {
  if (skip_guarded(A)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int wsum[32];
  const int G = A.G;
  uint4* sorted = reinterpret_cast<uint4*>(smem);                          // [S_TILE]
  unsigned short* own = reinterpret_cast<unsigned short*>(sorted + S_TILE); // [S_TILE] owner per point
  int* cursor = reinterpret_cast<int*>(own + S_TILE);                      // [G + 1] global run positions
  int* tcnt = cursor + (G + 1);                                            // [G + 1] tile counts -> offsets
  int* tcur = tcnt + (G + 1);                                              // [G] fill cursors inside the tile
  const int tid = threadIdx.x;
  owner_bases(A.tot, G, cursor, wsum);
  for (int o = tid; o < G; o += S_THREADS) cursor[o] += A.off[static_cast<size_t>(blockIdx.x) * G + o];
  const int64_t s0 = static_cast<int64_t>(blockIdx.x) * A.range;
  const int64_t e0 = min(A.n, s0 + A.range);
  for (int64_t t0 = s0; t0 < e0; t0 += S_TILE) {
    const int cnt = (e0 - t0 < S_TILE) ? static_cast<int>(e0 - t0) : S_TILE;
    for (int o = tid; o <= G; o += S_THREADS) tcnt[o] = 0;
    __syncthreads();
    // pass 1: owners and tile histogram
    auto own_of = [&](int i, float a0, float a1) {
      float f0, f1;
      uint32_t k;
      unsigned short o = 0xFFFF;
      if (point_key(a0, a1, A, &f0, &f1, &k)) {
        o = static_cast<unsigned short>(k >> 16);
        atomicAdd(&tcnt[o], 1);
      }
      own[i] = o;
    };
    if (A.vec_ok) {
      for (int i = 4 * tid; i < cnt; i += 4 * S_THREADS) {
        if (i + 3 < cnt) {
          const float4 a = __ldg(reinterpret_cast<const float4*>(A.x + t0 + i));
          const float4 c = __ldg(reinterpret_cast<const float4*>(A.x1 + t0 + i));
          own_of(i, a.x, c.x);
          own_of(i + 1, a.y, c.y);
          own_of(i + 2, a.z, c.z);
          own_of(i + 3, a.w, c.w);
        } else {
          for (int j = i; j < cnt; ++j) own_of(j, __ldg(A.x + t0 + j), __ldg(A.x1 + t0 + j));
        }
      }
    } else {
      for (int i = tid; i < cnt; i += S_THREADS) own_of(i, __ldg(A.x + t0 + i), __ldg(A.x1 + t0 + i));
    }
    __syncthreads();
    if (tid < 32) {  // exclusive scan of the tile counts (one warp)
      int carry = 0;
      for (int o0 = 0; o0 <= G; o0 += 32) {
        const int o = o0 + tid;
        const int v = (o < G) ? tcnt[o] : 0;
        int incl = v;
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, incl, dd);
          if (tid >= dd) incl += t;
        }
        if (o <= G) tcnt[o] = carry + incl - v;
        carry += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
    __syncthreads();
    for (int o = tid; o < G; o += S_THREADS) tcur[o] = tcnt[o];
    __syncthreads();
    // pass 2: records straight into their sorted slots (inputs re-read, now from L2)
    for (int i = tid; i < cnt; i += S_THREADS) {
      const unsigned short o = own[i];
      if (o == 0xFFFF) continue;
      float f0, f1;
      uint32_t k;
      point_key(__ldg(A.x + t0 + i), __ldg(A.x1 + t0 + i), A, &f0, &f1, &k);
      const int pos = atomicAdd(&tcur[o], 1);
      sorted[pos] = make_uint4(k, __float_as_uint(f0), __float_as_uint(f1),
                               A.has_y ? __float_as_uint(__ldg(A.y + t0 + i)) : 0u);
    }
    __syncthreads();
    // coalesced copy-out: record j belongs to owner o = its high bits; its global slot is
    // the owner's cursor plus its rank inside the owner's run of this tile
    const int valid = tcnt[G];
    for (int j = tid; j < valid; j += S_THREADS) {
      const uint4 r = sorted[j];
      const int o = static_cast<int>(r.x >> 16);
      A.rec[cursor[o] + (j - tcnt[o])] = r;
    }
    __syncthreads();
    for (int o = tid; o < G; o += S_THREADS) cursor[o] += tcnt[o + 1] - tcnt[o];
    __syncthreads();
  }
  // sentinel records fill each run up to its padded length
  for (int o = tid; o < G; o += S_THREADS) {
    const int c = A.cnt[static_cast<size_t>(blockIdx.x) * G + o];
    for (int k = c; k < ((c + 7) & ~7); ++k) A.rec[cursor[o]++] = make_uint4(0xFFFFu, 0u, 0u, 0u);
  }
}

// Pipelined scatter for aligned inputs: the next tile's coordinates and strengths
// arrive by TMA bulk copies while the current tile is sorted and written out; each
// thread keeps its points' records in registers between the histogram and the
// placement, so every key is computed once.
constexpr int S2_THREADS = 1024;
constexpr int S2_PER = 7;                       // points per thread per tile
constexpr int S2_TILE = S2_THREADS * S2_PER;    // 7168

struct S2Layout {
  size_t stage, sorted, ints, bar, total;
};
__host__ __device__ inline S2Layout s2_layout(int G, int tile = S2_TILE) {
  S2Layout L;
  L.stage = 0;                                             // float [3][tile]
  L.sorted = L.stage + sizeof(float) * 3 * tile;           // uint4 [tile]
  L.ints = L.sorted + sizeof(uint4) * tile;                // int [4 (G + 1)]
  L.bar = (L.ints + sizeof(int) * 4 * (G + 1) + 15) & ~static_cast<size_t>(15);
  L.total = L.bar + 16;
  return L;
}

__global__ void __launch_bounds__(S2_THREADS, 1) k_bin_scatter2(PartArgs A) {
  if (skip_guarded(A)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int wsum[32];
  const int G = A.G;
  const S2Layout L = s2_layout(G);
  float* stage = reinterpret_cast<float*>(smem + L.stage);
  uint4* sorted = reinterpret_cast<uint4*>(smem + L.sorted);
  int* cursor = reinterpret_cast<int*>(smem + L.ints);  // [G + 1]
  int* tcnt = cursor + (G + 1);                          // [G + 1]
  int* tcur = tcnt + (G + 1);                            // [G + 1]
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
  const int tid = threadIdx.x;
  owner_bases(A.tot, G, cursor, wsum);
  for (int o = tid; o < G; o += S2_THREADS) cursor[o] += A.off[static_cast<size_t>(blockIdx.x) * G + o];
  const int64_t s0 = static_cast<int64_t>(blockIdx.x) * A.range;
  const int64_t e0 = min(A.n, s0 + A.range);
  if (tid == 0) {
    mbar_init(bar);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int64_t t0) {  // one thread: bulk copies of tile t0
    const int cnt = static_cast<int>(min(static_cast<int64_t>(S2_TILE), e0 - t0));
    const unsigned bytes = static_cast<unsigned>(cnt) * 4u;
    fence_proxy_async();
    mbar_arrive_expect(bar, bytes * (A.has_y ? 3u : 2u));
    bulk_g2s(stage, A.x + t0, bytes, bar);
    bulk_g2s(stage + S2_TILE, A.x1 + t0, bytes, bar);
    if (A.has_y) bulk_g2s(stage + 2 * S2_TILE, A.y + t0, bytes, bar);
  };
  if (tid == 0 && s0 < e0) issue(s0);
  unsigned phase = 0;
  for (int64_t t0 = s0; t0 < e0; t0 += S2_TILE) {
    const int cnt = static_cast<int>(min(static_cast<int64_t>(S2_TILE), e0 - t0));
    for (int o = tid; o <= G; o += S2_THREADS) tcnt[o] = 0;
    if (!mbar_wait(bar, phase, A.flags)) {
      mbar_drain(bar, phase);
      return;
    }
    phase ^= 1u;
    __syncthreads();
    uint4 rec[S2_PER];
#pragma unroll
    for (int k = 0; k < S2_PER; ++k) {
      const int i = k * S2_THREADS + tid;
      rec[k].x = 0xFFFFFFFFu;
      if (i < cnt) {
        float f0, f1;
        uint32_t key;
        if (point_key(stage[i], stage[S2_TILE + i], A, &f0, &f1, &key)) {
          rec[k] = make_uint4(key, __float_as_uint(f0), __float_as_uint(f1),
                              A.has_y ? __float_as_uint(stage[2 * S2_TILE + i]) : 0u);
          atomicAdd(&tcnt[key >> 16], 1);
        }
      }
    }
    __syncthreads();
    if (tid == 0 && t0 + S2_TILE < e0) issue(t0 + S2_TILE);  // the stage is free again
    if (tid < 32) {  // exclusive scan of the tile counts (one warp)
      int carry = 0;
      for (int o0 = 0; o0 <= G; o0 += 32) {
        const int o = o0 + tid;
        const int v = (o < G) ? tcnt[o] : 0;
        int incl = v;
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, incl, dd);
          if (tid >= dd) incl += t;
        }
        if (o <= G) {
          tcnt[o] = carry + incl - v;
          tcur[o] = carry + incl - v;
        }
        carry += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < S2_PER; ++k) {
      if (rec[k].x != 0xFFFFFFFFu) {
        const int pos = atomicAdd(&tcur[rec[k].x >> 16], 1);
        sorted[pos] = rec[k];
      }
    }
    __syncthreads();
    const int valid = tcnt[G];
    for (int j = tid; j < valid; j += S2_THREADS) {
      const uint4 r = sorted[j];
      const int o = static_cast<int>(r.x >> 16);
      A.rec[cursor[o] + (j - tcnt[o])] = r;
    }
    __syncthreads();
    for (int o = tid; o < G; o += S2_THREADS) cursor[o] += tcnt[o + 1] - tcnt[o];
    __syncthreads();
  }
  for (int o = tid; o < G; o += S2_THREADS) {
    const int c = A.cnt[static_cast<size_t>(blockIdx.x) * G + o];
    for (int k = c; k < ((c + 7) & ~7); ++k) A.rec[cursor[o]++] = make_uint4(0xFFFFu, 0u, 0u, 0u);
  }
}

// One-pass scatter (no count pass): as k_bin_scatter2, but each tile reserves room
// for its owner runs in fixed-capacity buckets with one global atomic per (tile,
// owner).  A reservation that would pass the capacity writes nothing and sets ovf.
// T threads per block: 1024 (one block per SM) or 512 (two per SM, half the tile)
template <int PER, bool REC8, int T>
__global__ void __launch_bounds__(T, 1024 / T) k_bin_scatter1(PartArgs A) {
  constexpr int TILE = T * PER;
  extern __shared__ __align__(16) unsigned char smem[];
  const int G = A.G;
  const S2Layout L = s2_layout(G, TILE);
  float* stage = reinterpret_cast<float*>(smem + L.stage);
  uint4* sorted = reinterpret_cast<uint4*>(smem + L.sorted);
  int* tcnt = reinterpret_cast<int*>(smem + L.ints);  // [G + 1] counts of the tile
  int* toff = tcnt + (G + 1);                          // [G + 1] run starts inside the tile
  // [G + 1] bucket index of tile slot 0 for each owner's run (owner base + reserved
  // slot - run start; may be negative), or NO_ROOM
  long long* gdelta = reinterpret_cast<long long*>(toff + (G + 1));
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
  const int tid = threadIdx.x;
  const int64_t s0 = static_cast<int64_t>(blockIdx.x) * A.range;
  const int64_t e0 = min(A.n, s0 + A.range);
  if (tid == 0) {
    mbar_init(bar);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  for (int o = tid; o <= G; o += T) tcnt[o] = 0;
  __syncthreads();
  auto issue = [&](int64_t t0) {
    const int cnt = static_cast<int>(min(static_cast<int64_t>(TILE), e0 - t0));
    const unsigned bytes = static_cast<unsigned>(cnt) * 4u;
    fence_proxy_async();
    mbar_arrive_expect(bar, bytes * (A.has_y ? 3u : 2u));
    bulk_g2s(stage, A.x + t0, bytes, bar);
    bulk_g2s(stage + TILE, A.x1 + t0, bytes, bar);
    if (A.has_y) bulk_g2s(stage + 2 * TILE, A.y + t0, bytes, bar);
  };
  if (tid == 0 && s0 < e0) issue(s0);
  unsigned phase = 0;
  // Three barriers per tile.  Each thread waits for the tile's bulk copy itself; the
  // tile counts are zeroed after their last read of the tile before (between its
  // second and third barriers), and every shared array the next tile writes before its
  // first barrier (the counts) is one this tile no longer reads after its third, while
  // those it writes later (run starts, bucket positions, sorted records, the staged
  // points) are only written after that first barrier, which every thread reaches
  // after its copy-out.
  for (int64_t t0 = s0; t0 < e0; t0 += TILE) {
    const int cnt = static_cast<int>(min(static_cast<int64_t>(TILE), e0 - t0));
    if (!mbar_wait(bar, phase, A.flags)) {
      mbar_drain(bar, phase);
      return;
    }
    phase ^= 1u;
    // rk: the point's rank among the tile's points of its owner (its place in the
    // owner's run)
    uint4 rec[PER];
    int rk[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = k * T + tid;
      rec[k].x = 0xFFFFFFFFu;
      rk[k] = 0;
      if (i < cnt) {
        float f0, f1;
        uint32_t key;
        if (point_key(stage[i], stage[TILE + i], A, &f0, &f1, &key)) {
          rec[k] = make_uint4(key, __float_as_uint(f0), __float_as_uint(f1),
                              A.has_y ? __float_as_uint(stage[2 * TILE + i]) : 0u);
          rk[k] = atomicAdd(&tcnt[key >> 16], 1);
        } else {
          atomicOr(A.flags, FLAG_RANGE);
        }
      }
    }
    __syncthreads();
    if (tid == 0 && t0 + TILE < e0) issue(t0 + TILE);
    // reservations in the buckets, one global atomic per owner present in the tile;
    // the returned slot is needed only for the copy-out, so the atomic's latency
    // overlaps the scan and the placement
    int my_c = 0, my_pos = -1;
    if (tid < G) {
      my_c = tcnt[tid];
      if (my_c > 0) my_pos = atomicAdd(A.fill + tid, my_c);
    }
    if (tid >= T - 32) {  // exclusive scan of the tile counts (last warp)
      // each lane sums a run of consecutive owners, one warp scan of the run sums,
      // then each lane writes its run's prefixes: no serial loop over warp-wide chunks
      const int ln = tid - (T - 32);
      const int per = (G + 1 + 31) / 32;
      const int o0 = ln * per, o1 = min(o0 + per, G + 1);
      int run = 0;
      for (int o = o0; o < o1; ++o) run += (o < G) ? tcnt[o] : 0;
      int incl = run;
#pragma unroll
      for (int dd = 1; dd < 32; dd <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, dd);
        if (ln >= dd) incl += t;
      }
      int acc = incl - run;
      for (int o = o0; o < o1; ++o) {
        toff[o] = acc;
        acc += (o < G) ? tcnt[o] : 0;
      }
    }
    __syncthreads();
    for (int o = tid; o <= G; o += T) tcnt[o] = 0;  // the next tile's counts
#pragma unroll
    for (int k = 0; k < PER; ++k)
      if (rec[k].x != 0xFFFFFFFFu) sorted[toff[rec[k].x >> 16] + rk[k]] = rec[k];
    if (tid < G) {
      if (my_c > 0 && my_pos + my_c > bucket_cap(A.om, A.cap, A.cap_s, tid)) {
        atomicOr(A.ovf, 1u);
        my_pos = -1;
      }
      gdelta[tid] = my_pos >= 0 ? bucket_base(A.om, A.cap, A.cap_s, tid) + my_pos - toff[tid] : NO_ROOM;
    }
    __syncthreads();
    const int valid = toff[G];
    // a fixed trip count, so that every thread's PER loads are in flight at once
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int j = k * T + tid;
      if (j < valid) {
        const uint4 r = sorted[j];
        const long long gd = gdelta[r.x >> 16];
        const int64_t at = gd + j;
        if (gd != NO_ROOM &&
            fk_check(at >= 0 && at < bucket_base(A.om, A.cap, A.cap_s, A.G), A.flags)) {
          if (REC8) {
            reinterpret_cast<uint2*>(A.rec)[at] = pack_rec8(r, 0.5f * static_cast<float>(A.W));
            if (A.has_y) A.ybuf[at] = __uint_as_float(r.w);
          } else {
            A.rec[at] = r;
          }
        }
      }
    }
  }
}

struct AccArgs {
  int N, G, ncells;
  OwnerMap om;
  int cpc_max;  // cells of the largest owner (the shared-memory layout's size)
  float beta;
  EsPoly poly;  // tap polynomials of the plan's width
  int with_ones;
  const int* tot;   // [G]
  const uint4* rec;
  const float* ybuf;  // strengths beside 8-byte records (Rec8Y)
  double* grid;
  unsigned* flags;
  // mode 0: buckets from the exact partition (tot); 1: one-pass buckets (fill, cap),
  // skipped when ovf is set; 2: exact buckets, run only when ovf is set
  int mode;
  const int* fill;
  int cap, cap_s;
  const unsigned* ovf;
  float qmul;  // per-round quota = mean load + qmul sqrt(mean load)
  // several problems sharing the owner layout in one launch: CTA (b, sub) with
  // b = blockIdx / nsub; problem sub reads rec + sub sub_rec_stride (the parallel stream
  // ybuf is shared) and adds into grid + sub sub_grid_stride
  int nsub;
  int64_t sub_rec_stride, sub_grid_stride;
  int pad4;  // exact buckets (mode 0) start at multiples of 4 records (16-byte copies)
};

struct AccLayout {
  size_t stage, ystage, nxt, head, ccount, xcnt, total;
};
template <typename R>
__host__ __device__ inline AccLayout acc_layout(int cpc) {
  constexpr int CAPR = R::CAPR, CARRY = R::CARRY;
  AccLayout L{};
  L.stage = 0;                                                      // [2][CARRY + CAPR] records
  L.ystage = L.stage + sizeof(typename R::T) * 2 * (CARRY + CAPR);  // [2][CARRY + CAPR] floats
  const size_t yb = R::SPLIT_Y ? sizeof(float) * 2 * (CARRY + CAPR) : 0;
  L.nxt = L.ystage + yb;                                            // [CARRY + CAPR] u16
  L.head = (L.nxt + sizeof(unsigned short) * (CARRY + CAPR) + 15) & ~static_cast<size_t>(15);  // [cpc] int
  L.ccount = L.head + sizeof(int) * cpc;                            // [cpc] int
  L.xcnt = L.ccount + sizeof(int) * cpc;                            // [cpc] int
  L.total = L.xcnt + sizeof(int) * cpc;
  return L;
}

// W x W fp32 register window, acc[i][j] for tap i of the first coordinate and tap j of
// the second.  Scalar form: one fmaf per element.  Packed form: rows k and W - 1 - k
// of a column share a 64-bit register pair, so that one packed FMA (fma.rn.f32x2,
// sm_100 and later) updates both from the mirrored weight pair that the tap polynomial
// yields at once (es_taps_poly_pairs); every element is still one fused multiply-add
// rounded to nearest.  The packed form pays where each lane evaluates both
// coordinates' weights itself (one channel per lane); in pair mode the partner's
// weights arrive one by one through shuffles and the scalar form measured faster.
template <int W, bool PACKED>
struct Win;
template <int W>
struct Win<W, false> {
  float a[W][W];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < W; ++i)
#pragma unroll
      for (int j = 0; j < W; ++j) a[i][j] = 0.f;
  }
  __device__ __forceinline__ float get(int i, int j) const { return a[i][j]; }
  // column j += e t
  __device__ __forceinline__ void fma_col(const float* e, float t, int j) {
#pragma unroll
    for (int i = 0; i < W; ++i) a[i][j] = fmaf(e[i], t, a[i][j]);
  }
};
template <int W>
struct Win<W, true> {
  float2 p[W / 2][W];        // (row k, row W - 1 - k) of column j
  float r[(W & 1) ? W : 1];  // the middle row when W is odd
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int j = 0; j < W; ++j) {
#pragma unroll
      for (int k = 0; k < W / 2; ++k) p[k][j] = make_float2(0.f, 0.f);
      if constexpr (W & 1) r[j] = 0.f;
    }
  }
  __device__ __forceinline__ float get(int i, int j) const {
    if constexpr (W & 1) {
      if (i == W / 2) return r[j];
    }
    return i < W / 2 ? p[i][j].x : p[W - 1 - i][j].y;
  }
  // column j += e t, e as mirrored pairs (and the middle weight)
  __device__ __forceinline__ void fma_col(const float2* ep, float emid, float t, int j) {
    const float2 t2 = make_float2(t, t);
#pragma unroll
    for (int k = 0; k < W / 2; ++k) p[k][j] = __ffma2_rn(ep[k], t2, p[k][j]);
    if constexpr (W & 1) r[j] = fmaf(emid, t, r[j]);
  }
};

template <int W, bool PAIR, typename R>
__global__ void __launch_bounds__(PAIR ? Cfg<true>::THREADS : R::NP_THREADS, 1) k_bin_accumulate(AccArgs A) {
  static_assert(!PAIR || R::HAS_Y, "pair mode carries a strength");
  using RT = typename R::T;
  constexpr int THREADS = PAIR ? Cfg<true>::THREADS : R::NP_THREADS;
  constexpr int CAPR = R::CAPR, CARRY = R::CARRY;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_base, s_count, s_abort;
  __shared__ int s_ncar[2];  // records deferred into buffer b (counted during the round before)
  __shared__ __align__(8) uint64_t s_bar[2];
  const int tid = threadIdx.x, lane = tid & 31;
  const int nsub = A.nsub > 0 ? A.nsub : 1;
  const int b = blockIdx.x / nsub;
  const int sub = blockIdx.x - b * nsub;
  const typename R::T* recs = reinterpret_cast<const typename R::T*>(A.rec) + sub * A.sub_rec_stride;
  double* grid_s = A.grid + sub * A.sub_grid_stride;
  const int N = A.N;
  const int cpc = A.cpc_max;
  const int cell = PAIR ? (tid >> 1) : tid;
  const int ch = PAIR ? (tid & 1) : 0;
  const unsigned pmask = 3u << (lane & 30);
  const int my_first_cell = A.om.first(b);
  const int my_ncells = max(0, min(A.om.cells(b), A.ncells - my_first_cell));
  const bool owns = cell < my_ncells;
  const float gc = 0.5f * static_cast<float>(W - 1);  // window centre: g = f - gc
  const AccLayout L = acc_layout<R>(cpc);
  RT* stage = reinterpret_cast<RT*>(smem + L.stage);
  float* ystage = reinterpret_cast<float*>(smem + L.ystage);  // SPLIT_Y only
  unsigned short* nxt = reinterpret_cast<unsigned short*>(smem + L.nxt);
  int* head = reinterpret_cast<int*>(smem + L.head);
  int* ccount = reinterpret_cast<int*>(smem + L.ccount);
  int* xcnt = reinterpret_cast<int*>(smem + L.xcnt);  // records linked beyond the quota

  if (A.mode != 0) {
    const bool ov = *reinterpret_cast<const volatile unsigned*>(A.ovf) != 0u;
    if (ov != (A.mode == 2)) return;
  }
  if (A.mode == 1) {
    if (tid == 0) {
      s_base = static_cast<int>(bucket_base(A.om, A.cap, A.cap_s, b));
      s_count = min(__ldg(A.fill + b), bucket_cap(A.om, A.cap, A.cap_s, b));
      s_ncar[0] = s_ncar[1] = 0;
      s_abort = 0;
      mbar_init(&s_bar[0]);
      mbar_init(&s_bar[1]);
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
  } else {
    // bucket of this owner = [sum of earlier totals, + tot[b]): one load per thread
    __shared__ int wsum[32];
    int v = 0;
    for (int o = tid; o < b; o += THREADS) v += A.pad4 ? ((__ldg(A.tot + o) + 3) & ~3) : __ldg(A.tot + o);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if (lane == 0) wsum[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      int sum = 0;
      for (int w = 0; w < THREADS / 32; ++w) sum += wsum[w];
      s_base = sum;
      s_count = __ldg(A.tot + b);
      s_ncar[0] = s_ncar[1] = 0;
      s_abort = 0;
      mbar_init(&s_bar[0]);
      mbar_init(&s_bar[1]);
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
  }
  for (int i = tid; i < cpc; i += THREADS) {
    head[i] = 0xFFFF;
    ccount[i] = 0;
    xcnt[i] = 0;
  }
  __syncthreads();
  const int base = s_base, count = s_count;
  const int nrounds = (count + CAPR - 1) / CAPR;
  if (nrounds == 0) return;

  Win<W, !PAIR> acc;
  acc.zero();
  // the register window goes into the fp64 grid at the end, and also whenever FLUSH_PTS
  // points have been added since the last flush, so that an fp32 running sum never
  // spans more than that many points (crowded cells)
  int since = 0;
  auto flush = [&]() {
    const int key = my_first_cell + cell;
    const int64_t GN = static_cast<int64_t>(N) * N;
    const int c0 = key / N;
    const int c1 = key - c0 * N;
    double* g = grid_s + (PAIR ? ch : 0) * GN;
    const bool transposed = PAIR && ch == 1;
#pragma unroll
    for (int i = 0; i < W; ++i)
#pragma unroll
      for (int j = 0; j < W; ++j) {
        const int a = transposed ? j : i, bb = transposed ? i : j;
        if (fk_check(key < A.ncells, A.flags))
          atomicAdd(g + static_cast<int64_t>((c0 + a) & (N - 1)) * N + ((c1 + bb) & (N - 1)),
                    static_cast<double>(acc.get(i, j)));
      }
    acc.zero();
  };

  auto issue = [&](int r) {
    const int nr = min(CAPR, count - r * CAPR);
    RT* dst = stage + (r & 1) * (CARRY + CAPR) + CARRY;
    // whole 16-byte units (an 8-byte record list of odd length reads one record past its
    // end, inside the record buffer, which the round never links)
    const unsigned bytes = (static_cast<unsigned>(nr) * static_cast<unsigned>(sizeof(RT)) + 15u) & ~15u;
    const unsigned ybytes = R::SPLIT_Y ? ((static_cast<unsigned>(nr) * 4u + 15u) & ~15u) : 0u;
    fence_proxy_async();
    mbar_arrive_expect(&s_bar[r & 1], bytes + ybytes);
    bulk_g2s(dst, recs + base + static_cast<int64_t>(r) * CAPR, bytes, &s_bar[r & 1]);
    if (R::SPLIT_Y)
      bulk_g2s(ystage + (r & 1) * (CARRY + CAPR) + CARRY, A.ybuf + base + static_cast<int64_t>(r) * CAPR, ybytes,
               &s_bar[r & 1]);
  };
  if (tid == 0) issue(0);

  for (int r = 0; r < nrounds; ++r) {
    const int buf = r & 1, nb = buf ^ 1;
    RT* st = stage + buf * (CARRY + CAPR);
    const float* yst = ystage + buf * (CARRY + CAPR);
    RT* nst = stage + nb * (CARRY + CAPR);
    float* nyst = ystage + nb * (CARRY + CAPR);
    const int nr = min(CAPR, count - r * CAPR);
    const int nc = min(s_ncar[buf], CARRY);
    if (!mbar_wait(&s_bar[buf], (r >> 1) & 1, A.flags)) s_abort = 1;
    __syncthreads();
    if (s_abort) {
      mbar_drain(&s_bar[buf], (r >> 1) & 1);
      return;
    }
    if (tid == 0 && r + 1 < nrounds) issue(r + 1);
    // records of this round: [CARRY - nc, CARRY + nr) of the buffer, the ones deferred
    // from the last round in front
    const int lo = CARRY - nc, hi = CARRY + nr;
    const bool last = (r == nrounds - 1);
    int q = 0x7FFFFFFF;
    if (!last && my_ncells > 0) {
      const float lam = static_cast<float>(hi - lo) / static_cast<float>(my_ncells);
      q = static_cast<int>(ceilf(lam + A.qmul * sqrtf(lam)));
    }
    // A record's rank in its cell (the count atomic's old value) decides at once: below
    // the quota it is linked into the cell's list, else it moves to the front of the
    // next buffer (deferred to the next round) while there is room, and is linked
    // beyond the quota (xcnt) when there is not.  LU records per thread and trip, so
    // that their shared-memory atomics overlap (measured best: 4 in pair mode, 2 with one
    // lane per cell).
    constexpr int LU = PAIR ? 4 : 2;
    for (int base = lo + tid; base < hi; base += LU * THREADS) {
      int cl[LU], rk[LU];
#pragma unroll
      for (int u = 0; u < LU; ++u) {
        const int idx = base + u * THREADS;
        cl[u] = (idx < hi) ? R::cell(st[idx]) : 0xFFFF;  // 0xFFFF: run padding
        if (R::CHECK_CELL || kChecked) {
          if (cl[u] >= cpc) {  // a record that names no cell of this owner
            if (cl[u] != 0xFFFF) atomicOr(A.flags, FLAG_INTERNAL);
            cl[u] = 0xFFFF;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < LU; ++u)
        if (cl[u] != 0xFFFF) rk[u] = atomicAdd(&ccount[cl[u]], 1);
#pragma unroll
      for (int u = 0; u < LU; ++u)
        if (cl[u] != 0xFFFF) {
          const int idx = base + u * THREADS;
          bool link = rk[u] < q;
          if (!link) {
            const int pd = atomicAdd(&s_ncar[nb], 1);
            if (pd < CARRY) {
              nst[CARRY - 1 - pd] = st[idx];
              if (R::SPLIT_Y) nyst[CARRY - 1 - pd] = yst[idx];
            } else {
              link = true;
              atomicAdd(&xcnt[cl[u]], 1);
            }
          }
          if (link) nxt[idx] = static_cast<unsigned short>(atomicExch(&head[cl[u]], idx));
        }
    }
    __syncthreads();
    if (tid == 0) s_ncar[buf] = 0;  // read by every thread before this round's first barrier
    const int mine = owns ? min(ccount[cell], q) + xcnt[cell] : 0;
    int ri = owns ? head[cell] : 0xFFFF;
    // walk the next nproc records of this lane's list into the window
    auto walk = [&](const int nproc) {
      if constexpr (PAIR) {
        // lane 0 of the pair: ones channel, window [a][b]; lane 1: strength channel,
        // window transposed ([b][a]) because it holds the second coordinate's weights.
        // Two records per iteration for independent work in flight.
        int k = 0;
        // strength of the record at index i (the ones lane uses 1)
        auto strength = [&](const RT& r, int i) {
          if constexpr (R::SPLIT_Y) return yst[i];
          else return R::y(r);
        };
        for (; k + 1 < nproc; k += 2) {
          const int ia = ri;
          if (!fk_check(ia < hi, A.flags)) break;
          const RT ra = st[ia];
          const int rj = nxt[ia];
          if (!fk_check(rj < hi, A.flags)) break;
          const RT rb = st[rj];
          ri = nxt[rj];
          float ea[W], eb[W];
          es_taps_poly<W, true>(ch == 0 ? R::g0(ra, gc) : R::g1(ra, gc), A.poly, ea);
          es_taps_poly<W, true>(ch == 0 ? R::g0(rb, gc) : R::g1(rb, gc), A.poly, eb);
          const float wa = (ch == 0) ? 1.0f : strength(ra, ia);
          const float wb = (ch == 0) ? 1.0f : strength(rb, rj);
#pragma unroll
          for (int j = 0; j < W; ++j) {
            const float ta = wa * __shfl_xor_sync(pmask, ea[j], 1);
            const float tb = wb * __shfl_xor_sync(pmask, eb[j], 1);
            acc.fma_col(ea, ta, j);
            acc.fma_col(eb, tb, j);
          }
        }
        if (k < nproc && fk_check(ri < hi, A.flags)) {
          const int ia = ri;
          const RT ra = st[ia];
          ri = nxt[ia];
          float ea[W];
          es_taps_poly<W, true>(ch == 0 ? R::g0(ra, gc) : R::g1(ra, gc), A.poly, ea);
          const float wa = (ch == 0) ? 1.0f : strength(ra, ia);
#pragma unroll
          for (int j = 0; j < W; ++j) {
            const float ta = wa * __shfl_xor_sync(pmask, ea[j], 1);
            acc.fma_col(ea, ta, j);
          }
        }
      } else {
        // one channel: ones (no strength multiply) or the strengths
        auto one_channel = [&](auto ones_tag) {
          constexpr bool ONES = decltype(ones_tag)::value;
          for (int k = 0; k < nproc; ++k) {
            const int ir = ri;
            if (!fk_check(ir < hi, A.flags)) break;
            const RT rec = st[ir];
            ri = nxt[ir];
            float2 px[W / 2];
            float pm = 0.f, py[W];
            es_taps_poly_pairs<W>(R::g0x(rec, yst, ir, gc), A.poly, px, &pm);
            es_taps_poly<W>(R::g1(rec, gc), A.poly, py);
            if (!ONES) {
              float sv;
              if constexpr (R::SPLIT_Y) sv = yst[ir];
              else sv = R::y(rec);
#pragma unroll
              for (int t = 0; t < W / 2; ++t) px[t] = __fmul2_rn(px[t], make_float2(sv, sv));
              pm *= sv;
            }
#pragma unroll
            for (int j = 0; j < W; ++j) acc.fma_col(px, pm, py[j], j);
          }
        };
        if (A.with_ones)
          one_channel(std::true_type{});
        else
          one_channel(std::false_type{});
      }
    };
    // the lane's records of this round: in one run, flushed once FLUSH_PTS points have
    // gone into the window since its last flush; a crowded round (more than CROWD_RUN
    // records) in runs of CROWD_RUN, each flushed.  So no fp32 running sum spans more
    // than FLUSH_PTS + CROWD_RUN points, and a crowded cell's no more than CROWD_RUN
    // besides what came before it.  (Splitting ordinary rounds at FLUSH_PTS instead
    // makes the lanes of a warp diverge where one of them crosses it.)
    // (The two forms below differ only in where the ordinary round's flush check sits;
    // each measured fastest for its mode.)
    const bool crowded = mine > CROWD_RUN;
    int left = mine;
    if constexpr (PAIR) {
      do {
        const int nproc = crowded ? min(left, CROWD_RUN) : left;
        walk(nproc);
        left -= nproc;
        if (crowded) {
          flush();
          since = 0;
        }
      } while (left > 0);
      if (!crowded) {
        since += mine;
        if (since >= FLUSH_PTS) {
          flush();
          since = 0;
        }
      }
    } else {
      do {
        const int nproc = crowded ? min(left, CROWD_RUN) : left;
        walk(nproc);
        left -= nproc;
        since += nproc;
        if (since >= FLUSH_PTS || crowded) {
          flush();
          since = 0;
        }
      } while (left > 0);
    }
    if (owns) {
      // this cell's lists are done (both lanes of a pair read them before their loop);
      // the next round's linking starts after its first barrier
      if constexpr (PAIR) __syncwarp(pmask);
      if (ch == 0) {
        head[cell] = 0xFFFF;
        ccount[cell] = 0;
        xcnt[cell] = 0;
      }
    }
  }
  // flush the register window into the fp64 grid
  if (owns && since > 0) flush();
}

using KFn = void (*)(AccArgs);

template <bool PAIR, typename R>
KFn pick2d(int w) {
  switch (w) {
    case 4: return k_bin_accumulate<4, PAIR, R>;
    case 5: return k_bin_accumulate<5, PAIR, R>;
    case 6: return k_bin_accumulate<6, PAIR, R>;
    case 7: return k_bin_accumulate<7, PAIR, R>;
    case 8: return k_bin_accumulate<8, PAIR, R>;
    default: return nullptr;
  }
}

}  // namespace

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

// Owners.  Pair mode by default, when the cells fill between one and two waves of
// 16-warp owners: one wave (one per SM) of Cfg::CELLS cells, then owners of 3/4 of
// that (12 warps), so that each wave keeps the four schedulers of an SM equally busy.
// Otherwise (or with an explicit `cells`): uniform owners of at most `cells` cells
// (Cfg::CELLS by default), at least one per SM.
struct OwnerPlan {
  OwnerMap om;
  int G;
};
static OwnerPlan owner_plan(int64_t ncells, bool pair, int sms, int cells = 0) {
  const int cmax = pair ? Cfg<true>::CELLS : Cfg<false>::CELLS;
  OwnerPlan P{};
  if (cells <= 0 && pair && sms > 0) {
    const int cb = cmax, cs = cmax * 3 / 4;
    const int64_t kb = static_cast<int64_t>(sms) * cb;
    if (ncells > kb && ncells <= kb + static_cast<int64_t>(sms) * cs) {
      const int ns = static_cast<int>((ncells - kb + cs - 1) / cs);
      P.om = OwnerMap{sms, cb, cs, owner_magic(cb), owner_magic(cs)};
      P.G = sms + ns;
      return P;
    }
  }
  if (cells <= 0 || cells > cmax) cells = cmax;
  int64_t G = (ncells + cells - 1) / cells;
  if (G < sms) G = sms;
  if (G > ncells) G = ncells;
  const int cpc = static_cast<int>((ncells + G - 1) / G);
  P.om = OwnerMap{static_cast<int>(G), cpc, cpc, owner_magic(cpc), owner_magic(cpc)};
  P.G = static_cast<int>(G);
  return P;
}

bool spread_binned_supported(const EsPlan& p, int n_y, bool with_ones) {
  const int nch = n_y + (with_ones ? 1 : 0);
  if (p.d != 2 || nch < 1 || nch > 2 || n_y > 1 || p.w < 4 || p.w > 8) return false;
  const int sms = sm_count();
  if (sms <= 0) return false;
  const int64_t ncells = static_cast<int64_t>(p.N) * p.N;
  // the owner division (OwnerMap) is exact for cell indices below 2^18
  return ncells <= (1 << 18) && owner_plan(ncells, nch == 2, sms).G <= MAX_G;
}

fk_status spread_binned(const EsPlan& p, int64_t n, const float* x, const float* y, int n_y, bool with_ones,
                        double* grid, unsigned* flags, cudaStream_t st, Scratch& scr, bool autotune) {
  return spread_binned_xy(p, n, x, x + n, 1.0f, y, n_y, with_ones, grid, flags, st, scr, autotune);
}

namespace {

using Scatter1Fn = void (*)(PartArgs);
template <bool REC8, int T>
Scatter1Fn pick_scatter1_t(int per, int* tile) {
  switch (per) {
    case 5: *tile = T * 5; return k_bin_scatter1<5, REC8, T>;
    case 6: *tile = T * 6; return k_bin_scatter1<6, REC8, T>;
    default: *tile = T * 7; return k_bin_scatter1<7, REC8, T>;
  }
}
template <bool REC8>
Scatter1Fn pick_scatter1(int per, bool half, int* tile, int* threads) {
  *threads = half ? S2_THREADS / 2 : S2_THREADS;
  return half ? pick_scatter1_t<REC8, S2_THREADS / 2>(per, tile) : pick_scatter1_t<REC8, S2_THREADS>(per, tile);
}

// one run of the 2-D binned spreader with explicit tunables
fk_status spread_binned_run(const EsPlan& p, int64_t n, const float* x, const float* x1, float s1, const float* y,
                            int n_y, bool with_ones, double* grid, unsigned* flags, cudaStream_t st, Scratch& scr,
                            const BinCfg& cfg) {
  const int nch = n_y + (with_ones ? 1 : 0);
  const bool pair = (nch == 2);
  const int64_t ncells = static_cast<int64_t>(p.N) * p.N;
  const OwnerPlan op = owner_plan(ncells, pair, sm_count(), cfg.cells);
  const int G = op.G;
  if (G > MAX_G) return set_error(FK_EINVAL, "binned spreading: %d owners exceed %d", G, MAX_G);
  const int cpc = op.om.cb;  // the largest owner
  const double c = p.N / (2.0 * M_PI);

  FK_CUDA(cudaMemsetAsync(grid, 0, sizeof(double) * ncells * nch, st));
  if (n == 0) return FK_OK;

  PartArgs P{};
  P.N = p.N;
  P.W = p.w;
  P.G = G;
  P.om = op.om;
  P.n = n;
  P.x = x;
  P.x1 = x1;
  P.s1 = s1;
  P.y = y;
  P.has_y = n_y > 0 ? 1 : 0;
  // one partition block per SM; count and scatter use the same block ranges
  P.nblk = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n + P_TILE - 1) / P_TILE,
                                                                    static_cast<int64_t>(sm_count()) * (cfg.half ? 2 : 1))));
  P.range = ((n + P.nblk - 1) / P.nblk + 3) & ~static_cast<int64_t>(3);
  P.vec_ok = ((reinterpret_cast<uintptr_t>(x) & 15) == 0 && (reinterpret_cast<uintptr_t>(x1) & 15) == 0 &&
              (n & 3) == 0 &&
              (n_y == 0 || (reinterpret_cast<uintptr_t>(y) & 15) == 0))
                 ? 1
                 : 0;
  P.flags = flags;
  P.c_hi = static_cast<float>(c);
  P.c_lo = static_cast<float>(c - static_cast<double>(P.c_hi));
  FK_TRY(scr.alloc(&P.cnt, static_cast<size_t>(P.nblk) * G));
  FK_TRY(scr.alloc(&P.off, static_cast<size_t>(P.nblk) * G));
  FK_TRY(scr.alloc(&P.tot, static_cast<size_t>(G)));
  // one-pass bucket capacity: an owner's mean load (points x its share of the cells)
  // plus 2 % and 4096 records (a uniform sample's counts are within a few standard
  // deviations, sqrt(load), of the mean)
  const int64_t exact_len = n + static_cast<int64_t>(P.nblk) * G * 7;  // + run padding
  auto cap_for = [&](int cells) {
    const int64_t load = static_cast<int64_t>(static_cast<double>(n) * cells / static_cast<double>(ncells)) + 1;
    return (load + load / 50 + 4096 + 7) & ~static_cast<int64_t>(7);
  };
  const int64_t cap = cap_for(op.om.cb), cap_s = cap_for(op.om.cs);
  const int64_t rec_total =
      op.om.nb < G ? op.om.nb * cap + static_cast<int64_t>(G - op.om.nb) * cap_s : static_cast<int64_t>(G) * cap;
  const bool one_pass = P.vec_ok && rec_total < (static_cast<int64_t>(1) << 31);
  FK_TRY(scr.alloc(&P.rec, static_cast<size_t>(one_pass ? std::max<int64_t>(exact_len, rec_total) : exact_len)));
  unsigned* ovf = nullptr;
  if (one_pass) {
    FK_TRY(scr.alloc(&P.fill, static_cast<size_t>(G) + 1));
    ovf = reinterpret_cast<unsigned*>(P.fill + G);
    FK_CUDA(cudaMemsetAsync(P.fill, 0, sizeof(int) * (G + 1), st));
    P.cap = static_cast<int>(cap);
    P.cap_s = static_cast<int>(cap_s);
    P.ovf = ovf;
  }

  AccArgs A{};
  A.N = p.N;
  A.G = G;
  A.om = op.om;
  A.cpc_max = cpc;
  A.ncells = static_cast<int>(ncells);
  A.beta = static_cast<float>(p.beta);
  A.poly = es_poly(p.w, p.beta);
  A.with_ones = with_ones ? 1 : 0;
  A.tot = P.tot;
  A.rec = P.rec;
  A.grid = grid;
  A.flags = flags;
  A.fill = P.fill;
  A.cap = P.cap;
  A.cap_s = P.cap_s;
  A.ovf = ovf;
  A.qmul = cfg.qmul;
  // exact-partition (and strength-carrying) records: Rec16; the one-pass partition of
  // ones only writes Rec8
  const KFn fn = pair ? pick2d<true, Rec16>(p.w) : pick2d<false, Rec16>(p.w);
  if (!fn) return set_error(FK_EINVAL, "binned spreading: w = %d not built", p.w);
  const int threads = pair ? Cfg<true>::THREADS : Cfg<false>::THREADS;
  const size_t sm = acc_layout<Rec16>(cpc).total;
  FK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm)));
  // the one-pass partition writes 8-byte records, with the strengths in a parallel
  // stream when there are any
  const bool rec8 = one_pass;
  const bool spl = n_y > 0;
  KFn fn1 = fn;
  size_t sm_1 = sm;
  if (rec8) {
    fn1 = spl ? (pair ? pick2d<true, Rec8Y>(p.w) : pick2d<false, Rec8Y>(p.w)) : pick2d<false, Rec8>(p.w);
    sm_1 = spl ? acc_layout<Rec8Y>(cpc).total : acc_layout<Rec8>(cpc).total;
    FK_CUDA(cudaFuncSetAttribute(fn1, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm_1)));
    if (spl) {
      // + 4: a round's bulk copy rounds its byte count up to 16 (reads <= 3 floats past)
      FK_TRY(scr.alloc(&P.ybuf, static_cast<size_t>(rec_total) + 4));
      A.ybuf = P.ybuf;
    }
  }
  const size_t sm2 = s2_layout(G).total;
  KernelTimer* kt = kernel_timer();

  if (one_pass) {
    int tile1 = S2_TILE, threads1 = S2_THREADS;
    const Scatter1Fn s1fn = rec8 ? pick_scatter1<true>(cfg.per, cfg.half != 0, &tile1, &threads1)
                                 : pick_scatter1<false>(cfg.per, cfg.half != 0, &tile1, &threads1);
    const size_t sm1 = s2_layout(G, tile1).total;
    FK_CUDA(cudaFuncSetAttribute(s1fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm1)));
    s1fn<<<P.nblk, threads1, sm1, st>>>(P); note_launch();
    FK_CUDA(cudaGetLastError());
    A.mode = 1;
    if (kt->on) cudaEventRecordWithFlags(kt->start, st, kt->rec_flags);
    fn1<<<G, threads, sm_1, st>>>(A); note_launch();
    if (kt->on) {
      cudaEventRecordWithFlags(kt->stop, st, kt->rec_flags);
      kt->recorded = true;
    }
    FK_CUDA(cudaGetLastError());
    // exact partition, run only if a bucket overflowed (each kernel returns at once
    // otherwise); no host round trip either way
    P.guarded = 1;
    A.mode = 2;
  }
  const size_t sm_count_k = sizeof(int) * P_NWARPS * G;
  k_bin_count<<<P.nblk, P_THREADS, sm_count_k, st>>>(P); note_launch();
  FK_CUDA(cudaGetLastError());
  k_bin_scan<<<G, 256, 0, st>>>(P); note_launch();
  FK_CUDA(cudaGetLastError());
  if (P.vec_ok) {
    FK_CUDA(cudaFuncSetAttribute(k_bin_scatter2, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm2)));
    k_bin_scatter2<<<P.nblk, S2_THREADS, sm2, st>>>(P); note_launch();
  } else {
    const size_t sm_scatter = sizeof(uint4) * S_TILE + sizeof(unsigned short) * S_TILE + sizeof(int) * (3 * G + 2);
    FK_CUDA(cudaFuncSetAttribute(k_bin_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm_scatter)));
    k_bin_scatter<<<P.nblk, S_THREADS, sm_scatter, st>>>(P); note_launch();
  }
  FK_CUDA(cudaGetLastError());
  if (!one_pass && kt->on) cudaEventRecordWithFlags(kt->start, st, kt->rec_flags);
  fn<<<G, threads, sm, st>>>(A); note_launch();
  if (!one_pass && kt->on) {
    cudaEventRecordWithFlags(kt->stop, st, kt->rec_flags);
    kt->recorded = true;
  }
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}

}  // namespace

fk_status spread_binned_xy(const EsPlan& p, int64_t n, const float* x, const float* x1, float s1, const float* y,
                           int n_y, bool with_ones, double* grid, unsigned* flags, cudaStream_t st, Scratch& scr,
                           bool autotune) {
  if (!spread_binned_supported(p, n_y, with_ones)) return set_error(FK_EINVAL, "binned spreading: unsupported shape");
  if (n >= (static_cast<int64_t>(1) << 31)) return set_error(FK_EINVAL, "binned spreading: n >= 2^31 per call");
  const int nch = n_y + (with_ones ? 1 : 0);
  int lg = 0;
  while ((static_cast<int64_t>(1) << (lg + 1)) <= n) ++lg;
  const TuneKey key{TUNE_SPREAD2D, p.N, p.w, nch, lg};
  BinCfg cfg;
  if (tune_lookup(key, &cfg)) {
    return spread_binned_run(p, n, x, x1, s1, y, n_y, with_ones, grid, flags, st, scr, cfg);
  }
  if (!autotune || n < (1 << 20)) return spread_binned_run(p, n, x, x1, s1, y, n_y, with_ones, grid, flags, st, scr, cfg);
  // Coordinate search over the tunables, each trial a full run timed with events on
  // this stream; the winner is cached for this (grid, width, channels, size class).
  const bool pair = (nch == 2);
  const int cmax = pair ? Cfg<true>::CELLS : Cfg<false>::CELLS;
  const int64_t ncells = static_cast<int64_t>(p.N) * p.N;
  const int sms = std::max(1, sm_count());
  // cells per owner that give whole waves of owners over the SMs, and the default
  const int waves_cells = static_cast<int>((ncells + 2 * sms - 1) / (2 * sms));
  std::vector<int> cells_opts = {cmax};
  if (waves_cells < cmax) cells_opts.push_back(waves_cells);
  if (cmax * 7 / 8 != waves_cells) cells_opts.push_back(cmax * 7 / 8);
  const std::vector<int> per_opts = {7, 6, 5};
  const std::vector<float> q_opts = {0.5f, 0.25f, 1.0f, 0.125f};
  const std::vector<int> half_opts = {0, 1};
  cudaEvent_t e0, e1;
  FK_CUDA(cudaEventCreate(&e0));
  FK_CUDA(cudaEventCreate(&e1));
  auto trial = [&](const BinCfg& c, float* ms) -> fk_status {
    cudaEventRecord(e0, st);
    {
      Scratch inner(st);
      FK_TRY(spread_binned_run(p, n, x, x1, s1, y, n_y, with_ones, grid, flags, st, inner, c));
    }
    cudaEventRecord(e1, st);
    FK_CUDA(cudaEventSynchronize(e1));
    FK_CUDA(cudaEventElapsedTime(ms, e0, e1));
    return FK_OK;
  };
  BinCfg best;
  float best_ms = 0.f;
  std::string log;
  fk_status rc = trial(best, &best_ms);  // the default (first trial also warms caches)
  if (rc == FK_OK) rc = trial(best, &best_ms);
  char line[160];
  snprintf(line, sizeof(line), "default %.3f ms", best_ms);
  log += line;
  for (int knob = 0; knob < 4 && rc == FK_OK; ++knob) {
    const size_t cnt = knob == 0 ? half_opts.size()
                                 : (knob == 1 ? per_opts.size() : (knob == 2 ? cells_opts.size() : q_opts.size()));
    for (size_t i = 0; i < cnt && rc == FK_OK; ++i) {
      BinCfg c = best;
      if (knob == 0) c.half = half_opts[i];
      if (knob == 1) c.per = per_opts[i];
      if (knob == 2) c.cells = cells_opts[i];
      if (knob == 3) c.qmul = q_opts[i];
      if (c.half == best.half && c.per == best.per && c.cells == best.cells && c.qmul == best.qmul) continue;
      float ms = 0.f;
      rc = trial(c, &ms);
      snprintf(line, sizeof(line), "; half=%d per=%d cells=%d q=%.2f %.3f ms", c.half, c.per, c.cells, c.qmul, ms);
      log += line;
      if (rc == FK_OK && ms < best_ms) {
        best = c;
        best_ms = ms;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  FK_TRY(rc);
  snprintf(line, sizeof(line), "  ->  half=%d per=%d cells=%d q=%.2f (%.3f ms)", best.half, best.per, best.cells,
           best.qmul, best_ms);
  log += line;
  tune_store(key, best, log);
  return spread_binned_run(p, n, x, x1, s1, y, n_y, with_ones, grid, flags, st, scr, best);
}

}  // namespace fk

// ---------------------------------------------------------------- additive-model pairs
// The 2-D transforms of ones at (X_l1, -X_l2), l2 > l1 (Sec. 5, Complexity), grouped by
// their first coordinate l1.  Owners are pairs of grid rows of coordinate l1, so a
// point has the same owner for every partner l2: one partition per l1 sorts the points
// by row owner and writes the row word once plus one code word per partner (RecAdd),
// and one accumulation launch runs the (owner, partner) CTAs of all partners of l1.
// Bucket sizes are exact, counted before the partitions for every coordinate by
// k_add_codes (which also computes each partner coordinate's code words once), so no
// bucket overflows; buckets start at multiples of 4 records for the 16-byte copies.
namespace fk {
namespace {

constexpr int AP_THREADS = 512;               // partition CTA (two per SM)
constexpr int AP_PER = 4;                     // points per thread and tile
constexpr int AP_TILE = AP_THREADS * AP_PER;  // 2048

struct AddPartArgs {
  int N, W, G, P;   // grid nodes per dimension (<= 256), width, row owners (N / 2), partners
  int64_t n;
  const float* xl1;  // coordinate l1 (n floats); partner p is the row xl1 + (1 + p) n
  // precomputed partner code words (k_add_codes): partner p's are the row pre + p n, and
  // the partition takes them instead of the partners' coordinates (null: computes them)
  const unsigned* pre;
  int vec_ok;        // 16-byte aligned rows and n % 4 == 0: bulk copies of the tiles
  int64_t range;     // points per CTA (multiple of 4)
  const int* cnt;    // [G] exact bucket sizes of this l1
  int* fill;         // [G] reservation counters (zeroed)
  unsigned* o1;      // row words, bucketed
  unsigned* code;    // [P][stride] code words, bucketed like o1
  int64_t stride;
  unsigned* flags;
  float c_hi, c_lo;
};

// window of one coordinate on the pair grid: window-start node and the 23-bit offset
// v = (w/2 - f) 2^23 (exact for w >= 4); false outside [-3 pi, 3 pi)
__device__ __forceinline__ bool add_window(float x, const AddPartArgs& A, int* node, unsigned* v) {
  int l0;
  float f;
  if (!window_f32(x, A.N, A.c_hi, A.c_lo, A.W, &l0, &f)) return false;
  *node = wrap_node(l0, A.N);
  *v = static_cast<unsigned>((0.5f * static_cast<float>(A.W) - f) * 8388608.0f);
  return true;
}

// Once per fit, for every coordinate l: the row owners' counts of l (l < d - 1) into
// cnt[l][G], and the code word of -X_l (l >= 1) into codes[l - 1][n], c << 23 | v with
// the window-start column c and v = (w/2 - f) 2^23, or 0xFFFFFFFF for a point out of
// range (flagged).  A partition then adds the row bit (r N << 23) to a partner's code
// word, so each coordinate's window is computed here once instead of once per pair.
struct AddCodeArgs {
  int d, N, W, G;
  int64_t n;
  const float* x;  // [d][n]
  int* cnt;        // [d][G]
  unsigned* codes; // [d - 1][n]
  unsigned* flags;
  float c_hi, c_lo;
};
constexpr int AC_MAXD = 16;
// DMAX: coordinates held at once (d <= DMAX); 8 keeps three 512-thread CTAs per SM
template <int DMAX>
__global__ void __launch_bounds__(512, DMAX <= 8 ? 3 : 2) k_add_codes(AddCodeArgs C) {
  __shared__ int h[AC_MAXD - 1][128];
  AddPartArgs A{};
  A.N = C.N;
  A.W = C.W;
  A.c_hi = C.c_hi;
  A.c_lo = C.c_lo;
  for (int t = threadIdx.x; t < (C.d - 1) * 128; t += blockDim.x) h[t / 128][t % 128] = 0;
  __syncthreads();
  // one coordinate value: its row owner counted (l < d - 1), its code word returned (l >= 1)
  auto one = [&](int l, float xv) -> unsigned {
    int c;
    unsigned v, code = 0xFFFFFFFFu;
    if (l + 1 < C.d) {
      if (add_window(xv, A, &c, &v)) atomicAdd(&h[l][c >> 1], 1);
      else atomicOr(C.flags, FLAG_RANGE);
    }
    if (l >= 1) {
      if (add_window(-xv, A, &c, &v)) code = (static_cast<unsigned>(c) << 23) | v;
      else atomicOr(C.flags, FLAG_RANGE);
    }
    return code;
  };
  // one point per thread (the window arithmetic is latency bound: many warps per SM),
  // every coordinate's load in flight before the arithmetic
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < C.n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float xv[DMAX];
#pragma unroll
    for (int l = 0; l < DMAX; ++l)
      if (l < C.d) xv[l] = __ldg(C.x + static_cast<int64_t>(l) * C.n + i);
#pragma unroll
    for (int l = 0; l < DMAX; ++l) {
      if (l >= C.d) break;
      const unsigned code = one(l, xv[l]);
      if (l >= 1) C.codes[static_cast<int64_t>(l - 1) * C.n + i] = code;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < (C.d - 1) * C.G; t += blockDim.x) {
    const int l = t / C.G, o = t - l * C.G;
    if (h[l][o]) atomicAdd(C.cnt + t, h[l][o]);
  }
}

struct ApLayout {
  size_t stage, srow, scode, base, tcnt, toff, gdelta, bar, total;
};
__host__ __device__ inline ApLayout ap_layout(int P, int G) {
  ApLayout L;
  L.stage = 0;                                                     // float [P + 1][AP_TILE]
  L.srow = L.stage + sizeof(float) * (P + 1) * AP_TILE;            // unsigned [AP_TILE]
  L.scode = L.srow + sizeof(unsigned) * AP_TILE;                   // unsigned [2][AP_TILE]
  L.base = L.scode + sizeof(unsigned) * 2 * AP_TILE;               // int [G]
  L.tcnt = L.base + sizeof(int) * G;                               // int [G + 1]
  L.toff = L.tcnt + sizeof(int) * (G + 1);                         // int [G + 1]
  L.gdelta = (L.toff + sizeof(int) * (G + 1) + 7) & ~static_cast<size_t>(7);  // long long [G]
  L.bar = (L.gdelta + sizeof(long long) * G + 15) & ~static_cast<size_t>(15);  // uint64_t [P + 1]
  L.total = L.bar + sizeof(uint64_t) * (P + 1);
  return L;
}

__global__ void __launch_bounds__(AP_THREADS, 2) k_add_part(AddPartArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int wsum[AP_THREADS / 32];
  const int G = A.G, P = A.P, tid = threadIdx.x;
  const ApLayout L = ap_layout(P, G);
  float* stage = reinterpret_cast<float*>(smem + L.stage);
  unsigned* srow = reinterpret_cast<unsigned*>(smem + L.srow);    // row words in owner order
  unsigned* scode = reinterpret_cast<unsigned*>(smem + L.scode);  // two partners' codes in owner order
  int* base = reinterpret_cast<int*>(smem + L.base);              // bucket starts
  int* tcnt = reinterpret_cast<int*>(smem + L.tcnt);              // tile counts
  int* toff = reinterpret_cast<int*>(smem + L.toff);              // tile run starts
  long long* gdelta = reinterpret_cast<long long*>(smem + L.gdelta);  // bucket slot of tile slot 0
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);     // one per staged row
  // bucket starts: exclusive scan of the counts padded to 4 (G <= blockDim)
  {
    const int lane = tid & 31, warp = tid >> 5;
    const int v = tid < G ? ((__ldg(A.cnt + tid) + 3) & ~3) : 0;
    int incl = v;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, dd);
      if (lane >= dd) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int pre = 0;
    for (int w = 0; w < warp; ++w) pre += wsum[w];
    if (tid < G) base[tid] = pre + incl - v;
  }
  if (tid == 0) {
    for (int q = 0; q <= P; ++q) mbar_init(bar + q);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  for (int o = tid; o <= G; o += AP_THREADS) tcnt[o] = 0;
  __syncthreads();
  const int64_t s0 = static_cast<int64_t>(blockIdx.x) * A.range;
  const int64_t e0 = min(A.n, s0 + A.range);
  // Staged row q (0: coordinate l1, 1 + p: partner p) of the tile at t0 arrives on
  // bar[q].  Each row of the next tile is requested as soon as every thread has passed
  // the barrier after the row's last read in this tile (row 0 after the row words,
  // row 1 + p after partner p's codes), so the loads overlap this tile's work.
  // staged row q: coordinate l1 (q = 0), then partner q - 1's coordinate or code words
  auto row_src = [&](int q) -> const float* {
    if (q > 0 && A.pre) return reinterpret_cast<const float*>(A.pre + static_cast<int64_t>(q - 1) * A.n);
    return A.xl1 + q * A.n;
  };
  auto issue_row = [&](int q, int64_t t) {
    const unsigned bytes = static_cast<unsigned>(min(static_cast<int64_t>(AP_TILE), e0 - t)) * 4u;  // % 16 == 0
    fence_proxy_async();
    mbar_arrive_expect(bar + q, bytes);
    bulk_g2s(stage + q * AP_TILE, row_src(q) + t, bytes, bar + q);
  };
  if (A.vec_ok && tid == 0 && s0 < e0)
    for (int q = 0; q <= P; ++q) issue_row(q, s0);
  unsigned phase = 0;
  // after a wait gave up: wait (bounded) for each row copy still in flight, that of the
  // next tile (parity phase ^ 1) for rows 0 .. last when the next tile was requested,
  // else that of this tile (a phase already complete returns at once)
  auto drain = [&](int last, bool next) {
    for (int q = 0; q <= P; ++q) mbar_drain(bar + q, (next && q <= last) ? (phase ^ 1u) : phase);
  };
  for (int64_t t0 = s0; t0 < e0; t0 += AP_TILE) {
    const int cnt = static_cast<int>(min(static_cast<int64_t>(AP_TILE), e0 - t0));
    const bool next = t0 + AP_TILE < e0;
    // the tile counts were zeroed after their last read of the tile before; with bulk
    // copies each thread waits for the staged rows itself, plain loads need a barrier
    if (A.vec_ok) {
      if (!mbar_wait(bar, phase, A.flags)) {
        drain(-1, next);
        return;
      }
    } else {
      for (int q = 0; q <= P; ++q)
        for (int i = tid; i < cnt; i += AP_THREADS) stage[q * AP_TILE + i] = __ldg(row_src(q) + t0 + i);
      __syncthreads();
    }
    // row word and rank of each point inside its owner's run of the tile
    unsigned w1[AP_PER];
    int rk[AP_PER];
#pragma unroll
    for (int k = 0; k < AP_PER; ++k) {
      const int i = k * AP_THREADS + tid;
      w1[k] = 0xFFFFFFFFu;
      rk[k] = 0;
      if (i < cnt) {
        int c;
        unsigned v;
        if (add_window(stage[i], A, &c, &v)) {
          w1[k] = (static_cast<unsigned>(c) << 24) | v;
          rk[k] = atomicAdd(&tcnt[c >> 1], 1);
        } else {
          atomicOr(A.flags, FLAG_RANGE);
        }
      }
    }
    __syncthreads();
    if (A.vec_ok && tid == 0 && next) issue_row(0, t0 + AP_TILE);
    // bucket room: one global atomic per owner present; exclusive scan of the tile counts
    int my_c = 0, my_pos = 0;
    if (tid < G) {
      my_c = tcnt[tid];
      if (my_c > 0) my_pos = atomicAdd(A.fill + tid, my_c);
    }
    if (tid >= AP_THREADS - 32) {
      const int ln = tid - (AP_THREADS - 32);
      const int per = (G + 1 + 31) / 32;
      const int o0 = ln * per, o1 = min(o0 + per, G + 1);
      int run = 0;
      for (int o = o0; o < o1; ++o) run += (o < G) ? tcnt[o] : 0;
      int incl = run;
#pragma unroll
      for (int dd = 1; dd < 32; dd <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, dd);
        if (ln >= dd) incl += t;
      }
      int acc = incl - run;
      for (int o = o0; o < o1; ++o) {
        toff[o] = acc;
        acc += (o < G) ? tcnt[o] : 0;
      }
    }
    __syncthreads();
    for (int o = tid; o <= G; o += AP_THREADS) tcnt[o] = 0;  // the next tile's counts
    if (tid < G) {
      // the buckets are exact; a reservation beyond one (a count that disagrees with the
      // placement) is reported and its run is not written
      const bool room = my_pos + my_c <= __ldg(A.cnt + tid);
      if (!room) atomicOr(A.flags, FLAG_INTERNAL);
      gdelta[tid] = room ? static_cast<long long>(base[tid]) + my_pos - toff[tid] : NO_ROOM;
    }
    // each point's slot in the tile's owner order, the same for the row word and every
    // partner's code word: looked up once
    int pos[AP_PER];
#pragma unroll
    for (int k = 0; k < AP_PER; ++k) {
      pos[k] = (w1[k] != 0xFFFFFFFFu) ? toff[w1[k] >> 25] + rk[k] : 0;
      if (w1[k] != 0xFFFFFFFFu) srow[pos[k]] = w1[k];
    }
    __syncthreads();
    const int valid = toff[G];
    // bucket index of this thread's tile slots j = k AP_THREADS + tid (or -1), kept in
    // registers for the partners' copies
    long long at[AP_PER];
#pragma unroll
    for (int k = 0; k < AP_PER; ++k) {
      const int j = k * AP_THREADS + tid;
      at[k] = -1;
      if (j < valid) {
        const unsigned w = srow[j];
        const long long gd = gdelta[w >> 25];
        if (gd != NO_ROOM && fk_check(gd + j >= 0 && gd + j < A.stride, A.flags)) {
          at[k] = gd + j;
          A.o1[at[k]] = w;
        }
      }
    }
    // one code stream per partner, in the same order; two code buffers, so that one
    // barrier per partner suffices (a buffer is rewritten two partners later, after
    // every thread has passed the barrier in between)
    for (int p = 0; p < P; ++p) {
      unsigned* sc = scode + (p & 1) * AP_TILE;
      if (A.vec_ok && !mbar_wait(bar + 1 + p, phase, A.flags)) {
        drain(p, next);
        return;
      }
#pragma unroll
      for (int k = 0; k < AP_PER; ++k) {
        if (w1[k] == 0xFFFFFFFFu) continue;
        const int i = k * AP_THREADS + tid;
        int c;
        unsigned v, code = 0u;
        if (A.pre) {
          // precomputed c << 23 | v (out-of-range points were flagged there)
          const unsigned pc = __float_as_uint(stage[(1 + p) * AP_TILE + i]);
          if (pc != 0xFFFFFFFFu) code = pc + ((((w1[k] >> 24) & 1u) * static_cast<unsigned>(A.N)) << 23);
        } else if (add_window(-stage[(1 + p) * AP_TILE + i], A, &c, &v)) {
          code = ((((w1[k] >> 24) & 1u) * static_cast<unsigned>(A.N) + static_cast<unsigned>(c)) << 23) | v;
        } else {
          atomicOr(A.flags, FLAG_RANGE);
        }
        sc[pos[k]] = code;
      }
      __syncthreads();
      if (A.vec_ok && tid == 0 && next) issue_row(1 + p, t0 + AP_TILE);
      unsigned* out = A.code + p * A.stride;
#pragma unroll
      for (int k = 0; k < AP_PER; ++k)
        if (at[k] >= 0) out[at[k]] = sc[k * AP_THREADS + tid];
    }
    __syncthreads();  // the code buffers are free for the next tile
    phase ^= 1u;
  }
}

}  // namespace

bool additive_pairs_supported(const EsPlan& p, int d, int64_t n) {
  return p.d == 2 && p.N >= 16 && p.N <= 256 && p.w >= 4 && p.w <= 8 && d >= 2 && d <= AC_MAXD && n >= 1 &&
         n + 4LL * 256 + 16 < (static_cast<int64_t>(1) << 31) && sm_count() > 0;
}

fk_status additive_pairs_begin(const EsPlan& p, int d, int64_t n, const float* x, unsigned* flags, cudaStream_t st,
                               Scratch& scr, AddPairState* S) {
  if (!additive_pairs_supported(p, d, n)) return set_error(FK_EINTERNAL, "additive pairs: unsupported shape");
  *S = AddPairState{};
  S->p = p;
  S->d = d;
  S->n = n;
  S->x = x;
  S->G = p.N / 2;
  S->stride = (n + 4LL * S->G + 16 + 3) & ~static_cast<int64_t>(3);
  // counts of each coordinate's rows: [d][G]; fill [G]
  FK_TRY(scr.alloc(&S->cnt, (static_cast<size_t>(d) + 1) * S->G));
  for (int s = 0; s < 2 && s < d - 1; ++s) {
    FK_TRY(scr.alloc(&S->o1[s], static_cast<size_t>(S->stride)));
    FK_TRY(scr.alloc(&S->code[s], static_cast<size_t>(S->stride) * (d - 1 - s)));
  }
  FK_TRY(scr.alloc(&S->codes, static_cast<size_t>(n) * (d - 1)));
  FK_CUDA(cudaMemsetAsync(S->cnt, 0, sizeof(int) * (d + 1) * S->G, st));
  AddCodeArgs C{};
  const CoordConst cc = coord_const(p.N);
  C.d = d;
  C.N = p.N;
  C.W = p.w;
  C.G = S->G;
  C.n = n;
  C.x = x;
  C.cnt = S->cnt;
  C.codes = S->codes;
  C.flags = flags;
  C.c_hi = cc.hi;
  C.c_lo = cc.lo;
  if (d <= 8) k_add_codes<8><<<grid_for(n, 512, 6 * sm_count()), 512, 0, st>>>(C);
  else k_add_codes<AC_MAXD><<<grid_for(n, 512, 4 * sm_count()), 512, 0, st>>>(C);
  note_launch();
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}

fk_status additive_pairs_part(AddPairState& S, int l1, unsigned* flags, cudaStream_t st) {
  const EsPlan& p = S.p;
  const int G = S.G, P = S.d - 1 - l1, N = p.N;
  if (P < 1) return FK_OK;
  int* cnt = S.cnt + l1 * G;
  int* fill = S.cnt + S.d * G;
  const int sms = sm_count();
  FK_CUDA(cudaMemsetAsync(fill, 0, sizeof(int) * G, st));
  AddPartArgs A{};
  const CoordConst cc = coord_const(N);
  A.N = N;
  A.W = p.w;
  A.G = G;
  A.P = P;
  A.n = S.n;
  A.xl1 = S.x + static_cast<int64_t>(l1) * S.n;
  A.vec_ok = ((reinterpret_cast<uintptr_t>(S.x) & 15) == 0 && (S.n & 3) == 0) ? 1 : 0;
  const int nblk = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((S.n + AP_TILE - 1) / AP_TILE, 2LL * sms)));
  A.range = ((S.n + nblk - 1) / nblk + 3) & ~static_cast<int64_t>(3);
  A.cnt = cnt;
  A.fill = fill;
  A.pre = S.codes + static_cast<int64_t>(l1) * S.n;  // partner p = coordinate l1 + 1 + p
  A.o1 = S.o1[l1 & 1];
  A.code = S.code[l1 & 1];
  A.stride = S.stride;
  A.flags = flags;
  A.c_hi = cc.hi;
  A.c_lo = cc.lo;
  const size_t sm_part = ap_layout(P, G).total;
  FK_CUDA(cudaFuncSetAttribute(k_add_part, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm_part)));
  k_add_part<<<nblk, AP_THREADS, sm_part, st>>>(A); note_launch();
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}

fk_status additive_pairs_acc(AddPairState& S, int l1, double* grids, unsigned* flags, cudaStream_t st) {
  const EsPlan& p = S.p;
  const int G = S.G, P = S.d - 1 - l1, N = p.N;
  if (P < 1) return FK_OK;
  // accumulation: CTA (owner b, partner sub), owners of two rows (2N cells, one lane each)
  FK_CUDA(cudaMemsetAsync(grids, 0, sizeof(double) * N * N * P, st));
  AccArgs B{};
  B.N = N;
  B.G = G;
  B.om = OwnerMap{G, 2 * N, 2 * N, owner_magic(2 * N), owner_magic(2 * N)};
  B.cpc_max = 2 * N;
  B.ncells = N * N;
  B.beta = static_cast<float>(p.beta);
  B.poly = es_poly(p.w, p.beta);
  B.with_ones = 1;
  B.tot = S.cnt + l1 * G;
  B.rec = reinterpret_cast<const uint4*>(S.code[l1 & 1]);
  B.ybuf = reinterpret_cast<const float*>(S.o1[l1 & 1]);
  B.grid = grids;
  B.flags = flags;
  B.mode = 0;
  B.qmul = 0.5f;
  B.nsub = P;
  B.sub_rec_stride = S.stride;
  B.sub_grid_stride = static_cast<int64_t>(N) * N;
  B.pad4 = 1;
  const KFn fn = pick2d<false, RecAdd>(p.w);
  if (!fn) return set_error(FK_EINVAL, "additive pairs: w = %d not built", p.w);
  const size_t sm_acc = acc_layout<RecAdd>(2 * N).total;
  FK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm_acc)));
  KernelTimer* kt = kernel_timer();
  if (kt->on) cudaEventRecordWithFlags(kt->start, st, kt->rec_flags);
  fn<<<G * P, RecAdd::NP_THREADS, sm_acc, st>>>(B); note_launch();
  if (kt->on) {
    cudaEventRecordWithFlags(kt->stop, st, kt->rec_flags);
    kt->recorded = true;
  }
  FK_CUDA(cudaGetLastError());
  return FK_OK;
}

}  // namespace fk
