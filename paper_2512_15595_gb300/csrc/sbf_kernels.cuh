// Bulk construction and lookup kernels of the sectorized blocked Bloom filter.
//
// One template per operation, specialised at compile time on the geometry
// (B block bits, S word bits, K pattern bits) and on the execution layout
// (THETA threads per key, PHI words per thread per step, KPT keys per thread),
// as Sec. IV-A/IV-B prescribe (salts and word offsets become literals).
//
// Work mapping (Sec. IV-C, work-efficient cooperation): a warp takes a tile of
// 32*KPT consecutive keys, lane L owning keys [L*KPT, L*KPT+KPT).  Every lane
// hashes its own keys once; each cooperative group (CG) of THETA lanes then
// walks over its members' keys, receiving hash and block index by register
// shuffles, and touches the key's block together: lane r of the CG handles
// words q*THETA*PHI + r*PHI + [0, PHI) in step q.  Lookup results stay in the
// owning lane and are written back as one packed store per lane.
#pragma once

#include <cstdint>
#include <vector>

#include "registry.h"
#include "sbf_device.cuh"

namespace bloomgb {

enum : uint32_t { kHintFilterEvictLast = 1u << 0, kHintKeysEvictNormal = 1u << 1, kHintWarpAggregate = 1u << 3 };

// SALTS_: the salt set (0: SplitMix64 tables; 1: the Parquet split-block
// multipliers, valid for B = 256, S = 32, K = 8 only)
template <int B_, int S_, int K_, int THETA_, int PHI_, int KPT_, int SALTS_ = 0>
struct Cfg {
  static constexpr int B = B_, S = S_, K = K_, THETA = THETA_, PHI = PHI_, KPT = KPT_, SALTS = SALTS_;
  using word_t = typename WordOf<S>::type;
  static constexpr int s = B / S;            // words per block
  static constexpr int kp = K / s;           // pattern bits per word
  static constexpr int chunk = THETA * PHI;  // words the CG covers per step
  static constexpr int steps = s / chunk;    // steps per block
  static_assert(s >= 1 && B % S == 0, "geometry");
  static_assert(K % s == 0 && K >= s && K <= kMaxSalts, "SBF needs s | K");
  static_assert(THETA >= 1 && THETA <= 32 && (THETA & (THETA - 1)) == 0, "THETA");
  static_assert(PHI >= 1 && (PHI & (PHI - 1)) == 0 && chunk <= s, "PHI");
  static_assert(KPT == 1 || KPT == 2 || KPT == 4, "KPT");
  static_assert(SALTS == 0 || (SALTS == 1 && B == 256 && S == 32 && K == 8), "salt set");
};

constexpr unsigned kFullMask = 0xFFFFFFFFu;

template <class C>
using W_of = typename C::word_t;

constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x / 2); }
// CTA size bound the kernels are compiled for (leaves up to 128 registers per thread)
constexpr int kMaxBlockThreads = 512;

// Per-lane multipliers: salt index of (step q, word p, bit t) for CG rank r is
// q*chunk + r*PHI + p + s*t.  For THETA == 1 these fold to literals.
template <class C>
struct LaneSalts {
  typename C::word_t v[C::steps][C::PHI][C::kp];
  __device__ __forceinline__ explicit LaneSalts(uint32_t r) {
    static_for<C::steps>([&](auto q) {
      static_for<C::PHI>([&](auto p) {
        static_for<C::kp>([&](auto t) {
          constexpr int Q = decltype(q)::value, P = decltype(p)::value, T = decltype(t)::value;
          v[Q][P][T] = salt_select<C::S, Q * C::chunk + P + C::s * T, C::PHI, C::THETA, C::SALTS>(r);
        });
      });
    });
  }
  __device__ __forceinline__ typename C::word_t pattern(uint32_t hlo, int q, int p) const {
    typename C::word_t pat = 0;
#pragma unroll
    for (int t = 0; t < C::kp; ++t) pat |= pattern_bit(hlo, v[q][p][t]);
    return pat;
  }
  // 1 if word w has every pattern bit of (q, p) set.  For 64-bit words each
  // bit is read out of w by a shift (no 64-bit one-hot pattern is built).
  __device__ __forceinline__ uint32_t covers(uint32_t hlo, int q, int p, typename C::word_t w) const {
    if constexpr (C::S == 64) {
      uint32_t all = 1u;
#pragma unroll
      for (int t = 0; t < C::kp; ++t) all &= static_cast<uint32_t>(w >> pattern_pos(hlo, v[q][p][t]));
      return all & 1u;
    } else {
      const typename C::word_t pat = pattern(hlo, q, p);
      return (w & pat) == pat;
    }
  }
};

// OR one lane's PHI consecutive pattern words of step q into the filter at
// `bp` (the lane's first word of the step).  For 32-bit words and an even PHI,
// neighbouring words are merged into one 64-bit red (bits of word 2i in the
// low half, word 2i+1 in the high half: the same bits, half the red
// instructions through L1); word addresses are then 8-byte aligned because
// block starts, steps and lane offsets are all even.
template <class C>
__device__ __forceinline__ void red_lane_words(typename C::word_t* bp, const LaneSalts<C>& salts, uint32_t hlo,
                                               int q, uint64_t pol) {
  if constexpr (C::S == 32 && C::PHI % 2 == 0) {
    uint64_t* bp64 = reinterpret_cast<uint64_t*>(bp);
#pragma unroll
    for (int p = 0; p < C::PHI / 2; ++p) {
      const uint64_t v = static_cast<uint64_t>(salts.pattern(hlo, q, 2 * p)) |
                         (static_cast<uint64_t>(salts.pattern(hlo, q, 2 * p + 1)) << 32);
      red_or(bp64 + p, v, pol);
    }
  } else {
#pragma unroll
    for (int p = 0; p < C::PHI; ++p) red_or(bp + p, salts.pattern(hlo, q, p), pol);
  }
}

// Warp aggregation of construction updates (kHintWarpAggregate): a key equal
// to the key before it in the warp's tile (the previous key of the same lane,
// or for a lane's first key the previous lane's last) sets exactly the same
// bits, so it is dropped from the valid mask before any atomic; a run of
// repeated keys then costs one update.  Called by all 32 lanes together.
template <int KPT>
__device__ __forceinline__ uint32_t drop_repeats(const uint64_t (&key)[KPT], uint32_t valid) {
  const uint64_t prev = __shfl_up_sync(kFullMask, key[KPT - 1], 1);
  const bool first_lane = (threadIdx.x & 31u) == 0;
  uint32_t rep = 0;
#pragma unroll
  for (int u = 0; u < KPT; ++u) {
    const uint64_t before = u ? key[u - 1] : prev;
    if ((u || !first_lane) && key[u] == before) rep |= 1u << u;
  }
  return valid & ~rep;
}

// Load the lane's KPT keys; returns the validity mask.
template <int KPT>
__device__ __forceinline__ uint32_t load_keys(const uint64_t* keys, uint64_t n, uint64_t base,
                                              bool vec_ok, uint64_t pol, uint64_t (&key)[KPT]) {
  if (vec_ok && base + KPT <= n) {
    if constexpr (KPT == 1) key[0] = ld_key1(keys + base, pol);
    else if constexpr (KPT == 2) ld_key2(keys + base, pol, key);
    else ld_key4(keys + base, pol, key);
    return (1u << KPT) - 1u;
  }
  uint32_t valid = 0;
#pragma unroll
  for (int u = 0; u < KPT; ++u) {
    key[u] = 0;
    if (base + u < n) {
      key[u] = ld_key1(keys + base + u, pol);
      valid |= 1u << u;
    }
  }
  return valid;
}

// Everything a tile needs that does not change from tile to tile.
template <class C>
struct TileCtx {
  LaneSalts<C> salts;
  uint32_t lane, r, g0;
  uint64_t pol_keys, pol_filter;
  __device__ __forceinline__ TileCtx(uint32_t flags)
      : salts(threadIdx.x & (C::THETA - 1)),
        lane(threadIdx.x & 31u),
        r(threadIdx.x & (C::THETA - 1)),
        g0((threadIdx.x & 31u) - (threadIdx.x & (C::THETA - 1))),
        pol_keys((flags & kHintKeysEvictNormal) ? policy_evict_normal() : policy_evict_first()),
        pol_filter((flags & kHintFilterEvictLast) ? policy_evict_last() : policy_evict_normal()) {}
};

// Lookup of the warp's tile of 32*KPT keys starting at key `tile_base`
// (lane L owns keys tile_base + L*KPT + [0, KPT)); warp-uniform call.
template <class C>
__device__ __forceinline__ void contains_tile(const TileCtx<C>& t, const typename C::word_t* __restrict__ filter,
                                              uint64_t nblocks, int block_mode, const uint64_t* keys, uint64_t n,
                                              uint8_t* out, uint64_t acc0, bool vec_ok, uint64_t tile_base) {
  using W = typename C::word_t;
  constexpr int KPT = C::KPT, THETA = C::THETA, PHI = C::PHI, STEPS = C::steps;
  const uint64_t base = tile_base + static_cast<uint64_t>(t.lane) * KPT;
  uint64_t key[KPT];
  const uint32_t valid = load_keys<KPT>(keys, n, base, vec_ok, t.pol_keys, key);
  uint32_t hlo[KPT];
  uint64_t blk[KPT];
#pragma unroll
  for (int u = 0; u < KPT; ++u) {
    const uint64_t h = xxh64_key(key[u], acc0);
    hlo[u] = static_cast<uint32_t>(h);
    // invalid (tail) keys read block 0, which always exists; their result is dropped
    blk[u] = ((valid >> u) & 1u) ? block_of(h, nblocks, block_mode) : 0;
  }
  // phase 1: issue every load of the tile before any test (memory-level parallelism)
  W data[KPT][THETA][STEPS][PHI];
  uint32_t hk[KPT][THETA];
#pragma unroll
  for (int u = 0; u < KPT; ++u) {
#pragma unroll
    for (int m = 0; m < THETA; ++m) {
      uint64_t bm = blk[u];
      uint32_t hm = hlo[u];
      if constexpr (THETA > 1) {
        bm = __shfl_sync(kFullMask, bm, m, THETA);
        hm = __shfl_sync(kFullMask, hm, m, THETA);
      }
      hk[u][m] = hm;
      const W* bp = filter + bm * C::s + t.r * PHI;
#pragma unroll
      for (int q = 0; q < STEPS; ++q) ld_words<PHI>(bp + q * C::chunk, t.pol_filter, data[u][m][q]);
    }
  }
  // phase 2: test every word against its pattern; AND across the CG
  uint32_t res = 0;
#pragma unroll
  for (int u = 0; u < KPT; ++u) {
#pragma unroll
    for (int m = 0; m < THETA; ++m) {
      uint32_t all = 1u;
#pragma unroll
      for (int q = 0; q < STEPS; ++q) {
#pragma unroll
        for (int p = 0; p < PHI; ++p) all &= t.salts.covers(hk[u][m], q, p, data[u][m][q][p]);
      }
      bool ok = all != 0;
      if constexpr (THETA > 1) {
        const uint32_t seg = (__ballot_sync(kFullMask, ok) >> t.g0) & ((1u << THETA) - 1u);
        ok = (seg == (1u << THETA) - 1u);
        ok = ok && (t.r == static_cast<uint32_t>(m));
      }
      res |= static_cast<uint32_t>(ok) << u;
    }
  }
  // coalesced write-back of the lane's own results
  if (vec_ok && valid == (1u << KPT) - 1u) {
    if constexpr (KPT == 1) st_out1(out + base, res);
    else if constexpr (KPT == 2) st_out2(out + base, (res & 1u) | ((res & 2u) << 7));
    else st_out4(out + base, (res & 1u) | ((res & 2u) << 7) | ((res & 4u) << 14) | ((res & 8u) << 21));
  } else {
#pragma unroll
    for (int u = 0; u < KPT; ++u)
      if ((valid >> u) & 1u) st_out1(out + base + u, (res >> u) & 1u);
  }
}

// Construction of the warp's tile of 32*KPT keys starting at `tile_base`.
template <class C>
__device__ __forceinline__ void add_tile(const TileCtx<C>& t, typename C::word_t* __restrict__ filter,
                                         uint64_t nblocks, int block_mode, const uint64_t* keys, uint64_t n,
                                         uint64_t acc0, bool vec_ok, uint64_t tile_base, bool agg = false) {
  using W = typename C::word_t;
  constexpr int KPT = C::KPT, THETA = C::THETA, PHI = C::PHI, STEPS = C::steps;
  const uint64_t base = tile_base + static_cast<uint64_t>(t.lane) * KPT;
  uint64_t key[KPT];
  uint32_t valid = load_keys<KPT>(keys, n, base, vec_ok, t.pol_keys, key);
  if (agg) valid = drop_repeats<KPT>(key, valid);
  uint32_t hlo[KPT];
  uint64_t blk[KPT];
#pragma unroll
  for (int u = 0; u < KPT; ++u) {
    const uint64_t h = xxh64_key(key[u], acc0);
    hlo[u] = static_cast<uint32_t>(h);
    blk[u] = block_of(h, nblocks, block_mode);
  }
#pragma unroll
  for (int u = 0; u < KPT; ++u) {
#pragma unroll
    for (int m = 0; m < THETA; ++m) {
      uint64_t bm = blk[u];
      uint32_t hm = hlo[u];
      uint32_t vm = valid;
      if constexpr (THETA > 1) {
        bm = __shfl_sync(kFullMask, bm, m, THETA);
        hm = __shfl_sync(kFullMask, hm, m, THETA);
        vm = __shfl_sync(kFullMask, vm, m, THETA);
      }
      if ((vm >> u) & 1u) {
        // the CG's lanes update neighbouring words of one block in the same
        // instruction, so L1 merges them into one request per sector
        W* bp = filter + bm * C::s + t.r * PHI;
#pragma unroll
        for (int q = 0; q < STEPS; ++q) red_lane_words<C>(bp + q * C::chunk, t.salts, hm, q, t.pol_filter);
      }
    }
  }
}

template <class C>
__global__ void __launch_bounds__(kMaxBlockThreads) sbf_contains_kernel(const SbfArgs a) {
  const TileCtx<C> t(a.flags);
  const W_of<C>* filter = static_cast<const W_of<C>*>(a.filter);
  constexpr uint64_t kTile = 32u * C::KPT;
  const uint64_t ntiles = (a.n + kTile - 1) / kTile;
  const uint64_t warps_per_cta = blockDim.x >> 5;
  const uint64_t nwarps = static_cast<uint64_t>(gridDim.x) * warps_per_cta;
  const bool vec_ok = (reinterpret_cast<uintptr_t>(a.keys) % (8u * C::KPT) == 0) &&
                      (reinterpret_cast<uintptr_t>(a.out) % C::KPT == 0);
  for (uint64_t tile = blockIdx.x * warps_per_cta + (threadIdx.x >> 5); tile < ntiles; tile += nwarps)
    contains_tile<C>(t, filter, a.nblocks, a.block_mode, a.keys, a.n, a.out, a.acc0, vec_ok, tile * kTile);
}

template <class C>
__global__ void __launch_bounds__(kMaxBlockThreads) sbf_add_kernel(const SbfArgs a) {
  const TileCtx<C> t(a.flags);
  W_of<C>* filter = static_cast<W_of<C>*>(a.filter);
  constexpr uint64_t kTile = 32u * C::KPT;
  const uint64_t ntiles = (a.n + kTile - 1) / kTile;
  const uint64_t warps_per_cta = blockDim.x >> 5;
  const uint64_t nwarps = static_cast<uint64_t>(gridDim.x) * warps_per_cta;
  const bool vec_ok = reinterpret_cast<uintptr_t>(a.keys) % (8u * C::KPT) == 0;
  for (uint64_t tile = blockIdx.x * warps_per_cta + (threadIdx.x >> 5); tile < ntiles; tile += nwarps)
    add_tile<C>(t, filter, a.nblocks, a.block_mode, a.keys, a.n, a.acc0, vec_ok, tile * kTile,
                (a.flags & kHintWarpAggregate) != 0);
}

}  // namespace bloomgb
