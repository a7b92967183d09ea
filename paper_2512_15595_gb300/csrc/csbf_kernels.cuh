// Cache-sectorized blocked Bloom filter (CSBF, Sec. II-A): the s words of a
// block form Z groups of g = s/Z neighbouring words; in each group one word
// is selected by another odd multiplier (the top log2(g) bits of h_lo times
// salt[63 - q]) and receives K/Z pattern bits (salt q + Z*t for bit t).
// Only the Z selected words are read or updated, so a 512/1024-bit block
// costs Z sector accesses instead of all of its sectors (Sec. V-B, V-C).
//
// Work mapping as in sbf_kernels.cuh: a warp takes 32*KPT keys, each lane
// hashes its own, a cooperative group of THETA lanes shares (hash, block) by
// shuffles; lane r of the group handles groups q = r + THETA*j.
#pragma once

#include "sbf_kernels.cuh"

namespace bloomgb {

template <int B_, int S_, int K_, int Z_, int THETA_, int KPT_>
struct CCfg {
  static constexpr int B = B_, S = S_, K = K_, Z = Z_, THETA = THETA_, KPT = KPT_;
  using word_t = typename WordOf<S>::type;
  static constexpr int s = B / S;            // words per block
  static constexpr int g = s / Z;            // words per group
  static constexpr int log2g = ilog2c(g);
  static constexpr int kz = K / Z;           // bits in each selected word
  static constexpr int gpl = Z / THETA;      // groups per lane
  static_assert(Z >= 1 && Z < s && s % Z == 0, "1 <= Z < s, Z | s");
  static_assert(K % Z == 0 && K + Z <= kMaxSalts, "Z | K and K + Z <= 64");
  static_assert(THETA >= 1 && Z % THETA == 0, "THETA | Z");
  static_assert(KPT == 1 || KPT == 2 || KPT == 4, "KPT");
};

// Per-lane multipliers: pattern salt of (lane group j, bit t) is
// q + Z*t = THETA*j + Z*t + r; selection salt is 63 - q = 63 - THETA*j - r.
template <class C>
struct CsbfSalts {
  typename C::word_t pat[C::gpl][C::kz];
  typename C::word_t sel[C::gpl];
  __device__ __forceinline__ explicit CsbfSalts(uint32_t r) {
    static_for<C::gpl>([&](auto j) {
      constexpr int J = decltype(j)::value;
      sel[J] = salt_select<C::S, 63 - C::THETA * J, -1, C::THETA>(r);
      static_for<C::kz>([&](auto t) {
        constexpr int T = decltype(t)::value;
        pat[J][T] = salt_select<C::S, C::THETA * J + C::Z * T, 1, C::THETA>(r);
      });
    });
  }
  __device__ __forceinline__ typename C::word_t pattern(uint32_t hlo, int j) const {
    typename C::word_t p = 0;
#pragma unroll
    for (int t = 0; t < C::kz; ++t) p |= pattern_bit(hlo, pat[j][t]);
    return p;
  }
  // 1 if word w has every pattern bit of the lane's j-th group set (64-bit
  // words: each bit read out of w by a shift, no one-hot pattern built)
  __device__ __forceinline__ uint32_t covers(uint32_t hlo, int j, typename C::word_t w) const {
    if constexpr (C::S == 64) {
      uint32_t all = 1u;
#pragma unroll
      for (int t = 0; t < C::kz; ++t) all &= static_cast<uint32_t>(w >> pattern_pos(hlo, pat[j][t]));
      return all & 1u;
    } else {
      const typename C::word_t p = pattern(hlo, j);
      return (w & p) == p;
    }
  }
  // word of the lane's j-th group (group q = r + THETA*j) within the block
  __device__ __forceinline__ uint32_t word(uint32_t hlo, int j, uint32_t r) const {
    const uint32_t q = r + C::THETA * j;
    uint32_t pick = 0;
    if constexpr (C::log2g > 0) {
      if constexpr (C::S == 32) pick = (hlo * static_cast<uint32_t>(sel[j])) >> (32 - C::log2g);
      else pick = static_cast<uint32_t>((static_cast<uint64_t>(hlo) * sel[j]) >> (64 - C::log2g));
    }
    return q * C::g + pick;
  }
};

template <class C>
__global__ void __launch_bounds__(kMaxBlockThreads) csbf_contains_kernel(const SbfArgs a) {
  using W = typename C::word_t;
  constexpr int KPT = C::KPT, THETA = C::THETA, GPL = C::gpl;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t r = lane & (THETA - 1);
  const uint32_t g0 = lane - r;
  const CsbfSalts<C> salts(r);
  const uint64_t pol_keys = (a.flags & kHintKeysEvictNormal) ? policy_evict_normal() : policy_evict_first();
  const uint64_t pol_filter = (a.flags & kHintFilterEvictLast) ? policy_evict_last() : policy_evict_normal();
  const W* __restrict__ filter = static_cast<const W*>(a.filter);
  constexpr uint64_t kTile = 32u * KPT;
  const uint64_t ntiles = (a.n + kTile - 1) / kTile;
  const uint64_t warps_per_cta = blockDim.x >> 5;
  const uint64_t nwarps = static_cast<uint64_t>(gridDim.x) * warps_per_cta;
  const bool vec_ok = (reinterpret_cast<uintptr_t>(a.keys) % (8u * KPT) == 0) &&
                      (reinterpret_cast<uintptr_t>(a.out) % KPT == 0);
  for (uint64_t tile = blockIdx.x * warps_per_cta + (threadIdx.x >> 5); tile < ntiles; tile += nwarps) {
    const uint64_t base = tile * kTile + static_cast<uint64_t>(lane) * KPT;
    uint64_t key[KPT];
    const uint32_t valid = load_keys<KPT>(a.keys, a.n, base, vec_ok, pol_keys, key);
    uint32_t hlo[KPT];
    uint64_t blk[KPT];
#pragma unroll
    for (int u = 0; u < KPT; ++u) {
      const uint64_t h = xxh64_key(key[u], a.acc0);
      hlo[u] = static_cast<uint32_t>(h);
      blk[u] = ((valid >> u) & 1u) ? block_of(h, a.nblocks, a.block_mode) : 0;
    }
    W data[KPT][THETA][GPL];
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
#pragma unroll
        for (int j = 0; j < GPL; ++j) ld_words<1>(filter + bm * C::s + salts.word(hm, j, r), pol_filter, &data[u][m][j]);
      }
    }
    uint32_t res = 0;
#pragma unroll
    for (int u = 0; u < KPT; ++u) {
#pragma unroll
      for (int m = 0; m < THETA; ++m) {
        uint32_t all = 1u;
#pragma unroll
        for (int j = 0; j < GPL; ++j) all &= salts.covers(hk[u][m], j, data[u][m][j]);
        bool ok = all != 0;
        if constexpr (THETA > 1) {
          const uint32_t seg = (__ballot_sync(kFullMask, ok) >> g0) & ((1u << THETA) - 1u);
          ok = (seg == (1u << THETA) - 1u) && (r == static_cast<uint32_t>(m));
        }
        res |= static_cast<uint32_t>(ok) << u;
      }
    }
    if (vec_ok && valid == (1u << KPT) - 1u) {
      if constexpr (KPT == 1) st_out1(a.out + base, res);
      else if constexpr (KPT == 2) st_out2(a.out + base, (res & 1u) | ((res & 2u) << 7));
      else st_out4(a.out + base, (res & 1u) | ((res & 2u) << 7) | ((res & 4u) << 14) | ((res & 8u) << 21));
    } else {
#pragma unroll
      for (int u = 0; u < KPT; ++u)
        if ((valid >> u) & 1u) st_out1(a.out + base + u, (res >> u) & 1u);
    }
  }
}

template <class C>
__global__ void __launch_bounds__(kMaxBlockThreads) csbf_add_kernel(const SbfArgs a) {
  using W = typename C::word_t;
  constexpr int KPT = C::KPT, THETA = C::THETA, GPL = C::gpl;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t r = lane & (THETA - 1);
  const CsbfSalts<C> salts(r);
  const uint64_t pol_keys = (a.flags & kHintKeysEvictNormal) ? policy_evict_normal() : policy_evict_first();
  const uint64_t pol_filter = (a.flags & kHintFilterEvictLast) ? policy_evict_last() : policy_evict_normal();
  W* __restrict__ filter = static_cast<W*>(a.filter);
  constexpr uint64_t kTile = 32u * KPT;
  const uint64_t ntiles = (a.n + kTile - 1) / kTile;
  const uint64_t warps_per_cta = blockDim.x >> 5;
  const uint64_t nwarps = static_cast<uint64_t>(gridDim.x) * warps_per_cta;
  const bool vec_ok = reinterpret_cast<uintptr_t>(a.keys) % (8u * KPT) == 0;
  for (uint64_t tile = blockIdx.x * warps_per_cta + (threadIdx.x >> 5); tile < ntiles; tile += nwarps) {
    const uint64_t base = tile * kTile + static_cast<uint64_t>(lane) * KPT;
    uint64_t key[KPT];
    const uint32_t valid = load_keys<KPT>(a.keys, a.n, base, vec_ok, pol_keys, key);
    uint32_t hlo[KPT];
    uint64_t blk[KPT];
#pragma unroll
    for (int u = 0; u < KPT; ++u) {
      const uint64_t h = xxh64_key(key[u], a.acc0);
      hlo[u] = static_cast<uint32_t>(h);
      blk[u] = block_of(h, a.nblocks, a.block_mode);
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
#pragma unroll
          for (int j = 0; j < GPL; ++j)
            red_or(filter + bm * C::s + salts.word(hm, j, r), salts.pattern(hm, j), pol_filter);
        }
      }
    }
  }
}

}  // namespace bloomgb
