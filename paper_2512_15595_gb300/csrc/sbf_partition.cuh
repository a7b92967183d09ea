// L2-blocked construction for filters larger than L2.
//
// The direct construction kernel issues one random read-modify-write per key
// into HBM; its throughput is the number of atomic requests an SM keeps in
// flight divided by the DRAM-miss latency.  Here the keys are first hashed
// and radix-partitioned by filter slice (a slice is a power-of-two run of
// blocks sized to sit in L2), then each slice's atomic ORs are applied while
// the slice is L2-resident.  The set bits are the same as the direct
// kernel's: every key still ORs its own pattern into its own block (Sec. II-A);
// only the order of the ORs changes, and OR is commutative and idempotent.
//
//   sbf_partition_kernel: key -> XXH64 -> block j -> record (j << 32 | h_lo),
//     CTA-local counting sort by slice (j >> shift), one global atomic per
//     (tile, slice) to reserve space, coalesced record stores.  A record whose
//     slice buffer is full is inserted on the spot with direct atomics, so no
//     key distribution can lose a key.
//   sbf_add_records_kernel: the cooperative-group insert of sbf_add_kernel,
//     reading records slice by slice instead of keys (no hashing).
#pragma once

#include "sbf_kernels.cuh"

namespace bloomgb {

// OR a record's pattern into its block with one thread (Theta = 1, Phi = s):
// the overflow path of the partition kernel.
template <int B, int S, int K, int SALTS>
__device__ __forceinline__ void insert_one(typename WordOf<S>::type* filter, uint64_t blk, uint32_t hlo,
                                           uint64_t pol) {
  using C = Cfg<B, S, K, 1, B / S, 1, SALTS>;
  using W = typename C::word_t;
  W* bp = filter + blk * C::s;
  static_for<C::s>([&](auto w) {
    constexpr int Wd = decltype(w)::value;
    W pat = 0;
    static_for<C::kp>([&](auto t) { pat |= pattern_bit(hlo, salt_at<S, SALTS>(Wd + C::s * decltype(t)::value)); });
    red_or(bp + Wd, pat, pol);
  });
}

// Look a record up with one thread (Theta = 1, Phi = s): the overflow path of
// the lookup flavour of the partition kernel.
template <int B, int S, int K, int SALTS>
__device__ __forceinline__ bool lookup_one(const typename WordOf<S>::type* filter, uint64_t blk, uint32_t hlo,
                                           uint64_t pol) {
  using C = Cfg<B, S, K, 1, B / S, 1, SALTS>;
  using W = typename C::word_t;
  W data[C::s];
  ld_words<C::s>(filter + blk * C::s, pol, data);
  W miss = 0;
  static_for<C::s>([&](auto w) {
    constexpr int Wd = decltype(w)::value;
    W pat = 0;
    static_for<C::kp>([&](auto t) { pat |= pattern_bit(hlo, salt_at<S, SALTS>(Wd + C::s * decltype(t)::value)); });
    miss |= pat & ~data[Wd];
  });
  return miss == 0;
}

// LOOKUP = false: construction records.  LOOKUP = true: lookup records, each
// with the index of its query in `idx`; a query whose slice buffer is full is
// answered on the spot (its result bit is set if it is found).
template <int B, int S, int K, bool LOOKUP, int SALTS = 0>
__global__ void __launch_bounds__(kPartThreads, LOOKUP ? 3 : 4) sbf_partition_kernel(const PartArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* tile_rec = reinterpret_cast<uint64_t*>(smem);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(tile_rec + kPartTile);
  uint32_t* start = cnt + a.nparts;
  // per slice: reserved global position minus the slice's first position in
  // the tile (modulo 2^64), so that sorted position i goes to off[p] + i
  unsigned long long* off = reinterpret_cast<unsigned long long*>(start + a.nparts);
  uint32_t* warp_sum = reinterpret_cast<uint32_t*>(off + a.nparts);
  uint32_t* tile_idx = warp_sum + 64;  // lookup only (kPartTile entries)

  using W = typename WordOf<S>::type;
  const uint64_t pol_keys = policy_evict_first();
  const uint64_t pol_filter = policy_evict_normal();
  const uint32_t tid = threadIdx.x;
  const uint64_t ntiles = (a.n + kPartTile - 1) / kPartTile;

  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t base = tile * kPartTile;
    const uint32_t tile_n = static_cast<uint32_t>(a.n - base < kPartTile ? a.n - base : kPartTile);
    for (uint32_t p = tid; p < a.nparts; p += kPartThreads) cnt[p] = 0;
    __syncthreads();

    // key i of the tile is handled by thread i % kPartThreads; all loads are
    // issued before any hashing so that their latencies overlap
    uint64_t rec[kPartKeysPerThread];
#pragma unroll
    for (int u = 0; u < kPartKeysPerThread; ++u) {
      const uint32_t i = u * kPartThreads + tid;
      rec[u] = i < tile_n ? ld_key1(a.keys + base + i, pol_keys) : 0;
    }
    // hash, count; pr = slice << 12 | rank within the tile's slice run
    uint32_t pr[kPartKeysPerThread];
#pragma unroll
    for (int u = 0; u < kPartKeysPerThread; ++u) {
      pr[u] = 0xFFFFFFFFu;
      if (u * kPartThreads + tid < tile_n) {
        const uint64_t h = xxh64_key(rec[u], a.acc0);
        const uint64_t j = block_of(h, a.nblocks, a.block_mode);
        rec[u] = (j << 32) | static_cast<uint32_t>(h);
        const uint32_t part = static_cast<uint32_t>(j >> a.shift);
        pr[u] = (part << 12) | atomicAdd(&cnt[part], 1u);
      }
    }
    __syncthreads();

    // exclusive scan of the per-slice counts (nparts <= 1024, two per thread)
    {
      const uint32_t p0 = 2 * tid, p1 = 2 * tid + 1;
      const uint32_t c0 = p0 < a.nparts ? cnt[p0] : 0, c1 = p1 < a.nparts ? cnt[p1] : 0;
      uint32_t incl = c0 + c1;
      const uint32_t lane = tid & 31u, warp = tid >> 5;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t v = __shfl_up_sync(kFullMask, incl, d);
        if (lane >= static_cast<uint32_t>(d)) incl += v;
      }
      if (lane == 31) warp_sum[warp] = incl;
      __syncthreads();
      if (warp == 0) {
        uint32_t ws = lane < kPartThreads / 32 ? warp_sum[lane] : 0;
        uint32_t wi = ws;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t v = __shfl_up_sync(kFullMask, wi, d);
          if (lane >= static_cast<uint32_t>(d)) wi += v;
        }
        if (lane < kPartThreads / 32) warp_sum[lane] = wi - ws;  // exclusive
      }
      __syncthreads();
      const uint32_t excl = incl - (c0 + c1) + warp_sum[warp];
      if (p0 < a.nparts) start[p0] = excl;
      if (p1 < a.nparts) start[p1] = excl + c0;
    }
    __syncthreads();

    // reserve space in each slice's buffer, and scatter into shared memory
    for (uint32_t p = tid; p < a.nparts; p += kPartThreads)
      off[p] = (cnt[p] ? atomicAdd(a.counts + p, static_cast<unsigned long long>(cnt[p])) : 0ull) -
               static_cast<unsigned long long>(start[p]);
#pragma unroll
    for (int u = 0; u < kPartKeysPerThread; ++u) {
      if (pr[u] != 0xFFFFFFFFu) {
        const uint32_t part = pr[u] >> 12;
        const uint32_t pos = start[part] + (pr[u] & 0xFFFu);
        tile_rec[pos] = rec[u];
        if constexpr (LOOKUP) tile_idx[pos] = static_cast<uint32_t>(base) + u * kPartThreads + tid;
      }
    }
    __syncthreads();

    // coalesced write-out: consecutive positions of one slice go to
    // consecutive addresses of that slice's buffer (the slice is read back
    // from the record's block index)
    for (uint32_t i = tid; i < tile_n; i += kPartThreads) {
      const uint64_t r = tile_rec[i];
      const uint32_t p = static_cast<uint32_t>((r >> 32) >> a.shift);
      const uint64_t dst = off[p] + i;
      if constexpr (LOOKUP) {
        const uint32_t q = tile_idx[i];
        if (dst < a.cap) {
          a.records[static_cast<uint64_t>(p) * a.cap + dst] = r;
          a.idx[static_cast<uint64_t>(p) * a.cap + dst] = q;
        } else if (lookup_one<B, S, K, SALTS>(static_cast<const W*>(a.filter), r >> 32, static_cast<uint32_t>(r),
                                       pol_filter)) {
          atomicOr(a.bitmap + (q >> 5), 1u << (q & 31u));
        }
      } else {
        if (dst < a.cap) {
          a.records[static_cast<uint64_t>(p) * a.cap + dst] = r;
        } else {
          insert_one<B, S, K, SALTS>(static_cast<W*>(a.filter), r >> 32, static_cast<uint32_t>(r), pol_filter);
        }
      }
    }
    __syncthreads();
  }
}

// Insert the records of slices [part_lo, part_hi): record v of the virtual
// range [part_lo * cap, part_hi * cap) is slot v % cap of slice v / cap, valid
// below that slice's count.  cap is a multiple of the tile (32 * KPT), so a
// tile lies in one slice.
template <class C>
__global__ void __launch_bounds__(kMaxBlockThreads) sbf_add_records_kernel(const RecArgs a) {
  using W = typename C::word_t;
  constexpr int KPT = C::KPT, THETA = C::THETA, PHI = C::PHI, STEPS = C::steps;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t r = lane & (THETA - 1);
  const LaneSalts<C> salts(r);
  const uint64_t pol_rec = policy_evict_first();
  const uint64_t pol_filter = (a.flags & kHintFilterEvictLast) ? policy_evict_last() : policy_evict_normal();
  W* __restrict__ filter = static_cast<W*>(a.filter);
  constexpr uint64_t kTile = 32u * KPT;
  const uint64_t first_tile = static_cast<uint64_t>(a.part_lo) * a.cap / kTile;
  const uint64_t ntiles = static_cast<uint64_t>(a.part_hi) * a.cap / kTile;
  const uint64_t warps_per_cta = blockDim.x >> 5;
  const uint64_t nwarps = static_cast<uint64_t>(gridDim.x) * warps_per_cta;

  for (uint64_t tile = first_tile + blockIdx.x * warps_per_cta + (threadIdx.x >> 5); tile < ntiles;
       tile += nwarps) {
    const uint64_t v0 = tile * kTile;
    const uint64_t p = v0 / a.cap;
    const uint64_t slot0 = v0 - p * a.cap;
    const uint64_t count = a.counts[p];
    if (slot0 >= count) continue;  // the whole tile is past this slice's records (warp-uniform)
    const uint64_t base = slot0 + static_cast<uint64_t>(lane) * KPT;
    const uint64_t lim = count < a.cap ? count : a.cap;
    uint64_t rec[KPT];
    const uint32_t valid = load_keys<KPT>(a.records + p * a.cap, lim, base, true, pol_rec, rec);
#pragma unroll
    for (int u = 0; u < KPT; ++u) {
#pragma unroll
      for (int m = 0; m < THETA; ++m) {
        uint64_t rm = rec[u];
        uint32_t vm = valid;
        if constexpr (THETA > 1) {
          rm = __shfl_sync(kFullMask, rm, m, THETA);
          vm = __shfl_sync(kFullMask, vm, m, THETA);
        }
        if ((vm >> u) & 1u) {
          const uint32_t hm = static_cast<uint32_t>(rm);
          W* bp = filter + (rm >> 32) * C::s + r * PHI;
#pragma unroll
          for (int q = 0; q < STEPS; ++q) red_lane_words<C>(bp + q * C::chunk, salts, hm, q, pol_filter);
        }
      }
    }
  }
}

// Probe the records of slices [part_lo, part_hi) (lookup, slice-partitioned):
// the same cooperative-group test as sbf_contains_kernel, on records (no
// hashing) whose block lies in an L2-resident window of the filter; the
// owning lane of a found query sets the query's bit in the result bitmap
// (the bitmap starts zeroed, so only positives write).
template <class C>
__global__ void __launch_bounds__(kMaxBlockThreads) sbf_probe_records_kernel(const ProbeArgs a) {
  using W = typename C::word_t;
  constexpr int KPT = C::KPT, THETA = C::THETA, PHI = C::PHI, STEPS = C::steps;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t r = lane & (THETA - 1);
  const uint32_t g0 = lane - r;
  const LaneSalts<C> salts(r);
  const uint64_t pol_rec = policy_evict_first();
  const uint64_t pol_filter = (a.flags & kHintFilterEvictLast) ? policy_evict_last() : policy_evict_normal();
  const W* __restrict__ filter = static_cast<const W*>(a.filter);
  constexpr uint64_t kTile = 32u * KPT;
  const uint64_t first_tile = static_cast<uint64_t>(a.part_lo) * a.cap / kTile;
  const uint64_t ntiles = static_cast<uint64_t>(a.part_hi) * a.cap / kTile;
  const uint64_t warps_per_cta = blockDim.x >> 5;
  const uint64_t nwarps = static_cast<uint64_t>(gridDim.x) * warps_per_cta;

  for (uint64_t tile = first_tile + blockIdx.x * warps_per_cta + (threadIdx.x >> 5); tile < ntiles;
       tile += nwarps) {
    const uint64_t v0 = tile * kTile;
    const uint64_t p = v0 / a.cap;
    const uint64_t slot0 = v0 - p * a.cap;
    const uint64_t count = a.counts[p];
    if (slot0 >= count) continue;  // warp-uniform
    const uint64_t base = slot0 + static_cast<uint64_t>(lane) * KPT;
    const uint64_t lim = count < a.cap ? count : a.cap;
    uint64_t rec[KPT];
    const uint32_t valid = load_keys<KPT>(a.records + p * a.cap, lim, base, true, pol_rec, rec);
    uint32_t q[KPT];
#pragma unroll
    for (int u = 0; u < KPT; ++u) q[u] = ((valid >> u) & 1u) ? a.idx[p * a.cap + base + u] : 0u;
    W data[KPT][THETA][STEPS][PHI];
    uint32_t hk[KPT][THETA];
#pragma unroll
    for (int u = 0; u < KPT; ++u) {
#pragma unroll
      for (int m = 0; m < THETA; ++m) {
        uint64_t rm = ((valid >> u) & 1u) ? rec[u] : 0ull;  // invalid slots read block 0
        if constexpr (THETA > 1) rm = __shfl_sync(kFullMask, rm, m, THETA);
        hk[u][m] = static_cast<uint32_t>(rm);
        const W* bp = filter + (rm >> 32) * C::s + r * PHI;
#pragma unroll
        for (int qq = 0; qq < STEPS; ++qq) ld_words<PHI>(bp + qq * C::chunk, pol_filter, data[u][m][qq]);
      }
    }
#pragma unroll
    for (int u = 0; u < KPT; ++u) {
#pragma unroll
      for (int m = 0; m < THETA; ++m) {
        W miss = 0;
#pragma unroll
        for (int qq = 0; qq < STEPS; ++qq) {
#pragma unroll
          for (int pp = 0; pp < PHI; ++pp) miss |= salts.pattern(hk[u][m], qq, pp) & ~data[u][m][qq][pp];
        }
        bool ok = (miss == 0);
        if constexpr (THETA > 1) {
          const uint32_t seg = (__ballot_sync(kFullMask, ok) >> g0) & ((1u << THETA) - 1u);
          ok = (seg == (1u << THETA) - 1u) && (r == static_cast<uint32_t>(m));
        }
        if (ok && ((valid >> u) & 1u)) atomicOr(a.bitmap + (q[u] >> 5), 1u << (q[u] & 31u));
      }
    }
  }
}

}  // namespace bloomgb
