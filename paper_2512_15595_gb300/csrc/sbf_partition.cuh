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
//     key distribution can lose a key.  Few large slices (64 MiB) give long
//     runs per slice and tile, which is what the DRAM writes need.
//   sbf_add_records_kernel: the cooperative-group insert of sbf_add_kernel,
//     reading records slice by slice instead of keys (no hashing).
#pragma once

#include "sbf_kernels.cuh"

namespace bloomgb {

// a failed index check: set its bit in the status word (the access is skipped)
__device__ __forceinline__ void flag_status(uint32_t* status, uint32_t bit) { atomicOr(status, bit); }

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

// One tile of the slice partition (LOOKUP = false: construction records;
// LOOKUP = true: lookup records, each with the index of its query in `idx`).
// On entry key[] holds the tile's keys (loaded during the previous tile); on
// exit it holds the next tile's keys.  Three barriers per tile:
//   hash every key, rank it within its slice (shared-memory counters; two
//     sets that alternate between tiles, so clearing one needs no barrier)
//   B1 -> one warp scans the slice counts into start offsets; the other
//     counter set is cleared
//   B2 -> one global atomic per slice present reserves the slice's run in its
//     buffer; every thread scatters its records into sorted order in shared
//     memory and then loads the next tile's keys into the registers the
//     records left; the reservations become a packed (buffer index, limit)
//     per slice
//   B3 -> coalesced write-out: consecutive sorted positions of one slice go
//     to consecutive slots of that slice's buffer.
// FULL = a tile of exactly TILE keys (every tile but the last): no per-key
// bounds tests.  Indexes derived from data are clamped into their arrays;
// a record whose slice buffer is full takes the direct path (inserted, or
// looked up, on the spot), and one that fails a check is skipped and flagged
// in the status word.
template <int B, int S, int K, bool LOOKUP, int SALTS, int KPTH, bool FULL>
__device__ __forceinline__ void partition_tile(const PartArgs& a, uint64_t (&key)[KPTH], uint32_t it, uint64_t tile,
                                               uint64_t ntiles, uint64_t* trec, unsigned long long* oblim,
                                               uint32_t* cnt, uint32_t* start, uint16_t* tidx, uint64_t pol_keys,
                                               uint64_t pol_filter) {
  constexpr uint32_t TILE = kPartThreads * KPTH;
  constexpr uint64_t kMask48 = (1ull << 48) - 1;
  using W = typename WordOf<S>::type;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t nparts = a.nparts, shift = a.shift;
  const uint64_t base = tile * TILE;
  const uint32_t tile_n = FULL ? TILE : static_cast<uint32_t>(a.n - base);
  uint32_t* c = cnt + (it & 1u) * nparts;
  // block index ((h >> 32) * b) >> 32 for b <= 2^32 (b = bl + 2^32 * bh, bh in {0, 1})
  const uint32_t bl = static_cast<uint32_t>(a.nblocks), bh = static_cast<uint32_t>(a.nblocks >> 32);

  // hash and rank; pr = slice << 13 | rank within the tile's slice run
  uint32_t pr[KPTH];
#pragma unroll
  for (int u = 0; u < KPTH; ++u) {
    const uint64_t h = xxh64_key(key[u], a.acc0);
    const uint32_t hi = static_cast<uint32_t>(h >> 32);
    const uint32_t j = __umulhi(hi, bl) + hi * bh;
    key[u] = (static_cast<uint64_t>(j) << 32) | static_cast<uint32_t>(h);  // the record replaces the key
    const uint32_t part = min(j >> shift, nparts - 1u);
    if (FULL || u * kPartThreads + tid < tile_n) pr[u] = (part << 13) | atomicAdd(&c[part], 1u);
    else pr[u] = 0xFFFFFFFFu;
  }
  __syncthreads();  // B1

  if (warp == 0) {
    // exclusive scan of the counts; lane l owns slices l, l + 32, ... (any
    // slice order is a valid sort order: the runs only need disjoint ranges)
    const uint32_t nq = (nparts + 31u) >> 5;
    uint32_t sum = 0;
    for (uint32_t q = 0; q < nq; ++q) {
      const uint32_t p = q * 32u + lane;
      if (p < nparts) sum += c[p];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t v = __shfl_up_sync(kFullMask, incl, d);
      if (lane >= static_cast<uint32_t>(d)) incl += v;
    }
    uint32_t run = incl - sum;
    for (uint32_t q = 0; q < nq; ++q) {
      const uint32_t p = q * 32u + lane;
      if (p < nparts) {
        const uint32_t v = c[p];
        start[p] = run;
        run += v;
      }
    }
  }
  uint32_t* cn = cnt + ((it + 1u) & 1u) * nparts;  // the next tile's set (its last reader ran before B1)
  for (uint32_t p = tid; p < nparts; p += kPartThreads) cn[p] = 0;
  __syncthreads();  // B2

  const uint32_t c0 = tid < nparts ? c[tid] : 0u;
  const uint32_t c1 = tid + kPartThreads < nparts ? c[tid + kPartThreads] : 0u;
  unsigned long long r0 = 0, r1 = 0;
  if (c0) r0 = atomicAdd(a.counts + tid, static_cast<unsigned long long>(c0));
  if (c1) r1 = atomicAdd(a.counts + tid + kPartThreads, static_cast<unsigned long long>(c1));
#pragma unroll
  for (int u = 0; u < KPTH; ++u) {
    if (FULL || pr[u] != 0xFFFFFFFFu) {
      const uint32_t pos = min(start[pr[u] >> 13] + (pr[u] & 0x1FFFu), TILE - 1u);
      trec[pos] = key[u];
      if constexpr (LOOKUP) tidx[pos] = static_cast<uint16_t>(u * kPartThreads + tid);
    }
  }
  // the next tile's keys go into the registers the records just left
  const uint64_t next = tile + gridDim.x;
  if (next < ntiles) {
    const uint64_t nb = next * TILE;
    const uint64_t* kp = a.keys + nb + tid;
    if (a.n - nb >= TILE) {
#pragma unroll
      for (int u = 0; u < KPTH; ++u) key[u] = ld_key1(kp + u * kPartThreads, pol_keys);
    } else {
      const uint32_t tn = static_cast<uint32_t>(a.n - nb);
#pragma unroll
      for (int u = 0; u < KPTH; ++u)
        key[u] = u * kPartThreads + tid < tn ? ld_key1(kp + u * kPartThreads, pol_keys) : 0ull;
    }
  }
  // per present slice: buffer index of sorted position i is ob + i while i is
  // below the limit (the slots left in the slice buffer); ob mod 2^48 | limit << 48
  auto pack = [&](uint32_t p, uint32_t cp, unsigned long long res) {
    const uint32_t st = start[p];
    const uint64_t avail = a.cap > res ? a.cap - res : 0ull;
    const uint32_t lim = st + static_cast<uint32_t>(avail < cp ? avail : cp);
    const uint64_t ob = (static_cast<uint64_t>(p) * a.cap + res - st) & kMask48;
    oblim[p] = ob | (static_cast<uint64_t>(lim) << 48);
  };
  if (c0) pack(tid, c0, r0);
  if (c1) pack(tid + kPartThreads, c1, r1);
  __syncthreads();  // B3

  // coalesced write-out; the slice is read back from the record's block
  // index.  Records that do not go to their buffer here are handled after
  // the loop (one branch per thread, not per record).
  const uint64_t total = static_cast<uint64_t>(nparts) * a.cap;
  uint32_t slow = 0;
#pragma unroll
  for (int u = 0; u < KPTH; ++u) {
    const uint32_t i = u * kPartThreads + tid;
    if (FULL || i < tile_n) {
      const uint64_t r = trec[i];
      const uint32_t praw = static_cast<uint32_t>(r >> 32) >> shift;
      const unsigned long long pk = oblim[min(praw, nparts - 1u)];
      const uint64_t dst = (pk + i) & kMask48;
      const bool ok = i < static_cast<uint32_t>(pk >> 48) && praw < nparts && dst < total;
      if (ok) {
        st_u64_hint(a.records + dst, r, pol_keys);
        if constexpr (LOOKUP) st_u32_hint(a.idx + dst, static_cast<uint32_t>(base) + tidx[i], pol_keys);
      }
      slow |= static_cast<uint32_t>(!ok) << u;
    }
  }
  if (slow) {
#pragma unroll 1
    for (int u = 0; u < KPTH; ++u) {
      if (!((slow >> u) & 1u)) continue;
      const uint32_t i = u * kPartThreads + tid;
      const uint64_t r = trec[i];
      const uint32_t praw = static_cast<uint32_t>(r >> 32) >> shift;
      if (praw >= nparts || (r >> 32) >= a.nblocks) {
        flag_status(a.status, kStatusRecordSlice);
        continue;
      }
      if (i < static_cast<uint32_t>(oblim[praw] >> 48)) {  // it fit, so its buffer index failed the check
        flag_status(a.status, kStatusBufferIndex);
        continue;
      }
      // the slice buffer is full: the direct method
      if constexpr (LOOKUP) {
        const uint32_t q = static_cast<uint32_t>(base) + tidx[i];
        if (lookup_one<B, S, K, SALTS>(static_cast<const W*>(a.filter), r >> 32, static_cast<uint32_t>(r),
                                       pol_filter))
          atomicOr(a.bitmap + (q >> 5), 1u << (q & 31u));
      } else {
        insert_one<B, S, K, SALTS>(static_cast<W*>(a.filter), r >> 32, static_cast<uint32_t>(r), pol_filter);
      }
    }
  }
}

template <int B, int S, int K, bool LOOKUP, int SALTS = 0>
__global__ void __launch_bounds__(kPartThreads, LOOKUP ? 3 : 4) sbf_partition_kernel(const PartArgs a) {
  constexpr int KPTH = LOOKUP ? kPartKeysLookup : kPartKeysAdd;
  constexpr uint32_t TILE = kPartThreads * KPTH;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* trec = reinterpret_cast<uint64_t*>(smem);                               // [TILE] sorted records
  unsigned long long* oblim = reinterpret_cast<unsigned long long*>(trec + TILE);  // [nparts]
  uint32_t* cnt = reinterpret_cast<uint32_t*>(oblim + a.nparts);                   // [2][nparts]
  uint32_t* start = cnt + 2 * a.nparts;                                            // [nparts]
  uint16_t* tidx = reinterpret_cast<uint16_t*>(start + a.nparts);                  // lookup: [TILE]
  const uint64_t pol_keys = policy_evict_first();
  const uint64_t pol_filter = policy_evict_normal();
  const uint32_t tid = threadIdx.x;
  const uint64_t ntiles = (a.n + TILE - 1) / TILE;
  for (uint32_t p = tid; p < 2 * a.nparts; p += kPartThreads) cnt[p] = 0;
  uint64_t key[KPTH];
  uint64_t tile = blockIdx.x;
  if (tile < ntiles) {
    const uint64_t nb = tile * TILE;
    const uint64_t* kp = a.keys + nb + tid;
    const uint64_t tn = a.n - nb;
#pragma unroll
    for (int u = 0; u < KPTH; ++u)
      key[u] = u * kPartThreads + tid < tn ? ld_key1(kp + u * kPartThreads, pol_keys) : 0ull;
  }
  __syncthreads();
  for (uint32_t it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    if (a.n - tile * TILE >= TILE)
      partition_tile<B, S, K, LOOKUP, SALTS, KPTH, true>(a, key, it, tile, ntiles, trec, oblim, cnt, start, tidx,
                                                         pol_keys, pol_filter);
    else
      partition_tile<B, S, K, LOOKUP, SALTS, KPTH, false>(a, key, it, tile, ntiles, trec, oblim, cnt, start, tidx,
                                                          pol_keys, pol_filter);
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
  const bool agg = (a.flags & kHintWarpAggregate) != 0;
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
    uint32_t valid = load_keys<KPT>(a.records + p * a.cap, lim, base, true, pol_rec, rec);
    if (agg) valid = drop_repeats<KPT>(rec, valid);  // equal records: equal keys
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
        if (((vm >> u) & 1u) && (rm >> 32) >= a.nblocks) {
          flag_status(a.status, kStatusBlockRange);
          vm &= ~(1u << u);
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
        if ((rm >> 32) >= a.nblocks) {  // a record outside the filter reads block 0 instead
          flag_status(a.status, kStatusBlockRange);
          rm &= 0xFFFFFFFFull;
        }
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
        uint32_t all = 1u;
#pragma unroll
        for (int qq = 0; qq < STEPS; ++qq) {
#pragma unroll
          for (int pp = 0; pp < PHI; ++pp) all &= salts.covers(hk[u][m], qq, pp, data[u][m][qq][pp]);
        }
        bool ok = all != 0;
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
