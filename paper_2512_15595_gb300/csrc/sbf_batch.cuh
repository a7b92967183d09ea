// Batched construction and lookup: many independent filters (same geometry
// B, S, K; each its own number of blocks) processed by one launch.  The work
// unit is a chunk of kBatchChunk keys of one filter; a warp finds its chunk's
// filter by binary search over chunk_begin and runs the same per-tile code as
// the single-filter kernels on that filter.  No device-side waits: chunks are
// assigned statically (grid stride), so the launch can be captured into a
// CUDA graph and replayed.
#pragma once

#include "sbf_kernels.cuh"

namespace bloomgb {

__device__ __forceinline__ uint32_t batch_filter_of(const uint64_t* __restrict__ chunk_begin, uint32_t nfilters,
                                                    uint64_t chunk) {
  uint32_t lo = 0, hi = nfilters;  // chunk_begin[lo] <= chunk < chunk_begin[hi] (hi = nfilters: the total)
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(chunk_begin + mid) <= chunk) lo = mid;
    else hi = mid;
  }
  return lo;  // the last filter starting at or before `chunk` (empty filters are skipped)
}

// Bulk-prefetch into L2 the share of chunk c's filter that belongs to chunk c:
// bytes [i*F/n, (i+1)*F/n) of the filter's F bytes for its chunk i of n
// (widened to 128-byte lines, clipped to the bit array).  All chunks of a
// filter together prefetch the whole filter.  A hint: no completion is
// awaited and the bits do not depend on it.
template <class C>
__device__ __forceinline__ void batch_prefetch(const BatchArgs& a, uint64_t c) {
  if (c >= a.total_chunks) return;
  const uint32_t fi = batch_filter_of(a.chunk_begin, a.nfilters, c);
  const uint64_t c0 = __ldg(a.chunk_begin + fi), n = __ldg(a.chunk_begin + fi + 1) - c0;
  const BatchFilter e = a.filters[fi];
  const uint64_t bytes = (e.nblocks * (C::B / 8)) & ~15ull;
  const uint64_t i = c - c0, per = bytes / n;
  const uint64_t lo = (per * i) & ~127ull;
  uint64_t hi = i + 1 == n ? bytes : ((per * (i + 1) + 127) & ~127ull);
  if (hi > bytes) hi = bytes;
  const char* base = static_cast<const char*>(e.words);
  for (uint64_t p = lo; p < hi; p += (1u << 20)) {
    const uint32_t len = static_cast<uint32_t>(hi - p < (1u << 20) ? hi - p : (1u << 20));
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(base + p), "r"(len) : "memory");
  }
}

template <class C, bool ADD>
__global__ void __launch_bounds__(kMaxBlockThreads) sbf_batch_kernel(const BatchArgs a) {
  const TileCtx<C> t(a.flags);
  constexpr uint64_t kTile = 32u * C::KPT;
  static_assert(kBatchChunk % kTile == 0, "chunk must hold whole tiles");
  const uint64_t warps_per_cta = blockDim.x >> 5;
  const uint64_t nwarps = static_cast<uint64_t>(gridDim.x) * warps_per_cta;
  for (uint64_t c = blockIdx.x * warps_per_cta + (threadIdx.x >> 5); c < a.total_chunks; c += nwarps) {
    if (a.prefetch_chunks && (threadIdx.x & 31u) == 0) batch_prefetch<C>(a, c + a.prefetch_chunks);
    const uint32_t fi = batch_filter_of(a.chunk_begin, a.nfilters, c);
    const BatchFilter e = a.filters[fi];
    const uint64_t first = (c - __ldg(a.chunk_begin + fi)) * kBatchChunk;
    const uint64_t* keys = a.keys + e.key_offset;
    const int mode = e.nblocks < (1ull << 32) ? 0 : (e.nblocks == (1ull << 32) ? 1 : 2);
    bool vec_ok = reinterpret_cast<uintptr_t>(keys) % (8u * C::KPT) == 0;
    if constexpr (!ADD) vec_ok = vec_ok && (reinterpret_cast<uintptr_t>(a.out + e.key_offset) % C::KPT == 0);
#pragma unroll 1
    for (uint64_t tb = first; tb < first + kBatchChunk && tb < e.key_count; tb += kTile) {
      if constexpr (ADD) {
        add_tile<C>(t, static_cast<W_of<C>*>(e.words), e.nblocks, mode, keys, e.key_count, a.acc0, vec_ok, tb,
                    (a.flags & kHintWarpAggregate) != 0);
      } else {
        contains_tile<C>(t, static_cast<const W_of<C>*>(e.words), e.nblocks, mode, keys, e.key_count,
                         a.out + e.key_offset, a.acc0, vec_ok, tb);
      }
    }
  }
}

}  // namespace bloomgb
