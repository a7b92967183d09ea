// Staging of host-resident keys into device memory by the SMs.  On a
// Grace-coupled GPU the SMs read host memory coherently over NVLink-C2C; a
// light streaming kernel on one CTA slot per SM keeps the link busy while the
// rest of each SM partitions and inserts the previously staged pass.
#include <cstdint>

#include "host_stage.h"
#include "registry.h"

namespace bloomgb {

namespace {

// CTA b copies the contiguous range [b * per, (b + 1) * per) of n units;
// each iteration a thread issues four loads kHostStageThreads units apart
// (immediate offsets from one pointer), then the four stores.  Offsets
// within the range are of type I (32 bits when a range is below 2^31 units).
template <typename T, typename I>
__device__ __forceinline__ void copy_units(const T* __restrict__ s, T* __restrict__ d, uint64_t n) {
  constexpr uint32_t kT = kHostStageThreads;
  constexpr uint32_t kStep = 4 * kT;
  const uint64_t per = ((n + gridDim.x - 1) / gridDim.x + kStep - 1) / kStep * kStep;
  const uint64_t lo = static_cast<uint64_t>(blockIdx.x) * per;
  if (lo >= n) return;
  const I len = static_cast<I>((n - lo < per ? n - lo : per));
  s += lo;
  d += lo;
  I i = threadIdx.x;
  for (; i + 3 * kT < len; i += kStep) {
    const T v0 = __ldcs(s + i), v1 = __ldcs(s + i + kT), v2 = __ldcs(s + i + 2 * kT), v3 = __ldcs(s + i + 3 * kT);
    __stcs(d + i, v0);
    __stcs(d + i + kT, v1);
    __stcs(d + i + 2 * kT, v2);
    __stcs(d + i + 3 * kT, v3);
  }
#pragma unroll 1
  for (; i < len; i += kT) __stcs(d + i, __ldcs(s + i));
}

__global__ void __launch_bounds__(kHostStageThreads, 16)
    host_stage16_kernel(const ulonglong2* __restrict__ src, ulonglong2* __restrict__ dst, uint64_t n16) {
  copy_units<ulonglong2, uint32_t>(src, dst, n16);
}

__global__ void __launch_bounds__(kHostStageThreads, 16)
    host_stage8_kernel(const uint64_t* __restrict__ src, uint64_t* __restrict__ dst, uint64_t n) {
  copy_units<uint64_t, uint64_t>(src, dst, n);
}

// One chunk of a batch request: its host and arena element pointers and
// the number of its elements (1 to kBatchChunk).
template <typename T>
struct ChunkRef {
  T* host;
  T* arena;
  uint32_t cnt;
};

// The request owning chunk c, advanced from r (chunks are walked upwards;
// requests without elements own no chunk and are skipped).
__device__ __forceinline__ uint32_t owner(const uint64_t* __restrict__ begin, uint32_t r, uint64_t c) {
  while (begin[r + 1] <= c) ++r;
  return r;
}

template <typename T>
__device__ __forceinline__ ChunkRef<T> chunk_ref(const BatchFilter* __restrict__ desc, const uint64_t* __restrict__ begin,
                                                 const void* const* __restrict__ host, T* arena, uint32_t r, uint64_t c) {
  const uint64_t i0 = (c - begin[r]) * kBatchChunk;
  const uint64_t left = desc[r].key_count - i0;
  // host buffers of a gather are only read
  return {static_cast<T*>(const_cast<void*>(host[r])) + i0, arena + desc[r].key_offset + i0,
          static_cast<uint32_t>(left < kBatchChunk ? left : kBatchChunk)};
}

// The run of chunks [c, c_end) of this warp (warp w of all: chunks
// [w * per, (w + 1) * per)) and the request owning its first chunk, found
// by binary search (begin[0] = 0 <= c < begin[nreq]).  False if the run is
// empty.
__device__ __forceinline__ bool warp_run(const uint64_t* __restrict__ begin, uint32_t nreq, uint64_t chunks,
                                         uint64_t& c, uint64_t& c_end, uint32_t& r) {
  const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (blockDim.x / 32);
  const uint64_t w = static_cast<uint64_t>(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32;
  const uint64_t per = (chunks + warps - 1) / warps;
  c = w * per;
  c_end = c + per < chunks ? c + per : chunks;
  if (c >= c_end) return false;
  uint32_t lo = 0, hi = nreq;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) / 2;
    if (begin[mid] <= c) lo = mid;
    else hi = mid;
  }
  r = lo;
  return true;
}

// Keys of one chunk as 16-byte host loads: the chunk's keys from `h`
// (8-byte aligned) split into an optional head key (when h is 8 mod 16), 64
// or fewer 16-byte pairs, and an optional tail key; lane l loads pairs l and
// l + 32, lane 0 the head, lane 1 the tail.  Stores into the arena are
// 8-byte (any arena offset).
struct KeyChunk {
  ulonglong2 v[2];
  uint64_t head, tail;
};

__device__ __forceinline__ void load_chunk(const uint64_t* __restrict__ h, uint32_t cnt, uint32_t lane, KeyChunk& k) {
  const uint32_t mis = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(h) >> 3) & 1u;
  const uint32_t body = cnt - mis, npairs = body >> 1;
  const ulonglong2* hp = reinterpret_cast<const ulonglong2*>(h + mis);
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const uint32_t p = lane + 32u * j;
    if (p < npairs) k.v[j] = __ldcs(hp + p);
  }
  if (mis && lane == 0) k.head = __ldcs(h);
  if ((body & 1u) && lane == 1) k.tail = __ldcs(h + mis + 2 * npairs);
}

__device__ __forceinline__ void store_chunk(const uint64_t* h, uint64_t* __restrict__ a, uint32_t cnt, uint32_t lane,
                                            const KeyChunk& k) {
  const uint32_t mis = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(h) >> 3) & 1u;
  const uint32_t body = cnt - mis, npairs = body >> 1;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const uint32_t p = lane + 32u * j;
    if (p < npairs) {
      __stcs(a + mis + 2 * p, k.v[j].x);
      __stcs(a + mis + 2 * p + 1, k.v[j].y);
    }
  }
  if (mis && lane == 0) __stcs(a, k.head);
  if ((body & 1u) && lane == 1) __stcs(a + mis + 2 * npairs, k.tail);
}

// Gather of a batch's keys from host memory into the arena: warp w walks
// chunks [w * per, (w + 1) * per), two at a time (one search for its first
// request, then the owner advanced), all loads of both chunks before the
// stores; 16-byte host loads (half the requests of 8-byte ones over the link).
__global__ void __launch_bounds__(kHostStageThreads, 8)
    batch_gather_kernel(const BatchFilter* __restrict__ desc, const uint64_t* __restrict__ begin, uint32_t nreq,
                        uint64_t chunks, const void* const* __restrict__ host, uint64_t* __restrict__ arena) {
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t c, c_end;
  uint32_t r;
  if (!warp_run(begin, nreq, chunks, c, c_end, r)) return;
  for (; c < c_end; c += 2) {
    r = owner(begin, r, c);
    const ChunkRef<uint64_t> a = chunk_ref<uint64_t>(desc, begin, host, arena, r, c);
    const bool two = c + 1 < c_end;
    uint32_t r2 = r;
    ChunkRef<uint64_t> b{nullptr, nullptr, 0};
    if (two) {
      r2 = owner(begin, r, c + 1);
      b = chunk_ref<uint64_t>(desc, begin, host, arena, r2, c + 1);
    }
    KeyChunk ka, kb;
    load_chunk(a.host, a.cnt, lane, ka);
    if (two) load_chunk(b.host, b.cnt, lane, kb);
    store_chunk(a.host, a.arena, a.cnt, lane, ka);
    if (two) store_chunk(b.host, b.arena, b.cnt, lane, kb);
    r = r2;
  }
}

// Results of one chunk to host memory with 4-byte stores: the cnt result
// bytes at `a` (device) go to `h` (host, any alignment) as head bytes up to
// h's 4-byte boundary, 32 or fewer 4-byte words (lane l: word l, its bytes
// loaded one by one from the device) and tail bytes (lane l: byte l).
__device__ __forceinline__ void scatter_chunk(const uint8_t* __restrict__ a, uint8_t* __restrict__ h, uint32_t cnt,
                                              uint32_t lane) {
  const uint32_t lead = (4u - static_cast<uint32_t>(reinterpret_cast<uintptr_t>(h) & 3u)) & 3u;
  const uint32_t head = lead < cnt ? lead : cnt;
  const uint32_t nw = (cnt - head) >> 2, tail0 = head + 4 * nw;
  if (lane < nw) {
    const uint8_t* s = a + head + 4 * lane;
    const uint32_t v = static_cast<uint32_t>(s[0]) | (static_cast<uint32_t>(s[1]) << 8) |
                       (static_cast<uint32_t>(s[2]) << 16) | (static_cast<uint32_t>(s[3]) << 24);
    __stcs(reinterpret_cast<uint32_t*>(h + head) + lane, v);
  }
  if (lane < head) h[lane] = a[lane];
  if (lane < cnt - tail0) h[tail0 + lane] = a[tail0 + lane];
}

// Scatter of a batch's results from the arena into host memory: warp w walks
// chunks [w * per, (w + 1) * per), with 4-byte host stores.
__global__ void __launch_bounds__(kHostStageThreads, 8)
    batch_scatter_kernel(const BatchFilter* __restrict__ desc, const uint64_t* __restrict__ begin, uint32_t nreq,
                         uint64_t chunks, const void* const* __restrict__ host, uint8_t* __restrict__ arena) {
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t c, c_end;
  uint32_t r;
  if (!warp_run(begin, nreq, chunks, c, c_end, r)) return;
  for (; c < c_end; ++c) {
    r = owner(begin, r, c);
    const ChunkRef<uint8_t> k = chunk_ref<uint8_t>(desc, begin, host, arena, r, c);
    scatter_chunk(k.arena, k.host, k.cnt, lane);
  }
}

}  // namespace

cudaError_t launch_host_stage(const uint64_t* src, uint64_t* dst, uint64_t n, uint32_t ctas, cudaStream_t stream,
                              uint32_t* launches) {
  *launches = 0;
  if (n == 0) return cudaSuccess;
  if (n > (1ull << 32) || ctas == 0) return cudaErrorInvalidValue;  // 16-byte ranges stay below 2^31 units
  // The staging CTA stays resident for a whole pass beside the partition
  // kernel, whose CTAs need tens of KiB of shared memory: an SM brought up
  // with a large L1 (the default for a kernel without shared memory) would
  // take no partition CTA until it went idle.
  for (const void* fn : {reinterpret_cast<const void*>(&host_stage16_kernel),
                         reinterpret_cast<const void*>(&host_stage8_kernel)}) {
    const cudaError_t e =
        cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, kBesidePartitionCarveout);
    if (e != cudaSuccess) return e;
  }
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
    // 16-byte units, the odd last key (if any) by a one-thread launch
    if (n >= 2) {
      host_stage16_kernel<<<ctas, kHostStageThreads, 0, stream>>>(reinterpret_cast<const ulonglong2*>(src),
                                                                  reinterpret_cast<ulonglong2*>(dst), n / 2);
      ++*launches;
    }
    if (n & 1) {
      host_stage8_kernel<<<1, kHostStageThreads, 0, stream>>>(src + n - 1, dst + n - 1, 1);
      ++*launches;
    }
  } else {
    host_stage8_kernel<<<ctas, kHostStageThreads, 0, stream>>>(src, dst, n);
    *launches = 1;
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_gather(const BatchFilter* desc, const uint64_t* begin, uint32_t nreq, uint64_t chunks,
                                const uint64_t* const* host, uint64_t* arena_keys, uint32_t ctas,
                                cudaStream_t stream) {
  if (chunks == 0) return cudaSuccess;
  if (ctas == 0 || nreq == 0) return cudaErrorInvalidValue;
  batch_gather_kernel<<<ctas, kHostStageThreads, 0, stream>>>(desc, begin, nreq, chunks,
                                                               reinterpret_cast<const void* const*>(host), arena_keys);
  return cudaGetLastError();
}

cudaError_t launch_batch_scatter(const BatchFilter* desc, const uint64_t* begin, uint32_t nreq, uint64_t chunks,
                                 uint8_t* const* host, const uint8_t* arena_out, uint32_t ctas, cudaStream_t stream) {
  if (chunks == 0) return cudaSuccess;
  if (ctas == 0 || nreq == 0) return cudaErrorInvalidValue;
  batch_scatter_kernel<<<ctas, kHostStageThreads, 0, stream>>>(desc, begin, nreq, chunks,
                                                                reinterpret_cast<const void* const*>(host),
                                                                const_cast<uint8_t*>(arena_out));
  return cudaGetLastError();
}

}  // namespace bloomgb
