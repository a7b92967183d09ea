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

// GATHER: host keys -> arena; else arena results -> host.  Warp w walks
// chunks [w * per, (w + 1) * per), two at a time: all loads of both chunks,
// then the stores (lane l takes elements l, l + 32, l + 64, l + 96).
template <bool GATHER, typename T>
__global__ void __launch_bounds__(kHostStageThreads, 8)
    batch_stage_kernel(const BatchFilter* __restrict__ desc, const uint64_t* __restrict__ begin, uint32_t nreq,
                       uint64_t chunks, const void* const* __restrict__ host, T* __restrict__ arena) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (blockDim.x / 32);
  const uint64_t w = static_cast<uint64_t>(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32;
  const uint64_t per = (chunks + warps - 1) / warps;
  uint64_t c = w * per;
  const uint64_t c_end = c + per < chunks ? c + per : chunks;
  if (c >= c_end) return;
  // the last request whose first chunk is at or before c (begin[0] = 0 <= c < begin[nreq])
  uint32_t lo = 0, hi = nreq;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) / 2;
    if (begin[mid] <= c) lo = mid;
    else hi = mid;
  }
  uint32_t r = lo;
  constexpr uint32_t kStep = kBatchChunk / 4;  // 32: one element per lane per quarter chunk
  for (; c < c_end; c += 2) {
    r = owner(begin, r, c);
    const ChunkRef<T> a = chunk_ref<T>(desc, begin, host, arena, r, c);
    const bool two = c + 1 < c_end;
    uint32_t r2 = r;
    ChunkRef<T> b{nullptr, nullptr, 0};
    if (two) {
      r2 = owner(begin, r, c + 1);
      b = chunk_ref<T>(desc, begin, host, arena, r2, c + 1);
    }
    T va[4], vb[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t i = lane + j * kStep;
      if (i < a.cnt) va[j] = __ldcs(GATHER ? a.host + i : a.arena + i);
      if (i < b.cnt) vb[j] = __ldcs(GATHER ? b.host + i : b.arena + i);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t i = lane + j * kStep;
      if (i < a.cnt) __stcs(GATHER ? a.arena + i : a.host + i, va[j]);
      if (i < b.cnt) __stcs(GATHER ? b.arena + i : b.host + i, vb[j]);
    }
    r = r2;
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
  batch_stage_kernel<true, uint64_t><<<ctas, kHostStageThreads, 0, stream>>>(
      desc, begin, nreq, chunks, reinterpret_cast<const void* const*>(host), arena_keys);
  return cudaGetLastError();
}

cudaError_t launch_batch_scatter(const BatchFilter* desc, const uint64_t* begin, uint32_t nreq, uint64_t chunks,
                                 uint8_t* const* host, const uint8_t* arena_out, uint32_t ctas, cudaStream_t stream) {
  if (chunks == 0) return cudaSuccess;
  if (ctas == 0 || nreq == 0) return cudaErrorInvalidValue;
  batch_stage_kernel<false, uint8_t><<<ctas, kHostStageThreads, 0, stream>>>(
      desc, begin, nreq, chunks, reinterpret_cast<const void* const*>(host), const_cast<uint8_t*>(arena_out));
  return cudaGetLastError();
}

}  // namespace bloomgb
