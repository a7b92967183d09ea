// Staging of host-resident keys into device memory by the SMs.  On a
// Grace-coupled GPU the SMs read host memory coherently over NVLink-C2C; a
// light streaming kernel on one CTA slot per SM keeps the link busy while the
// rest of each SM partitions and inserts the previously staged pass.
#include <cstdint>

#include "host_stage.h"

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

}  // namespace bloomgb
