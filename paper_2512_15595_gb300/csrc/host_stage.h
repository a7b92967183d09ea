// Staging of host-resident keys into device memory by the SMs
// (host_stage.cu), used by the pass-wise host-buffer construction and lookup.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace bloomgb {

// Threads per CTA of the staging kernel: one such CTA (at most 32 registers
// per thread, 4096 registers in all) fits on an SM beside three partition
// CTAs of either kind, so the staging of the next pass runs beside the
// partition and the record kernels of the current one.
constexpr uint32_t kHostStageThreads = 128;

// Shared-memory carveout (percent of the maximum) preferred by the staging
// kernel and by every kernel that runs beside the slice partition.  A
// resident CTA pins its SM's L1 / shared-memory split until the SM goes
// idle, and the staging CTA stays resident for a whole pass, so all of them
// ask for one split: 50 % (the driver rounds up to a 132 KiB shared / 124
// KiB L1 configuration) holds three partition CTAs (27 to 33 KiB each with
// 128 slices) and leaves the record probes most of their L1.
constexpr int kBesidePartitionCarveout = 50;

// Enqueue dst[0, n) = src[0, n) on `stream` with `ctas` CTAs; *launches =
// the kernels enqueued (0 to 2).  src is host memory the kernels can address
// (page-locked, or pageable on a GPU with pageable memory access), dst
// device memory; both 8-byte aligned; n <= 2^32 and ctas >= 1, else
// cudaErrorInvalidValue with nothing enqueued.  Each thread keeps four
// 16-byte loads in flight when src and dst are both 16-byte aligned (the odd
// last key, if any, by a second one-thread launch), else four 8-byte loads;
// the stores are streaming (evict-first), so the staged keys do not displace
// the L2-resident filter window.
cudaError_t launch_host_stage(const uint64_t* src, uint64_t* dst, uint64_t n, uint32_t ctas, cudaStream_t stream,
                              uint32_t* launches);

// Staging of a batch of requests between their host buffers and a device
// arena by the SMs, in the chunk decomposition of the batched kernels:
// request r (of nreq) owns chunks [begin[r], begin[r + 1]) of kBatchChunk
// elements, and its element i lives at arena element desc[r].key_offset + i
// and at host element i of host[r]; desc[r].key_count elements in all.
// gather: the 8-byte keys from host[r] (8-byte aligned) into arena_keys;
// scatter: the 1-byte results from arena_out into host[r].  desc, begin and
// host are device arrays; the host buffers must be addressable by the
// kernels.  One warp walks a contiguous run of chunks (one search for its
// first request); the gather loads two chunks at a time as 16-byte host
// loads (a single key at either end where the host address is 8 mod 16),
// the scatter stores 4-byte words (single bytes up to the host address's
// 4-byte boundary and at the end); `ctas` CTAs of kHostStageThreads threads.
struct BatchFilter;
cudaError_t launch_batch_gather(const BatchFilter* desc, const uint64_t* begin, uint32_t nreq, uint64_t chunks,
                                const uint64_t* const* host, uint64_t* arena_keys, uint32_t ctas,
                                cudaStream_t stream);
cudaError_t launch_batch_scatter(const BatchFilter* desc, const uint64_t* begin, uint32_t nreq, uint64_t chunks,
                                 uint8_t* const* host, const uint8_t* arena_out, uint32_t ctas, cudaStream_t stream);

}  // namespace bloomgb
