// Cost of back-to-back tcgen05.mma kind::f16 instructions (M = 128, K = 16,
// bf16 operands, fp32 accumulation) by N and by where A comes from: one
// issuing thread per SM, every SM busy.  The learned prefilter's tile is a
// fixed set of such instructions (4 with N = 128 and A in shared memory, 8
// with N = 64 and A in tensor memory), so these costs bound its throughput
// from above the way the random-access microbenchmark bounds the filters'.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "bloomgb.h"

namespace {

constexpr int kCostSmem = 120 * 1024;  // one CTA per SM (each takes all 512 TMEM columns)

__device__ __forceinline__ uint64_t cost_desc(uint32_t saddr) {
  uint64_t d = static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;
  d |= static_cast<uint64_t>(1024 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(2) << 61;
  return d;
}

__host__ __device__ constexpr uint32_t cost_idesc(uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

// Operands are zeros (A: 16 KiB, B: up to 32 KiB of shared memory; A in
// tensor memory: columns 256..287); D takes columns 0..N-1.  Thread 0 issues
// `reps` MMAs, commits, waits (bounded, 2 s) and block 0 reports the cycles.
template <uint32_t N, bool TA>
__global__ void __launch_bounds__(128, 1) k_mma_cost(uint32_t reps, unsigned long long* out) {
  extern __shared__ uint8_t raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sb = static_cast<uint32_t>(__cvta_generic_to_shared(sm));
  for (int i = threadIdx.x; i < (48 * 1024) / 16; i += blockDim.x) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  __shared__ uint32_t holder;
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = static_cast<uint32_t>(__cvta_generic_to_shared(&bar));
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(&holder)))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = holder;
  if (threadIdx.x == 0) {
    const long long t0 = clock64();
    for (uint32_t i = 0; i < reps; ++i) {
      const uint32_t acc = i > 0;
      if (TA) {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
                tmem),
            "r"(tmem + 256 + 8 * (i & 3)), "l"(cost_desc(sb + 16384 + 32 * (i & 3))), "r"(cost_idesc(N)), "r"(acc));
      } else {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem),
            "l"(cost_desc(sb + 32 * (i & 3))), "l"(cost_desc(sb + 16384 + 32 * (i & 3))), "r"(cost_idesc(N)), "r"(acc));
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(b) : "memory");
    uint32_t done = 0;
    unsigned long long g0, g;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
    do {
      asm volatile(
          "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\nselp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(b)
          : "memory");
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g));
    } while (!done && g - g0 < 2000000000ull);
    const long long t1 = clock64();
    if (blockIdx.x == 0) {
      out[0] = static_cast<unsigned long long>(t1 - t0);
      out[1] = done;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

template <uint32_t N, bool TA>
cudaError_t run_cost(uint32_t reps, unsigned long long* d_out, int sms) {
  cudaError_t e = cudaFuncSetAttribute(k_mma_cost<N, TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCostSmem);
  if (e != cudaSuccess) return e;
  k_mma_cost<N, TA><<<sms, 128, kCostSmem>>>(64, d_out);  // warm-up
  k_mma_cost<N, TA><<<sms, 128, kCostSmem>>>(reps, d_out);
  return cudaGetLastError();
}

}  // namespace

extern "C" bf_status bf_mma_cost(uint32_t n, int a_tmem, uint32_t reps, double* cycles) {
  if (!cycles || reps == 0 || reps > (1u << 24)) return BF_EINVAL;
  if (n != 16 && n != 32 && n != 64 && n != 128 && n != 256) return BF_EINVAL;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, 16) != cudaSuccess) {
    cudaGetLastError();
    return BF_ENOMEM;
  }
  cudaError_t e = cudaSuccess;
  const bool ta = a_tmem != 0;
  switch (n) {
    case 16: e = ta ? run_cost<16, true>(reps, d, sms) : run_cost<16, false>(reps, d, sms); break;
    case 32: e = ta ? run_cost<32, true>(reps, d, sms) : run_cost<32, false>(reps, d, sms); break;
    case 64: e = ta ? run_cost<64, true>(reps, d, sms) : run_cost<64, false>(reps, d, sms); break;
    case 128: e = ta ? run_cost<128, true>(reps, d, sms) : run_cost<128, false>(reps, d, sms); break;
    default: e = ta ? run_cost<256, true>(reps, d, sms) : run_cost<256, false>(reps, d, sms); break;
  }
  unsigned long long h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return BF_ECUDA;
  if (!h[1]) return BF_ETIMEDOUT;
  *cycles = static_cast<double>(h[0]) / reps;
  return BF_OK;
}
