// Expansion of the slice-partitioned lookup's result bitmap into result bytes.
#include <cstdint>
#include <vector>

#include "registry.h"

namespace bloomgb {

// out[i] = bit i of the result bitmap: one 32-bit bitmap word per thread,
// written as 32 result bytes (two 16-byte stores when `out` allows it).
__global__ void __launch_bounds__(256) bitmap_expand_kernel(const ExpandArgs a) {
  const uint64_t nwords = (a.n + 31) / 32;
  const bool vec_ok = reinterpret_cast<uintptr_t>(a.out) % 16 == 0;
  for (uint64_t w = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; w < nwords;
       w += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint32_t bits = a.bitmap[w];
    const uint64_t base = w * 32;
    if (vec_ok && base + 32 <= a.n) {
      uint32_t v[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const uint32_t x = (bits >> (4 * c)) & 0xFu;
        v[c] = (x & 1u) | ((x & 2u) << 7) | ((x & 4u) << 14) | ((x & 8u) << 21);
      }
      asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(a.out + base), "r"(v[0]), "r"(v[1]), "r"(v[2]),
                   "r"(v[3])
                   : "memory");
      asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(a.out + base + 16), "r"(v[4]), "r"(v[5]),
                   "r"(v[6]), "r"(v[7])
                   : "memory");
    } else {
      for (uint32_t b = 0; b < 32 && base + b < a.n; ++b) a.out[base + b] = static_cast<uint8_t>((bits >> b) & 1u);
    }
  }
}

void register_expand(std::vector<KernelEntry>& v) {
  v.push_back({6, 0, 0, 0, 0, 0, 0, reinterpret_cast<const void*>(&bitmap_expand_kernel)});
}

}  // namespace bloomgb
