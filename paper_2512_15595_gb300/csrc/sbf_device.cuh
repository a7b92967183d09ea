// Device building blocks of the sectorized blocked Bloom filter kernels:
// XXH64 of one 64-bit key, block selection, salted bit positions, wide loads
// and cache-policy-tagged memory operations (inline PTX for sm_103a).
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>

#include "parquet_salts.cuh"
#include "salts.cuh"

namespace bloomgb {

// ---------------------------------------------------------------------------
// base hash (Sec. IV-B): XXH64 specialised to an 8-byte little-endian input
// ---------------------------------------------------------------------------
constexpr uint64_t kXP1 = 0x9E3779B185EBCA87ull;
constexpr uint64_t kXP2 = 0xC2B2AE3D27D4EB4Full;
constexpr uint64_t kXP3 = 0x165667B19E3779F9ull;
constexpr uint64_t kXP4 = 0x85EBCA77C2B2AE63ull;
constexpr uint64_t kXP5 = 0x27D4EB2F165667C5ull;

__device__ __forceinline__ uint64_t rotl64(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

// `acc0` = seed + P5 + 8 (input length), computed once per launch.
__device__ __forceinline__ uint64_t xxh64_key(uint64_t key, uint64_t acc0) {
  uint64_t lane = rotl64(key * kXP2, 31) * kXP1;
  uint64_t acc = rotl64(acc0 ^ lane, 27) * kXP1 + kXP4;
  acc ^= acc >> 33;
  acc *= kXP2;
  acc ^= acc >> 29;
  acc *= kXP3;
  acc ^= acc >> 32;
  return acc;
}

__host__ __device__ constexpr uint64_t xxh64_acc0(uint64_t seed) { return seed + kXP5 + 8; }

// ---------------------------------------------------------------------------
// block selection (Sec. II-A: "an additional hash selects one block"):
// multiply-shift range reduction of the high half of h.
// mode 0: b < 2^32, mode 1: b == 2^32, mode 2: b > 2^32 (128-bit product).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t block_of(uint64_t h, uint64_t nblocks, int mode) {
  const uint32_t hi = static_cast<uint32_t>(h >> 32);
  if (mode == 0) return __umulhi(hi, static_cast<uint32_t>(nblocks));
  if (mode == 1) return hi;
  return __umul64hi(h, nblocks);
}

inline int block_mode(uint64_t nblocks) {
  return nblocks < (1ull << 32) ? 0 : (nblocks == (1ull << 32) ? 1 : 2);
}

// ---------------------------------------------------------------------------
// salted bit positions (Sec. IV-B)
// ---------------------------------------------------------------------------
template <int S> struct WordOf;
template <> struct WordOf<32> { using type = uint32_t; };
template <> struct WordOf<64> { using type = uint64_t; };

// pattern bit for hash low half `hlo` and multiplier `salt`
__device__ __forceinline__ uint32_t pattern_bit(uint32_t hlo, uint32_t salt) {
  return (1u << ((hlo * salt) >> 27));
}
__device__ __forceinline__ uint64_t pattern_bit(uint32_t hlo, uint64_t salt) {
  return (1ull << ((static_cast<uint64_t>(hlo) * salt) >> 58));
}
// the bit position alone (S = 64): the top 6 bits of (hlo * salt) mod 2^64
__device__ __forceinline__ uint32_t pattern_pos(uint32_t hlo, uint64_t salt) {
  return static_cast<uint32_t>((static_cast<uint64_t>(hlo) * salt) >> 58);
}

// salt i of salt set SET (0: the SplitMix64 tables; 1: the Parquet
// split-block multipliers, 32-bit words only)
template <int S, int SET = 0> __host__ __device__ constexpr typename WordOf<S>::type salt_at(int i);
template <> __host__ __device__ constexpr uint32_t salt_at<32, 0>(int i) { return salt32_at(i); }
template <> __host__ __device__ constexpr uint64_t salt_at<64, 0>(int i) { return salt64_at(i); }
template <> __host__ __device__ constexpr uint32_t salt_at<32, 1>(int i) { return parquet_salt32_at(i); }

// Compile-time binary decision tree (Sec. IV-B, "mapping thread indices to
// salt indices"): returns salt_at(BASE + r * STRIDE) for a runtime r in
// [0, N) with log2(N) selects, every leaf a literal.
template <int S, int BASE, int STRIDE, int N, int SET = 0>
__device__ __forceinline__ typename WordOf<S>::type salt_select(uint32_t r) {
  if constexpr (N == 1) {
    return salt_at<S, SET>(BASE);
  } else {
    constexpr int H = N / 2;
    const auto lo = salt_select<S, BASE, STRIDE, H, SET>(r);
    const auto hi = salt_select<S, BASE + H * STRIDE, STRIDE, N - H, SET>(r - H);
    return r < static_cast<uint32_t>(H) ? lo : hi;
  }
}

// ---------------------------------------------------------------------------
// compile-time loops
// ---------------------------------------------------------------------------
template <class F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// ---------------------------------------------------------------------------
// cache policies (createpolicy) and tagged memory operations
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_normal() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// streaming key loads (read once): non-coherent path, no L1 allocation
__device__ __forceinline__ uint64_t ld_key1(const uint64_t* p, uint64_t pol) {
  uint64_t v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u64 %0, [%1], %2;"
               : "=l"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void ld_key2(const uint64_t* p, uint64_t pol, uint64_t (&v)[2]) {
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u64 {%0,%1}, [%2], %3;"
               : "=l"(v[0]), "=l"(v[1]) : "l"(p), "l"(pol));
}
__device__ __forceinline__ void ld_key4(const uint64_t* p, uint64_t pol, uint64_t (&v)[4]) {
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u64 {%0,%1,%2,%3}, [%4], %5;"
               : "=l"(v[0]), "=l"(v[1]), "=l"(v[2]), "=l"(v[3]) : "l"(p), "l"(pol));
}

// filter word loads for lookup: read-only during the kernel, no L1 allocation
// (random blocks have no reuse in L1), L2 policy chosen by the caller, and an
// L2 fetch of 64 bytes: a random 32-byte access otherwise pulls a whole
// 128-byte line from HBM (measured), wasting bandwidth the key stream needs.
// NWORDS contiguous words starting at p (aligned to the access width).
template <int NW>
__device__ __forceinline__ void ld_words(const uint32_t* p, uint64_t pol, uint32_t* w) {
  if constexpr (NW == 1) {
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.L2::64B.u32 %0, [%1], %2;"
                 : "=r"(w[0]) : "l"(p), "l"(pol));
  } else if constexpr (NW == 2) {
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.L2::64B.v2.u32 {%0,%1}, [%2], %3;"
                 : "=r"(w[0]), "=r"(w[1]) : "l"(p), "l"(pol));
  } else if constexpr (NW == 4) {
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.L2::64B.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "l"(p), "l"(pol));
  } else {
    static_assert(NW % 8 == 0, "word count");
#pragma unroll
    for (int c = 0; c < NW / 8; ++c) {
      uint32_t* o = w + 8 * c;
      asm volatile(
          "ld.global.nc.L1::no_allocate.L2::cache_hint.L2::64B.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
          : "=r"(o[0]), "=r"(o[1]), "=r"(o[2]), "=r"(o[3]), "=r"(o[4]), "=r"(o[5]), "=r"(o[6]),
            "=r"(o[7])
          : "l"(p + 8 * c), "l"(pol));
    }
  }
}
template <int NW>
__device__ __forceinline__ void ld_words(const uint64_t* p, uint64_t pol, uint64_t* w) {
  if constexpr (NW == 1) {
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.L2::64B.u64 %0, [%1], %2;"
                 : "=l"(w[0]) : "l"(p), "l"(pol));
  } else if constexpr (NW == 2) {
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.L2::64B.v2.u64 {%0,%1}, [%2], %3;"
                 : "=l"(w[0]), "=l"(w[1]) : "l"(p), "l"(pol));
  } else {
    static_assert(NW % 4 == 0, "word count");
#pragma unroll
    for (int c = 0; c < NW / 4; ++c) {
      uint64_t* o = w + 4 * c;
      asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.L2::64B.v4.u64 {%0,%1,%2,%3}, [%4], %5;"
                   : "=l"(o[0]), "=l"(o[1]), "=l"(o[2]), "=l"(o[3])
                   : "l"(p + 4 * c), "l"(pol));
    }
  }
}

// fire-and-forget atomic OR (no return value: red, not atom)
__device__ __forceinline__ void red_or(uint32_t* p, uint32_t v, uint64_t pol) {
  asm volatile("red.relaxed.gpu.global.or.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void red_or(uint64_t* p, uint64_t v, uint64_t pol) {
  asm volatile("red.relaxed.gpu.global.or.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol)
               : "memory");
}

// streaming 64-bit store with an L2 policy
__device__ __forceinline__ void st_u64_hint(uint64_t* p, uint64_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_u32_hint(uint32_t* p, uint32_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}

// result stores: streaming
__device__ __forceinline__ void st_out1(uint8_t* p, uint32_t v) {
  asm volatile("st.global.cs.u8 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_out2(uint8_t* p, uint32_t v) {
  asm volatile("st.global.cs.u16 [%0], %1;" ::"l"(p), "h"(static_cast<uint16_t>(v)) : "memory");
}
__device__ __forceinline__ void st_out4(uint8_t* p, uint32_t v) {
  asm volatile("st.global.cs.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

}  // namespace bloomgb
