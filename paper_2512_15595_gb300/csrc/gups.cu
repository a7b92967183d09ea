// Random-access microbenchmark that bounds the filter kernels.
//
// Sec. V-B bounds DRAM-resident filter throughput by measured random-access
// throughput (GUPS).  These kernels reproduce the filter kernels' memory
// traffic without their arithmetic: the same 8-byte key stream, the same
// multiply-shift unit selection (applied to the raw key instead of its hash),
// the same wide loads / fire-and-forget atomics, and for loads the same
// one-byte-per-key result stream.  MODE 0: loads of the unit; MODE 1: one
// 32-bit red.or per 32-byte sector of the unit; MODE 2: the record-insert
// kernel's traffic, four lanes per key each ORing 64 bits, so every 32-byte
// sector of the unit receives one full-width update (its 8 words).
#include <cstdint>
#include <vector>

#include "registry.h"
#include "sbf_register.cuh"

namespace bloomgb {

template <int UNIT, int KPT, int MODE>
__global__ void __launch_bounds__(kMaxBlockThreads) gups_kernel(const GupsArgs a) {
  constexpr bool RED = MODE == 1;
  static_assert(UNIT == 8 || UNIT % 32 == 0, "unit");
  constexpr int kSectors = UNIT >= 32 ? UNIT / 32 : 1;
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t pol_keys = policy_evict_first();
  const uint64_t pol_tab = policy_evict_normal();
  constexpr uint64_t kTile = 32u * KPT;
  const uint64_t ntiles = (a.n + kTile - 1) / kTile;
  const uint64_t warps_per_cta = blockDim.x >> 5;
  const uint64_t nwarps = static_cast<uint64_t>(gridDim.x) * warps_per_cta;
  const bool vec_ok = (reinterpret_cast<uintptr_t>(a.keys) % (8u * KPT) == 0) &&
                      (reinterpret_cast<uintptr_t>(a.out) % KPT == 0);
  for (uint64_t tile = blockIdx.x * warps_per_cta + (threadIdx.x >> 5); tile < ntiles; tile += nwarps) {
    const uint64_t base = tile * kTile + static_cast<uint64_t>(lane) * KPT;
    uint64_t key[KPT];
    const uint32_t valid = load_keys<KPT>(a.keys, a.n, base, vec_ok, pol_keys, key);
    uint64_t unit[KPT];
#pragma unroll
    for (int u = 0; u < KPT; ++u) unit[u] = ((valid >> u) & 1u) ? block_of(key[u], a.nunits, a.unit_mode) : 0;
    if constexpr (MODE == 2) {
      // lane r of each group of four lanes ORs 64-bit word r of every sector
      // of the group members' units (the Theta = 4, Phi = 2 insert layout)
      uint64_t* t = static_cast<uint64_t*>(a.table);
      const uint32_t r = lane & 3u;
#pragma unroll
      for (int u = 0; u < KPT; ++u) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const uint64_t km = __shfl_sync(0xFFFFFFFFu, key[u], m, 4);
          const uint64_t um = __shfl_sync(0xFFFFFFFFu, unit[u], m, 4);
          const uint32_t vm = __shfl_sync(0xFFFFFFFFu, valid, m, 4);
          if ((vm >> u) & 1u) {
            const uint64_t bits = (1ull << (km >> 58)) | (1ull << ((km >> 52) & 63u));
#pragma unroll
            for (int c = 0; c < kSectors; ++c) red_or(t + um * (UNIT / 8) + c * 4 + r, bits, pol_tab);
          }
        }
      }
    } else if constexpr (RED) {
      uint32_t* t = static_cast<uint32_t*>(a.table);
#pragma unroll
      for (int u = 0; u < KPT; ++u) {
        if ((valid >> u) & 1u) {
          const uint32_t bit = 1u << (key[u] >> 59);
#pragma unroll
          for (int c = 0; c < kSectors; ++c) {
            const uint64_t word = unit[u] * (UNIT / 4) + c * 8 + (UNIT == 8 ? (key[u] & 1u) : (key[u] & 7u));
            red_or(t + word, bit, pol_tab);
          }
        }
      }
    } else {
      uint32_t fold[KPT];
      if constexpr (UNIT == 8) {
        const uint64_t* t = static_cast<const uint64_t*>(a.table);
        uint64_t v[KPT];
#pragma unroll
        for (int u = 0; u < KPT; ++u) ld_words<1>(t + unit[u], pol_tab, &v[u]);
#pragma unroll
        for (int u = 0; u < KPT; ++u) fold[u] = __popcll(v[u]) & 1u;
      } else {
        const uint32_t* t = static_cast<const uint32_t*>(a.table);
        uint32_t w[KPT][UNIT / 4];
#pragma unroll
        for (int u = 0; u < KPT; ++u) ld_words<UNIT / 4>(t + unit[u] * (UNIT / 4), pol_tab, w[u]);
#pragma unroll
        for (int u = 0; u < KPT; ++u) {
          uint32_t x = 0;
#pragma unroll
          for (int i = 0; i < UNIT / 4; ++i) x ^= w[u][i];
          fold[u] = __popc(x) & 1u;
        }
      }
      if (vec_ok && valid == (1u << KPT) - 1u) {
        if constexpr (KPT == 1) st_out1(a.out + base, fold[0]);
        else if constexpr (KPT == 2) st_out2(a.out + base, fold[0] | (fold[1] << 8));
        else st_out4(a.out + base, fold[0] | (fold[1] << 8) | (fold[2] << 16) | (fold[3] << 24));
      } else {
#pragma unroll
        for (int u = 0; u < KPT; ++u)
          if ((valid >> u) & 1u) st_out1(a.out + base + u, fold[u]);
      }
    }
  }
}

template <int UNIT>
void register_gups_unit(std::vector<GupsEntry>& v) {
  host_static_for<3>([&](auto lk) {
    constexpr int KPT = 1 << decltype(lk)::value;
    v.push_back({0, UNIT, KPT, reinterpret_cast<const void*>(&gups_kernel<UNIT, KPT, 0>)});
    v.push_back({1, UNIT, KPT, reinterpret_cast<const void*>(&gups_kernel<UNIT, KPT, 1>)});
    if constexpr (UNIT >= 32) v.push_back({2, UNIT, KPT, reinterpret_cast<const void*>(&gups_kernel<UNIT, KPT, 2>)});
  });
}

void register_gups(std::vector<GupsEntry>& v) {
  register_gups_unit<8>(v);
  register_gups_unit<32>(v);
  register_gups_unit<64>(v);
  register_gups_unit<128>(v);
}

}  // namespace bloomgb
