// Registration of every compiled specialisation of the construction, lookup,
// record-insert and partition kernels for one geometry.
#pragma once

#include <vector>

#include "sbf_kernels.cuh"
#include "csbf_kernels.cuh"
#include "sbf_batch.cuh"
#include "sbf_partition.cuh"

namespace bloomgb {

template <class F, int... I>
__host__ void host_static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__host__ void host_static_for(F&& f) {
  host_static_for_impl(f, std::make_integer_sequence<int, N>{});
}

constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

template <int B, int S, int K, int SALTS = 0>
void register_k(std::vector<KernelEntry>& v) {
  constexpr int s = B / S;
  host_static_for<ilog2(s) + 1>([&](auto lt) {
    constexpr int T = 1 << decltype(lt)::value;
    host_static_for<ilog2(s / T) + 1>([&](auto lp) {
      constexpr int P = 1 << decltype(lp)::value;
      host_static_for<3>([&](auto lk) {
        constexpr int KPT = 1 << decltype(lk)::value;
        using C = Cfg<B, S, K, T, P, KPT, SALTS>;
        v.push_back({0, B, S, K, T, P, KPT, reinterpret_cast<const void*>(&sbf_add_kernel<C>), 0, SALTS});
        v.push_back({1, B, S, K, T, P, KPT, reinterpret_cast<const void*>(&sbf_contains_kernel<C>), 0, SALTS});
        v.push_back({2, B, S, K, T, P, KPT, reinterpret_cast<const void*>(&sbf_add_records_kernel<C>), 0, SALTS});
        v.push_back({4, B, S, K, T, P, KPT, reinterpret_cast<const void*>(&sbf_probe_records_kernel<C>), 0, SALTS});
        v.push_back({7, B, S, K, T, P, KPT, reinterpret_cast<const void*>(&sbf_batch_kernel<C, true>), 0, SALTS});
        v.push_back({8, B, S, K, T, P, KPT, reinterpret_cast<const void*>(&sbf_batch_kernel<C, false>), 0, SALTS});
      });
    });
  });
  v.push_back({3, B, S, K, 0, 0, 0, reinterpret_cast<const void*>(&sbf_partition_kernel<B, S, K, false, SALTS>), 0,
               SALTS});
  v.push_back({5, B, S, K, 0, 0, 0, reinterpret_cast<const void*>(&sbf_partition_kernel<B, S, K, true, SALTS>), 0,
               SALTS});
}

template <int B, int S, int K, int Z>
void register_csbf(std::vector<KernelEntry>& v) {
  host_static_for<ilog2(Z) + 1>([&](auto lt) {
    constexpr int T = 1 << decltype(lt)::value;
    host_static_for<3>([&](auto lk) {
      constexpr int KPT = 1 << decltype(lk)::value;
      using C = CCfg<B, S, K, Z, T, KPT>;
      v.push_back({9, B, S, K, T, 1, KPT, reinterpret_cast<const void*>(&csbf_add_kernel<C>), Z});
      v.push_back({10, B, S, K, T, 1, KPT, reinterpret_cast<const void*>(&csbf_contains_kernel<C>), Z});
    });
  });
}

// cache-sectorized kernels for groups Z in {1, 2, 4, 8} (Z < s) and K in {4, 8, 16} with Z | K
template <int B, int S, int Z>
void register_csbf_z(std::vector<KernelEntry>& v) {
  constexpr int s = B / S;
  if constexpr (Z < s) {
    if constexpr (4 % Z == 0) register_csbf<B, S, 4, Z>(v);
    if constexpr (8 % Z == 0) register_csbf<B, S, 8, Z>(v);
    if constexpr (16 % Z == 0) register_csbf<B, S, 16, Z>(v);
  }
}

template <int B, int S>
void register_geometry(std::vector<KernelEntry>& v) {
  register_csbf_z<B, S, 1>(v);
  register_csbf_z<B, S, 2>(v);
  register_csbf_z<B, S, 4>(v);
  register_csbf_z<B, S, 8>(v);
  constexpr int s = B / S;
  if constexpr (4 % s == 0) register_k<B, S, 4>(v);
  if constexpr (s <= 8) register_k<B, S, 8>(v);
  if constexpr (s <= 16) register_k<B, S, 16>(v);
  // the Parquet split-block salt set exists for its one geometry
  if constexpr (B == 256 && S == 32) register_k<256, 32, 8, 1>(v);
}

}  // namespace bloomgb
