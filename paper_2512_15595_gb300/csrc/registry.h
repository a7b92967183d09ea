// Kernel argument blocks and the registry that maps a compiled specialisation
// (operation, geometry, layout) to its kernel.  Plain structs, shared by the
// kernel translation units and the host API.
#pragma once
#include <cstdint>
#include <vector>

namespace bloomgb {

// Arguments of the construction / lookup kernels (passed by value).
struct SbfArgs {
  void* filter;          // b*s words of S bits
  uint64_t nblocks;      // b
  const uint64_t* keys;  // n keys
  uint64_t n;
  uint8_t* out;          // lookup results (n bytes); unused by construction
  uint64_t acc0;         // XXH64 start value: seed + P5 + 8
  uint32_t flags;        // kHint* bits
  int block_mode;        // 0: b < 2^32, 1: b == 2^32, 2: b > 2^32
};

// Arguments of the random-access microbenchmark kernels.
struct GupsArgs {
  void* table;
  uint64_t nunits;
  const uint64_t* keys;
  uint64_t n;
  uint8_t* out;
  int unit_mode;  // same encoding as SbfArgs::block_mode
};

struct KernelEntry {
  int op;  // 0 add, 1 contains
  int B, S, K, theta, phi, kpt;
  const void* fn;
};

struct GupsEntry {
  int mode;  // 0 load, 1 red.or
  int unit_bytes, kpt;
  const void* fn;
};

#define BLOOMGB_GEOMETRIES(X) \
  X(64, 32) X(128, 32) X(256, 32) X(512, 32) X(64, 64) X(128, 64) X(256, 64) X(512, 64) X(1024, 64)
#define BLOOMGB_DECLARE(B, S) void register_B##B##_S##S(std::vector<KernelEntry>& v);
BLOOMGB_GEOMETRIES(BLOOMGB_DECLARE)
#undef BLOOMGB_DECLARE
void register_gups(std::vector<GupsEntry>& v);

}  // namespace bloomgb
