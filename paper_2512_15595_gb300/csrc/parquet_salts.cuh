// Salt set 1: the eight odd multipliers of the Apache Parquet split-block
// Bloom filter.  With B = 256, S = 32, k = 8 (one bit in each of the block's
// eight words, word w using multiplier w) the sectorized filter then stores
// exactly the bit array a Parquet writer stores for the same keys and block
// count -- the bitwise compatibility the paper claims for this configuration
// (Sec. VI).  The paper does not give the values; they were recovered from
// the bit arrays of pyarrow's Parquet writer (the test suite recovers them
// again and checks the oracle's copy of this table, which is compared with
// this one).
#pragma once
#include <cstdint>
namespace bloomgb {
__host__ __device__ constexpr uint32_t parquet_salt32_at(int i) {
  switch (i) {
    case 0: return 0x47B6137Bu;
    case 1: return 0x44974D91u;
    case 2: return 0x8824AD5Bu;
    case 3: return 0xA2B7289Du;
    case 4: return 0x705495C7u;
    case 5: return 0x2DF1424Bu;
    case 6: return 0x9EFC4947u;
    case 7: return 0x5C6BFB31u;
    default: return 0;
  }
}
}  // namespace bloomgb
