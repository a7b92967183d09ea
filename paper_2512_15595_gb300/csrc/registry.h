// Kernel argument blocks and the registry that maps a compiled specialisation
// (operation, geometry, layout) to its kernel.  Plain structs, shared by the
// kernel translation units and the host API.
#pragma once
#include <cstddef>
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

// Launch geometry of the slice-partition kernel, shared by the kernel and the host.
// A CTA of kPartThreads threads partitions tiles of part_tile(lookup) keys,
// part_keys_per_thread(lookup) keys per thread.
constexpr int kPartThreads = 512;
constexpr int kPartKeysAdd = 6, kPartKeysLookup = 6;
constexpr int part_keys_per_thread(bool lookup) { return lookup ? kPartKeysLookup : kPartKeysAdd; }
constexpr int part_tile(bool lookup) { return kPartThreads * part_keys_per_thread(lookup); }
constexpr int kMaxParts = 1024;
constexpr uint64_t kRecTile = 128;  // slice buffer capacity granule: the largest record tile (32 x KPT)

// dynamic shared memory of the partition kernel for `nparts` slices (the
// lookup flavour also keeps each record's in-tile query index)
constexpr size_t partition_smem_bytes(int nparts, bool lookup = false) {
  return static_cast<size_t>(part_tile(lookup)) * 8                    // the tile's records, sorted by slice
         + static_cast<size_t>(nparts) * 8                               // per-slice packed buffer index and limit
         + static_cast<size_t>(nparts) * 4 * 3                           // per-slice counts (two tiles) and start
         + (lookup ? static_cast<size_t>(part_tile(lookup)) * 2 : 0);  // in-tile query index of each record
}

// Arguments of the slice-partition kernel (L2-blocked construction).
struct PartArgs {
  const uint64_t* keys;
  uint64_t n;
  uint64_t acc0;
  uint64_t nblocks;              // b <= 2^32 (records hold the block index in 32 bits)
  int block_mode;
  uint32_t shift;                // slice of block j = j >> shift
  uint32_t nparts;               // number of slices (<= 1024)
  uint64_t cap;                  // record slots per slice buffer (multiple of 128)
  unsigned long long* counts;    // [nparts] records reserved per slice (zeroed before launch)
  uint64_t* records;             // [nparts * cap] records (j << 32 | h_lo)
  void* filter;                  // overflow records are inserted (or looked up) here directly
  uint32_t* idx;                 // lookup: [nparts * cap] query index of each record
  uint32_t* bitmap;              // lookup: one result bit per query (zeroed before launch)
  uint32_t* status;              // kStatus* bits of index checks that failed (access skipped)
};

// Arguments of the record-probe kernel (slice-partitioned lookup): records
// of slices [part_lo, part_hi); a positive query sets its bit in `bitmap`.
struct ProbeArgs {
  const void* filter;
  const uint64_t* records;
  const uint32_t* idx;
  const unsigned long long* counts;
  uint32_t part_lo, part_hi;
  uint64_t cap;
  uint32_t* bitmap;
  uint32_t flags;
  uint64_t nblocks;   // b: a record's block index must be below it
  uint32_t* status;   // kStatus* bits of index checks that failed
};

// Arguments of the bitmap expansion: out[i] = bit i of `bitmap`, i < n.
struct ExpandArgs {
  const uint32_t* bitmap;
  uint64_t n;
  uint8_t* out;
};

// Arguments of the record-insert kernel: slices [part_lo, part_hi) of the
// slice buffers (one launch per group of slices keeps the warps within one
// L2-sized window of the filter; a kernel boundary re-synchronises them).
struct RecArgs {
  void* filter;
  const uint64_t* records;
  const unsigned long long* counts;
  uint32_t part_lo, part_hi;
  uint64_t cap;
  uint32_t flags;
  uint64_t nblocks;   // b: a record's block index must be below it
  uint32_t* status;   // kStatus* bits of index checks that failed
};

// Index checks of the slice-partitioned kernels.  Indexes derived from data
// are clamped into their arrays or checked before use; a failed check sets
// its bit in the status word and skips the access, so no index can leave its
// buffer.  None of them fails when the kernels are correct.
enum : uint32_t {
  kStatusBlockRange = 1u << 1,    // a record's block index >= b (record insert / probe)
  kStatusRecordSlice = 1u << 3,   // a sorted record outside the slices, or its block >= b (partition)
  kStatusBufferIndex = 1u << 4,   // a slice-buffer index outside the buffers (partition)
};

// One filter of a batch: its bit array and its run of the batch's keys.
struct BatchFilter {
  void* words;          // b*B/8 bytes
  uint64_t nblocks;     // b
  uint64_t key_offset;  // first key of this filter in the batch's key array
  uint64_t key_count;
};

// Batched construction / lookup over many filters in one launch.  The keys
// of all filters are cut into work chunks of kBatchChunk keys that never
// straddle two filters; chunk_begin[f] is the first chunk of filter f
// (nfilters + 1 entries).
constexpr uint64_t kBatchChunk = 128;
struct BatchArgs {
  const BatchFilter* filters;
  const uint64_t* chunk_begin;
  uint32_t nfilters;
  uint64_t total_chunks;
  const uint64_t* keys;
  uint8_t* out;         // lookup results, same indexing as keys
  uint64_t acc0;
  uint32_t flags;
  uint64_t prefetch_chunks;  // BF_HINT_PREFETCH_L2: lookahead in chunks (the grid's warp count); else 0
};

struct KernelEntry {
  // 0 add, 1 contains, 2 add from slice records, 3 slice partition (add),
  // 4 probe slice records, 5 slice partition (lookup), 6 bitmap expansion,
  // 7 batched add, 8 batched contains
  // 9 cache-sectorized add, 10 cache-sectorized contains (z = groups)
  int op;
  int B, S, K, theta, phi, kpt;
  const void* fn;
  int z = 0;      // groups of a cache-sectorized kernel; 0 = sectorized
  int salts = 0;  // salt set (bf_params.salts)
};

struct GupsEntry {
  int mode;  // 0 load, 1 red.or
  int unit_bytes, kpt;
  const void* fn;
};

// Lookup of a compiled kernel (implemented with the registry in bf_api.cu).
const KernelEntry* find_kernel(int op, int block_bits, int word_bits, int k, int theta, int phi, int kpt, int z,
                               int salts = 0);
// Resident CTAs per SM of a kernel at a CTA size (cached).
int kernel_resident_ctas(const void* fn, int threads, int device);

#define BLOOMGB_GEOMETRIES(X) \
  X(64, 32) X(128, 32) X(256, 32) X(512, 32) X(64, 64) X(128, 64) X(256, 64) X(512, 64) X(1024, 64)
#define BLOOMGB_DECLARE(B, S) void register_B##B##_S##S(std::vector<KernelEntry>& v);
BLOOMGB_GEOMETRIES(BLOOMGB_DECLARE)
#undef BLOOMGB_DECLARE
void register_gups(std::vector<GupsEntry>& v);
void register_expand(std::vector<KernelEntry>& v);

}  // namespace bloomgb
