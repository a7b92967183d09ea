/*
 * bloomgb -- sectorized blocked Bloom filter on one GB300 GPU (sm_103a).
 *
 * C ABI of the library built from paper_2512_15595_gb300/csrc.  The filter
 * and the operations follow "Optimizing Bloom Filters on Modern GPUs"
 * (arXiv 2512.15595):
 *
 *   - Sec. II-A: a Bloom filter approximates a set of n keys with a bit array
 *     of m bits; construction sets the k pattern bits of every key, lookup
 *     reports a key present iff all of its k bits are set (false positives
 *     possible, false negatives never).  The blocked form splits the array
 *     into b blocks of B bits and sends all k bits of a key into one block;
 *     the sectorized form splits a block into s = B/S words of S bits and
 *     puts k' = k/s bits into every word (k >= s, s | k).
 *   - Sec. IV-B: one 64-bit base hash per key (XXH64); the bit positions are
 *     the high bits of the base hash times odd constants (salts).
 *   - Sec. IV-A / IV-C: a key is processed by a cooperative group of Theta
 *     threads, each loading Phi contiguous words per step (1 <= Theta*Phi <= s,
 *     both powers of two); the group shares the key's hash by shuffles.
 *
 * Conventions (all entry points):
 *   - Pointers named d_* are device pointers owned by the caller; h_* are host
 *     pointers owned by the caller.  The library never frees caller memory.
 *   - Operations are asynchronous on the given stream (NULL = legacy default
 *     stream) and never synchronize the host, except where stated.
 *   - Argument errors are detected on the host before any launch and return
 *     BF_EINVAL / BF_EUNSUPPORTED; nothing is enqueued in that case.
 *   - A CUDA error reported at launch returns BF_ECUDA; bf_last_error() gives
 *     the message.  n = 0 is a no-op returning BF_OK.
 *   - Bit layout of the filter: block j occupies words j*s .. j*s+s-1; a word
 *     is S bits little-endian, bit p is the value 1 << p.
 *   - Hash readings the paper leaves open (fixed by this library):
 *       h     = XXH64 of the key's 8 little-endian bytes with params.seed;
 *       j     = ((h >> 32) * b) >> 32 if b <= 2^32, else high64(h * b);
 *       h_lo  = h mod 2^32;
 *       bit t of word w (t < k', w < s) uses salt i = w + s*t and is
 *         ((h_lo * salt32[i]) mod 2^32) >> 27          for S = 32,
 *         ((h_lo * salt64[i]) mod 2^64) >> 58          for S = 64,
 *       salt64[i] = (i-th output of SplitMix64 seeded 0x5A175EED) | 1,
 *       salt32[i] = (salt64[i] >> 32) | 1.
 *   - Thread safety: distinct filters may be used from distinct host threads.
 *     Calls on one filter from several host threads must be serialized by the
 *     caller.  A filter's slice-partitioned and host-buffer calls use
 *     workspaces and internal streams of that filter, so calls on one filter
 *     enqueued on different streams must be ordered by the caller (one
 *     stream, or events between them).
 */
#ifndef BLOOMGB_H
#define BLOOMGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL selects the legacy default stream. */
typedef struct CUstream_st* bf_stream_t;

typedef struct bf_filter bf_filter;

typedef enum {
    BF_OK = 0,
    BF_EINVAL = 1,         /* bad argument: null pointer, misalignment, bad geometry */
    BF_ENOMEM = 2,         /* device or pinned-host allocation failed */
    BF_ECUDA = 3,          /* a CUDA call failed; see bf_last_error() */
    BF_EUNSUPPORTED = 4,   /* valid by the definition, but not compiled into this library */
    BF_ETIMEDOUT = 5       /* a wait ran out of time (bf_server_wait) */
} bf_status;

/* Filter geometry (Sec. II-A).  num_blocks = b >= 1; block_bits = B in
   {64,128,256,512,1024}; word_bits = S in {32,64}; seed = XXH64 seed.
   groups = 0 (or s): sectorized filter (SBF): s = B/S words per block, k
   pattern bits with k >= s, s | k, k <= 64, k/s bits in every word.
   0 < groups = z < s: cache-sectorized filter (CSBF): the s words form z
   groups of s/z neighbouring words; in group q the word q*(s/z) + sel is
   selected, sel = the top log2(s/z) bits of (h_lo * salt[63 - q]) (mod 2^S,
   with a 64-bit product for S = 64), and it receives k/z bits (bit t from
   salt q + z*t); z | s, z | k, k + z <= 64.  Only the z selected words are
   read or updated.
   Builds compile k in {4,8,16} and, for the CSBF, z in {1,2,4,8}; other
   admissible values return BF_EUNSUPPORTED.  The slice-partitioned paths,
   batches and bf_add_noalloc serve sectorized filters only.
   salts: the odd multipliers of the bit positions (Sec. IV-B).  0 (default):
   the library's SplitMix64 tables.  1: the Apache Parquet split-block Bloom
   filter's eight multipliers, for block_bits = 256, word_bits = 32, k = 8,
   sectorized only (else BF_EINVAL); with seed 0 the bit array is then the one
   a Parquet writer stores for the same keys and block count (Sec. VI), so
   such filters can be read from or written into Parquet files as they are. */
typedef struct {
    uint64_t num_blocks;
    uint32_t block_bits;
    uint32_t word_bits;
    uint32_t k;
    uint32_t groups;        /* z; 0 = sectorized */
    uint64_t seed;
    uint32_t salts;         /* salt set: 0 default, 1 Parquet split-block */
    uint32_t reserved;      /* 0 */
} bf_params;

typedef enum { BF_OP_ADD = 0, BF_OP_CONTAINS = 1 } bf_op;

/* Cache-policy hints (bit flags of bf_layout.flags). */
enum {
    BF_HINT_FILTER_EVICT_LAST = 1u << 0,   /* filter accesses carry an L2 evict_last policy */
    BF_HINT_KEYS_EVICT_NORMAL = 1u << 1,   /* keys load with evict_normal instead of evict_first */
    BF_HINT_PREFETCH_L2 = 1u << 2,         /* batched kernels only (others ignore it): while a warp
                                              works on a key chunk, it bulk-prefetches into L2 the
                                              share of its filter's bit array that belongs to the
                                              chunk one grid-stride step ahead, so that filters
                                              are streamed into L2 before their keys arrive */
    BF_HINT_WARP_AGGREGATE = 1u << 3       /* construction (direct, record-insert and batched
                                              kernels; lookups ignore it): a key equal to the key
                                              before it in the warp's tile of keys (or, in the
                                              record-insert kernel, a record equal to the one
                                              before it) issues no atomics -- it sets the same
                                              bits -- so a run of repeated keys costs one update;
                                              the bits are those without the hint */
};

/* Execution layout of one operation (Sec. IV-A, IV-C).
   cg = Theta threads per key (power of two, 1..s; for a cache-sectorized
   filter a divisor of groups, each lane handling groups/cg groups); phi = Phi
   words per thread per step (power of two, cg*phi <= s; 1 for a
   cache-sectorized filter, which loads single words); kpt = keys each thread hashes per
   tile (1, 2 or 4); block_threads = CTA size (multiple of 32, <= 512);
   grid_ctas = number of CTAs (0 = SM count x resident CTAs per SM).
   A zero in cg/phi/kpt/block_threads selects the library default. */
typedef struct {
    uint32_t cg;
    uint32_t phi;
    uint32_t kpt;
    uint32_t block_threads;
    uint32_t grid_ctas;
    uint32_t flags;
} bf_layout;

/* Validate a geometry on the host.  BF_OK, BF_EINVAL (not an SBF by
   Sec. II-A) or BF_EUNSUPPORTED (admissible but not compiled). */
bf_status bf_params_check(const bf_params* params);

/* Validate a layout for a geometry and operation on the host (Sec. IV-A:
   1 <= cg*phi <= s, powers of two); zeros are resolved to defaults first. */
bf_status bf_layout_check(const bf_params* params, int op, const bf_layout* layout);

/* Create a filter on the current CUDA device: the empty m-bit array of Sec.
   II-A (m = b*B, all bits 0 for a library-allocated array), organised as b
   blocks of s words.  If d_words is NULL the library
   allocates b*B/8 bytes (owned, freed by bf_destroy) and zeroes them with a
   blocking memset.  Otherwise it adopts the caller's buffer, which must hold
   b*B/8 bytes, be aligned to max(32, B/8) bytes and stay valid until
   bf_destroy; an adopted buffer is neither cleared nor freed. */
bf_status bf_create(const bf_params* params, void* d_words, bf_filter** out);

/* Release the filter (and the bit array if the library allocated it).  The
   bits themselves are the filter of Sec. II-A; an adopted array keeps them
   after this call.  The caller must ensure no work on the filter is still
   in flight. */
bf_status bf_destroy(bf_filter* f);

/* Zero the bit array, asynchronously on stream: the empty filter of Sec.
   II-A (every lookup then reports absent). */
bf_status bf_clear(bf_filter* f, bf_stream_t stream);

/* Construction (Sec. II-A, Sec. IV): set the pattern of each of the n keys
   d_keys[0..n) (8-byte aligned device array).  Bitwise OR is commutative and
   idempotent, so the result does not depend on layout, order or duplicates. */
bf_status bf_add(bf_filter* f, const uint64_t* d_keys, uint64_t n, bf_stream_t stream);

/* Lookup (Sec. II-A, Sec. IV): d_out[i] = 1 if every pattern bit of d_keys[i]
   is set, else 0; d_out is a device array of n bytes (compatible with
   torch.bool).  Reads the filter only. */
bf_status bf_contains(const bf_filter* f, const uint64_t* d_keys, uint64_t n, uint8_t* d_out,
                      bf_stream_t stream);

/* End-to-end variants over HOST buffers.  The work is ordered after prior
   work on `stream` and all of it is complete when `stream` is; h_keys / h_out
   must stay valid until then.  The device "can address" a buffer when it is
   page-locked (cudaHostAlloc / cudaHostRegister) or the GPU has pageable
   memory access (as on Grace-coupled GB300), and for the keys when h_keys is
   also 8-byte aligned; bf_set_staging(BF_HOST_STAGED) makes every buffer
   count as one it cannot address.  Three ways, chosen per call:
     staged passes: when the call takes the slice-partitioned path (see
       bf_set_partition), unless bf_set_staging selected BF_HOST_DIRECT and
       the device can address the buffers: the call runs in (at least) eight
       passes.  On an internal copy-in stream (highest priority) each pass's
       keys are copied into one of two device staging slots, by a staging
       kernel on one CTA slot per SM when the device can address them, else
       by the copy engine, while `stream` partitions and inserts (or probes)
       the previous pass from device memory; for bf_contains_host the copy
       engine returns each pass's results on an internal copy-out stream, so
       the host link stays busy in both directions (into a pageable h_out
       the device can address, the kernels write the results in place).
       The staging slots (2 x 8 bytes per key of a pass, plus 2 x 1 byte for
       lookups) are kept until bf_set_staging or bf_destroy.  Without memory for them the call takes
       one of the next two ways;
     direct: otherwise, when the device can address the buffers, the kernels
       read the keys and write the results in place over the CPU-GPU link; a
       slice-partitioned call then runs in (at least) eight passes over two
       alternating workspaces, the record inserts (or probes and result
       expansion) of one pass on an internal stream while the next pass's
       partition reads the host buffer;
     chunked: otherwise keys are copied in chunks into device staging
       buffers on three internal streams and the direct kernels run on each
       chunk, overlapping the copies with the kernels, and results are copied
       back.  The first such call allocates the staging buffers (3 slots of
       about 9 x chunk_keys bytes) and keeps them until bf_destroy.
   Host keys need no alignment. */
bf_status bf_add_host(bf_filter* f, const uint64_t* h_keys, uint64_t n, bf_stream_t stream);
bf_status bf_contains_host(bf_filter* f, const uint64_t* h_keys, uint64_t n, uint8_t* h_out,
                           bf_stream_t stream);

/* Host-variant settings: keys per chunk of the chunked way (default 1<<24)
   and mode (BF_HOST_AUTO = as above, BF_HOST_STAGED = never read host
   memory from the kernels: copy-engine passes or chunks, BF_HOST_DIRECT =
   read it in place whenever the device can address it).
   Frees the current staging buffers; must not be called while host-variant
   work on this filter is in flight. */
typedef enum { BF_HOST_AUTO = 0, BF_HOST_STAGED = 1, BF_HOST_DIRECT = 2 } bf_host_mode;
bf_status bf_set_staging(bf_filter* f, uint64_t chunk_keys, int mode);

/* Raw bit array: device pointer and size in bytes (b*B/8).  Layout as in
   Sec. II-A (blocked) and Sec. II-A (sectorized): block j is words j*s ..
   j*s+s-1, each S-bit word little-endian, bit p = 1 << p; the array is the
   whole state of the filter (it can be saved and restored as bytes). */
bf_status bf_words(const bf_filter* f, void** d_ptr, uint64_t* nbytes);

/* Geometry of an existing filter. */
bf_status bf_get_params(const bf_filter* f, bf_params* out);

/* Select the layout of one operation (op = BF_OP_ADD or BF_OP_CONTAINS).  The
   construction layout also drives the record-insert kernel of the
   partitioned construction. */
bf_status bf_set_layout(bf_filter* f, int op, const bf_layout* layout);
bf_status bf_get_layout(const bf_filter* f, int op, bf_layout* out);

/* L2 persistence window over the bit array for `stream` (cache-resident
   filters, e.g. 32 MiB): sets the context's persisting-L2 limit to
   min(bytes, device maximum) and the stream's access-policy window with the
   given hit ratio.  hit_ratio <= 0 removes the window, resets persisting
   lines and sets the limit back to 0. */
bf_status bf_set_l2_persist(bf_filter* f, bf_stream_t stream, float hit_ratio);

/* Slice-partitioned construction and lookup (this library's addition; the
   paper's kernels are the direct ones).  For a filter larger than L2 the keys
   are hashed and radix-partitioned by filter slice (2^slice_log2 bytes of the
   bit array); then the slices are processed one L2-sized window
   (2^window_log2 bytes, at least one slice) per kernel launch, so the
   window's blocks are read and updated from L2 instead of HBM.
   Construction ORs each key's pattern into its block exactly as the direct
   kernel does (OR is commutative and idempotent: the same bits).  Lookup
   keeps each query's index with its record, sets one bit per positive query
   in a result bitmap, and expands the bitmap into the result bytes: the same
   answers as the direct kernel.  A key or query whose slice buffer is full
   is handled on the spot by the direct method, so any key distribution is
   handled.  The buffers (about 8 bytes per key of a construction pass; 12
   bytes per query plus a bit per query of a lookup pass) are allocated on
   first use and kept until bf_destroy; if an allocation fails the direct
   kernel runs.  Partitioning needs num_blocks <= 2^32 and more than one slice.
   mode (construction) and lookup_mode: BF_PART_OFF = direct kernel only;
   BF_PART_ON = partition whenever it applies; BF_PART_AUTO (default) =
   partition when the bit array is larger than half the L2 and the call has
   at least num_blocks/2 keys (construction) or num_blocks/4 queries (lookup).
   chunk_keys / lookup_chunk_keys: keys per pass (lookup default 2^28, so that
   the pass's result bitmap stays in L2).  cap_override: slots per slice
   buffer (0 = computed from the pass size; small values force the overflow
   path, for tests).
   passes: 0 or 1 = each pass of at most chunk_keys keys is partitioned, then
   its records inserted; >= 2 = the keys are split into at least this many
   passes over two alternating workspaces (twice the workspace of one such
   pass) and the phases overlap: the record inserts of pass i run on an
   internal stream while the partition of pass i + 1 runs on the caller's.
   part_ctas: partition CTAs per SM (0 = as many as fit; with passes >= 2 a
   smaller value leaves room for the record inserts beside the partition).
   The host-buffer variants always overlap, with at least max(8, passes)
   passes and part_ctas partition CTAs per SM (0 = one, enough for the
   CPU-GPU link). */
typedef enum { BF_PART_OFF = 0, BF_PART_ON = 1, BF_PART_AUTO = 2 } bf_part_mode;
typedef struct {
    uint32_t mode;               /* construction; default BF_PART_AUTO */
    uint32_t slice_log2;         /* 16..34; default 24 (16 MiB) */
    uint64_t chunk_keys;         /* >= 4096; default 2^32 */
    uint64_t cap_override;       /* 0 = computed; else a multiple of 128 */
    uint32_t window_log2;        /* 16..36; default 26 (64 MiB) */
    uint32_t lookup_mode;        /* default BF_PART_AUTO */
    uint64_t lookup_chunk_keys;  /* 4096..2^32; default 2^28 */
    uint32_t passes;             /* 0..64; default 0 (no overlap) */
    uint32_t part_ctas;          /* 0..8; default 0 */
} bf_partition;
bf_status bf_set_partition(bf_filter* f, const bf_partition* cfg);
bf_status bf_get_partition(const bf_filter* f, bf_partition* out);

/* Index checks of the slice-partitioned kernels.  Those kernels keep every
   index they derive from data inside its array (clamped, or checked before
   use); a failed check skips the access and sets a bit in a device status
   word of the filter -- 2: a record's block index beyond the filter (record
   insert, record probe), 8: a sorted record outside the slices (partition),
   16: a slice-buffer slot outside the buffers (partition) -- so no index can
   leave its buffer.  None of them fails when the kernels are correct; a
   nonzero value means the result of some call is incomplete.
   bf_device_status waits for `stream` (and the filter's internal stream),
   returns the bits accumulated since the last call in *codes (0 = none) and
   clears them. */
bf_status bf_device_status(bf_filter* f, bf_stream_t stream, uint32_t* codes);

/* Per-phase device time (a measurement aid).  After bf_set_timing(f, 1),
   every bf_add / bf_contains / host-buffer call records a CUDA event before
   and after each group of launches of one kind, on the stream that group
   runs on.  bf_get_timing waits for those events and returns, per phase, the
   summed duration of the groups recorded since the previous bf_get_timing (or
   bf_set_timing) in milliseconds and their number of launches, then starts a
   new sum.  Phases of the overlapped and staged schedules run concurrently,
   so their sums may exceed the calls' duration.  Timing costs two event
   records per group; bf_set_timing(f, 0) turns it off. */
enum {
    BF_PHASE_ADD_DIRECT = 0,        /* sbf_add_kernel (and the CSBF construction kernel) */
    BF_PHASE_CONTAINS_DIRECT = 1,   /* sbf_contains_kernel (and the CSBF lookup kernel) */
    BF_PHASE_PARTITION_ADD = 2,     /* slice partition of construction keys */
    BF_PHASE_RECORD_INSERT = 3,     /* record inserts, one launch per window */
    BF_PHASE_PARTITION_LOOKUP = 4,  /* slice partition of lookup queries */
    BF_PHASE_RECORD_PROBE = 5,      /* record probes, one launch per window */
    BF_PHASE_BITMAP_EXPAND = 6,     /* result bitmap to result bytes */
    BF_PHASE_HOST_STAGE = 7,        /* host keys into device staging slots on the copy-in stream of the
                                       staged host-buffer passes: staging kernels, or copy-engine copies
                                       (counted with 0 launches) */
    BF_PHASES = 8
};
typedef struct {
    float ms[BF_PHASES];
    uint32_t launches[BF_PHASES];
} bf_timing;
bf_status bf_set_timing(bf_filter* f, int enable);
bf_status bf_get_timing(bf_filter* f, bf_timing* out);

/* Kernel launches made by the last bf_add / bf_contains / bf_add_host /
   bf_contains_host call on this filter (1 for a direct call; per pass of a
   partitioned construction, one partition launch plus one record-insert
   launch per window; per chunk for the staged host variants). */
bf_status bf_last_launches(const bf_filter* f, uint32_t* n);

/* Random-access microbenchmark that bounds the filter kernels (Sec. V-B
   measures the bound with random 64-bit accesses, GUPS).  For each i in
   [0, n): u = unit index taken from d_keys[i] by the same multiply-shift
   rule as the block index, over table_bytes / unit_bytes units;
     mode BF_GUPS_LOAD:   load the unit_bytes at u (32-byte vector loads; 8-byte
                          load when unit_bytes = 8), fold them to one byte and
                          store it to d_out[i];
     mode BF_GUPS_RED_OR: one red.global.or of a 32-bit value derived from
                          d_keys[i] into each 32-byte sector of unit u;
     mode BF_GUPS_RED_OR_SECTOR: the record-insert kernel's traffic: each
                          32-byte sector of unit u receives four 64-bit
                          red.global.or (from four lanes, one instruction),
                          i.e. one full-width update of its eight 32-bit words.
   unit_bytes in {8, 32, 64, 128}; d_table aligned to unit_bytes; layout uses
   kpt, block_threads and grid_ctas (cg/phi ignored). */
typedef enum { BF_GUPS_LOAD = 0, BF_GUPS_RED_OR = 1, BF_GUPS_RED_OR_SECTOR = 2 } bf_gups_mode;
bf_status bf_gups(int mode, void* d_table, uint64_t table_bytes, uint32_t unit_bytes,
                  const uint64_t* d_keys, uint64_t n, uint8_t* d_out, const bf_layout* layout,
                  bf_stream_t stream);

/* Batched filters (an extension of the paper's bulk operations to many
   independent filters): one launch builds, or probes, every filter of
   a batch.  All filters share params->block_bits / word_bits / k / seed
   (params->num_blocks is ignored); each has its own bit array and its own
   run [key_offset, key_offset + key_count) of one key array, and lookup
   results use the same indexing in one result array.  Per filter the bits
   and answers are exactly those of bf_add / bf_contains on that filter
   (Sec. II-A).  bf_batch_create copies the descriptors to the device (a
   blocking copy) and resolves kernels and grids; bf_batch_add /
   bf_batch_contains then only enqueue one kernel each, so they can be
   captured into a CUDA graph and replayed.  Filters may share bit arrays or
   key runs (ORs commute); filters with key_count = 0 are skipped. */
typedef struct bf_batch bf_batch;
typedef struct {
    void* d_words;         /* num_blocks * block_bits / 8 bytes, aligned to max(32, block_bits/8) */
    uint64_t num_blocks;
    uint64_t key_offset;
    uint64_t key_count;
} bf_batch_filter;
bf_status bf_batch_create(const bf_params* params, const bf_batch_filter* h_filters, uint32_t nfilters,
                          bf_batch** out);
bf_status bf_batch_destroy(bf_batch* b);
bf_status bf_batch_set_layout(bf_batch* b, int op, const bf_layout* layout);
bf_status bf_batch_get_layout(const bf_batch* b, int op, bf_layout* out);
bf_status bf_batch_add(bf_batch* b, const uint64_t* d_keys, bf_stream_t stream);
bf_status bf_batch_contains(const bf_batch* b, const uint64_t* d_keys, uint8_t* d_out, bf_stream_t stream);
/* Number of filters, and the length the key / result arrays must have. */
bf_status bf_batch_info(const bf_batch* b, uint32_t* nfilters, uint64_t* total_keys);

/* Lookup server (an extension of the bulk lookup to request traffic): many
   device-resident filters of one geometry (sectorized), lookup requests
   (filter, host keys, host results) arriving over time.  A worker thread
   admits pending requests in arrival order while a device key arena of
   arena_keys slots, the per-launch request limit and the launch's share of
   the arena (a quarter; a larger request goes alone) have room, copies their
   keys in, runs one batched lookup launch over all of them (across filters),
   copies each request's results back, and frees the arena in completion
   order; up to four launches are in flight.  When the kernels can address
   every request's buffers of a launch (pinned memory, or any host memory on
   a GPU with pageable memory access, and 8-byte aligned keys), staging
   kernels on high-priority streams gather the keys and scatter the results;
   otherwise the copy engine copies each request's keys and results.
   Answers are those of bf_contains on the request's filter.  Host buffers
   must stay valid until the request completes.
   bf_server_create allocates the arena (9 bytes per slot) and a stream and
   starts the worker; bf_server_destroy completes in-flight work and stops it. */
typedef struct bf_server bf_server;
typedef struct {
    uint64_t requests;     /* completed since the last reset */
    uint64_t keys;
    uint64_t launches;
    double p50_s, p99_s, mean_s, max_s;  /* request latency: submit -> results on the host */
    double span_s;         /* first submit -> last completion */
    double offered_s;      /* bf_server_run_poisson: the arrival window */
    /* device time summed over the completed launches (CUDA events on each
       stream): keys into the arena, batched lookup kernels, results out */
    double stage_in_s, lookup_s, stage_out_s;
} bf_server_stats;
bf_status bf_server_create(const bf_params* params, const bf_batch_filter* filters /* d_words, num_blocks */,
                           uint32_t nfilters, uint64_t arena_keys, uint32_t max_requests_per_launch,
                           bf_server** out);
bf_status bf_server_destroy(bf_server* s);
/* Queue a lookup of n keys of filter `filter` (n <= arena_keys); *ticket identifies it. */
bf_status bf_server_submit(bf_server* s, uint32_t filter, const uint64_t* h_keys, uint64_t n, uint8_t* h_out,
                           uint64_t* ticket);
/* Block until the request is complete (BF_OK, its latency in *latency_s if not NULL),
   timeout_s passes (BF_ETIMEDOUT) or a CUDA error occurred (BF_ECUDA).  A completed
   ticket is forgotten. */
bf_status bf_server_wait(bf_server* s, uint64_t ticket, double timeout_s, double* latency_s);
/* Counters and latency percentiles of the requests completed since the last reset. */
bf_status bf_server_get_stats(bf_server* s, int reset, bf_server_stats* out);
/* Load generator: for duration_s seconds, requests arrive as a Poisson process of
   rate_per_s; each picks a filter uniformly and log-uniform(min_keys, max_keys) keys,
   taken as consecutive runs of the pinned host pool h_key_pool (results to the same
   runs of h_out_pool); waits for all, then reports their statistics (SplitMix64 seed). */
bf_status bf_server_run_poisson(bf_server* s, double rate_per_s, double duration_s, uint64_t min_keys,
                                uint64_t max_keys, const uint64_t* h_key_pool, uint64_t pool_keys,
                                uint8_t* h_out_pool, uint64_t seed, bf_server_stats* out);

/* Construction that allocates nothing (the paper has no counterpart: this is
   an interface for callers of this library).  Some callers cannot let a
   library call cudaMalloc -- services whose own caching allocator owns the
   GPU's free memory, and latency-critical loops that must not pay for the
   device synchronization cudaMalloc / cudaFree imply.  bf_add_noalloc sets
   the same bits as bf_add (slice-partitioned construction with the default
   layout) into the caller's bit array d_words (geometry `params`, alignment as
   for bf_create), with its scratch in one 16 MiB array that the library keeps
   on every GPU that loads it, until the process exits.  No filter handle is
   needed.
   Limits: num_blocks <= 2^32, and n must fit the array: *max_keys (if not
   NULL) receives the largest n accepted for this geometry (from about 2.08
   million keys for a filter of one 16 MiB slice down to about 1.40 million
   for 1024 slices), and a larger n returns BF_EINVAL with nothing enqueued --
   split the keys over several calls.
   Every call shares the one array (the call clears the counters it needs):
   calls whose work overlaps on the GPU -- other streams, other host threads --
   race and corrupt each other's scratch; serialize them.  The first call on
   each device looks up the array's device address (cudaGetSymbolAddress) with
   that device current; make that first call before any stream capture.
   Errors are reported by the status only (bf_last_error is not updated). */
bf_status bf_add_noalloc(const bf_params* params, void* d_words, const uint64_t* d_keys, uint64_t n,
                         uint64_t* max_keys, bf_stream_t stream);

/* The index-check bits (as for bf_device_status) that bf_add_noalloc calls on
   the current device have accumulated in the shared array since the last
   bf_noalloc_status; clears them.  A synchronous copy: call it once those
   calls have completed. */
bf_status bf_noalloc_status(uint32_t* codes);

/* ---------------------------------------------------------------------------
   Learned prefilter (an extension beside the paper's filters; the paper has no
   learned component).  A small network over the 64 bits of a key -- inputs
   x_i = (key >> i) & 1, layers 64 -> 128 -> 64 -> 1 with ReLU -- scores keys;
   a key is reported present when its score reaches the threshold tau or when
   a backup blocked filter (bf_create / bf_add), which holds the members the
   network scores below tau, contains it.  No false negatives by
   construction.
   Training is in fp32 on the GPU (mean binary cross-entropy of the logit,
   Adam), with the three weight matrices fake-quantized in the forward pass:
   W -> s * clamp(round(W / s), -127, 127), s = max|W| / 127, rounding half
   away from zero, the quotient and rounding taken in fp64; the gradient
   passes straight through the rounding.
   Parameter vector (BF_MLP_PARAMS fp32 values, device memory, caller-owned):
   W1 [64][128] row-major (input-major), b1 [128], W2 [128][64], b2 [64],
   W3 [64], b3.
   The exported integer model computes exactly:
     a1 = x . W1q + b1q,   h1 = min(max(a1, 0) >> sh1, 127)
     a2 = h1 . W2q + b2q,  h2 = min(max(a2, 0) >> sh2, 127)
     score = h2 . W3q + b3q, saturated to int32
   with int8 weights Wq = clamp(round(W / s)), biases rounded to the units of
   their layer's accumulator (s1; s1 2^sh1 s2; s1 2^sh1 s2 2^sh2 s3) and
   saturated to int32, and sh1 / sh2 the smallest shifts that bring the
   largest max(a, 0) of their layer over the calibration keys to <= 127.
   ------------------------------------------------------------------------- */
#define BF_MLP_PARAMS 16641

typedef struct {
    int8_t w1[64 * 128]; /* W1q[i][j] at i * 128 + j */
    int8_t w2[128 * 64]; /* W2q[i][j] at i * 64 + j */
    int8_t w3[64];
    int32_t b1[128];
    int32_t b2[64];
    int32_t b3;
    int32_t sh1, sh2;
    double unit; /* value of one score unit in logit units */
} bf_mlp_int8;

typedef struct bf_mlp_model bf_mlp_model;

/* Device workspace a training call needs for `batch` samples (bytes). */
uint64_t bf_mlp_workspace_bytes(uint32_t batch);

/* Gradient of the mean loss over one batch into d_grads (BF_MLP_PARAMS
   floats) and the loss into *d_loss (if not NULL).  The training set is
   d_keys / d_labels (n <= 2^32 - 1 entries, labels 0.0 or 1.0); sample i of
   the batch is element ((first + i) mod n) * mult mod n, so with mult coprime
   to n (1 <= mult < 2^32; else BF_EINVAL) n consecutive samples visit every
   element once.  d_ws: bf_mlp_workspace_bytes(batch) bytes, 256-byte aligned. */
bf_status bf_mlp_grad(const float* d_params, const uint64_t* d_keys, const float* d_labels, uint64_t n,
                      uint64_t first, uint64_t mult, uint32_t batch, float* d_grads, float* d_loss, void* d_ws,
                      uint64_t ws_bytes, bf_stream_t stream);

/* One Adam step (step >= 1 counts from 1):  m = b1 m + (1-b1) g,
   v = b2 v + (1-b2) g^2,  p -= lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps). */
bf_status bf_mlp_adam(float* d_params, const float* d_grads, float* d_m, float* d_v, uint32_t step, float lr,
                      float beta1, float beta2, float eps, bf_stream_t stream);

/* `steps` training steps (gradient + Adam) numbered first_step, first_step+1,
   ...; step t uses the batch that starts at sample (t-1)*batch.  Per-step
   losses into d_loss[0..steps) if not NULL.  Enqueued only. */
bf_status bf_mlp_train(float* d_params, float* d_m, float* d_v, const uint64_t* d_keys, const float* d_labels,
                       uint64_t n, uint64_t mult, uint32_t batch, uint32_t first_step, uint32_t steps, float lr,
                       float beta1, float beta2, float eps, float* d_loss, void* d_ws, uint64_t ws_bytes,
                       bf_stream_t stream);

/* Export the host parameter vector h_params to the integer model *out,
   calibrating the shifts on the device keys d_calib[0..n_calib).
   Synchronizes `stream`. */
bf_status bf_mlp_export(const float* h_params, const uint64_t* d_calib, uint64_t n_calib, bf_mlp_int8* out,
                        bf_stream_t stream);

/* Copy an integer model to the current device (BF_EINVAL for shifts outside 0..62). */
bf_status bf_mlp_load(const bf_mlp_int8* m, bf_mlp_model** out);
bf_status bf_mlp_free(bf_mlp_model* m);

/* Engines of the integer model.  TENSOR: tcgen05 MMAs in bf16 with fp32
   accumulation on values for which that arithmetic is exact (models whose
   shifts sh1, sh2 are <= 15); DP4A: CUDA-core int8 dot products.  Both give
   the integer model's results bit for bit.  AUTO (default) takes TENSOR when
   the model allows it. */
#define BF_MLP_ENGINE_AUTO 0
#define BF_MLP_ENGINE_TENSOR 1
#define BF_MLP_ENGINE_DP4A 2
/* BF_EUNSUPPORTED when TENSOR is asked of a model that does not allow it. */
bf_status bf_mlp_set_engine(bf_mlp_model* m, int engine);
/* The engine lookups of this model use (TENSOR or DP4A). */
bf_status bf_mlp_get_engine(const bf_mlp_model* m, int* engine);
/* Synchronizes the device; BF_ETIMEDOUT if a bounded wait of a tensor-core
   launch of this model ran out (its results are then incomplete). */
bf_status bf_mlp_check(const bf_mlp_model* m);

/* Integer scores of n device keys into d_scores (int32). */
bf_status bf_mlp_scores(const bf_mlp_model* m, const uint64_t* d_keys, uint64_t n, int32_t* d_scores,
                        bf_stream_t stream);

/* Compaction: the keys whose score is below tau, in no particular order, into
   d_out_keys (room for n keys), their number into *d_count (device). */
bf_status bf_mlp_select_below(const bf_mlp_model* m, int32_t tau, const uint64_t* d_keys, uint64_t n,
                              uint64_t* d_out_keys, uint64_t* d_count, bf_stream_t stream);

/* Learned-filter lookup: d_out[i] = (score(key_i) >= tau) || backup contains key_i. */
bf_status bf_mlp_contains(const bf_mlp_model* m, int32_t tau, const bf_filter* backup, const uint64_t* d_keys,
                          uint64_t n, uint8_t* d_out, bf_stream_t stream);

/* The same from host buffers (pinned for overlap): chunks of 2^24 keys are
   copied in, looked up and copied out on three internal streams that follow
   `stream` and are joined back into it.  The model keeps the staging
   buffers (3 x 144 MiB of device memory) from the first call until
   bf_mlp_free.  Calls on one model must not overlap. */
bf_status bf_mlp_contains_host(bf_mlp_model* m, int32_t tau, const bf_filter* backup, const uint64_t* h_keys,
                               uint64_t n, uint8_t* h_out, bf_stream_t stream);

/* Measured cost of back-to-back 5th-generation tensor-core MMAs (tcgen05.mma
   kind::f16, M = 128, K = 16, bf16 operands, fp32 accumulation) with n
   columns (16, 32, 64, 128 or 256), A from shared memory (a_tmem = 0) or
   tensor memory (1): one issuing thread per SM on every SM issues `reps`
   instructions (1 <= reps <= 2^24); *cycles = SM clock cycles per
   instruction.  The learned prefilter's tile is a fixed set of such
   instructions, so this bounds its throughput (as bf_gups bounds the
   filters').  Synchronizes the device; BF_ETIMEDOUT if the instructions did
   not complete within 2 s. */
bf_status bf_mma_cost(uint32_t n, int a_tmem, uint32_t reps, double* cycles);

const char* bf_status_str(bf_status s);

/* Message of the last error on the calling host thread ("" if none). */
const char* bf_last_error(void);

/* Library version string. */
const char* bf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BLOOMGB_H */
