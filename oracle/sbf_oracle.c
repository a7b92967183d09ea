/*
 * Plain CPU oracle for the sectorized blocked Bloom filter (SBF).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library: every step below is written out again from
 * its definition, one key at a time, with no blocking, fusion or reordering.
 *
 * Definitions followed (paper: "Optimizing Bloom Filters on Modern GPUs"):
 *   - Sec. II-A (CBF, BBF, SBF): a filter of b blocks of B bits; a key selects
 *     one block; the block is s = B/S machine words of S bits; the k pattern
 *     bits of a key are spread evenly, k' = k/s bits per word; construction
 *     sets the bits, lookup reports membership iff all of them are set.
 *   - Sec. IV-B: one 64-bit base hash per key (xxHash, 64-bit variant); each
 *     pattern bit position comes from multiplying the base hash by an odd
 *     constant (a salt) and keeping the high bits of the product.
 *
 * Readings taken where the paper is silent (each is also listed in the
 * design notes):
 *   - base hash: XXH64 over the 8 little-endian bytes of the key, written
 *     here for inputs of any length from the public xxHash specification;
 *   - block index: j = ((h >> 32) * b) >> 32 when b <= 2^32, otherwise the
 *     high 64 bits of the 128-bit product h * b;
 *   - pattern hash: h_lo = low 32 bits of h; for S = 32 the bit is
 *     ((h_lo * salt32) mod 2^32) >> 27, for S = 64 it is
 *     ((h_lo * salt64) mod 2^64) >> 58;
 *   - salt i of the 64-bit table is (i-th output of SplitMix64 seeded with
 *     0x5A175EED) | 1; salt i of the 32-bit table is (salt64_i >> 32) | 1;
 *   - bit t (t = 0..k'-1) of word w (w = 0..s-1) uses salt index w + s*t;
 *   - a word's bit p is the value 1 << p (bit 0 = least significant); block
 *     j occupies words j*s .. j*s+s-1; words are stored little-endian.
 *
 * Cache-sectorized form (Sec. II-A, CSBF; Sec. V-A for the extra multiplier),
 * selected by groups = z with 0 < z < s: the s words form z groups of
 * g = s/z neighbouring words; in group q one word is selected, and it
 * receives k/z bits.  Readings:
 *   - the selected word of group q is q*g + sel, with sel the top log2(g)
 *     bits of (h_lo * salt[63 - q]) (mod 2^32 for S = 32, mod 2^64 for
 *     S = 64): "another odd multiplier", taken from the top of the table;
 *   - bit t (t = 0..k/z-1) of group q uses salt index q + z*t (with z = s
 *     this is the sectorized rule, and the two forms coincide);
 *   - k must be a multiple of z and k + z <= 64 (the pattern and selection
 *     multipliers then never share a table entry).
 *
 * Salt set 1 (salts = 1, only B = 256, S = 32, k = 8, sectorized): the
 * multipliers are those of the Apache Parquet split-block Bloom filter, so
 * the bit array is the one a Parquet writer stores for the same keys and
 * block count (the paper's compatibility claim, Sec. VI); everything else
 * above is unchanged.
 */
#include <stddef.h>
#include <stdint.h>

/* ---------------------------------------------------------------------- */
/* xxHash64, general input length (xxHash specification, XXH64 section)     */
/* ---------------------------------------------------------------------- */
#define XXP1 0x9E3779B185EBCA87ULL
#define XXP2 0xC2B2AE3D27D4EB4FULL
#define XXP3 0x165667B19E3779F9ULL
#define XXP4 0x85EBCA77C2B2AE63ULL
#define XXP5 0x27D4EB2F165667C5ULL

static uint64_t rotate_left(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

static uint64_t load_le64(const uint8_t* p)
{
    uint64_t v = 0;
    for (int i = 7; i >= 0; --i) v = (v << 8) | (uint64_t)p[i];
    return v;
}

static uint64_t load_le32(const uint8_t* p)
{
    uint64_t v = 0;
    for (int i = 3; i >= 0; --i) v = (v << 8) | (uint64_t)p[i];
    return v;
}

/* one accumulator round: acc + lane*P2, rotate by 31, times P1 */
static uint64_t xxh64_round(uint64_t acc, uint64_t lane)
{
    acc = acc + lane * XXP2;
    acc = rotate_left(acc, 31);
    return acc * XXP1;
}

/* fold one of the four stripe accumulators into the running value */
static uint64_t xxh64_merge(uint64_t acc, uint64_t stripe_acc)
{
    acc = acc ^ xxh64_round(0, stripe_acc);
    return acc * XXP1 + XXP4;
}

uint64_t orc_xxh64(const uint8_t* input, uint64_t len, uint64_t seed)
{
    const uint8_t* p = input;
    uint64_t left = len;
    uint64_t acc;

    if (len >= 32) {
        uint64_t a1 = seed + XXP1 + XXP2;
        uint64_t a2 = seed + XXP2;
        uint64_t a3 = seed;
        uint64_t a4 = seed - XXP1;
        while (left >= 32) {
            a1 = xxh64_round(a1, load_le64(p));
            a2 = xxh64_round(a2, load_le64(p + 8));
            a3 = xxh64_round(a3, load_le64(p + 16));
            a4 = xxh64_round(a4, load_le64(p + 24));
            p += 32;
            left -= 32;
        }
        acc = rotate_left(a1, 1) + rotate_left(a2, 7) + rotate_left(a3, 12) + rotate_left(a4, 18);
        acc = xxh64_merge(acc, a1);
        acc = xxh64_merge(acc, a2);
        acc = xxh64_merge(acc, a3);
        acc = xxh64_merge(acc, a4);
    } else {
        acc = seed + XXP5;
    }

    acc = acc + len;

    while (left >= 8) {
        acc = acc ^ xxh64_round(0, load_le64(p));
        acc = rotate_left(acc, 27) * XXP1 + XXP4;
        p += 8;
        left -= 8;
    }
    if (left >= 4) {
        acc = acc ^ (load_le32(p) * XXP1);
        acc = rotate_left(acc, 23) * XXP2 + XXP3;
        p += 4;
        left -= 4;
    }
    while (left > 0) {
        acc = acc ^ ((uint64_t)(*p) * XXP5);
        acc = rotate_left(acc, 11) * XXP1;
        p += 1;
        left -= 1;
    }

    /* avalanche */
    acc = acc ^ (acc >> 33);
    acc = acc * XXP2;
    acc = acc ^ (acc >> 29);
    acc = acc * XXP3;
    acc = acc ^ (acc >> 32);
    return acc;
}

/* base hash of a 64-bit key: XXH64 of its 8 little-endian bytes */
uint64_t orc_key_hash(uint64_t key, uint64_t seed)
{
    uint8_t bytes[8];
    for (int i = 0; i < 8; ++i) bytes[i] = (uint8_t)(key >> (8 * i));
    return orc_xxh64(bytes, 8, seed);
}

/* ---------------------------------------------------------------------- */
/* salts                                                                    */
/* ---------------------------------------------------------------------- */
#define ORC_SALT_SEED 0x5A175EEDULL
#define ORC_MAX_SALTS 64

static uint64_t splitmix64_next(uint64_t* state)
{
    uint64_t z;
    *state = *state + 0x9E3779B97F4A7C15ULL;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* the 64-entry table is filled once, when the library is loaded */
static uint64_t salt64_table[ORC_MAX_SALTS];

__attribute__((constructor)) static void fill_salt_table(void)
{
    uint64_t state = ORC_SALT_SEED;
    for (uint32_t i = 0; i < ORC_MAX_SALTS; ++i) salt64_table[i] = splitmix64_next(&state) | 1ULL;
}

uint64_t orc_salt64(uint32_t i)
{
    return salt64_table[i];
}

uint32_t orc_salt32(uint32_t i)
{
    return (uint32_t)(orc_salt64(i) >> 32) | 1u;
}

/* Salt set 1: the eight odd multipliers of the Apache Parquet split-block
   filter (256-bit blocks of eight 32-bit words, one bit per word), which the
   paper's filter with B = 256, S = 32, k = 8 reproduces bit for bit (Sec. VI).
   The values are not in the paper; they were recovered from the bit arrays
   pyarrow's Parquet writer produces (tests/test_oracle_hash_pins.py recovers
   them again on every run and compares). */
static const uint32_t parquet_salt32[8] = {
    0x47B6137Bu, 0x44974D91u, 0x8824AD5Bu, 0xA2B7289Du,
    0x705495C7u, 0x2DF1424Bu, 0x9EFC4947u, 0x5C6BFB31u,
};

uint32_t orc_parquet_salt32(uint32_t i)
{
    return i < 8 ? parquet_salt32[i] : 0u;
}

/* ---------------------------------------------------------------------- */
/* block selection and bit positions                                        */
/* ---------------------------------------------------------------------- */
uint64_t orc_block_index(uint64_t h, uint64_t num_blocks)
{
    if (num_blocks <= (1ULL << 32)) return ((h >> 32) * num_blocks) >> 32;
    return (uint64_t)(((unsigned __int128)h * num_blocks) >> 64);
}

uint32_t orc_bit_position(uint64_t h, uint32_t salt_index, uint32_t word_bits)
{
    uint64_t h_lo = h & 0xFFFFFFFFULL;
    if (word_bits == 32) {
        uint32_t product = (uint32_t)(h_lo * (uint64_t)orc_salt32(salt_index));
        return product >> 27;
    }
    return (uint32_t)((h_lo * orc_salt64(salt_index)) >> 58);
}

/* ---------------------------------------------------------------------- */
/* filter                                                                   */
/* ---------------------------------------------------------------------- */
typedef struct {
    uint64_t num_blocks;
    uint32_t block_bits;
    uint32_t word_bits;
    uint32_t k;
    uint32_t groups;    /* z: 0 (or s) = sectorized; 0 < z < s = cache-sectorized */
    uint64_t seed;
    uint32_t salts;     /* 0: SplitMix64 salts; 1: the Parquet split-block salts */
    uint32_t reserved;
} orc_params;

/* bit position of salt index i under the geometry's salt set */
static uint32_t bit_position_p(const orc_params* p, uint64_t h, uint32_t salt_index)
{
    if (p->salts == 1) {
        uint64_t h_lo = h & 0xFFFFFFFFULL;
        return (uint32_t)(h_lo * (uint64_t)orc_parquet_salt32(salt_index)) >> 27;
    }
    return orc_bit_position(h, salt_index, p->word_bits);
}

static uint32_t effective_groups(const orc_params* p)
{
    uint32_t s = p->block_bits / p->word_bits;
    return (p->groups == 0) ? s : p->groups;
}

/* 0 if the geometry is one the definitions admit, else -1.
   SBF (Sec. II-A): s = B/S words, k >= s and s | k.
   CSBF (Sec. II-A): z groups with z | s, z | k, and k + z <= 64. */
int orc_check(const orc_params* p)
{
    if (p->num_blocks == 0) return -1;
    if (p->word_bits != 32 && p->word_bits != 64) return -1;
    if (p->block_bits < p->word_bits || p->block_bits % p->word_bits != 0) return -1;
    uint32_t s = p->block_bits / p->word_bits;
    uint32_t z = effective_groups(p);
    if (z == 0 || z > s || s % z != 0) return -1;
    if (p->k < z || p->k % z != 0) return -1;
    if (p->k > ORC_MAX_SALTS) return -1;
    if (z < s && p->k + z > ORC_MAX_SALTS) return -1;
    if (p->salts > 1) return -1;
    if (p->salts == 1 && !(p->block_bits == 256 && p->word_bits == 32 && p->k == 8 && z == s)) return -1;
    return 0;
}

/* word of group q selected by h (CSBF); for groups of one word it is that word */
uint32_t orc_group_word(const orc_params* p, uint64_t h, uint32_t q)
{
    uint32_t s = p->block_bits / p->word_bits;
    uint32_t z = effective_groups(p);
    uint32_t g = s / z;
    uint32_t log2g = 0;
    while ((1u << log2g) < g) log2g++;
    if (log2g == 0) return q;
    uint64_t h_lo = h & 0xFFFFFFFFULL;
    uint32_t sel;
    if (p->word_bits == 32) {
        uint32_t product = (uint32_t)(h_lo * (uint64_t)orc_salt32(63 - q));
        sel = product >> (32 - log2g);
    } else {
        sel = (uint32_t)((h_lo * orc_salt64(63 - q)) >> (64 - log2g));
    }
    return q * g + sel;
}

/* pattern of the selected word of group q: the OR of its k/z bits */
uint64_t orc_group_pattern(const orc_params* p, uint64_t h, uint32_t q)
{
    uint32_t z = effective_groups(p);
    uint32_t kz = p->k / z;
    uint64_t pattern = 0;
    for (uint32_t t = 0; t < kz; ++t) pattern |= 1ULL << bit_position_p(p, h, q + z * t);
    return pattern;
}

static uint64_t word_get(const void* words, uint32_t word_bits, uint64_t index)
{
    if (word_bits == 32) return ((const uint32_t*)words)[index];
    return ((const uint64_t*)words)[index];
}

static void word_or(void* words, uint32_t word_bits, uint64_t index, uint64_t bits)
{
    if (word_bits == 32) ((uint32_t*)words)[index] |= (uint32_t)bits;
    else ((uint64_t*)words)[index] |= bits;
}

/* pattern of word w of the block chosen by h: the OR of its k' bits */
uint64_t orc_word_pattern(const orc_params* p, uint64_t h, uint32_t w)
{
    uint32_t s = p->block_bits / p->word_bits;
    uint32_t kp = p->k / s;
    uint64_t pattern = 0;
    for (uint32_t t = 0; t < kp; ++t) {
        uint32_t bit = bit_position_p(p, h, w + s * t);
        pattern |= 1ULL << bit;
    }
    return pattern;
}

int orc_add(const orc_params* p, void* words, const uint64_t* keys, uint64_t n)
{
    if (orc_check(p) != 0) return -1;
    uint32_t s = p->block_bits / p->word_bits;
    uint32_t z = effective_groups(p);
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t h = orc_key_hash(keys[i], p->seed);
        uint64_t j = orc_block_index(h, p->num_blocks);
        for (uint32_t q = 0; q < z; ++q)
            word_or(words, p->word_bits, j * s + orc_group_word(p, h, q), orc_group_pattern(p, h, q));
    }
    return 0;
}

/* Construction restricted to the blocks [block_lo, block_hi): keys whose
   block lies outside are skipped; `words` holds only that slice. */
int orc_add_block_range(const orc_params* p, void* words, uint64_t block_lo, uint64_t block_hi,
                        const uint64_t* keys, uint64_t n)
{
    if (orc_check(p) != 0) return -1;
    uint32_t s = p->block_bits / p->word_bits;
    uint32_t z = effective_groups(p);
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t h = orc_key_hash(keys[i], p->seed);
        uint64_t j = orc_block_index(h, p->num_blocks);
        if (j < block_lo || j >= block_hi) continue;
        for (uint32_t q = 0; q < z; ++q)
            word_or(words, p->word_bits, (j - block_lo) * s + orc_group_word(p, h, q), orc_group_pattern(p, h, q));
    }
    return 0;
}

int orc_contains(const orc_params* p, const void* words, const uint64_t* keys, uint64_t n, uint8_t* out)
{
    if (orc_check(p) != 0) return -1;
    uint32_t s = p->block_bits / p->word_bits;
    uint32_t z = effective_groups(p);
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t h = orc_key_hash(keys[i], p->seed);
        uint64_t j = orc_block_index(h, p->num_blocks);
        int member = 1;
        for (uint32_t q = 0; q < z; ++q) {
            uint64_t pattern = orc_group_pattern(p, h, q);
            if ((word_get(words, p->word_bits, j * s + orc_group_word(p, h, q)) & pattern) != pattern) member = 0;
        }
        out[i] = (uint8_t)member;
    }
    return 0;
}

/* Lookup against the slice [block_lo, block_hi); keys whose block lies
   outside the slice get 2 (not decided here). */
int orc_contains_block_range(const orc_params* p, const void* words, uint64_t block_lo,
                             uint64_t block_hi, const uint64_t* keys, uint64_t n, uint8_t* out)
{
    if (orc_check(p) != 0) return -1;
    uint32_t s = p->block_bits / p->word_bits;
    uint32_t z = effective_groups(p);
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t h = orc_key_hash(keys[i], p->seed);
        uint64_t j = orc_block_index(h, p->num_blocks);
        if (j < block_lo || j >= block_hi) { out[i] = 2; continue; }
        int member = 1;
        for (uint32_t q = 0; q < z; ++q) {
            uint64_t pattern = orc_group_pattern(p, h, q);
            uint64_t idx = (j - block_lo) * s + orc_group_word(p, h, q);
            if ((word_get(words, p->word_bits, idx) & pattern) != pattern) member = 0;
        }
        out[i] = (uint8_t)member;
    }
    return 0;
}

/* Each key's own contribution: its block index in out_block[i] and the s
   words of that block with only this key's pattern set, in
   out_words[i*s .. i*s+s-1] (S-bit words).  Construction is the OR of these
   images into their blocks; used to check very sparse filters block by block
   without a full-size array. */
int orc_key_blocks(const orc_params* p, const uint64_t* keys, uint64_t n, uint64_t* out_block, void* out_words)
{
    if (orc_check(p) != 0) return -1;
    uint32_t s = p->block_bits / p->word_bits;
    uint32_t z = effective_groups(p);
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t h = orc_key_hash(keys[i], p->seed);
        out_block[i] = orc_block_index(h, p->num_blocks);
        for (uint32_t w = 0; w < s; ++w) {
            if (p->word_bits == 32) ((uint32_t*)out_words)[i * s + w] = 0;
            else ((uint64_t*)out_words)[i * s + w] = 0;
        }
        for (uint32_t q = 0; q < z; ++q)
            word_or(out_words, p->word_bits, i * s + orc_group_word(p, h, q), orc_group_pattern(p, h, q));
    }
    return 0;
}

/* per-key base hash and block index, for statistics tests */
void orc_hash_keys(const uint64_t* keys, uint64_t n, uint64_t seed, uint64_t* out)
{
    for (uint64_t i = 0; i < n; ++i) out[i] = orc_key_hash(keys[i], seed);
}

void orc_block_indices(const uint64_t* keys, uint64_t n, uint64_t seed, uint64_t num_blocks, uint64_t* out)
{
    for (uint64_t i = 0; i < n; ++i) out[i] = orc_block_index(orc_key_hash(keys[i], seed), num_blocks);
}
