// Learned prefilter, integer model on the 5th-generation tensor cores.
//
// The exported model is integer arithmetic (int8 weights, ReLU + shift +
// saturation, int32 score).  sm_103a has no int8 tensor-core MMA, so the two
// matrix products run as bf16 MMAs with fp32 accumulation (tcgen05.mma
// kind::f16) on values chosen so that every product and every partial sum is
// an exactly representable integer multiple of a power of two:
//   * A1 = the key bits (0/1), B1 = W1q * 2^-sh1 (int8 times a power of two:
//     exact in bf16); |sum x W1q| <= 64 * 127.
//   * a per-unit constant c1 = (b1' + 128 * 2^sh1) 2^-sh1 (b1' = b1q
//     clamped to the range where it still changes the result) is the first
//     product of the layer: one more MMA of K = 16 over a constant A (1.0 in
//     k = 0..2) and B = the three bf16 parts of c1 (an integer below 2^24
//     times 2^-sh1 is the sum of three 8-bit parts, each exact), so
//     y1 = 128 + a1 / 2^sh1 exactly; the epilogue converts to bf16 rounding
//     toward zero (the bf16 spacing on [128, 256) is 1, so this is the floor)
//     and clamps to [128, 255]: A2 = 128 + h1, exact in bf16.
//   * B2 = W2q * 2^-sh2; the offset 128 * colsum(W2q) is folded into c2
//     (added by the layer's bias MMA the same way), and
//     likewise 128 + h2 (exact in bf16 and fp32) is dotted with W3q on the
//     CUDA cores in fp32 (integer partial sums below 2^24), score = acc3 +
//     (b3q - 128 sum W3q).
// Every magnitude stays below 2^24 when sh1, sh2 <= 15 (checked on the host;
// other models use the dp4a kernel), so the results equal the integer
// model's bit for bit.
//
// Kernel shape: persistent, one CTA per SM, warp-specialized: four epilogue
// warpgroups and one MMA warp.  Each warpgroup owns 16 KiB of shared memory
// (A1) and 128 TMEM columns and walks its tiles of 128 keys (one key per
// thread, one TMEM lane per key): it writes A1 and signals the MMA warp,
// waits for L1, requantizes (TMEM -> registers -> TMEM), signals, writes the
// next tile's A1 while L2 runs, waits for L2, finishes layer 3 and the score,
// and releases its TMEM columns to the next L1.  The MMA warp's elected thread
// issues every product (L1 of each warpgroup, then L2 of each, in turn) and
// commits it to that warpgroup's mbarrier, so no epilogue thread ever blocks
// on issuing MMAs.
// All waits are bounded (2 s); a time-out sets the model's error word.
// TMEM columns of a warpgroup over one tile:
//   L1: D1 -> 0..127;  E1: A2 (128 bf16 = 64 columns) -> 0..63;
//   L2: A = 0..63 (A from tensor memory), D2 -> 64..127;  E2: reads 64..127.
// Shared-memory operands (A1, B1, B2) use the K-major 128-byte-swizzled
// layout (8-row groups of 128-byte rows, 16-byte chunks XOR-permuted by row).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "bloomgb.h"
#include "lbf.h"
#include "sbf_device.cuh"

namespace lbf {
namespace {

// shared-memory map (offsets from a 1024-byte aligned base)
constexpr uint32_t kB1 = 0;                     // 128 rows (unit j) x 64 bf16 (input i)
constexpr uint32_t kB2 = kB1 + 128 * 128;       // 2 k-blocks x 64 rows x 64 bf16
// bias k-block: A = 1.0 in k = 0..2 of every row, B = the three bf16 parts of
// each unit's requantization constant (zero elsewhere), so one more MMA of
// K = 16 per layer adds the constant to the accumulator
constexpr uint32_t kAx = kB2 + 2 * 64 * 128;    // 128 rows x 64 bf16 (k < 3 used)
constexpr uint32_t kB1x = kAx + 128 * 128;      // 128 rows (unit j)
constexpr uint32_t kB2x = kB1x + 128 * 128;     // 64 rows (unit j)
constexpr uint32_t kImage = kB2x + 64 * 128;    // bytes copied from the device image
constexpr uint32_t kSlots = (kImage + 1023) / 1024 * 1024;  // 4 slots of 16 KiB (A1)
constexpr uint32_t kSlotBytes = 16384;
constexpr int kWG = 4;
constexpr uint32_t kBar = kSlots + kWG * kSlotBytes;  // 4 mbarriers per warpgroup, TMEM base, flags
// + alignment slack; at least 120 KiB so that no second CTA (which would
// wait for this one's tensor memory) is ever placed on the same SM
constexpr uint32_t kSmemBytes = kBar + 256 + 1024 > 120 * 1024 ? kBar + 256 + 1024 : 120 * 1024;
static_assert(kSlots % 1024 == 0 && kB2 % 1024 == 0 && kAx % 1024 == 0 && kB1x % 1024 == 0 && kB2x % 1024 == 0,
              "swizzled operands must be 1024-byte aligned");
static_assert(kSmemBytes <= 227 * 1024, "shared memory");
constexpr int kEpiThreads = 128 * kWG;
constexpr int kThreads = kEpiThreads + 32;  // + the MMA warp
constexpr uint32_t kTmemCols = 512;
// mbarriers of a warpgroup: A1 ready (128 arrivals), A2 ready (128), D1 full
// and D2 full (one tcgen05.commit each)
constexpr int kBarA1 = 0, kBarA2 = 1, kBarD1 = 2, kBarD2 = 3;

// instruction descriptor, kind::f16: fp32 D, bf16 A and B, both K-major, M = 128
__host__ __device__ constexpr uint32_t idesc(uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

struct TcArgs {
  const uint64_t* keys;
  uint64_t n;
  const uint8_t* image;  // kImage bytes, laid out as in shared memory
  int mode;              // 0 scores, 1 out8 |= score >= tau, 4 compaction below tau,
                         // 5 out8 = score >= tau || backup filter (fused lookup)
  int tau;
  int32_t* out32;
  uint8_t* out8;
  unsigned long long* count;
  uint64_t* out_keys;
  unsigned int* err;
  long long s3;
  float w3[64];   // W3q as fp32 (layer 3 runs on the CUDA cores)
  // mode 5: the backup filter (256-bit blocks, S = 32, K = 8, sectorized)
  const uint32_t* bk_words;
  uint64_t bk_blocks;
  uint64_t bk_acc0;
  int bk_mode;
};

// Backup-filter membership of one key (sectorized filter, 256-bit blocks,
// S = 32, K = 8: one bit in each of the block's eight words; Sec. II-A and
// Sec. IV-B): the block's 32 bytes are loaded here, tested by backup_test.
__device__ __forceinline__ void backup_load(const TcArgs& P, uint64_t key, uint32_t& hlo, uint32_t (&w)[8]) {
  const uint64_t h = bloomgb::xxh64_key(key, P.bk_acc0);
  const uint64_t j = bloomgb::block_of(h, P.bk_blocks, P.bk_mode);
  hlo = static_cast<uint32_t>(h);
  bloomgb::ld_words<8>(P.bk_words + j * 8, bloomgb::policy_evict_normal(), w);
}

__device__ __forceinline__ bool backup_test(uint32_t hlo, const uint32_t (&w)[8]) {
  bool in = true;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const uint32_t bit = bloomgb::pattern_bit(hlo, bloomgb::salt_at<32>(t));
    in = in && ((w[t] & bit) != 0);
  }
  return in;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);  // start address
  d |= static_cast<uint64_t>(1) << 16;                          // leading offset (unused when swizzled)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;                  // stride offset: 8 rows x 128 B
  d |= static_cast<uint64_t>(1) << 46;                          // descriptor version
  d |= static_cast<uint64_t>(2) << 61;                          // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id, uint32_t accum) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(id), "r"(accum));
}

__device__ __forceinline__ void mma_bf16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t id,
                                            uint32_t accum) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(id), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void wg_bar(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded wait on an mbarrier phase: false when it did not complete within
// limit_ns.  Each try_wait may sleep in hardware (suspend-time hint 20 us)
// until the phase completes, so a waiting thread takes almost no issue slots.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, uint64_t limit_ns) {
  const uint64_t t0 = globaltimer();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase), "r"(20000u)
        : "memory");
    if (done) return true;
    if (globaltimer() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void sts128(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}



// bf16 pair: floor of (lo, hi) on [128, 256) by conversion toward zero, then clamped to [128, 255]
__device__ __forceinline__ uint32_t requant2(float lo, float hi) {
  uint32_t d;
  asm("{\ncvt.rz.bf16x2.f32 %0, %1, %2;\nmax.bf16x2 %0, %0, %3;\nmin.bf16x2 %0, %0, %4;\n}\n"
      : "=r"(d)
      : "f"(hi), "f"(lo), "r"(0x43004300u), "r"(0x437F437Fu));
  return d;
}

// A-operand byte offset of (row, 16-byte chunk) within a k-block of 128 rows
__device__ __forceinline__ uint32_t swz(uint32_t row, uint32_t chunk) {
  return row * 128u + (((chunk ^ (row & 7u)) & 7u) << 4);
}

#define LBF_LD32(dst, addr)                                                                                        \
  asm volatile(                                                                                                    \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "   \
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"                \
      : "=r"(dst[0]), "=r"(dst[1]), "=r"(dst[2]), "=r"(dst[3]), "=r"(dst[4]), "=r"(dst[5]), "=r"(dst[6]),           \
        "=r"(dst[7]), "=r"(dst[8]), "=r"(dst[9]), "=r"(dst[10]), "=r"(dst[11]), "=r"(dst[12]), "=r"(dst[13]),       \
        "=r"(dst[14]), "=r"(dst[15]), "=r"(dst[16]), "=r"(dst[17]), "=r"(dst[18]), "=r"(dst[19]), "=r"(dst[20]),    \
        "=r"(dst[21]), "=r"(dst[22]), "=r"(dst[23]), "=r"(dst[24]), "=r"(dst[25]), "=r"(dst[26]), "=r"(dst[27]),    \
        "=r"(dst[28]), "=r"(dst[29]), "=r"(dst[30]), "=r"(dst[31])                                                  \
      : "r"(addr))

#define LBF_ST16(addr, src)                                                                                        \
  asm volatile(                                                                                                    \
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "  \
      "%15, %16};" ::"r"(addr),                                                                                     \
      "r"(src[0]), "r"(src[1]), "r"(src[2]), "r"(src[3]), "r"(src[4]), "r"(src[5]), "r"(src[6]), "r"(src[7]),       \
      "r"(src[8]), "r"(src[9]), "r"(src[10]), "r"(src[11]), "r"(src[12]), "r"(src[13]), "r"(src[14]), "r"(src[15])  \
      : "memory")

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// two fp32 lanes in one 64-bit register pair (sm_100 f32x2 arithmetic)
__device__ __forceinline__ uint64_t pack2(uint32_t lo, uint32_t hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
  return r;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ float lo_of(uint64_t v) { return __uint_as_float(static_cast<uint32_t>(v)); }
__device__ __forceinline__ float hi_of(uint64_t v) { return __uint_as_float(static_cast<uint32_t>(v >> 32)); }

// 32 loaded layer-1 accumulator columns (the constant already added by the
// bias MMA) -> 16 columns of packed bf16 (128 + h) at `to`
__device__ __forceinline__ void requant_store(const uint32_t (&a)[32], uint32_t to) {
  uint32_t w[16];
#pragma unroll
  for (int p = 0; p < 16; ++p) w[p] = requant2(__uint_as_float(a[2 * p]), __uint_as_float(a[2 * p + 1]));
  LBF_ST16(to, w);
}

// Layer-1 accumulators (columns from[0..128)) -> packed bf16 at to[0..64), in
// chunks of 32 columns with the next chunk's load in flight while the current
// one is converted; chunk c is stored over columns that chunk c/2 already
// loaded (to <= from), so no store overwrites an unread column.
__device__ __forceinline__ void epilogue1(uint32_t from, uint32_t to) {
  uint32_t a[32], b[32];
  LBF_LD32(a, from);
  tmem_wait_ld();
  LBF_LD32(b, from + 32);
  requant_store(a, to);
  tmem_wait_ld();
  LBF_LD32(a, from + 64);
  requant_store(b, to + 16);
  tmem_wait_ld();
  LBF_LD32(b, from + 96);
  requant_store(a, to + 32);
  tmem_wait_ld();
  requant_store(b, to + 48);
}

// Layer-2 accumulators (64 columns at `from`) -> 128 + h2 -> dot with W3q
// (fp32, even and odd units in the two lanes; every partial sum is an integer
// below 2^24, so exact)
__device__ __forceinline__ float epilogue2(const TcArgs& P, uint32_t from) {
  uint32_t a[32], b[32];
  LBF_LD32(a, from);
  LBF_LD32(b, from + 32);
  tmem_wait_ld();
  auto wp = [&](int u) { return pack2(__float_as_uint(P.w3[u]), __float_as_uint(P.w3[u + 1])); };
  uint64_t acc = 0;
#pragma unroll
  for (int p = 0; p < 16; ++p) {
    const uint32_t w = requant2(__uint_as_float(a[2 * p]), __uint_as_float(a[2 * p + 1]));
    acc = fma2(pack2(w << 16, w & 0xFFFF0000u), wp(2 * p), acc);
  }
#pragma unroll
  for (int p = 0; p < 16; ++p) {
    const uint32_t w = requant2(__uint_as_float(b[2 * p]), __uint_as_float(b[2 * p + 1]));
    acc = fma2(pack2(w << 16, w & 0xFFFF0000u), wp(32 + 2 * p), acc);
  }
  return lo_of(acc) + hi_of(acc);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ uint64_t tiles_of(uint64_t ntiles, uint64_t first, uint64_t stride) {
  return first < ntiles ? (ntiles - first + stride - 1) / stride : 0;
}

// The MMA warp's elected thread issues the warpgroups' products in a fixed
// round: L1 of every warpgroup, then L2 of every warpgroup, and so on (the
// warpgroups run the same work, so they become ready in about this order).
// Each layer starts with its bias product.  Each wait is a blocking try_wait
// (the thread sleeps in hardware).  Returns false when a request did not come
// within 2 s.  (Issuing whichever warpgroup's request is ready first, by
// polling, was measured slower: 21.9 vs 24.1 G scores/s.)
__device__ bool mma_issuer(uint32_t sb, uint32_t tmem, uint64_t ntiles) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kWG;
  uint64_t left[kWG];
  uint64_t most = 0;
  for (int w = 0; w < kWG; ++w) {
    left[w] = tiles_of(ntiles, static_cast<uint64_t>(blockIdx.x) * kWG + w, stride);
    most = left[w] > most ? left[w] : most;
  }
  const uint64_t limit = 2000000000ull;
  for (uint64_t t = 0; t < most; ++t) {
    const uint32_t ph = static_cast<uint32_t>(t & 1);
#pragma unroll
    for (int w = 0; w < kWG; ++w) {
      if (t >= left[w]) continue;
      const uint32_t bars = sb + kBar + 32 * w;
      if (!mbar_wait(bars + 8 * kBarA1, ph, limit)) return false;
      fence_after();
      const uint32_t a1 = sb + kSlots + w * kSlotBytes;
      const uint32_t tm = tmem + 128 * w;
      mma_bf16(tm, sdesc(sb + kAx), sdesc(sb + kB1x), idesc(128), 0);  // D1 = the layer-1 constants
#pragma unroll
      for (uint32_t s = 0; s < 4; ++s) mma_bf16(tm, sdesc(a1 + s * 32), sdesc(sb + kB1 + s * 32), idesc(128), 1);
      mma_commit(bars + 8 * kBarD1);
    }
#pragma unroll
    for (int w = 0; w < kWG; ++w) {
      if (t >= left[w]) continue;
      const uint32_t bars = sb + kBar + 32 * w;
      if (!mbar_wait(bars + 8 * kBarA2, ph, limit)) return false;
      fence_after();
      const uint32_t tm = tmem + 128 * w;
      mma_bf16(tm + 64, sdesc(sb + kAx), sdesc(sb + kB2x), idesc(64), 0);  // D2 = the layer-2 constants
#pragma unroll
      for (uint32_t s = 0; s < 8; ++s)
        mma_bf16_ta(tm + 64, tm + 8 * s, sdesc(sb + kB2 + (s >> 2) * 8192u + (s & 3) * 32), idesc(64), 1);
      mma_commit(bars + 8 * kBarD2);
    }
  }
  return true;
}

__global__ void __launch_bounds__(kThreads, 1) k_tc_mlp(const __grid_constant__ TcArgs P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sb = smem_u32(smem);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;

  for (uint32_t i = tid; i < kImage / 16; i += kThreads)
    reinterpret_cast<uint4*>(smem)[i] = reinterpret_cast<const uint4*>(P.image)[i];
  uint32_t* holder = reinterpret_cast<uint32_t*>(smem + kBar + 128);
  volatile int* flag = reinterpret_cast<volatile int*>(smem + kBar + 144);
  if (tid == 0) {
    for (int w = 0; w < kWG; ++w) {
      const uint32_t bars = sb + kBar + 32 * w;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(bars + 8 * kBarA1) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(bars + 8 * kBarA2) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bars + 8 * kBarD1) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bars + 8 * kBarD2) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const int mma_warp = kEpiThreads / 32;
  if (warp == mma_warp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *holder;
  const uint64_t ntiles = (P.n + 127) / 128;
  const uint64_t limit = 2000000000ull;

  if (warp == mma_warp) {
    if ((tid & 31) == 0 && !mma_issuer(sb, tmem, ntiles)) atomicOr(P.err, 1u);
  } else {
    const int wg = tid >> 7;
    const uint32_t r = tid & 127;
    const uint32_t a1 = sb + kSlots + wg * kSlotBytes;  // this warpgroup's A1 (shared memory)
    const uint32_t bars = sb + kBar + 32 * wg;
    const uint32_t tm = tmem + wg * 128;                 // this warpgroup's columns
    const uint32_t tm_row = tm + ((r & ~31u) << 16);     // this warp's lane quarter
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kWG;
    uint32_t phase = 0;  // each barrier completes once per tile
    bool failed = false;

    // one elected thread waits (bounded) on a commit; the warpgroup then
    // agrees on the outcome through a named barrier (a flag slot per barrier)
    auto wait_on = [&](int which) -> bool {
      if (r == 0) flag[4 * wg + which] = mbar_wait(bars + 8 * which, phase, limit) ? 0 : 1;
      wg_bar(1 + wg);
      fence_after();
      return flag[4 * wg + which] == 0;
    };
    // A1 of a tile: row r = the 64 key bits as bf16 0 / 1.  For 16 bits x,
    // X = (even bits of x) | (odd bits of x) << 16 puts bits 2j and 2j+1 at
    // positions 2j and 16 + 2j, so ((X >> 2j) & 0x10001) * 0x3F80 is the bf16
    // pair (bit 2j, bit 2j+1) with 1.0 = 0x3F80.
    auto build_a1 = [&](uint64_t key) {
#pragma unroll
      for (uint32_t g = 0; g < 4; ++g) {
        const uint32_t x = static_cast<uint32_t>(key >> (16 * g)) & 0xFFFFu;
        const uint32_t X = (x & 0x5555u) | (((x >> 1) & 0x5555u) << 16);
        uint32_t w[8];
#pragma unroll
        for (uint32_t j = 0; j < 8; ++j) w[j] = ((X >> (2 * j)) & 0x00010001u) * 0x3F80u;
        sts128(a1 + swz(r, 2 * g), w[0], w[1], w[2], w[3]);
        sts128(a1 + swz(r, 2 * g + 1), w[4], w[5], w[6], w[7]);
      }
      fence_async_smem();
    };

    uint64_t tile = static_cast<uint64_t>(blockIdx.x) * kWG + wg;
    uint64_t key = 0;
    if (tile < ntiles) {
      const uint64_t i0 = tile * 128 + r;
      key = i0 < P.n ? __ldg(P.keys + i0) : 0;
      build_a1(key);
      mbar_arrive(bars + 8 * kBarA1);
    }
    for (; tile < ntiles; tile += stride) {
      const uint64_t i = tile * 128 + r;
      const bool live = i < P.n;
      // the next tile's keys, loaded early
      const uint64_t ntile = tile + stride;
      const uint64_t ni = ntile * 128 + r;
      const uint64_t nkey = (ntile < ntiles && ni < P.n) ? __ldg(P.keys + ni) : 0;
      // fused lookup: the backup filter's block is fetched while L1 runs
      bool in_backup = false;
      if (P.mode == 5) {
        uint32_t hlo, bw[8];
        backup_load(P, key, hlo, bw);
        in_backup = backup_test(hlo, bw);
      }
      // epilogue 1: D1 (columns 0..127) + c1 -> A2 = 128 + h1 packed in columns 0..63
      if (!wait_on(kBarD1)) { failed = true; break; }
      epilogue1(tm_row, tm_row);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      fence_before();
      mbar_arrive(bars + 8 * kBarA2);
      // the next tile's A1 while L2 runs (L1, its only reader, is complete)
      if (ntile < ntiles) build_a1(nkey);
      // epilogue 2 and layer 3: D2 (columns 64..127)
      if (!wait_on(kBarD2)) { failed = true; break; }
      const float acc3 = epilogue2(P, tm_row + 64);
      fence_before();
      // TMEM and the next A1 are ready for the next L1
      if (ntile < ntiles) mbar_arrive(bars + 8 * kBarA1);
      phase ^= 1;
      long long sc = static_cast<long long>(__float2int_rn(acc3)) + P.s3;
      sc = sc < INT32_MIN ? INT32_MIN : (sc > INT32_MAX ? INT32_MAX : sc);
      if (P.mode == 0) {
        if (live) P.out32[i] = static_cast<int32_t>(sc);
      } else if (P.mode == 1) {
        if (live && sc >= P.tau) P.out8[i] = 1;
      } else if (P.mode == 5) {
        if (live) P.out8[i] = (sc >= P.tau || in_backup) ? 1 : 0;
      } else {
        const bool take = live && sc < P.tau;
        const unsigned vote = __ballot_sync(0xFFFFFFFFu, take);
        const uint32_t lane = r & 31u;
        unsigned long long base = 0;
        if (lane == 0 && vote) base = atomicAdd(P.count, static_cast<unsigned long long>(__popc(vote)));
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (take) P.out_keys[base + __popc(vote & ((1u << lane) - 1u))] = key;
      }
      key = nkey;
    }
    if (failed && r == 0) atomicOr(P.err, 1u);
  }
  fence_before();
  __syncthreads();
  if (warp == mma_warp) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

uint16_t bf16_of(double v) {  // exact for the values used here (<= 8 significant bits)
  const float f = static_cast<float>(v);
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return static_cast<uint16_t>(u >> 16);
}

void put16(std::vector<uint8_t>& img, uint32_t off, uint16_t v) {
  img[off] = static_cast<uint8_t>(v & 0xFF);
  img[off + 1] = static_cast<uint8_t>(v >> 8);
}

uint32_t swz_host(uint32_t row, uint32_t k) {  // element k (< 64) of a 128-byte row
  return row * 128u + ((((k >> 3) ^ (row & 7u)) & 7u) << 4) + (k & 7u) * 2u;
}

double double_of_bf16(uint16_t b) {
  const uint32_t u = static_cast<uint32_t>(b) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// The three bf16 parts of N * s for an integer |N| < 2^24 and s a power of
// two: N = hi + mid + lo with hi = floor(N / 2^16) * 2^16 (at most 8
// significant bits), mid a multiple of 2^8 below 2^16 and lo below 2^8, each
// exact in bf16; the tensor core adds them (and the layer's products) as
// integer multiples of s below 2^24, exactly.  False if a part is not exact.
bool split3(long long n, double s, uint16_t (&out)[3]) {
  if (n <= -(1LL << 24) || n >= (1LL << 24)) return false;
  const long long q = n >= 0 ? n / 65536 : -((-n + 65535) / 65536);
  const long long hi = q * 65536, r = n - hi, mid = (r / 256) * 256, lo = r - mid;
  const long long parts[3] = {lo, mid, hi};
  for (int k = 0; k < 3; ++k) {
    const double v = static_cast<double>(parts[k]) * s;
    out[k] = bf16_of(v);
    if (double_of_bf16(out[k]) != v) return false;
  }
  return true;
}

}  // namespace

bool tc_eligible(const bf_mlp_int8* m) { return m->sh1 >= 0 && m->sh1 <= 15 && m->sh2 >= 0 && m->sh2 <= 15; }

bool tc_prepare(const bf_mlp_int8* m, TcModel* out) {
  if (!tc_eligible(m)) return false;
  std::vector<uint8_t> img(kImage, 0);
  const double s1 = std::ldexp(1.0, -m->sh1), s2 = std::ldexp(1.0, -m->sh2);
  for (uint32_t j = 0; j < 128; ++j)
    for (uint32_t i = 0; i < 64; ++i) put16(img, kB1 + swz_host(j, i), bf16_of(m->w1[i * 128 + j] * s1));
  for (uint32_t j = 0; j < 64; ++j)
    for (uint32_t i = 0; i < 128; ++i)
      put16(img, kB2 + (i >> 6) * 8192u + swz_host(j, i & 63u), bf16_of(m->w2[i * 64 + j] * s2));
  long long sum3 = 0;
  for (uint32_t i = 0; i < 64; ++i) sum3 += m->w3[i];
  // per-unit constants: integers below 2^24 times 2^-sh, exact in fp32
  const long long A1 = 64LL * 127, A2 = 128LL * 127 * 127;
  const long long p1 = 1LL << m->sh1, p2 = 1LL << m->sh2;
  // ... written into the image as the bias k-block (A = 1.0 in k < 3, B = the parts)
  for (uint32_t row = 0; row < 128; ++row)
    for (uint32_t k = 0; k < 3; ++k) put16(img, kAx + swz_host(row, k), 0x3F80u);
  uint16_t part[3];
  for (uint32_t j = 0; j < 128; ++j) {
    const long long b = std::min(std::max<long long>(m->b1[j], -(A1 + 1)), 128 * p1 + A1);
    const double c = static_cast<double>(b + 128 * p1) * s1;
    out->c1[j] = static_cast<float>(c);
    if (static_cast<double>(out->c1[j]) != c || !split3(b + 128 * p1, s1, part)) return false;
    for (uint32_t k = 0; k < 3; ++k) put16(img, kB1x + swz_host(j, k), part[k]);
  }
  for (uint32_t j = 0; j < 64; ++j) {
    long long col = 0;
    for (int i = 0; i < 128; ++i) col += m->w2[i * 64 + j];
    const long long b = std::min(std::max<long long>(m->b2[j], -(A2 + 1)), 128 * p2 + A2);
    const double c = static_cast<double>(b - 128 * col + 128 * p2) * s2;
    out->c2[j] = static_cast<float>(c);
    if (static_cast<double>(out->c2[j]) != c || !split3(b - 128 * col + 128 * p2, s2, part)) return false;
    for (uint32_t k = 0; k < 3; ++k) put16(img, kB2x + swz_host(j, k), part[k]);
  }
  out->s3 = static_cast<long long>(m->b3) - 128 * sum3;
  for (int i = 0; i < 64; ++i) out->w3[i] = static_cast<float>(m->w3[i]);
  out->image = std::move(img);
  return true;
}

uint32_t tc_image_bytes() { return kImage; }

cudaError_t tc_run(const uint8_t* d_image, const TcModel& tm, const uint64_t* d_keys, uint64_t n, int mode, int tau,
                   int32_t* out32, uint8_t* out8, unsigned long long* count, uint64_t* out_keys, unsigned int* err,
                   cudaStream_t st, const TcBackup* backup) {
  if (n == 0) return cudaSuccess;
  static thread_local int configured_device = -1;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (configured_device != dev) {
    const cudaError_t e = cudaFuncSetAttribute(k_tc_mlp, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    configured_device = dev;
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t ntiles = (n + 127) / 128;
  const uint32_t grid = static_cast<uint32_t>(std::min<uint64_t>((ntiles + kWG - 1) / kWG, static_cast<uint64_t>(sms)));
  TcArgs a;
  a.keys = d_keys;
  a.n = n;
  a.image = d_image;
  a.mode = mode;
  a.tau = tau;
  a.out32 = out32;
  a.out8 = out8;
  a.count = count;
  a.out_keys = out_keys;
  a.err = err;
  a.s3 = tm.s3;
  std::memcpy(a.w3, tm.w3, sizeof(a.w3));
  a.bk_words = backup ? backup->words : nullptr;
  a.bk_blocks = backup ? backup->num_blocks : 0;
  a.bk_acc0 = backup ? bloomgb::xxh64_acc0(backup->seed) : 0;
  a.bk_mode = backup ? bloomgb::block_mode(backup->num_blocks) : 0;
  if (mode == 5 && !backup) return cudaErrorInvalidValue;
  k_tc_mlp<<<grid, kThreads, kSmemBytes, st>>>(a);
  return cudaGetLastError();
}

}  // namespace lbf
