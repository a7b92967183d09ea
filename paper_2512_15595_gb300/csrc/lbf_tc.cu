// Learned prefilter, integer model on the 5th-generation tensor cores.
//
// The exported model is integer arithmetic (int8 weights, ReLU + shift +
// saturation, int32 score).  sm_103a has no int8 tensor-core MMA, so the
// three products run as bf16 MMAs with fp32 accumulation (tcgen05.mma
// kind::f16) on values chosen so that every product and every partial sum is
// an exactly representable integer multiple of a power of two:
//   * A1 = the key bits (0/1), B1 = W1q * 2^-sh1 (int8 times a power of two:
//     exact in bf16); |sum x W1q| <= 64 * 127.
//   * the epilogue adds a per-column constant c1 = (b1' + 128 * 2^sh1) 2^-sh1,
//     so y1 = 128 + a1 / 2^sh1 exactly (b1' = b1q clamped to the range where
//     it still changes the result), converts to bf16 rounding toward zero
//     (the bf16 spacing on [128, 256) is 1, so this is the floor) and clamps
//     to [128, 255]: A2 = 128 + h1, exact in bf16.
//   * B2 = W2q * 2^-sh2; the offset 128 * colsum(W2q) is folded into c2, and
//     likewise A3 = 128 + h2, B3 = W3q, score = acc3 + (b3q - 128 sum W3q).
// Every magnitude stays below 2^24 when sh1, sh2 <= 15 (checked on the host;
// other models use the dp4a kernel), so the results equal the integer
// model's bit for bit.
//
// Kernel shape: persistent, one CTA per SM, four warpgroups.  Each warpgroup
// owns a 32 KiB shared-memory slot and 128 TMEM columns and runs its tiles of
// 128 keys through build A1 -> MMA L1 -> epilogue -> MMA L2 -> epilogue ->
// MMA L3 -> score on its own; one elected thread issues its MMAs and commits
// them to the warpgroup's mbarrier.  Four independent pipelines keep the
// tensor core busy while the other warpgroups run their epilogues.  Operands
// use the K-major 128-byte-swizzled layout (8-row groups of 128-byte rows,
// 16-byte chunks XOR-permuted by row), written by the threads themselves.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "bloomgb.h"
#include "lbf.h"

namespace lbf {
namespace {

// shared-memory map (offsets from a 1024-byte aligned base)
constexpr uint32_t kB1 = 0;                     // 128 rows (unit j) x 64 bf16 (input i)
constexpr uint32_t kB2 = kB1 + 128 * 128;       // 2 k-blocks x 64 rows x 64 bf16
constexpr uint32_t kB3 = kB2 + 2 * 64 * 128;    // 16 rows x 64 bf16 (row 0 = W3q)
constexpr uint32_t kLut = kB3 + 16 * 128;       // 256 x 8 bf16: bits of a byte as 0/1
constexpr uint32_t kImage = kLut + 256 * 16;    // bytes copied from the device image
constexpr uint32_t kSlots = kImage;             // 4 slots of 32 KiB
constexpr uint32_t kSlotBytes = 32768;
constexpr int kWG = 4;
constexpr uint32_t kBar = kSlots + kWG * kSlotBytes;  // 4 mbarriers, TMEM base, flags
constexpr uint32_t kSmemBytes = kBar + 64 + 1024;     // + alignment slack
static_assert(kSlots % 1024 == 0, "slots must be 1024-byte aligned");
constexpr int kThreads = 128 * kWG;
constexpr uint32_t kTmemCols = 512;

// instruction descriptor, kind::f16: fp32 D, bf16 A and B, both K-major, M = 128
__host__ __device__ constexpr uint32_t idesc(uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

struct TcArgs {
  const uint64_t* keys;
  uint64_t n;
  const uint8_t* image;  // kImage bytes, laid out as in shared memory
  int mode;              // 0 scores, 1 out8 |= score >= tau, 4 compaction below tau
  int tau;
  int32_t* out32;
  uint8_t* out8;
  unsigned long long* count;
  uint64_t* out_keys;
  unsigned int* err;
  long long s3;
  float c1[128];
  float c2[64];
};

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

// bounded wait on an mbarrier phase (2 s): false when it did not complete
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, uint64_t limit_ns) {
  const uint64_t t0 = globaltimer();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
    if (globaltimer() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void sts128(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}

__device__ __forceinline__ uint4 lds128(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}

// 32 consecutive fp32 columns of this thread's TMEM row
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tmem_ld1(uint32_t taddr) {
  uint32_t r;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  return __uint_as_float(r);
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

__global__ void __launch_bounds__(kThreads, 1) k_tc_mlp(const __grid_constant__ TcArgs P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sb = smem_u32(smem);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;

  for (uint32_t i = tid; i < kImage / 16; i += kThreads)
    reinterpret_cast<uint4*>(smem)[i] = reinterpret_cast<const uint4*>(P.image)[i];
  uint32_t* holder = reinterpret_cast<uint32_t*>(smem + kBar + 32);
  volatile int* flag = reinterpret_cast<volatile int*>(smem + kBar + 48);
  if (tid == 0) {
    for (int s = 0; s < kWG; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sb + kBar + 8 * s) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
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

  const int wg = tid >> 7;
  const uint32_t r = tid & 127;
  const uint32_t slot = sb + kSlots + wg * kSlotBytes;
  const uint32_t bar = sb + kBar + 8 * wg;
  const uint32_t tm = tmem + wg * 128;                      // this warpgroup's columns
  const uint32_t tm_row = tm + ((r & ~31u) << 16);          // this warp's lane quarter
  const uint64_t ntiles = (P.n + 127) / 128;
  const uint64_t limit = 2000000000ull;
  uint32_t phase = 0;
  bool failed = false;

  // one elected thread waits (bounded) on the MMA commit; the warpgroup then
  // agrees on the outcome through a named barrier
  auto wait_mma = [&]() -> bool {
    if (r == 0) flag[wg] = mbar_wait(bar, phase, limit) ? 0 : 1;
    wg_bar(1 + wg);
    phase ^= 1;
    fence_after();
    return flag[wg] == 0;
  };

  for (uint64_t tile = static_cast<uint64_t>(blockIdx.x) * kWG + wg; tile < ntiles;
       tile += static_cast<uint64_t>(gridDim.x) * kWG) {
    const uint64_t i = tile * 128 + r;
    const bool live = i < P.n;
    const uint64_t key = live ? __ldg(P.keys + i) : 0;
    // A1: row r = the 64 key bits as bf16 0 / 1
#pragma unroll
    for (uint32_t c = 0; c < 8; ++c) {
      const uint4 v = lds128(sb + kLut + ((static_cast<uint32_t>(key >> (8 * c)) & 0xFFu) << 4));
      sts128(slot + swz(r, c), v.x, v.y, v.z, v.w);
    }
    fence_async_smem();
    wg_bar(1 + wg);
    if (r == 0) {
      fence_after();
#pragma unroll
      for (uint32_t s = 0; s < 4; ++s) mma_bf16(tm, sdesc(slot + s * 32), sdesc(sb + kB1 + s * 32), idesc(128), s);
      mma_commit(bar);
    }
    if (!wait_mma()) { failed = true; break; }
    // epilogue 1: 128 columns -> A2 = 128 + h1 (two k-blocks)
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      float v[32];
      tmem_ld32(tm_row + q * 32, v);
      uint32_t w[16];
#pragma unroll
      for (int p = 0; p < 16; ++p) w[p] = requant2(v[2 * p] + P.c1[q * 32 + 2 * p], v[2 * p + 1] + P.c1[q * 32 + 2 * p + 1]);
      const uint32_t kb = slot + (q >> 1) * 16384u;
#pragma unroll
      for (uint32_t t = 0; t < 4; ++t) sts128(kb + swz(r, (q & 1) * 4 + t), w[4 * t], w[4 * t + 1], w[4 * t + 2], w[4 * t + 3]);
    }
    fence_before();
    fence_async_smem();
    wg_bar(1 + wg);
    if (r == 0) {
      fence_after();
#pragma unroll
      for (uint32_t s = 0; s < 8; ++s)
        mma_bf16(tm, sdesc(slot + (s >> 2) * 16384u + (s & 3) * 32), sdesc(sb + kB2 + (s >> 2) * 8192u + (s & 3) * 32),
                 idesc(64), s);
      mma_commit(bar);
    }
    if (!wait_mma()) { failed = true; break; }
    // epilogue 2: 64 columns -> A3 = 128 + h2 (one k-block)
#pragma unroll
    for (uint32_t q = 0; q < 2; ++q) {
      float v[32];
      tmem_ld32(tm_row + q * 32, v);
      uint32_t w[16];
#pragma unroll
      for (int p = 0; p < 16; ++p) w[p] = requant2(v[2 * p] + P.c2[q * 32 + 2 * p], v[2 * p + 1] + P.c2[q * 32 + 2 * p + 1]);
#pragma unroll
      for (uint32_t t = 0; t < 4; ++t) sts128(slot + swz(r, q * 4 + t), w[4 * t], w[4 * t + 1], w[4 * t + 2], w[4 * t + 3]);
    }
    fence_before();
    fence_async_smem();
    wg_bar(1 + wg);
    if (r == 0) {
      fence_after();
#pragma unroll
      for (uint32_t s = 0; s < 4; ++s) mma_bf16(tm, sdesc(slot + s * 32), sdesc(sb + kB3 + s * 32), idesc(16), s);
      mma_commit(bar);
    }
    if (!wait_mma()) { failed = true; break; }
    // score: column 0
    const float acc3 = tmem_ld1(tm_row);
    fence_before();
    long long sc = static_cast<long long>(__float2int_rn(acc3)) + P.s3;
    sc = sc < INT32_MIN ? INT32_MIN : (sc > INT32_MAX ? INT32_MAX : sc);
    if (P.mode == 0) {
      if (live) P.out32[i] = static_cast<int32_t>(sc);
    } else if (P.mode == 1) {
      if (live && sc >= P.tau) P.out8[i] = 1;
    } else {
      const bool take = live && sc < P.tau;
      const unsigned vote = __ballot_sync(0xFFFFFFFFu, take);
      const uint32_t lane = r & 31u;
      unsigned long long base = 0;
      if (lane == 0 && vote) base = atomicAdd(P.count, static_cast<unsigned long long>(__popc(vote)));
      base = __shfl_sync(0xFFFFFFFFu, base, 0);
      if (take) P.out_keys[base + __popc(vote & ((1u << lane) - 1u))] = key;
    }
  }
  if (failed && r == 0) {
    atomicOr(P.err, 1u);
    mbar_wait(bar, phase ^ 1, limit);  // the MMAs still in flight, once more (bounded)
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
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
  for (uint32_t i = 0; i < 64; ++i) {
    put16(img, kB3 + swz_host(0, i), bf16_of(m->w3[i]));
    sum3 += m->w3[i];
  }
  for (uint32_t b = 0; b < 256; ++b)
    for (uint32_t e = 0; e < 8; ++e) put16(img, kLut + b * 16 + e * 2, ((b >> e) & 1u) ? 0x3F80 : 0);
  const long long A1 = 64LL * 127, A2 = 128LL * 127 * 127;
  const long long p1 = 1LL << m->sh1, p2 = 1LL << m->sh2;
  for (int j = 0; j < 128; ++j) {
    const long long b = std::min(std::max<long long>(m->b1[j], -(A1 + 1)), 128 * p1 + A1);
    out->c1[j] = static_cast<float>(static_cast<double>(b + 128 * p1) * s1);
  }
  for (int j = 0; j < 64; ++j) {
    long long col = 0;
    for (int i = 0; i < 128; ++i) col += m->w2[i * 64 + j];
    const long long b = std::min(std::max<long long>(m->b2[j], -(A2 + 1)), 128 * p2 + A2);
    out->c2[j] = static_cast<float>(static_cast<double>(b - 128 * col + 128 * p2) * s2);
  }
  out->s3 = static_cast<long long>(m->b3) - 128 * sum3;
  out->image = std::move(img);
  return true;
}

uint32_t tc_image_bytes() { return kImage; }

cudaError_t tc_run(const uint8_t* d_image, const TcModel& tm, const uint64_t* d_keys, uint64_t n, int mode, int tau,
                   int32_t* out32, uint8_t* out8, unsigned long long* count, uint64_t* out_keys, unsigned int* err,
                   cudaStream_t st) {
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
  std::memcpy(a.c1, tm.c1, sizeof(a.c1));
  std::memcpy(a.c2, tm.c2, sizeof(a.c2));
  k_tc_mlp<<<grid, kThreads, kSmemBytes, st>>>(a);
  return cudaGetLastError();
}

}  // namespace lbf
